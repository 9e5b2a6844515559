"""CPU FP64 oracle of the proposal network -- TEST INFRASTRUCTURE.

The learned starting-point proposal has no counterpart in the paper: it is a
plain multilayer perceptron, written out here from its definition (affine
layers, GELU in its tanh form, a weighted squared error with 1 - cos for
periodic outputs, averaged over the rows) with the backward pass by the chain
rule, in float64.  With quantize=True the operands are rounded to BF16 at the
points where the library's kernels hold them in BF16 (inputs, weights, hidden
activations, the output and hidden gradients that enter matrix products), so
that the library and this oracle differ only by FP32 accumulation order.
Nothing here is imported by the library.
"""
from __future__ import annotations

import numpy as np

_C = 0.7978845608028654  # sqrt(2 / pi)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_C * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3 * 0.044715 * z * z)


def init_params(sizes, seed: int):
    """Weights uniform in +-sqrt(6 / (fan_in + fan_out)), biases 0 (numpy generator)."""
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / (fi + fo))
        out.append((rng.uniform(-lim, lim, size=(fo, fi)), np.zeros(fo)))
    return out


def forward(params, x, quantize=False):
    """Pre-activations z_l and layer inputs h_l; returns (y, zs, hs)."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    h = q(x)
    zs, hs = [], []
    for i, (W, b) in enumerate(params):
        hs.append(h)
        z = h @ q(W).T + b
        zs.append(z)
        if i < len(params) - 1:
            h = q(gelu(z))
    return zs[-1], zs, hs


def loss_and_grads(params, x, t, weight, periodic, quantize=False):
    """Mean loss over the rows and the gradients [(dW, db), ...]."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    y, zs, hs = forward(params, x, quantize)
    B = y.shape[0]
    d = y - t
    per = np.asarray(periodic, dtype=bool)
    lc = np.where(per, 1.0 - np.cos(d), 0.5 * d * d)
    gc = np.where(per, np.sin(d), d)
    loss = float(np.sum(lc * weight) / B)
    dz32 = gc * weight / B
    grads = [None] * len(params)
    dzq = q(dz32)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (dzq.T @ hs[l], dz32.sum(axis=0))
        if l == 0:
            break
        dh = dzq @ q(W)
        dz32 = dh * gelu_grad(zs[l - 1])
        dzq = q(dz32)
    return loss, grads
