"""The learned proposal's network on the GPU against the CPU FP64 oracle.

The library runs every matrix product on the tensor cores with BF16 operands
and FP32 accumulation; the oracle (oracle/mlp.py) rounds the same operands to
BF16 at the same points and accumulates in FP64, so the two differ by FP32
accumulation order and by the rare BF16 rounding decision that the FP32 and
FP64 values of an operand take differently.  Bars:
  * a single product, K terms: |C - C_ref| <= 4 K 2^-24 (|A| |B|^T) + 1e-30
    elementwise (FP32 accumulation error bound with a factor 4 of slack);
  * forward outputs and gradients, per layer: relative Frobenius error
    against the BF16-rounding oracle <= max(2e-3, 0.25 e_q), with e_q the
    relative Frobenius distance between that oracle and the plain FP64
    network.  A hidden activation whose FP32 and FP64 values round to
    different BF16 neighbours moves by 2^-8 of itself; such flips hit a
    fraction of order (relative FP32 error of the pre-activation) / 2^-8 of
    the activations, while the BF16 storage itself moves every activation, so
    their effect is a small fraction of e_q as long as the pre-activations
    carry little FP32 error (the 4096-input network gets an exactly summed
    first layer for that reason, see its test).  Any wrong index or a dropped
    term gives an O(1) error.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _net(n_in, hidden, layers, n_out, max_batch, seed=5, periodic=None, weight=None):
    from paper_2403_09225_b300 import binding
    return binding.ProposalMLP(n_in, hidden, layers, n_out, max_batch, seed=seed, periodic=periodic,
                               loss_weight=weight)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 192, 320), (384, 128, 4096)])
def test_gemm_matches_bf16_product(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    net = _net(64, 128, 1, 4, 128)
    C = net.gemm_check(A, B)
    Aq, Bq = omlp.bf16(A), omlp.bf16(B)
    ref = Aq @ Bq.T
    bound = 4 * K * 2.0 ** -24 * (np.abs(Aq) @ np.abs(Bq).T) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    net.close()


def test_gemm_rejects_unaligned_shapes():
    from paper_2403_09225_b300 import binding
    net = _net(64, 128, 1, 4, 128)
    with pytest.raises(binding.PwaError):
        net.gemm_check(np.zeros((100, 64), np.float32), np.zeros((64, 64), np.float32))
    net.close()


def _setup(n_in, hidden, layers, n_out, B, seed, exact_first=False):
    import torch
    rng = np.random.default_rng(seed)
    periodic = [int(i % 3 == 2) for i in range(n_out)]
    weight = 0.5 + rng.random(n_out)
    net = _net(n_in, hidden, layers, n_out, B, seed=seed, periodic=periodic, weight=weight)
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    if exact_first:
        # small integers and weights on a 2^-12 grid: every product and partial
        # sum of the first layer is exact in FP32, so both sides see the same
        # pre-activations and only GELU's last-bit differences can move a BF16
        # rounding decision
        x = rng.integers(-4, 5, size=(B, n_in)).astype(np.float32)
        W0 = net.get(0, 0)
        net.set(0, 0, np.round(W0 * 4096) / 4096)
    t = rng.standard_normal((B, n_out)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    return net, x, t, xd, td, periodic, np.asarray(weight, np.float32).astype(np.float64)


@pytest.mark.parametrize("n_in,hidden,layers,n_out,B,exact_first", [(64, 128, 1, 5, 128, False),
                                                                    (256, 256, 2, 78, 256, False),
                                                                    (4096, 512, 3, 78, 128, True)])
def test_forward_and_gradients_match_oracle(n_in, hidden, layers, n_out, B, exact_first):
    """exact_first for the 4096-input network: with random FP32 operands a
    fan-in of 4096 leaves pre-activations whose FP32 rounding error is a few
    1e-4 of their value (cancellation), and several per cent of the hidden
    activations then round to the other BF16 neighbour than in FP64 -- as
    large an effect as the BF16 storage itself, which would leave nothing to
    compare against."""
    net, x, t, xd, td, periodic, weight = _setup(n_in, hidden, layers, n_out, B, seed=n_in + n_out,
                                                 exact_first=exact_first)
    # biases away from zero so that the bias path is exercised (a 2^-10 grid
    # keeps the first layer's sums exact)
    rng = np.random.default_rng(7)
    for l in range(layers + 1):
        net.set(l, 1, np.round(0.1 * rng.standard_normal(net.get(l, 1).shape) * 1024) / 1024)
    params = net.params()
    y = net.forward(xd).cpu().numpy()
    y_q, _, _ = omlp.forward(params, x, quantize=True)
    y_64, _, _ = omlp.forward(params, x, quantize=False)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    e_q = rel(y_q, y_64)
    assert rel(y, y_q) <= max(2e-3, 0.25 * e_q), (rel(y, y_q), e_q)
    loss = net.gradients(xd, td)
    loss_ref, grads = omlp.loss_and_grads(params, x, t, weight, periodic, quantize=True)
    loss_64, g64 = omlp.loss_and_grads(params, x, t, weight, periodic, quantize=False)
    assert abs(loss - loss_ref) <= max(1e-4 * abs(loss_ref), 0.25 * abs(loss_ref - loss_64))
    for l in range(layers + 1):
        dW, db = net.get(l, 2), net.get(l, 3)
        eW, eb = rel(dW, grads[l][0]), rel(db, grads[l][1])
        qW, qb = rel(grads[l][0], g64[l][0]), rel(grads[l][1], g64[l][1])
        print("layer %d: weight grad %.2e (BF16 effect %.2e), bias grad %.2e (%.2e)" % (l, eW, qW, eb, qb))
        assert eW <= max(2e-3, 0.25 * qW) and eb <= max(2e-3, 0.25 * qb), (l, eW, qW, eb, qb)
        # and the BF16 storage costs well under 5 % against the plain FP64 network
        assert qW <= 0.05
    net.close()


def test_adam_step_matches_definition():
    """One train step: loss and gradients as above, then Adam (bias-corrected
    first and second moments, beta 0.9 / 0.999, eps 1e-8) from zero moments,
    which for the first step moves every weight by lr * g / (|g| + eps)."""
    net, x, t, xd, td, periodic, weight = _setup(64, 128, 1, 5, 128, seed=11)
    params = net.params()
    lr = 1e-3
    net.train_step(xd, td, lr)
    _, grads = omlp.loss_and_grads(params, x, t, weight, periodic, quantize=True)
    for l in range(2):
        W1 = net.get(l, 0).astype(np.float64)
        g = net.get(l, 2).astype(np.float64)
        expect = params[l][0] - lr * g / (np.abs(g) + 1e-8)
        assert np.max(np.abs(W1 - expect)) <= 1e-6, l
    net.close()


def test_training_fits_a_smooth_map():
    """Plain regression on a fixed smooth target: 300 Adam steps take the
    loss down by more than 10x (checks that forward, backward and the
    optimizer work together on the tensor-core products)."""
    import torch
    rng = np.random.default_rng(0)
    n_in, n_out, B = 128, 6, 256
    P = rng.standard_normal((n_in, n_out)) / np.sqrt(n_in)
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    t = np.tanh(x @ P).astype(np.float32)
    net = _net(n_in, 256, 2, n_out, B, seed=3)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = net.train_step(xd, td, 1e-3)
    for _ in range(300):
        last = net.train_step(xd, td, 1e-3)
    assert last < first / 10, (first, last)
    net.close()


def test_graph_replayed_gradients_equal_the_eager_ones():
    """The gradient pass of a batch size runs eagerly twice, is captured into a
    CUDA graph on the third call and replayed from then on: the same kernels in
    the same order, so the results are bit-identical; a new input reaches the
    replayed graph (it is copied into the network's buffers first)."""
    import torch
    net, x, t, xd, td, periodic, weight = _setup(256, 256, 2, 12, 256, seed=21)
    ref_loss = net.gradients(xd, td)
    ref = [net.get(l, 2).copy() for l in range(3)]
    for _ in range(4):
        assert net.gradients(xd, td) == ref_loss
        for l in range(3):
            assert np.array_equal(net.get(l, 2), ref[l])
    x2 = torch.flip(xd, dims=[0]).contiguous()
    l2 = net.gradients(x2, td)
    params = net.params()
    lo, _ = omlp.loss_and_grads(params, x2.cpu().numpy(), t, weight, periodic, quantize=True)
    assert abs(l2 - lo) <= 1e-3 * abs(lo) and l2 != ref_loss
    net.close()
