"""torch.autograd.Function wrappers around the fused pass.

``nll(theta, L)`` returns -ln L as a 0-d tensor whose gradient is the
library's adjoint gradient and whose second derivative (double backward,
e.g. ``torch.autograd.grad(g, theta, v)`` with ``create_graph=True``) is the
library's Hessian-vector product.  No arithmetic happens here: every value
comes from one launch of the CUDA pass (theta on a CUDA device: the launch is
enqueued on the current stream; theta on the CPU: the synchronous host entry
point is used).  Device-side errors of asynchronous launches are reported by
``L.sync()``.
"""
from __future__ import annotations

import torch


def _launch(L, theta: torch.Tensor, v, want_grad: bool, want_hv: bool) -> torch.Tensor:
    """(NLL, grad[P], hv[P]) as one float64 tensor of length 1 + 2P."""
    P = L.P
    if theta.is_cuda:
        th = theta.detach().to(torch.float64).contiguous()
        vv = th if v is None else v.detach().to(device=th.device, dtype=torch.float64).contiguous()
        out = torch.empty(1 + 2 * P, dtype=torch.float64, device=th.device)
        L.set_stream(torch.cuda.current_stream(th.device).cuda_stream)
        L.eval_device(th.data_ptr(), vv.data_ptr(), out.data_ptr(), want_grad, want_hv)
        return out
    th = theta.detach().to(torch.float64).numpy()
    f, g, hv = L.eval(th, None if v is None else v.detach().to(torch.float64).numpy())
    out = torch.zeros(1 + 2 * P, dtype=torch.float64)
    out[0] = f
    out[1:1 + P] = torch.from_numpy(g)
    if hv is not None:
        out[1 + P:] = torch.from_numpy(hv)
    return out


class _Grad(torch.autograd.Function):
    """theta -> grad NLL(theta); its backward is the Hessian-vector product."""

    @staticmethod
    def forward(ctx, theta, L):
        ctx.L = L
        ctx.save_for_backward(theta)
        P = L.P
        return _launch(L, theta, None, True, False)[1:1 + P].to(theta.dtype)

    @staticmethod
    def backward(ctx, v):
        (theta,) = ctx.saved_tensors
        P = ctx.L.P
        hv = _launch(ctx.L, theta, v, True, True)[1 + P:].to(theta.dtype)
        return hv, None


class _NLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, L):
        ctx.L = L
        ctx.save_for_backward(theta)
        return _launch(L, theta, None, False, False)[0].to(theta.dtype)

    @staticmethod
    def backward(ctx, gout):
        (theta,) = ctx.saved_tensors
        return gout * _Grad.apply(theta, ctx.L), None


def nll(theta: torch.Tensor, L) -> torch.Tensor:
    """-ln L(theta) (paper Eq. 3, negated) with exact first and second derivatives."""
    return _NLL.apply(theta, L)
