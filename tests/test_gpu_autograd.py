"""The torch.autograd.Function wrapper: first and second derivatives of the
GPU NLL through torch.autograd, checked against the FP64 oracle (analytic
gradient and HVP) and against central differences of the GPU gradient."""
import numpy as np
import pytest

import oracle
from paper_2403_09225_b300 import workload as W

from conftest import small_workload

pytestmark = pytest.mark.gpu


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_autograd_gradient_and_hvp(device):
    import torch
    from paper_2403_09225_b300 import autograd, binding
    wl, model = small_workload("paper", 1500 + 3, 6000 + 29)
    L = binding.make_likelihood(wl)
    th0 = W.random_starts(wl, 1)[0]
    v0 = np.cos(np.arange(model.P))
    theta = torch.tensor(th0, dtype=torch.float64, device=device, requires_grad=True)
    f = autograd.nll(theta, L)
    (g,) = torch.autograd.grad(f, theta, create_graph=True)
    v = torch.tensor(v0, dtype=torch.float64, device=device)
    (hv,) = torch.autograd.grad(g, theta, grad_outputs=v)
    L.sync()
    fo, go, hvo = oracle.nll_grad_hvp(model, th0, v0, wl.data, wl.mc)
    assert relmax(g.detach().cpu().numpy(), go) <= 1e-5
    assert relmax(hv.detach().cpu().numpy(), hvo) <= 1e-4
    # HVP against central differences of the GPU gradient (FP32 noise: loose bar)
    h = 1e-4
    gp = L.grad(th0 + h * v0)[1]
    gm = L.grad(th0 - h * v0)[1]
    assert relmax(hv.detach().cpu().numpy(), (gp - gm) / (2 * h)) <= 1e-3
