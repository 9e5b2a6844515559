"""Newton-CG fit parity (paper Sec. 3): the GPU fit and the oracle's FP64
textbook Newton-CG, started from the same point on the full tiny
configuration, reach the same minimum within 1e-3 of the oracle's parameter
errors (after mapping (rho, phi) ~ (-rho, phi + pi) to one representative)."""
import numpy as np
import pytest

import oracle
from oracle import newton_cg as ncg
from paper_2403_09225_b300 import workload as W

from conftest import small_workload

pytestmark = pytest.mark.gpu


def test_fit_matches_oracle_fit_on_tiny():
    from paper_2403_09225_b300 import binding
    cfg = W.CONFIGS["tiny"]
    wl, model = small_workload("tiny", cfg.n_data, cfg.n_mc)
    rng = np.random.default_rng(4)
    th0 = wl.theta_true * (1 + 0.03 * rng.standard_normal(model.P))
    fg = lambda x: oracle.nll_grad(model, x, wl.data, wl.mc)
    hp = lambda x, v: oracle.nll_grad_hvp(model, x, v, wl.data, wl.mc)[2]
    ref = ncg.newton_cg(fg, hp, th0, xtol=1e-10, maxiter=200)
    assert ref.status in ncg.CONVERGED, ref.status_name
    L = binding.make_likelihood(wl)
    th, info = L.fit(th0, xtol=1e-10)
    assert info["converged"], info
    sig = oracle.parameter_errors(oracle.hessian(model, ref.x, wl.data, wl.mc))
    pull = (oracle.canonical(model, th) - oracle.canonical(model, ref.x)) / sig
    assert np.max(np.abs(pull)) <= 1e-3, (pull, info)
    assert abs(info["nll"] - ref.fun) <= 1e-6 * abs(ref.fun)
