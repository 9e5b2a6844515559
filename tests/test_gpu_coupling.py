"""The fixed-mass coupling sub-problem on the tensor cores (Eq. 1 with the
couplings outside the sum): the integral matrix against the oracle's, and
NLL, gradient and H v in the coupling parameters for many coupling vectors
against the oracle's full NLL, gradient and H v at the same full theta
(restricted to the coupling block) and against the fused pass.

Bars (as test_gpu_parity): NLL within 1e-6 of max(|NLL|, sum w |ln I|)
(the small-sample reading: the two terms of Eq. 3 nearly cancel on these
samples; the full-size test uses the literal 1e-6 |NLL|), gradient within
1e-5 and H v within 1e-4 of their largest component."""
import numpy as np
import pytest

import oracle
from paper_2403_09225_b300 import workload as W

from conftest import small_workload
from test_gpu_parity import TOL_GRAD, TOL_HVP, TOL_NLL, nll_scale, relmax

pytestmark = pytest.mark.gpu


def coupling_points(wl, model, C, seed):
    """C coupling vectors around and away from the generating couplings, with
    the masses and widths of theta_true, and directions in the coupling block."""
    from paper_2403_09225_b300 import binding
    rng = np.random.default_rng(seed)
    Pc = int(np.sum([not r.fix_coupling for r in wl.table])) * 2
    th0 = wl.theta_true
    rows = [th0[:Pc] * (1 + 0.05 * rng.standard_normal(Pc)) for _ in range(C)]
    rows[0] = th0[:Pc].copy()
    starts = W.random_starts(wl, C)
    for c in range(1, C, 2):
        rows[c] = starts[c][:Pc]
    return th0, np.array(rows), rng.standard_normal((C, Pc)), Pc


def full_theta(th0, row):
    th = th0.copy()
    th[:row.size] = row
    return th


GRAD_BAR = {}  # every shape at the spec bars


@pytest.mark.parametrize("name,nd,nm,C", [("tiny", 4000 + 17, 20000 + 5, 5), ("paper", 1500 + 3, 6000 + 29, 20),
                                          ("tiny_k4", 3001, 9999, 16)])
def test_coupling_eval_matches_oracle(name, nd, nm, C):
    from paper_2403_09225_b300 import binding
    wl, model = small_workload(name, nd, nm)
    L = binding.make_likelihood(wl)
    th0, rows, vs, Pc = coupling_points(wl, model, C, seed=13)
    cp = binding.Coupling(L, th0)
    assert cp.Pc == Pc
    f, g, hv = cp.eval(rows, vs)
    for c in range(C):
        th = full_theta(th0, rows[c])
        vfull = np.zeros(model.P)
        vfull[:Pc] = vs[c]
        fo, go, hvo = oracle.nll_grad_hvp(model, th, vfull, wl.data, wl.mc)
        assert abs(f[c] - fo) <= TOL_NLL * nll_scale(model, th, wl, fo), (c, f[c], fo)
        assert relmax(g[c], go[:Pc]) <= GRAD_BAR.get(name, TOL_GRAD), (c, relmax(g[c], go[:Pc]))
        assert relmax(hv[c], hvo[:Pc]) <= TOL_HVP, (c, relmax(hv[c], hvo[:Pc]))
        # the fused pass at the same point: both paths carry FP32 rounding of
        # their own, so they agree to the same bars as each does with the oracle
        f1, g1, hv1 = L.eval(th, vfull)
        assert abs(f[c] - f1) <= TOL_NLL * nll_scale(model, th, wl, f1)
        assert relmax(g[c], g1[:Pc]) <= GRAD_BAR.get(name, TOL_GRAD) and relmax(hv[c], hv1[:Pc]) <= TOL_HVP
    f2, g2, none = cp.eval(rows)
    assert none is None and np.allclose(f2, f, rtol=0, atol=0) and np.array_equal(g2, g)
    cp.close()


def test_integral_matrix_matches_oracle():
    from paper_2403_09225_b300 import binding
    wl, model = small_workload("paper", 1500 + 3, 6000 + 29)
    L = binding.make_likelihood(wl)
    th = W.random_starts(wl, 1)[0]
    cp = binding.Coupling(L, th)
    phi = cp.integral_matrix()
    phio = oracle.integral_matrix(model, th, wl.mc.m2, wl.mc.F)
    assert relmax(phi, phio) <= 1e-6, relmax(phi, phio)
    cp.close()


def test_projection_count_three_and_ragged_tiles():
    """S = 3 leaves two unused rows per warp in every tile; sizes end in a
    ragged tile."""
    from paper_2403_09225_b300 import binding
    cfg = W.Config("s3", 7, 3, 1234, 5000, 4, False, 42)
    table = W.make_table(cfg)
    model = oracle.Model.from_table(table, cfg.S)
    wl = W.make_workload(cfg, intensity=None)
    L = binding.make_likelihood(wl)
    th0, rows, vs, Pc = coupling_points(wl, model, 3, seed=5)
    cp = binding.Coupling(L, th0)
    f, g, hv = cp.eval(rows, vs)
    for c in range(3):
        th = full_theta(th0, rows[c])
        vfull = np.zeros(model.P)
        vfull[:Pc] = vs[c]
        fo, go, hvo = oracle.nll_grad_hvp(model, th, vfull, wl.data, wl.mc)
        assert abs(f[c] - fo) <= TOL_NLL * nll_scale(model, th, wl, fo)
        assert relmax(g[c], go[:Pc]) <= TOL_GRAD and relmax(hv[c], hvo[:Pc]) <= TOL_HVP
    cp.close()


def test_coupling_refuses_large_k():
    from paper_2403_09225_b300 import binding
    wl, model = small_workload("diff", 700, 3001, from_model=False)
    L = binding.make_likelihood(wl)
    with pytest.raises(binding.PwaError):
        binding.Coupling(L, wl.theta_true)


@pytest.mark.parametrize("name,nd,nm", [("tiny_k4", 3001, 9999), ("paper", 1500 + 3, 6000 + 29)])
def test_coupling_fit_reaches_the_oracle_coupling_minimum(name, nd, nm):
    """Coupling-only fits (masses and widths fixed at theta_true) from starts
    scattered around the generating couplings all converge to the minimum the
    oracle's textbook Newton-CG finds over the same coupling parameters, within
    1e-3 of the oracle's errors of those parameters."""
    from oracle import newton_cg as ncg
    from paper_2403_09225_b300 import binding
    wl, model = small_workload(name, nd, nm)
    th0 = wl.theta_true
    Pc = int(np.sum([not r.fix_coupling for r in wl.table])) * 2
    full = lambda xc: full_theta(th0, xc)

    def fg(xc):
        f, g = oracle.nll_grad(model, full(xc), wl.data, wl.mc)
        return f, g[:Pc]

    def hp(xc, v):
        vf = np.zeros(model.P)
        vf[:Pc] = v
        return oracle.nll_grad_hvp(model, full(xc), vf, wl.data, wl.mc)[2][:Pc]

    rng = np.random.default_rng(17)
    starts = th0[:Pc] * (1 + 0.02 * rng.standard_normal((4, Pc)))
    ref = ncg.newton_cg(fg, hp, starts[0], xtol=1e-10, maxiter=200)
    assert ref.status in ncg.CONVERGED, ref.status_name
    H = oracle.hessian(model, full(ref.x), wl.data, wl.mc)[:Pc, :Pc]
    sig = oracle.parameter_errors(H)
    L = binding.make_likelihood(wl)
    cp = binding.Coupling(L, th0)
    xs, infos, ok = cp.fit(starts, xtol=1e-10)
    assert ok, infos
    for b in range(len(starts)):
        d = oracle.canonical(model, full(xs[b]))[:Pc] - oracle.canonical(model, full(ref.x))[:Pc]
        assert np.max(np.abs(d / sig)) <= 1e-3, (b, np.max(np.abs(d / sig)), infos[b])
        assert abs(infos[b]["nll"] - ref.fun) <= 1e-6 * abs(ref.fun)
    cp.close()
