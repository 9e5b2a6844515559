"""Batched evaluation (several parameter vectors of one model in one launch)
and lockstep multi-start fits built on it.

Each vector of a batch gets the NLL, gradient and H v of paper Eqs. 3, 6, 7 at
that vector: checked against the FP64 oracle at the benchmark spec's tolerances and
against the single-vector pass (whose event sums are split over a different
block grid, so agreement is to FP32 summation accuracy, not bit for bit).
The batched fits follow the same Newton-CG iteration as the single fit and
reach the oracle fit's minimum.

Bars (as test_gpu_parity): NLL within 1e-6 of max(|NLL|, sum w |ln I|)
(the small-sample reading: the two terms of Eq. 3 nearly cancel on these
samples; the full-size test uses the literal 1e-6 |NLL|), gradient within
1e-5 and H v within 1e-4 of their largest component.
"""
import numpy as np
import pytest

import oracle
from oracle import newton_cg as ncg
from paper_2403_09225_b300 import workload as W

from conftest import small_workload
from test_gpu_parity import TOL_GRAD, TOL_HVP, TOL_NLL, nll_scale, relmax

pytestmark = pytest.mark.gpu


def make_L(wl, **kw):
    from paper_2403_09225_b300 import binding
    return binding.make_likelihood(wl, **kw)


def batch_points(wl, B, seed):
    rng = np.random.default_rng(seed)
    th = wl.theta_true
    pts = [th, th + 0.02 * rng.standard_normal(th.size)] + (list(W.random_starts(wl, B - 2)) if B > 2 else [])
    return np.array(pts[:B]), rng.standard_normal((B, th.size))


@pytest.mark.parametrize("name,nd,nm,B", [("tiny", 4000 + 17, 20000 + 5, 7), ("paper", 1500 + 3, 6000 + 29, 5),
                                          ("tiny_k4", 3001, 9999, 1)])
def test_batch_rows_match_oracle_and_single_pass(name, nd, nm, B):
    wl, model = small_workload(name, nd, nm)
    L = make_L(wl)
    ths, vs = batch_points(wl, B, seed=11)
    f, g, hv = L.eval_batch(ths, vs)
    for b in range(B):
        fo, go, hvo = oracle.nll_grad_hvp(model, ths[b], vs[b], wl.data, wl.mc)
        assert abs(f[b] - fo) <= TOL_NLL * nll_scale(model, ths[b], wl, fo), (b, f[b], fo)
        assert relmax(g[b], go) <= TOL_GRAD, (b, relmax(g[b], go))
        assert relmax(hv[b], hvo) <= TOL_HVP, (b, relmax(hv[b], hvo))
        f1, g1, hv1 = L.eval(ths[b], vs[b])
        assert abs(f[b] - f1) <= 1e-7 * nll_scale(model, ths[b], wl, f1)
        assert relmax(g[b], g1) <= 1e-6 and relmax(hv[b], hv1) <= 1e-5
    # gradient-only batch: the same f and g as the fused one up to FP32 summation
    f2, g2, none = L.eval_batch(ths)
    assert none is None
    for b in range(B):
        assert abs(f2[b] - f[b]) <= 1e-7 * nll_scale(model, ths[b], wl, f[b])
        assert relmax(g2[b], g[b]) <= 1e-6


def test_batch_is_reproducible_and_order_free():
    """Each row depends only on its own vector: the same vector gives the same
    bits wherever it sits in a batch of the same size, and run to run."""
    wl, model = small_workload("tiny", 4000 + 17, 20000 + 5)
    L = make_L(wl)
    ths, vs = batch_points(wl, 6, seed=3)
    f, g, hv = L.eval_batch(ths, vs)
    f_again, g_again, hv_again = L.eval_batch(ths, vs)
    assert np.array_equal(f, f_again) and np.array_equal(g, g_again) and np.array_equal(hv, hv_again)
    perm = np.array([5, 3, 1, 0, 2, 4])
    fp, gp, hvp = L.eval_batch(ths[perm], vs[perm])
    assert np.array_equal(fp, f[perm]) and np.array_equal(gp, g[perm]) and np.array_equal(hvp, hv[perm])


def test_batch_device_entry_point():
    import torch
    wl, model = small_workload("tiny", 4000 + 17, 20000 + 5)
    L = make_L(wl, stream=torch.cuda.current_stream().cuda_stream)
    ths, vs = batch_points(wl, 4, seed=8)
    d_th = torch.tensor(ths, device="cuda")
    d_v = torch.tensor(vs, device="cuda")
    out = torch.zeros((4, 1 + 2 * L.P), dtype=torch.float64, device="cuda")
    L.eval_batch_device(4, d_th.data_ptr(), d_v.data_ptr(), out.data_ptr(), True, True)
    L.sync()
    f, g, hv = L.eval_batch(ths, vs)
    o = out.cpu().numpy()
    assert np.array_equal(o[:, 0], f) and np.array_equal(o[:, 1:1 + L.P], g) and np.array_equal(o[:, 1 + L.P:], hv)


def test_batched_fits_reach_the_oracle_minimum():
    """Starts scattered around the generating point of the full tiny
    configuration: every lockstep fit converges to the minimum that the
    oracle's textbook Newton-CG finds, within 1e-3 of the parameter errors."""
    cfg = W.CONFIGS["tiny"]
    wl, model = small_workload("tiny", cfg.n_data, cfg.n_mc)
    rng = np.random.default_rng(4)
    B = 4
    th0 = wl.theta_true * (1 + 0.03 * rng.standard_normal((B, model.P)))
    fg = lambda x: oracle.nll_grad(model, x, wl.data, wl.mc)
    hp = lambda x, v: oracle.nll_grad_hvp(model, x, v, wl.data, wl.mc)[2]
    ref = ncg.newton_cg(fg, hp, th0[0], xtol=1e-10, maxiter=200)
    assert ref.status in ncg.CONVERGED, ref.status_name
    sig = oracle.parameter_errors(oracle.hessian(model, ref.x, wl.data, wl.mc))
    L = make_L(wl)
    th, infos, all_converged = L.fit_batch(th0, xtol=1e-10)
    assert all_converged, infos
    for b in range(B):
        pull = (oracle.canonical(model, th[b]) - oracle.canonical(model, ref.x)) / sig
        assert np.max(np.abs(pull)) <= 1e-3, (b, pull, infos[b])
        assert abs(infos[b]["nll"] - ref.fun) <= 1e-6 * abs(ref.fun)
        assert infos[b]["n_hess"] > 0 and infos[b]["n_fev"] > 0  # one Hessian pass per outer iteration


def test_batched_fit_reports_a_bad_start_per_fit():
    """A start whose NLL is not finite (every Breit-Wigner underflows, so some
    data event has I = 0) ends that fit with status 'error' and leaves the
    other fits of the batch untouched."""
    cfg = W.CONFIGS["tiny"]
    wl, model = small_workload("tiny", 4000 + 17, 20000 + 5)
    L = make_L(wl)
    good = wl.theta_true.copy()
    bad = good.copy()
    K = cfg.K
    # theta order: rho_1..rho_{K-1}, phi_1..phi_{K-1}, M_0..M_{K-1}, Gamma_0..Gamma_{K-1}
    bad[2 * (K - 1):2 * (K - 1) + K] = 1e20
    th, infos, all_converged = L.fit_batch(np.array([good, bad]), xtol=1e-8)
    assert not all_converged
    assert infos[1]["status"] == "error"
    assert infos[0]["status"] in ("xtol", "gtol", "precision_limit"), infos[0]
    th_single, info_single = L.fit(good, xtol=1e-8)
    assert abs(infos[0]["nll"] - info_single["nll"]) <= 1e-6 * abs(info_single["nll"])


def _toys():
    """Three toy likelihoods of different K, S and sizes (ragged tiles)."""
    wls = [small_workload("tiny", 3000 + 7, 15000 + 3), small_workload("tiny_k4", 2001, 8001),
           small_workload("paper", 800 + 5, 3000 + 11)]
    cfg = W.Config("k7s3", 7, 3, 0, 0, 2, False, 11)
    wl = W.make_workload(cfg, intensity=None, n_data=1234, n_mc=5077)
    wls.append((wl, oracle.Model.from_table(wl.table, cfg.S)))
    return wls


def test_one_launch_over_several_handles_matches_the_oracle():
    """pwa_eval_multi_device: one launch over toys of K = 3, 4, 20, 7 and
    S = 2, 2, 4, 3, two parameter vectors each (theta_true and a prior start),
    every row at the oracle's bars; then a gradient-only launch."""
    from paper_2403_09225_b300 import binding
    toys = _toys()
    Ls = [make_L(wl) for wl, _ in toys]
    thetas, vs = [], []
    for wl, model in toys:
        thetas.append(np.stack([wl.theta_true, W.random_starts(wl, 1)[0]]))
        vs.append(np.stack([np.linspace(-1, 1, model.P), np.cos(np.arange(model.P))]))
    res = binding.eval_multi(Ls, thetas, vs)
    for (wl, model), th, v, (f, g, hv) in zip(toys, thetas, vs, res):
        for b in range(2):
            fo, go, hvo = oracle.nll_grad_hvp(model, th[b], v[b], wl.data, wl.mc)
            assert abs(f[b] - fo) <= TOL_NLL * nll_scale(model, th[b], wl, fo), (f[b], fo)
            assert relmax(g[b], go) <= TOL_GRAD, relmax(g[b], go)
            assert relmax(hv[b], hvo) <= TOL_HVP, relmax(hv[b], hvo)
    res2 = binding.eval_multi(Ls, thetas)
    for (f, g, _), (f2, g2, hv2) in zip(res, res2):
        assert hv2 is None and np.allclose(f2, f, rtol=1e-12, atol=0) and relmax(g2, g) <= 1e-6


def test_one_launch_over_many_handles_sharing_ctas():
    """Ten toys of K 5..30 and S 2..4, eight vectors each: the work list is
    several times longer than the CTAs that fit on the GPU, so CTAs run
    entries of different handles one after another (different shared-memory
    layouts).  Every row agrees with the handle's own batched pass."""
    from paper_2403_09225_b300 import binding
    rng = np.random.default_rng(31)
    toys, Ls = [], []
    for i, (K, S) in enumerate(((5, 2), (30, 3), (12, 4), (26, 2), (8, 3), (22, 4), (17, 4), (13, 2), (25, 4),
                                (7, 2))):
        cfg = W.Config("t%d" % i, K, S, 0, 0, 4, False, 200 + i)
        wl = W.make_workload(cfg, intensity=None, n_data=int(rng.integers(2000, 9000)),
                             n_mc=int(rng.integers(8000, 30000)))
        toys.append(wl)
        Ls.append(make_L(wl))
    thetas = [W.random_starts(wl, 8) for wl in toys]
    vs = [np.tile(np.linspace(-1, 1, L.P), (8, 1)) for L in Ls]
    res = binding.eval_multi(Ls, thetas, vs)
    for L, th, v, (f, g, hv) in zip(Ls, thetas, vs, res):
        f2, g2, hv2 = L.eval_batch(th, v)
        assert np.all(np.isfinite(f)) and np.all(np.isfinite(hv))
        assert np.max(np.abs(f - f2) / np.maximum(np.abs(f2), 1.0)) <= 1e-6
        for b in range(8):
            assert relmax(g[b], g2[b]) <= 1e-5 and relmax(hv[b], hv2[b]) <= 1e-4


def test_fits_over_several_handles_reach_the_oracle_minima():
    """Toy fits of different models and sample sizes (K, S, N differ) in
    lockstep over several handles -- one launch per round over all of them
    (pwa_eval_multi_device, its rounds captured into CUDA graphs) -- reach,
    toy by toy, the minimum the oracle's textbook Newton-CG finds, within
    1e-3 of the oracle's parameter errors.  Each toy's data are drawn from its
    own model and its starts lie 0.2 sigma per parameter from the oracle's
    minimum (inside the basin: paths from far away can end in different
    local minima under different FP32 rounding)."""
    from paper_2403_09225_b300 import binding
    toys = [small_workload("tiny", 3000 + 7, 15000 + 3), small_workload("tiny_k4", 2001, 8001)]
    for K, S, seed in ((5, 3, 13), (6, 2, 17)):
        cfg = W.Config("k%ds%d" % (K, S), K, S, 0, 0, 2, False, seed)
        model = oracle.Model.from_table(W.make_table(cfg), S)
        fn = lambda m2, F, cfg=cfg, model=model: oracle.intensity_full(cfg.K, cfg.S, model.channels, model.par0, m2, F)
        toys.append((W.make_workload(cfg, intensity=fn, n_data=6001, n_mc=24001), model))
    refs, starts = [], []
    for i, (wl, model) in enumerate(toys):
        fg = lambda x, wl=wl, model=model: oracle.nll_grad(model, x, wl.data, wl.mc)
        hp = lambda x, v, wl=wl, model=model: oracle.nll_grad_hvp(model, x, v, wl.data, wl.mc)[2]
        ref = ncg.newton_cg(fg, hp, wl.theta_true, xtol=1e-10, maxiter=300)
        assert ref.status in ncg.CONVERGED, ref.status_name
        sig = oracle.parameter_errors(oracle.hessian(model, ref.x, wl.data, wl.mc))
        refs.append((ref.x, sig))
        rng = np.random.default_rng(20 + i)
        starts.append(ref.x + 0.2 * sig * rng.standard_normal((3, ref.x.size)))
    Ls = [make_L(wl) for wl, _ in toys]
    for matrix_free, one_launch in ((False, False), (False, True), (True, True)):
        outs, infos, ok = binding.fit_multi(Ls, starts, xtol=1e-10, matrix_free=matrix_free, one_launch=one_launch)
        assert ok, infos
        for (wl, model), (x_ref, sig), o in zip(toys, refs, outs):
            for th in o:
                pull = (oracle.canonical(model, th) - oracle.canonical(model, x_ref)) / sig
                assert np.max(np.abs(pull)) <= 1e-3, (matrix_free, one_launch, np.max(np.abs(pull)))


def test_autotune_keeps_results_within_tolerance():
    wl, model = small_workload("paper", 1500 + 3, 6000 + 29)
    L = make_L(wl)
    th = wl.theta_true
    v = np.random.default_rng(2).standard_normal(model.P)
    til = L.autotune(th, batch=4)
    assert til["warps"] in (1, 2, 4, 8) and til["stages"] in (2, 3) and til["blocks_per_sm"] >= 1
    f, g, hv = L.eval(th, v)
    fo, go, hvo = oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
    assert abs(f - fo) <= TOL_NLL * nll_scale(model, th, wl, fo)
    assert relmax(g, go) <= TOL_GRAD and relmax(hv, hvo) <= TOL_HVP
