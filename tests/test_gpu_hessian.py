"""The Hessian pass (pwa_hessian) against the FP64 oracle's full Hessian.

Eq. 7 written out without the contraction with a direction: the oracle forms
every entry per event from the analytic first and second derivatives of the
couplings (oracle.hessian, itself pinned by its agreement with the oracle's
H v and by symmetry).  Bars: Hessian 1e-4 relative in max-norm (the HVP's
bar), gradient 1e-5 relative in max-norm, NLL 1e-6 of the summand scale
(the small-sample reading of the NLL bar, as in test_gpu_parity).  Sizes span
several tiles and end in ragged tiles; points are theta_true, an offset from
it and random starts of the prior.
"""
import numpy as np
import pytest

import oracle
from paper_2403_09225_b300 import workload as W

from conftest import small_workload
from test_gpu_parity import TOL_GRAD, TOL_HVP, TOL_NLL, nll_scale, points, relmax

pytestmark = pytest.mark.gpu


def _check(L, model, wl, th):
    f, g, H = L.hessian(th)
    fo, go = oracle.nll_grad(model, th, wl.data, wl.mc)
    Ho = oracle.hessian(model, th, wl.data, wl.mc)
    assert abs(f - fo) <= TOL_NLL * nll_scale(model, th, wl, fo), (f, fo)
    assert relmax(g, go) <= TOL_GRAD, relmax(g, go)
    assert relmax(H, Ho) <= TOL_HVP, relmax(H, Ho)
    assert np.array_equal(H, H.T)
    # H v from the Hessian and from the fused pass agree
    v = np.linspace(-1.0, 1.0, model.P)
    hv = L.hvp(th, v)
    assert relmax(H @ v, hv) <= 2 * TOL_HVP, relmax(H @ v, hv)
    return relmax(H, Ho)


@pytest.mark.parametrize("name,nd,nm", [("tiny", 4000 + 17, 20000 + 5), ("tiny_k4", 3001, 9999),
                                        ("paper", 1500 + 3, 6000 + 29)])
def test_hessian_matches_oracle(name, nd, nm):
    from paper_2403_09225_b300 import binding
    wl, model = small_workload(name, nd, nm)
    L = binding.make_likelihood(wl)
    for th in points(wl, n_random=1):
        _check(L, model, wl, th)
    L.close()


def test_hessian_k40_fixed_parameters_and_tilings():
    """K = 40 (the differentiation model: 512-thread instance, two Gram
    blocks per thread), odd S with fixed parameters, and a re-tiled handle
    (the tile rotation depends on the tiling)."""
    from paper_2403_09225_b300 import binding
    wl, model = small_workload("diff", 700, 3001, from_model=False)
    L = binding.make_likelihood(wl)
    _check(L, model, wl, W.random_starts(wl, 1)[0])
    L.close()
    cfg = W.Config("k7s3", 7, 3, 0, 0, 2, False, 11)
    base = W.make_workload(cfg, intensity=None, n_data=1234, n_mc=5077)
    table = [W.Resonance(**{**r.__dict__}) for r in base.table]
    table[2].fix_mass = True
    table[4].fix_width = True
    table[5].fix_coupling = True
    wl = W.Workload(cfg, table, W.free_parameter_vector(table), base.data, base.mc, {})
    model = oracle.Model.from_table(table, cfg.S)
    L = binding.make_likelihood(wl)
    assert L.P == model.P == 4 * 7 - 2 - 1 - 1 - 2
    th = wl.theta_true * 1.02
    _check(L, model, wl, th)
    for tiling in ((1, 2), (2, 3), (8, 2)):
        L.set_tiling(*tiling)
        _check(L, model, wl, th)
    L.close()


@pytest.mark.parametrize("K,S", [(30, 3), (28, 4), (25, 2)])
def test_hessian_tensor_core_path_above_k24(K, S):
    """K = 25..32 on the tensor-core path (every event-phase warp owns up to
    four resonances), against the oracle, and against the CUDA-core path."""
    from paper_2403_09225_b300 import binding
    cfg = W.Config("k%ds%d" % (K, S), K, S, 0, 0, 4, False, 40 + K)
    wl = W.make_workload(cfg, intensity=None, n_data=1500 + K, n_mc=4000 + 3 * K)
    model = oracle.Model.from_table(wl.table, S)
    L = binding.make_likelihood(wl)
    th = W.random_starts(wl, 1)[0]
    _check(L, model, wl, th)
    _, _, H = L.hessian(th)
    L.set_hessian_cuda_cores(True)
    _, _, Hc = L.hessian(th)
    assert relmax(H, Hc) <= TOL_HVP, relmax(H, Hc)
    L.close()


@pytest.mark.parametrize("name,nd,nm,B", [("tiny", 2001, 8003, 5), ("tiny_k4", 1500, 6001, 200),
                                           ("paper", 1203, 4099, 3)])
def test_hessian_batch_matches_oracle_and_single_calls(name, nd, nm, B):
    """B vectors in one launch (B = 200 exceeds the resident CTAs: one CTA per
    vector) against the oracle and against single-vector calls; a vector whose
    intensity overflows is flagged in its status while the others are still
    combined."""
    from paper_2403_09225_b300 import binding
    wl, model = small_workload(name, nd, nm)
    L = binding.make_likelihood(wl)
    # the oracle-checked rows at theta_true and an offset from it (as the
    # parity tests); random starts of the prior for the rest
    pts = points(wl, n_random=1)
    ths = np.array([pts[0]] + [pts[0]] + [pts[1]] + list(W.random_starts(wl, B)))[:B]
    bad = wl.theta_true.copy()
    bad[0] = 1e30  # the first free magnitude (magnitudes lead theta): I overflows FP32
    ths[1] = bad
    f, g, H, st = L.hessian_batch(ths)
    for b in range(B):
        if b == 1:
            assert st[b] == binding.PWA_ENONFINITE
            assert np.all(np.isnan(H[b]))
            continue
        assert st[b] == binding.PWA_OK
        if b in (0, 2):
            fo, go = oracle.nll_grad(model, ths[b], wl.data, wl.mc)
            Ho = oracle.hessian(model, ths[b], wl.data, wl.mc)
            assert abs(f[b] - fo) <= TOL_NLL * nll_scale(model, ths[b], wl, fo), (b, f[b], fo)
            assert relmax(g[b], go) <= TOL_GRAD, (b, relmax(g[b], go))
            assert relmax(H[b], Ho) <= TOL_HVP, (b, relmax(H[b], Ho))
        f1, g1, H1 = L.hessian(ths[b])
        assert relmax(H[b], H1) <= 1e-5 and relmax(g[b], g1) <= 1e-6, (b, relmax(H[b], H1))
        assert np.array_equal(H[b], H[b].T)
    # the handle stays usable and a single call after the flagged batch is clean
    f1, g1, H1 = L.hessian(ths[0])
    assert np.isfinite(H1).all()
    L.close()


def test_hessian_is_reproducible_and_refuses_large_k():
    from paper_2403_09225_b300 import binding
    wl, model = small_workload("paper", 1500 + 3, 6000 + 29)
    L = binding.make_likelihood(wl)
    th = W.random_starts(wl, 1)[0]
    a, b = L.hessian(th), L.hessian(th)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    L.close()
    cfg = W.Config("k48", 48, 1, 0, 0, 2, False, 7)
    wl = W.make_workload(cfg, intensity=None, n_data=500, n_mc=2000)
    L = binding.make_likelihood(wl)
    with pytest.raises(binding.PwaError) as e:
        L.hessian(wl.theta_true)
    assert e.value.status == binding.PWA_EINVAL
    L.close()
