"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (the spec bar, norm-wise so that near-stationary points do
not inflate them): NLL 1e-6 relative, gradient 1e-5 relative in max-norm, HVP
1e-4 relative in max-norm.  Points: theta_true, offsets from it, random
starts from the prior.  Sizes span several tiles and end in a ragged tile.
"""
import numpy as np
import pytest

import oracle
from paper_2403_09225_b300 import workload as W

from conftest import small_workload

pytestmark = pytest.mark.gpu

TOL_NLL, TOL_GRAD, TOL_HVP = 1e-6, 1e-5, 1e-4


def nll_scale(model, th, wl, fo):
    """Scale for the NLL's relative bar.  NLL = -sum w ln I + N_d ln(G/N_mc)
    is a difference of two terms of size ~ N_d that nearly cancel for small
    samples at some points; FP32 rounding is relative to the summands, so the
    bar is 1e-6 of max(|NLL|, sum_data w |ln I|).  At the full configuration
    sizes both scales coincide (tested separately)."""
    I = oracle.intensity(model, th, wl.data.m2, wl.data.F)
    w = np.ones_like(I) if wl.data.w is None else wl.data.w.astype(np.float64)
    return max(abs(fo), float(np.sum(w * np.abs(np.log(I)))))


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def make_L(wl, **kw):
    from paper_2403_09225_b300 import binding
    return binding.make_likelihood(wl, **kw)


def check_point(L, model, wl, th, v):
    f, g, hv = L.eval(th, v)
    fo, go, hvo = oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
    assert abs(f - fo) <= TOL_NLL * nll_scale(model, th, wl, fo), (f, fo)
    assert relmax(g, go) <= TOL_GRAD, relmax(g, go)
    assert relmax(hv, hvo) <= TOL_HVP, relmax(hv, hvo)
    # the reuse pass (Q sums, G and the gradient kept from the full pass at th)
    # for this v and for another direction
    assert relmax(L.hvp_reuse(th, v), hvo) <= TOL_HVP
    v2 = np.asarray(v)[::-1] * np.linspace(0.5, 1.5, len(v))
    hvo2 = oracle.nll_grad_hvp(model, th, v2, wl.data, wl.mc)[2]
    assert relmax(L.hvp_reuse(th, v2), hvo2) <= TOL_HVP, relmax(L.hvp_reuse(th, v2), hvo2)
    # the cheaper passes agree with the fused one
    assert L.nll(th) == f  # same summation order in every mode
    f2, g2 = L.grad(th)
    assert relmax(g2, go) <= TOL_GRAD
    return relmax(g, go), relmax(hv, hvo)


def points(wl, n_random=2, seed=1):
    rng = np.random.default_rng(seed)
    th = wl.theta_true
    return [th, th + 0.01 * rng.standard_normal(th.size)] + list(W.random_starts(wl, n_random))


@pytest.mark.parametrize("name,nd,nm", [("tiny", 4000 + 17, 20000 + 5), ("tiny_k4", 3001, 9999),
                                        ("paper", 1500 + 3, 6000 + 29)])
def test_parity_against_oracle(name, nd, nm):
    wl, model = small_workload(name, nd, nm)
    L = make_L(wl)
    rng = np.random.default_rng(5)
    for th in points(wl):
        check_point(L, model, wl, th, rng.standard_normal(model.P))


def test_parity_k40_and_device_inputs():
    """K = 40 (the differentiation configuration's model) with inputs handed
    over as torch CUDA tensors."""
    wl, model = small_workload("diff", 700, 3001, from_model=False)
    L = make_L(wl, device_inputs=True)
    rng = np.random.default_rng(9)
    for th in points(wl, n_random=1):
        check_point(L, model, wl, th, rng.standard_normal(model.P))


@pytest.mark.parametrize("tiling", [(1, 2), (2, 3), (4, 2), (4, 3), (4, 4), (8, 2), (8, 3, 1)])
def test_every_tiling_gives_the_same_answer(tiling):
    wl, model = small_workload("paper", 1500 + 3, 6000 + 29)
    L = make_L(wl)
    if tiling[0] < 4:  # K = 20 needs at least 3 warps (at most 8 resonances per warp)
        with pytest.raises(Exception) as e:
            L.set_tiling(*tiling)
        assert "PWA_EINVAL" in str(e.value)
        return
    try:
        L.set_tiling(*tiling)
    except Exception as e:  # a tiling that does not fit must be refused cleanly
        assert "PWA_EINVAL" in str(e)
        return
    th = W.random_starts(wl, 1)[0]
    v = np.linspace(-1, 1, model.P)
    check_point(L, model, wl, th, v)


def test_runs_are_bit_identical():
    wl, model = small_workload("paper", 1500 + 3, 6000 + 29)
    L = make_L(wl)
    th = W.random_starts(wl, 1)[0]
    v = np.cos(np.arange(model.P))
    a = L.eval(th, v)
    for _ in range(3):
        b = L.eval(th, v)
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_weights_fixed_parameters_and_free_reference_coupling():
    """Non-unit data weights, fixed masses/widths, and resonance 0's coupling
    left free (the NLL is then flat along global phase and scale)."""
    wl, _ = small_workload("tiny_k4", 3001, 9999)
    rng = np.random.default_rng(2)
    w = rng.uniform(0.2, 2.0, wl.data.n).astype(np.float32)
    data = W.Sample(m2=wl.data.m2, F=wl.data.F, w=w)
    table = [W.Resonance(**{**r.__dict__}) for r in wl.table]
    table[0].fix_coupling = False
    table[1].fix_mass = True
    table[2].fix_width = True
    wl2 = W.Workload(wl.config, table, W.free_parameter_vector(table), data, wl.mc, {})
    model = oracle.Model.from_table(table, wl.S)
    L = make_L(wl2)
    assert L.P == model.P == 4 * 4 - 2
    for th in [wl2.theta_true, wl2.theta_true * 1.01]:
        check_point(L, model, wl2, th, rng.standard_normal(model.P))


def test_smallest_shapes():
    """K = 1, S = 1, one data event and one MC event."""
    t = [W.Resonance(0, 0, 1.0, 0.1, 1.0, 0.0, fix_coupling=True)]
    d = W.Sample(m2=np.array([[0.9], [2.0], [3.0]], np.float32), F=np.array([[[0.5 + 0.25j]]], np.complex64))
    m = W.Sample(m2=np.array([[1.1], [2.0], [3.0]], np.float32), F=np.array([[[1.5 - 0.5j]]], np.complex64))
    cfg = W.Config("one", 1, 1, 1, 1, 0, True, 0)
    wl = W.Workload(cfg, t, W.free_parameter_vector(t), d, m, {})
    model = oracle.Model.from_table(t, 1)
    L = make_L(wl)
    for th in [np.array([1.0, 0.1]), np.array([1.3, 0.05])]:
        check_point(L, model, wl, th, np.array([0.3, -1.0]))


def test_event_intensity_matches_oracle():
    wl, model = small_workload("paper", 1500 + 3, 6000 + 29)
    L = make_L(wl)
    th = W.random_starts(wl, 1)[0]
    for smp, s in ((0, wl.data), (1, wl.mc)):
        I = L.intensity(th, sample=smp)
        Io = oracle.intensity(model, th, s.m2, s.F)
        assert np.max(np.abs(I - Io) / Io) < 2e-4


def test_nonfinite_inputs_and_zero_intensity_are_reported():
    from paper_2403_09225_b300 import binding
    wl, _ = small_workload("tiny", 4000 + 17, 20000 + 5)
    bad = W.Sample(m2=wl.data.m2, F=wl.data.F.copy())
    bad.F[123, 1, 0] = np.nan
    with pytest.raises(binding.PwaError) as e:
        make_L(W.Workload(wl.config, wl.table, wl.theta_true, bad, wl.mc, {}))
    assert e.value.status == binding.PWA_EINVAL and "123" in str(e.value)
    zero = W.Sample(m2=wl.data.m2, F=wl.data.F.copy())
    zero.F[77] = 0  # I = 0 for data event 77: ln I is undefined
    L = make_L(W.Workload(wl.config, wl.table, wl.theta_true, zero, wl.mc, {}))
    with pytest.raises(binding.PwaError) as e:
        L.nll(wl.theta_true)
    assert e.value.status == binding.PWA_ENONFINITE and "77" in str(e.value)
    # the handle stays usable after the report
    L2 = make_L(wl)
    assert np.isfinite(L2.nll(wl.theta_true))


@pytest.mark.parametrize("warps", [1, 2, 4])
def test_small_k_tilings(warps):
    """K = 3 (tiny): one, two or four warps per block (one or several lanes per event)."""
    wl, model = small_workload("tiny", 4000 + 17, 20000 + 5)
    L = make_L(wl)
    L.set_tiling(warps, 2)
    th = W.random_starts(wl, 1)[0]
    check_point(L, model, wl, th, np.linspace(-1, 1, model.P))


def test_reuse_pass_needs_a_full_pass_at_the_same_theta():
    """pwa_hvp_reuse refuses a theta other than the last full H v pass's,
    through the host call (PWA_EINVAL) and the device call (NaN output and a
    device error reported by the next synchronising call)."""
    import torch
    from paper_2403_09225_b300 import binding
    wl, model = small_workload("tiny", 4000 + 17, 20000 + 5)
    L = make_L(wl, stream=torch.cuda.current_stream().cuda_stream)
    th = W.random_starts(wl, 2)
    v = np.linspace(-1, 1, model.P)
    with pytest.raises(binding.PwaError) as e:  # no full pass yet
        L.hvp_reuse(th[0], v)
    assert e.value.status == binding.PWA_EINVAL
    L.eval(th[0], v)
    ok = L.hvp_reuse(th[0], v)
    with pytest.raises(binding.PwaError) as e:
        L.hvp_reuse(th[1], v)
    assert e.value.status == binding.PWA_EINVAL and "theta" in str(e.value)
    d_th = torch.tensor(th[1], dtype=torch.float64, device="cuda")
    d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
    out = torch.zeros(1 + 2 * model.P, dtype=torch.float64, device="cuda")
    L.hvp_reuse_device(d_th.data_ptr(), d_v.data_ptr(), out.data_ptr())
    with pytest.raises(binding.PwaError):
        L.sync()
    assert torch.isnan(out).all()
    # after a full pass at th[1] (device call) the reuse at th[1] is served
    L.eval_device(d_th.data_ptr(), d_v.data_ptr(), out.data_ptr(), True, True)
    ref = out.cpu().numpy().copy()
    L.hvp_reuse_device(d_th.data_ptr(), d_v.data_ptr(), out.data_ptr())
    L.sync()
    got = out.cpu().numpy()
    assert relmax(got[1 + model.P:], ref[1 + model.P:]) <= 1e-5 and got[0] == ref[0]
    assert np.array_equal(got[1:1 + model.P], ref[1:1 + model.P])
    assert relmax(L.hvp_reuse(th[1], v), ref[1 + model.P:]) <= 1e-5
    assert np.isfinite(ok).all()
