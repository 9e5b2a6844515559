"""Pins of the physics-variant oracle (oracle/variants.py) against things
other than itself: the C oracle on the constant-width model it shares with
the main path, closed forms of the hyper-dual arithmetic and of the line
shapes at special points, reductions between the coupling modes, finite
differences, Hessian symmetry and the phase invariance of each projection."""
import math

import numpy as np
import pytest

import oracle
from oracle import variants as V
from paper_2403_09225_b300 import workload as W

PI_MASS, K_MASS = 0.1396, 0.4937


def tiny_samples(nd=300, nm=900, seed=3):
    cfg = W.CONFIGS["tiny"]
    table = W.make_table(cfg)
    data = W.phase_space_sample(W.rng_stream(seed, W.STREAM_DATA), nd, table, cfg.S)
    mc = W.phase_space_sample(W.rng_stream(seed, W.STREAM_MC), nm, table, cfg.S)
    return cfg, table, data, mc


def variant_model(table, S, per_projection=False, fix_first=True):
    shapes = [V.Shape(V.KIND_CONSTANT),
              V.Shape(V.KIND_MASS_DEPENDENT, ma=PI_MASS, mb=PI_MASS, radius=3.0),
              V.Shape(V.KIND_FLATTE, ma=PI_MASS, mb=PI_MASS, mc=K_MASS, md=K_MASS, width2=0.3)]
    m = V.VariantModel.from_table(table, S, shapes, per_projection)
    if not fix_first:
        m.fix_coupling[:] = False
    return m


def test_hyper_dual_closed_form():
    """f(x, y) = ln(x) / x + x y^2 at (2, 3): e2 part = df/dx, e1 e2 part =
    d2f/dx dy along (e1 = y, e2 = x)."""
    x = V.HD(2.0, 0.0, 1.0, 0.0)
    y = V.HD(3.0, 1.0, 0.0, 0.0)
    f = x.log() / x + x * y * y
    assert abs(f.a - (math.log(2) / 2 + 18)) < 1e-14
    assert abs(f.c - ((1 - math.log(2)) / 4 + 9)) < 1e-14
    assert abs(f.d - 2 * 3) < 1e-14
    assert abs(V.HD(4.0, 1.0, 1.0).sqrt().d - (-0.25 / 8)) < 1e-15


def test_constant_width_matches_the_c_oracle():
    cfg, table, data, mc = tiny_samples()
    vm = V.VariantModel.from_table(table, cfg.S)
    cm = oracle.Model.from_table(table, cfg.S)
    assert vm.P == cm.P
    rng = np.random.default_rng(1)
    th = W.free_parameter_vector(table) * (1 + 0.05 * rng.standard_normal(vm.P))
    v = rng.standard_normal(vm.P)
    f, g, hv = V.nll_grad_hvp(vm, th, v, data, mc)
    fo, go, hvo = oracle.nll_grad_hvp(cm, th, v, data, mc)
    assert abs(f - fo) <= 1e-11 * abs(fo)
    assert np.max(np.abs(g - go)) <= 1e-9 * np.max(np.abs(go))
    assert np.max(np.abs(hv - hvo)) <= 1e-9 * np.max(np.abs(hvo))


def test_equal_projection_couplings_reduce_to_one_coupling():
    cfg, table, data, mc = tiny_samples()
    m1 = variant_model(table, cfg.S, per_projection=False)
    mS = variant_model(table, cfg.S, per_projection=True)
    th1 = m1.theta0()
    lay1, layS = m1.layout(), mS.layout()
    thS = np.array([th1[[i for i, (n1, k1, _) in enumerate(lay1) if (n1, k1) == (n, k)][0]] for n, k, s in layS])
    f1, g1, _ = V.nll_grad_hvp(m1, th1, np.zeros(m1.P), data, mc)
    fS, gS, _ = V.nll_grad_hvp(mS, thS, np.zeros(mS.P), data, mc)
    assert abs(f1 - fS) <= 1e-12 * abs(f1)
    # a coupling shared by all projections: its derivative is the sum over projections
    for i, (n, k, _) in enumerate(lay1):
        js = [j for j, (nS, kS, _) in enumerate(layS) if (nS, kS) == (n, k)]
        assert abs(g1[i] - sum(gS[j] for j in js)) <= 1e-9 * max(1.0, abs(g1[i]))


def test_line_shapes_at_special_points():
    # mass-dependent width at m = M: Gamma(M) = Gamma0, so D = -i M Gamma0
    cfg, table, _, _ = tiny_samples(10, 10)
    vm = variant_model(table, cfg.S)
    M, G0 = 1.2, 0.15
    bw = V.breit_wigner(vm, 1, np.array([M * M]), V.HD(M), V.HD(G0), V.HD(0.0))
    assert abs(bw.a[0] - 1.0 / (-1j * M * G0)) <= 1e-14 * abs(bw.a[0])
    # Flatte below the KK threshold: the gamma2 term is real and moves Re D only
    m2 = np.array([0.8 ** 2])
    g1, g2 = 0.2, 0.5
    D = V.breit_wigner(vm, 2, m2, V.HD(0.98), V.HD(g1), V.HD(g2)).inv().a[0]
    q1 = math.sqrt((0.64 - (2 * PI_MASS) ** 2) / 4)
    k2 = math.sqrt((2 * K_MASS) ** 2 / 4 - 0.64 / 4)  # |q_KK| below threshold
    assert abs(D.imag - (-g1 * 2 * q1 / 0.8)) <= 1e-14
    assert abs(D.real - (0.98 ** 2 - 0.64 + g2 * 2 * k2 / 0.8)) <= 1e-14
    # the barrier factor: F_1^2(z) = 2 z / (1 + z)
    assert abs(V.barrier_sq(1, 3.0) - 1.5) < 1e-15


@pytest.mark.parametrize("per_projection", [False, True])
def test_variants_match_finite_differences(per_projection):
    cfg, table, data, mc = tiny_samples()
    vm = variant_model(table, cfg.S, per_projection)
    rng = np.random.default_rng(2)
    th = vm.theta0() * (1 + 0.05 * rng.standard_normal(vm.P))
    v = rng.standard_normal(vm.P)
    f, g, hv = V.nll_grad_hvp(vm, th, v, data, mc)
    h = 1e-5
    for j in range(vm.P):
        e = np.zeros(vm.P)
        e[j] = h
        fd = (-V.nll(vm, th + 2 * e, data, mc) + 8 * V.nll(vm, th + e, data, mc)
              - 8 * V.nll(vm, th - e, data, mc) + V.nll(vm, th - 2 * e, data, mc)) / (12 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, np.max(np.abs(g))), (j, fd, g[j])
    # H v from central differences of the gradient along v
    t = 1e-5
    _, gp, _ = V.nll_grad_hvp(vm, th + t * v, v, data, mc)
    _, gm, _ = V.nll_grad_hvp(vm, th - t * v, v, data, mc)
    fd_hv = (gp - gm) / (2 * t)
    assert np.max(np.abs(fd_hv - hv)) <= 1e-5 * np.max(np.abs(hv))


def test_variant_hessian_is_symmetric():
    cfg, table, data, mc = tiny_samples()
    vm = variant_model(table, cfg.S, per_projection=True)
    rng = np.random.default_rng(4)
    th = vm.theta0()
    u, v = rng.standard_normal(vm.P), rng.standard_normal(vm.P)
    uhv = float(np.real(V.nll_hd(vm, th, data, mc, v=v, u=u).d))
    vhu = float(np.real(V.nll_hd(vm, th, data, mc, v=u, u=v).d))
    assert abs(uhv - vhu) <= 1e-10 * max(abs(uhv), 1.0)


def test_each_projection_has_its_own_phase_invariance():
    """With one coupling per (resonance, projection), rotating every coupling
    of one projection s by the same phase leaves I unchanged, and the
    gradient is orthogonal to that direction."""
    cfg, table, data, mc = tiny_samples()
    vm = variant_model(table, cfg.S, per_projection=True, fix_first=False)
    th = vm.theta0() + 0.1 * np.arange(vm.P) / vm.P
    lay = vm.layout()
    d = np.array([1.0 if (n == "phase" and s == 1) else 0.0 for n, k, s in lay])
    f0 = V.nll(vm, th, data, mc)
    assert abs(V.nll(vm, th + 0.7 * d, data, mc) - f0) <= 1e-12 * abs(f0)
    _, g, _ = V.nll_grad_hvp(vm, th, np.zeros(vm.P), data, mc)
    assert abs(g @ d) <= 1e-9 * np.max(np.abs(g))


@pytest.mark.parametrize("per_projection", [False, True])
def test_integral_matrices_give_the_mc_sum(per_projection):
    """sum_e I(e) = sum_s g_s^H Phi_s g_s for any couplings (the MC term of
    Eq. 3 from the integral matrices), and each Phi_s is Hermitian."""
    cfg, table, data, mc = tiny_samples()
    vm = variant_model(table, cfg.S, per_projection)
    rng = np.random.default_rng(9)
    th = vm.theta0() * (1 + 0.05 * rng.standard_normal(vm.P))
    phi = V.integral_matrices(vm, th, mc.m2, mc.F)
    for s in range(cfg.S):
        assert np.allclose(phi[s], np.conj(phi[s].T), rtol=0, atol=1e-9 * np.abs(phi[s]).max())
    pars = V._params(vm, th)
    mag, phase = pars[0], pars[1]
    G = 0.0
    for s in range(cfg.S):
        j = s if per_projection else 0
        g = np.array([mag[k][j].a * np.exp(1j * phase[k][j].a) for k in range(vm.K)])
        G += float(np.real(np.conj(g) @ phi[s] @ g))
    I = V.intensity(vm, th, mc.m2, mc.F)
    assert abs(G - I.sum()) <= 1e-10 * I.sum()
    assert V.coupling_count(vm) == (4 * cfg.S if per_projection else 4)
