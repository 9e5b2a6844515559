"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test checks the oracle against something the mathematics or the paper
fixes, chosen so that a plausible slip (a dropped term, a wrong sign or index,
a transposed operand) fails at least one of them:
  * central finite differences of the NLL (gradient) and of the gradient (HVP);
  * the full Hessian, built by a second code path, against the HVP, and its symmetry;
  * the closed form for one resonance with a constant amplitude projection;
  * invariance under a global phase and scale of all couplings;
  * independence of S when every resonance sits in one channel;
  * additivity of the per-shard sums (paper Eqs. 4-5);
  * error reporting for non-finite or vanishing intensities.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2403_09225_b300 import workload as W


def rel(a, b):
    a, b = np.atleast_1d(a), np.atleast_1d(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def points(wl, model, n_random=2, seed=7):
    """theta_true, theta_true + offsets, and random starts from the prior."""
    rng = np.random.default_rng(seed)
    th = wl.theta_true
    pts = [th, th + 0.02 * rng.standard_normal(th.size)]
    pts += list(W.random_starts(wl, n_random))
    return pts


def fd_grad(f, x, rel_step=2e-5):
    """Five-point central differences (truncation O(h^4)): narrow widths make
    the third derivative large, which a plain two-point stencil would see."""
    g = np.empty_like(x)
    for i in range(x.size):
        h = rel_step * max(1.0, abs(x[i]))

        def at(t):
            xx = x.copy()
            xx[i] += t
            return f(xx)
        g[i] = (8 * (at(h) - at(-h)) - (at(2 * h) - at(-2 * h))) / (12 * h)
    return g


def fd_dir(gfun, x, v, h=2e-5):
    """Five-point central difference of a vector function along v."""
    return (8 * (gfun(x + h * v) - gfun(x - h * v)) - (gfun(x + 2 * h * v) - gfun(x - 2 * h * v))) / (12 * h)


@pytest.mark.parametrize("which", ["tiny_small", "paper_small"])
def test_gradient_matches_central_differences(which, request):
    wl, model = request.getfixturevalue(which)
    for th in points(wl, model, n_random=1):
        f, g = oracle.nll_grad(model, th, wl.data, wl.mc)
        g_fd = fd_grad(lambda x: oracle.nll(model, x, wl.data, wl.mc), th)
        assert rel(g, g_fd) < 1e-8, (which, rel(g, g_fd))


@pytest.mark.parametrize("which", ["tiny_small", "paper_small"])
def test_hvp_matches_differences_of_gradient(which, request):
    wl, model = request.getfixturevalue(which)
    rng = np.random.default_rng(3)
    for th in points(wl, model, n_random=1):
        v = rng.standard_normal(model.P)
        _, _, hv = oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
        hv_fd = fd_dir(lambda x: oracle.nll_grad(model, x, wl.data, wl.mc)[1], th, v)
        assert rel(hv, hv_fd) < 1e-7, (which, rel(hv, hv_fd))


def test_full_hessian_agrees_with_hvp_and_is_symmetric(tiny_small):
    wl, model = tiny_small
    rng = np.random.default_rng(11)
    th = W.random_starts(wl, 1)[0]
    H = oracle.hessian(model, th, wl.data, wl.mc)
    assert rel(H, H.T) < 1e-12
    for _ in range(3):
        v = rng.standard_normal(model.P)
        u = rng.standard_normal(model.P)
        hv = oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)[2]
        hu = oracle.nll_grad_hvp(model, th, u, wl.data, wl.mc)[2]
        assert rel(hv, H @ v) < 1e-10
        assert abs(u @ hv - v @ hu) <= 1e-10 * max(abs(u @ hv), 1.0)


def _k1_constant_F(n_data, n_mc, S=2, seed=5):
    rng = np.random.default_rng(seed)
    lo, hi = W.channel_mass_range(0)
    md = rng.uniform(lo, hi, n_data) ** 2
    mm = rng.uniform(lo, hi, n_mc) ** 2
    f = np.array([0.7 - 0.4j, 0.2 + 1.1j][:S], dtype=np.complex64)
    mk = lambda m: np.stack([m, np.full_like(m, 2.0), np.full_like(m, 3.0)]).astype(np.float32)
    data = W.Sample(m2=mk(md), F=np.tile(f, (n_data, 1, 1)).reshape(n_data, 1, S))
    mc = W.Sample(m2=mk(mm), F=np.tile(f, (n_mc, 1, 1)).reshape(n_mc, 1, S))
    return data, mc


def test_closed_form_one_resonance_constant_F():
    """K = 1, F constant: I = rho^2 |BW|^2 sum_s |F_s|^2, so
    NLL = sum_d ln((M^2 - m^2)^2 + M^2 G^2) + N_d ln(mean_mc 1/((M^2 - m^2)^2 + M^2 G^2)),
    independent of the coupling, whose derivatives vanish."""
    data, mc = _k1_constant_F(700, 3000)
    model = oracle.Model([0], [1.3], [0.4], [1.1], [0.15], [False], [False], [False], S=2)
    for (rho, phi, M, G) in [(1.3, 0.4, 1.1, 0.15), (0.2, -2.0, 0.8, 0.05), (5.0, 3.0, 1.9, 0.3)]:
        th = np.array([rho, phi, M, G])
        md = data.m2[0].astype(np.float64)
        mm = mc.m2[0].astype(np.float64)
        den = lambda m: (M * M - m) ** 2 + M * M * G * G
        expect = np.sum(np.log(den(md))) + md.size * math.log(np.mean(1.0 / den(mm)))
        f, g = oracle.nll_grad(model, th, data, mc)
        assert abs(f - expect) <= 1e-11 * abs(expect)
        scale = np.max(np.abs(g))
        assert abs(g[0]) <= 1e-9 * scale and abs(g[1]) <= 1e-9 * scale


def _all_couplings_free(wl):
    t = wl.table
    return oracle.Model([r.channel for r in t], [r.mag for r in t], [r.phase for r in t],
                        [r.mass for r in t], [r.width for r in t],
                        [False] * len(t), [False] * len(t), [False] * len(t), wl.S)


@pytest.mark.parametrize("which", ["tiny_small", "paper_small"])
def test_global_phase_and_scale_invariance(which, request):
    wl, _ = request.getfixturevalue(which)
    model = _all_couplings_free(wl)
    K = model.K
    th = model.par0.copy()
    f0, g0 = oracle.nll_grad(model, th, wl.data, wl.mc)
    for lam, alpha in [(2.5, 0.0), (1.0, 1.1), (0.3, -2.7)]:
        t2 = th.copy()
        t2[:K] *= lam
        t2[K:2 * K] += alpha
        f2 = oracle.nll(model, t2, wl.data, wl.mc)
        assert abs(f2 - f0) <= 1e-11 * abs(f0)
    d_scale = np.zeros(4 * K); d_scale[:K] = th[:K]
    d_phase = np.zeros(4 * K); d_phase[K:2 * K] = 1.0
    gn = np.linalg.norm(g0)
    assert abs(g0 @ d_scale) <= 1e-10 * gn * np.linalg.norm(d_scale)
    assert abs(g0 @ d_phase) <= 1e-10 * gn * np.linalg.norm(d_phase)


def test_s_independence_in_a_single_channel(tiny_small):
    """All resonances in m12: e^{i s phi} is common to every term of A_s, so
    I = S * I_{S=1} and the NLL does not depend on S (up to FP32 rounding of F)."""
    wl, model = tiny_small
    assert all(r.channel == 0 for r in wl.table)
    m1 = oracle.Model.from_table(wl.table, 1)
    d1 = W.Sample(m2=wl.data.m2, F=np.ascontiguousarray(wl.data.F[:, :, :1]))
    c1 = W.Sample(m2=wl.mc.m2, F=np.ascontiguousarray(wl.mc.F[:, :, :1]))
    for th in W.random_starts(wl, 2):
        f2 = oracle.nll(model, th, wl.data, wl.mc)
        f1 = oracle.nll(m1, th, d1, c1)
        assert abs(f2 - f1) <= 1e-8 * abs(f1), (f1, f2)


def test_shard_sums_add_up(paper_small):
    """Eqs. 4-5: sums over disjoint event shards combine to the whole."""
    wl, model = paper_small
    th = W.random_starts(wl, 1)[0]
    v = np.linspace(-1, 1, model.P)
    whole = oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
    parts = oracle.sharded_nll_grad_hvp(model, th, v, wl.data, wl.mc, workers=2, shard=1000)
    assert abs(parts[0] - whole[0]) <= 1e-12 * abs(whole[0])
    assert rel(parts[1], whole[1]) < 1e-11
    assert rel(parts[2], whole[2]) < 1e-11


def test_bad_events_are_reported(tiny_small):
    wl, model = tiny_small
    data = W.Sample(m2=wl.data.m2.copy(), F=wl.data.F.copy())
    data.F[17] = 0  # I = 0 for a data event: ln I undefined
    with pytest.raises(oracle.OracleError) as e:
        oracle.nll(model, wl.theta_true, data, wl.mc)
    assert e.value.index == 17
    mc = W.Sample(m2=wl.mc.m2.copy(), F=wl.mc.F.copy())
    mc.F[5, 0, 0] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.nll(model, wl.theta_true, wl.data, mc)
    assert e.value.index == wl.data.n + 5


def test_integral_matrix_reproduces_the_mc_sum(paper_small):
    """Eq. 1 with the couplings factored out: sum_mc I(e) = g^H Phi g for any
    couplings at fixed masses and widths; Phi is Hermitian positive
    semi-definite.  Pins the oracle's integral matrix against its own
    intensity (an independent loop over events)."""
    wl, model = paper_small
    rng = np.random.default_rng(31)
    for th in (wl.theta_true, W.random_starts(wl, 1)[0]):
        phi = oracle.integral_matrix(model, th, wl.mc.m2, wl.mc.F)
        assert np.allclose(phi, phi.conj().T, rtol=0, atol=1e-10 * np.abs(phi).max())
        assert np.linalg.eigvalsh(phi).min() >= -1e-9 * np.abs(phi).max()
        # other couplings at the same masses and widths
        th2 = th.copy()
        nc = int(np.sum([not r.fix_coupling for r in wl.table]))
        th2[:2 * nc] += 0.3 * rng.standard_normal(2 * nc)
        g = oracle.couplings(model, th2)
        total = float(np.sum(oracle.intensity(model, th2, wl.mc.m2, wl.mc.F)))
        assert abs(np.real(g.conj() @ phi @ g) - total) <= 1e-11 * total


def test_mlp_oracle_gradients_match_finite_differences():
    """The proposal network's oracle (plain FP64, no rounding): backward pass
    against central differences of its own loss, for squared-error and
    periodic (1 - cos) outputs."""
    from oracle import mlp
    rng = np.random.default_rng(3)
    sizes = [12, 8, 8, 5]
    params = mlp.init_params(sizes, seed=1)
    x = rng.standard_normal((7, 12))
    t = rng.standard_normal((7, 5))
    weight = np.array([1.0, 0.5, 2.0, 1.0, 1.0])
    periodic = [0, 0, 1, 0, 1]
    loss, grads = mlp.loss_and_grads(params, x, t, weight, periodic)
    h = 1e-6

    def perturbed(l, which, idx, s):
        ps = [(w.copy(), bb.copy()) for w, bb in params]
        ps[l][which][idx] += s
        return mlp.loss_and_grads(ps, x, t, weight, periodic)[0]

    for l, (W, b) in enumerate(params):
        for idx in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            fd = (perturbed(l, 0, idx, h) - perturbed(l, 0, idx, -h)) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, grads[l][0][idx])
        k = (b.size - 1,)
        fd = (perturbed(l, 1, k, h) - perturbed(l, 1, k, -h)) / (2 * h)
        assert abs(fd - grads[l][1][k]) <= 1e-6 * max(1.0, abs(fd))


def test_mlp_oracle_reduces_to_least_squares():
    """One affine layer with squared error: the loss is the least-squares
    objective, whose gradient vanishes at numpy's lstsq solution."""
    from oracle import mlp
    rng = np.random.default_rng(4)
    x = rng.standard_normal((40, 6))
    t = rng.standard_normal((40, 3))
    X1 = np.hstack([x, np.ones((40, 1))])
    sol = np.linalg.lstsq(X1, t, rcond=None)[0]
    params = [(sol[:6].T.copy(), sol[6].copy())]
    loss, grads = mlp.loss_and_grads(params, x, t, np.ones(3), [0, 0, 0])
    assert np.max(np.abs(grads[0][0])) < 1e-12 and np.max(np.abs(grads[0][1])) < 1e-12
    assert abs(loss - 0.5 * np.sum((X1 @ sol - t) ** 2) / 40) < 1e-12


def test_bf16_rounding_is_nearest_even():
    from oracle import mlp
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even 1
    assert mlp.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert mlp.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    x = np.random.default_rng(0).standard_normal(1000)
    assert np.max(np.abs(mlp.bf16(x) - x) / np.abs(x)) <= 2 ** -8


def test_splitmix64_known_answers():
    """splitmix64 started at 0: its first three outputs as published with the
    reference implementation (Vigna, splitmix64.c)."""
    from oracle import generate as og
    out = og.splitmix64(0, np.arange(3))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_accept_reject_oracle_against_a_plain_loop_and_its_distribution():
    from oracle import generate as og
    rng = np.random.default_rng(5)
    n = 3000
    I = rng.random(n).astype(np.float32) * 4
    idx, C = og.accept_reject(I, 0.0, seed=77, start=1234, n_target=400)
    assert C == float(np.float32(I).max())
    # brute force: walk the pool from `start`, keep while fewer than n_target
    want = []
    for i in range(n):
        j = (1234 + i) % n
        u = int(og.splitmix64(77, np.array([j]))[0] >> np.uint64(11)) * 2.0 ** -53
        if u * C < float(I[j]) and len(want) < 400:
            want.append(j)
    assert idx.tolist() == want
    # I = C everywhere keeps every event in order; I = 0 keeps none
    full, _ = og.accept_reject(np.full(50, 2.0, np.float32), 2.0, seed=1, start=45, n_target=50)
    assert full.tolist() == list(range(45, 50)) + list(range(45))
    none, _ = og.accept_reject(np.zeros(50, np.float32), 1.0, seed=1, start=0, n_target=50)
    assert none.size == 0
    # kept fraction per intensity band follows I / C (binomial, 5 sigma)
    I = np.repeat(np.array([0.1, 0.5, 0.9], np.float32), 20000)
    idx, _ = og.accept_reject(I, 1.0, seed=9, start=0, n_target=10 ** 9)
    for b, p in enumerate([0.1, 0.5, 0.9]):
        k = np.sum((idx >= 20000 * b) & (idx < 20000 * (b + 1)))
        assert abs(k - 20000 * p) < 5 * np.sqrt(20000 * p * (1 - p))


def test_dalitz_histogram_oracle_against_a_plain_loop():
    from oracle import generate as og
    rng = np.random.default_rng(8)
    m2 = rng.uniform(0.0, 9.0, size=(3, 500)).astype(np.float32)
    idx = rng.choice(500, size=300, replace=False)
    bounds = (0.5, 8.0, 0.25, 7.5)
    h = og.dalitz_histogram(m2, idx, 8, bounds, log_scale=False)
    want = np.zeros(64)
    for e in idx:
        bx = min(max(int(math.floor((float(m2[0, e]) - 0.5) * 8 / 7.5)), 0), 7)
        by = min(max(int(math.floor((float(m2[2, e]) - 0.25) * 8 / 7.25)), 0), 7)
        want[bx * 8 + by] += 1
    assert np.array_equal(h, want) and h.sum() == 300
    hl = og.dalitz_histogram(m2, idx, 8, bounds, log_scale=True)
    assert np.allclose(hl, np.log(1 + want * 64 / 300), rtol=0, atol=1e-15)


def test_sharded_hessian_matches_the_single_pass_hessian(paper_small):
    """Shard sums of the second derivatives combined by Eq. 7 on the host
    (oracle.sharded_hessian) equal the C combination of the whole-sample sums
    (oracle.hessian): shard additivity (Eqs. 4-5) for the Hessian, and the two
    combinations of Eq. 7 agree."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    wl, model = paper_small
    th = W.random_starts(wl, 1)[0]
    with ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context("spawn")) as pool:
        f, g, H = oracle.sharded_hessian(model, th, wl.data, wl.mc, pool=pool, shard=1000)
    fo, go = oracle.nll_grad(model, th, wl.data, wl.mc)
    Ho = oracle.hessian(model, th, wl.data, wl.mc)
    assert abs(f - fo) <= 1e-12 * abs(fo)
    assert rel(g, go) <= 1e-12
    assert rel(H, Ho) <= 1e-12
