"""Pseudo-experiment generation on the GPU (accept-reject from a pool,
binned Dalitz plot, gather) against the CPU oracle (oracle/generate.py).

Index and count outputs are integer results: bit-exact.  The log-scaled
histogram is one FP32 log1p per bin: within 1e-6 relative.  Inputs are
seeded synthetic intensities and coordinates, so no oracle input comes from
the library."""
import numpy as np
import pytest

from oracle import generate as og

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,start,n_target,C", [(1, 0, 1, 0.0), (1000, 999, 10 ** 6, 0.0),
                                                (50_000 + 17, 12_345, 5_000, 0.0),
                                                (3 * 1024 * 1024 + 5, 7, 300_000, 9.0),
                                                (200_003, 100_000, 0, 0.0)])
def test_accept_reject_bit_exact(n, start, n_target, C):
    from paper_2403_09225_b300 import binding
    rng = np.random.default_rng(n)
    # a peaked intensity with some exact zeros: acceptance varies along the pool
    I = (rng.random(n) ** 4 * 8).astype(np.float32)
    I[rng.random(n) < 0.05] = 0.0
    idx, C_used = binding.accept_reject(_cuda(I), seed=n + 3, start=start, n_target=n_target, C=C)
    want, C_want = og.accept_reject(I, C, seed=n + 3, start=start, n_target=n_target)
    assert C_used == C_want
    got = idx.cpu().numpy().astype(np.int64)
    assert got.shape == want.shape and np.array_equal(got, want)


def test_accept_reject_rejects_bad_input():
    from paper_2403_09225_b300 import binding
    I = np.ones(100, np.float32)
    I[50] = np.nan
    with pytest.raises(binding.PwaError):
        binding.accept_reject(_cuda(I), seed=1, start=0, n_target=10)
    I[50] = -1.0
    with pytest.raises(binding.PwaError):
        binding.accept_reject(_cuda(I), seed=1, start=0, n_target=10)
    with pytest.raises(binding.PwaError):
        binding.accept_reject(_cuda(np.ones(10, np.float32)), seed=1, start=10, n_target=10)


@pytest.mark.parametrize("nb,n", [(64, 100_000 + 3), (8, 1), (64, 0), (128, 5000)])
def test_dalitz_histogram(nb, n):
    import torch
    from paper_2403_09225_b300 import binding, workload as W
    rng = np.random.default_rng(nb + n)
    ld = max(2 * n, 10)
    bounds = W.dalitz_bounds()
    m2 = np.stack([rng.uniform(bounds[0] - 0.1, bounds[1] + 0.1, ld), rng.uniform(0, 9, ld),
                   rng.uniform(bounds[2] - 0.1, bounds[3] + 0.1, ld)]).astype(np.float32)
    idx = rng.choice(ld, size=n, replace=False).astype(np.int32)
    idx_d = _cuda(idx) if n else torch.empty(0, dtype=torch.int32, device="cuda")
    raw = binding.dalitz_histogram(_cuda(m2), idx_d, nb, bounds, log_scale=False).cpu().numpy()
    want = og.dalitz_histogram(m2, idx.astype(np.int64), nb, bounds, log_scale=False)
    assert np.array_equal(raw.astype(np.float64), want)
    lg = binding.dalitz_histogram(_cuda(m2), idx_d, nb, bounds, log_scale=True).cpu().numpy()
    wl = og.dalitz_histogram(m2, idx.astype(np.int64), nb, bounds, log_scale=True)
    assert np.allclose(lg, wl, rtol=1e-6, atol=0)


def test_gather_events_bit_exact():
    from paper_2403_09225_b300 import binding
    rng = np.random.default_rng(4)
    ld, K, S = 10_007, 20, 4
    m2 = rng.random((3, ld)).astype(np.float32)
    F = rng.standard_normal((ld, K, S, 2)).astype(np.float32)
    idx = rng.choice(ld, size=3001, replace=True).astype(np.int32)
    m2o, Fo = binding.gather_events(_cuda(m2), _cuda(F), _cuda(idx))
    assert np.array_equal(m2o.cpu().numpy(), m2[:, idx])
    assert np.array_equal(Fo.cpu().numpy(), F[idx])


def test_pool_pseudo_experiment_follows_the_model():
    """End to end at the tiny model: I of a phase-space pool from the
    library, accept-reject, and the kept events' histogram against the
    oracle's intensity-weighted histogram of the same pool (chi-square)."""
    import oracle
    from paper_2403_09225_b300 import proposal, workload as W
    cfg = W.CONFIGS["tiny"]
    table = W.make_table(cfg)
    gen = proposal.Generator(table, cfg.S, pool_size=1_000_000, n_mc=20_000, seed=11, nb=8)
    theta = W.free_parameter_vector(table)
    idx = gen.draw(theta, 20_000, seed=5)
    n = idx.numel()
    assert n == 20_000
    h = gen.features(idx)  # log scaled
    counts = np.round(np.expm1(h.cpu().numpy()) * n / 64).astype(np.int64)
    assert counts.sum() == n
    # the oracle: expected counts from I over the same pool (FP64)
    model = oracle.Model.from_table(table, cfg.S)
    m2 = gen.pool_m2.cpu().numpy()
    F = gen.pool_F.cpu().numpy().view(np.complex64)[..., 0]
    I = oracle.intensity(model, theta, m2, F)
    x0, x1, y0, y1 = gen.bounds
    bx = np.clip(np.floor((m2[0].astype(np.float64) - x0) * 8 / (x1 - x0)), 0, 7).astype(int)
    by = np.clip(np.floor((m2[2].astype(np.float64) - y0) * 8 / (y1 - y0)), 0, 7).astype(int)
    expect = np.bincount(bx * 8 + by, weights=I, minlength=64)
    expect = expect / expect.sum() * n
    ok = expect > 5
    chi2 = np.sum((counts[ok] - expect[ok]) ** 2 / expect[ok])
    dof = int(ok.sum()) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)
    gen.close()
