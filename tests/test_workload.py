"""Checks of the seeded input generator (shared by the oracle and the GPU path)."""
import numpy as np

import oracle
from paper_2403_09225_b300 import workload as W


def test_phase_space_events_are_physical():
    cfg = W.CONFIGS["paper"]
    table = W.make_table(cfg)
    s = W.phase_space_sample(W.rng_stream(1, W.STREAM_MC), 20000, table, cfg.S)
    m2 = s.m2.astype(np.float64)
    # m12^2 + m13^2 + m23^2 = M^2 + sum m_i^2
    total = W.PARENT_MASS ** 2 + sum(m * m for m in W.DAUGHTER_MASSES)
    assert np.allclose(m2.sum(axis=0), total, rtol=1e-6)
    for ch in range(3):
        lo, hi = W.channel_mass_range(ch)
        assert m2[ch].min() >= lo * lo * (1 - 1e-6) and m2[ch].max() <= hi * hi * (1 + 1e-6)
    assert np.all(W.inside_dalitz(m2[0] * (1 + 1e-7) - 1e-9, m2[2]) | W.inside_dalitz(m2[0], m2[2]))
    assert s.F.shape == (20000, cfg.K, cfg.S) and s.F.dtype == np.complex64
    assert np.all(np.isfinite(s.F.view(np.float32)))


def test_same_seed_same_events():
    cfg = W.CONFIGS["tiny"]
    table = W.make_table(cfg)
    a = W.phase_space_sample(W.rng_stream(5, W.STREAM_MC), 3000, table, cfg.S)
    b = W.phase_space_sample(W.rng_stream(5, W.STREAM_MC), 3000, table, cfg.S)
    assert np.array_equal(a.m2, b.m2) and np.array_equal(a.F, b.F)


def test_proposal_density_is_normalised():
    """The accept-reject proposal must be an exact density: its mean over
    uniform Dalitz points times the Dalitz area is 1."""
    for name in ("tiny", "paper"):
        table = W.make_table(W.CONFIGS[name])
        prop = W.Proposal(table)
        x, y = W.uniform_dalitz(np.random.default_rng(3), 1_000_000)
        q = prop.density(x, y)
        est = np.mean(q) * prop.area
        err = np.std(q) * prop.area / np.sqrt(q.size)
        assert abs(est - 1) < 5 * err + 1e-3, (name, est, err)


def test_accept_reject_sample_follows_the_intensity():
    """Histogram of m12^2 in a sample drawn from I agrees (chi^2) with phase
    space reweighted by I."""
    cfg = W.CONFIGS["tiny"]
    table = W.make_table(cfg)
    model = oracle.Model.from_table(table, cfg.S)
    fn = lambda m2, F: oracle.intensity_full(cfg.K, cfg.S, model.channels, model.par0, m2, F)
    data, stats = W.accept_reject_sample(W.rng_stream(8, W.STREAM_DATA), 20000, table, cfg.S, fn)
    assert stats["restarts"] == 0 or stats["C"] > 0
    ps = W.phase_space_sample(W.rng_stream(9, W.STREAM_MC), 300000, table, cfg.S)
    wgt = fn(ps.m2, ps.F)
    edges = np.linspace(ps.m2[0].min(), ps.m2[0].max(), 31)
    h_data, _ = np.histogram(data.m2[0], edges)
    h_ps, _ = np.histogram(ps.m2[0], edges, weights=wgt)
    h_ps2, _ = np.histogram(ps.m2[0], edges, weights=wgt ** 2)
    expect = h_ps / h_ps.sum() * data.n
    var = expect + h_ps2 / h_ps.sum() ** 2 * data.n ** 2
    ok = expect > 5
    chi2 = np.sum((h_data[ok] - expect[ok]) ** 2 / var[ok])
    dof = int(ok.sum())
    assert chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof)
