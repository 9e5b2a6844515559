"""Host logic of the learned proposal (no GPU): canonical labels, the
target codec and the time-to-minimum summary."""
import math

import numpy as np

from paper_2403_09225_b300 import proposal, workload as W


def _table():
    return W.make_table(W.CONFIGS["paper"])


def test_layout_matches_the_library_theta_order():
    table = _table()
    lay = proposal.Layout.of(table)
    th = W.free_parameter_vector(table)
    assert lay.P == th.size == 78
    for k, r in enumerate(table):
        if lay.rho[k] >= 0:
            assert th[lay.rho[k]] == r.mag and th[lay.phi[k]] == r.phase
        assert th[lay.mass[k]] == r.mass and th[lay.width[k]] == r.width
    assert lay.periodic().sum() == 19


def test_canonical_sorts_groups_flips_signs_and_is_idempotent():
    table = _table()
    lay = proposal.Layout.of(table)
    groups = proposal.exchangeable_groups(table)
    assert len(groups) >= 3 and all(len(g) >= 2 for g in groups)
    rng = np.random.default_rng(0)
    th = np.stack([W.sample_start(rng, table) for _ in range(5)])
    g = groups[0]
    th[0, lay.rho[g[0]]] = -0.7
    th[0, lay.phi[g[0]]] = 3.0
    c = proposal.canonical(table, th)
    assert np.allclose(proposal.canonical(table, c), c)
    assert np.all(c[:, lay.rho[lay.rho >= 0]] >= 0)
    assert np.all(np.abs(c[:, lay.phi[lay.phi >= 0]]) <= math.pi + 1e-12)
    for grp in groups:
        assert np.all(np.diff(c[:, lay.mass[grp]], axis=1) >= 0)
    # the flipped coupling is the same complex number
    k = g[0]
    row = c[0]
    # find where resonance k's (rho, phi, M, Gamma) went after sorting: the mass is unique
    M = th[0, lay.mass[k]]
    kk = [q for q in g if abs(row[lay.mass[q]] - M) < 1e-15][0]
    z0 = -0.7 * np.exp(3.0j)
    z1 = row[lay.rho[kk]] * np.exp(1j * row[lay.phi[kk]])
    assert abs(z0 - z1) < 1e-12


def test_codec_round_trip_and_box():
    table = _table()
    rng = np.random.default_rng(1)
    labels = np.stack([W.sample_start(rng, table) for _ in range(200)])
    codec = proposal.Codec(table, labels)
    t = codec.encode(labels)
    back = codec.decode(t)
    # decode maps into the prior's box (masses 1e-3 inside the channel range)
    assert np.max(np.abs(back - np.clip(labels, codec.lo, codec.hi))) < 1e-5
    wild = codec.decode(100 * np.ones_like(t))
    lay = codec.lay
    for k, r in enumerate(table):
        lo, hi = W.channel_mass_range(r.channel)
        assert lo < wild[0, lay.mass[k]] < hi
    assert np.all(np.abs(wild[:, codec.periodic]) <= math.pi)


def test_summary_time_to_minimum():
    recs = [dict(t_random=2.0, random_hits=1, t_mlp=0.5, mlp_hit=True, nll_mlp=0.0, best=0.0, nll_random=[0.0, 1.0],
                 t_learned_batch=0.8, learned_batch_hit=True),
            dict(t_random=2.0, random_hits=0, t_mlp=0.5, mlp_hit=False, nll_mlp=5.0, best=0.0, nll_random=[2.0, 3.0],
                 t_learned_batch=0.8, learned_batch_hit=False)]
    s = proposal.summarize(recs, n_random=2, n_learned=4)
    p = 1 / 4
    e = 2.0 / (1 - (1 - p) ** 2)
    assert math.isclose(s["random_hit_rate"], p)
    assert math.isclose(s["random_s_to_min"], e)
    assert math.isclose(s["learned_s_to_min"], (0.5 + 0.5 + e) / 2)
    assert math.isclose(s["learned_batch_s_to_min"], (0.8 + 0.8 + e) / 2)
    assert s["mlp_hit_rate"] == 0.5


def test_summary_of_the_polished_forms():
    recs = [dict(t_random=2.0, random_hits=1, t_mlp=0.5, mlp_hit=False, nll_mlp=1.0, best=0.0,
                 nll_random=[0.0, 1.0], t_learned_batch=0.8, learned_batch_hit=True,
                 t_polish=0.6, polish_hit=True, t_polish_batch=0.9, polish_batch_hit=False)]
    s = proposal.summarize(recs, n_random=2, n_learned=4)
    e = 2.0 / (1 - (1 - 0.5) ** 2)
    assert math.isclose(s["polish_s_to_min"], 0.6)
    assert math.isclose(s["polish_batch_s_to_min"], 0.9 + e)
    assert s["polish_hit_rate"] == 1.0 and s["polish_batch_hit_rate"] == 0.0
