"""The learned starting-point proposal end to end on the GPU, at the tiny
model (K = 3, S = 2, 10 real parameters): pseudo-experiments generated and
labelled by the library, the network trained by its own kernels, and its
gain over random multi-start on held-out pseudo-experiments measured.

What is compared (proposal.evaluate): on each held-out experiment one fit
from the network's start and one batched call of 8 fits from prior starts,
all with the same fit options; the experiment's global minimum is the lowest
NLL of those 9 fits, and a fit reaches it within 0.01.  The test requires
the network's start to reach the minimum more often than a random start, and
the expected GPU-seconds to the minimum (network start, with random
multi-start as the fallback when it misses) to be lower than random
multi-start's own, alone and in the batched form (the network's start and
three draws around it fitted in one lockstep call).  The batched form is at
least as likely to reach the minimum as the single start whose draws it
adds (its first row is that start; the lockstep path may end one such fit
elsewhere, so one experiment of slack)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_canonical_labels_are_fixed_points_and_preserve_the_likelihood():
    """Sorting an exchangeable group and flipping a magnitude's sign leave the
    NLL unchanged (library evaluation), and canonical() is idempotent."""
    from paper_2403_09225_b300 import binding, proposal, workload as W
    import oracle
    cfg = W.CONFIGS["paper"]
    table = W.make_table(cfg)
    groups = proposal.exchangeable_groups(table)
    assert groups, "the K = 20 table has exchangeable resonances"
    model = oracle.Model.from_table(table, cfg.S)
    wl = W.make_workload(cfg, n_data=3000, n_mc=12000,
                         intensity=lambda m2, F: oracle.intensity_full(cfg.K, cfg.S, model.channels, model.par0,
                                                                      m2, F))
    L = binding.make_likelihood(wl)
    rng = np.random.default_rng(0)
    th = W.sample_start(rng, table)
    lay = proposal.Layout.of(table)
    th[lay.rho[groups[0][0]]] *= -1  # a negative magnitude
    c = proposal.canonical(table, th)
    assert np.allclose(proposal.canonical(table, c), c)
    assert abs(L.nll(c) - L.nll(th)) <= 1e-6 * abs(L.nll(th))
    for g in groups:
        m = c[lay.mass[g]]
        assert np.all(np.diff(m) >= 0)
    L.close()


def test_learned_proposal_beats_random_starts():
    from paper_2403_09225_b300 import proposal, workload as W
    cfg = W.CONFIGS["tiny"]
    table = W.make_table(cfg)
    gen = proposal.Generator(table, cfg.S, pool_size=1_000_000, n_mc=50_000, seed=7)
    ex = proposal.make_experiments(gen, 1536, 10_000, seed=100)
    assert ex.n_events.min() > 1000
    net, codec, hist = proposal.train(ex, table, epochs=60, batch=128, lr=1e-3)
    assert hist[-1] < 0.2 * hist[0], hist
    recs, s = proposal.evaluate(gen, net, codec, 24, 10_000, 8, seed=999)
    print(s)
    assert s["mlp_hit_rate"] > s["random_hit_rate"] + 0.1, s
    assert s["learned_s_to_min"] < s["random_s_to_min"], s
    # the batched form (the network's start and three draws around it in one call)
    assert s["learned_batch_hit_rate"] >= s["mlp_hit_rate"] - 1.0 / 24, s
    assert s["learned_batch_s_to_min"] < s["random_s_to_min"], s
    net.close()
    gen.close()
