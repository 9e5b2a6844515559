"""Parity at the full paper-scale size (1e6 data + 5e6 MC events, K = 20,
S = 4) in the launch configuration the benchmark times, against the oracle
evaluated over event shards in spawned worker processes (paper Eqs. 4-5:
shard sums add up).  Data events are phase-space events here (accept-reject
from I at this size is left to the benchmark); the likelihood is defined for
any event sample."""
import os

import numpy as np
import pytest

import oracle
from paper_2403_09225_b300 import workload as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_full_paper_scale_against_sharded_oracle():
    from paper_2403_09225_b300 import binding
    cfg = W.CONFIGS["paper"]
    wl = W.make_workload(cfg, intensity=None)
    model = oracle.Model.from_table(wl.table, cfg.S)
    L = binding.make_likelihood(wl)
    th = W.random_starts(wl, 1)[0]
    v = np.linspace(-1.0, 1.0, model.P)
    f, g, hv = L.eval(th, v)
    fo, go, hvo = oracle.sharded_nll_grad_hvp(model, th, v, wl.data, wl.mc,
                                              workers=max(2, min(32, os.cpu_count() or 2)), shard=100_000)
    assert abs(f - fo) <= 1e-6 * abs(fo), (f, fo)
    assert np.max(np.abs(g - go)) <= 1e-5 * np.max(np.abs(go))
    assert np.max(np.abs(hv - hvo)) <= 1e-4 * np.max(np.abs(hvo))
