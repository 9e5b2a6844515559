import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


_CACHE = {}


def small_workload(name: str, n_data: int, n_mc: int, from_model: bool = True):
    """A reduced-size workload of a named configuration, data drawn from the
    model with the oracle's intensity (cached per session)."""
    key = (name, n_data, n_mc, from_model)
    if key not in _CACHE:
        import oracle
        from paper_2403_09225_b300 import workload as W
        cfg = W.CONFIGS[name]
        table = W.make_table(cfg)
        model = oracle.Model.from_table(table, cfg.S)
        fn = None
        if from_model:
            fn = lambda m2, F: oracle.intensity_full(cfg.K, cfg.S, model.channels, model.par0, m2, F)
        wl = W.make_workload(cfg, intensity=fn, n_data=n_data, n_mc=n_mc)
        _CACHE[key] = (wl, model)
    return _CACHE[key]


@pytest.fixture(scope="session")
def tiny_small():
    return small_workload("tiny", 4000, 20000)


@pytest.fixture(scope="session")
def paper_small():
    return small_workload("paper", 1500, 6000)
