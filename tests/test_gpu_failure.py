"""Failure detection without a GPU fault: a device-side wait that nothing
completes runs out after its limit and the library reports PWA_ETIMEOUT,
leaving the context usable."""
import numpy as np
import pytest

from paper_2403_09225_b300 import workload as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_2403_09225_b300 import binding
    assert binding.lib().pwa_selftest_bounded_wait(0.05) == binding.PWA_ETIMEOUT
    assert binding.lib().pwa_selftest_bounded_wait(-1.0) == binding.PWA_EINVAL
    cfg = W.CONFIGS["tiny"]
    wl = W.make_workload(cfg, intensity=None, n_data=1000, n_mc=5000)
    L = binding.make_likelihood(wl)
    assert np.isfinite(L.nll(wl.theta_true))
