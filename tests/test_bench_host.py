"""Host logic of bench.py (no GPU): the roofline's committed DRAM-traffic
figure is used only for the kernel revision and tiling it was captured on,
fits are scored against the best NLL with the 0.01 criterion, and the
oracle legs time what they say on bounded samples."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_figure_matches_revision_and_tiling():
    t = bench.measured_traffic({"warps": 4, "stages": 2})
    assert t is not None and 3.9e9 < t < 4.0e9  # 32.6 B per event-amplitude, 1.2e8 of them
    assert bench.measured_traffic({"warps": 8, "stages": 2}) is None
    assert bench.measured_traffic({"warps": 4, "stages": 3}) is None


def test_traffic_figure_refused_for_another_revision(monkeypatch):
    monkeypatch.setattr(bench, "KERNEL_REVISION", "some other revision")
    assert bench.measured_traffic({"warps": 4, "stages": 2}) is None


def test_fit_scoring_uses_the_best_nll_and_0_01():
    arms = {"a": {"nll": [-10.0, -9.995, -9.9], "gpu_seconds": 2.0},
            "b": {"nll": [-9.0], "gpu_seconds": 1.0}}
    bench._score(arms, -10.0)
    assert arms["a"]["reached_global_min"] == 2
    assert arms["b"]["reached_global_min"] == 0
    assert arms["a"]["fits_to_global_min_per_s"] == 1.0


def test_oracle_eval_rate_on_a_tiny_sample():
    r = bench._oracle_eval_rate("tiny", 0.01)
    assert r["events"] == 200 + 1000 and r["K"] == 3 and r["eval_s"] > 0
    assert np.isclose(r["event_amps_per_s"], r["events"] * r["K"] / r["eval_s"])
