"""Host logic of the physics variants (no GPU): the library's theta layout
(binding.Variant.initial_theta, the order pwa_variant_create uses) against
the oracle's layout for both coupling modes and mixed line shapes."""
import numpy as np
import pytest

from oracle import variants as V
from paper_2403_09225_b300 import binding, workload as W


def _shapes(table):
    out = []
    for k, r in enumerate(table):
        a, b, _ = W.CHANNEL_PAIRS[r.channel]
        ma, mb = W.DAUGHTER_MASSES[a], W.DAUGHTER_MASSES[b]
        if k % 4 == 2:
            out.append(V.Shape(V.KIND_FLATTE, ma=ma, mb=mb, mc=0.4937, md=0.4937, width2=0.1 + 0.01 * k))
        elif k % 4 == 1:
            out.append(V.Shape(V.KIND_MASS_DEPENDENT, ma=ma, mb=mb, radius=3.0))
        else:
            out.append(V.Shape(V.KIND_CONSTANT))
    return out


@pytest.mark.parametrize("name", ["tiny", "tiny_k4", "paper"])
@pytest.mark.parametrize("per_projection", [False, True])
def test_initial_theta_follows_the_oracle_layout(name, per_projection):
    cfg = W.CONFIGS[name]
    table = W.make_table(cfg)
    table[-1].fix_width = True  # a fixed width (and, for a Flatte shape, its gamma2) leaves theta
    shapes = _shapes(table)
    vm = V.VariantModel.from_table(table, cfg.S, shapes, per_projection)
    th = binding.Variant.initial_theta(table, shapes, cfg.S, per_projection)
    assert th.shape == (vm.P,)
    assert np.array_equal(th, vm.theta0())
    assert V.coupling_count(vm) == 2 * sum(not r.fix_coupling for r in table) * (cfg.S if per_projection else 1)
