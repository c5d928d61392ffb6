"""Host-side pieces of bench.py (no GPU): every named workload builds with the sizes it states,
the energy-subset option keeps weights and order, and the stored DRAM traffic figure is looked
up only for the walk sources it was measured on."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("name,W,L,n_e", [("wire_10x50", 10, 50, 64), ("chain_l20", 1, 20, 1),
                                          ("wire_16x100", 16, 100, 16),
                                          ("wire_32x100", 32, 100, 8),
                                          ("wire_64x100", 64, 100, 8)])
def test_named_workloads(name, W, L, n_e):
    wl = bench.workload(name)
    w = wl.wires[0]
    assert (w.W, w.L, w.energy.size) == (W, L, n_e)


def test_energy_subset_keeps_order_and_weights():
    full = bench.workload("wire_10x50").wires[0]
    sub = bench.workload("wire_10x50", energies=8)
    w = sub.wires[0]
    assert w.energy.size == 8 and np.all(np.diff(w.energy) > 0)
    assert w.energy[0] == full.energy[0] and w.energy[-1] == full.energy[-1]
    assert np.allclose(w.energy_weight, full.energy_weight[0])
    assert sub.name.endswith("_sub8E")


def test_unknown_workload_is_refused():
    with pytest.raises(SystemExit):
        bench.workload("no_such_workload")


def test_traffic_figure_is_keyed_to_the_sources():
    assert bench.measured_traffic("walk_kernel", "no_such_workload") is None
    assert bench.measured_traffic("alias_kernel", "wire_W10_L50_eta0.05_64E") is None
