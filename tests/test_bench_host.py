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


def test_fp32_peak_from_unit_counts():
    pk, src = bench.fp32_peak()
    # 152 SMs x 128 lanes x 2 flop at 2070 MHz = 80.5 TFLOP/s
    assert 60.0 < pk < 90.0 and "152 SMs" in src


def test_cta_chain_flops_count_the_symmetric_chain():
    wl = bench.workload("wire_64x1000", energies=2)
    L, W = 1000, 64
    assert bench.cta_chain_flops(wl, "fp32") == 2 * 8 * W**3 * (L * (L - 1) // 2 + 2 * (L - 1))
    assert bench.cta_chain_flops(wl, "fp64") == 0
    narrow = bench.workload("wire_32x100")
    assert bench.cta_chain_flops(narrow, "fp32") == 8 * 8 * 32**3 * (102 * 99)


def test_local_workload_partitions_energies():
    wl = bench.workload("wire_64x1000")
    parts = [bench.local_workload(wl, r, 3) for r in range(3)]
    E = np.sort(np.concatenate([p.wires[0].energy for p in parts]))
    assert np.array_equal(E, wl.wires[0].energy)
    assert bench.local_workload(wl, 0, 1) is wl


def test_rooflines_of_a_step():
    wl = bench.workload("wire_64x1000", energies=8)
    counts = np.zeros((8, 5), dtype=np.uint64)
    counts[:, 0] = 32_000_000
    counts[:, 4] = 100_000_000
    counts[:, 2] = 32_000_000
    prof = {"chain_cta_kernel": (8, 245.0), "two_level_kernel": (8, 82.0), "walk_kernel": (1, 35.0),
            "rgf_sweep_kernel": (1, 64.0)}
    r = bench.rooflines(prof, wl, "fp32", counts, 1)
    assert r["chain_cta_kernel"]["bound"] == "alu" and 0.3 < r["chain_cta_kernel"]["frac"] < 0.6
    assert r["two_level_kernel"]["bound"] == "hbm" and 0.2 < r["two_level_kernel"]["frac"] < 1.0
    assert r["walk_kernel"]["bound"] == "hbm"
    assert "rgf_sweep_kernel" not in r


def test_traffic_is_reported_per_launch():
    """The measured DRAM traffic of the headline chain (keyed to the current sources) over the
    launches of a step: the figure of the average launch, as achieved is its rate."""
    wl = bench.workload("wire_64x1000")
    tps = bench.measured_traffic("chain_cta_kernel", wl.name)
    assert tps is not None and tps > 0
    prof = {"chain_cta_kernel": (2 * 86, 2 * 7706.0)}
    counts = np.zeros((256, 5), dtype=np.uint64)
    r = bench.rooflines(prof, wl, "fp32", counts, 2)["chain_cta_kernel"]
    assert r["traffic_per_step"] == tps
    assert r["traffic"] == int(tps / 86)
