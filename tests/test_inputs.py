"""The seeded input recipe: every workload is reproducible from its seed and has the sizes and
distributions it states (the configurations the benchmark and the parity tests run)."""
import numpy as np

from paper_1805_10164_gb300 import inputs


def test_workloads_are_seeded_and_shaped():
    cases = [
        (inputs.chain_l20, 1, 20, 0.5, 0.1, 1, "fp64"),
        (inputs.wire_10x50, 10, 50, 1.0, 0.05, 64, "fp32"),
        (inputs.wire_16x100, 16, 100, 1.0, 0.05, 16, "fp64"),
        (inputs.wire_32x100, 32, 100, 1.0, 0.05, 8, "fp32"),
        (inputs.wire_64x100, 64, 100, 0.5, 0.005, 8, "fp32"),
    ]
    for make, W, L, dis, eta, ne, prec in cases:
        a, b = make(), make()
        w = a.wires[0]
        assert (w.W, w.L) == (W, L) and w.onsite.shape == (L, W) and w.eta.shape == (L, W)
        assert np.array_equal(w.onsite, b.wires[0].onsite)           # seeded
        assert np.all(np.abs(w.onsite) <= dis) and np.all(w.eta == eta)
        assert w.energy.size == ne and a.precision == prec
        assert np.all(np.diff(w.energy) > 0) and np.all(w.energy_weight > 0)


def test_midpoint_grid_covers_the_window():
    E, wE = inputs.midpoint_grid(-3.5, 3.5, 64)
    assert abs(wE.sum() - 7.0) < 1e-12
    assert abs(E[0] - (-3.5 + 7.0 / 128)) < 1e-12 and abs(E[-1] - (3.5 - 7.0 / 128)) < 1e-12


def test_batched_uneven_recipe():
    wl = inputs.batched_uneven()
    assert len(wl.wires) == 256
    W = np.array([w.W for w in wl.wires])
    L = np.array([w.L for w in wl.wires])
    eta = np.array([w.eta[0, 0] for w in wl.wires])
    assert W.min() >= 4 and W.max() <= 32 and L.min() >= 20 and L.max() <= 200
    assert np.all((eta >= 0.01) & (eta <= 0.2))
    # log-uniform: log(eta) roughly uniform over [log 0.01, log 0.2]
    u = (np.log(eta) - np.log(0.01)) / (np.log(0.2) - np.log(0.01))
    assert abs(u.mean() - 0.5) < 0.06 and 0.2 < np.median(u) < 0.8
    # widths and lengths spread over their ranges
    assert len(set(W.tolist())) > 20 and np.std(L) > 35
    assert all(w.energy.size == 32 for w in wl.wires)
    again = inputs.batched_uneven()
    assert all(np.array_equal(x.onsite, y.onsite) for x, y in zip(wl.wires, again.wires))
