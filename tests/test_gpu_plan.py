"""Captured plans (CUDA graph of the whole path) and the launch-shape autotuner, through the C ABI.

A plan relaunched with (seed, walker-id offset) must give exactly the tallies, transmissions
and currents of the uncaptured calls (negf_build_tables + negf_walk + negf_current, or negf_run)
with the same seed and walker ids, whatever launch shapes the autotuner picked: launch shapes
change which thread runs which walker, never a walker's draws.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10164_gb300 import inputs, negf  # noqa: E402

MU = (3.5, -3.5, 0.025)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    c = negf.negf_create(0)
    yield c
    negf.negf_destroy(c)


def _wires():
    return [inputs.small_wire(91, W=3, L=7, n_energy=3, eta=0.1),
            inputs.small_wire(92, W=6, L=4, n_energy=2, eta=0.2),
            inputs.small_wire(93, W=1, L=15, n_energy=4, eta=0.05, e_lo=-1.9, e_hi=1.9),
            inputs.small_wire(94, W=20, L=3, n_energy=1, eta=0.3)]


def _reference(ctx, wires, seed, offset, N, start_lead=0, precision="fp32"):
    n_tasks = sum(len(w.energy) for w in wires)
    t = negf.negf_build_tables(ctx, wires, precision=precision)
    tl = negf.negf_walk(ctx, t, start_lead, seed, N, walker_id_offset=offset)
    try:
        counts = negf.negf_tally_counts(ctx, tl, n_tasks)
        cur = negf.negf_current(ctx, t, tl, *MU)
    finally:
        negf.negf_tally_free(tl)
        negf.negf_tables_free(t)
    return counts, cur


@pytest.mark.parametrize("autotune", [True, False])
def test_plan_equals_uncaptured_calls(ctx, autotune):
    wires = _wires()
    N = 20000
    plan = negf.negf_plan_create(ctx, wires, 0, N, *MU, precision="fp32", autotune=autotune)
    try:
        tune = negf.negf_plan_get_tuning(plan)
        assert tune["tuned"] == autotune
        if autotune:
            assert 2 <= tune["walk_blocks_per_sm"] <= 5
            assert tune["chain_warps"] >= 1 and tune["alias_warps"] >= 1
            assert tune["walk_ms"] > 0 and tune["chain_ms"] > 0 and tune["alias_ms"] > 0
        assert negf.negf_plan_num_waves(plan) == 1
        for seed, off in ((11, 0), (12, 5 * N), (11, 0)):
            negf.negf_plan_launch(ctx, plan, seed, off)
            got = negf.negf_plan_result(ctx, plan)
            ref_counts, ref_cur = _reference(ctx, wires, seed, off, N)
            assert np.array_equal(got["counts"], ref_counts), (seed, off)
            assert np.array_equal(got["T"], ref_cur["T"]) and np.array_equal(got["I"], ref_cur["I"])
            assert np.array_equal(got["se"], ref_cur["se"])
            assert not got["stepcap"]
    finally:
        negf.negf_plan_destroy(plan)


def test_plan_waves_and_device_inputs(ctx):
    """Several waves (two slots, walks overlapped on the second stream), device-resident
    inputs re-read by every launch: an in-place change of onsite shows up in the next launch."""
    wires = _wires()
    N = 15000
    dev = [inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite.copy()).cuda(),
                       eta=torch.from_numpy(w.eta.copy()).cuda(),
                       energy=torch.from_numpy(w.energy).cuda(),
                       energy_weight=torch.from_numpy(w.energy_weight).cuda()) for w in wires]
    plan = negf.negf_plan_create(ctx, dev, 1, N, *MU, precision="fp32", memspace="device",
                                 tasks_per_wave=2, autotune=True)
    try:
        assert negf.negf_plan_num_waves(plan) == 5
        negf.negf_plan_launch(ctx, plan, 77, 3)
        got = negf.negf_plan_result(ctx, plan)
        ref_counts, ref_cur = _reference(ctx, wires, 77, 3, N, start_lead=1)
        assert np.array_equal(got["counts"], ref_counts)
        assert np.array_equal(got["I"], ref_cur["I"])
        # change one wire's potential in place: the next launch must see it
        dev[1].onsite.add_(0.25)
        torch.cuda.synchronize()
        negf.negf_plan_launch(ctx, plan, 77, 3)
        got2 = negf.negf_plan_result(ctx, plan)
        w2 = [w for w in wires]
        w2[1] = inputs.Wire(W=wires[1].W, L=wires[1].L, t=wires[1].t,
                            onsite=wires[1].onsite + 0.25, eta=wires[1].eta,
                            energy=wires[1].energy, energy_weight=wires[1].energy_weight)
        ref2, _ = _reference(ctx, w2, 77, 3, N, start_lead=1)
        assert np.array_equal(got2["counts"], ref2)
        assert not np.array_equal(got2["counts"], got["counts"])
        # a bad value in a device input is reported by the launch that reads it
        dev[0].eta[0, 0] = -1.0
        torch.cuda.synchronize()
        negf.negf_plan_launch(ctx, plan, 77, 3)
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_plan_result(ctx, plan)
    finally:
        negf.negf_plan_destroy(plan)


def test_plan_profile_segments(ctx):
    """With profiling on, every launch adds the device time of its kernel groups (timed by
    event nodes inside the graph) to the context's profile."""
    wires = _wires()
    plan = negf.negf_plan_create(ctx, wires, 0, 50000, *MU, precision="fp32", autotune=False)
    try:
        negf.negf_profile_enable(ctx, True)
        for k in range(3):
            negf.negf_plan_launch(ctx, plan, 5, k * 50000)
        prof = negf.negf_profile_read(ctx)
        negf.negf_profile_enable(ctx, False)
        for name in ("rgf_sweep_kernel", "diag_chain_kernels", "alias_kernel", "walk_kernel",
                     "current_kernel"):
            assert name in prof, (name, prof)
            assert prof[name][0] >= 3 and prof[name][1] > 0.0, (name, prof[name])
    finally:
        negf.negf_plan_destroy(plan)


def test_plan_rejects_bad_options(ctx):
    wires = _wires()
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        negf.negf_plan_create(ctx, wires, 2, 100, *MU)
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        negf.negf_plan_create(ctx, wires, 0, 100, 0.0, 0.0, 0.0)
