"""Parity of the benchmark's own workload and of every compiled slice width, through the C ABI.

The kernels for slices of W <= 16 sites (register RGF sweeps, register diagonal blocks, block
columns with one column per lane) are compiled once per width, so each width is separate code:
every width 10..16 is compared here elementwise with the oracle, in FP32 and FP64 (widths 1..9
are in test_gpu_parity.py).  The benchmark's wire (W = 10 x L = 50, 64 energies, 1e6 walkers
per energy, FP32 tables) runs through an autotuned, captured plan exactly as bench.py runs it,
and its tables, transmissions and current are compared with the oracle.

Bars:
  * tables: FP64 |w - w_ref| <= 1e-10 |w_ref| + 1e-13 rowsum_ref; FP32 |w - w_ref| <= 1e-5
    rowsum_ref (per element); c_p, row sums and mode weights relative 1e-10 (FP64) / 1e-5 (FP32).
  * Monte Carlo transmissions against the direct probe solve (Eq. buteq): every |z| <= z_bar(m)
    and sum z^2 <= chi2_bar(m) for the m tasks with an open channel (mc_bars: the 3-SE bar as a
    0.27 % family-wise false-alarm rate).
  * the current (Eq. iqof_t_el_db on the grid): within 3 SE(I) of the current of the direct
    solve's transmissions; equal to the oracle's formula on the same tallies to 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import chi2_bar, z_bar  # noqa: E402
from oracle import current as ocur, pipeline  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402

BENCH_SEED = 20240607          # bench.py's default seed


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    c = negf.negf_create(0)
    yield c
    negf.negf_destroy(c)


def _check_tables(ctx, tables, refs, precision, task0=0):
    rt = 1e-10 if precision == "fp64" else 1e-5
    for k, ref in enumerate(refs):
        task = task0 + k
        tab = ref["tab"]
        w_ref = tab["w"]
        rs_ref = w_ref.sum(1)
        w = negf.negf_export_tables(ctx, tables, task, "weights").reshape(w_ref.shape)
        if precision == "fp64":
            tol = 1e-10 * np.abs(w_ref) + 1e-13 * rs_ref[:, None] + 1e-300
        else:
            tol = 1e-5 * rs_ref[:, None] + 1e-30
        bad = np.abs(w - w_ref) > tol
        assert not bad.any(), (task, np.argwhere(bad)[:5])
        rs = negf.negf_export_tables(ctx, tables, task, "rowsum")
        assert np.allclose(rs, rs_ref, rtol=rt, atol=1e-300), task
        mw = negf.negf_export_tables(ctx, tables, task, "mode_weights").reshape(2, -1)
        assert np.allclose(mw, tab["mode_w"], rtol=rt, atol=rt * tab["c"].max() + 1e-300), task
        info = negf.negf_get_task_info(ctx, tables, task)
        assert np.allclose(info["c"], tab["c"], rtol=rt, atol=1e-300), task


def _register_width_wires():
    # every width compiled separately, each long enough for several slices of every kind
    return [inputs.small_wire(300 + W, W=W, L=20 + (W % 3), n_energy=2, eta=0.06 + 0.01 * (W % 4),
                              e_lo=-3.3, e_hi=3.1)
            for W in range(10, 17)]


@pytest.fixture(scope="module")
def width_refs():
    wires = _register_width_wires()
    refs = [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)
            for w in wires for E in w.energy]
    return wires, refs


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tables_of_every_register_width(ctx, width_refs, precision):
    wires, refs = width_refs
    tables = negf.negf_build_tables(ctx, wires, precision=precision, keep_weights=True)
    try:
        assert negf.negf_tables_num_tasks(tables) == len(refs)
        _check_tables(ctx, tables, refs, precision)
    finally:
        negf.negf_tables_free(tables)
    # each width alone (its instantiation is the only one the launch takes)
    for wi, w in enumerate(wires[::3]):
        tables = negf.negf_build_tables(ctx, [w], precision=precision, keep_weights=True)
        try:
            k0 = 2 * (3 * wi)
            _check_tables(ctx, tables, refs[k0:k0 + 2], precision)
        finally:
            negf.negf_tables_free(tables)


def test_transmission_of_every_register_width(ctx, width_refs):
    wires, refs = width_refs
    tables = negf.negf_build_tables(ctx, wires, precision="fp32")
    try:
        N = 400_000
        z = []
        for lead0 in (0, 1):
            tally = negf.negf_walk(ctx, tables, lead0, 7100 + lead0, N)
            res = negf.negf_current(ctx, tables, tally, 3.5, -3.5, 0.025)
            negf.negf_tally_free(tally)
            assert not res["stepcap"]
            for task, ref in enumerate(refs):
                if ref["tab"]["c"][lead0] > 0:
                    z.append((res["T"][task] - ref["T_direct"][1 - lead0, lead0])
                             / res["T_se"][task])
        z = np.asarray(z)
        assert np.max(np.abs(z)) <= z_bar(z.size), z
        assert np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tables_free(tables)


@pytest.fixture(scope="module")
def bench_case():
    wl = inputs.wire_10x50()
    w = wl.wires[0]
    refs = [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False) for E in w.energy]
    return wl, refs


def test_benchmark_tables_match_oracle(ctx, bench_case):
    wl, refs = bench_case
    tables = negf.negf_build_tables(ctx, wl.wires, precision=wl.precision, keep_weights=True)
    try:
        assert negf.negf_tables_num_tasks(tables) == 64
        _check_tables(ctx, tables, refs, wl.precision)
    finally:
        negf.negf_tables_free(tables)


def test_benchmark_plan_against_direct_solve(ctx, bench_case):
    """The benchmark's step as bench.py runs it: device-resident inputs, autotuned plan, one
    launch with the benchmark's seed and the first walker range."""
    wl, refs = bench_case
    w = wl.wires[0]
    dev = inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                      eta=torch.from_numpy(w.eta).cuda(), energy=torch.from_numpy(w.energy).cuda(),
                      energy_weight=torch.from_numpy(w.energy_weight).cuda())
    N = wl.walkers_per_task
    plan = negf.negf_plan_create(ctx, [dev], 0, N, wl.mu_p, wl.mu_q, wl.kT,
                                 precision=wl.precision, memspace="device", autotune=True)
    try:
        negf.negf_plan_launch(ctx, plan, BENCH_SEED, 0)
        r = negf.negf_plan_result(ctx, plan)
    finally:
        negf.negf_plan_destroy(plan)
    assert not r["stepcap"]
    counts = r["counts"]
    assert np.all(counts[:, 0] == N)
    T_dir = np.array([ref["T_direct"][1, 0] for ref in refs])
    c = np.array([ref["tab"]["c"][0] for ref in refs])
    open_ = c > 0
    assert np.all(counts[open_, 1] + counts[open_, 2] == N)
    assert np.all(counts[~open_, 1] + counts[~open_, 2] == 0)
    z = (r["T"][open_] - T_dir[open_]) / r["T_se"][open_]
    assert np.max(np.abs(z)) <= z_bar(z.size), (np.argmax(np.abs(z)), z)
    assert np.sum(z ** 2) <= chi2_bar(z.size), np.sum(z ** 2)
    # current of the direct solve on the same grid (Eq. iqof_t_el_db), one comparison at 3 SE
    I_dir, _ = ocur.current(w.energy, w.energy_weight, T_dir, np.zeros_like(T_dir), wl.mu_p,
                            wl.mu_q, wl.kT)
    assert abs(r["I"][0] - I_dir) <= 3.0 * r["se"][0], (r["I"][0], I_dir, r["se"][0])
    # the current assembly equals the oracle's formula on the same tallies (the device's c_p)
    T_o, se_o = ocur.mc_transmission(r["T"] / np.where(counts[:, 2] > 0,
                                                       counts[:, 2] / counts[:, 0], 1.0),
                                     counts[:, 2], counts[:, 0])
    I_o, dI_o = ocur.current(w.energy, w.energy_weight, T_o, se_o, wl.mu_p, wl.mu_q, wl.kT)
    assert abs(r["I"][0] - I_o) <= 1e-12 * abs(I_o)
    assert abs(r["se"][0] - dI_o) <= 1e-12 * abs(dI_o)
