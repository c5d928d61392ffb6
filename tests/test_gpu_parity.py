"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Bars (stated once, used below):
  * FP64 tables: |w - w_ref| <= 1e-10 |w_ref| + 1e-13 * rowsum_ref, per element.
  * FP32 tables: |w - w_ref| <= 1e-5 rowsum_ref per element (FP32 propagation, FP64 inversions).
  * c_p and row sums: relative 1e-10 (FP64) / 1e-5 (FP32).
  * alias rows: the exact integer-implied distribution equals the row's own weights / rowsum
    within (K + 2) 2^-32 + 4 eps_row (quantisation of thresholds and slots).
  * walks: bit-exact (lead and steps per walker) against the oracle walker replaying the
    exported integer tables with the same Philox counters.
  * Monte Carlo transmission against the direct probe solve, and mean walk length against the
    fundamental matrix of the chain: every |z| <= z_bar(m) and sum z^2 <= chi2_bar(m) over the
    m comparisons of a test (mc_bars: the 3-SE bar as a 0.27 % family-wise false-alarm rate).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import chi2_bar, z_bar  # noqa: E402
from oracle import alias, current as ocur, pipeline, walker  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402


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
    ws = [
        inputs.chain_l20().wires[0],                                     # W=1, L=20, E=0.5
        inputs.small_wire(11, W=3, L=9, n_energy=4, eta=0.1),
        inputs.small_wire(12, W=5, L=13, n_energy=3, eta=0.07, e_lo=-3.8, e_hi=3.8),
        inputs.small_wire(13, W=7, L=4, n_energy=2, eta=0.3),
        inputs.small_wire(14, W=2, L=1, n_energy=2, eta=0.2),           # single slice
        inputs.small_wire(15, W=1, L=6, n_energy=3, eta=0.1, e_lo=-3.3, e_hi=3.3),  # closed E
        inputs.small_wire(16, W=4, L=5, n_energy=2, eta=0.15, lead_model=1, gamma_lead=0.8),
        inputs.small_wire(17, W=33, L=3, n_energy=1, eta=0.05),         # > 32 rows per slice
    ]
    return ws


def _refs(wires):
    out = []
    for w in wires:
        for E in w.energy:
            out.append(pipeline.task_reference(w.onsite, w.eta, w.t, E, w.lead_model,
                                               w.gamma_lead, with_alias=False))
    return out


@pytest.fixture(scope="module")
def batch(ctx):
    wires = _wires()
    return wires, _refs(wires)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tables_match_oracle(ctx, batch, precision):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision=precision, keep_weights=True)
    try:
        assert negf.negf_tables_num_tasks(tables) == len(refs)
        rt = 1e-10 if precision == "fp64" else 1e-5
        for task, ref in enumerate(refs):
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
            assert np.allclose(rs, rs_ref, rtol=rt, atol=1e-300)
            mw = negf.negf_export_tables(ctx, tables, task, "mode_weights").reshape(2, -1)
            assert np.allclose(mw, tab["mode_w"], rtol=rt, atol=rt * tab["c"].max() + 1e-300)
            info = negf.negf_get_task_info(ctx, tables, task)
            assert np.allclose(info["c"], tab["c"], rtol=rt, atol=1e-300)
    finally:
        negf.negf_tables_free(tables)


def test_alias_rows_realise_their_weights(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32", keep_weights=True)
    try:
        rng = np.random.default_rng(0)
        for task, ref in enumerate(refs):
            shape = ref["tab"]["w"].shape
            w = negf.negf_export_tables(ctx, tables, task, "weights").reshape(shape)
            rs = negf.negf_export_tables(ctx, tables, task, "rowsum")
            ent = negf.negf_export_tables(ctx, tables, task, "alias").reshape(shape)
            K = shape[1]
            rows = rng.choice(shape[0], size=min(12, shape[0]), replace=False)
            for r in rows:
                if rs[r] <= 0:
                    continue
                p = alias.implied_distribution(ent[r])
                err = np.max(np.abs(p - w[r] / rs[r]))
                assert err <= (K + 2) / 2**32 + 1e-12, (task, r, err)
            mw = negf.negf_export_tables(ctx, tables, task, "mode_weights").reshape(2, -1)
            me = negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, -1)
            for p_ in range(2):
                if mw[p_].sum() > 0:
                    p = alias.implied_distribution(me[p_])
                    assert np.max(np.abs(p - mw[p_] / mw[p_].sum())) <= (mw.shape[1] + 2) / 2**32 + 1e-13
    finally:
        negf.negf_tables_free(tables)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_walks_bit_exact_against_oracle_walker(ctx, batch, precision):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision=precision)
    try:
        n_w = 3000
        for task in range(len(refs)):
            info = negf.negf_get_task_info(ctx, tables, task)
            ent = negf.negf_export_tables(ctx, tables, task, "alias").reshape(info["rows"], info["K"])
            ment = negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, info["W"])
            for lead0, cap, off in ((0, 1 << 20, 0), (1, 1 << 20, 2**33 + 5), (0, 2, 77)):
                d_lead = torch.empty(n_w, dtype=torch.int32, device="cuda")
                d_steps = torch.empty(n_w, dtype=torch.int32, device="cuda")
                negf.negf_walk_trace(ctx, tables, task, lead0, 0xC0FFEE + task, off, d_lead,
                                     d_steps, max_steps=cap)
                lead, steps = walker.walk(ent, ment, info["n"], info["W"], info["c"] > 0, task,
                                          lead0, 0xC0FFEE + task, off + np.arange(n_w), cap)
                assert np.array_equal(d_lead.cpu().numpy(), lead), (task, lead0, cap)
                assert np.array_equal(d_steps.cpu().numpy().astype(np.uint32), steps)
    finally:
        negf.negf_tables_free(tables)


def test_monte_carlo_transmission_and_current(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp64")
    try:
        N = 400_000
        z_T, z_steps = [], []
        for lead0 in (0, 1):
            tally = negf.negf_walk(ctx, tables, lead0, 2024 + lead0, N)
            counts = negf.negf_tally_counts(ctx, tally, len(refs))
            res = negf.negf_current(ctx, tables, tally, 3.5, -3.5, 0.025)
            negf.negf_tally_free(tally)
            assert not res["stepcap"]
            q = 1 - lead0
            c_all = []
            for task, ref in enumerate(refs):
                c = ref["tab"]["c"][lead0]
                c_all.append(negf.negf_get_task_info(ctx, tables, task)["c"][lead0])
                assert counts[task, 0] == N
                if c > 0:
                    assert counts[task, 1] + counts[task, 2] == N
                else:
                    assert counts[task, 1] + counts[task, 2] == 0
                    assert res["T"][task] == 0.0
                    continue
                T_ref = ref["T_direct"][q, lead0]
                z_T.append((res["T"][task] - T_ref) / res["T_se"][task])
                # mean steps against the fundamental matrix of the chain
                ms = counts[task, 4] / N
                m_ref = ref["exact"]["steps_inj"][lead0]
                var = ref["exact"]["steps2_inj"][lead0] - m_ref**2
                z_steps.append((ms - m_ref) / np.sqrt(var / N))
            # current assembly: same formula in the oracle on the same tallies
            k = 0
            for wi, w in enumerate(wires):
                nE = len(w.energy)
                sl = slice(k, k + nE)
                T_o, se_o = ocur.mc_transmission(np.array(c_all[sl]), counts[sl, 1 + q],
                                                 counts[sl, 0])
                I_o, dI_o = ocur.current(w.energy, w.energy_weight, T_o, se_o, 3.5, -3.5, 0.025)
                assert np.allclose(res["T"][sl], T_o, rtol=1e-12, atol=1e-15)
                assert abs(res["I"][wi] - I_o) <= 1e-12 * abs(I_o) + 1e-15
                assert abs(res["se"][wi] - dI_o) <= 1e-12 * abs(dI_o) + 1e-15
                k += nE
        for z in (np.asarray(z_T), np.asarray(z_steps)):
            assert np.max(np.abs(z)) <= z_bar(z.size), z
            assert np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tables_free(tables)


def test_batching_and_device_inputs_do_not_change_tables(ctx):
    """A task's tables do not depend on what else is in the batch, nor on where the inputs
    live (bit-identical alias entries)."""
    wires = [inputs.small_wire(21, W=4, L=6, n_energy=2), inputs.small_wire(22, W=9, L=5, n_energy=3)]
    big = negf.negf_build_tables(ctx, wires, precision="fp32")
    dev_wires = []
    for w in wires:
        dw = inputs.Wire(W=w.W, L=w.L, t=w.t,
                         onsite=torch.from_numpy(w.onsite).cuda(), eta=torch.from_numpy(w.eta).cuda(),
                         energy=torch.from_numpy(w.energy).cuda(),
                         energy_weight=torch.from_numpy(w.energy_weight).cuda())
        dev_wires.append(dw)
    dev = negf.negf_build_tables(ctx, dev_wires, precision="fp32", memspace="device")
    single = negf.negf_build_tables(ctx, wires[1:], precision="fp32")
    try:
        for task in range(5):
            a = negf.negf_export_tables(ctx, big, task, "alias")
            b = negf.negf_export_tables(ctx, dev, task, "alias")
            assert np.array_equal(a, b)
        for task in range(3):
            a = negf.negf_export_tables(ctx, big, task + 2, "alias")
            b = negf.negf_export_tables(ctx, single, task, "alias")
            assert np.array_equal(a, b)
    finally:
        for t in (big, dev, single):
            negf.negf_tables_free(t)


def test_invalid_inputs_are_rejected(ctx):
    w = inputs.small_wire(31, W=3, L=4, n_energy=1)
    bad = inputs.Wire(**{**w.__dict__, "eta": -w.eta})
    with pytest.raises(negf.NegfError, match="INVALID"):
        negf.negf_build_tables(ctx, [bad])
    edge = inputs.Wire(**{**w.__dict__, "W": 1, "L": 4, "onsite": np.zeros((4, 1)),
                          "eta": np.full((4, 1), 0.1), "energy": np.array([2.0]),
                          "energy_weight": np.array([1.0])})
    with pytest.raises(negf.NegfError, match="band edge"):
        negf.negf_build_tables(ctx, [edge])
    tables = negf.negf_build_tables(ctx, [w])
    try:
        with pytest.raises(negf.NegfError, match="max_steps"):
            negf.negf_walk(ctx, tables, 0, 1, 10, max_steps=0)
        with pytest.raises(negf.NegfError, match="start_lead"):
            negf.negf_walk(ctx, tables, 2, 1, 10)
    finally:
        negf.negf_tables_free(tables)
    # device-resident inputs are checked on the device and reported at the next sync
    dw = inputs.Wire(W=3, L=4, t=1.0, onsite=torch.full((4, 3), float("nan"), device="cuda",
                                                        dtype=torch.float64),
                     eta=torch.full((4, 3), 0.1, device="cuda", dtype=torch.float64),
                     energy=torch.tensor([0.3], device="cuda", dtype=torch.float64),
                     energy_weight=None)
    t2 = negf.negf_build_tables(ctx, [dw], memspace="device")
    try:
        with pytest.raises(negf.NegfError, match="INVALID"):
            negf.negf_get_task_info(ctx, t2, 0)
    finally:
        negf.negf_tables_free(t2)


def test_step_cap_reported(ctx):
    w = inputs.small_wire(41, W=2, L=30, n_energy=1, eta=0.8)
    tables = negf.negf_build_tables(ctx, [w])
    try:
        tally = negf.negf_walk(ctx, tables, 0, 5, 20000, max_steps=1)
        counts = negf.negf_tally_counts(ctx, tally, 1)
        res = negf.negf_current(ctx, tables, tally, 0.5, -0.5, 0.025)
        negf.negf_tally_free(tally)
        assert counts[0, 3] > 0 and res["stepcap"]
        assert counts[0, 1] + counts[0, 2] + counts[0, 3] == 20000
    finally:
        negf.negf_tables_free(tables)


def test_tally_accumulate_resumes_exactly(ctx):
    """Walks over disjoint walker-id ranges add up to one run over the union."""
    w = inputs.small_wire(51, W=3, L=7, n_energy=2)
    tables = negf.negf_build_tables(ctx, [w])
    try:
        a = negf.negf_walk(ctx, tables, 0, 9, 5000, walker_id_offset=0)
        b = negf.negf_walk(ctx, tables, 0, 9, 5000, walker_id_offset=5000)
        ab = negf.negf_walk(ctx, tables, 0, 9, 10000, walker_id_offset=0)
        cb = negf.negf_tally_counts(ctx, b, 2)
        negf.negf_tally_accumulate(ctx, a, cb)
        assert np.array_equal(negf.negf_tally_counts(ctx, a, 2), negf.negf_tally_counts(ctx, ab, 2))
        for t in (a, b, ab):
            negf.negf_tally_free(t)
    finally:
        negf.negf_tables_free(tables)


def test_run_pipeline_matches_build_and_walk(ctx):
    """negf_run (waves built on one stream while the previous wave walks on another, tables
    freed per wave) gives bit-identical tallies to negf_build_tables + negf_walk, for uneven
    wires and several wave sizes, and its task handle serves negf_current."""
    wires = [inputs.small_wire(71, W=3, L=7, n_energy=3, eta=0.1),
             inputs.small_wire(72, W=6, L=4, n_energy=2, eta=0.2),
             inputs.small_wire(73, W=1, L=15, n_energy=4, eta=0.05, e_lo=-1.9, e_hi=1.9),
             inputs.small_wire(74, W=9, L=3, n_energy=1, eta=0.3)]
    n_tasks = sum(len(w.energy) for w in wires)
    N = 30000
    ref_t = negf.negf_build_tables(ctx, wires, precision="fp32")
    ref_tl = negf.negf_walk(ctx, ref_t, 1, 4242, N, walker_id_offset=17)
    ref = negf.negf_tally_counts(ctx, ref_tl, n_tasks)
    ref_cur = negf.negf_current(ctx, ref_t, ref_tl, 3.5, -3.5, 0.025)
    try:
        for per_wave, budget in ((0, 0), (1, 0), (3, 0), (0, 1)):
            t, tl = negf.negf_run(ctx, wires, 1, 4242, N, precision="fp32", walker_id_offset=17,
                                  tasks_per_wave=per_wave, memory_budget=budget)
            try:
                got = negf.negf_tally_counts(ctx, tl, n_tasks)
                assert np.array_equal(got, ref), (per_wave, budget)
                cur = negf.negf_current(ctx, t, tl, 3.5, -3.5, 0.025)
                assert np.array_equal(cur["T"], ref_cur["T"]) and np.array_equal(cur["I"], ref_cur["I"])
                if budget == 1:
                    assert negf.negf_tables_num_waves(t) == n_tasks     # one task per wave
                with pytest.raises(negf.NegfError, match="released"):
                    negf.negf_export_tables(ctx, t, 0, "alias")
            finally:
                negf.negf_tally_free(tl)
                negf.negf_tables_free(t)
    finally:
        negf.negf_tally_free(ref_tl)
        negf.negf_tables_free(ref_t)
