"""Tensor-core block columns (precision "split_tf32": W = 64 slices as 3xTF32 GEMMs on tcgen05,
two-level tables) against the oracle.

Bars: weights elementwise within 1e-5 of the row sum (the FP32 table bar; chains here are at
most 40 slices, where the tensor-core accumulation bias stays below it); realised two-level
distributions within the quantisation bound (L + W + 4) 2^-32 plus 1e-5 of the row of the
oracle's FP64 weights; row sums (the sum rule,
checked again by the alias build) 1e-5; walks bit-exact against the oracle's two-level walker on
the exported tables; Monte Carlo T against the direct probe solve with every |z| <= z_bar(m)
and sum z^2 <= chi2_bar(m) (mc_bars); negf_run and plans
equal to build + walk for a batch mixing tensor-core and CUDA-core wires.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import chi2_bar, z_bar  # noqa: E402
from oracle import alias, pipeline, walker  # noqa: E402
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
    return [inputs.small_wire(121, W=64, L=1, n_energy=1, eta=0.05, disorder=0.5),
            inputs.small_wire(122, W=64, L=4, n_energy=2, eta=0.02, disorder=0.5, e_lo=-1.0,
                              e_hi=1.0),
            inputs.small_wire(123, W=64, L=7, n_energy=1, eta=0.005, disorder=0.5),
            inputs.small_wire(124, W=64, L=40, n_energy=1, eta=0.05, disorder=1.0, e_lo=0.37,
                              e_hi=0.37),
            inputs.small_wire(125, W=64, L=5, n_energy=1, eta=0.1, lead_model=1, gamma_lead=0.8)]


@pytest.fixture(scope="module")
def batch(ctx):
    wires = _wires()
    refs = []
    for w in wires:
        for E in w.energy:
            refs.append(pipeline.task_reference(w.onsite, w.eta, w.t, E, w.lead_model,
                                                w.gamma_lead, with_alias=False))
    return wires, refs


def _export(ctx, tables, task):
    info = negf.negf_get_task_info(ctx, tables, task)
    assert info["layout"] == "two_level"
    rows, L, W = info["rows"], info["L"], info["W"]
    l2 = negf.negf_export_tables(ctx, tables, task, "alias").view(np.uint32).reshape(
        rows, L, negf.level2_words(W))
    l1 = negf.negf_export_tables(ctx, tables, task, "alias_level1").reshape(rows, L + 2)
    return info, l1, l2


def test_tensor_core_tables_realise_oracle_weights(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="split_tf32", keep_weights=True)
    try:
        rng = np.random.default_rng(3)
        for task, ref in enumerate(refs):
            info, l1, l2 = _export(ctx, tables, task)
            w_ref = ref["tab"]["w"]
            rs_ref = w_ref.sum(1)
            rs = negf.negf_export_tables(ctx, tables, task, "rowsum")
            assert np.allclose(rs, rs_ref, rtol=1e-5), task
            assert np.allclose(info["c"], ref["tab"]["c"], rtol=1e-5)
            L, W = info["L"], info["W"]
            quant = (L + W + 4) * 2.0**-32
            rows = np.concatenate([rng.choice(info["rows"], size=min(24, info["rows"]),
                                              replace=False),
                                   np.arange(info["n"], info["rows"], 17)])   # injection rows
            w = negf.negf_export_tables(ctx, tables, task, "weights").reshape(w_ref.shape)
            bad = np.abs(w - w_ref) > 1e-5 * rs_ref[:, None] + 1e-30
            assert not bad.any(), (task, np.argwhere(bad)[:5])
            for r in rows:
                p = alias.implied_two_level(l1[r], l2[r], W)
                err = np.max(np.abs(p - w_ref[r] / rs_ref[r]))
                assert err <= quant + 1e-5, (task, r, err)
    finally:
        negf.negf_tables_free(tables)


def test_tensor_core_walks_bit_exact(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="split_tf32")
    try:
        n_w = 2000
        for task in range(len(refs)):
            info, l1, l2 = _export(ctx, tables, task)
            ment = negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, info["W"])
            for lead0, off in ((0, 0), (1, 2**34 + 1)):
                d_lead = torch.empty(n_w, dtype=torch.int32, device="cuda")
                d_steps = torch.empty(n_w, dtype=torch.int32, device="cuda")
                negf.negf_walk_trace(ctx, tables, task, lead0, 0xACE + task, off, d_lead, d_steps)
                lead, steps = walker.walk_two_level(l1, l2, ment, info["n"], info["L"], info["W"],
                                                    info["c"] > 0, task, lead0, 0xACE + task,
                                                    off + np.arange(n_w), 1 << 20)
                assert np.array_equal(d_lead.cpu().numpy(), lead), (task, lead0)
                assert np.array_equal(d_steps.cpu().numpy().astype(np.uint32), steps)
    finally:
        negf.negf_tables_free(tables)


def test_tensor_core_monte_carlo_transmission(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="split_tf32")
    try:
        N = 400_000
        z = []
        for lead0 in (0, 1):
            tally = negf.negf_walk(ctx, tables, lead0, 17 + lead0, N)
            res = negf.negf_current(ctx, tables, tally, 3.5, -3.5, 0.025)
            negf.negf_tally_free(tally)
            for task, ref in enumerate(refs):
                T_ref = ref["T_direct"][1 - lead0, lead0]
                if res["T_se"][task] > 0:
                    z.append((res["T"][task] - T_ref) / (res["T_se"][task] + 1e-5 * T_ref))
                else:
                    assert abs(res["T"][task] - T_ref) <= 1e-5 * T_ref + 1e-12, task
        z = np.asarray(z)
        assert np.max(np.abs(z)) <= z_bar(z.size) and np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tables_free(tables)


def test_tensor_core_mixed_batch_run_and_plan(ctx):
    """W = 64 wires (tensor cores) and narrower ones (CUDA cores, one-level) in one batch:
    negf_run waves and a captured plan reproduce build + walk."""
    wires = [inputs.small_wire(131, W=64, L=6, n_energy=2, eta=0.03, disorder=0.5),
             inputs.small_wire(132, W=5, L=9, n_energy=2, eta=0.1),
             inputs.small_wire(133, W=64, L=3, n_energy=1, eta=0.05, disorder=0.5)]
    n_tasks = 5
    N = 20000
    t = negf.negf_build_tables(ctx, wires, precision="split_tf32")
    try:
        layouts = [negf.negf_get_task_info(ctx, t, k)["layout"] for k in range(n_tasks)]
        assert layouts == ["two_level", "two_level", "one_level", "one_level", "two_level"]
        tl = negf.negf_walk(ctx, t, 0, 555, N, walker_id_offset=3)
        ref = negf.negf_tally_counts(ctx, tl, n_tasks)
        negf.negf_tally_free(tl)
    finally:
        negf.negf_tables_free(t)
    for per_wave in (0, 1, 2):
        t, tl = negf.negf_run(ctx, wires, 0, 555, N, precision="split_tf32", walker_id_offset=3,
                              tasks_per_wave=per_wave)
        got = negf.negf_tally_counts(ctx, tl, n_tasks)
        negf.negf_tally_free(tl)
        negf.negf_tables_free(t)
        assert np.array_equal(got, ref), per_wave
    plan = negf.negf_plan_create(ctx, wires, 0, N, 3.5, -3.5, 0.025, precision="split_tf32",
                                 tasks_per_wave=2, autotune=True)
    try:
        negf.negf_plan_launch(ctx, plan, 555, 3)
        assert np.array_equal(negf.negf_plan_result(ctx, plan)["counts"], ref)
    finally:
        negf.negf_plan_destroy(plan)
