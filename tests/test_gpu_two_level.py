"""Two-level tables (slice or lead, then the site within the slice) on the GPU against the oracle.

Bars:
  * the distribution a two-level row realises (exact product of its level-1 alias row and its
    level-2 inverse-CDF blocks) against the oracle's FP64 weights / row sum: the quantisation bound
    (L + W + 4) 2^-32 plus 1e-10 (FP64 build) or 1e-5 (FP32 build) of the row;
  * the same distribution against the kernel's own weights (keep_weights): within the
    quantisation bound (L + W + 4) 2^-32 + 4 eps;
  * walks bit-exact against the oracle's two-level walker on the exported tables;
  * Monte Carlo T against the direct probe solve and mean steps against the exact chain, every
    |z| <= z_bar(m) and sum z^2 <= chi2_bar(m) (mc_bars: the 3-SE bar as a 0.27 % family-wise
    false-alarm rate); a single comparison at 3 SE;
  * negf_run and captured plans give the same tallies as build + walk.
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
    return [inputs.chain_l20().wires[0],
            inputs.small_wire(111, W=3, L=9, n_energy=2, eta=0.1),
            inputs.small_wire(112, W=5, L=13, n_energy=2, eta=0.07, e_lo=-3.8, e_hi=3.8),
            inputs.small_wire(113, W=33, L=3, n_energy=1, eta=0.05),
            inputs.small_wire(114, W=64, L=3, n_energy=1, eta=0.02, disorder=0.5),
            inputs.small_wire(115, W=4, L=5, n_energy=1, eta=0.15, lead_model=1, gamma_lead=0.8)]


@pytest.fixture(scope="module")
def batch(ctx):
    wires = _wires()
    refs = []
    for w in wires:
        for E in w.energy:
            refs.append(pipeline.task_reference(w.onsite, w.eta, w.t, E, w.lead_model,
                                                w.gamma_lead, with_alias=False))
    return wires, refs


def _export_two_level(ctx, tables, task):
    info = negf.negf_get_task_info(ctx, tables, task)
    assert info["layout"] == "two_level"
    rows, L, W = info["rows"], info["L"], info["W"]
    l2 = negf.negf_export_tables(ctx, tables, task, "alias").view(np.uint32).reshape(
        rows, L, negf.level2_words(W))
    l1 = negf.negf_export_tables(ctx, tables, task, "alias_level1").reshape(rows, L + 2)
    return info, l1, l2


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_two_level_tables_realise_oracle_weights(ctx, batch, precision, tol):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision=precision, keep_weights=True,
                                    layout="two_level")
    try:
        rng = np.random.default_rng(1)
        for task, ref in enumerate(refs):
            info, l1, l2 = _export_two_level(ctx, tables, task)
            w_ref = ref["tab"]["w"]
            rs_ref = w_ref.sum(1)
            w = negf.negf_export_tables(ctx, tables, task, "weights").reshape(w_ref.shape)
            rs = negf.negf_export_tables(ctx, tables, task, "rowsum")
            assert np.allclose(rs, rs_ref, rtol=1e-10 if precision == "fp64" else 1e-5)
            L, W = info["L"], info["W"]
            rows = rng.choice(info["rows"], size=min(10, info["rows"]), replace=False)
            quant = (L + W + 4) * 2.0**-32
            for r in rows:
                p = alias.implied_two_level(l1[r], l2[r], W)
                assert np.max(np.abs(p - w_ref[r] / rs_ref[r])) <= quant + tol, (task, r)
                own = w[r] / w[r].sum()
                assert np.max(np.abs(p - own)) <= (L + W + 4) * 2.0**-32 + 4e-7, (task, r)
    finally:
        negf.negf_tables_free(tables)


def test_two_level_walks_bit_exact(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32", layout="two_level")
    try:
        n_w = 2000
        for task in range(len(refs)):
            info, l1, l2 = _export_two_level(ctx, tables, task)
            ment = negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, info["W"])
            for lead0, cap, off in ((0, 1 << 20, 0), (1, 1 << 20, 2**33 + 5), (0, 2, 77)):
                d_lead = torch.empty(n_w, dtype=torch.int32, device="cuda")
                d_steps = torch.empty(n_w, dtype=torch.int32, device="cuda")
                negf.negf_walk_trace(ctx, tables, task, lead0, 0xBEEF + task, off, d_lead,
                                     d_steps, max_steps=cap)
                lead, steps = walker.walk_two_level(l1, l2, ment, info["n"], info["L"],
                                                    info["W"], info["c"] > 0, task, lead0,
                                                    0xBEEF + task, off + np.arange(n_w), cap)
                assert np.array_equal(d_lead.cpu().numpy(), lead), (task, lead0, cap)
                assert np.array_equal(d_steps.cpu().numpy().astype(np.uint32), steps)
    finally:
        negf.negf_tables_free(tables)


def test_two_level_monte_carlo_transmission(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32", layout="two_level")
    try:
        N = 400_000
        z_T, z_steps = [], []
        for lead0 in (0, 1):
            tally = negf.negf_walk(ctx, tables, lead0, 99 + lead0, N)
            counts = negf.negf_tally_counts(ctx, tally, len(refs))
            res = negf.negf_current(ctx, tables, tally, 3.5, -3.5, 0.025)
            negf.negf_tally_free(tally)
            q = 1 - lead0
            for task, ref in enumerate(refs):
                T_ref = ref["T_direct"][q, lead0]
                if ref["tab"]["c"][lead0] > 0:
                    z_T.append((res["T"][task] - T_ref) / (res["T_se"][task] + 1e-6 * T_ref))
                    ms = counts[task, 4] / N
                    m_ref = ref["exact"]["steps_inj"][lead0]
                    var = ref["exact"]["steps2_inj"][lead0] - m_ref**2
                    z_steps.append((ms - m_ref) / np.sqrt(var / N))
                else:
                    assert res["T"][task] == 0.0 and T_ref <= 1e-12, task
        for z in (np.asarray(z_T), np.asarray(z_steps)):
            assert np.max(np.abs(z)) <= z_bar(z.size) and np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tables_free(tables)


def test_two_level_through_run_and_plan(ctx, batch):
    """negf_run waves and a captured plan give the tallies of build + walk on two-level tables."""
    wires, refs = batch
    n_tasks = len(refs)
    N = 20000
    ref_t = negf.negf_build_tables(ctx, wires, precision="fp32", layout="two_level")
    ref_tl = negf.negf_walk(ctx, ref_t, 0, 4321, N, walker_id_offset=9)
    ref = negf.negf_tally_counts(ctx, ref_tl, n_tasks)
    negf.negf_tally_free(ref_tl)
    negf.negf_tables_free(ref_t)
    for per_wave in (0, 2):
        t, tl = negf.negf_run(ctx, wires, 0, 4321, N, precision="fp32", walker_id_offset=9,
                              tasks_per_wave=per_wave, layout="two_level")
        got = negf.negf_tally_counts(ctx, tl, n_tasks)
        negf.negf_tally_free(tl)
        negf.negf_tables_free(t)
        assert np.array_equal(got, ref), per_wave
    plan = negf.negf_plan_create(ctx, wires, 0, N, 3.5, -3.5, 0.025, precision="fp32",
                                 tasks_per_wave=3, layout="two_level", autotune=True)
    try:
        negf.negf_plan_launch(ctx, plan, 4321, 9)
        assert np.array_equal(negf.negf_plan_result(ctx, plan)["counts"], ref)
    finally:
        negf.negf_plan_destroy(plan)


def test_auto_layout_for_long_wire(ctx):
    """W = 64, L = 101 (6464 sites, above the automatic two-level threshold and the one-level
    limit) builds two-level tables by itself;
    sampled rows realise the oracle's weights and the transmission matches the direct solve."""
    w = inputs.small_wire(116, W=64, L=101, n_energy=1, eta=0.02, disorder=0.5, e_lo=-0.3,
                          e_hi=-0.3)
    ref = pipeline.task_reference(w.onsite, w.eta, w.t, w.energy[0], with_alias=False)
    tables = negf.negf_build_tables(ctx, [w], precision="fp32")
    try:
        info, l1, l2 = _export_two_level(ctx, tables, 0)
        w_ref = ref["tab"]["w"]
        rs_ref = w_ref.sum(1)
        rng = np.random.default_rng(2)
        for r in rng.choice(info["rows"], size=6, replace=False):
            p = alias.implied_two_level(l1[r], l2[r], 64)
            assert np.max(np.abs(p - w_ref[r] / rs_ref[r])) <= (101 + 64 + 4) * 2.0**-32 + 1e-5, r
        N = 200_000
        tally = negf.negf_walk(ctx, tables, 0, 5, N)
        res = negf.negf_current(ctx, tables, tally, 3.5, -3.5, 0.025)
        negf.negf_tally_free(tally)
        T_ref = ref["T_direct"][1, 0]
        assert abs(res["T"][0] - T_ref) <= 3.0 * res["T_se"][0] + 1e-6 * T_ref
    finally:
        negf.negf_tables_free(tables)


def test_two_level_refusals(ctx):
    w = inputs.small_wire(117, W=3, L=4, n_energy=1)
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        negf.negf_build_tables(ctx, [w], layout="two_level", keep_green=True)
    t = negf.negf_build_tables(ctx, [w], layout="one_level")
    try:
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_export_tables(ctx, t, 0, "alias_level1")
    finally:
        negf.negf_tables_free(t)
