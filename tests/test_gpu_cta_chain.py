"""FP32 block columns by the CTA-wide kernels against the oracle: W = 64 wires
(chain_cta_kernel), 16 < W <= 32 wires (chain_cta_narrow_kernel, odd and even widths, both
ends of the range, ragged lengths down to L = 1), and a batch mixing both with a W <= 16 wire
(whose columns the column-per-lane chain builds in the same wave).  Bars: weights elementwise within 1e-5 of
the row sum (the FP32 table bar), one-level and two-level tables, lead weights at both boundary
slices, and bit-exact walks on the exported tables."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _wires(kind):
    if kind == "mixed":
        # one batch whose tasks take three block-column kernels: W = 64 and 16 < W <= 32 the
        # CTA chains, W <= 16 the column-per-lane chain
        return [inputs.small_wire(161, W=64, L=3, n_energy=1, eta=0.05, disorder=0.5),
                inputs.small_wire(162, W=9, L=6, n_energy=2, eta=0.04, disorder=0.7),
                inputs.small_wire(163, W=19, L=4, n_energy=1, eta=0.06, disorder=0.6)]
    if kind == "narrow":
        return [inputs.small_wire(151, W=17, L=1, n_energy=1, eta=0.05, disorder=0.5),
                inputs.small_wire(152, W=20, L=7, n_energy=2, eta=0.03, disorder=0.8,
                                  e_lo=-1.5, e_hi=1.2),
                inputs.small_wire(153, W=25, L=2, n_energy=1, eta=0.1, disorder=0.5),
                inputs.small_wire(154, W=31, L=12, n_energy=1, eta=0.01, disorder=0.5,
                                  e_lo=0.41, e_hi=0.41),
                inputs.small_wire(155, W=32, L=5, n_energy=1, eta=0.08, lead_model=1,
                                  gamma_lead=0.7),
                inputs.small_wire(156, W=24, L=9, n_energy=1, eta=0.05, disorder=1.0)]
    return [inputs.small_wire(141, W=64, L=1, n_energy=1, eta=0.05, disorder=0.5),
            inputs.small_wire(142, W=64, L=3, n_energy=2, eta=0.02, disorder=0.5, e_lo=-1.0,
                              e_hi=1.0),
            inputs.small_wire(143, W=64, L=40, n_energy=1, eta=0.005, disorder=0.5, e_lo=0.37,
                              e_hi=0.37),
            inputs.small_wire(144, W=64, L=6, n_energy=1, eta=0.1, lead_model=1, gamma_lead=0.8)]


@pytest.fixture(scope="module", params=["wide", "narrow", "mixed"])
def batch(ctx, request):
    wires = _wires(request.param)
    refs = []
    for w in wires:
        for E in w.energy:
            refs.append(pipeline.task_reference(w.onsite, w.eta, w.t, E, w.lead_model,
                                                w.gamma_lead, with_alias=False))
    return wires, refs


@pytest.mark.parametrize("layout", ["one_level", "two_level"])
def test_cta_chain_weights_match_oracle(ctx, batch, layout):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32", keep_weights=True,
                                    layout=layout)
    try:
        for task, ref in enumerate(refs):
            w_ref = ref["tab"]["w"]
            rs_ref = w_ref.sum(1)
            w = negf.negf_export_tables(ctx, tables, task, "weights").reshape(w_ref.shape)
            bad = np.abs(w - w_ref) > 1e-5 * rs_ref[:, None] + 1e-30
            assert not bad.any(), (task, np.argwhere(bad)[:5])
            rs = negf.negf_export_tables(ctx, tables, task, "rowsum")
            assert np.allclose(rs, rs_ref, rtol=1e-5)
            info = negf.negf_get_task_info(ctx, tables, task)
            assert info["layout"] == layout
            if layout == "two_level":
                L, W = info["L"], info["W"]
                l2 = negf.negf_export_tables(ctx, tables, task, "alias").view(np.uint32).reshape(
                    info["rows"], L, negf.level2_words(W))
                l1 = negf.negf_export_tables(ctx, tables, task, "alias_level1").reshape(info["rows"], L + 2)
                for r in (0, info["n"] - 1, info["n"], info["rows"] - 1):
                    p = alias.implied_two_level(l1[r], l2[r], W)
                    assert np.max(np.abs(p - w_ref[r] / rs_ref[r])) <= (L + W + 4) * 2.0**-32 + 1e-5
    finally:
        negf.negf_tables_free(tables)


def test_cta_chain_walks_bit_exact(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32", layout="one_level")
    try:
        n_w = 2000
        for task in range(len(refs)):
            info = negf.negf_get_task_info(ctx, tables, task)
            ent = negf.negf_export_tables(ctx, tables, task, "alias").reshape(info["rows"], info["K"])
            ment = negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, info["W"])
            d_lead = torch.empty(n_w, dtype=torch.int32, device="cuda")
            d_steps = torch.empty(n_w, dtype=torch.int32, device="cuda")
            negf.negf_walk_trace(ctx, tables, task, 1, 0xF00D + task, 5, d_lead, d_steps)
            lead, steps = walker.walk(ent, ment, info["n"], info["W"], info["c"] > 0, task, 1,
                                      0xF00D + task, 5 + np.arange(n_w), 1 << 20)
            assert np.array_equal(d_lead.cpu().numpy(), lead), task
            assert np.array_equal(d_steps.cpu().numpy().astype(np.uint32), steps)
    finally:
        negf.negf_tables_free(tables)


def _two_level_export(ctx, tables, task):
    info = negf.negf_get_task_info(ctx, tables, task)
    l2 = negf.negf_export_tables(ctx, tables, task, "alias")
    l1 = negf.negf_export_tables(ctx, tables, task, "alias_level1")
    return info, l1, l2


def test_fused_level2_equals_stored_weights_path(ctx):
    """W = 64 two-level tables built without kept weights take the fused path (the chain
    writes the level-2 blocks and level-1 weights); with keep_weights the weights are stored
    and the level-2 pass builds them.  Both must give the same bits, for single builds, the
    batched run's waves and a captured plan, and realise the oracle's weights."""
    wires = _wires("wide") + [inputs.small_wire(145, W=9, L=5, n_energy=1, eta=0.07)]
    stored = negf.negf_build_tables(ctx, wires, precision="fp32", keep_weights=True,
                                    layout="two_level")
    fused = negf.negf_build_tables(ctx, wires, precision="fp32", layout="two_level")
    try:
        n_tasks = negf.negf_tables_num_tasks(fused)
        ref = [_two_level_export(ctx, stored, k) for k in range(n_tasks)]
        for k in range(n_tasks):
            info, l1, l2 = _two_level_export(ctx, fused, k)
            assert info["layout"] == "two_level"
            assert np.array_equal(l1, ref[k][1]), k
            assert np.array_equal(l2, ref[k][2]), k
            assert np.array_equal(negf.negf_export_tables(ctx, fused, k, "rowsum"),
                                  negf.negf_export_tables(ctx, stored, k, "rowsum")), k
        # against the oracle: sampled rows' realised distributions
        rng = np.random.default_rng(9)
        task = 0
        for w in wires:
            for E in w.energy:
                info, l1, l2 = _two_level_export(ctx, fused, task)
                rows, L, W = info["rows"], info["L"], info["W"]
                l1 = l1.reshape(rows, L + 2)
                l2 = l2.view(np.uint32).reshape(rows, L, negf.level2_words(W))
                tab = pipeline.task_reference(w.onsite, w.eta, w.t, E, w.lead_model,
                                              w.gamma_lead, with_alias=False)["tab"]
                rs = tab["w"].sum(1)
                for r in rng.choice(rows, size=min(12, rows), replace=False):
                    if rs[r] > 0:
                        p = alias.implied_two_level(l1[r], l2[r], W)
                        assert np.max(np.abs(p - tab["w"][r] / rs[r])) <= \
                            (L + W + 4) * 2.0**-32 + 1e-5, (task, r)
                task += 1
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_walk_score(ctx, fused, 0, 1, 10)      # no weights for the score seeds
        # batched waves and a captured plan take the fused path too: same tallies as the
        # stored-weights tables
        N = 20000
        tl = negf.negf_walk(ctx, stored, 0, 4242, N, walker_id_offset=3)
        want = negf.negf_tally_counts(ctx, tl, n_tasks)
        negf.negf_tally_free(tl)
        for per_wave in (0, 2):
            t, tl = negf.negf_run(ctx, wires, 0, 4242, N, precision="fp32", walker_id_offset=3,
                                  tasks_per_wave=per_wave, layout="two_level")
            got = negf.negf_tally_counts(ctx, tl, n_tasks)
            negf.negf_tally_free(tl)
            negf.negf_tables_free(t)
            assert np.array_equal(got, want), per_wave
        plan = negf.negf_plan_create(ctx, wires, 0, N, 3.5, -3.5, 0.025, precision="fp32",
                                     tasks_per_wave=2, layout="two_level", autotune=False)
        try:
            negf.negf_plan_launch(ctx, plan, 4242, walker_id_offset=3)
            got = negf.negf_plan_result(ctx, plan)["counts"]
            assert np.array_equal(got, want)
        finally:
            negf.negf_plan_destroy(plan)
    finally:
        negf.negf_tables_free(stored)
        negf.negf_tables_free(fused)
