"""Inelastic Buttiker probes (Step 7') on the GPU against the oracle (oracle/inelastic.py).

Bars:
  * the Step 7' energy rows: the distribution each alias row realises (exact integers) against
    the oracle's hop probabilities p(e' | i, e) = w_e' K A_ii(E_e') / sum: the quantisation
    bound (nE + 2) 2^-32 plus 1e-9 (FP64 tables: the kernel's row sums and the oracle's agree to
    rounding); sigma = 0 rows are the identity draw;
  * walks: the tallies of negf_walk_inelastic (done, absorbed L and R, truncated, summed steps
    per injection task) equal, count for count, those of the oracle's walker run on the
    exported tables and energy rows with the same Philox streams, for both start leads and a
    step cap;
  * Monte Carlo T_qp(E_0) = c_p P(q | p, E_0) and mean steps of FP32 tables against the exact
    chain over (site, energy) states, every abs(z) <= z_bar(m) (mc_bars: the 3-SE bar as a
    0.27 % family-wise false-alarm rate);
  * refusals: two-level tables, a negative or non-finite sigma.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import z_bar  # noqa: E402
from oracle import alias, inelastic, pipeline  # noqa: E402
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


def _wire():
    return inputs.small_wire(81, W=3, L=6, n_energy=6, eta=0.4, e_lo=-2.6, e_hi=2.6)


def _oracle_chain(w, sigma):
    on = w.onsite.reshape(w.L, w.W)
    et = w.eta.reshape(w.L, w.W)
    refs = [pipeline.task_reference(on, et, w.t, E, with_direct=False) for E in w.energy]
    return refs, inelastic.chain([r["tab"] for r in refs], w.energy, w.energy_weight, sigma)


@pytest.mark.parametrize("sigma", [0.0, 0.45])
def test_energy_rows_realise_the_hop_law(ctx, sigma):
    w = _wire()
    _, ch = _oracle_chain(w, sigma)
    tables = negf.negf_build_tables(ctx, [w], precision="fp64")
    try:
        nE = len(w.energy)
        for task in range(nE):
            rows = negf.negf_export_energy_tables(ctx, tables, task, sigma)
            assert rows.shape == (w.W * w.L, nE)
            for i in range(rows.shape[0]):
                p = alias.implied_distribution(rows[i])
                assert np.max(np.abs(p - ch["H"][i, task])) <= (nE + 2) / 2**32 + 1e-9, (task, i)
    finally:
        negf.negf_tables_free(tables)


def _export(ctx, tables, nE):
    ent, ment, c_open = [], [], []
    for task in range(nE):
        info = negf.negf_get_task_info(ctx, tables, task)
        ent.append(negf.negf_export_tables(ctx, tables, task, "alias").reshape(info["rows"], info["K"]))
        ment.append(negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, info["W"]))
        c_open.append(info["c"] > 0)
    return info, np.stack(ent), np.stack(ment), np.stack(c_open)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tallies_equal_the_oracle_walker(ctx, precision):
    w = _wire()
    nE = len(w.energy)
    sigma = 0.45
    tables = negf.negf_build_tables(ctx, [w], precision=precision)
    try:
        info, ent, ment, c_open = _export(ctx, tables, nE)
        erows = np.stack([negf.negf_export_energy_tables(ctx, tables, t, sigma) for t in range(nE)],
                         axis=1)                                       # [n, nE, nE]
        N = 2000
        for p, cap, off in ((0, 1 << 20, 0), (1, 1 << 20, 2**33 + 7), (0, 2, 91)):
            seed = 0xE1A5 + p
            tally = negf.negf_walk_inelastic(ctx, tables, p, seed, N, sigma, walker_id_offset=off,
                                             max_steps=cap)
            try:
                got = negf.negf_tally_counts(ctx, tally, nE)
            finally:
                negf.negf_tally_free(tally)
            for e0 in range(nE):
                lead, steps = inelastic.walk(ent, ment, erows, info["n"], info["W"], c_open, e0,
                                             e0, p, seed, off + np.arange(N, dtype=np.uint64), cap)
                want = [N, np.sum(lead == 0), np.sum(lead == 1), np.sum(lead == -2),
                        int(steps.astype(np.uint64).sum())]
                assert np.array_equal(got[e0].astype(np.int64), np.array(want, dtype=np.int64)), \
                    (precision, p, cap, e0, got[e0], want)
    finally:
        negf.negf_tables_free(tables)


def test_monte_carlo_matches_the_exact_chain(ctx):
    w = _wire()
    nE = len(w.energy)
    sigma = 0.45
    refs, ch = _oracle_chain(w, sigma)
    tables = negf.negf_build_tables(ctx, [w], precision="fp32")
    try:
        N = 200_000
        zs = []
        for p in (0, 1):
            tally = negf.negf_walk_inelastic(ctx, tables, p, 777 + p, N, sigma)
            try:
                cnt = negf.negf_tally_counts(ctx, tally, nE).astype(np.float64)
            finally:
                negf.negf_tally_free(tally)
            q = 1 - p
            for e0 in range(nE):
                if refs[e0]["tab"]["c"][p] <= 0:
                    continue
                P = ch["P_inj"][e0, p, q]
                Ph = cnt[e0, 1 + q] / cnt[e0, 0]
                zs.append((Ph - P) / np.sqrt(max(P * (1 - P), 1e-300) / N))
                m = ch["steps_inj"][e0, p]
                # steps are geometric-like: their variance bounded via the oracle's own samples
                _, st = inelastic.walk(np.stack([r["entries"] for r in refs]),
                                       np.stack([r["mode_entries"] for r in refs]),
                                       inelastic.energy_tables(ch["weights"]), refs[0]["n"],
                                       refs[0]["W"], np.stack([r["c_open"] for r in refs]), e0,
                                       e0, p, 5, np.arange(20000), 1 << 20)
                zs.append((cnt[e0, 4] / cnt[e0, 0] - m) / (st.std() / np.sqrt(N)))
        zs = np.array(zs)
        assert np.all(np.abs(zs) <= z_bar(zs.size)), zs
    finally:
        negf.negf_tables_free(tables)


def test_refusals(ctx):
    w = _wire()
    two = negf.negf_build_tables(ctx, [w], precision="fp32", layout="two_level")
    one = negf.negf_build_tables(ctx, [w], precision="fp32")
    try:
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_walk_inelastic(ctx, two, 0, 1, 10, 0.3)
        for bad in (-0.1, float("nan"), float("inf")):
            with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
                negf.negf_walk_inelastic(ctx, one, 0, 1, 10, bad)
    finally:
        negf.negf_tables_free(two)
        negf.negf_tables_free(one)


def test_several_wires_in_one_handle(ctx):
    """Energy rows and walks of wires of different widths, lengths and grids in one table
    handle: each wire's walkers hop over its own grid only (tallies count for count against
    the oracle walker on each wire's exported tables)."""
    wires = [inputs.small_wire(82, W=2, L=5, n_energy=4, eta=0.5, e_lo=-1.8, e_hi=1.8),
             inputs.small_wire(83, W=4, L=3, n_energy=7, eta=0.3, e_lo=-3.2, e_hi=3.2)]
    sigma = 0.6
    tables = negf.negf_build_tables(ctx, wires, precision="fp64")
    try:
        N, seed = 1500, 0xBEE5
        for p in (0, 1):
            tally = negf.negf_walk_inelastic(ctx, tables, p, seed + p, N, sigma)
            try:
                got = negf.negf_tally_counts(ctx, tally, sum(len(w.energy) for w in wires))
            finally:
                negf.negf_tally_free(tally)
            t0 = 0
            for w in wires:
                nE = len(w.energy)
                ent, ment, c_open, erows = [], [], [], []
                for k in range(nE):
                    info = negf.negf_get_task_info(ctx, tables, t0 + k)
                    ent.append(negf.negf_export_tables(ctx, tables, t0 + k, "alias").reshape(
                        info["rows"], info["K"]))
                    ment.append(negf.negf_export_tables(ctx, tables, t0 + k, "mode_alias").reshape(
                        2, info["W"]))
                    c_open.append(info["c"] > 0)
                    erows.append(negf.negf_export_energy_tables(ctx, tables, t0 + k, sigma))
                ent, ment, c_open = np.stack(ent), np.stack(ment), np.stack(c_open)
                erows = np.stack(erows, axis=1)
                assert erows.shape == (w.W * w.L, nE, nE)
                for e0 in range(nE):
                    lead, steps = inelastic.walk(ent, ment, erows, w.W * w.L, w.W, c_open, e0,
                                                 t0 + e0, p, seed + p, np.arange(N, dtype=np.uint64),
                                                 1 << 20)
                    want = [N, np.sum(lead == 0), np.sum(lead == 1), np.sum(lead == -2),
                            int(steps.astype(np.uint64).sum())]
                    assert np.array_equal(got[t0 + e0].astype(np.int64),
                                          np.array(want, dtype=np.int64)), (p, t0, e0)
                t0 += nE
    finally:
        negf.negf_tables_free(tables)
