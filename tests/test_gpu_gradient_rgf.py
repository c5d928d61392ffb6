"""Block-column adjoint with checkpointed RGF blocks (negf_current_backward_rgf) against the
oracle's exact FP64 derivative (oracle.adjoint, pinned to finite differences of the direct
probe solve).

* Exact tallies (the score counts replaced by their expectations for N = 2^52 walks, from the
  oracle's absorbing chain; the largest N whose counts a double holds exactly: the counts are
  integers, and a count rounded by 1/2 moves the seed of a transition of weight w by 1/(2 N w),
  which far-apart sites' tiny weights amplify): every component within rel |ref| + floor
  max|ref| of the exact derivative: FP64 rel 1e-6, floor 1e-9; FP32 rel 1e-4, floor 1e-6,
  except on the two-level W = 64 x L = 150 wire in FP32: rel 1e-3, floor 1e-4 (there the FP32
  tables hold a weight to the FP32 table bar, 1e-5 of its row, after chains of up to 150
  slices, and the FP64 expectations of the counts meet those weights in every seed s / w;
  measured 2.4e-5 of the largest component).  Wires: W = 3 x L = 5,
  W = 7 x L = 23 (several row tiles and a ragged one), and a two-level W = 64 x L = 150 wire
  (FP64 and FP32, compared at sampled sites: the oracle's forward-mode derivative costs one
  dense tangent per site).
* The dense adjoint (negf_current_backward, dense G) on the same tallies: equal to 1e-10 of the
  largest component (FP64).
* Checkpoint strides 1, 2, 3, 7, L, L + 4 and the default: equal to 1e-12 of the largest
  component (the recomputed blocks are the swept ones bit for bit; only the order of the FP64
  atomic sums differs).
* Two-level score walks: the score tallies hold every transition of every absorbed walk
  (sum = the walks' steps, mode counts = absorbed walks), and the gradient from real two-level
  walks is unbiased: projections within the family-wise 3-SE bar of Student's t over 20 batches.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import t_bar  # noqa: E402
from oracle import adjoint, current as ocur, markov, wire  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402

MU_P, MU_Q, KT = 0.6, -0.4, 0.3
BARS = {"fp64": (1e-6, 1e-9), "fp32": (1e-4, 1e-6), "fp32_long": (1e-3, 1e-4)}
N_EXACT = float(2 ** 52)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    c = negf.negf_create(0)
    yield c
    negf.negf_destroy(c)


def _weights_df(w):
    return w.energy_weight * (ocur.fermi(w.energy, MU_P, KT) - ocur.fermi(w.energy, MU_Q, KT))


def _exact_grad(w, p, sites=None):
    """dI/dV, dI/deta [L*W] (oracle, FP64; only `sites` when given)."""
    q = 1 - p
    gV = np.zeros(w.W * w.L)
    gE = np.zeros(w.W * w.L)
    for k, (E, f) in enumerate(zip(w.energy, _weights_df(w))):
        _, dV, dE = adjoint.transmission_gradient(w.onsite, w.eta, w.t, E, p, q, sites=sites)
        gV += f * dV.reshape(-1)
        gE += f * dE.reshape(-1)
    return gV, gE


def _expected_counts(w, E, p, N):
    """Exact expected tallies of N walks from lead p (oracle absorbing chain): basic counts,
    score counts [2, rows*K], mode counts [2, 2W]."""
    g = wire.green_retarded(E, w.onsite, w.eta, w.t)
    phi, _, gam = wire.lead_modes(E, w.W, w.t)
    tab = markov.transition_weights(g, (phi, gam))
    n, W = w.W * w.L, w.W
    rs = tab["w"].sum(1, keepdims=True)
    P = np.divide(tab["w"], rs, out=np.zeros_like(tab["w"]), where=rs > 0)
    rows, K = P.shape
    IQ = np.eye(n) - P[:n, :n]
    h = np.linalg.solve(IQ, P[:n, n:])
    u = tab["mode_w"][p] / tab["mode_w"][p].sum()
    inj = slice(n + p * W, n + (p + 1) * W)
    nu = np.zeros(rows)
    nu[inj] = u
    nu[:n] = np.linalg.solve(IQ.T, P[inj, :n].T @ u)
    score = np.empty((2, rows * K), dtype=np.uint64)
    for rr in range(2):
        hb = np.concatenate([h[:, rr], [1.0 if rr == 0 else 0.0, 1.0 if rr == 1 else 0.0]])
        score[rr] = np.rint(N * (nu[:, None] * P * hb[None, :])).reshape(-1)
    v = P[inj, n:] + P[inj, :n] @ h
    mode = np.zeros((2, 2 * W))
    for rr in range(2):
        mode[rr, p * W:(p + 1) * W] = u * v[:, rr]
    Pr = u @ v
    counts = np.array([N, N * Pr[0], N * Pr[1], 0, 0], dtype=np.float64)
    return np.rint(counts).astype(np.uint64), score, np.rint(N * mode).astype(np.uint64)


def _exact_tally(ctx, tables, w, p, N=N_EXACT):
    tally = negf.negf_walk_score(ctx, tables, p, 1, 0)      # allocated, all counts zero
    ns = negf.load().negf_tally_score_size(tally)
    nm = negf.load().negf_tally_mode_size(tally)
    basic = np.zeros((len(w.energy), negf.TALLY_FIELDS), dtype=np.uint64)
    sc = np.zeros((2, ns), dtype=np.uint64)
    md = np.zeros((2, nm), dtype=np.uint64)
    for k, E in enumerate(w.energy):
        info = negf.negf_get_task_info(ctx, tables, k)
        b, s_, m_ = _expected_counts(w, E, p, N)
        basic[k] = b
        off, moff = info["table_offset"], info["mode_offset"]
        sc[:, off:off + s_.shape[1]] = s_
        md[:, moff:moff + m_.shape[1]] = m_
    negf.negf_tally_accumulate(ctx, tally, basic)
    negf.negf_tally_score_accumulate(ctx, tally, sc, md)
    return tally


def _check(got, ref, precision, scale, what):
    rel, floor = BARS[precision]
    err = np.abs(got - ref)
    bound = rel * np.abs(ref) + floor * scale
    worst = int(np.argmax(err - bound))
    assert np.all(err <= bound), (what, worst, got[worst], ref[worst], err.max() / scale)


def _wire(size):
    if size == "multi_tile":
        return inputs.small_wire(84, W=7, L=23, n_energy=2, eta=0.15, e_lo=-1.2, e_hi=0.9)
    if size == "w24":          # FP32: the CTA-wide chains of 16 < W <= 32
        return inputs.small_wire(86, W=24, L=9, n_energy=1, eta=0.08, e_lo=-0.7, e_hi=0.7)
    if size == "w64":          # FP32: the symmetric CTA-wide chain of W = 64
        return inputs.small_wire(87, W=64, L=12, n_energy=1, eta=0.05, disorder=0.5)
    return inputs.small_wire(81, W=3, L=5, n_energy=2, eta=0.2, e_lo=-1.0, e_hi=1.0)


@pytest.mark.parametrize("size", ["small", "multi_tile", "w24", "w64"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rgf_gradient_with_exact_tallies(ctx, precision, size):
    w = _wire(size)
    p = 0
    tables = negf.negf_build_tables(ctx, [w], precision=precision, keep_weights=True)
    tally = _exact_tally(ctx, tables, w, p)
    try:
        dV, dE, cap = negf.negf_current_backward_rgf(ctx, tables, tally, MU_P, MU_Q, KT, [1.0],
                                                     w.W * w.L)
        assert not cap
        gV, gE = _exact_grad(w, p)
        scale = max(np.abs(gV).max(), np.abs(gE).max())
        _check(dV, gV, precision, scale, "dV")
        _check(dE, gE, precision, scale, "deta")
    finally:
        negf.negf_tally_free(tally)
        negf.negf_tables_free(tables)


def test_rgf_equals_dense_adjoint_and_stride_invariant(ctx):
    w = _wire("multi_tile")
    p = 1
    t_dense = negf.negf_build_tables(ctx, [w], precision="fp64", keep_green=True)
    t_rgf = negf.negf_build_tables(ctx, [w], precision="fp64", keep_weights=True)
    tl_dense = _exact_tally(ctx, t_dense, w, p)
    tl_rgf = _exact_tally(ctx, t_rgf, w, p)
    try:
        ref = np.concatenate(negf.negf_current_backward(ctx, t_dense, tl_dense, MU_P, MU_Q, KT,
                                                        [2.5], w.W * w.L)[:2])
        scale = np.abs(ref).max()
        base = None
        for stride in (0, 1, 2, 3, 7, w.L, w.L + 4):
            dV, dE, cap = negf.negf_current_backward_rgf(ctx, t_rgf, tl_rgf, MU_P, MU_Q, KT,
                                                         [2.5], w.W * w.L, ckpt_stride=stride)
            assert not cap
            got = np.concatenate([dV, dE])
            assert np.max(np.abs(got - ref)) <= 1e-10 * scale, (stride, np.abs(got - ref).max())
            if base is None:
                base = got
            assert np.max(np.abs(got - base)) <= 1e-12 * scale, stride
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_current_backward_rgf(ctx, t_rgf, tl_rgf, MU_P, MU_Q, KT, [1.0], w.W * w.L,
                                           ckpt_stride=-1)
        # tables kept for the dense adjoint keep their weights too: both adjoints run on them
        dV, dE, _ = negf.negf_current_backward_rgf(ctx, t_dense, tl_dense, MU_P, MU_Q, KT,
                                                   [2.5], w.W * w.L)
        assert np.max(np.abs(np.concatenate([dV, dE]) - ref)) <= 1e-10 * scale
        t_plain = negf.negf_build_tables(ctx, [w], precision="fp64")
        tl_plain = negf.negf_walk_score(ctx, t_plain, p, 1, 10)
        try:
            with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
                negf.negf_current_backward_rgf(ctx, t_plain, tl_plain, MU_P, MU_Q, KT, [1.0],
                                               w.W * w.L)      # no keep_weights
        finally:
            negf.negf_tally_free(tl_plain)
            negf.negf_tables_free(t_plain)
    finally:
        negf.negf_tally_free(tl_dense)
        negf.negf_tally_free(tl_rgf)
        negf.negf_tables_free(t_dense)
        negf.negf_tables_free(t_rgf)


_W64 = {}


def _w64_reference():
    """The two-level W = 64 x L = 150 wire, its sampled sites and the oracle's derivative there
    (computed once for both precisions)."""
    if not _W64:
        w = inputs.small_wire(90, W=64, L=150, n_energy=1, eta=0.05, disorder=0.5)
        n = w.W * w.L
        rng = np.random.default_rng(3)
        sites = np.unique(np.concatenate([[0, 63, 64 * 75 + 31, n - 64, n - 1],
                                          rng.choice(n, size=3, replace=False)]))
        gV, gE = _exact_grad(w, 0, sites=sites)
        _W64.update(w=w, sites=sites, gV=gV[sites], gE=gE[sites],
                    counts=_expected_counts(w, float(w.energy[0]), 0, N_EXACT))
    return _W64


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rgf_gradient_two_level_w64(ctx, precision):
    ref = _w64_reference()
    w, sites = ref["w"], ref["sites"]
    tables = negf.negf_build_tables(ctx, [w], precision=precision, keep_weights=True,
                                    layout="two_level")
    tally = negf.negf_walk_score(ctx, tables, 0, 1, 0)
    try:
        info = negf.negf_get_task_info(ctx, tables, 0)
        assert info["layout"] == "two_level"
        ns = negf.load().negf_tally_score_size(tally)
        nm = negf.load().negf_tally_mode_size(tally)
        b, s_, m_ = ref["counts"]
        sc = np.zeros((2, ns), dtype=np.uint64)
        md = np.zeros((2, nm), dtype=np.uint64)
        sc[:, info["table_offset"]:info["table_offset"] + s_.shape[1]] = s_
        md[:, info["mode_offset"]:info["mode_offset"] + m_.shape[1]] = m_
        negf.negf_tally_accumulate(ctx, tally, b[None, :])
        negf.negf_tally_score_accumulate(ctx, tally, sc, md)
        dV, dE, cap = negf.negf_current_backward_rgf(ctx, tables, tally, MU_P, MU_Q, KT, [1.0],
                                                     w.W * w.L)
        assert not cap
        scale = max(np.abs(ref["gV"]).max(), np.abs(ref["gE"]).max())
        bar = "fp32_long" if precision == "fp32" else precision
        _check(dV[sites], ref["gV"], bar, scale, "dV")
        _check(dE[sites], ref["gE"], bar, scale, "deta")
    finally:
        negf.negf_tally_free(tally)
        negf.negf_tables_free(tables)


def test_two_level_score_walks(ctx):
    w = inputs.small_wire(85, W=4, L=6, n_energy=2, eta=0.25, e_lo=-0.8, e_hi=0.8)
    p = 0
    gV, gE = _exact_grad(w, p)
    g_exact = np.concatenate([gV, gE])
    rng = np.random.default_rng(7)
    dirs = [g_exact / np.linalg.norm(g_exact)] + [d / np.linalg.norm(d) for d in
                                                  rng.normal(size=(3, g_exact.size))]
    tables = negf.negf_build_tables(ctx, [w], precision="fp64", keep_weights=True,
                                    layout="two_level")
    try:
        est = []
        n_batch, N = 20, 200_000
        for b in range(n_batch):
            tally = negf.negf_walk_score(ctx, tables, p, 11, N, walker_id_offset=b * N)
            if b == 0:
                counts = negf.negf_tally_counts(ctx, tally, len(w.energy))
                sc, md = negf.negf_tally_score_counts(ctx, tally)
                for k in range(len(w.energy)):
                    info = negf.negf_get_task_info(ctx, tables, k)
                    rows, K = info["rows"], info["K"]
                    o, mo = info["table_offset"], info["mode_offset"]
                    assert int(sc[:, o:o + rows * K].sum()) == int(counts[k, 4])
                    assert int(md[:, mo:mo + 2 * w.W].sum()) == int(counts[k, 1] + counts[k, 2])
            dV, dE, cap = negf.negf_current_backward_rgf(ctx, tables, tally, MU_P, MU_Q, KT,
                                                         [1.0], w.W * w.L)
            negf.negf_tally_free(tally)
            assert not cap
            est.append(np.concatenate([dV, dE]))
        est = np.array(est)
        for d in dirs:
            proj = est @ d
            se = proj.std(ddof=1) / np.sqrt(len(proj))
            assert abs(proj.mean() - g_exact @ d) <= t_bar(len(dirs), n_batch - 1) * se + 1e-12, \
                (proj.mean(), g_exact @ d, se)
    finally:
        negf.negf_tables_free(tables)
