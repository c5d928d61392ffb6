"""GPU gradient of the Monte Carlo current (negf_walk_score + negf_current_backward) against
the oracle's exact FP64 derivative (pinned to finite differences of the direct probe solve).

* Deterministic: the score tallies are replaced by their exact expectations (N = 2^52 walkers'
  worth of counts, computed by the oracle from the absorbing chain; integers a double holds
  exactly, so that their rounding stays far below the bar), so the GPU result must
  equal the exact derivative: 1e-8 of the largest component in FP64, 1e-4 in FP32 (the bar
  for gradients against finite differences); a 15-site wire and a 161-site one whose
  adjoint product spans several tiles of the tensor-core kernel with ragged tails.
* Statistical: real walks; the gradient's projections on fixed directions must lie within the
  family-wise 3-SE bar of Student's t (mc_bars.t_bar; means of 20 batches over independent
  walker-id ranges, their standard error from the batches' spread) of the exact values.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import t_bar  # noqa: E402
from oracle import adjoint, current as ocur, markov, pipeline, wire  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402

MU_P, MU_Q, KT = 0.6, -0.4, 0.3


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    c = negf.negf_create(0)
    yield c
    negf.negf_destroy(c)


def _exact_grad(w, p):
    """dI/dV, dI/deta [L*W] of the wire's current (oracle, FP64)."""
    q = 1 - p
    gV = np.zeros(w.W * w.L)
    gE = np.zeros(w.W * w.L)
    df = ocur.fermi(w.energy, MU_P, KT) - ocur.fermi(w.energy, MU_Q, KT)
    for k, E in enumerate(w.energy):
        _, dV, dE = adjoint.transmission_gradient(w.onsite, w.eta, w.t, E, p, q)
        gV += w.energy_weight[k] * df[k] * dV.reshape(-1)
        gE += w.energy_weight[k] * df[k] * dE.reshape(-1)
    return gV, gE


def _expected_counts(w, E, p, N):
    """Exact expected tallies of N walks from lead p (oracle): (basic counts, score counts
    [2, rows*K], mode counts [2, 2W])."""
    r = pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)
    tab, n, W = r["tab"], r["n"], w.W
    P = tab["w"] / tab["w"].sum(1, keepdims=True)
    rows, K = P.shape
    Q = P[:n, :n]
    IQ = np.eye(n) - Q
    h = np.linalg.solve(IQ, P[:n, n:])                       # [n, 2] absorption from sites
    H = np.vstack([h, np.zeros((2 * W, 2))])                 # rows: sites then injection rows
    u = tab["mode_w"][p] / tab["mode_w"][p].sum()
    inj = slice(n + p * W, n + (p + 1) * W)
    nu = np.zeros(rows)
    nu[inj] = u
    nu[:n] = np.linalg.solve(IQ.T, P[inj, :n].T @ u)        # expected visits of each site
    score = np.zeros((2, rows, K))
    for rr in range(2):
        hb = np.concatenate([h[:, rr], [1.0 if rr == 0 else 0.0, 1.0 if rr == 1 else 0.0]])
        score[rr] = nu[:, None] * P * hb[None, :]
    v = P[inj, n:] + P[inj, :n] @ h                          # [W, 2]
    mode = np.zeros((2, 2 * W))
    for rr in range(2):
        mode[rr, p * W:(p + 1) * W] = u * v[:, rr]
    Pr = u @ v
    counts = np.array([N, N * Pr[0], N * Pr[1], 0, 0], dtype=np.float64)
    return (np.rint(counts).astype(np.uint64), np.rint(N * score.reshape(2, -1)).astype(np.uint64),
            np.rint(N * mode).astype(np.uint64))


def _exact_tally_wire(size):
    if size == "wide":
        # W > 32: the start lead's mode seeds take two per lane of the seeds kernel
        return inputs.small_wire(88, W=40, L=5, n_energy=1, eta=0.1, disorder=0.7)
    if size == "multi_tile":
        # n = 161 sites: the adjoint's dense product spans two row tiles, three column tiles
        # and eleven k stages of the tensor-core kernel, each with a ragged tail
        return inputs.small_wire(84, W=7, L=23, n_energy=2, eta=0.15, e_lo=-1.2, e_hi=0.9)
    return inputs.small_wire(81, W=3, L=5, n_energy=2, eta=0.2, e_lo=-1.0, e_hi=1.0)


@pytest.mark.parametrize("size", ["small", "multi_tile", "wide"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-4)])
def test_gradient_with_exact_tallies(ctx, precision, tol, size):
    w = _exact_tally_wire(size)
    p, N = 0, float(2 ** 52)
    tables = negf.negf_build_tables(ctx, [w], precision=precision, keep_green=True)
    tally = negf.negf_walk_score(ctx, tables, p, 1, 0)      # allocated, all counts zero
    try:
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
        dV, dE, cap = negf.negf_current_backward(ctx, tables, tally, MU_P, MU_Q, KT, [1.0],
                                                 w.W * w.L)
        gV, gE = _exact_grad(w, p)
        scale = max(np.abs(gV).max(), np.abs(gE).max())
        assert not cap
        assert np.max(np.abs(dV - gV)) <= tol * scale, (dV, gV)
        assert np.max(np.abs(dE - gE)) <= tol * scale, (dE, gE)
    finally:
        negf.negf_tally_free(tally)
        negf.negf_tables_free(tables)


def test_gradient_from_walks_is_unbiased(ctx):
    w = inputs.small_wire(82, W=2, L=4, n_energy=2, eta=0.3, e_lo=-0.8, e_hi=0.8)
    p = 0
    gV, gE = _exact_grad(w, p)
    g_exact = np.concatenate([gV, gE])
    rng = np.random.default_rng(5)
    dirs = [g_exact / np.linalg.norm(g_exact)] + [d / np.linalg.norm(d) for d in
                                                  rng.normal(size=(3, g_exact.size))]
    tables = negf.negf_build_tables(ctx, [w], precision="fp64", keep_green=True)
    try:
        est = []
        n_batch = 20
        for b in range(n_batch):
            tally = negf.negf_walk_score(ctx, tables, p, 7, 200_000, walker_id_offset=b * 200_000)
            dV, dE, cap = negf.negf_current_backward(ctx, tables, tally, MU_P, MU_Q, KT, [1.0],
                                                     w.W * w.L)
            negf.negf_tally_free(tally)
            assert not cap
            est.append(np.concatenate([dV, dE]))
        est = np.array(est)
        for d in dirs:
            proj = est @ d
            se = proj.std(ddof=1) / np.sqrt(len(proj))
            # batch means with their sample spread: Student t, n_batch - 1 degrees of freedom
            assert abs(proj.mean() - g_exact @ d) <= t_bar(len(dirs), n_batch - 1) * se + 1e-12, \
                (proj.mean(), g_exact @ d, se)
    finally:
        negf.negf_tables_free(tables)


@pytest.mark.parametrize("adjoint_kind", ["rgf", "dense"])
def test_autograd_function_matches_abi(ctx, adjoint_kind):
    """NegfCurrent (torch.autograd.Function) makes exactly the C-ABI calls: same current, same
    gradient as negf_build_tables + negf_walk_score + negf_current + negf_current_backward_rgf
    (default) or negf_current_backward (dense G)."""
    from paper_1805_10164_gb300 import autograd as nag
    w = inputs.small_wire(83, W=3, L=5, n_energy=2, eta=0.2, e_lo=-1.0, e_hi=1.0)
    dense = adjoint_kind == "dense"
    spec = nag.CurrentSpec(W=w.W, L=w.L, t=w.t, energy=w.energy, energy_weight=w.energy_weight,
                           mu_p=MU_P, mu_q=MU_Q, kT=KT, walkers_per_task=100_000, seed=9,
                           precision="fp64", adjoint=adjoint_kind, ckpt_stride=2)
    V = torch.tensor(w.onsite, device="cuda", requires_grad=True)
    eta = torch.tensor(w.eta, device="cuda", requires_grad=True)
    I, se = nag.current(V, eta, ctx, spec)
    (3.0 * I).backward()
    tables = negf.negf_build_tables(ctx, [w], precision="fp64", keep_green=dense,
                                    keep_weights=not dense)
    tally = negf.negf_walk_score(ctx, tables, 0, 9, 100_000)
    try:
        res = negf.negf_current(ctx, tables, tally, MU_P, MU_Q, KT)
        if dense:
            dV, dE, cap = negf.negf_current_backward(ctx, tables, tally, MU_P, MU_Q, KT, [3.0],
                                                     w.W * w.L)
        else:
            dV, dE, cap = negf.negf_current_backward_rgf(ctx, tables, tally, MU_P, MU_Q, KT,
                                                         [3.0], w.W * w.L, ckpt_stride=2)
    finally:
        negf.negf_tally_free(tally)
        negf.negf_tables_free(tables)
    assert not cap
    assert I.item() == res["I"][0] and se.item() == res["se"][0]
    # the block-column adjoint sums with FP64 atomics: equal up to the order of those sums
    tol = 1e-12 * max(np.abs(dV).max(), np.abs(dE).max())
    np.testing.assert_allclose(V.grad.cpu().numpy().reshape(-1), dV, rtol=1e-12, atol=tol)
    np.testing.assert_allclose(eta.grad.cpu().numpy().reshape(-1), dE, rtol=1e-12, atol=tol)
    # without a gradient the plain walk runs: same walks, same current
    with torch.no_grad():
        I2, _ = nag.current(V, eta, ctx, spec)
    assert I2.item() == I.item()
