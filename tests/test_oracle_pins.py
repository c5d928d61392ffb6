"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics, independent
of the oracle itself (closed forms, identities between independent routes, brute force, an
independent implementation of the RNG).  CPU only."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from mc_bars import z_bar
from oracle import alias, buttiker, current, markov, neumann, philox, pipeline, walker, wire

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _wire(seed, W, L, eta, disorder=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-disorder, disorder, (L, W)), np.full((L, W), float(eta))


# ---------------------------------------------------------------- lead self-energies, G^r

@pytest.mark.parametrize("e", [-3.0, -2.5, -1.2, 0.0, 0.7, 1.99, 2.4, 5.0])
def test_surface_green_function_solves_dyson(e):
    """g_s of a semi-infinite chain satisfies g = 1/(e - t^2 g) (removing one site leaves the
    same chain) on the retarded branch: Im g <= 0 in band, |g| < 1/t outside."""
    t = 1.3
    s, gam = wire.chain_surface_self_energy(e, t)
    g = s / t**2
    assert abs(g - 1.0 / (e - t**2 * g)) < 1e-12
    if abs(e) < 2 * t:
        assert g.imag < 0 and gam > 0
    else:
        assert abs(g) < 1.0 / t and gam == 0.0


def test_surface_green_function_matches_long_finite_chain():
    """Brute force: the corner element of (E + i delta - H_chain)^{-1} for a long chain with a
    small damping approaches the surface Green's function."""
    t, e, N, delta = 1.0, 0.6, 3000, 2e-3
    H = np.diag(np.full(N - 1, -t), 1)
    H = H + H.T
    g_fin = np.linalg.solve((e + 1j * delta) * np.eye(N) - H, np.eye(N)[:, 0])[0]
    s, _ = wire.chain_surface_self_energy(e, t)
    assert abs(g_fin - s / t**2) < 5e-3


def test_transverse_modes_diagonalise_the_slice():
    W, t = 7, 1.4
    phi, eps = wire.transverse_modes(W, t)
    Hs = np.diag(np.full(W - 1, -t), 1)
    Hs = Hs + Hs.T
    assert np.allclose(phi.T @ phi, np.eye(W), atol=1e-13)
    assert np.allclose(phi.T @ Hs @ phi, np.diag(eps), atol=1e-13)


def test_two_site_chain_cramer():
    """W=1, L=2: the 2x2 inverse by Cramer's rule (independent of the LU solve)."""
    V1, V2, eta, E, t = 0.3, -0.2, 0.15, 0.4, 1.0
    s, _ = wire.chain_surface_self_energy(E, t)
    a = E - V1 - s + 0.5j * eta
    d = E - V2 - s + 0.5j * eta
    b = t                                    # E - H has +t off the diagonal (H_12 = -t)
    det = a * d - b * b
    G_ref = np.array([[d, -b], [-b, a]]) / det
    g = wire.green_retarded(E, [[V1], [V2]], [[eta], [eta]], t)
    assert np.allclose(g["G"], G_ref, atol=1e-14)


@pytest.mark.parametrize("E,expect", [(0.5, 1.0), (-1.9, 1.0), (1.2, 1.0), (2.1, 0.0), (-3.0, 0.0)])
def test_clean_chain_ballistic(E, expect):
    """Clean 1D chain without dephasing: T = 1 inside the band |E| < 2t, 0 outside."""
    L = 9
    r = pipeline.task_reference(np.zeros((L, 1)), np.zeros((L, 1)), 1.0, E)
    assert abs(r["T_direct"][1, 0] - expect) < 1e-10
    assert abs(r["exact"]["T_eff"][1, 0] - expect) < 1e-10


@pytest.mark.parametrize("E", [-3.3, -2.05, -0.4, 0.9, 2.7, 3.9])
def test_clean_strip_channel_staircase(E):
    """Clean W-wide strip without dephasing: T = number of open transverse channels."""
    W, L, t = 5, 6, 1.0
    _, eps = wire.transverse_modes(W, t)
    n_open = int(np.sum(np.abs(E - eps) < 2 * t))
    r = pipeline.task_reference(np.zeros((L, W)), np.zeros((L, W)), t, E)
    assert abs(r["T_direct"][1, 0] - n_open) < 1e-9
    assert abs(r["exact"]["T_eff"][1, 0] - n_open) < 1e-9


# ---------------------------------------------------------------- identities

@pytest.mark.parametrize("seed,W,L,eta,E,lm", [(0, 1, 20, 0.1, 0.5, 0), (1, 3, 7, 0.1, 0.3, 0),
                                               (2, 4, 9, 0.3, -1.7, 0), (3, 2, 5, 0.05, 2.6, 0),
                                               (4, 3, 6, 0.2, 0.4, 1)])
def test_three_routes_agree(seed, W, L, eta, E, lm):
    """Probe solve (Eq. buteq), the Neumann series (Eq. iqof_t_el_db) and the absorbing-chain
    expectation of the Step 6' walk give the same T^eff (Appendix B identity)."""
    on, et = _wire(seed, W, L, eta)
    r = pipeline.task_reference(on, et, 1.0, E, lead_model=lm, gamma_lead=0.7)
    Td = r["T_direct"]
    Tx = r["exact"]["T_eff"]
    for q in range(2):
        for p in range(2):
            Tn = neumann.neumann_transmission(r["g"], q, p)
            assert abs(Td[q, p] - Tx[q, p]) <= 1e-10 * abs(Td[q, p]) + 1e-13
            assert abs(Tn - Td[q, p]) <= 1e-9 * abs(Td[q, p]) + 1e-13


def test_symmetry_sum_rule_reciprocity_conservation():
    on, et = _wire(7, 4, 8, 0.12)
    r = pipeline.task_reference(on, et, 1.0, -0.8)
    G = r["g"]["G"]
    assert np.allclose(G, G.T, atol=1e-13)                            # real H, symmetric Sigma
    tab = r["tab"]
    assert np.allclose(tab["w"].sum(1), tab["A_row"], rtol=1e-12)    # A = G Gamma G^dag
    assert np.all(tab["w"] >= 0)
    T = r["exact"]["T_eff"]
    assert abs(T[1, 0] - T[0, 1]) < 1e-11 * T[1, 0]                   # reciprocity
    P = r["exact"]["P_inj"]
    assert np.allclose(P.sum(1), 1.0, atol=1e-12)                     # absorbed somewhere
    assert np.allclose(T[:, 0].sum(), tab["c"][0], rtol=1e-12)
    # c_p = Tr Gamma_p A equals the sum of the mode weights lambda_m <phi_m|A|phi_m>
    assert np.allclose(tab["mode_w"].sum(1), tab["c"], rtol=1e-12)


def test_probe_current_conservation():
    """With the probe occupations solved, every probe's net current vanishes and the two lead
    currents cancel (charge conservation, Appendix on assumption (iv))."""
    on, et = _wire(8, 3, 6, 0.2)
    g = wire.green_retarded(0.2, on, et, 1.0)
    probes, x, (T_PP, T_Pq, T_qP, T_qp) = buttiker.probe_occupations(g, [1.0, 0.0])
    f_lead = np.array([1.0, 0.0])
    A = -2 * np.imag(np.diag(g["G"]))[probes]
    gam = g["gamma"][probes]
    net_probe = gam * A * x - T_PP @ x - T_Pq @ f_lead
    assert np.max(np.abs(net_probe)) < 1e-12
    tot_q = T_qP.sum(1) + T_qp.sum(1)                    # sum_b T_qb
    I = np.array([T_qP[q] @ x + T_qp[q] @ f_lead - tot_q[q] * f_lead[q] for q in range(2)])
    assert abs(I[0] + I[1]) < 1e-11


def test_ohmic_resistance_linear_in_length():
    """Strong dephasing makes transport diffusive: 1/T^eff = A + L/lambda (Sec. IV.B.2), with
    the mean free path shrinking as the dephasing grows."""
    Ls = np.arange(10, 101, 10)
    slopes = []
    for eta in (0.5, 1.0):
        R = []
        for L in Ls:
            g = wire.green_retarded(0.3, np.zeros((L, 1)), np.full((L, 1), eta), 1.0)
            R.append(1.0 / buttiker.effective_transmission(g)[1, 0])
        R = np.array(R)
        c = np.polyfit(Ls, R, 1)
        fit = np.polyval(c, Ls)
        r2 = 1 - np.sum((R - fit) ** 2) / np.sum((R - R.mean()) ** 2)
        assert r2 > 0.9999
        slopes.append(c[0])
    assert 1.6 < slopes[1] / slopes[0] < 2.4


# ---------------------------------------------------------------- alias tables

@pytest.mark.parametrize("w", [[1.0], [0.0, 3.0], [1, 1, 1, 1, 1], [5, 0, 0, 1e-9, 2.5],
                               list(np.random.default_rng(1).exponential(size=37)),
                               list(np.random.default_rng(2).uniform(size=502) ** 6)])
def test_vose_implied_distribution(w):
    w = np.asarray(w, dtype=np.float64)
    e = alias.vose(w)
    p = alias.implied_distribution(e)
    K = w.size
    assert np.max(np.abs(p - w / w.sum())) <= (K + 2) / 2**32
    thr, ali = alias.split(e)
    assert np.all(ali[thr == 2**32 - 1] == np.arange(K)[thr == 2**32 - 1])   # full slots
    assert np.all(p[w == 0] == 0.0)                                         # never drawn


def test_alias_slot_mass_is_exact():
    for K in (1, 2, 3, 7, 502, 2**20 + 3):
        m = alias.slot_mass(K) if K < 10000 else None
        if m is not None:
            assert sum(m) == 2**32 and max(m) - min(m) <= 1
    # brute force on a tiny "2^32": the same formula with 2^8 counts (x*K)>>8
    for K in (3, 5, 7):
        counts = np.bincount([(x * K) >> 8 for x in range(256)], minlength=K)
        ref = [(-(-((c + 1) * 256) // K)) - (-(-(c * 256) // K)) for c in range(K)]
        assert list(counts) == ref


def test_alias_detects_planted_mistake():
    """A wrong threshold anywhere in a row moves the implied distribution past the bound."""
    w = np.random.default_rng(3).exponential(size=40)
    e = alias.vose(w).copy()
    thr, ali = alias.split(e)
    c = int(np.argmax((thr > 2**30) & (ali != np.arange(40))))
    e[c] = np.uint64(thr[c] // 2) | (np.uint64(ali[c]) << np.uint64(32))
    p = alias.implied_distribution(e)
    assert np.max(np.abs(p - w / w.sum())) > 1e-4


# ---------------------------------------------------------------- Philox

_TRITON_CHECK = textwrap.dedent("""
    import numpy as np, torch, triton, triton.language as tl, sys
    sys.path.insert(0, %r)
    from oracle.philox import philox4x32_10
    @triton.jit
    def k(c0p, c1p, c2p, c3p, o0, o1, o2, o3, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i),
                               tl.load(c3p + i))
        tl.store(o0 + i, a); tl.store(o1 + i, b); tl.store(o2 + i, c); tl.store(o3 + i, d)
    N = 64
    rng = np.random.default_rng(11)
    cs = [rng.integers(0, 2**32, N, dtype=np.uint64).astype(np.uint32) for _ in range(4)]
    cs[0][:4] = 0; cs[1][:4] = [0, 1, 0xFFFFFFFF, 7]
    for seed in (0, 1, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF):
        outs = [torch.empty(N, dtype=torch.int32) for _ in range(4)]
        k[(1,)](*[torch.from_numpy(c.view(np.int32).copy()) for c in cs], *outs, seed, N=N)
        ref = philox4x32_10(*cs, seed & 0xFFFFFFFF, seed >> 32)
        for o, r in zip(outs, ref):
            assert np.array_equal(o.numpy().view(np.uint32), r), seed
    print("OK")
""")


def test_philox_matches_independent_implementation():
    """Triton ships its own Philox4x32-10 (Python source, run here by Triton's CPU
    interpreter); the oracle's words must agree bit for bit."""
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, "-c", _TRITON_CHECK % ROOT], env=env,
                         capture_output=True, text=True, timeout=600)
    if "OK" not in res.stdout:
        if "No module named" in res.stderr or "interpret" in res.stderr.lower():
            pytest.skip("triton interpreter unavailable: " + res.stderr[-200:])
        raise AssertionError(res.stdout + res.stderr)


def test_philox_uniformity():
    x0, x1, x2, x3 = philox.philox4x32_10(np.zeros(1 << 16), np.arange(1 << 16), 0, 5, 9, 3)
    for x in (x0, x1, x2, x3):
        h = np.bincount(x >> np.uint32(28), minlength=16)
        chi2 = np.sum((h - 4096.0) ** 2 / 4096.0)
        assert chi2 < 45.0                   # 15 dof, p ~ 1e-4


# ---------------------------------------------------------------- walker

def test_walker_statistics_match_exact_chain():
    on, et = _wire(5, 3, 8, 0.15)
    r = pipeline.task_reference(on, et, 1.0, 0.45)
    N = 60000
    lead, steps = walker.walk(r["entries"], r["mode_entries"], r["n"], r["W"], r["c_open"],
                              task=3, start_lead=0, seed=1234, wids=np.arange(N), max_steps=10**6)
    assert np.all(lead >= 0)
    P = r["exact"]["P_inj"][0, 1]
    Phat = np.mean(lead == 1)
    assert abs(Phat - P) < z_bar(2) * np.sqrt(P * (1 - P) / N)
    m = r["exact"]["steps_inj"][0]
    var = r["exact"]["steps2_inj"][0] - m * m
    assert abs(steps.mean() - m) < z_bar(2) * np.sqrt(var / N)
    assert abs(steps.var() / var - 1.0) < 0.1


@pytest.mark.parametrize("L,W", [(5, 4), (3, 13), (2, 64)])
def test_two_level_tables_realise_the_weights(L, W):
    """Level 1 over slice totals and leads, level 2 the inverse-CDF draw within a slice (a
    guide for W > 8): the product of the exact implied distributions equals weights / row sum
    (an empty slice, zero weights inside a slice and at its end, a row without lead weight)."""
    rng = np.random.default_rng(31 + W)
    w = rng.exponential(size=(6, L * W + 2))
    w[1, W:2 * W] = 0.0                           # an empty slice
    w[2, L * W:] = 0.0                            # no lead weight
    w[3, 1:W:3] = 0.0                             # zeros inside slice 0
    w[4, W - 2:W] = 0.0                           # zeros at the end of slice 0
    l1, l2 = alias.build_two_level(w, L, W)
    assert l1.shape == (6, L + 2) and l2.shape == (6, L, alias.level2_words(W))
    assert l2.dtype == np.uint32
    for i in range(6):
        p = alias.implied_two_level(l1[i], l2[i], W)
        assert np.max(np.abs(p - w[i] / w[i].sum())) <= (L + W + 4) * 2.0**-32
        assert np.all(p[:L * W][w[i, :L * W] == 0] == 0.0)    # zero weight: never drawn


@pytest.mark.parametrize("W", [1, 5, 8, 9, 16, 31, 64])
def test_level2_guided_draw_is_the_inverse_cdf(W):
    """The two-stage draw (guide, then octet) equals the plain inverse-CDF count
    #{a < W - 1 : c_a <= v} of Sec. III.B's draw, for every v at and around each threshold."""
    rng = np.random.default_rng(W)
    wk = rng.exponential(size=W) * (rng.random(W) < 0.7)
    wk[0] += 0.1
    blk = alias.cdf_block(wk)
    G = -(-W // 8)
    c = blk.astype(np.int64)[8:] if G > 1 else blk.astype(np.int64)
    v = np.unique(np.clip(np.concatenate([c[:W - 1] + d for d in (-1, 0, 1)]
                                         + [rng.integers(0, 2**31, size=200), [0, 2**31 - 1]]),
                          0, 2**31 - 1))
    plain = (c[None, :W - 1] <= v[:, None]).sum(1)
    assert np.array_equal(alias.draw_level2(np.broadcast_to(blk, (v.size, blk.size)), W, v), plain)


def test_level2_planted_mistakes_are_caught():
    """A wrong guide word or a shifted threshold changes the realised distribution beyond the
    quantisation bound, so the implied-distribution check catches it."""
    rng = np.random.default_rng(7)
    W = 40
    wk = rng.exponential(size=W)
    blk = alias.cdf_block(wk)
    ok = alias.implied_level2(blk, W)
    assert np.max(np.abs(ok - wk / wk.sum())) <= 2.0**-30
    bad = blk.copy()
    bad[1] = bad[0]                               # guide of octet 1 replaced by octet 0's
    assert np.max(np.abs(alias.implied_level2(bad, W) - wk / wk.sum())) > 1e-3
    bad = blk.copy()
    bad[8 + 3:8 + 8] = bad[8 + 4:8 + 9]           # thresholds shifted by one site
    assert np.max(np.abs(alias.implied_level2(bad, W) - wk / wk.sum())) > 1e-3


def test_two_level_walker_statistics_match_exact_chain():
    on, et = _wire(5, 3, 8, 0.15)
    r = pipeline.task_reference(on, et, 1.0, 0.45)
    l1, l2 = alias.build_two_level(r["tab"]["w"], 8, 3)
    N = 60000
    lead, steps = walker.walk_two_level(l1, l2, r["mode_entries"], r["n"], 8, 3, r["c_open"],
                                        task=3, start_lead=0, seed=1234, wids=np.arange(N),
                                        max_steps=10**6)
    assert np.all(lead >= 0)
    P = r["exact"]["P_inj"][0, 1]
    assert abs(np.mean(lead == 1) - P) < z_bar(2) * np.sqrt(P * (1 - P) / N)
    m = r["exact"]["steps_inj"][0]
    var = r["exact"]["steps2_inj"][0] - m * m
    assert abs(steps.mean() - m) < z_bar(2) * np.sqrt(var / N)
    # truncation as in the one-level walker
    lead2, steps2 = walker.walk_two_level(l1, l2, r["mode_entries"], r["n"], 8, 3, r["c_open"],
                                          3, 0, 1234, np.arange(2000), 2)
    assert np.all((lead2 >= 0) | ((lead2 == -2) & (steps2 == 2)))
    assert np.array_equal(lead2 >= 0, steps[:2000] <= 2)


@pytest.mark.parametrize("seed,W,L,E,lm", [(41, 3, 6, 0.3, 0), (42, 1, 9, -1.1, 0), (43, 4, 3, 0.8, 1)])
def test_sparse_column_rows_match_dense(seed, W, L, E, lm):
    """Sampled table rows from sparse LU column solves equal the dense transition weights."""
    from oracle import columns
    rng = np.random.default_rng(seed)
    on = rng.uniform(-1, 1, (L, W))
    et = rng.uniform(0.02, 0.3, (L, W))
    g = wire.green_retarded(E, on, et, 1.0, lm, 0.7)
    tab = markov.transition_weights(g, wire.lead_modes(E, W, 1.0, lm, 0.7)[0::2])
    n = L * W
    rows = np.array([0, n // 2, n - 1, n, n + W - 1, n + W, n + 2 * W - 1])
    got = columns.sampled_rows(E, on, et, 1.0, rows, lm, 0.7)
    scale = tab["w"].sum(1).max()
    assert np.allclose(got["w"], tab["w"][rows], rtol=1e-10, atol=1e-13 * scale)
    assert np.allclose(got["A_row"], tab["A_row"][rows], rtol=1e-10, atol=1e-13 * scale)
    assert np.allclose(got["mode_w"], tab["mode_w"], rtol=1e-10, atol=1e-13 * scale)
    assert np.allclose(got["c"], tab["c"], rtol=1e-10, atol=1e-13 * scale)


def test_step_moments_brute_force():
    """Second moment of the number of steps: the fundamental-matrix identity against direct
    iteration of the chain's step distribution P(S = k) on a small wire."""
    on, et = _wire(12, 2, 4, 0.6)
    r = pipeline.task_reference(on, et, 1.0, 0.2, with_alias=False)
    tab, ex = r["tab"], r["exact"]
    n, W = r["n"], r["W"]
    P = tab["w"] / tab["w"].sum(1, keepdims=True)
    u = tab["mode_w"][0] / tab["mode_w"][0].sum()
    dist = u @ P[n:n + W]                     # state after draw 1 (sites then leads)
    alive = dist[:n].copy()
    m1 = m2 = 0.0
    k = 1
    absorbed = dist[n:].sum()
    m1 += k * absorbed
    m2 += k * k * absorbed
    while alive.sum() > 1e-16 and k < 100000:
        k += 1
        nxt = alive @ P[:n]
        absorbed = nxt[n:].sum()
        m1 += k * absorbed
        m2 += k * k * absorbed
        alive = nxt[:n]
    assert abs(m1 - ex["steps_inj"][0]) < 1e-10 * m1
    assert abs(m2 - ex["steps2_inj"][0]) < 1e-10 * m2


def test_walker_reproducible_and_truncation():
    on, et = _wire(6, 2, 10, 0.5)
    r = pipeline.task_reference(on, et, 1.0, -0.3)
    ids = np.arange(5000, 7000)
    a = walker.walk(r["entries"], r["mode_entries"], r["n"], r["W"], r["c_open"], 0, 1, 77, ids, 1000)
    b = walker.walk(r["entries"], r["mode_entries"], r["n"], r["W"], r["c_open"], 0, 1, 77, ids[::-1], 1000)
    assert np.array_equal(a[0], b[0][::-1]) and np.array_equal(a[1], b[1][::-1])
    lead, steps = walker.walk(r["entries"], r["mode_entries"], r["n"], r["W"], r["c_open"], 0, 1,
                              77, ids, 2)
    assert np.all((lead >= 0) | ((lead == -2) & (steps == 2)))
    assert np.all(steps <= 2)
    assert np.array_equal(lead >= 0, (a[1] <= 2))


@pytest.mark.parametrize("two_level", [False, True])
def test_walker_path_is_the_walk(two_level):
    """The recorded path is the walk itself: one transition per step, the first row the
    injection row of the drawn mode, each later row the previous column, the last column of an
    absorbed walk its lead, and the empirical transition frequencies out of a row those of the
    row's weights."""
    on, et = _wire(6, 2, 10, 0.5)
    r = pipeline.task_reference(on, et, 1.0, -0.3)
    n, W = r["n"], r["W"]
    ids = np.arange(3000)
    path = {}
    if two_level:
        l1, l2 = alias.build_two_level(r["tab"]["w"], 10, 2)
        lead, steps = walker.walk_two_level(l1, l2, r["mode_entries"], n, 10, W, r["c_open"], 5,
                                            1, 77, ids, 10**6, path=path)
    else:
        lead, steps = walker.walk(r["entries"], r["mode_entries"], n, W, r["c_open"], 5, 1, 77,
                                  ids, 10**6, path=path)
    assert np.all(lead >= 0)
    seen = np.zeros(ids.size, dtype=np.int64)
    cur = n + 1 * W + path["mode"]
    counts = np.zeros_like(r["tab"]["w"])
    for idx, row, col in path["steps"]:
        assert np.array_equal(row, cur[idx])
        seen[idx] += 1
        cur[idx] = col
        np.add.at(counts, (row, col), 1.0)
    assert np.array_equal(seen, steps.astype(np.int64))
    assert np.array_equal(cur - n, lead)
    P = r["tab"]["w"] / r["tab"]["w"].sum(1, keepdims=True)
    busy = counts.sum(1) > 2000
    assert busy.any()
    emp = counts[busy] / counts[busy].sum(1, keepdims=True)
    assert np.max(np.abs(emp - P[busy])) < 6 * np.sqrt(0.25 / 2000)


def test_walker_closed_lead():
    """Energy outside the lead band: no open channel, nothing is injected."""
    r = pipeline.task_reference(np.zeros((6, 1)), np.full((6, 1), 0.1), 1.0, 2.5)
    assert not r["c_open"][0]
    lead, steps = walker.walk(r["entries"], r["mode_entries"], r["n"], r["W"], r["c_open"], 0, 0,
                              1, np.arange(10), 100)
    assert np.all(lead == -1) and np.all(steps == 0)


def test_binomial_standard_error_is_honest():
    """The binomial SE of Sec. IV.B.2 matches the spread of independent estimates."""
    on, et = _wire(9, 2, 6, 0.2)
    r = pipeline.task_reference(on, et, 1.0, 0.1)
    c = r["tab"]["c"][0]
    est, ses = [], []
    for b in range(40):
        lead, _ = walker.walk(r["entries"], r["mode_entries"], r["n"], r["W"], r["c_open"], 0, 0,
                              99, np.arange(b * 1500, (b + 1) * 1500), 10**5)
        T, se = current.mc_transmission(c, np.sum(lead == 1), lead.size)
        est.append(T)
        ses.append(se)
    ratio = np.std(est, ddof=1) / np.mean(ses)
    assert 0.7 < ratio < 1.35


def test_fermi_and_current():
    E = np.linspace(-1, 1, 11)
    f = current.fermi(E, 0.2, 0.05)
    assert abs(current.fermi(0.2, 0.2, 0.05) - 0.5) < 1e-15
    assert np.allclose(current.fermi(0.2 + E, 0.2, 0.05) + current.fermi(0.2 - E, 0.2, 0.05), 1.0)
    assert np.allclose(f, 1 / (1 + np.exp((E - 0.2) / 0.05)))
    I, dI = current.current(E, np.full(11, 0.2), np.ones(11), np.zeros(11), 0.5, -0.5, 1e-3)
    assert abs(I - 0.2 * np.sum(np.abs(E) < 0.5) - 0.2 * 0.5 * 2 * 0) < 0.2 + 1e-12 and dI == 0


def test_current_integrates_to_the_bias():
    """With T = 1 at every energy the current is the integral of f_p - f_q, which equals
    mu_p - mu_q exactly (Landauer: one open channel carries the bias window); a sharp window
    with T = 0.2 inside it gives 0.2 per grid weight inside."""
    h = 1e-3
    E = np.arange(-6.0 + h / 2, 6.0, h)
    for mu_p, mu_q, kT in ((0.3, -0.1, 0.05), (-0.2, 0.45, 0.1), (0.0, 0.0, 0.02)):
        I, dI = current.current(E, np.full(E.size, h), np.ones(E.size), np.zeros(E.size),
                                mu_p, mu_q, kT)
        assert abs(I - (mu_p - mu_q)) < 1e-9, (mu_p, mu_q, I)
        assert dI == 0.0
    Eg = np.linspace(-1, 1, 11)
    I, _ = current.current(Eg, np.full(11, 0.2), np.ones(11), np.zeros(11), 0.5, -0.5, 1e-3)
    assert abs(I - 0.2 * 5) < 1e-12


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_a_dropped_scattering_term(monkeypatch):
    """Plant a mistake in the oracle (drop Sigma_s from G): the sum-rule pin must fail."""
    orig = wire.green_retarded

    def broken(E, onsite, eta, t, lead_model=0, gamma_lead=0.0, slice_h=None):
        g = orig(E, onsite, np.zeros_like(np.asarray(eta)), t, lead_model, gamma_lead, slice_h)
        g["gamma"] = np.asarray(eta, dtype=np.float64).reshape(-1)
        return g

    monkeypatch.setattr(wire, "green_retarded", broken)
    on, et = _wire(10, 3, 5, 0.2)
    r = pipeline.task_reference(on, et, 1.0, 0.3, with_alias=False)
    tab = r["tab"]
    assert not np.allclose(tab["w"].sum(1), tab["A_row"], rtol=1e-6)


def test_pins_catch_a_wrong_lead_sign(monkeypatch):
    """Plant an advanced (wrong-branch) lead self-energy: the clean-chain pin must fail."""
    orig = wire.chain_surface_self_energy

    def broken(e, t):
        s, gam = orig(e, t)
        return np.conj(s), gam

    monkeypatch.setattr(wire, "chain_surface_self_energy", broken)
    # the retarded-branch pin fails ...
    s, _ = wire.chain_surface_self_energy(0.5, 1.0)
    assert not s.imag < 0
    # ... and so does the sum rule once dephasing mixes with the lead self-energy
    on, et = _wire(11, 1, 9, 0.1)
    r = pipeline.task_reference(on, et, 1.0, 0.5, with_alias=False)
    tab = r["tab"]
    assert not np.allclose(tab["w"].sum(1), tab["A_row"], rtol=1e-6)


def _vary_eta(seed, W, L):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (L, W)), rng.uniform(0.05, 0.4, (L, W))


def test_pins_catch_transposed_site_weights(monkeypatch):
    """Plant gamma_i |G_ij|^2 in place of gamma_j |G_ji|^2 (source and destination swapped):
    the walk's exact expectation must leave the direct probe solve."""
    orig = markov.transition_weights

    def broken(g, modes):
        tab = orig(g, modes)
        n = tab["n"]
        tab["w"][:n, :n] = np.abs(g["G"]) ** 2 * g["gamma"][:, None]
        return tab

    on, et = _vary_eta(12, 2, 5)
    good = pipeline.task_reference(on, et, 1.0, 0.4, with_alias=False)
    assert abs(good["exact"]["T_eff"][1, 0] - good["T_direct"][1, 0]) <= 1e-10
    monkeypatch.setattr(markov, "transition_weights", broken)
    r = pipeline.task_reference(on, et, 1.0, 0.4, with_alias=False)
    assert abs(r["exact"]["T_eff"][1, 0] - r["T_direct"][1, 0]) > 1e-4 * r["T_direct"][1, 0]


def test_pins_catch_a_dropped_self_transition(monkeypatch):
    """Plant j != i in the Step 6' sum (drop the self-transition): the row-sum pin fails."""
    orig = markov.transition_weights

    def broken(g, modes):
        tab = orig(g, modes)
        n = tab["n"]
        tab["w"][np.arange(n), np.arange(n)] = 0.0
        return tab

    monkeypatch.setattr(markov, "transition_weights", broken)
    on, et = _vary_eta(13, 2, 4)
    r = pipeline.task_reference(on, et, 1.0, -0.6, with_alias=False)
    tab = r["tab"]
    assert not np.allclose(tab["w"].sum(1), tab["A_row"], rtol=1e-6)


# ---------------------------------------------------------------- gradients

@pytest.mark.parametrize("seed,W,L,E,lm", [(21, 3, 5, 0.4, 0), (22, 1, 8, -0.7, 0), (23, 2, 4, 1.1, 1)])
def test_gradient_matches_finite_differences_of_direct_solve(seed, W, L, E, lm):
    """The FP64 tangent of T_qp (through the walk's absorbing chain) against central
    differences (h = 1e-5) of the direct probe solve, an independent route to T."""
    from oracle import adjoint
    rng = np.random.default_rng(seed)
    on = rng.uniform(-1, 1, (L, W))
    et = 0.1 + rng.uniform(0, 0.05, (L, W))
    T, gV, gE = adjoint.transmission_gradient(on, et, 1.0, E, 0, 1, lm, 0.6)

    def Td(o, e):
        return buttiker.effective_transmission(wire.green_retarded(E, o, e, 1.0, lm, 0.6))[1, 0]

    assert abs(T - Td(on, et)) < 1e-11 * T
    h = 1e-5
    for a in range(L):
        for b in range(W):
            d = np.zeros((L, W))
            d[a, b] = h
            fdV = (Td(on + d, et) - Td(on - d, et)) / (2 * h)
            fdE = (Td(on, et + d) - Td(on, et - d)) / (2 * h)
            assert abs(fdV - gV[a, b]) <= 1e-6 * max(abs(fdV), 1e-3 * abs(T))
            assert abs(fdE - gE[a, b]) <= 1e-6 * max(abs(fdE), 1e-3 * abs(T))


def test_gradient_reciprocity():
    from oracle import adjoint
    on, et = _wire(24, 3, 4, 0.15)
    T1, gV1, gE1 = adjoint.transmission_gradient(on, et, 1.0, -0.3, 0, 1)
    T2, gV2, gE2 = adjoint.transmission_gradient(on, et, 1.0, -0.3, 1, 0)
    assert abs(T1 - T2) < 1e-12 * T1
    assert np.allclose(gV1, gV2, atol=1e-12 * np.abs(gV1).max())
    assert np.allclose(gE1, gE2, atol=1e-12 * np.abs(gE1).max())
