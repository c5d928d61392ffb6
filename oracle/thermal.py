"""Continuous-energy sampling of the linear-response conductance (oracle; test infrastructure
only).

Sec. II.E: the linear conductance is G_qp = (e^2/h) integral dE T_qp(E) Th(E) with
Th(E) = -df/dE (Eq. Gqp_expression); drawing the energy E_0 of each Monte Carlo sample from
h(E) = Th(E) makes the sampled variable X_pq = Tr[Gamma_p A](E_0) delta_rq (Eq. gpq_formula,
Eq. elast_lin_xpq).  Sec. "Interpolation" (discussion) replaces the transition probabilities at
E_0 by linear interpolation between two nearby energies where they were computed.

Here the energies are restricted to the span [E_0, E_{M-1}] of a grid on which tables exist:
  * Th(E) = 1 / (4 kT cosh^2((E - mu) / (2 kT))) is the logistic density with scale kT, CDF
    F(E) = 1 / (1 + exp(-(E - mu) / kT)), inverse mu + kT log(p / (1 - p));
  * G_grid = integral over [E_0, E_{M-1}] of Th(E) T(E) dE = (F(E_{M-1}) - F(E_0)) E[X] with E
    drawn from Th restricted to the span;
  * with E in grid interval i (E_i <= E < E_{i+1}, alpha = (E - E_i) / (E_{i+1} - E_i)) the walk
    uses the transition probabilities (1 - alpha) p(E_i) + alpha p(E_{i+1}) (each draw picks the
    table of E_{i+1} with probability alpha, else that of E_i), the injection distribution
    likewise, and X = c(E) = (1 - alpha) c_i + alpha c_{i+1} when absorbed at q = 1 - p;
  * an interval with no open channel of lead p at one end (c = 0 there) interpolates c only and
    walks with the open end's probabilities alone: a chain without an open lead never absorbs,
    so mixing it in would make the walks' mean length diverge as alpha approaches that end
    (both ends closed: X = 0).

Random numbers of walker ``wid`` in wire ``wire`` (seed -> key (lo, hi)), Philox4x32-10 block
b with counter (b, wid_lo, wid_hi, 0x80000000 | wire):
  block 0: (x0, x1) -> u = (((x0 << 32 | x1) >> 11) + 1/2) / 2^53, the energy's CDF value
           F = F(E_0) + u (F(E_{M-1}) - F(E_0)) (its interval: F(E_i) <= F < F(E_{i+1})) and
           E = F^-1(F); x2 picks the injection table
           (E_{i+1}'s iff x2 < a, a = min(floor(alpha 2^32), 2^32 - 1));
  block 1: the injection mode draw (x0, x1) on the picked table's mode row;
  block b >= 2: transition b - 1: (x0, x1) on the current row of the table picked by x2 < a.
A draw with words (x, y) over a K-entry row picks c = (x K) >> 32 and keeps c if y < thr[c],
else alias[c].

The interpolating sampler's grid (``refine_grid``): intervals whose two ends' Step 6'
probabilities differ by more than a tolerance (``interval_distance``, five percent in the
paper) are split at their midpoints until every interval passes.

Pinned by (tests/test_oracle_thermal.py): Th against the central difference of the Fermi
function and its integral against the closed-form CDF; the interval distance zero on equal
tables, symmetric, within [0, 1], and the refined grid's intervals all within the tolerance with
the interpolated conductance converging to the direct one as the tolerance shrinks (error
falling about as its square); the direct conductance of a clean chain
and of a clean wire's channel staircase in closed form; the interpolated chain equal to the
exact absorbing chain at alpha = 0 and 1 and converging to the direct conductance at the h^2
rate of linear interpolation; the replay walker within 4 SE of the interpolated chain's exact
expectation and its energies Kolmogorov-Smirnov-consistent with Th; planted mistakes caught.
"""
import numpy as np

from . import buttiker, markov, wire
from .alias import draw_level2
from .philox import philox4x32_10

MASK32 = np.uint64(0xFFFFFFFF)
TWO32 = float(2 ** 32)


def th_density(E, mu, kT):
    """Th(E) = -df/dE for the Fermi function f(E) = 1 / (1 + exp((E - mu) / kT))."""
    x = (np.asarray(E, dtype=np.float64) - mu) / (2.0 * kT)
    return 1.0 / (4.0 * kT * np.cosh(x) ** 2)


def th_cdf(E, mu, kT):
    """integral from -infinity to E of Th = 1 - f(E)."""
    return 1.0 / (1.0 + np.exp(-(np.asarray(E, dtype=np.float64) - mu) / kT))


def th_inverse(p, mu, kT):
    return mu + kT * np.log(p / (1.0 - p))


def energy_draw(x0, x1, grid, mu, kT):
    """(E, interval i, a) of the energy words (x0, x1) (uint32 arrays) on an ascending grid."""
    grid = np.asarray(grid, dtype=np.float64)
    v = ((x0.astype(np.uint64) << np.uint64(32)) | x1.astype(np.uint64)) >> np.uint64(11)
    u = (v.astype(np.float64) + 0.5) / 2.0 ** 53
    F = th_cdf(grid, mu, kT)
    pE = F[0] + u * (F[-1] - F[0])
    E = th_inverse(pE, mu, kT)
    # the interval: the CDF value placed among the grid's CDF values (F is increasing)
    i = np.clip(np.searchsorted(F, pE, side="right") - 1, 0, grid.size - 2)
    alpha = np.clip((E - grid[i]) / (grid[i + 1] - grid[i]), 0.0, 1.0)
    a = np.minimum(np.floor(alpha * TWO32), TWO32 - 1).astype(np.uint64)
    return E, i, a


def conductance_direct(onsite, eta, t, grid, mu, kT, n_quad=16, lead_model=0, gamma_lead=0.0,
                       q=1, p=0):
    """G_grid = integral over [grid[0], grid[-1]] of Th(E) T^eff_qp(E) dE (units e^2/h), by
    Gauss-Legendre quadrature with n_quad nodes on each grid interval of the direct probe solve
    (Eq. buteq)."""
    grid = np.asarray(grid, dtype=np.float64)
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    total = 0.0
    for i in range(grid.size - 1):
        lo, hi = grid[i], grid[i + 1]
        for x, wq in zip(xg, wg):
            E = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
            g = wire.green_retarded(E, onsite, eta, t, lead_model, gamma_lead)
            T = buttiker.effective_transmission(g)[q, p]
            total += 0.5 * (hi - lo) * wq * th_density(E, mu, kT) * T
    return total


def _chain(tab):
    w, n = tab["w"], tab["n"]
    tot = w.sum(axis=1)
    P = np.zeros_like(w)
    live = tot > 0
    P[live] = w[live] / tot[live, None]
    return P


def interpolated_absorption(tab_i, tab_j, alpha, p=0):
    """P(q | p) for q = 0, 1 of the chain whose transition probabilities are (1 - alpha) times
    those of tab_i plus alpha times those of tab_j, injected from lead p with the interpolated
    mode distribution; when lead p has no open channel at one end, the chain and injection of
    the open end alone."""
    n, W = tab_i["n"], tab_i["W"]
    mi, mj = tab_i["mode_w"][p], tab_j["mode_w"][p]
    open_i, open_j = tab_i["c"][p] > 0.0, tab_j["c"][p] > 0.0
    if not (open_i or open_j):
        return np.zeros(2)
    if open_i and open_j:
        P = (1.0 - alpha) * _chain(tab_i) + alpha * _chain(tab_j)
        u = (1.0 - alpha) * mi / mi.sum() + alpha * mj / mj.sum()
    elif open_i:
        P, u = _chain(tab_i), mi / mi.sum()
    else:
        P, u = _chain(tab_j), mj / mj.sum()
    Q, R = P[:n, :n], P[:n, n:]
    P_site = np.linalg.solve(np.eye(n) - Q, R)
    Pi = P[n + p * W:n + (p + 1) * W]
    return u @ (Pi[:, n:] + Pi[:, :n] @ P_site)


def interval_distance(tab_i, tab_j, p=0):
    """How far apart the Step 6' probabilities of two grid energies are (Sec. "Interpolation":
    where two nearby energies' probabilities p_i differ by less than five percent, the p_i in
    between are interpolated linearly).  The largest of: the total-variation distance
    (1/2) sum_b |P_ab(E_i) - P_ab(E_j)| of every row a (rows normalised to their sums; a row of
    zero sum is all zeros), the same for the injection-mode distributions of lead p, and the
    relative change |c_i - c_j| / max(c_i, c_j) of c = Tr Gamma_p A (0 when both vanish)."""
    d = 0.5 * np.abs(_chain(tab_i) - _chain(tab_j)).sum(axis=1).max()
    mi, mj = tab_i["mode_w"][p], tab_j["mode_w"][p]
    ui = mi / mi.sum() if mi.sum() > 0 else np.zeros_like(mi)
    uj = mj / mj.sum() if mj.sum() > 0 else np.zeros_like(mj)
    d = max(d, 0.5 * np.abs(ui - uj).sum())
    ci, cj = tab_i["c"][p], tab_j["c"][p]
    if max(ci, cj) > 0.0:
        d = max(d, abs(ci - cj) / max(ci, cj))
    return float(d)


def refine_grid(onsite, eta, t, e_lo, e_hi, n_init, tol=0.05, max_points=257, p=0,
                lead_model=0, gamma_lead=0.0):
    """The energy grid of the interpolating sampler (Sec. "Interpolation"): start from n_init
    evenly spaced energies on [e_lo, e_hi]; in each round every interval whose two ends are
    farther apart than tol (interval_distance) is split at its midpoint (E_i + E_{i+1}) / 2, in
    the order of the grid, as long as the grid stays within max_points energies; stop when every
    interval passes or no point can be added.  Returns (grid, distances of its intervals)."""
    W = np.asarray(onsite).shape[1]

    def table(E):
        g = wire.green_retarded(E, onsite, eta, t, lead_model, gamma_lead)
        phi, _, gam = wire.lead_modes(E, W, t, lead_model, gamma_lead)
        return markov.transition_weights(g, (phi, gam))
    grid = [float(E) for E in np.linspace(e_lo, e_hi, n_init)]
    tabs = {E: table(E) for E in grid}
    while True:
        d = [interval_distance(tabs[grid[i]], tabs[grid[i + 1]], p) for i in range(len(grid) - 1)]
        new = []
        for i, di in enumerate(d):
            if di > tol and len(grid) + len(new) < max_points:
                new.append(0.5 * (grid[i] + grid[i + 1]))
        if not new:
            return np.array(grid), np.array(d)
        for E in new:
            tabs[E] = table(E)
        grid = sorted(grid + new)


def conductance_interpolated(tabs, grid, mu, kT, n_quad=16, p=0):
    """The exact expectation of the sampler: integral over the span of Th(E) c(E) P(q|p; E) dE
    with c and the chain interpolated linearly between grid energies (q = 1 - p)."""
    grid = np.asarray(grid, dtype=np.float64)
    q = 1 - p
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    total = 0.0
    for i in range(grid.size - 1):
        lo, hi = grid[i], grid[i + 1]
        ci, cj = tabs[i]["c"][p], tabs[i + 1]["c"][p]
        for x, wq in zip(xg, wg):
            alpha = 0.5 * (x + 1.0)
            E = lo + alpha * (hi - lo)
            c = (1.0 - alpha) * ci + alpha * cj
            if c <= 0.0:
                continue
            P = interpolated_absorption(tabs[i], tabs[i + 1], alpha, p)
            total += 0.5 * (hi - lo) * wq * th_density(E, mu, kT) * c * P[q]
    return total


def walk(entries, mode_entries, c, n, W, wire_index, start_lead, seed, wids, grid, mu, kT,
         max_steps, energy=None, level2=None):
    """Replay walkers ``wids`` of the thermal sampler over integer alias tables.

    entries[e] [n + 2W, n + 2] and mode_entries[e] [2, W] (uint64) and c[e] (Tr Gamma_p A at the
    two leads) of every grid energy e.  ``energy``: optional (interval, a) arrays that replace the
    energy draw (the replay of a trace).  ``level2``: for two-level tables, (blocks, L) with
    blocks[e] [n + 2W, L, alias.level2_words(W)] the level-2 inverse-CDF blocks, entries[e] then
    being the level-1 alias rows [n + 2W, L + 2]; a transition draws the slice or lead with
    (x0, x1) and the site of a drawn slice with v = x3 >> 1 (alias.draw_level2).  Returns
    (lead int32: 0 / 1, -1 no open channel, -2 truncated; steps uint32; interval int64; a uint64).
    """
    wids = np.asarray(wids, dtype=np.uint64)
    m = wids.size
    wlo, whi = wids & MASK32, wids >> np.uint64(32)
    k0, k1 = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    ctr3 = np.full(m, 0x80000000 | int(wire_index), dtype=np.uint64)
    x = philox4x32_10(np.zeros(m, dtype=np.uint64), wlo, whi, ctr3, k0, k1)
    if energy is None:
        _, iv, a = energy_draw(x[0], x[1], grid, mu, kT)
    else:
        iv, a = np.asarray(energy[0], dtype=np.int64), np.asarray(energy[1], dtype=np.uint64)
    K = n + 2
    lead = np.full(m, -2, dtype=np.int32)
    steps = np.zeros(m, dtype=np.uint32)
    for w in range(m):
        i = int(iv[w])
        open_lo, open_hi = c[i][start_lead] > 0.0, c[i + 1][start_lead] > 0.0
        if not (open_lo or open_hi):
            lead[w] = -1
            continue

        def pick(word):
            # the table of the draw: mixed on an interval open at both ends, else the open end
            if open_lo and open_hi:
                return i + 1 if int(word) < int(a[w]) else i
            return i if open_lo else i + 1
        t = pick(x[2][w])
        y = philox4x32_10(np.array([1], np.uint64), wlo[w:w + 1], whi[w:w + 1], ctr3[w:w + 1],
                          k0, k1)
        cc = (int(y[0][0]) * W) >> 32
        e = int(mode_entries[t][start_lead][cc])
        mode = cc if int(y[1][0]) < (e & 0xFFFFFFFF) else (e >> 32)
        row = n + start_lead * W + mode
        b = 2
        while True:
            z = philox4x32_10(np.array([b], np.uint64), wlo[w:w + 1], whi[w:w + 1],
                              ctr3[w:w + 1], k0, k1)
            t = pick(z[2][0])
            if level2 is None:
                cc = (int(z[0][0]) * K) >> 32
                e = int(entries[t][row, cc])
                j = cc if int(z[1][0]) < (e & 0xFFFFFFFF) else (e >> 32)
            else:
                blocks, L = level2
                cc = (int(z[0][0]) * (L + 2)) >> 32
                e = int(entries[t][row, cc])
                k = cc if int(z[1][0]) < (e & 0xFFFFFFFF) else (e >> 32)
                j = n + (k - L) if k >= L else \
                    k * W + int(draw_level2(blocks[t][row, k], W, [int(z[3][0]) >> 1])[0])
            steps[w] += 1
            if j >= n:
                lead[w] = j - n
                break
            if steps[w] >= max_steps:
                break
            row = j
            b += 1
    return lead, steps, iv, a


def estimate(lead, a, iv, c, window, start_lead=0):
    """(G, SE) of the sampled X = c(E) 1[absorbed at q], scaled by the window F1 - F0."""
    q = 1 - start_lead
    alpha = a.astype(np.float64) / TWO32
    cE = np.array([(1.0 - al) * c[i][start_lead] + al * c[i + 1][start_lead]
                   for i, al in zip(iv, alpha)])
    X = np.where(lead == q, cE, 0.0)
    return window * X.mean(), window * X.std(ddof=0) / np.sqrt(X.size)
