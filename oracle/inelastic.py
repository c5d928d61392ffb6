"""Inelastic Buttiker probes: Step 6' followed by the energy draw of Step 7' (oracle; test
infrastructure only).

Sec. II.F.  With Buttiker's approximation a probe i scatters out at the rate
lambda~_i(E, E') <i|G|i>, and charge conservation (assumption (iv)) ties that rate to the probe's
broadening: gamma_i(E) = int dE' lambda~_i(E', E) A_ii(E') (Eq. condition4_buttiker).  Once
Step 6' has drawn an internal index i, Step 7' draws the walker's next energy with
p(E) = lambda~_i(E, E_n) A_ii(E) / gamma_i(E_n) (Eq. draw_E_last); the walk then goes on from
the state at that energy.

Model (a reading: the paper leaves lambda~ open).  On the energy grid {E_e} with quadrature
weights w_e, a redistribution kernel K(dE) (a Gaussian of width sigma; the identity for
sigma = 0) is scaled so that gamma_i = eta_i at every energy,
    lambda~_i(E_e', E_e) = eta_i K(E_e' - E_e) / sum_e'' w_e'' K(E_e'' - E_e) A_ii(E_e''),
which satisfies Eq. condition4_buttiker exactly and leaves G^r, and so every Step 6' table, the
elastic one.  The energy draw is then
    p(e' | i, e) = w_e' K(E_e' - E_e) A_ii(E_e') / sum_e'' w_e'' K(E_e'' - E_e) A_ii(E_e''),
and sigma = 0 is the elastic limit lambda~ ~ delta(E - E').

The chain's states are (site, energy).  A walker injected from lead p at energy E_0 is absorbed
at lead q with probability P(q | p, E_0); T_qp(E_0) = c_p(E_0) P(q | p, E_0) is the estimator of
Eq. elast_lin_xpq with the walker's energy free to change on the way.
"""
import numpy as np

from . import alias
from .philox import philox4x32_10

MASK32 = np.uint64(0xFFFFFFFF)


def energy_kernel(E, sigma):
    """K[e, e'] = exp(-(E_e' - E_e)^2 / (2 sigma^2)); the identity for sigma = 0."""
    E = np.asarray(E, dtype=np.float64)
    if sigma <= 0.0:
        return np.eye(E.size)
    d = E[None, :] - E[:, None]
    return np.exp(-d * d / (2.0 * sigma * sigma))


def energy_weights(A, E, wE, sigma):
    """Step 7' weights [n, nE, nE]: wts[i, e, e'] = w_e' K(E_e' - E_e) A_ii(E_e') for the site
    spectral weights A [nE, n] (A_ii at each grid energy)."""
    K = energy_kernel(E, sigma)
    A = np.asarray(A, dtype=np.float64)
    wE = np.asarray(wE, dtype=np.float64)
    return (K[None, :, :] * (wE[None, None, :] * A.T[:, None, :]))


def energy_tables(wts):
    """Alias rows [n, nE, nE] (uint64 entries) of the Step 7' weights, one per (site, energy)."""
    n, nE, _ = wts.shape
    out = np.zeros((n, nE, nE), dtype=np.uint64)
    for i in range(n):
        for e in range(nE):
            out[i, e] = alias.vose(wts[i, e])
    return out


def chain(tabs, E, wE, sigma):
    """Exact absorption of the inelastic chain of one wire.

    tabs: the Step 6' tables (markov.transition_weights) of the wire at each grid energy.
    Returns P_inj [nE, p, q] = P(q | p, E_0 = E_e), steps_inj [nE, p] (mean transitions drawn,
    the absorbing one included), T [nE, q, p] = c_p(E_0) P(q | p, E_0) and the hop
    probabilities H [n, nE, nE] = p(e' | i, e).
    Pinned by: the elastic limit sigma = 0 (every energy's own chain, markov.absorption), a grid
    of one repeated energy (any sigma), P(L) + P(R) = 1, and the CPU walker's samples.
    """
    nE = len(tabs)
    n, W = tabs[0]["n"], tabs[0]["W"]
    A = np.stack([t["w"][:n].sum(axis=1) for t in tabs])            # [nE, n] row sums = A_ii
    wts = energy_weights(A, E, wE, sigma)
    tot = wts.sum(axis=2, keepdims=True)
    H = np.divide(wts, tot, out=np.zeros_like(wts), where=tot > 0)
    P = []
    for t in tabs:
        s = t["w"].sum(axis=1, keepdims=True)
        P.append(np.divide(t["w"], s, out=np.zeros_like(t["w"]), where=s > 0))
    S = n * nE                                                       # state (i, e) -> e n + i
    Q = np.zeros((S, S))
    R = np.zeros((S, 2))
    for e in range(nE):
        Pe = P[e]
        for ep in range(nE):
            # (i, e) -> (j, e'): P_e[i, j] H[j, e, e']
            Q[e * n:(e + 1) * n, ep * n:(ep + 1) * n] = Pe[:n, :n] * H[None, :, e, ep]
        R[e * n:(e + 1) * n] = Pe[:n, n:]
    IQ = np.eye(S) - Q
    P_site = np.linalg.solve(IQ, R)
    steps_site = np.linalg.solve(IQ, np.ones(S))
    P_inj = np.zeros((nE, 2, 2))
    steps_inj = np.zeros((nE, 2))
    T = np.zeros((nE, 2, 2))
    for e0 in range(nE):
        Pe = P[e0]
        for p in range(2):
            mw = tabs[e0]["mode_w"][p]
            if mw.sum() <= 0:
                continue
            u = mw / mw.sum()
            Pi = Pe[n + p * W:n + (p + 1) * W]                       # [W, n + 2]
            # first transition to site j, then the energy hop from E_0: weights over (j, e')
            first = Pi[:, :n, None] * H[None, :, e0, :]               # [W, n, nE]
            reach = first.transpose(0, 2, 1).reshape(W, S)           # state e' n + j
            P_inj[e0, p] = u @ (Pi[:, n:] + reach @ P_site)
            steps_inj[e0, p] = u @ (1.0 + reach @ steps_site)
            T[e0, :, p] = tabs[e0]["c"][p] * P_inj[e0, p]
    return dict(P_inj=P_inj, steps_inj=steps_inj, T=T, H=H, weights=wts)


def walk(entries, mode_entries, energy_entries, n, W, c_open, e0, task, start_lead, seed,
         wids, max_steps):
    """Inelastic walkers injected at energy index e0.  Returns (lead, steps) as walker.walk.

    entries [nE, n + 2W, n + 2] and mode_entries [nE, 2, W]: the Step 6' alias rows at every
    grid energy; energy_entries [n, nE, nE]: the Step 7' alias rows; c_open [nE, 2].
    Random numbers: Philox4x32-10 block b of walker wid with counter (b, wid_lo, wid_hi, task)
    and key (seed_lo, seed_hi), task being the injection task's number.  Block 0 is the
    injection draw (words x0, x1 over the W modes at E_0); block s >= 1 is transition s: words
    (x0, x1) draw the next index from the current row at the walker's energy e (K = n + 2,
    leads n and n + 1), and for a site j words (x2, x3) draw the next energy e' from the energy
    row (j, e).  A draw with words (x, y) over a K-entry row picks c = (x K) >> 32 and keeps c
    if y < thr[c], else takes alias[c].
    Pinned by: absorption probabilities and mean steps against ``chain``.
    """
    wids = np.asarray(wids, dtype=np.uint64)
    m = wids.size
    nE = energy_entries.shape[1]
    K = n + 2
    lead = np.full(m, -2, dtype=np.int32)
    steps = np.zeros(m, dtype=np.uint32)
    if m == 0:
        return lead, steps
    if not c_open[e0][start_lead]:
        lead[:] = -1
        return lead, steps
    wlo = wids & MASK32
    whi = wids >> np.uint64(32)
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    active = np.arange(m)
    row = np.zeros(m, dtype=np.int64)
    ene = np.full(m, e0, dtype=np.int64)
    s = 0
    while active.size:
        if s >= 1 and s > max_steps:
            break
        b = np.full(active.size, s, dtype=np.uint64)
        x0, x1, x2, x3 = (v.astype(np.uint64) for v in
                          philox4x32_10(b, wlo[active], whi[active], np.full(active.size, task),
                                        k0, k1))
        if s == 0:
            c = ((x0 * np.uint64(W)) >> np.uint64(32)).astype(np.int64)
            ent = mode_entries[e0][start_lead][c]
            mode = np.where(x1 < (ent & MASK32), c, (ent >> np.uint64(32)).astype(np.int64))
            row[active] = n + start_lead * W + mode
        else:
            r, e = row[active], ene[active]
            c = ((x0 * np.uint64(K)) >> np.uint64(32)).astype(np.int64)
            ent = entries[e, r, c]
            j = np.where(x1 < (ent & MASK32), c, (ent >> np.uint64(32)).astype(np.int64))
            steps[active] = s
            done = j >= n
            lead[active[done]] = (j[done] - n).astype(np.int32)
            jj = np.where(done, 0, j)
            ce = ((x2 * np.uint64(nE)) >> np.uint64(32)).astype(np.int64)
            ent = energy_entries[jj, e, ce]
            ep = np.where(x3 < (ent & MASK32), ce, (ent >> np.uint64(32)).astype(np.int64))
            row[active] = jj
            ene[active] = ep
            active = active[~done]
        s += 1
    return lead, steps
