"""Alias tables for the categorical draw of Step 6' (oracle; test infrastructure only).

The paper draws the next index by inverse CDF: cumulative sum of the weight array a_j,
normalised, and the first entry above a uniform x (Sec. III.B).  The walk instead uses Walker's
alias method, built here by Vose's algorithm (M. D. Vose, IEEE TSE 17(9), 1991), so one draw
costs O(1).  Integer form of one slot c of a K-entry row, as the walk consumes it:

    entry = thr | (alias << 32),   thr = floor(prob_c * 2^32) (a full slot stores alias = c),
    draw  : c = (x * K) >> 32 for a uniform u32 x (multiply-shift), then
            outcome = c if y < thr else alias, for a second uniform u32 y.

``implied_distribution`` recomputes, exactly in integers, the distribution a table realises, so
any table (this one or one exported from the GPU) can be checked against the FP weights.
"""
from fractions import Fraction

import numpy as np

TWO32 = 1 << 32


def vose(weights):
    """Vose's alias construction for one row of nonnegative weights.  Returns uint64 entries.

    Rows whose weights sum to zero get all-full slots (never drawn in a valid walk).
    Pinned by: the exact implied distribution equals weights/sum within the quantisation bound.
    """
    w = np.asarray(weights, dtype=np.float64)
    K = w.size
    total = float(w.sum())
    prob = np.ones(K)
    alias = np.arange(K, dtype=np.int64)
    if total > 0.0:
        q = w * (K / total)
        small = [i for i in range(K) if q[i] < 1.0]
        large = [i for i in range(K) if q[i] >= 1.0]
        while small and large:
            l = small.pop()
            g = large.pop()
            prob[l] = q[l]
            alias[l] = g
            q[g] = (q[g] + q[l]) - 1.0
            if q[g] < 1.0:
                small.append(g)
            else:
                large.append(g)
        # leftovers are full slots (exactly 1 in exact arithmetic)
        for i in large + small:
            prob[i] = 1.0
            alias[i] = i
    thr = np.minimum(np.floor(prob * TWO32), TWO32 - 1).astype(np.uint64)
    full = prob >= 1.0
    alias[full] = np.arange(K)[full]
    return thr | (alias.astype(np.uint64) << np.uint64(32))


def build_tables(w):
    """Vose tables for every row of a weight matrix [rows, K]."""
    return np.stack([vose(row) for row in w])


def split(entries):
    e = np.asarray(entries, dtype=np.uint64)
    return (e & np.uint64(0xFFFFFFFF)).astype(np.int64), (e >> np.uint64(32)).astype(np.int64)


def slot_mass(K):
    """Exact number of u32 values x with (x*K)>>32 == c, for c = 0..K-1 (Python ints)."""
    return [(-(-((c + 1) * TWO32) // K)) - (-(-(c * TWO32) // K)) for c in range(K)]


def implied_distribution(entries, exact=False):
    """Exact outcome distribution of one integer alias row under the draw above."""
    thr, ali = split(entries)
    K = thr.size
    mass = slot_mass(K)
    if exact:
        p = [Fraction(0)] * K
        for c in range(K):
            keep = Fraction(mass[c] * int(thr[c]), TWO32 * TWO32)
            p[c] += keep
            p[int(ali[c])] += Fraction(mass[c], TWO32) - keep
        return p
    p = np.zeros(K)
    for c in range(K):
        m = mass[c] / TWO32
        keep = m * (int(thr[c]) / TWO32)
        p[c] += keep
        p[int(ali[c])] += m - keep
    return p


def build_two_level(w, L, W):
    """Two-level alias tables of a weight matrix [rows, L*W + 2] whose first L*W columns are the
    sites of L slices of W sites each and whose last two are the leads.

    The Step 6' draw over K = L*W + 2 outcomes factorises exactly: P(slice k, site a) =
    P1(k) P2(a | k) with P1 over the L slice totals and the two lead weights, and P2 the slice's
    own weights over its total.  Returns (level1 [rows, L + 2], level2 [rows, L, W]) uint64
    entries; a slice of zero total gets all-full slots (never drawn).
    Pinned by: the product of the two implied distributions equals weights / row sum.
    """
    w = np.asarray(w, dtype=np.float64)
    rows = w.shape[0]
    sites = w[:, :L * W].reshape(rows, L, W)
    w1 = np.concatenate([sites.sum(axis=2), w[:, L * W:]], axis=1)
    level1 = np.stack([vose(r) for r in w1])
    level2 = np.stack([np.stack([vose(sites[i, k]) for k in range(L)]) for i in range(rows)])
    return level1, level2


def implied_two_level(level1_row, level2_row):
    """Distribution over the L*W + 2 outcomes realised by one two-level row."""
    p1 = implied_distribution(level1_row)
    L = level2_row.shape[0]
    out = [p1[k] * implied_distribution(level2_row[k]) for k in range(L)]
    return np.concatenate(out + [p1[L:]])
