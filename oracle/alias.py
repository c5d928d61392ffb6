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

Two-level tables (long wires) draw the slice (or a lead) from an alias row over the slice
totals and then the site within the slice by the paper's own inverse-CDF draw, as 31-bit
cumulative thresholds in octets behind an 8-word guide (``cdf_block``).
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


CDF_ONE = 1 << 31     # level-2 thresholds are 31-bit: v = x >> 1 is uniform on [0, 2^31)


def level2_words(W):
    """u32 words of one level-2 block: one octet for W <= 8, else an 8-word guide followed by
    ceil(W / 8) octets."""
    G = -(-W // 8)
    return 8 if G == 1 else 8 + 8 * G


def cdf_block(wk):
    """Level-2 block of one slice: the inverse-CDF draw of Sec. III.B (cumulative sum,
    normalised, first entry above a uniform) over the slice's W site weights wk, in integers.

    c_a = floor(2^31 P_a / S) with P_a = sum_{b <= a} wk_b and S = P_{W-1}, for a < W - 1;
    c_{W-1} and the padding of the last octet are 2^31.  Words: octet g holds c_{8g .. 8g+7};
    for W > 8 an 8-word guide comes first, guide_g = c_{8g+7} for g < G - 1 and 2^31 after.
    Draw (v = x >> 1 for a uniform u32 x): g = #{guide words <= v} (0 without a guide), then
    site = 8g + #{words of octet g <= v}.  Site a is drawn with probability
    (c_a - c_{a-1}) / 2^31 (c_{-1} = 0), so a zero weight is never drawn.  A slice of zero total
    gets c = 2^31 everywhere (it is never drawn at level 1).
    """
    wk = np.asarray(wk, dtype=np.float64)
    W = wk.size
    G = -(-W // 8)
    c = np.full(8 * G, CDF_ONE, dtype=np.int64)
    P = np.cumsum(wk)
    S = P[-1] if W else 0.0
    if S > 0.0:
        c[:W - 1] = np.floor(P[:W - 1] / S * CDF_ONE).astype(np.int64)
    if G == 1:
        return c.astype(np.uint32)
    guide = np.full(8, CDF_ONE, dtype=np.int64)
    guide[:G - 1] = c[8 * np.arange(G - 1) + 7]
    return np.concatenate([guide, c]).astype(np.uint32)


def draw_level2(blocks, W, v):
    """Sites drawn from level-2 blocks [m, level2_words(W)] for 31-bit values v [m]."""
    blocks = np.asarray(blocks, dtype=np.int64).reshape(-1, level2_words(W))
    v = np.asarray(v, dtype=np.int64).reshape(-1)
    m = blocks.shape[0]
    G = -(-W // 8)
    if G == 1:
        g = np.zeros(m, dtype=np.int64)
        octs = blocks[:, :8]
    else:
        g = (blocks[:, :8] <= v[:, None]).sum(1)
        octs = blocks[:, 8:].reshape(m, G, 8)[np.arange(m), np.minimum(g, G - 1)]
    return 8 * g + (octs <= v[:, None]).sum(1)


def implied_level2(block, W):
    """Exact distribution over the W sites realised by the draw of ``draw_level2`` (evaluated
    on every interval between the block's distinct values)."""
    block = np.asarray(block, dtype=np.int64)
    cuts = np.unique(np.concatenate([[0, CDF_ONE], block[(block >= 0) & (block <= CDF_ONE)]]))
    p = np.zeros(W)
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        a = int(draw_level2(block, W, [lo])[0])
        if a >= W:
            raise ValueError("level-2 block draws a site beyond W")
        p[a] += (hi - lo) / CDF_ONE
    return p


def build_two_level(w, L, W):
    """Two-level tables of a weight matrix [rows, L*W + 2] whose first L*W columns are the
    sites of L slices of W sites each and whose last two are the leads.

    The Step 6' draw over K = L*W + 2 outcomes factorises exactly: P(slice k, site a) =
    P1(k) P2(a | k) with P1 over the L slice totals and the two lead weights, and P2 the slice's
    own weights over its total.  Returns (level1 [rows, L + 2] uint64 alias entries, level2
    [rows, L, level2_words(W)] uint32 inverse-CDF blocks).
    Pinned by: the product of the two implied distributions equals weights / row sum.
    """
    w = np.asarray(w, dtype=np.float64)
    rows = w.shape[0]
    sites = w[:, :L * W].reshape(rows, L, W)
    w1 = np.concatenate([sites.sum(axis=2), w[:, L * W:]], axis=1)
    level1 = np.stack([vose(r) for r in w1])
    level2 = np.stack([np.stack([cdf_block(sites[i, k]) for k in range(L)]) for i in range(rows)])
    return level1, level2


def implied_two_level(level1_row, level2_row, W):
    """Distribution over the L*W + 2 outcomes realised by one two-level row."""
    p1 = implied_distribution(level1_row)
    L = level2_row.shape[0]
    out = [p1[k] * implied_level2(level2_row[k], W) for k in range(L)]
    return np.concatenate(out + [p1[L:]])
