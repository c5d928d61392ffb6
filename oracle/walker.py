"""The Step 6' random walk over integer alias tables, driven by Philox4x32-10
(oracle; test infrastructure only).

One walker = one Monte Carlo sample of Sec. II.E with fixed start lead p (Eq. elast_lin_xpq):
Step 4 draws the injection eigenvector of Gamma_p, then Step 6' repeats (site or lead) until a
lead is drawn.  Random numbers: draw s of walker ``wid`` in task ``task`` uses Philox block
b = s // 2 with counter (b, wid_lo, wid_hi, task) and key (seed_lo, seed_hi); even s takes output
words (x0, x1), odd s takes (x2, x3).  Draw 0 is the injection draw (always consumed); draws
1, 2, ... are transitions and each one counts as a step.  A draw with words (x, y) over a K-entry
row picks c = (x*K)>>32 and keeps c if y < thr[c], else takes alias[c].

Outcomes per walker: lead 0 (L) or 1 (R); -1 when the start lead has no open channel at this
energy (Tr Gamma_p A = 0, nothing to inject); -2 when ``max_steps`` transitions were drawn without
absorption (the walk is cut, the sample is counted as truncated).
"""
import numpy as np

from .alias import draw_level2
from .philox import philox4x32_10

MASK32 = np.uint64(0xFFFFFFFF)


def walk(entries, mode_entries, n, W, c_open, task, start_lead, seed, wids, max_steps,
         path=None):
    """Run walkers ``wids`` (uint64 array) to absorption.  Returns (lead int32, steps uint32).

    entries [n + 2W, n + 2] uint64 alias rows, mode_entries [2, W] uint64 injection alias rows,
    c_open [2] bool (lead p has an open channel).  ``path``, a dict, receives the walk itself:
    "mode" (the injection mode of every walker) and "steps", one (walker positions, row, column)
    triple per transition drawn.  Pinned by: the empirical absorption probabilities and mean
    steps of many walkers against the exact chain expectation.
    """
    wids = np.asarray(wids, dtype=np.uint64)
    m = wids.size
    K = n + 2
    lead = np.full(m, -2, dtype=np.int32)
    steps = np.zeros(m, dtype=np.uint32)
    if path is not None:
        path["mode"] = np.zeros(m, dtype=np.int64)
        path["steps"] = []
    if m == 0:
        return lead, steps
    if not c_open[start_lead]:
        lead[:] = -1
        return lead, steps
    wlo = wids & MASK32
    whi = wids >> np.uint64(32)
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    active = np.arange(m)
    row = np.zeros(m, dtype=np.int64)
    words = None
    s = 0
    while active.size:
        if s >= 1 and s > max_steps:
            break
        if s % 2 == 0:
            b = np.full(active.size, s // 2, dtype=np.uint64)
            words = philox4x32_10(b, wlo[active], whi[active], np.full(active.size, task), k0, k1)
            x, y = words[0], words[1]
        else:
            x, y = words[2], words[3]
        x = x.astype(np.uint64)
        y = y.astype(np.uint64)
        if s == 0:
            c = ((x * np.uint64(W)) >> np.uint64(32)).astype(np.int64)
            e = mode_entries[start_lead][c]
            keep = y < (e & MASK32)
            mode = np.where(keep, c, (e >> np.uint64(32)).astype(np.int64))
            row[active] = n + start_lead * W + mode
            if path is not None:
                path["mode"][active] = mode
        else:
            c = ((x * np.uint64(K)) >> np.uint64(32)).astype(np.int64)
            e = entries[row[active], c]
            keep = y < (e & MASK32)
            j = np.where(keep, c, (e >> np.uint64(32)).astype(np.int64))
            if path is not None:
                path["steps"].append((active.copy(), row[active].copy(), j.copy()))
            steps[active] = s
            done = j >= n
            lead[active[done]] = (j[done] - n).astype(np.int32)
            row[active] = np.where(done, 0, j)
            sel = ~done
            active = active[sel]
            if words is not None:
                words = tuple(wd[sel] for wd in words)
        s += 1
    return lead, steps


def walk_two_level(level1, level2, mode_entries, n, L, W, c_open, task, start_lead, seed, wids,
                   max_steps, path=None):
    """The same walk over two-level tables (level1 [n + 2W, L + 2] alias entries, level2
    [n + 2W, L, alias.level2_words(W)] inverse-CDF blocks).

    Random numbers: Philox block 0 of the walker is the injection draw (words x0, x1); block
    s >= 1 is transition s: words (x0, x1) draw the slice or lead from the row's level-1 entries
    (K1 = L + 2), and for a slice k the word x2 draws the site a from level-2 block (row, k)
    with v = x2 >> 1 (alias.draw_level2); the next row is k*W + a.  Outcomes and step counts as
    in ``walk``; ``path`` as in ``walk``, the column of a transition being the site k W + a or
    the lead n + r.
    Pinned by: absorption probabilities and mean steps against the exact chain expectation.
    """
    wids = np.asarray(wids, dtype=np.uint64)
    m = wids.size
    K1 = L + 2
    lead = np.full(m, -2, dtype=np.int32)
    steps = np.zeros(m, dtype=np.uint32)
    if path is not None:
        path["mode"] = np.zeros(m, dtype=np.int64)
        path["steps"] = []
    if m == 0:
        return lead, steps
    if not c_open[start_lead]:
        lead[:] = -1
        return lead, steps
    wlo = wids & MASK32
    whi = wids >> np.uint64(32)
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    active = np.arange(m)
    row = np.zeros(m, dtype=np.int64)
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
            e = mode_entries[start_lead][c]
            mode = np.where(x1 < (e & MASK32), c, (e >> np.uint64(32)).astype(np.int64))
            row[active] = n + start_lead * W + mode
            if path is not None:
                path["mode"][active] = mode
        else:
            r = row[active]
            c = ((x0 * np.uint64(K1)) >> np.uint64(32)).astype(np.int64)
            e = level1[r, c]
            k = np.where(x1 < (e & MASK32), c, (e >> np.uint64(32)).astype(np.int64))
            steps[active] = s
            done = k >= L
            lead[active[done]] = (k[done] - L).astype(np.int32)
            kk = np.where(done, 0, k)
            v = (x2 >> np.uint64(1)).astype(np.int64)
            a = draw_level2(level2[r, kk], W, v)
            if path is not None:
                path["steps"].append((active.copy(), r.copy(), np.where(done, n + k - L, kk * W + a)))
            row[active] = np.where(done, 0, kk * W + a)
            active = active[~done]
        s += 1
    return lead, steps
