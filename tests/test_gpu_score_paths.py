"""Score tallies of negf_walk_score against the oracle's walks, count for count.

Every transition a -> b of a walk absorbed at lead r adds one to score[r][a][b] of its task, and
its injection mode m to mode_score[r][m]: the counts the score-function gradient is formed
from.  Here the GPU's counts over N walkers equal, exactly, those of the oracle walker run on
the exported tables with the same Philox streams (its recorded paths), for one- and two-level
tables, both start leads, and strongly dephasing wires whose walks run shorter than the walk
kernel's shared-memory record, into its local-memory extension, and beyond both (so that the
recorded commits of both parts and the replayed commit are exercised).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import walker  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402

RECORD = 16          # transitions the walk kernel records per walker in shared memory
RECORD_ALL = 128     # ... and in all, before it replays a walk


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    c = negf.negf_create(0)
    yield c
    negf.negf_destroy(c)


def _oracle_counts(ctx, tables, task, p, seed, N, offset):
    info = negf.negf_get_task_info(ctx, tables, task)
    n, W, L, rows, K = info["n"], info["W"], info["L"], info["rows"], info["K"]
    ment = negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, W)
    path = {}
    ids = offset + np.arange(N, dtype=np.uint64)
    if info["layout"] == "two_level":
        l2 = negf.negf_export_tables(ctx, tables, task, "alias").view(np.uint32).reshape(
            rows, L, negf.level2_words(W))
        l1 = negf.negf_export_tables(ctx, tables, task, "alias_level1").reshape(rows, L + 2)
        lead, steps = walker.walk_two_level(l1, l2, ment, n, L, W, info["c"] > 0, task, p, seed,
                                            ids, 1 << 20, path=path)
    else:
        ent = negf.negf_export_tables(ctx, tables, task, "alias").reshape(rows, K)
        lead, steps = walker.walk(ent, ment, n, W, info["c"] > 0, task, p, seed, ids, 1 << 20,
                                  path=path)
    score = np.zeros((2, rows * K), dtype=np.uint64)
    mode = np.zeros((2, 2 * W), dtype=np.uint64)
    for idx, row, col in path["steps"]:
        r = lead[idx]
        ok = r >= 0
        np.add.at(score, (r[ok], row[ok] * K + col[ok]), np.uint64(1))
    ok = lead >= 0
    np.add.at(mode, (lead[ok], p * W + path["mode"][ok]), np.uint64(1))
    return info, score, mode, steps[ok]


@pytest.mark.parametrize("layout", ["one_level", "two_level"])
def test_score_counts_equal_the_oracle_walks(ctx, layout):
    wires = [inputs.small_wire(71, W=3, L=8, n_energy=2, eta=0.8),
             inputs.small_wire(72, W=5, L=6, n_energy=1, eta=0.3),
             inputs.small_wire(73, W=2, L=30, n_energy=1, eta=1.0)]     # ~1 % beyond 128
    tables = negf.negf_build_tables(ctx, wires, precision="fp64", layout=layout)
    N, offset = 3000, 2**33 + 11
    lengths = []
    try:
        for p in (0, 1):
            seed = 0x5C0DE + p
            tally = negf.negf_walk_score(ctx, tables, p, seed, N, walker_id_offset=offset)
            try:
                sc, md = negf.negf_tally_score_counts(ctx, tally)
            finally:
                negf.negf_tally_free(tally)
            for task in range(sum(len(w.energy) for w in wires)):
                info, score, mode, steps = _oracle_counts(ctx, tables, task, p, seed, N, offset)
                off, moff = info["table_offset"], info["mode_offset"]
                assert np.array_equal(sc[:, off:off + score.shape[1]], score), (layout, p, task)
                assert np.array_equal(md[:, moff:moff + mode.shape[1]], mode), (layout, p, task)
                lengths.append(steps)
    finally:
        negf.negf_tables_free(tables)
    lengths = np.concatenate(lengths)
    short = int((lengths <= RECORD).sum())
    ext = int(((lengths > RECORD) & (lengths <= RECORD_ALL)).sum())
    long_ = int((lengths > RECORD_ALL).sum())
    assert short > 0 and ext >= 20 and long_ >= 10, (short, ext, long_)
