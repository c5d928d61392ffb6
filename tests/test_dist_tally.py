"""Multi-process path on CPU (gloo, world size 2): walker-id ranges split over ranks give
disjoint Philox streams, and the summed tallies equal a single process's tallies over the union
of walker ids bit for bit.  The CPU walker of the oracle stands in for the walk kernel (the GPU
parity tests show the two are bit-identical on shared tables)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1805_10164_gb300 import dist as ndist, inputs  # noqa: E402

N_WALKERS = 3001          # odd: the split is uneven
SEED = 77


def _tally(ref, task, start_lead, wids):
    from oracle import walker
    lead, steps = walker.walk(ref["entries"], ref["mode_entries"], ref["n"], ref["W"],
                              ref["c_open"], task, start_lead, SEED,
                              np.asarray(wids, dtype=np.uint64), 1 << 16)
    return np.array([lead.size, (lead == 0).sum(), (lead == 1).sum(), (lead == -2).sum(),
                     steps.astype(np.uint64).sum()], dtype=np.uint64)


def _refs():
    from oracle import pipeline
    w = inputs.small_wire(5, W=2, L=4, n_energy=2, eta=0.3, e_lo=-1.5, e_hi=1.5)
    out = []
    for E in w.energy:
        r = pipeline.task_reference(w.onsite, w.eta, w.t, E, with_direct=False)
        r["W"] = w.W
        out.append(r)
    return out


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        refs = _refs()
        off, cnt = ndist.walker_range(rank, world, N_WALKERS)
        local = np.stack([_tally(r, k, 0, np.arange(off, off + cnt)) for k, r in enumerate(refs)])
        merged = ndist.allreduce_tally(local)
        q.put((rank, local, merged))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_walker_range_partitions():
    for world in (1, 2, 3, 8):
        for n in (0, 1, 7, 3001):
            spans = [ndist.walker_range(r, world, n) for r in range(world)]
            ids = np.concatenate([np.arange(o, o + c) for o, c in spans])
            assert np.array_equal(ids, np.arange(n))
    with pytest.raises(ValueError):
        ndist.walker_range(2, 2, 10)
    a = ndist.weak_walker_offset(0, 5, 1000)
    b = ndist.weak_walker_offset(1, 0, 1000)
    assert a + 1000 <= b


def test_allreduce_single_process_is_identity():
    c = np.arange(10, dtype=np.uint64).reshape(2, 5)
    assert np.array_equal(ndist.allreduce_tally(c), c)
    with pytest.raises(ValueError):
        ndist.allreduce_tally(np.zeros((2, 4), dtype=np.uint64))


def test_gloo_two_ranks_tally_equals_single_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, local, merged = q.get(timeout=240)
        res[rank] = (local, merged)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    refs = _refs()
    single = np.stack([_tally(r, k, 0, np.arange(N_WALKERS)) for k, r in enumerate(refs)])
    for rank in range(world):
        assert np.array_equal(res[rank][1], single)
    # the shards really are different samples
    assert not np.array_equal(res[0][0], res[1][0])
    assert int(res[0][0][:, 0].sum() + res[1][0][:, 0].sum()) == 2 * N_WALKERS
