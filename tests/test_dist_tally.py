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


# ---- task partition: ranks own disjoint energies; the current and its gradient are sums ----

MU = (0.6, -0.4, 0.3)
N_PART = 20000


def _part_wire():
    return inputs.small_wire(9, W=2, L=3, n_energy=5, eta=0.25, e_lo=-1.7, e_hi=1.7)


def _partial(w, idx):
    """Oracle current, SE and exact gradient over the energies ``idx`` of wire ``w``."""
    from oracle import adjoint, current, pipeline
    E, wE = w.energy[idx], w.energy_weight[idx]
    T, se = [], []
    gV = np.zeros(w.W * w.L)
    gE = np.zeros(w.W * w.L)
    df = current.fermi(E, MU[0], MU[2]) - current.fermi(E, MU[1], MU[2])
    for k, Ek in zip(idx, E):
        r = pipeline.task_reference(w.onsite, w.eta, w.t, Ek, with_direct=False)
        r["W"] = w.W
        c = _tally(r, int(k), 0, np.arange(N_PART))
        Tk, sk = current.mc_transmission(r["tab"]["c"][0], c[2], c[0])
        T.append(Tk)
        se.append(sk)
        _, dV, dEta = adjoint.transmission_gradient(w.onsite, w.eta, w.t, Ek, 0, 1)
        j = list(E).index(Ek)
        gV += wE[j] * df[j] * dV.reshape(-1)
        gE += wE[j] * df[j] * dEta.reshape(-1)
    I, dI = current.current(E, wE, np.array(T), np.array(se), *MU)
    return I, dI, gV, gE


def _part_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _part_wire()
        idx = ndist.task_partition(len(w.energy), rank, world)
        I, dI, gV, gE = _partial(w, idx)
        It, st = ndist.reduce_current(np.array([I]), np.array([dI]))
        gVt, gEt = ndist.reduce_gradient(gV, gE)
        q.put((rank, idx, It, st, gVt, gEt))
    finally:
        dist.destroy_process_group()


def test_task_partition_covers_every_energy_once():
    for world in (1, 2, 3, 8):
        for n in (0, 1, 5, 256):
            parts = [ndist.task_partition(n, r, world) for r in range(world)]
            assert np.array_equal(np.sort(np.concatenate(parts)), np.arange(n))
    with pytest.raises(ValueError):
        ndist.task_partition(4, 2, 2)


def test_gloo_two_ranks_task_partition_current_and_gradient():
    """Each rank builds and walks only its own energies; one all-reduce of the partial current,
    SE^2 and gradient reproduces the single-process result over all energies."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_part_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, idx, It, st, gVt, gEt = q.get(timeout=240)
        res[rank] = (idx, It, st, gVt, gEt)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _part_wire()
    assert not set(res[0][0]) & set(res[1][0])
    I, dI, gV, gE = _partial(w, np.arange(len(w.energy)))
    for rank in range(world):
        _, It, st, gVt, gEt = res[rank]
        assert np.allclose(It, I, rtol=1e-13, atol=1e-15)
        assert np.allclose(st, dI, rtol=1e-13, atol=1e-15)
        assert np.allclose(gVt, gV, rtol=1e-12, atol=1e-14)
        assert np.allclose(gEt, gE, rtol=1e-12, atol=1e-14)
