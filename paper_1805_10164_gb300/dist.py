"""Host logic of the multi-process path (one process per GPU).

Tasks (wire, energy) and walkers are independent, and every walker's random numbers are a
function of (seed, task, walker id, draw) alone (counter-based Philox4x32-10).  The path
shards by tasks: every rank owns a disjoint set of a wire's energies (``task_partition``),
builds only their tables and walks only their walkers, so no data moves during a step.  The one
exchange step is a sum: the current of a wire is a sum over energies of independent terms,
I = sum_E w_E (f_p - f_q) T(E) with SE(I)^2 = sum_E (w_E (f_p - f_q) SE(T(E)))^2 (Eq.
iqof_t_el_db and the binomial SE of Sec. IV.B.2), so each rank's partial I and SE^2 add
(``reduce_current``), and so do the gradients of that current (``reduce_gradient``).  Walks
over disjoint walker-id ranges of the same task are also disjoint samples of one estimator, so
their per-task u64 tallies add too (``allreduce_tally``).
"""
import numpy as np

TALLY_FIELDS = 5


def task_partition(n_energies, rank, world):
    """Energy indices owned by ``rank`` when a wire's ``n_energies`` energies are split over
    ``world`` ranks: round-robin (rank r takes r, r + world, ...), so that neighbouring grid
    energies, which cost about the same, land on different ranks."""
    if world < 1 or not 0 <= rank < world or n_energies < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_energies >= 0")
    return np.arange(rank, int(n_energies), int(world), dtype=np.int64)


def _allreduce_sum(a, group=None):
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(a, dtype=np.float64)
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return a.copy()
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(a.copy()).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def reduce_current(I, se, group=None):
    """Current and standard error of every wire from each rank's partial current over its own
    energies: I = sum of the partial currents, SE = sqrt(sum of the partial SE^2)."""
    I = np.asarray(I, dtype=np.float64)
    se = np.asarray(se, dtype=np.float64)
    both = _allreduce_sum(np.concatenate([I.ravel(), (se ** 2).ravel()]), group)
    n = I.size
    return both[:n].reshape(I.shape), np.sqrt(both[n:]).reshape(se.shape)


def reduce_gradient(d_onsite, d_eta, group=None):
    """Gradient of the current w.r.t. onsite energies and dephasing rates from each rank's
    gradient over its own energies (a sum)."""
    d_onsite = np.asarray(d_onsite, dtype=np.float64)
    d_eta = np.asarray(d_eta, dtype=np.float64)
    both = _allreduce_sum(np.concatenate([d_onsite.ravel(), d_eta.ravel()]), group)
    n = d_onsite.size
    return both[:n].reshape(d_onsite.shape), both[n:].reshape(d_eta.shape)


def walker_range(rank, world, walkers_per_task):
    """Walker ids [offset, offset + count) of ``rank`` when ``walkers_per_task`` walkers per
    task are split over ``world`` ranks (strong scaling: the first ranks take the remainder)."""
    if world < 1 or not 0 <= rank < world or walkers_per_task < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, walkers_per_task >= 0")
    base, extra = divmod(int(walkers_per_task), int(world))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def weak_walker_offset(rank, step, walkers_per_task, steps_per_rank=1 << 20):
    """First walker id of ``rank``'s ``step``-th batch when every rank walks
    ``walkers_per_task`` walkers per task per step (weak scaling); ranges never overlap."""
    return (int(rank) * int(steps_per_rank) + int(step)) * int(walkers_per_task)


def allreduce_tally(counts, group=None):
    """Sum per-task tallies [n_tasks, 5] (uint64) over all ranks; returns the merged array.

    The counts travel as int64 (every field stays far below 2^63)."""
    import torch
    import torch.distributed as dist
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    if c.ndim != 2 or c.shape[1] != TALLY_FIELDS:
        raise ValueError("counts must have shape [n_tasks, 5]")
    if c.size and int(c.max()) >= 1 << 63:
        raise OverflowError("tally count does not fit in int64")
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return c.copy()
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.from_numpy(c.view(np.int64).copy()).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy().view(np.uint64).copy()
