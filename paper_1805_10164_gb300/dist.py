"""Host logic of the multi-process path (one process per GPU).

Tasks and walkers are independent, and every walker's random numbers are a function of
(seed, task, walker id, draw) alone (counter-based Philox4x32-10), so walks over disjoint
walker-id ranges are disjoint samples of the same estimator and their tallies add.  The only
exchange step of the path is therefore the sum of the per-task u64 tallies (walkers, absorbed
at L, absorbed at R, truncated, steps), which this module performs with torch.distributed.
"""
import numpy as np

TALLY_FIELDS = 5


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
