"""One registration shared by several processes, one GPU each.

The measurement (Fig. 1 "measurement", > 99 % of an iteration) is
independent per particle, so each rank measures a disjoint slice of the
particles; the moment buffers are then summed over the ranks (each word has
exactly one non-zero contributor, so the integer sum is exact) and every
rank runs the prediction and the update itself.  Those are deterministic
(counter-based random numbers, integer weights and resampling), so all ranks
hold the same cloud, bit for bit equal to stepping the registration on one
GPU.  Per iteration the only exchange is that one sum of 96 N bytes.
"""
from __future__ import annotations


def slice_bounds(n_particles: int, rank: int, world: int):
    """Particles [lo, hi) measured by ``rank``: contiguous, sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    base, extra = divmod(int(n_particles), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _torch_all_reduce_sum(t):
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM)


class ShardedRegistration:
    """Steps ``reg`` (a :class:`Registration`, created identically on every
    rank) with the measurement split over ``world`` ranks.

    ``all_reduce_sum(t)`` sums the int64 tensor ``t`` over the ranks in place;
    the default is ``torch.distributed.all_reduce`` (NCCL for CUDA tensors),
    which is ordered on the current CUDA stream, the stream the context was
    created on by default.
    """

    def __init__(self, reg, rank: int, world: int, all_reduce_sum=None):
        self.reg = reg
        self.rank, self.world = int(rank), int(world)
        self.bounds = slice_bounds(reg.N, self.rank, self.world)
        self.all_reduce_sum = all_reduce_sum or _torch_all_reduce_sum
        self.moments = reg.moments()

    def step(self, n_iters: int = 1):
        lo, hi = self.bounds
        for _ in range(int(n_iters)):
            self.reg.step_measure(lo, hi)
            self.all_reduce_sum(self.moments)
            self.reg.step_update()
        return self
