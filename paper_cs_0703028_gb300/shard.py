"""Ray-sharded Monte-Carlo runs over several ranks (one process per GPU).

Section 3 of the paper averages the effect of all rays on the host.  The
estimate partitions by ray range: rank r traces rays [r R, (r + 1) R) of an
N R-ray estimate (the Philox counters make each ray the same wherever it runs,
and every rank builds the same kappa table), so the only exchange is one
binary64 all-reduce (sum) of each rank's per-cell absorbed power together with
its emitted and escaped totals.  The energy balance is then formed on the
combined tally (``rt_tally`` on the combined buffers, or ``energy_residual``).
Enclosures of a batched run partition the same way with no exchange at all.
"""
from __future__ import annotations


def ray_range(rank: int, world: int, rays_per_rank: int):
    """Weak scaling: (first ray, rays of this rank, rays of the whole estimate)."""
    if not (0 <= rank < world) or rays_per_rank < 0:
        raise ValueError(f"bad partition: rank {rank} of {world}, {rays_per_rank} rays per rank")
    return rank * rays_per_rank, rays_per_rank, world * rays_per_rank


def combine_tally(tally, group=None):
    """Sum the ranks' tallies in place: one all-reduce of ``tally.flat`` (binary64,
    [absorbed | emitted, absorbed total, escaped, residual]) and one of the step
    counter.  The absorbed total and residual slots are summed too; they are
    recomputed from the combined buffers by ``rt_tally`` (or ``energy_residual``)."""
    import torch.distributed as dist
    dist.all_reduce(tally.flat, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(tally.steps, op=dist.ReduceOp.SUM, group=group)
    return tally


def energy_residual(absorbed, emitted: float, escaped: float) -> float:
    """|emitted - sum(absorbed) - escaped| / emitted of a (combined) tally on the host."""
    import math
    tot = math.fsum(float(v) for v in absorbed)
    return abs(emitted - tot - escaped) / emitted if emitted else 0.0
