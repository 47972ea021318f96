"""Cube-range sharding of one integral over several ranks (host side).

The sub-cubes [0, m) of an iteration are split into contiguous ranges, one
per rank; each rank samples its range (mcubes_shard_sample), the partials are
gathered in rank order, and every rank finishes the iteration from the same
gathered array (mcubes_shard_finish), whose kernel sums the partials in rank
order.  Alg. 3 reduces the block results and bin contributions of one
iteration and Alg. 2 refines from them; the ranges only decide which GPU
computes which part of that reduction.
"""
from __future__ import annotations


def cube_ranges(m: int, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges covering [0, m) once: rank r gets
    [r m / world, (r + 1) m / world) (floors), so sizes differ by at most one
    and a rank may get an empty range when m < world."""
    if world < 1 or m < 0:
        raise ValueError("world >= 1 and m >= 0 required")
    return [(r * m // world, (r + 1) * m // world) for r in range(world)]


def iterate_sharded(ctx, rank: int, world: int, m: int, n_iter: int, gather) -> None:
    """Runs n_iter iterations of ctx's problem as rank `rank` of `world`:
    sample this rank's cube range, gather every rank's partial (in rank
    order) with gather(partial) -> gathered, finish the iteration.
    `partial` and the gathered array are device tensors (torch, float64);
    gather is e.g. torch.distributed.all_gather_into_tensor wrapped."""
    import torch
    c0, c1 = cube_ranges(m, world)[rank]
    n = ctx.shard_partial_len()
    part = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(n_iter):
        ctx.shard_sample(c0, c1, part.data_ptr())
        gathered = gather(part)
        ctx.shard_finish(gathered.data_ptr(), world)
