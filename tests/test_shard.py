"""Host side of the cube-range sharding of one integral (no GPU): the
ranges every rank samples, and the gather-then-combine protocol on CPU ranks
(gloo, world size 2).  Alg. 3 reduces one iteration's block results and bin
contributions; sharding only decides which rank computes which part of that
sum, so the ranges must cover the sub-cubes exactly once and every rank must
combine the same gathered partials in the same (rank) order."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2202_01753_gb300.shard import cube_ranges

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("m,world", [(64, 2), (47_045_881, 8), (7, 3), (3, 8), (0, 2), (1, 1), (101, 4)])
def test_ranges_cover_every_cube_once(m, world):
    r = cube_ranges(m, world)
    assert len(r) == world
    assert r[0][0] == 0 and r[-1][1] == m
    for (a0, a1), (b0, b1) in zip(r, r[1:]):
        assert a1 == b0                       # contiguous, no gap or overlap
    sizes = [b - a for a, b in r]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    assert sum(sizes) == m


def test_ranges_reject_bad_world():
    with pytest.raises(ValueError):
        cube_ranges(10, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_partial(rank, m, world, d, nb):
    """Synthetic partial of one rank: a function of the global cube indices
    it owns only (as a real rank's sums are), so that the union over ranks
    does not depend on the world size."""
    c0, c1 = cube_ranges(m, world)[rank]
    cubes = np.arange(c0, c1, dtype=np.float64)
    vals = np.sin(0.37 * cubes) * 1e3 + 1e-3 * cubes
    head = np.array([vals.sum(), (vals ** 2).sum(), np.abs(vals).sum()])
    hist = np.zeros(d * nb)
    np.add.at(hist, (np.arange(c0, c1) * 7919) % (d * nb), vals ** 2)
    return np.concatenate([head, hist])


def _combine_in_rank_order(gathered):
    out = gathered[0].copy()
    for r in range(1, gathered.shape[0]):
        out += gathered[r]
    return out


def _worker(rank, world, port, m, d, nb, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    part = torch.from_numpy(_rank_partial(rank, m, world, d, nb))
    gathered = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(gathered, part)
    comb = _combine_in_rank_order(torch.stack(gathered).numpy())
    q.put((rank, comb.tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_gather_and_combine_identically():
    m, d, nb = 1001, 3, 50        # ragged: 500 + 501 cubes
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, m, d, nb, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1]                       # every rank holds the same bits
    comb = np.frombuffer(res[0])
    whole = _rank_partial(0, m, 1, d, nb)         # the same cubes on one rank
    np.testing.assert_allclose(comb, whole, rtol=1e-13, atol=1e-9)
