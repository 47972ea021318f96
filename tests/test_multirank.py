"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2): every
rank integrates its own independent copy of the workload, and the job's
throughput is all ranks' samples over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    args = type("A", (), {"config": "cosmo6", "ncall": None})()
    w = bench.workload(args, rank)
    # rank r is slower by 10 ms and does 100 + r samples
    value, max_ms, total = bench.aggregate_ranks(50.0 + 10.0 * rank, 100 + rank, "cpu")
    out.put((rank, w.seed, value, max_ms, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_aggregate_max_time_and_sum_of_samples():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seed0, v0, m0, n0), (r1, seed1, v1, m1, n1) = res
    assert seed0 != seed1                 # independent integrals per rank
    assert m0 == m1 == 60.0               # slowest rank's time everywhere
    assert n0 == n1 == 201.0              # all ranks' samples
    assert v0 == pytest.approx(201.0 / 0.060)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"config": "cosmo6", "ncall": None, "steps": 1, "warmup": 0})()
    assert bench.reference_arm(args) == 0
    assert capsys.readouterr().out == ""
