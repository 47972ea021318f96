"""Cube-range sharding of one integral (mcubes_shard_sample/_finish) on one
GPU: several contexts, each standing for one rank, sample disjoint cube
ranges of the same iteration; the partials are gathered in rank order and
every context finishes the iteration from the same gathered array.  Each
context's trace, grid and histogram must match the oracle's whole iteration
(Alg. 3's reduction over all cubes, Alg. 2's refinement) at the FP64
tolerances of the other parity tests, and all ranks must hold the same bits.
The contexts share one stream and never wait on each other: the host
sequences the passes, as NCCL would between GPUs."""
import numpy as np
import pytest

from paper_2202_01753_gb300 import mcubes
from paper_2202_01753_gb300 import workloads as W
from paper_2202_01753_gb300.shard import cube_ranges
from test_gpu_parity import assert_parity, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(gpu_ctx_factory):
    torch = pytest.importorskip("torch")
    return torch


def sharded_run(torch, w, world, **opts):
    stream = torch.cuda.current_stream().cuda_stream
    ita = -1 if w.ita is None else w.ita
    ctxs = [mcubes.Context(0, stream=stream, nbins=w.nb, ita=ita, g_override=w.g_override, seed=w.seed, **opts)
            for _ in range(world)]
    for c in ctxs:
        c.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, w.rel_tol, w.abs_tol)
    m = ctxs[0].geometry()["m"]
    n = ctxs[0].shard_partial_len()
    parts = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(world)]
    for _ in range(w.itmax):
        for r, (c, (c0, c1)) in enumerate(zip(ctxs, cube_ranges(m, world))):
            c.shard_sample(c0, c1, parts[r].data_ptr())
        gathered = torch.cat(parts)
        for c in ctxs:
            c.shard_finish(gathered.data_ptr(), world)
    outs = []
    for c in ctxs:
        res = c.result()
        I, V = c.trace()
        outs.append(dict(res=res, I=I, V=V, grid=c.grid(), hist=c.hist(), geom=c.geometry()))
        c.close()
    return outs


def assert_ranks_identical(outs):
    for o in outs[1:]:
        assert np.array_equal(o["I"], outs[0]["I"]) and np.array_equal(o["V"], outs[0]["V"])
        assert np.array_equal(o["grid"], outs[0]["grid"])
        assert o["res"]["estimate"] == outs[0]["res"]["estimate"]


@pytest.mark.parametrize("world", [2, 3])
def test_cosmo6_shards_match_whole_iteration_oracle(torch_cuda, world):
    # histogram bins within 2e-12 (the whole-run test holds 1e-12): the ridge
    # exp(-(x1 + x2 - r)^2 / (2 0.01^2)) turns the last-bit differences of the
    # mapped x (grid edges rounded differently by the kernels and the oracle)
    # into ~1e3 times larger relative changes of F^2, and the ranks' partial
    # histograms add one more grouping of the bin sums (observed 1.005e-12)
    w = W.cosmo6().scaled(400_000, itmax=5)
    outs = sharded_run(torch_cuda, w, world)
    assert_ranks_identical(outs)
    o = oracle_run(w)
    assert_parity(w, o, outs[0], hist_tol=2e-12 * np.abs(o["hist"]) + 1e-300)


def test_suite_shards_with_plain_iterations_and_early_stop(torch_cuda):
    # two adjusting iterations then plain ones; a tolerance that stops early
    w = W.suite("f4", 5, ncall=300_000, itmax=8)
    w.ita = 2
    w.rel_tol = 2e-3
    outs = sharded_run(torch_cuda, w, 2)
    assert_ranks_identical(outs)
    o = oracle_run(w)
    assert o["iterations"] < 8            # the early stop is exercised
    assert_parity(w, o, outs[0])


def test_shards_more_ranks_than_cubes(torch_cuda):
    # 64 cubes of 16384 samples over 5 ranks (ragged 12/13) and 100 ranks
    # (most ranges empty): the same whole iteration
    w = W.gauss3()
    w.itmax = 3
    o = oracle_run(w)
    for world in (5, 100):
        outs = sharded_run(torch_cuda, w, world)
        assert_ranks_identical(outs)
        assert_parity(w, o, outs[0])


def test_onedim_shards(torch_cuda):
    w = W.suite("f2", 4, ncall=200_000, itmax=4)
    outs = sharded_run(torch_cuda, w, 2, one_dim=1)
    assert_ranks_identical(outs)
    o = oracle_run(w, one_dim=True)
    assert_parity(w, o, outs[0])


def test_shard_call_order_is_checked(torch_cuda):
    torch = torch_cuda
    w = W.cosmo6().scaled(100_000, itmax=2)
    ctx = mcubes.Context(0, seed=w.seed)
    ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax)
    n = ctx.shard_partial_len()
    assert n == 3 + w.d * w.nb
    part = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(mcubes.McubesError):            # nothing sampled yet
        ctx.shard_finish(part.data_ptr(), 1)
    m = ctx.geometry()["m"]
    with pytest.raises(mcubes.McubesError):            # range beyond m
        ctx.shard_sample(0, m + 1, part.data_ptr())
    ctx.shard_sample(0, m, part.data_ptr())
    with pytest.raises(mcubes.McubesError):            # a pass is open
        ctx.shard_sample(0, m, part.data_ptr())
    with pytest.raises(mcubes.McubesError):
        ctx.iterate(1)
    with pytest.raises(mcubes.McubesError):            # no checkpoint between sample and finish
        ctx.state_export()
    ctx.shard_finish(part.data_ptr(), 1)
    ctx.iterate(1)                                      # the last iteration, unsharded
    with pytest.raises(mcubes.McubesError):            # every iteration enqueued
        ctx.shard_sample(0, m, part.data_ptr())
    assert ctx.result()["iterations"] == 2
    ctx.close()
