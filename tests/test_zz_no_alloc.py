"""The allocation-free sampling entry point (mcubes_sample_range_noalloc).

It serves callers that cannot allocate device memory -- hosts whose device
memory belongs to another allocator (a framework's caching pool, a fixed
arena), processes that must not grow their device footprint or stall on an
allocation once running -- by keeping its per-block partial sums and its
histogram accumulator in a static device array of the library.  These tests call it through the C ABI with device buffers the
caller owns and check its output against the context-based entry point
(mcubes_sample_range) on the same inputs, within the tolerance of the other
parity tests (1e-12 relative), on consecutive calls that reuse the shared
array: the common shape (many cubes of two or three samples, one thread per
cube), few cubes of many samples (several lanes per cube), and a grid of
exactly the array's bin limit.  The file sorts last so that a run stopping at the first failure has
run every other test first.
"""
import numpy as np
import pytest

from paper_2202_01753_gb300 import build, mcubes
from paper_2202_01753_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12
# the mixed path adds single-precision F^2 into shared memory with atomics,
# whose order varies from run to run: its histograms agree to rounding of
# single-precision sums, not bitwise (the parity tests allow 1e-3)
RTOL_HIST_MIXED = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    mcubes.lib()
    return torch


def _skewed_grid(d, nb, power):
    k = np.arange(1, nb + 1, dtype=np.float64) / nb
    B = np.tile(k ** power, (d, 1))
    B[:, -1] = 1.0
    return B


def _noalloc(torch, w, prec, it, adjust, c0, c1, d_grid, d_sums, d_hist):
    st = mcubes.mcubes_sample_range_noalloc(
        0, w.fid, w.params, w.lo, w.hi, w.ncall, w.nb, w.g_override, w.seed, prec, it, adjust, c0, c1,
        d_grid.data_ptr(), d_sums.data_ptr(), 0 if d_hist is None else d_hist.data_ptr(),
        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_context_entry_point_on_consecutive_calls(torch_cuda, prec):
    torch = torch_cuda
    w = W.cosmo6().scaled(3_000_000)
    B = _skewed_grid(w.d, w.nb, 1.4)
    ctx = mcubes.Context(0, seed=w.seed, precision=prec, nbins=w.nb)
    ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, 4)
    ctx.set_grid(B)
    m = ctx.geometry()["m"]
    d_grid = torch.tensor(B.reshape(-1), dtype=torch.float64, device="cuda")
    d_sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    d_hist = torch.zeros(w.d * w.nb, dtype=torch.float64, device="cuda")
    # two calls in a row over different iterations and cube ranges: the
    # second must not see anything the first left in the shared array
    for it, c0, c1 in [(0, 0, m), (3, m // 3, m // 3 + 12345)]:
        ref_sums, ref_C = ctx.sample_range(it, True, c0, c1)
        assert _noalloc(torch, w, prec, it, True, c0, c1, d_grid, d_sums, d_hist) == mcubes.OK
        np.testing.assert_allclose(d_sums.cpu().numpy(), ref_sums, rtol=RTOL)
        np.testing.assert_allclose(d_hist.cpu().numpy().reshape(w.d, w.nb), ref_C,
                                   rtol=RTOL if prec == "fp64" else RTOL_HIST_MIXED, atol=1e-300)
    # a non-adjusting pass needs no histogram output
    ref_sums, _ = ctx.sample_range(1, False, 0, m)
    assert _noalloc(torch, w, prec, 1, False, 0, m, d_grid, d_sums, None) == mcubes.OK
    np.testing.assert_allclose(d_sums.cpu().numpy(), ref_sums, rtol=RTOL)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array(torch_cuda):
    torch = torch_cuda
    w = W.suite("f3", 8, ncall=100_000)
    w.nb = 500                      # 8 x 500 = 4000 bins > MCUBES_NOALLOC_MAX_BINS (3072)
    d_grid = torch.tensor(_skewed_grid(w.d, w.nb, 1.0).reshape(-1), dtype=torch.float64, device="cuda")
    d_sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    d_hist = torch.zeros(w.d * w.nb, dtype=torch.float64, device="cuda")
    assert _noalloc(torch, w, "fp64", 0, True, 0, 10, d_grid, d_sums, d_hist) == mcubes.EINVAL


def test_noalloc_few_large_cubes_several_lanes(torch_cuda):
    # 64 cubes of 16384 samples: the context shares each cube among 32 lanes
    # (its iterations would even split cubes over blocks; a range pass keeps
    # one block per group of cubes), and so must the allocation-free pass
    torch = torch_cuda
    w = W.gauss3()
    B = _skewed_grid(w.d, w.nb, 1.3)
    ctx = mcubes.Context(0, seed=w.seed, nbins=w.nb, g_override=w.g_override)
    ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, 4)
    ctx.set_grid(B)
    geo = ctx.geometry()
    assert geo["m"] == 64 and geo["p"] == 16384 and geo["lanes"] > 1
    d_grid = torch.tensor(B.reshape(-1), dtype=torch.float64, device="cuda")
    d_sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    d_hist = torch.zeros(w.d * w.nb, dtype=torch.float64, device="cuda")
    for it, c0, c1 in [(0, 0, 64), (2, 5, 41)]:
        ref_sums, ref_C = ctx.sample_range(it, True, c0, c1)
        assert _noalloc(torch, w, "fp64", it, True, c0, c1, d_grid, d_sums, d_hist) == mcubes.OK
        np.testing.assert_allclose(d_sums.cpu().numpy(), ref_sums, rtol=RTOL)
        np.testing.assert_allclose(d_hist.cpu().numpy().reshape(w.d, w.nb), ref_C, rtol=RTOL, atol=1e-300)
    ctx.close()


def test_noalloc_at_exactly_the_bin_limit(torch_cuda):
    torch = torch_cuda
    w = W.suite("f3", 6, ncall=400_000)
    w.nb = 512                      # 6 x 512 = 3072 = MCUBES_NOALLOC_MAX_BINS
    B = _skewed_grid(w.d, w.nb, 0.8)
    ctx = mcubes.Context(0, seed=w.seed, nbins=w.nb)
    ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, 4)
    ctx.set_grid(B)
    m = ctx.geometry()["m"]
    d_grid = torch.tensor(B.reshape(-1), dtype=torch.float64, device="cuda")
    d_sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    d_hist = torch.zeros(w.d * w.nb, dtype=torch.float64, device="cuda")
    for it in (0, 1):
        ref_sums, ref_C = ctx.sample_range(it, True, 0, m)
        assert _noalloc(torch, w, "fp64", it, True, 0, m, d_grid, d_sums, d_hist) == mcubes.OK
        np.testing.assert_allclose(d_sums.cpu().numpy(), ref_sums, rtol=RTOL)
        np.testing.assert_allclose(d_hist.cpu().numpy().reshape(w.d, w.nb), ref_C, rtol=RTOL, atol=1e-300)
    ctx.close()
