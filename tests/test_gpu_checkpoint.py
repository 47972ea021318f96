"""Checkpoint and resume through the C ABI: a run stopped after k iterations,
exported, imported into a fresh context (created with other options) and
continued.  Every input of an iteration (double-double grid, iteration
index, history, flags) travels in the checkpoint and the launch shape is
rebuilt from the stored options, so the checkpoint round-trips byte for byte
and a run resumed after its adjusting iterations reproduces the
uninterrupted run bit for bit (estimate, sigma, chi2, every iteration's
estimate and variance, the grid)."""
import numpy as np
import pytest

from paper_2202_01753_gb300 import mcubes
from paper_2202_01753_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(name):
    make = {"gauss3": W.gauss3, "cosmo6": W.cosmo6, "corner8": W.corner8}[name]
    ncall = {"gauss3": 200_000, "cosmo6": 300_000, "corner8": 400_000}[name]
    return make().scaled(ncall, itmax=10)


def _ctx(make_ctx, w, precision="fp64", ita=-1):
    return make_ctx(seed=w.seed, precision=precision, ita=ita, nbins=w.nb, g_override=w.g_override)


def _resume(make_ctx, w, precision, ita, k):
    """Runs k iterations, exports; continues that context to itmax (the
    uninterrupted run) and a fresh context from the checkpoint (the resumed
    run).  Returns both (result, trace, grid)."""
    a = _ctx(make_ctx, w, precision, ita)
    a.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, w.rel_tol, w.abs_tol)
    a.iterate(k)
    blob = a.state_export()
    a.iterate(w.itmax - k)
    full = a.result(), a.trace(), a.grid()
    a.close()
    b = make_ctx(seed=12345, precision="mixed" if precision == "fp64" else "fp64", nbins=64)
    b.state_import(blob)
    pr = b.problem()
    assert (pr["d"], pr["nb"], pr["itmax"], pr["enqueued"]) == (len(w.lo), w.nb, w.itmax, k)
    b.iterate(w.itmax - k)
    resumed = b.result(), b.trace(), b.grid()
    with pytest.raises(mcubes.McubesError) as e:
        b.iterate(1)                                  # beyond itmax
    assert e.value.status == mcubes.ESTATE
    b.close()
    return full, resumed


@pytest.mark.parametrize("name,precision,k,ita", [
    ("gauss3", "fp64", 4, 4), ("cosmo6", "fp64", 7, 5), ("corner8", "mixed", 3, 2), ("gauss3", "mixed", 6, 6),
])
def test_resume_is_bit_identical(gpu_ctx_factory, name, precision, k, ita):
    """Resumed after the last adjusting iteration (k >= ita): every later
    iteration samples the restored grid with fixed-order reductions, so the
    resumed run equals the uninterrupted one bit for bit."""
    w = _problem(name)
    w.rel_tol = w.abs_tol = 0.0                       # run all iterations
    (res, (I, V), B), (res2, (I2, V2), B2) = _resume(gpu_ctx_factory, w, precision, ita, k)
    for key in ("estimate", "sigma", "chi2_dof", "iterations", "converged", "status"):
        assert res2[key] == res[key], key
    assert np.array_equal(I2, I) and np.array_equal(V2, V)
    assert np.array_equal(B2, B)


@pytest.mark.parametrize("name,precision,k", [("gauss3", "fp64", 3), ("cosmo6", "fp64", 5), ("corner8", "mixed", 2)])
def test_resume_with_adjusting_iterations(gpu_ctx_factory, name, precision, k):
    """Resumed before the adjusting iterations end: the per-block histograms
    add F^2 with shared-memory atomics in an unspecified order, so adjusting
    iterations are reproducible (resumed or not) to the rounding of those
    sums; the resumed run agrees with the uninterrupted one to that level
    (FP64: 1e-12 relative; mixed, single-precision histograms: 1e-7)."""
    w = _problem(name)
    w.rel_tol = w.abs_tol = 0.0
    (res, (I, V), B), (res2, (I2, V2), B2) = _resume(gpu_ctx_factory, w, precision, -1, k)
    tol = 1e-12 if precision == "fp64" else 1e-7
    assert np.array_equal(I2[:k], I[:k]) and np.array_equal(V2[:k], V[:k])   # the restored history
    np.testing.assert_allclose(I2, I, rtol=tol)
    np.testing.assert_allclose(V2, V, rtol=100 * tol)
    np.testing.assert_allclose(B2, B, rtol=0, atol=100 * tol)
    assert res2["estimate"] == pytest.approx(res["estimate"], rel=tol)


def test_resume_after_convergence_stays_done(gpu_ctx_factory):
    """A checkpoint taken after convergence: the imported run is done, later
    iterations are skipped and the result is the exported one, bit for bit."""
    w = _problem("gauss3")
    w.rel_tol = 1e-2                                   # converges within a few iterations
    a = _ctx(gpu_ctx_factory, w)
    a.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, w.rel_tol, w.abs_tol)
    a.iterate(6)
    res, B = a.result(), a.grid()
    assert res["converged"] and res["iterations"] < 6
    blob = a.state_export()
    a.close()
    b = gpu_ctx_factory()
    b.state_import(blob)
    b.iterate(w.itmax - 6)
    assert b.result() == res
    assert np.array_equal(b.grid(), B)
    b.close()


def test_checkpoint_round_trip_is_stable(gpu_ctx_factory):
    w = _problem("gauss3")
    a = _ctx(gpu_ctx_factory, w)
    a.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax)
    a.iterate(3)
    blob = a.state_export()
    b = gpu_ctx_factory()
    b.state_import(blob)
    assert b.state_export() == blob                    # export(import(x)) == x
    a.close()
    b.close()


def test_bad_checkpoints_are_rejected(gpu_ctx_factory):
    w = _problem("gauss3")
    a = _ctx(gpu_ctx_factory, w)
    with pytest.raises(mcubes.McubesError) as e:
        a.state_export()                               # no problem yet
    assert e.value.status == mcubes.ESTATE
    a.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax)
    a.iterate(2)
    blob = bytearray(a.state_export())
    for bad in (bytes(blob[:-1]), bytes(blob[:40]), b"X" + bytes(blob[1:]), bytes(blob) + b"\0"):
        b = gpu_ctx_factory()
        with pytest.raises(mcubes.McubesError) as e:
            b.state_import(bad)
        assert e.value.status == mcubes.EINVAL
        with pytest.raises(mcubes.McubesError) as e:
            b.iterate(1)                               # a failed import leaves no problem
        assert e.value.status == mcubes.ESTATE
        b.close()
    a.close()
