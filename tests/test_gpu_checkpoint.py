"""Checkpoint and resume through the C ABI: a run stopped after k iterations,
exported, imported into a fresh context (created with other options) and
continued must reproduce the uninterrupted run bit for bit: estimate, sigma,
chi2, every iteration's estimate and variance, and the grid.  Every input of
an iteration (double-double grid, iteration index, history, flags) travels in
the checkpoint, and the launch shape is rebuilt from the stored options."""
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


def _full(make_ctx, w, precision, ita):
    ctx = _ctx(make_ctx, w, precision, ita)
    ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, w.rel_tol, w.abs_tol)
    ctx.iterate(w.itmax)
    out = ctx.result(), ctx.trace(), ctx.grid()
    ctx.close()
    return out


@pytest.mark.parametrize("name,precision,k,ita", [
    ("gauss3", "fp64", 4, -1), ("cosmo6", "fp64", 7, 5), ("corner8", "mixed", 3, -1), ("gauss3", "mixed", 1, 6),
])
def test_resume_is_bit_identical(gpu_ctx_factory, name, precision, k, ita):
    w = _problem(name)
    w.rel_tol = w.abs_tol = 0.0                       # run all iterations
    res, (I, V), B = _full(gpu_ctx_factory, w, precision, ita)

    a = _ctx(gpu_ctx_factory, w, precision, ita)
    a.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, w.rel_tol, w.abs_tol)
    a.iterate(k)
    blob = a.state_export()
    a.close()

    b = gpu_ctx_factory(seed=12345, precision="mixed" if precision == "fp64" else "fp64", nbins=64)
    b.state_import(blob)
    pr = b.problem()
    assert (pr["d"], pr["nb"], pr["itmax"], pr["enqueued"]) == (len(w.lo), w.nb, w.itmax, k)
    b.iterate(w.itmax - k)
    res2, (I2, V2), B2 = b.result(), b.trace(), b.grid()
    with pytest.raises(mcubes.McubesError) as e:
        b.iterate(1)                                  # beyond itmax
    assert e.value.status == mcubes.ESTATE
    b.close()

    for key in ("estimate", "sigma", "chi2_dof", "iterations", "converged", "status"):
        assert res2[key] == res[key], key
    assert np.array_equal(I2, I) and np.array_equal(V2, V)
    assert np.array_equal(B2, B)


def test_resume_after_convergence_stays_done(gpu_ctx_factory):
    w = _problem("gauss3")
    w.rel_tol = 1e-2                                   # converges within a few iterations
    res, (I, V), B = _full(gpu_ctx_factory, w, "fp64", -1)
    assert res["converged"] and res["iterations"] < w.itmax
    a = _ctx(gpu_ctx_factory, w)
    a.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, w.rel_tol, w.abs_tol)
    a.iterate(res["iterations"] + 1)
    blob = a.state_export()
    a.close()
    b = gpu_ctx_factory()
    b.state_import(blob)
    b.iterate(w.itmax - res["iterations"] - 1)
    res2 = b.result()
    assert res2 == res
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
