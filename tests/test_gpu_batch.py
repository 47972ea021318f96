"""The batched path (mcubes_integrate_batch): many independent integrals
iterated together by one persistent sampling launch and one refinement
launch per iteration, replayed as a CUDA graph.

Every integral draws the same Philox words as when it runs alone (its own
seed and iteration index), so batch and solo results differ only in how the
per-block partial sums are grouped: at rounding level in FP64, at the level
of single-precision histogram sums in mixed precision, amplified mildly by
the grid adaptation.  Tolerances below are those levels with margin.
"""
import numpy as np
import pytest

from paper_2202_01753_gb300 import closed_forms as CF
import oracle
from paper_2202_01753_gb300 import mcubes
from paper_2202_01753_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mix(n, seed, ncall_lo=1e4, ncall_hi=3e5, itmax=5, dmax=8):
    rng = np.random.Generator(np.random.PCG64(seed))
    ws = []
    for i in range(n):
        d = int(rng.integers(2, dmax + 1))
        fam = int(rng.choice([W.F_GAUSS, W.F_CORNER, W.F_OSC]))
        ncall = int(round(10 ** rng.uniform(np.log10(ncall_lo), np.log10(ncall_hi))))
        ws.append(W.random_integral(rng, d, fam, ncall, itmax, seed=7000 + i))
    return ws


def _req(w):
    return dict(fid=w.fid, params=w.params, lo=w.lo, hi=w.hi, ncall=w.ncall, itmax=w.itmax, rel_tol=w.rel_tol,
                abs_tol=w.abs_tol, seed=w.seed)


def _solo(make_ctx, w, precision):
    ctx = make_ctx(seed=w.seed, precision=precision)
    r = ctx.integrate(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, w.rel_tol, w.abs_tol)
    ctx.close()
    return r


# Batch against solo, about ten times the largest differences observed on
# GB300 in three runs (estimate relative to max(|I|, sigma), sigma
# relative): FP64 4.1e-16 and 6.5e-15 on the mix, 7.2e-15 and 1.1e-14 over
# every class; mixed 3.9e-8 and 3.8e-7 on the mix, 1.4e-7 and 3.3e-6 over
# every class (single-precision histogram sums grouped by segment instead
# of by block: the grids differ by their rounding, and each rebin carries
# it into the next iteration).
@pytest.mark.parametrize("precision,rtol,stol", [("fp64", 1e-13, 1e-13), ("mixed", 3e-7, 4e-6)])
def test_batch_matches_solo(gpu_ctx_factory, precision, rtol, stol):
    ws = _mix(40, seed=11)
    ctx = gpu_ctx_factory(precision=precision)
    out = ctx.integrate_batch([_req(w) for w in ws])
    ctx.close()
    for w, b in zip(ws, out):
        s = _solo(gpu_ctx_factory, w, precision)
        assert b["status"] == s["status"] == mcubes.ENOCONV
        assert b["iterations"] == s["iterations"] == w.itmax
        assert (b["g"], b["m"], b["p"]) == (s["g"], s["m"], s["p"])
        # |I|, sigma, and a floor for oscillatory integrals that cancel to
        # near zero (far below the integrands' O(1) values)
        scale = max(abs(s["estimate"]), s["sigma"], 1e-9)
        assert abs(b["estimate"] - s["estimate"]) <= rtol * scale, (w.name, b["estimate"], s["estimate"])
        assert b["sigma"] == pytest.approx(s["sigma"], rel=stol)


def _every_class(precision):
    """One integral per batched kernel class: gauss / corner / osc at every
    dimension 1..12, and in FP64 also the other batched families."""
    rng = np.random.Generator(np.random.PCG64(15))
    ws = [W.random_integral(rng, d, fam, 20_000, 3, seed=7500 + 3 * d + k)
          for d in range(1, 13) for k, fam in enumerate((W.F_GAUSS, W.F_CORNER, W.F_OSC))]
    if precision == "fp64":
        ws += [W.suite(f, d, ncall=20_000, itmax=3, seed=7600 + d) for f in ("f2", "f5", "f6") for d in (1, 5)]
        ws.append(W.cosmo6(seed=7700).scaled(30_000, itmax=3))
    return ws


@pytest.mark.parametrize("precision,rtol,stol", [("fp64", 1e-13, 1e-13), ("mixed", 1.5e-6, 3e-5)])
def test_batch_every_class_matches_solo(gpu_ctx_factory, precision, rtol, stol):
    """All class kernels of one iteration run as concurrent graph branches;
    each integral still matches its solo run (disjoint segments, no
    cross-talk between the classes)."""
    ws = _every_class(precision)
    ctx = gpu_ctx_factory(precision=precision)
    out = ctx.integrate_batch([_req(w) for w in ws])
    ctx.close()
    for w, b in zip(ws, out):
        s = _solo(gpu_ctx_factory, w, precision)
        assert b["status"] == s["status"], w.name
        assert b["iterations"] == s["iterations"] == 3
        scale = max(abs(s["estimate"]), s["sigma"], 1e-9)
        assert abs(b["estimate"] - s["estimate"]) <= rtol * scale, (w.name, b["estimate"], s["estimate"])
        assert b["sigma"] == pytest.approx(s["sigma"], rel=stol), w.name


def _oracle_set():
    """Every batched family at several dimensions (and the six-dimensional
    power-law x lognormal x ridge integrand), small enough for the oracle."""
    rng = np.random.Generator(np.random.PCG64(12))
    ws = [W.random_integral(rng, d, fam, 60_000, 4, seed=7800 + 10 * d + k)
          for d in (2, 5, 9) for k, fam in enumerate((W.F_GAUSS, W.F_CORNER, W.F_OSC))]
    ws += [W.suite(f, d, ncall=60_000, itmax=4, seed=7900 + d) for f in ("f2", "f5", "f6") for d in (3, 7)]
    ws.append(W.cosmo6(seed=7950).scaled(120_000, itmax=4))
    return ws


def test_batch_fp64_traces_match_oracle(gpu_ctx_factory):
    """Batched FP64 integrals against the oracle at the single-integral
    path's tolerances (test_gpu_parity): each iteration's estimate within
    1e-12 of its conditioning scale and its variance within 1e-12 (1e-10 for
    the oscillatory family), the final grid within 1e-12, chi^2 within
    1e-9, and the last histogram within 1e-11 of each axis's largest bin.
    The histogram sums F^2, whose relative error is the mapped points'
    last-bit differences (grids equal to ~1e-16, not bit for bit) times the
    integrand's sensitivity: f6's F^2 = exp(2 sum c_i x_i) multiplies them
    by 2 sum c_i ~ 70 (observed 3.1e-12 of the axis's largest bin; corner9's
    bins 3e-12 relative to themselves).  The batch draws each
    integral's own samples; only the grouping of the partial sums into
    segments differs from the oracle's compensated sums."""
    from test_gpu_parity import cond_scale
    ws = _oracle_set()
    ctx = gpu_ctx_factory()
    out = ctx.integrate_batch([_req(w) for w in ws])
    for i, (w, b) in enumerate(zip(ws, out)):
        o = oracle.integrate(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, nb=w.nb, seed=w.seed)
        I, V, B, C = ctx.batch_trace(i, w.d)
        assert b["iterations"] == o["iterations"] == len(I), w.name
        assert (b["g"], b["m"], b["p"]) == (o["g"], o["m"], o["p"])
        scale = cond_scale(w, o)
        vtol = 1e-10 if w.fid == W.F_OSC else 1e-12
        np.testing.assert_allclose(I, o["trace_I"], rtol=0, atol=1e-12 * scale, err_msg=w.name)
        np.testing.assert_allclose(V, o["trace_var"], rtol=vtol, atol=0, err_msg=w.name)
        np.testing.assert_allclose(B, o["grid"], rtol=0, atol=1e-12, err_msg=w.name)
        rowmax = np.abs(o["hist"]).max(axis=1, keepdims=True)
        worst = float(np.max(np.abs(C - o["hist"]) / rowmax))
        assert worst <= 1e-11, (w.name, worst, np.unravel_index(np.argmax(np.abs(C - o["hist"]) / rowmax), C.shape))
        assert b["estimate"] == pytest.approx(o["estimate"], abs=1e-12 * scale), w.name
        assert b["sigma"] == pytest.approx(o["sigma"], rel=vtol), w.name
        assert b["chi2_dof"] == pytest.approx(o["chi2_dof"], rel=1e-9, abs=1e-12), w.name
    ctx.close()


def test_batch_early_convergence_per_integral(gpu_ctx_factory):
    ws = _mix(30, seed=13, ncall_lo=3e4, ncall_hi=3e5, itmax=12)
    for i, w in enumerate(ws):
        w.rel_tol = [1e-2, 3e-3, 1e-3][i % 3]
    ctx = gpu_ctx_factory()
    out = ctx.integrate_batch([_req(w) for w in ws])
    ctx.close()
    its = set()
    for w, b in zip(ws, out):
        s = _solo(gpu_ctx_factory, w, "fp64")
        assert b["iterations"] == s["iterations"]
        assert b["converged"] == s["converged"]
        # the FP64 batch-against-solo bound of test_batch_matches_solo
        scale = max(abs(s["estimate"]), s["sigma"], 1e-9)
        assert abs(b["estimate"] - s["estimate"]) <= 1e-13 * scale, (w.name, b["estimate"], s["estimate"])
        its.add(b["iterations"])
        if b["converged"]:
            assert b["sigma"] <= w.rel_tol * abs(b["estimate"])
            assert abs(b["estimate"] - CF.exact(w)) < 6 * b["sigma"]
    assert len(its) > 1   # integrals left the batch at different iterations


def test_batch_rejects_invalid_request(gpu_ctx_factory):
    ws = _mix(3, seed=14)
    reqs = [_req(w) for w in ws]
    reqs[1]["lo"] = reqs[1]["hi"]
    ctx = gpu_ctx_factory()
    with pytest.raises(mcubes.McubesError) as e:
        ctx.integrate_batch(reqs)
    assert e.value.status == mcubes.EINVAL
    # the context is still usable
    out = ctx.integrate_batch([_req(w) for w in ws])
    assert all(r["status"] == mcubes.ENOCONV for r in out)
    ctx.close()


def test_batch_4096_uneven_integrals(gpu_ctx_factory):
    """The batched configuration's shape (4096 integrals, d in 2..10, three
    families, ncall log-uniform) scaled to 1e4..1e5 calls: every integral
    finishes and agrees with its closed form."""
    ws = W.batch4096(n=4096, itmax=4)
    ws = [w.scaled(min(w.ncall, 100_000)) for w in ws]
    ctx = gpu_ctx_factory(precision="mixed")
    out = ctx.integrate_batch([_req(w) for w in ws])
    ctx.close()
    z = []
    for w, b in zip(ws, out):
        assert b["status"] == mcubes.ENOCONV and b["iterations"] == 4
        z.append((b["estimate"] - CF.exact(w)) / b["sigma"])
    z = np.abs(np.array(z))
    assert np.mean(z < 3) > 0.97
