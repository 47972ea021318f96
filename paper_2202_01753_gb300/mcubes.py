"""Thin ctypes binding of the C ABI in include/mcubes.h.

Argument marshalling only: every step of an integration runs in the CUDA
kernels of libmcubes.  Functions keep the C names.  Loading fails loudly if
the library has not been built (``python -m paper_2202_01753_gb300.build``);
there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ENOCONV, ETIMEOUT, ESTATE = range(8)
FP64, MIXED = 0, 1
DMAX, NBMAX, PARAMS_MAX, ITMAX_MAX = 12, 1024, 32, 4096

EXPORTED = [
    "mcubes_default_opts", "mcubes_create", "mcubes_create_on_stream", "mcubes_set_opts",
    "mcubes_destroy", "mcubes_strerror", "mcubes_last_cuda_error", "mcubes_integrate",
    "mcubes_integrate_batch", "mcubes_setup", "mcubes_iterate", "mcubes_result_get",
    "mcubes_trace_get", "mcubes_grid_get", "mcubes_grid_set", "mcubes_hist_get",
    "mcubes_sample_range", "mcubes_geometry_get", "mcubes_timing_reset", "mcubes_timing_get",
    "mcubes_sample_range_noalloc", "mcubes_server_create", "mcubes_server_destroy", "mcubes_server_submit",
    "mcubes_server_step", "mcubes_server_poll", "mcubes_server_stats", "mcubes_server_run_stream",
    "mcubes_selftest_fxmath", "mcubes_state_size", "mcubes_state_export", "mcubes_state_import",
    "mcubes_problem_get", "mcubes_get_opts", "mcubes_tables_set", "mcubes_server_set_step_iterations",
    "mcubes_selftest_rebin", "mcubes_shard_partial_len", "mcubes_shard_sample", "mcubes_shard_finish",
    "mcubes_server_set_escalation", "mcubes_batch_trace_get", "mcubes_server_set_retry_sized",
]


class mcubes_opts(ctypes.Structure):
    _fields_ = [("nbins", ctypes.c_int), ("ita", ctypes.c_int), ("g_override", ctypes.c_longlong),
                ("alpha", ctypes.c_double), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int),
                ("lanes_per_cube", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("one_dim", ctypes.c_int)]


class mcubes_table(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 2), ("lo", ctypes.c_double * 2),
                ("hi", ctypes.c_double * 2), ("values", ctypes.POINTER(ctypes.c_double))]


class mcubes_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("sigma", ctypes.c_double), ("chi2_dof", ctypes.c_double),
                ("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("samples_per_iter", ctypes.c_longlong), ("g", ctypes.c_longlong),
                ("m", ctypes.c_longlong), ("p", ctypes.c_longlong), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mcubes_request(ctypes.Structure):
    _fields_ = [("integrand_id", ctypes.c_int), ("params", ctypes.POINTER(ctypes.c_double)),
                ("nparams", ctypes.c_int), ("d", ctypes.c_int), ("lo", ctypes.POINTER(ctypes.c_double)),
                ("hi", ctypes.POINTER(ctypes.c_double)), ("ncall", ctypes.c_longlong),
                ("itmax", ctypes.c_int), ("rel_tol", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.lib_path()


def lib():
    """The loaded libmcubes (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libmcubes is not built ({path} missing): run "
                                   "`python -m paper_2202_01753_gb300.build` on a machine with nvcc")
            h = ctypes.CDLL(path)
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            ctx = ctypes.c_void_p
            ll = ctypes.c_longlong
            sig = {
                "mcubes_default_opts": (None, [P(mcubes_opts)]),
                "mcubes_create": (ctypes.c_int, [P(ctx), ctypes.c_int, P(mcubes_opts)]),
                "mcubes_create_on_stream": (ctypes.c_int, [P(ctx), ctypes.c_int, P(mcubes_opts), ctypes.c_void_p]),
                "mcubes_set_opts": (ctypes.c_int, [ctx, P(mcubes_opts)]),
                "mcubes_destroy": (ctypes.c_int, [ctx]),
                "mcubes_strerror": (ctypes.c_char_p, [ctypes.c_int]),
                "mcubes_last_cuda_error": (ctypes.c_char_p, [ctx]),
                "mcubes_integrate": (ctypes.c_int, [ctx, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp, ll,
                                                    ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                    P(mcubes_result)]),
                "mcubes_integrate_batch": (ctypes.c_int, [ctx, ctypes.c_int, P(mcubes_request), P(mcubes_result)]),
                "mcubes_setup": (ctypes.c_int, [ctx, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp, ll,
                                                ctypes.c_int, ctypes.c_double, ctypes.c_double]),
                "mcubes_iterate": (ctypes.c_int, [ctx, ctypes.c_int]),
                "mcubes_result_get": (ctypes.c_int, [ctx, P(mcubes_result)]),
                "mcubes_trace_get": (ctypes.c_int, [ctx, dp, dp, ctypes.c_int, P(ctypes.c_int)]),
                "mcubes_grid_get": (ctypes.c_int, [ctx, dp, ll]),
                "mcubes_grid_set": (ctypes.c_int, [ctx, dp, ll]),
                "mcubes_hist_get": (ctypes.c_int, [ctx, dp, ll]),
                "mcubes_sample_range": (ctypes.c_int, [ctx, ctypes.c_uint, ctypes.c_int, ll, ll, dp, dp]),
                "mcubes_geometry_get": (ctypes.c_int, [ctx, P(ll), P(ll), P(ll), P(ctypes.c_int),
                                                       P(ctypes.c_int)]),
                "mcubes_timing_reset": (ctypes.c_int, [ctx, ctypes.c_int]),
                "mcubes_timing_get": (ctypes.c_int, [ctx, dp, P(ctypes.c_int), dp, P(ctypes.c_int)]),
                "mcubes_server_create": (ctypes.c_int, [P(ctypes.c_void_p), ctx, ll, ctypes.c_int]),
                "mcubes_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
                "mcubes_server_submit": (ctypes.c_int, [ctypes.c_void_p, P(mcubes_request), ll]),
                "mcubes_server_step": (ctypes.c_int, [ctypes.c_void_p, P(ctypes.c_int)]),
                "mcubes_server_set_step_iterations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
                "mcubes_server_set_escalation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ll]),
                "mcubes_server_set_retry_sized": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                                                  ll]),
                "mcubes_server_poll": (ctypes.c_int, [ctypes.c_void_p, P(ll), P(mcubes_result), ctypes.c_int,
                                                      P(ctypes.c_int)]),
                "mcubes_server_stats": (ctypes.c_int, [ctypes.c_void_p, P(ll), P(ll), P(ll), P(ll), P(ll)]),
                "mcubes_server_run_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, P(mcubes_request), dp,
                                                            P(mcubes_result), dp, dp]),
                "mcubes_get_opts": (ctypes.c_int, [ctx, P(mcubes_opts)]),
                "mcubes_tables_set": (ctypes.c_int, [ctx, ctypes.c_int, P(mcubes_table)]),
                "mcubes_state_size": (ctypes.c_int, [ctx, P(ll)]),
                "mcubes_state_export": (ctypes.c_int, [ctx, ctypes.c_void_p, ll]),
                "mcubes_state_import": (ctypes.c_int, [ctx, ctypes.c_void_p, ll]),
                "mcubes_problem_get": (ctypes.c_int, [ctx, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                                      P(ctypes.c_int), P(ctypes.c_int)]),
                "mcubes_selftest_fxmath": (ctypes.c_int, [ctypes.c_int, ll, ctypes.c_void_p, ctypes.c_void_p,
                                                          ctypes.c_void_p]),
                "mcubes_selftest_rebin": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
                "mcubes_batch_trace_get": (ctypes.c_int, [ctx, ctypes.c_int, dp, dp, ctypes.c_int, P(ctypes.c_int),
                                                          dp, dp]),
                "mcubes_shard_partial_len": (ctypes.c_int, [ctx, P(ll)]),
                "mcubes_shard_sample": (ctypes.c_int, [ctx, ll, ll, ctypes.c_void_p]),
                "mcubes_shard_finish": (ctypes.c_int, [ctx, ctypes.c_void_p, ctypes.c_int]),
                "mcubes_sample_range_noalloc": (ctypes.c_int, [
                    ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp, ll, ctypes.c_int, ll,
                    ctypes.c_uint64, ctypes.c_int, ctypes.c_uint, ctypes.c_int, ll, ll, ctypes.c_void_p,
                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _lib = h
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def mcubes_sample_range_noalloc(device, fid, params, lo, hi, ncall, nbins, g_override, seed, precision, it,
                                adjust, cube_begin, cube_end, d_grid, d_sums, d_hist, stream=0):
    """Binding of the allocation-free sampling pass: d_grid, d_sums and d_hist
    are device addresses (ints) owned by the caller; returns the status."""
    p, lo, hi = _f64(params), _f64(lo), _f64(hi)
    if isinstance(precision, str):
        precision = {"fp64": FP64, "mixed": MIXED}[precision]
    return lib().mcubes_sample_range_noalloc(device, fid, _dp(p), len(p), len(lo), _dp(lo), _dp(hi), int(ncall),
                                             nbins, int(g_override), int(seed), precision, it, int(adjust),
                                             int(cube_begin), int(cube_end), ctypes.c_void_p(d_grid),
                                             ctypes.c_void_p(d_sums), ctypes.c_void_p(d_hist),
                                             ctypes.c_void_p(stream))


class McubesError(RuntimeError):
    def __init__(self, status, where, detail=""):
        msg = lib().mcubes_strerror(status).decode()
        super().__init__(f"{where}: {msg} ({status}){' ' + detail if detail else ''}")
        self.status = status


def mcubes_default_opts() -> mcubes_opts:
    o = mcubes_opts()
    lib().mcubes_default_opts(ctypes.byref(o))
    return o


def make_opts(**kw) -> mcubes_opts:
    o = mcubes_default_opts()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "mixed": MIXED}[v]
        setattr(o, k, v)
    return o


class Context:
    """One mcubes_ctx: a device, a stream and the buffers of one integral."""

    def __init__(self, device: int = 0, stream: int | None = None, **opts):
        self._h = ctypes.c_void_p()
        o = make_opts(**opts)
        if stream is None:
            st = lib().mcubes_create(ctypes.byref(self._h), device, ctypes.byref(o))
        else:
            st = lib().mcubes_create_on_stream(ctypes.byref(self._h), device, ctypes.byref(o),
                                               ctypes.c_void_p(stream))
        if st != OK:
            raise McubesError(st, "mcubes_create")
        self.d = self.nb = 0
        self.opts = o

    # -- lifecycle -----------------------------------------------------
    def close(self):
        if self._h:
            lib().mcubes_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where, ok=(OK,)):
        if st not in ok:
            detail = lib().mcubes_last_cuda_error(self._h).decode() if st == ECUDA else ""
            raise McubesError(st, where, detail)
        return st

    def set_opts(self, **opts):
        o = make_opts(**opts)
        self._check(lib().mcubes_set_opts(self._h, ctypes.byref(o)), "mcubes_set_opts")
        self.opts = o

    # -- whole integrations --------------------------------------------
    def integrate(self, fid, params, lo, hi, ncall, itmax, rel_tol=0.0, abs_tol=0.0):
        p, lo, hi = _f64(params), _f64(lo), _f64(hi)
        res = mcubes_result()
        st = lib().mcubes_integrate(self._h, fid, _dp(p), len(p), len(lo), _dp(lo), _dp(hi), int(ncall), itmax,
                                    rel_tol, abs_tol, ctypes.byref(res))
        self._check(st, "mcubes_integrate", ok=(OK, ENOCONV))
        self.d, self.nb = len(lo), self.opts.nbins
        return res.as_dict()

    def integrate_batch(self, requests):
        """requests: iterable of dicts with keys fid, params, lo, hi, ncall, itmax, rel_tol, abs_tol, seed."""
        reqs = list(requests)
        keep = []
        arr = (mcubes_request * len(reqs))()
        for i, r in enumerate(reqs):
            p, lo, hi = _f64(r["params"]), _f64(r["lo"]), _f64(r["hi"])
            keep += [p, lo, hi]
            arr[i] = mcubes_request(r["fid"], _dp(p), len(p), len(lo), _dp(lo), _dp(hi), int(r["ncall"]),
                                    int(r["itmax"]), float(r.get("rel_tol", 0.0)), float(r.get("abs_tol", 0.0)),
                                    int(r.get("seed", 0)))
        outs = (mcubes_result * len(reqs))()
        self._check(lib().mcubes_integrate_batch(self._h, len(reqs), arr, outs), "mcubes_integrate_batch")
        return [o.as_dict() for o in outs]

    # -- step-level -------------------------------------------------------
    def setup(self, fid, params, lo, hi, ncall, itmax, rel_tol=0.0, abs_tol=0.0):
        p, lo, hi = _f64(params), _f64(lo), _f64(hi)
        self._check(lib().mcubes_setup(self._h, fid, _dp(p), len(p), len(lo), _dp(lo), _dp(hi), int(ncall), itmax,
                                       rel_tol, abs_tol), "mcubes_setup")
        self.d, self.nb = len(lo), self.opts.nbins

    def iterate(self, n_iter=1):
        self._check(lib().mcubes_iterate(self._h, n_iter), "mcubes_iterate")

    def result(self):
        res = mcubes_result()
        self._check(lib().mcubes_result_get(self._h, ctypes.byref(res)), "mcubes_result_get",
                    ok=(OK, ENOCONV, ENONFINITE))
        return res.as_dict()

    def trace(self, cap=ITMAX_MAX):
        I = np.zeros(cap)
        V = np.zeros(cap)
        n = ctypes.c_int()
        self._check(lib().mcubes_trace_get(self._h, _dp(I), _dp(V), cap, ctypes.byref(n)), "mcubes_trace_get")
        k = min(n.value, cap)
        return I[:k], V[:k]

    def grid(self):
        B = np.zeros(self.d * self.nb)
        self._check(lib().mcubes_grid_get(self._h, _dp(B), B.size), "mcubes_grid_get")
        return B.reshape(self.d, self.nb)

    def set_grid(self, B):
        B = _f64(B).reshape(-1)
        self._check(lib().mcubes_grid_set(self._h, _dp(B), B.size), "mcubes_grid_set")

    def set_tables(self, tables):
        """Interpolation tables of TABLE integrands: dicts with ndim (1 or 2),
        values (array of n0 or n0 x n1 knot values), lo and hi (scalars, or
        pairs for 2-D).  Ends the current problem (set up again after it)."""
        arr = (mcubes_table * max(len(tables), 1))()
        keep = []
        for i, tb in enumerate(tables):
            v = _f64(tb["values"])
            keep.append(v)
            lo, hi = np.atleast_1d(tb["lo"]).astype(float), np.atleast_1d(tb["hi"]).astype(float)
            arr[i].ndim = int(tb["ndim"])
            arr[i].n[0] = v.shape[0]
            arr[i].n[1] = v.shape[1] if arr[i].ndim == 2 else 1
            arr[i].lo[0], arr[i].hi[0] = lo[0], hi[0]
            if arr[i].ndim == 2:
                arr[i].lo[1], arr[i].hi[1] = lo[1], hi[1]
            arr[i].values = _dp(np.ascontiguousarray(v).reshape(-1))
        self._check(lib().mcubes_tables_set(self._h, len(tables), arr), "mcubes_tables_set")

    def problem(self):
        v = [ctypes.c_int() for _ in range(5)]
        self._check(lib().mcubes_problem_get(self._h, *[ctypes.byref(x) for x in v]), "mcubes_problem_get")
        return dict(zip(["fid", "d", "nb", "itmax", "enqueued"], [x.value for x in v]))

    def state_export(self):
        """Checkpoint of the current problem (waits for the stream) as bytes."""
        n = ctypes.c_longlong()
        self._check(lib().mcubes_state_size(self._h, ctypes.byref(n)), "mcubes_state_size")
        buf = ctypes.create_string_buffer(n.value)
        self._check(lib().mcubes_state_export(self._h, buf, n.value), "mcubes_state_export")
        return buf.raw

    def state_import(self, blob):
        """Restores a checkpoint made by state_export: options, problem, grid and iteration state."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        self._check(lib().mcubes_state_import(self._h, buf, len(blob)), "mcubes_state_import")
        o = mcubes_opts()
        self._check(lib().mcubes_get_opts(self._h, ctypes.byref(o)), "mcubes_get_opts")
        self.opts = o
        pr = self.problem()
        self.d, self.nb = pr["d"], pr["nb"]

    def hist(self):
        C = np.zeros(self.d * self.nb)
        self._check(lib().mcubes_hist_get(self._h, _dp(C), C.size), "mcubes_hist_get")
        return C.reshape(self.d, self.nb)

    def sample_range(self, it, adjust, cube_begin, cube_end):
        sums = np.zeros(3)
        C = np.zeros(self.d * self.nb) if adjust else None
        self._check(lib().mcubes_sample_range(self._h, it, int(adjust), int(cube_begin), int(cube_end), _dp(sums),
                                              _dp(C)), "mcubes_sample_range")
        return sums, (None if C is None else C.reshape(self.d, self.nb))

    def batch_trace(self, i, d, cap=ITMAX_MAX):
        """Integral i of the last integrate_batch: (I_it, var_it, grid [d][nb], C [d][nb])."""
        I, V = np.zeros(cap), np.zeros(cap)
        n = ctypes.c_int()
        B = np.zeros(d * self.opts_nb())
        C = np.zeros(d * self.opts_nb())
        self._check(lib().mcubes_batch_trace_get(self._h, int(i), _dp(I), _dp(V), cap, ctypes.byref(n), _dp(B),
                                                 _dp(C)), "mcubes_batch_trace_get")
        k = n.value
        return I[:k], V[:k], B.reshape(d, -1), C.reshape(d, -1)

    def opts_nb(self):
        o = mcubes_opts()
        self._check(lib().mcubes_get_opts(self._h, ctypes.byref(o)), "mcubes_get_opts")
        return o.nbins

    def shard_partial_len(self):
        n = ctypes.c_longlong()
        self._check(lib().mcubes_shard_partial_len(self._h, ctypes.byref(n)), "mcubes_shard_partial_len")
        return n.value

    def shard_sample(self, cube_begin, cube_end, d_partial):
        """Samples cubes [cube_begin, cube_end) of the next iteration into the
        device array at address d_partial (shard_partial_len() doubles)."""
        self._check(lib().mcubes_shard_sample(self._h, int(cube_begin), int(cube_end), ctypes.c_void_p(d_partial)),
                    "mcubes_shard_sample")

    def shard_finish(self, d_gathered, nranks):
        """Finishes the iteration from nranks gathered partials (device
        address, [nranks][shard_partial_len()] in rank order)."""
        self._check(lib().mcubes_shard_finish(self._h, ctypes.c_void_p(d_gathered), int(nranks)),
                    "mcubes_shard_finish")

    def geometry(self):
        g, m, p = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        lanes, blocks = ctypes.c_int(), ctypes.c_int()
        self._check(lib().mcubes_geometry_get(self._h, ctypes.byref(g), ctypes.byref(m), ctypes.byref(p),
                                              ctypes.byref(lanes), ctypes.byref(blocks)), "mcubes_geometry_get")
        return dict(g=g.value, m=m.value, p=p.value, lanes=lanes.value, blocks=blocks.value)

    def timing_reset(self, enable=True):
        self._check(lib().mcubes_timing_reset(self._h, int(enable)), "mcubes_timing_reset")

    def timing(self):
        sm, rm = ctypes.c_double(), ctypes.c_double()
        sn, rn = ctypes.c_int(), ctypes.c_int()
        self._check(lib().mcubes_timing_get(self._h, ctypes.byref(sm), ctypes.byref(sn), ctypes.byref(rm),
                                            ctypes.byref(rn)), "mcubes_timing_get")
        return dict(sample_ms=sm.value, sample_launches=sn.value, refine_ms=rm.value, refine_launches=rn.value)


def _requests(requests):
    """ctypes array of mcubes_request from dicts (fid, params, lo, hi, ncall,
    itmax, rel_tol, abs_tol, seed); returns (array, arrays kept alive)."""
    reqs = list(requests)
    keep = []
    arr = (mcubes_request * len(reqs))()
    for i, r in enumerate(reqs):
        p, lo, hi = _f64(r["params"]), _f64(r["lo"]), _f64(r["hi"])
        keep += [p, lo, hi]
        arr[i] = mcubes_request(r["fid"], _dp(p), len(p), len(lo), _dp(lo), _dp(hi), int(r["ncall"]),
                                int(r["itmax"]), float(r.get("rel_tol", 0.0)), float(r.get("abs_tol", 0.0)),
                                int(r.get("seed", 0)))
    return arr, keep


class Server:
    """mcubes_server: continuous batching of integration requests on one context."""

    def __init__(self, ctx: Context, budget_bytes: int = 0, itcap: int = 32):
        self._h = ctypes.c_void_p()
        self.ctx = ctx
        ctx._check(lib().mcubes_server_create(ctypes.byref(self._h), ctx._h, int(budget_bytes), itcap),
                   "mcubes_server_create")

    def close(self):
        if self._h:
            lib().mcubes_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, request, tag):
        arr, keep = _requests([request])
        self.ctx._check(lib().mcubes_server_submit(self._h, arr, int(tag)), "mcubes_server_submit")

    def set_step_iterations(self, iters: int):
        """Iterations each step runs before reading back which requests finished."""
        self.ctx._check(lib().mcubes_server_set_step_iterations(self._h, int(iters)),
                        "mcubes_server_set_step_iterations")

    def set_escalation(self, factor: float, ncall_max: int):
        """Retry a request that ends unconverged with factor x its calls (up to ncall_max)."""
        self.ctx._check(lib().mcubes_server_set_escalation(self._h, float(factor), int(ncall_max)),
                        "mcubes_server_set_escalation")

    def set_retry_sized(self, min_factor: float, max_factor: float, ncall_max: int):
        """Retry an unconverged request with its calls sized from its sigma (see mcubes.h)."""
        self.ctx._check(lib().mcubes_server_set_retry_sized(self._h, float(min_factor), float(max_factor),
                                                            int(ncall_max)), "mcubes_server_set_retry_sized")

    def step(self):
        ran = ctypes.c_int()
        self.ctx._check(lib().mcubes_server_step(self._h, ctypes.byref(ran)), "mcubes_server_step")
        return ran.value

    def poll(self, cap=65536):
        tags = (ctypes.c_longlong * cap)()
        res = (mcubes_result * cap)()
        n = ctypes.c_int()
        self.ctx._check(lib().mcubes_server_poll(self._h, tags, res, cap, ctypes.byref(n)), "mcubes_server_poll")
        return [(tags[i], res[i].as_dict()) for i in range(n.value)]

    def stats(self):
        v = [ctypes.c_longlong() for _ in range(5)]
        self.ctx._check(lib().mcubes_server_stats(self._h, *[ctypes.byref(x) for x in v]), "mcubes_server_stats")
        return dict(zip(["queued", "resident", "completed", "capacity", "slot_bytes"], [x.value for x in v]))

    def run_stream(self, requests, arrival_s):
        arr, keep = _requests(requests)
        n = len(keep) // 3
        arrival = _f64(arrival_s)
        res = (mcubes_result * n)()
        lat = np.zeros(n)
        wall = ctypes.c_double()
        self.ctx._check(lib().mcubes_server_run_stream(self._h, n, arr, _dp(arrival), res, _dp(lat),
                                                        ctypes.byref(wall)), "mcubes_server_run_stream")
        return [r.as_dict() for r in res], lat, wall.value
