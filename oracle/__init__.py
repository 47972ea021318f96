"""CPU oracle of the m-Cubes VEGAS iteration (arXiv 2202.01753), for tests only.

TEST INFRASTRUCTURE.  The oracle is a plain, slow, double-precision C
implementation of what the method computes (``mcubes_oracle.c``), loaded
here through ctypes.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the library
itself never does, and shares no code with it.

Each wrapper names the paper passage its C function follows (Alg. 1-3,
Sec. 3-5); the readings taken where the paper is silent are stated in the C
source.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcubes_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

OK, EINVAL, ENOMEM, ENONFINITE, ENOCONV = 0, 1, 2, 4, 5
DMAX, NBMAX = 12, 1024

# integrand family ids (same values as the CUDA library's registry)
F_CONST, F_GAUSS, F_CORNER, F_OSC, F_PRODPEAK, F_C0, F_DISCONT, F_COSMO6, F_TABLE = range(9)

_tables_keep = []   # the arrays the C oracle points to

_lock = threading.Lock()
_lib_handle = None


def lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction, no fast-math)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            h = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            h.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            h.oracle_sample_words.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_int, u32p]
            h.oracle_geometry.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                          i64p, i64p, i64p]
            h.oracle_init_grid.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            h.oracle_bin_of.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), dp]
            h.oracle_nparams.argtypes = [ctypes.c_int, ctypes.c_int]
            h.oracle_integrand.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
            h.oracle_integrand.restype = ctypes.c_double
            h.oracle_vsample.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_uint32, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_uint64, dp, dp,
                                         ctypes.POINTER(ctypes.c_uint64)]
            ip = ctypes.POINTER(ctypes.c_int)
            h.oracle_set_tables.argtypes = [ctypes.c_int, ip, ip, ip, dp, dp, dp, dp,
                                            ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
            h.oracle_table_params.argtypes = [dp, ctypes.c_int, ctypes.c_int]
            h.oracle_rebin_axis.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
            h.oracle_weighted.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                          dp, dp, dp, ctypes.POINTER(ctypes.c_int)]
            h.oracle_integrate.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_int64,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                           ctypes.c_double, ctypes.c_uint64, ctypes.c_double,
                                           ctypes.c_double, dp, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), i64p, dp, dp, dp, dp, ctypes.c_int]
            _lib_handle = h
    return _lib_handle


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _Problem(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int), ("params", ctypes.POINTER(ctypes.c_double)),
                ("d", ctypes.c_int), ("nb", ctypes.c_int),
                ("lo", ctypes.POINTER(ctypes.c_double)), ("hi", ctypes.POINTER(ctypes.c_double)),
                ("g", ctypes.c_int64), ("m", ctypes.c_int64), ("p", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("one_dim", ctypes.c_int)]


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter block (Salmon et al., SC'11)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    _lib().oracle_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def sample_words(seed, it, cube, s, d):
    """The d 32-bit words of one sample (counter (s, cube, it, dim block))."""
    out = np.zeros(d, dtype=np.uint32)
    _lib().oracle_sample_words(seed, it, cube, s, d, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def geometry(d, ncall, g_override=0, nb=500):
    """(g, m, p) of Alg. 2, or raises ValueError on invalid arguments."""
    g, m, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = _lib().oracle_geometry(d, ncall, g_override, nb, ctypes.byref(g), ctypes.byref(m), ctypes.byref(p))
    if st:
        raise ValueError(f"invalid geometry d={d} ncall={ncall} g={g_override} nb={nb}")
    return g.value, m.value, p.value


def init_grid(d, nb, with_lo=False):
    """Init-Bins of Alg. 2: [d][nb] right edges of equal bins (and, with
    with_lo, the low parts of their double-double values)."""
    B = np.zeros(d * nb)
    L = np.zeros(d * nb)
    _lib().oracle_init_grid(d, nb, _dp(B), _dp(L))
    return (B.reshape(d, nb), L.reshape(d, nb)) if with_lo else B.reshape(d, nb)


def bin_of(c, w, g, nb):
    """(k, phi) of one coordinate: sub-cube digit c, random word w."""
    k = ctypes.c_int()
    phi = ctypes.c_double()
    _lib().oracle_bin_of(c, w, g, nb, ctypes.byref(k), ctypes.byref(phi))
    return k.value, phi.value


def set_tables(tables):
    """Interpolation tables of the TABLE family (Sec. 6.1's stateful
    integrands): a list of dicts with ndim (1 or 2), values (n0 or n0 x n1
    array, row-major) and the knot ranges lo, hi (scalars, or pairs for 2-D)."""
    global _tables_keep
    n = len(tables)
    nd = (ctypes.c_int * max(n, 1))()
    n0 = (ctypes.c_int * max(n, 1))()
    n1 = (ctypes.c_int * max(n, 1))()
    lo0, hi0, lo1, hi1 = (np.zeros(max(n, 1)) for _ in range(4))
    vals = (ctypes.POINTER(ctypes.c_double) * max(n, 1))()
    keep = []
    for t, tb in enumerate(tables):
        v = _f64(tb["values"])
        keep.append(v)
        nd[t] = int(tb["ndim"])
        lo, hi = np.atleast_1d(tb["lo"]).astype(float), np.atleast_1d(tb["hi"]).astype(float)
        n0[t] = v.shape[0]
        n1[t] = v.shape[1] if nd[t] == 2 else 1
        lo0[t], hi0[t] = lo[0], hi[0]
        lo1[t], hi1[t] = (lo[1], hi[1]) if nd[t] == 2 else (0.0, 1.0)
        vals[t] = _dp(v)
    st = _lib().oracle_set_tables(n, nd, n0, n1, _dp(lo0), _dp(hi0), _dp(lo1), _dp(hi1), vals)
    if st != OK:
        raise ValueError("oracle_set_tables rejected the tables")
    _tables_keep = keep


def table_params_ok(params, d):
    p = _f64(params)
    return bool(_lib().oracle_table_params(_dp(p), len(p), d))


def nparams(fid, d):
    return _lib().oracle_nparams(fid, d)


def integrand(fid, params, x):
    """f(x) of one registered family (Sec. 5 eqs. 1-6, Table 1, Sec. 6.1)."""
    p = _f64(params)
    xx = _f64(x)
    return _lib().oracle_integrand(fid, _dp(p), len(xx), _dp(xx))


class Problem:
    """One integral: family id, parameters, box, calls per iteration."""

    def __init__(self, fid, params, lo, hi, ncall, nb=500, g_override=0, seed=0, one_dim=False):
        self.fid = fid
        self.params = _f64(params)
        self.lo = _f64(lo)
        self.hi = _f64(hi)
        self.d = len(self.lo)
        self.nb = nb
        self.seed = seed
        self.ncall = ncall
        self.g, self.m, self.p = geometry(self.d, ncall, g_override, nb)
        self.one_dim = bool(one_dim)
        self._c = _Problem(fid, _dp(self.params), self.d, nb, _dp(self.lo), _dp(self.hi),
                           self.g, self.m, self.p, seed, int(one_dim))

    @property
    def n_samples(self):
        return self.m * self.p

    def vsample(self, B, it, adjust, cube_begin=0, cube_end=None, hits=False, Blo=None):
        """One V-Sample pass (Alg. 3) over a cube range.

        Returns (sums, C, H): sums = [sum of cube means, sum of cube mean
        variances, sum of |cube means|]; C = [d][nb] per-bin sum of F^2 (adjust
        only); H = [d][nb] per-bin hit counts (adjust and hits only).  With
        one_dim (m-Cubes1D, Sec. 3) only row 0 of C and H is filled.
        """
        cube_end = self.m if cube_end is None else cube_end
        B = _f64(B).reshape(-1)
        L = None if Blo is None else _f64(Blo).reshape(-1)
        sums = np.zeros(3)
        C = np.zeros(self.d * self.nb) if adjust else None
        H = np.zeros(self.d * self.nb, dtype=np.uint64) if (adjust and hits) else None
        st = _lib().oracle_vsample(ctypes.byref(self._c), _dp(B), _dp(L), it, int(adjust), cube_begin, cube_end,
                                   _dp(sums), _dp(C),
                                   H.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if H is not None else None)
        if st not in (OK, ENONFINITE):
            raise RuntimeError(f"oracle_vsample failed: {st}")
        return (sums, None if C is None else C.reshape(self.d, self.nb),
                None if H is None else H.reshape(self.d, self.nb), st)


def rebin_axis(Cj, Bj, alpha=1.5, Blo=None, with_lo=False):
    """Adjust-Bin-Bounds of one axis (Alg. 2; Lepage 1978). Returns (status,
    new edges) or, with with_lo, (status, new edges, their low parts)."""
    C = _f64(Cj).copy()
    B = _f64(Bj).copy()
    L = np.zeros_like(B) if Blo is None else _f64(Blo).copy()
    st = _lib().oracle_rebin_axis(len(B), alpha, _dp(C), _dp(B), _dp(L))
    return (st, B, L) if with_lo else (st, B)


def weighted(I_it, var_it, rel_tol=0.0, abs_tol=0.0):
    """Weighted-Estimates + Check-Convergence (Alg. 2, Sec. 5.1)."""
    I = _f64(I_it)
    V = _f64(var_it)
    est, sig, chi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    conv = ctypes.c_int()
    _lib().oracle_weighted(len(I), _dp(I), _dp(V), rel_tol, abs_tol, ctypes.byref(est),
                           ctypes.byref(sig), ctypes.byref(chi), ctypes.byref(conv))
    return est.value, sig.value, chi.value, bool(conv.value)


def integrate(fid, params, lo, hi, ncall, itmax, ita=None, nb=500, g_override=0, alpha=1.5,
              seed=0, rel_tol=0.0, abs_tol=0.0, one_dim=False):
    """The whole m-Cubes driver (Alg. 2), or with one_dim the m-Cubes1D
    variant (Sec. 3: one grid shared by all axes). Returns a dict."""
    lo = _f64(lo)
    hi = _f64(hi)
    p = _f64(params)
    d = len(lo)
    ita = itmax if ita is None else ita
    res = np.zeros(3)
    iters = ctypes.c_int()
    conv = ctypes.c_int()
    geom = np.zeros(3, dtype=np.int64)
    tI = np.full(itmax, np.nan)
    tV = np.full(itmax, np.nan)
    B = np.zeros(d * nb)
    C = np.zeros(d * nb)
    st = _lib().oracle_integrate(fid, _dp(p), d, _dp(lo), _dp(hi), ncall, itmax, ita, nb, g_override,
                                 alpha, seed, rel_tol, abs_tol, _dp(res), ctypes.byref(iters),
                                 ctypes.byref(conv), geom.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 _dp(tI), _dp(tV), _dp(B), _dp(C), int(one_dim))
    n = iters.value
    return dict(status=st, estimate=res[0], sigma=res[1], chi2_dof=res[2], iterations=n,
                converged=bool(conv.value), g=int(geom[0]), m=int(geom[1]), p=int(geom[2]),
                trace_I=tI[:n], trace_var=tV[:n], grid=B.reshape(d, nb), hist=C.reshape(d, nb))
