"""Measured ALU peaks of the device (FFMA, DFMA, DADD and DMUL throughput), the
denominators of the sampling kernel's roofline.  Built in-tree by
paper_2202_01753_gb300.build alongside libmcubes."""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

from .. import build as _build

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "alu_peaks.cu")


def lib_path() -> str:
    return os.path.join(_build.BUILD, "libmcpeaks.so")


def build() -> str:
    out = lib_path()
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(_build.BUILD, exist_ok=True)
    cmd = [_build.nvcc(), "-shared", "-o", out + ".tmp", SRC] + _build.ARCH + [
        "-O3", "-Xcompiler", "-fPIC", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(out + ".tmp", out)
    return out


def measure(device: int = 0) -> dict:
    """FMA/s in FP32 and FP64 on `device` (one FMA = 2 flops), and FP64 adds/s and multiplies/s."""
    h = ctypes.CDLL(build())
    h.mcpeaks_fma.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    f, d = ctypes.c_double(), ctypes.c_double()
    mf, md = ctypes.c_float(), ctypes.c_float()
    st = h.mcpeaks_fma(device, ctypes.byref(f), ctypes.byref(d), ctypes.byref(mf), ctypes.byref(md))
    if st:
        raise RuntimeError(f"peak measurement failed ({st})")
    h.mcpeaks_fp64_addmul.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    a, m = ctypes.c_double(), ctypes.c_double()
    st = h.mcpeaks_fp64_addmul(device, ctypes.byref(a), ctypes.byref(m))
    if st:
        raise RuntimeError(f"peak measurement failed ({st})")
    return {"ffma_per_s": f.value, "dfma_per_s": d.value, "dadd_per_s": a.value, "dmul_per_s": m.value,
            "ms_f32": mf.value, "ms_f64": md.value, "host": platform.machine()}
