"""Generates csrc/fx_tables.h: the tables of the fixed-point logarithm and
exponential used by the double-precision kernels (csrc/fx_math.cuh).

Table-driven reduction after P. T. P. Tang, "Table-driven implementation of
the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4),
1990, and "Table-driven implementation of the exponential function in IEEE
floating-point arithmetic", ACM TOMS 15(2), 1989:

* log: c_j = 1 + j/256 for j = 0..255 (the left end of each mantissa
  interval, so that the reduced argument is never negative); 1/c_j as an
  unsigned Q63 integer and ln(c_j) as an unsigned Q64 fraction, stored side
  by side (one 16-byte load per lookup); ln 2 as a Q64 integer.  A second
  reduction step (Tang's method applied once more to the reduced argument
  r < 2^-8): d_k = 1 + k/65536 for k = 0..255, 1/d_k as Q63 and ln(d_k) as
  Q64, side by side as well.
* exp: 2^(j/256) for j = 0..255 as unsigned Q62 integers; ln 2 / 256 as a
  128-bit Q115 integer for the fixed-point argument reduction and as a Q62
  integer for the step that makes the reduced argument non-negative; 256/ln 2
  as a Q53 integer for the integer choice of n.  A second step splits the
  reduced argument r < ln2/256 at multiples of 2^-16: exp(k/65536) for
  k = 0..255 as Q62.
* single-precision cosine: pi/2 as the sum of three floats (each the float
  nearest to what remains of pi/2) for a Cody-Waite reduction (Cody and
  Waite, "Software Manual for the Elementary Functions", 1980), and 2/pi.

Values are computed with 60-digit mpmath arithmetic and rounded once.
Run from the repository root: python -m paper_2202_01753_gb300.gen_fx_tables
"""
from __future__ import annotations

import os

import mpmath

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "fx_tables.h")


def _f32(x):
    """x rounded to the nearest single-precision value (returned as a Python float)."""
    import struct
    return struct.unpack("<f", struct.pack("<f", float(mpmath.mpf(x))))[0]


def _dd(x):
    hi = float(x)
    lo = float(x - mpmath.mpf(hi))
    return hi, lo


def tables():
    mpmath.mp.dps = 60
    inv_c, log_q64, exp2 = [], [], []
    for j in range(256):
        c = 1 + mpmath.mpf(j) / 256
        inv_c.append(int(mpmath.nint(2 ** 63 / c)))
        log_q64.append(int(mpmath.nint(2 ** 64 * mpmath.log(c))))
        exp2.append(int(mpmath.nint(2 ** 62 * mpmath.power(2, mpmath.mpf(j) / 256))))
    ln2 = mpmath.log(2)
    return inv_c, log_q64, exp2, ln2


def second_step_tables():
    mpmath.mp.dps = 60
    inv_d, log_d, exp_k = [], [], []
    for k in range(256):
        dk = 1 + mpmath.mpf(k) / 65536
        inv_d.append(int(mpmath.nint(2 ** 63 / dk)))
        log_d.append(int(mpmath.nint(2 ** 64 * mpmath.log(dk))))
        exp_k.append(int(mpmath.nint(2 ** 62 * mpmath.exp(mpmath.mpf(k) / 65536))))
    return inv_d, log_d, exp_k


def _table(lines, comment, name, vals):
    lines += [comment, f"__device__ const uint64_t {name}[256] = {{"]
    for i in range(0, 256, 4):
        lines.append("    " + ", ".join(f"0x{v:016x}ull" for v in vals[i:i + 4]) + ",")
    lines += ["};", ""]


def _pair_table(lines, comment, name, inv, ln):
    lines += [comment, f"__device__ const LogPair {name}[256] = {{"]
    for i in range(0, 256, 2):
        lines.append("    " + " ".join(f"{{0x{a:016x}ull, 0x{b:016x}ull}}," for a, b in zip(inv[i:i + 2], ln[i:i + 2])))
    lines += ["};", ""]


def render():
    inv_c, log_q64, exp2, ln2 = tables()
    mpmath.mp.dps = 60
    ln2_q64 = int(mpmath.nint(ln2 * 2 ** 64))
    c = ln2 / 256
    hp = mpmath.pi / 2
    c_q115 = int(mpmath.nint(c * mpmath.mpf(2) ** 115))
    lines = [
        "// fx_tables.h -- generated by paper_2202_01753_gb300/gen_fx_tables.py (do not edit).",
        "// Tables of the fixed-point logarithm and exponential (fx_math.cuh).",
        "#pragma once",
        "",
        "#include <cstdint>",
        "",
        "namespace mc {",
        "namespace fx {",
        "",
        f"constexpr uint64_t kLn2Q64 = 0x{ln2_q64:016x}ull;  // ln 2 as Q64",
        f"constexpr double k256OverLn2 = {float(256 / ln2)!r};",
        f"constexpr uint64_t k256OverLn2Q53 = 0x{int(mpmath.nint(256 / ln2 * mpmath.mpf(2) ** 53)):016x}ull;  // 256/ln2 as Q53",
        f"constexpr uint64_t kLn2Over256Q115Hi = 0x{c_q115 >> 64:016x}ull;  // ln2/256 = (Hi 2^64 + Lo) 2^-115",
        f"constexpr uint64_t kLn2Over256Q115Lo = 0x{c_q115 & (2 ** 64 - 1):016x}ull;",
        f"constexpr uint64_t kLn2Over256Q62 = 0x{int(mpmath.nint(c * mpmath.mpf(2) ** 62)):016x}ull;  // ln2/256 as Q62",
        f"constexpr float kHalfPiF1 = {_f32(hp)!r}f;  // pi/2 = F1 + F2 + F3 (+ ~1e-23)",
        f"constexpr float kHalfPiF2 = {_f32(hp - _f32(hp))!r}f;",
        f"constexpr float kHalfPiF3 = {_f32(hp - _f32(hp) - _f32(hp - _f32(hp)))!r}f;",
        f"constexpr float kTwoOverPiF = {_f32(2 / mpmath.pi)!r}f;",
        "",
        "// A logarithm table entry: 1/c as Q63 and ln c as Q64, loaded together",
        "struct alignas(16) LogPair {",
        "    uint64_t inv, ln;",
        "};",
        "",
    ]
    _pair_table(lines, "// c_j = 1 + j/256: 1/c_j as Q63 (j = 0: exactly 2^63), ln c_j as Q64 (0 <= ln c_j < ln 2)",
                "kLogC", inv_c, log_q64)
    lines += ["// 2^(j/256) as Q62", "__device__ const uint64_t kExp2[256] = {"]
    for i in range(0, 256, 4):
        lines.append("    " + ", ".join(f"0x{v:016x}ull" for v in exp2[i:i + 4]) + ",")
    lines += ["};", ""]
    inv_d, log_d, exp_k = second_step_tables()
    _pair_table(lines, "// d_k = 1 + k/65536: 1/d_k as Q63 (k = 0: exactly 2^63), ln d_k as Q64", "kLogD", inv_d, log_d)
    _table(lines, "// exp(k/65536) as Q62", "kExpK16", exp_k)
    lines += ["}  // namespace fx", "}  // namespace mc", ""]
    return "\n".join(lines)


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write(render())
    print(OUT)
