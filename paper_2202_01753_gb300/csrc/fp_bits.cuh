// fp_bits.cuh -- the IEEE-754 double addition of two non-negative numbers
// (round to nearest, ties to even) in 64-bit integer arithmetic.
//
// The sampling kernels add F^2 >= 0 into shared-memory histograms with a
// compare-and-swap loop.  Its first attempt adds on the FP64 pipe with the
// whole warp; a retry (another lane of the warp, or another warp, changed
// the bin in between) runs for a few lanes only, and on GB300, whose SM
// issues one FP64 warp instruction per 16 cycles whatever the number of
// active lanes, a retried FP64 add costs as much pipe time as a full one.
// Retries therefore add with this function on the integer pipes.  Both
// operands and the result are bit patterns of doubles; the result equals
// the hardware's a + b bit for bit (tested against it on the host).
#pragma once

#include <cstdint>

namespace mc {

// a + b for non-negative doubles a, b given by their bits (either may be a
// subnormal or zero; a NaN or infinite operand is not expected: the
// histogram of a non-finite sample is reported as ENONFINITE elsewhere, and
// here it yields +inf).
__host__ __device__ __forceinline__ uint64_t add_nonneg_bits(uint64_t x, uint64_t y)
{
    constexpr uint64_t kFrac = (1ull << 52) - 1ull;
    const uint64_t a = x > y ? x : y;   // non-negative doubles order as integers
    const uint64_t b = x > y ? y : x;
    if (b == 0ull) return a;
    const int ea = (int)(a >> 52), eb = (int)(b >> 52);
    if (ea == 0x7FF) return 0x7FF0000000000000ull;
    // significands with the implicit bit (none for subnormals, whose
    // exponent acts as 1), three guard bits below
    const uint64_t A = ((a & kFrac) | (ea ? (1ull << 52) : 0ull)) << 3;
    const uint64_t B = ((b & kFrac) | (eb ? (1ull << 52) : 0ull)) << 3;
    const int sh = (ea ? ea : 1) - (eb ? eb : 1);
    if (sh > 55) return a;  // b is below a quarter of a's last place: a + b rounds to a
    const uint64_t Bs = sh ? ((B >> sh) | ((B << (64 - sh)) != 0ull ? 1ull : 0ull)) : B;  // sticky bit
    uint64_t S = A + Bs;    // < 2^57
    int E = ea ? ea : 1;
    if (S >> 56) {          // carry into a new leading bit
        S = (S >> 1) | (S & 1ull);
        ++E;
    }
    const uint64_t low = S & 7ull;
    uint64_t m = S >> 3;
    if (low > 4ull || (low == 4ull && (m & 1ull))) ++m;
    if (m >> 53) {          // rounding carried out
        m >>= 1;
        ++E;
    }
    if (E >= 0x7FF) return 0x7FF0000000000000ull;
    return (m >> 52) ? (((uint64_t)E << 52) | (m & kFrac)) : m;  // normal, or subnormal (E == 1, no implicit bit)
}

}  // namespace mc
