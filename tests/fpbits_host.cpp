// Host build of the integer addition of non-negative doubles
// (csrc/fp_bits.cuh).  Reads pairs of hex doubles from stdin and prints the
// bits of add_nonneg_bits and of the hardware sum, for a bit-for-bit
// comparison.
#include <cstdint>
#include <cstdio>
#include <cstring>
#define __device__
#define __host__
#define __forceinline__ inline
#include "fp_bits.cuh"
static uint64_t bits(double d) { uint64_t x; std::memcpy(&x, &d, 8); return x; }
int main()
{
    double a, b;
    while (std::scanf("%la %la", &a, &b) == 2) {
        volatile double s = a + b;  // an SSE2 / AArch64 double add: round to nearest even
        std::printf("%016llx %016llx\n", (unsigned long long)mc::add_nonneg_bits(bits(a), bits(b)),
                    (unsigned long long)bits(s));
    }
    return 0;
}
