// Host build of the kernels' fixed-point log and exp (csrc/fx_math.cuh) with
// plain C++ stand-ins for the device intrinsics they use, so that their
// integer arithmetic can be checked bit for bit on the CPU.  Reads lines of
// one hex double x and prints fx_log(x) and fx_exp(-x), or of a hex double v,
// a decimal 64-bit jm and a decimal je and prints fx_exp_neg_scaled(v, jm, je).
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cstdio>
#define __device__
#define __forceinline__ inline
#define __noinline__
#define __host__
static inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
static inline int64_t __mul64hi(int64_t a, int64_t b) { return (int64_t)(((__int128)a * b) >> 64); }
static inline uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
template <class T> static inline T __ldg(const T* p) { return *p; }
static inline long long __double_as_longlong(double d) { long long x; std::memcpy(&x, &d, 8); return x; }
static inline double __longlong_as_double(long long x) { double d; std::memcpy(&d, &x, 8); return d; }
using std::log; using std::exp; using std::ldexp;
#include "fx_math.cuh"
int main()
{
    char line[256];
    while (std::fgets(line, sizeof line, stdin)) {
        double x;
        unsigned long long jm;
        int je;
        if (std::sscanf(line, "%la %llu %d", &x, &jm, &je) == 3)
            std::printf("%a\n", mc::fx::fx_exp_neg_scaled(x, (uint64_t)jm, je));
        else if (std::sscanf(line, "%la", &x) == 1)
            std::printf("%a %a\n", mc::fx::fx_log(x), mc::fx::fx_exp(-x));
    }
    return 0;
}
