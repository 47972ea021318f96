// vsample.cuh -- the sampling kernel (V-Sample / V-Sample-No-Adjust of
// Alg. 3 in the paper), instantiated once per integrand family by the
// vsample_<family>.cu translation units, and the device pieces it shares with
// the batched kernel (batch.cuh).
//
// Work layout.  A run of `lanes` consecutive threads of a warp owns one
// sub-cube; lane l of the run draws samples l, l + lanes, ... of it.  With
// lanes == 1 (the common case: p is 2 or 3 at 1e8-1e9 calls) a thread owns
// whole cubes and its cube moments need no communication; larger p spreads a
// cube over up to 32 lanes whose moments are merged by XOR shuffles.  Blocks
// walk the cube range with a grid stride.  The bin grid of all axes is staged
// in shared memory once per block as (left edge, nb * width) cells in the
// integration box's coordinates.  In adjusting iterations every sample adds
// F^2 to a per-block shared-memory histogram [d][nb], which the block adds
// to the pass's global histogram once at its end (one global reduction per
// non-empty bin; no per-sample global atomics).  Each block writes three
// double partials (sum of cube means, of their variances, of |means|) which
// the refinement launch reduces in fixed order.
#pragma once

#include <type_traits>

#include "mc_device.cuh"

namespace mc {

// Adds v to the shared-memory histogram word at byte offset `off` of the
// histogram whose shared-window address is `base` (a reduction: no value
// comes back, so nothing waits on it).
__device__ __forceinline__ void hist_add(uint32_t base, uint32_t idx, float v)
{
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(base + 4u * idx), "f"(v));
}
__device__ __forceinline__ void hist_add(uint32_t base, uint32_t idx, double v)
{
    asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(base + 8u * idx), "d"(v));
}

// Adds F2 to the sample's bin on each of the first hist_d axes; idx holds the
// flat bin indices two per word (axis 2k in the low half of idx[k]).  In
// double precision, where a shared-memory add is a compare-and-swap loop that
// repeats while lanes of the warp collide on one bin, odd lanes take the two
// axes of each word in the opposite order: at every step the warp adds to two
// different axes' histograms and half as many lanes compete for the same
// bins.  The single-precision add is a native reduction; there the swap
// measured slower and is not made.
template <int NB4, class HT>
__device__ __forceinline__ void hist_add_sample(uint32_t hist_s, const uint32_t (&idx)[2 * NB4], uint32_t hist_d,
                                                HT F2)
{
    const uint32_t odd = sizeof(HT) == 8 ? (threadIdx.x & 1u) : 0u;
#pragma unroll
    for (int k = 0; k < 2 * NB4; ++k) {
        if (2 * k < (int)hist_d) {
            const uint32_t w = __funnelshift_l(idx[k], idx[k], odd << 4);  // halves swapped on odd lanes
            if (((2u * k) ^ odd) < hist_d) hist_add(hist_s, w & 0xFFFFu, F2);
            if (((2u * k + 1u) ^ odd) < hist_d) hist_add(hist_s, w >> 16, F2);
        }
    }
}

// The same for a sample of DC axes, every one with a histogram (hist_d =
// DC): the lanes start at different index words and take the words in turn
// from there, NW = ceil(DC/2) words in all.  In double precision lane pair t
// (lanes 2t, 2t+1) starts at word (t mod NW), the odd lane of the pair with
// the two halves swapped as above, so each of the NW steps adds to 2 NW
// different axes' histograms, about 32 / (2 NW) lanes each, instead of two
// axes with 16 lanes each; in single precision lane l starts at word
// (l mod NW), no halves swapped (measured faster: corner8 17.57 -> 17.42 ms,
// osc10 21.69 -> 21.00 ms per 1e9-call pass, against 17.65 and 21.33 with
// the swap).  Fewer lanes of a warp collide on one bin, and each collision
// repeats the shared-memory compare-and-swap for the whole warp.  The words
// are picked with selects (static register indices).
template <int NW, int NB4, class HT>
__device__ __forceinline__ void hist_add_sample_rotated(uint32_t hist_s, const uint32_t (&idx)[2 * NB4],
                                                        uint32_t hist_d, HT F2)
{
    static_assert(NW >= 2 && NW <= 2 * NB4, "rotation over the words in use");
    constexpr bool kSwap = sizeof(HT) == 8;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t odd = kSwap ? (lane & 1u) : 0u;
    const uint32_t rot = (kSwap ? (lane >> 1) : lane) % (uint32_t)NW;
#pragma unroll
    for (int t = 0; t < NW; ++t) {
        uint32_t w = idx[t], k = (uint32_t)t;
#pragma unroll
        for (int q = 1; q < NW; ++q) {
            if (rot == (uint32_t)q) {
                w = idx[(t + q) % NW];
                k = (uint32_t)((t + q) % NW);
            }
        }
        w = __funnelshift_l(w, w, odd << 4);  // halves swapped on odd lanes
        if (((2u * k) ^ odd) < hist_d) hist_add(hist_s, w & 0xFFFFu, F2);
        if (((2u * k + 1u) ^ odd) < hist_d) hist_add(hist_s, w >> 16, F2);
    }
}

// The histogram adds of one sample: rotated where the axis count is a
// compile-time DC >= 3 with a histogram on every axis.
template <int DC, int NB4, class HT>
__device__ __forceinline__ void hist_add_one(uint32_t hist_s, const uint32_t (&idx)[2 * NB4], uint32_t hist_d, HT F2)
{
    if constexpr (DC >= 3) {
        if (hist_d == (uint32_t)DC) {
            hist_add_sample_rotated<(DC + 1) / 2, NB4, HT>(hist_s, idx, hist_d, F2);
            return;
        }
    }
    hist_add_sample<NB4>(hist_s, idx, hist_d, F2);
}

template <bool MIXED> struct Prec;
#ifndef MC_MIXED_CUBE_F64
#define MC_MIXED_CUBE_F64 0
#endif
// R: map and integrand; Cell: shared-memory map cell; H: histogram entry;
// S: a cube's shifted sums S1, S2 and its mean and variance.
template <> struct Prec<false> {
    using R = double;
    using Cell = double2;  // (x left edge, x width / g): x = left + (width/g)(g phi), J factor = (g nb)(width/g)
    using H = double;
    using S = double;
};
template <> struct Prec<true> {
    using R = float;
    using Cell = float2;   // (x left edge, nb * x width): x = left + (nb width)(phi/nb), J factor = nb width
    using H = float;
    using S = std::conditional_t<MC_MIXED_CUBE_F64 != 0, double, float>;
};

// Stages the grid of all axes into shared-memory cells and clears the
// histogram ([hist_d][nb]).  grid/grid_lo: [d][nb] double-double right
// edges (unit cube); lo/scale: the box's lower corner and hi - lo; g:
// sub-cubes per axis.
template <bool MIXED, bool ADJ, class Arr>
__device__ __forceinline__ void stage_grid(typename Prec<MIXED>::Cell* cells, typename Prec<MIXED>::H* hist,
                                           const double* grid, const double* grid_lo, const Arr& lo,
                                           const Arr& scale, uint32_t d, uint32_t nb, uint32_t g, uint32_t hist_d)
{
    if constexpr (ADJ)
        for (uint32_t i = threadIdx.x; i < hist_d * nb; i += blockDim.x) hist[i] = typename Prec<MIXED>::H(0);
    const double inv_g = 1.0 / (double)g;  // one division per thread, a multiply per cell
    for (uint32_t i = threadIdx.x; i < d * nb; i += blockDim.x) {
        const uint32_t j = i / nb, k = i - j * nb;
        if constexpr (MIXED) cells[i] = map_cell_f32(grid + j * nb, grid_lo + j * nb, k, lo[j], scale[j], nb);
        else cells[i] = map_cell_f64(grid + j * nb, grid_lo + j * nb, k, lo[j], scale[j], inv_g);
    }
}

// The same staging from cells already built in global memory (by the
// refinement after each rebin, and at set-up): a copy, 16-byte words.
template <bool MIXED, bool ADJ>
__device__ __forceinline__ void stage_cells(typename Prec<MIXED>::Cell* cells, typename Prec<MIXED>::H* hist,
                                            const void* cells_g, uint32_t d, uint32_t nb, uint32_t hist_d)
{
    if constexpr (ADJ)
        for (uint32_t i = threadIdx.x; i < hist_d * nb; i += blockDim.x) hist[i] = typename Prec<MIXED>::H(0);
    const uint32_t bytes = d * nb * (uint32_t)sizeof(typename Prec<MIXED>::Cell);
    const uint4* src = static_cast<const uint4*>(cells_g);
    uint4* dst = reinterpret_cast<uint4*>(cells);
    for (uint32_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0 && (bytes & 15u))  // an odd number of 8-byte cells
        reinterpret_cast<uint2*>(cells)[bytes / 8 - 1] = static_cast<const uint2*>(cells_g)[bytes / 8 - 1];
}

// Whether a family runs its FP64 axes as a loop (Family::kRolled, default no).
template <class F, class = void> struct RolledAxes { static constexpr bool value = false; };
template <class F> struct RolledAxes<F, decltype((void)F::kRolled)> { static constexpr bool value = F::kRolled; };

// Only FP64 families with heavy per-axis work are rolled.  The mixed corner
// and oscillatory kernels, whose per-axis work is a few instructions with
// the axis's constants folded into constant-bank operands when unrolled,
// measured slower rolled (corner8 17.7 -> 21.1-23.1 ms, osc10 21.8 ->
// 26.6-30.2 ms per 1e9-call pass, blocks of 256 to 1024 threads).
template <int FAM, bool MIXED>
constexpr bool rolled_axes()
{
    if constexpr (MIXED) return false;
    else return RolledAxes<Family<FAM, double>>::value;
}

// sample_point for FP64 families with heavy per-axis work (a logarithm per
// axis): the same arithmetic with the axes as a loop that is not unrolled,
// so the per-axis code exists once instead of D times.  Unrolled, a six-axis
// sample is thousands of instructions, more than the SM's instruction
// caches keep close, and warps wait on instruction fetch.  In the loop the
// sub-cube digit of axis j is peeled off the cube index (one high multiply),
// the Philox block of axes 4b..4b+3 is drawn at j = 4b and its words are
// rotated into place, and the flat bin indices are shifted into idx from the
// top, so that after the last axis axis j's index is field j (the layout
// sample_point leaves).  (Unrolled by two or three the loop measured slower:
// 9.55 and 9.69 ms against 8.80 ms per 1e8-call cosmo6 pass.)
template <int FAM, bool MIXED, int NB4, int D, class A>
__device__ __forceinline__ typename Prec<MIXED>::R
sample_point_rolled(const A& a, const typename Prec<MIXED>::Cell* cells, uint32_t c, uint32_t s, uint32_t it,
                    uint32_t (&idx)[2 * NB4])
{
    using R = typename Prec<MIXED>::R;
    using Fam = Family<FAM, R>;
    constexpr int NW = (D + 1) / 2;  // index words in use
    const uint32_t nb = a.nb;
    typename Fam::S fs;
    Fam::begin(fs);
    R jac = R(1);          // mixed: single-precision product of the widths
    IntProd jp{0, 0};      // FP64: the product in integer arithmetic, from jac0
    if constexpr (!MIXED) jp = int_prod_of(a.jac0);
    uint32_t rest = c;
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int k = 0; k < 2 * NB4; ++k) idx[k] = 0u;
#pragma unroll 1
    for (int j = 0; j < D; ++j) {
        if ((j & 3) == 0) r = sample_words(a, make_uint4(s, c, it, (uint32_t)(j >> 2)));
        const uint32_t w = r.x;
        r = make_uint4(r.y, r.z, r.w, r.x);
        uint32_t q = __umulhi(rest, a.gmagic);
        uint32_t dig = rest - q * a.g;
        if (dig >= a.g) { ++q; dig -= a.g; }
        if (dig >= a.g) { ++q; dig -= a.g; }
        rest = q;
        const BinPos bp = bin_pos(w, dig * nb, nb, a.g, a.gmagic);
        const uint32_t flat = (uint32_t)j * nb + bp.k;
        const auto cell = cells[flat];
        R x;
        if constexpr (MIXED) {
            x = fmaf(cell.y, bin_phi_f32(bp, a.phi_scale_f), cell.x);   // (nb width)(phi/nb)
            jac *= cell.y;
        } else {
            x = fma(cell.y, bin_gphi_f64(bp), cell.x);                    // (width/g)(g phi)
            int_prod_mul(jp, cell.y);
        }
        Fam::add(fs, j, x, a.fam);
#pragma unroll
        for (int k = 0; k < NW - 1; ++k) idx[k] = __funnelshift_r(idx[k], idx[k + 1], 16);
        idx[NW - 1] = (idx[NW - 1] >> 16) | (flat << 16);
    }
    if constexpr (D & 1) {  // one field short of the top: move every field down once more
#pragma unroll
        for (int k = 0; k < NW - 1; ++k) idx[k] = __funnelshift_r(idx[k], idx[k + 1], 16);
        idx[NW - 1] >>= 16;
    }
    if constexpr (!MIXED) return Fam::end_scaled(fs, a.fam, jp.m, jp.e);  // f J, rounded once
    else return Fam::end(fs, D, a.fam) * jac;
}

// One sample: random words -> exact bin position -> map -> integrand.
// Returns F = f(x) * J and leaves the flat histogram index of every axis in
// idx (16 bits each, two per word).  A provides d, nb, g, gmagic, jac0 ((g nb)^d), phi_scale_f
// (1/(g nb)), hist_d and fam, and sample_words(a, counter) its Philox block.
template <int FAM, bool MIXED, int NB4, int DC = 0, class A>
__device__ __forceinline__ typename Prec<MIXED>::R
sample_point(const A& a, const typename Prec<MIXED>::Cell* cells, uint32_t c, uint32_t s, uint32_t it,
             const uint32_t (&nbc)[4 * NB4], uint32_t (&idx)[2 * NB4])
{
    using R = typename Prec<MIXED>::R;
    using Fam = Family<FAM, R>;
    if constexpr (DC > 0 && rolled_axes<FAM, MIXED>()) {
        return sample_point_rolled<FAM, MIXED, NB4, DC>(a, cells, c, s, it, idx);
    }
    constexpr int DN = 4 * NB4;  // axes handled by this instantiation (d <= DN)
    const uint32_t d = DC ? (uint32_t)DC : a.d, nb = a.nb;  // DC: the dimension when fixed at compile time
    uint32_t w[DN];
#pragma unroll
    for (int b = 0; b < NB4; ++b) {
        if (4 * b < (int)d) {
            const uint4 r = sample_words(a, make_uint4(s, c, it, (uint32_t)b));
            w[4 * b + 0] = r.x;
            w[4 * b + 1] = r.y;
            w[4 * b + 2] = r.z;
            w[4 * b + 3] = r.w;
        }
    }
    typename Fam::S fs;
    Fam::begin(fs);
    R jac = R(1);                          // mixed: single-precision product of the widths
    IntProd jp{0, 0};                      // FP64: the product in integer arithmetic, from jac0
    if constexpr (!MIXED) jp = int_prod_of(a.jac0);
#pragma unroll
    for (int j = 0; j < DN; ++j) {
        if (j < (int)d) {
            const BinPos bp = bin_pos(w[j], nbc[j], nb, a.g, a.gmagic);
            const uint32_t flat = (uint32_t)j * nb + bp.k;
            const auto cell = cells[flat];
            R x;
            if constexpr (MIXED) {
                const float phin = bin_phi_f32(bp, a.phi_scale_f);   // phi / nb
                x = fmaf(cell.y, phin, cell.x);
            } else {
                x = fma(cell.y, bin_gphi_f64(bp), cell.x);            // (width/g)(g phi)
            }
            if constexpr (MIXED) jac *= cell.y;
            else int_prod_mul(jp, cell.y);
            Fam::add(fs, j, x, a.fam);
            // flat histogram indices (< 2^16) packed two per register
            if (j & 1) idx[j >> 1] |= flat << 16;
            else idx[j >> 1] = flat;
        }
    }
    if constexpr (!MIXED) jac = int_prod_value(jp);
    return Fam::end(fs, d, a.fam) * jac;
}

// Per-thread sums over the cubes a thread finishes: double, or a compensated
// single-precision pair in the mixed path (no FP64 work per cube).
struct CubeSums {
    double I = 0.0, V = 0.0, A = 0.0;
    DFloat fI{0.f, 0.f}, fV{0.f, 0.f}, fA{0.f, 0.f};
    __device__ double vI() const { return I + fI.value(); }
    __device__ double vV() const { return V + fV.value(); }
    __device__ double vA() const { return A + fA.value(); }
};

// Samples cubes [cube_lo, cube_lo + ncubes) of one integral.  The block takes
// groups of (blockDim / lanes) logical cube indices: group0, group0 + gstride,
// ...; logical index i is cube cube_lo + (i * perm_k mod ncubes), a bijection
// of the range (gcd(perm_k, ncubes) = 1) that gives the lanes of a warp
// cubes with unrelated digits on every axis, so that their samples spread
// over all bins instead of crowding the same few (fewer shared-memory atomic
// conflicts and bank conflicts).  Besides what sample_point reads, A provides
// inv_p = 1/p and inv_var_den = 1/(p (p-1)) (inv_p_f, inv_var_den_f in single
// precision) and want_abs (whether the sums of |cube mean| are needed: they
// are reported by the sampling-pass calls, not used by an iteration).
template <int FAM, bool MIXED, bool ADJ, int NB4, int DC = 0, class A>
__device__ __forceinline__ void sample_cubes(const A& a, const typename Prec<MIXED>::Cell* cells,
                                             typename Prec<MIXED>::H* hist, uint64_t cube_lo, uint64_t ncubes,
                                             uint64_t perm_k, uint64_t group0, uint64_t gstride, uint32_t it,
                                             uint32_t lanes, uint32_t p, CubeSums& acc)
{
    using R = typename Prec<MIXED>::R;
    using HT = typename Prec<MIXED>::H;
    constexpr int DN = 4 * NB4;
    const uint32_t d = DC ? (uint32_t)DC : a.d, nb = a.nb;
    const uint32_t hist_d = a.hist_d;  // axes with a histogram: d, or 1 (m-Cubes1D, Sec. 3)
    const uint32_t hist_s = (uint32_t)__cvta_generic_to_shared(hist);
    const uint32_t L = lanes;
    const uint32_t seg_lane = threadIdx.x & (L - 1u);
    const uint32_t cubes_per_group = blockDim.x / L;
    // 1/p and 1/(p (p-1)), rounded once on the host: a division here would be
    // recomputed inside the cube loop when registers run short
    using RS = typename Prec<MIXED>::S;  // per-cube shifted sums and moments
    RS inv_p, inv_var_den;
    if constexpr (sizeof(RS) == 4) {
        inv_p = a.inv_p_f;
        inv_var_den = a.inv_var_den_f;
    } else {
        inv_p = a.inv_p;
        inv_var_den = a.inv_var_den;
    }
    const uint64_t first = group0 * cubes_per_group + threadIdx.x / L;
    uint64_t off = ncubes ? (first % ncubes) * perm_k % ncubes : 0;               // physical offset of `first`
    const uint64_t step = ncubes ? (gstride * cubes_per_group % ncubes) * perm_k % ncubes : 0;
    for (uint64_t base = group0 * cubes_per_group; base < ncubes; base += gstride * cubes_per_group) {
        const uint64_t ci = base + threadIdx.x / L;
        const bool valid = ci < ncubes;
        const uint32_t c = (uint32_t)(cube_lo + (valid ? off : 0));
        off += step;
        if (off >= ncubes) off -= ncubes;
        // sub-cube digits (axis 0 fastest), kept as nb * digit
        uint32_t nbc[DN];
        {
            uint32_t rest = c;
#pragma unroll
            for (int j = 0; j < DN; ++j) {
                if (j < (int)d) {
                    uint32_t q = __umulhi(rest, a.gmagic);
                    uint32_t r = rest - q * a.g;
                    if (r >= a.g) { ++q; r -= a.g; }
                    if (r >= a.g) { ++q; r -= a.g; }
                    nbc[j] = r * nb;
                    rest = q;
                }
            }
        }
        // this lane's samples of the cube, shifted by its first value
        R K = R(0);
        RS S1 = RS(0), S2 = RS(0);
        uint32_t n = 0;
        if (valid) {
            for (uint32_t s = seg_lane; s < p; s += L) {
                uint32_t idx[2 * NB4];
                const R F = sample_point<FAM, MIXED, NB4, DC>(a, cells, c, s, it, nbc, idx);
                if (n == 0) {
                    K = F;  // the shift: its own term is zero
                } else if (n == 1) {
                    S1 = (RS)F - (RS)K;  // S2 = S1^2 is formed when needed
                } else {
                    if (n == 2) S2 = S1 * S1;
                    const RS z = (RS)F - (RS)K;
                    S1 += z;
                    S2 += z * z;
                }
                ++n;
                if constexpr (ADJ) {
                    hist_add_one<DC, NB4>(hist_s, idx, hist_d, (HT)(F * F));
                }
            }
        }
        if (L == 1u) {
            if (valid) {
                // UpdateVariance (Alg. 3): cube mean and the variance of that
                // mean; at p = 2 (every 1e8-call geometry) S1 = z, S2 = z^2 and
                // the variance (z^2 - z^2/2)/2 is exactly z^2/4: the z^2 are
                // summed and the sum scaled once after the loop (exact)
                RS mean, var;
                if (p == 2u) {
                    mean = (RS)K + S1 * RS(0.5);
                    var = S1 * S1;
                } else {
                    mean = (RS)K + S1 * inv_p;
                    var = (S2 - S1 * S1 * inv_p) * inv_var_den;
                }
                if constexpr (sizeof(RS) == 4) {
                    acc.fI.add(mean);
                    acc.fV.add(var);
                    if (a.want_abs) acc.fA.add(fabsf(mean));
                } else {
                    acc.I += mean;
                    if (p == 2u) acc.V = fma(S1, S1, acc.V);  // one FMA for the z^2
                    else acc.V += var;
                    if (a.want_abs) acc.A += fabs(mean);
                }
            }
        } else {
            if (n == 2) S2 = S1 * S1;
            // the cube's lanes re-base their sums on the shift of its first lane
            // (S1 += n dK, S2 += dK (2 S1 + n dK), dK = K_l - K_0; a lane without
            // samples adds nothing) and add them with XOR shuffles: no division
            const double K0 = __shfl_sync(0xffffffffu, (double)K, (int)((threadIdx.x & 31u) & ~(L - 1u)));
            const double dK = (double)K - K0, cnt = (double)n;
            double s1 = (double)S1, s2 = (double)S2;
            s2 = fma(dK, fma(cnt, dK, 2.0 * s1), s2);
            s1 = fma(cnt, dK, s1);
            for (uint32_t off = 1; off < L; off <<= 1) {
                s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            }
            if (valid && seg_lane == 0) {
                const double mean = K0 + s1 * a.inv_p;
                acc.I += mean;
                acc.V += (s2 - s1 * s1 * a.inv_p) * a.inv_var_den;
                if (a.want_abs) acc.A += fabs(mean);
            }
        }
    }
    if (L == 1u && p == 2u) {  // the z^2 / 4 of every cube, scaled once
        acc.V *= 0.25;
        acc.fV.hi *= 0.25f;
        acc.fV.lo *= 0.25f;
    }
}

// Cube-split sampling, for geometries with few cubes and many samples each
// (e.g. 64 cubes of 16384 samples): `split` blocks share one cube, block k
// drawing samples [k q, min(p, (k+1) q)), q = ceil(p / split), spread over
// its threads.  Every thread keeps sums of its samples shifted by its first
// value K_t; they are re-based on thread 0's shift K (S1 += n dK,
// S2 += dK (2 S1 + n dK), dK = K_t - K: no division) and summed in a fixed
// order; the block writes (K, S1, S2) to out[0..2] and the refinement
// combines a cube's blocks the same way.
template <int FAM, bool MIXED, bool ADJ, int NB4, int DC = 0, class A>
__device__ __forceinline__ void sample_cube_slice(const A& a, const typename Prec<MIXED>::Cell* cells,
                                                  typename Prec<MIXED>::H* hist, uint64_t cube, uint32_t k,
                                                  uint32_t split, uint32_t it, uint32_t p,
                                                  double (*red)[kVsThreadsMax / 32], double* out)
{
    using R = typename Prec<MIXED>::R;
    using HT = typename Prec<MIXED>::H;
    constexpr int DN = 4 * NB4;
    const uint32_t d = DC ? (uint32_t)DC : a.d, nb = a.nb;
    const uint32_t hist_d = a.hist_d;
    const uint32_t q = (p + split - 1) / split;
    const uint32_t s_lo = k * q, s_hi = min(p, s_lo + q);
    const uint32_t hist_s = (uint32_t)__cvta_generic_to_shared(hist);
    const uint32_t c = (uint32_t)cube;
    uint32_t nbc[DN];
    {
        uint32_t rest = c;
#pragma unroll
        for (int j = 0; j < DN; ++j) {
            if (j < (int)d) {
                uint32_t qq = __umulhi(rest, a.gmagic);
                uint32_t r = rest - qq * a.g;
                if (r >= a.g) { ++qq; r -= a.g; }
                if (r >= a.g) { ++qq; r -= a.g; }
                nbc[j] = r * nb;
                rest = qq;
            }
        }
    }
    R K = R(0), S1 = R(0), S2 = R(0);
    uint32_t n = 0;
    for (uint32_t s = s_lo + threadIdx.x; s < s_hi; s += blockDim.x) {
        uint32_t idx[2 * NB4];
        const R F = sample_point<FAM, MIXED, NB4, DC>(a, cells, c, s, it, nbc, idx);
        if (n == 0) {
            K = F;  // the shift: its own term is zero
        } else {
            const R z = F - K;
            S1 += z;
            S2 += z * z;
        }
        ++n;
        if constexpr (ADJ) {
            hist_add_one<DC, NB4>(hist_s, idx, hist_d, (HT)(F * F));
        }
    }
    // re-base on thread 0's shift (every thread has a sample: q >= blockDim;
    // a thread without one adds nothing)
    __syncthreads();
    if (threadIdx.x == 0) red[0][0] = (double)K;
    __syncthreads();
    const double K0 = red[0][0];
    __syncthreads();
    const double dK = (double)K - K0, cnt = (double)n;
    double s1 = (double)S1, s2 = (double)S2;
    s2 = fma(dK, fma(cnt, dK, 2.0 * s1), s2);
    s1 = fma(cnt, dK, s1);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, off);
        s2 += __shfl_down_sync(0xffffffffu, s2, off);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[1][warp] = s1;
        red[2][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b1 = 0.0, b2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            b1 += red[1][w];
            b2 += red[2][w];
        }
        out[0] = K0;
        out[1] = b1;
        out[2] = b2;
    }
}

// Fixed-order block sum of the three per-thread sums; thread 0 writes them.
template <int NW>
__device__ __forceinline__ void block_write_sums(const CubeSums& acc, double (*red)[NW], double* out)
{
    double v0 = acc.vI(), v1 = acc.vV(), v2 = acc.vA();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, off);
        v1 += __shfl_down_sync(0xffffffffu, v1, off);
        v2 += __shfl_down_sync(0xffffffffu, v2, off);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][warp] = v0;
        red[1][warp] = v1;
        red[2][warp] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
        }
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
    }
}

// Resident blocks per SM the register allocation is bounded for: three (80
// registers, 24 warps) — measured against two: osc10 mixed +10% despite 132
// bytes of spills, cosmo6 FP64 +4% and gauss3 FP64 +9% with none — except
// for the table integrands in FP64, whose spills and larger table footprint
// in L1/L2 cost a third (two blocks; table6 at three: 16.6 ms per 1e8 calls
// against 10.0 ms).  Four blocks (64 registers) for the mixed kernels up to
// d = 8 measured slower too (corner8: 23.3 ms per 1e9 calls against 21.3);
// for d <= 4 four blocks fit in 64 registers without spills (gauss3 in
// cube-split mode lives on resident warps).
template <int FAM, bool MIXED, int NB4>
constexpr int vsample_min_blocks() { return (FAM == MCUBES_F_TABLE && !MIXED) ? 2 : (NB4 == 1 ? 4 : 3); }

// The same for the single-integral kernel, whose block size can differ
// (vsample_threads): blocks that fill the register file at its size.
template <int FAM, bool MIXED, int D>
constexpr int vsample_kernel_min_blocks()
{
    return vsample_threads(FAM, MIXED, D) == kVsThreads ? vsample_min_blocks<FAM, MIXED, (D + 3) / 4>()
                                                        : 1024 / vsample_threads(FAM, MIXED, D);
}

// One instantiation per dimension D: with the axis count a compile-time
// constant every per-axis loop is unrolled without guards and the families'
// dimension-dependent code (the corner family's power) folds (corner8: 21.4
// -> 17.7 ms per 1e9-call launch against a runtime count).
template <int FAM, bool MIXED, bool ADJ, int D>
__global__ void __launch_bounds__(vsample_threads(FAM, MIXED, D), vsample_kernel_min_blocks<FAM, MIXED, D>())
vsample_kernel(const __grid_constant__ VsArgs a)
{
    constexpr int NB4 = (D + 3) / 4;  // Philox blocks per sample
    if constexpr (FAM == MCUBES_F_COSMO6 && D != 6) {
        return;  // six axes only: never launched
    } else {
    using Cell = typename Prec<MIXED>::Cell;
    using HT = typename Prec<MIXED>::H;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[3][kVsThreadsMax / 32];

    constexpr uint32_t d = D;
    const uint32_t nb = a.nb;
    uint32_t it = a.it_fixed;
    if (a.st != nullptr) {
        const int done = *(volatile const int*)&a.st->done;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.st->active = done ? 0 : 1;
        if (done) return;
        it = *(volatile const uint32_t*)&a.st->it;
    }

    Cell* cells = reinterpret_cast<Cell*>(smem);
    HT* hist = reinterpret_cast<HT*>(smem + cell_bytes(MIXED) * d * nb);
    if (a.cells_g) stage_cells<MIXED, ADJ>(cells, hist, a.cells_g, d, nb, a.hist_d);
    else stage_grid<MIXED, ADJ>(cells, hist, a.grid, a.grid_lo, a.lo, a.scale, d, nb, a.g, a.hist_d);
    __syncthreads();

    if (a.split > 1) {
        sample_cube_slice<FAM, MIXED, ADJ, NB4, D>(a, cells, hist, a.cube_begin + blockIdx.x / a.split,
                                                blockIdx.x % a.split, a.split, it, a.p, red,
                                                a.part + 3 * (size_t)blockIdx.x);
    } else {
        CubeSums acc;
        sample_cubes<FAM, MIXED, ADJ, NB4, D>(a, cells, hist, a.cube_begin, a.cube_end - a.cube_begin, a.perm_k,
                                           blockIdx.x, gridDim.x, it, a.lanes, a.p, acc);
        block_write_sums(acc, red, a.part + 3 * (size_t)blockIdx.x);
    }
    if constexpr (ADJ) {
        __syncthreads();
        // the block's histogram goes into the pass's accumulator once: one
        // global reduction per non-empty bin (no per-sample global atomics)
        for (uint32_t i = threadIdx.x; i < a.hist_d * nb; i += blockDim.x) {
            const double v = (double)hist[i];
            if (v != 0.0) atomicAdd(a.hist_acc + i, v);
        }
    }
    }
}

template <int FAM, bool MIXED, bool ADJ>
inline auto vsample_kernel_d(int d)
{
    using K = void (*)(VsArgs);
    switch (d) {
    case 1: return (K)vsample_kernel<FAM, MIXED, ADJ, 1>;
    case 2: return (K)vsample_kernel<FAM, MIXED, ADJ, 2>;
    case 3: return (K)vsample_kernel<FAM, MIXED, ADJ, 3>;
    case 4: return (K)vsample_kernel<FAM, MIXED, ADJ, 4>;
    case 5: return (K)vsample_kernel<FAM, MIXED, ADJ, 5>;
    case 6: return (K)vsample_kernel<FAM, MIXED, ADJ, 6>;
    case 7: return (K)vsample_kernel<FAM, MIXED, ADJ, 7>;
    case 8: return (K)vsample_kernel<FAM, MIXED, ADJ, 8>;
    case 9: return (K)vsample_kernel<FAM, MIXED, ADJ, 9>;
    case 10: return (K)vsample_kernel<FAM, MIXED, ADJ, 10>;
    case 11: return (K)vsample_kernel<FAM, MIXED, ADJ, 11>;
    default: return (K)vsample_kernel<FAM, MIXED, ADJ, 12>;  // d is checked to be 1..12
    }
}

template <int FAM>
inline auto vsample_kernel_ptr(bool mixed, bool adjust, int d)
{
    if (mixed) return adjust ? vsample_kernel_d<FAM, true, true>(d) : vsample_kernel_d<FAM, true, false>(d);
    return adjust ? vsample_kernel_d<FAM, false, true>(d) : vsample_kernel_d<FAM, false, false>(d);
}

template <int FAM>
cudaError_t launch_vsample_family(bool mixed, bool adjust, const VsArgs& a, int grid, size_t smem,
                                  cudaStream_t s)
{
    auto k = vsample_kernel_ptr<FAM>(mixed, adjust, (int)a.d);
    cudaError_t e = raise_smem_limit((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, vsample_threads(FAM, mixed, (int)a.d), smem, s>>>(a);
    return cudaGetLastError();
}

template <int FAM>
cudaError_t occupancy_family(bool mixed, bool adjust, int d, size_t smem, int* blocks)
{
    auto k = vsample_kernel_ptr<FAM>(mixed, adjust, d);
    cudaError_t e = raise_smem_limit((const void*)k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, vsample_threads(FAM, mixed, d), smem);
}

}  // namespace mc

#define MC_INSTANTIATE_FAMILY(FAM, NAME)                                                          \
    namespace mc {                                                                                \
    cudaError_t launch_vsample_##NAME(bool mixed, bool adjust, const VsArgs& a, int grid,         \
                                      size_t smem, cudaStream_t s)                                \
    {                                                                                             \
        return launch_vsample_family<FAM>(mixed, adjust, a, grid, smem, s);                       \
    }                                                                                             \
    cudaError_t occupancy_##NAME(bool mixed, bool adjust, int d, size_t smem, int* blocks)        \
    {                                                                                             \
        return occupancy_family<FAM>(mixed, adjust, d, smem, blocks);                             \
    }                                                                                             \
    }
