// noalloc.cu -- one sampling pass over a cube range that allocates no device
// memory, for callers that cannot call cudaMalloc: hosts whose device memory
// is owned by another allocator (a framework's caching pool, a fixed arena in
// an embedded or real-time service), and processes that must not grow their
// device footprint, or stall on an allocation, once running.  The kernels are
// the ones mcubes_sample_range launches; only the per-block partial sums and
// the histogram accumulator live in a static device array of this file
// instead of a context's buffers.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "mc_internal.h"

namespace mc {
bool integrand_prepare(int id, const double* p, int np, int d, FamParams* out);
bool geometry(int d, long long ncall, long long g_override, int nb, long long* g, long long* m,
              long long* p);
void philox_round_keys(uint64_t seed, uint32_t rk[10][2]);
}  // namespace mc

using namespace mc;

namespace {

// Layout of the static scratch: [block partials: kMaxBlocks x 3 doubles]
// [the pass's histogram accumulator: kMaxBins doubles] [zero low parts of
// the grid edges: kMaxBins doubles].
constexpr int kMaxBlocks = MCUBES_NOALLOC_MAX_BLOCKS;
constexpr int kMaxBins = MCUBES_NOALLOC_MAX_BINS;
constexpr size_t kPartBytes = sizeof(double) * 3 * kMaxBlocks;
constexpr size_t kHistBytes = sizeof(double) * (size_t)kMaxBins;
constexpr size_t kLoBytes = sizeof(double) * kMaxBins;
constexpr size_t kScratchBytes = kPartBytes + kHistBytes + kLoBytes;

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (in host code the symbol is only a host-side stand-in).
cudaError_t scratch_address(int device, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" mcubes_status mcubes_sample_range_noalloc(
    int device, int integrand_id, const double* params, int nparams, int d, const double* lo, const double* hi,
    long long ncall, int nbins, long long g_override, uint64_t seed, int precision, unsigned it, int adjust,
    long long cube_begin, long long cube_end, const double* d_grid, double* d_sums, double* d_hist,
    void* cuda_stream)
{
    if (device < 0 || device >= kMaxDevices || d < 1 || d > MCUBES_DMAX || nbins < 2 || nbins > MCUBES_NBMAX)
        return MCUBES_EINVAL;
    if ((long long)d * nbins > kMaxBins) return MCUBES_EINVAL;  // beyond the static scratch
    if (!lo || !hi || !d_grid || !d_sums || (adjust && !d_hist) || (nparams > 0 && !params)) return MCUBES_EINVAL;
    if (precision != MCUBES_FP64 && precision != MCUBES_MIXED) return MCUBES_EINVAL;
    FamParams fp;
    if (!integrand_prepare(integrand_id, params, nparams, d, &fp)) return MCUBES_EINVAL;
    for (int j = 0; j < d; ++j)
        if (!(lo[j] < hi[j])) return MCUBES_EINVAL;
    long long g, m, p;
    if (!geometry(d, ncall, g_override, nbins, &g, &m, &p)) return MCUBES_EINVAL;
    if (cube_begin < 0 || cube_end < cube_begin || cube_end > m) return MCUBES_EINVAL;

    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return MCUBES_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return MCUBES_EINVAL;
    mcubes_status st = MCUBES_OK;
    do {
        const bool mixed = precision == MCUBES_MIXED;
        const bool adj = adjust != 0;
        cudaStream_t s = (cudaStream_t)cuda_stream;
        unsigned char* scratch = nullptr;
        if (scratch_address(device, &scratch) != cudaSuccess) { st = MCUBES_ECUDA; break; }
        double* part = reinterpret_cast<double*>(scratch);
        double* hist_acc = reinterpret_cast<double*>(scratch + kPartBytes);
        double* grid_lo = reinterpret_cast<double*>(scratch + kPartBytes + kHistBytes);

        const size_t smem = vsample_smem_bytes(mixed, adj, d, nbins, d);
        const size_t smem_other = vsample_smem_bytes(mixed, !adj, d, nbins, d);
        int smem_limit = 0, sms = 0, occ = 0, occ_other = 0;
        if (cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            st = MCUBES_ECUDA;
            break;
        }
        if (smem + 1024 > (size_t)smem_limit) { st = MCUBES_EINVAL; break; }
        if (vsample_occupancy(integrand_id, mixed, adj, d, smem, &occ) != cudaSuccess || occ < 1 ||
            vsample_occupancy(integrand_id, mixed, !adj, d, smem_other, &occ_other) != cudaSuccess) {
            st = MCUBES_ECUDA;
            break;
        }
        int grid = occ * sms;
        if (grid > kMaxBlocks) grid = kMaxBlocks;

        VsArgs a;
        std::memset(&a, 0, sizeof a);
        a.grid = d_grid;
        a.grid_lo = grid_lo;
        a.part = part;
        a.hist_acc = hist_acc;
        a.st = nullptr;
        a.it_fixed = it;
        a.d = (uint32_t)d;
        a.nb = (uint32_t)nbins;
        a.g = (uint32_t)g;
        a.gmagic = (uint32_t)(0xFFFFFFFFu / (uint32_t)g);
        a.p = (uint32_t)p;
        // lanes per cube: a context's default rule, from the residency of both
        // the adjusting and the plain kernel.  The block count differs (at most
        // kMaxBlocks here), so the cubes' sums are grouped into other block
        // partials: results agree with mcubes_sample_range to rounding, not
        // bit for bit.
        int lanes = 1;
        const long long resident = (long long)std::max(occ, occ_other) * sms * vsample_threads(integrand_id, mixed, d);
        while (lanes < 32 && 2 * lanes <= p && (m * lanes < 4 * resident || p / lanes > 64)) lanes *= 2;
        a.lanes = (uint32_t)lanes;
        a.hist_d = (uint32_t)d;
        a.split = 1;
        a.cube_begin = (uint64_t)cube_begin;
        a.cube_end = (uint64_t)cube_end;
        a.perm_k = cube_permutation((uint64_t)(cube_end - cube_begin));
        philox_round_keys(seed, a.rk);
        for (int j = 0; j < d; ++j) {
            a.lo[j] = lo[j];
            a.scale[j] = hi[j] - lo[j];
        }
        a.jac0 = jacobian_scale(g, nbins, d) * family_jac_factor(integrand_id, fp);
        a.phi_scale_f = (float)(1.0 / ((double)g * nbins));
        a.nb_f = (float)nbins;
        set_moment_scales(a, p);
        a.want_abs = 1;  // the pass reports the sum of |cube mean|
        a.fam = fp;

        // the grid's low parts must read as zero and the histogram accumulator
        // start empty; the partials are overwritten
        if (cudaMemsetAsync(grid_lo, 0, sizeof(double) * d * nbins, s) != cudaSuccess ||
            (adj && cudaMemsetAsync(hist_acc, 0, sizeof(double) * d * nbins, s) != cudaSuccess) ||
            launch_vsample(integrand_id, mixed, adj, a, grid, smem, s) != cudaSuccess ||
            launch_reduce_range(part, hist_acc, grid, d, nbins, adj ? 1 : 0, d_sums, d_hist, s) != cudaSuccess) {
            st = MCUBES_ECUDA;
            break;
        }
    } while (0);
    cudaSetDevice(prev);
    return st;
}
