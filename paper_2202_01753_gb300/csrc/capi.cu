// capi.cu -- host driver and C ABI (include/mcubes.h) of the single-integral
// path: argument validation, geometry (Alg. 2), device buffers, and the
// enqueueing of the sampling and refinement launches of every iteration.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "ctx_internal.h"

using namespace mc;

namespace mc {
cudaError_t launch_vsample_const(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_gauss(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_corner(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_osc(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_prodpeak(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_c0(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_discont(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_cosmo6(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t launch_vsample_table(bool, bool, const VsArgs&, int, size_t, cudaStream_t);
cudaError_t occupancy_const(bool, bool, int, size_t, int*);
cudaError_t occupancy_gauss(bool, bool, int, size_t, int*);
cudaError_t occupancy_corner(bool, bool, int, size_t, int*);
cudaError_t occupancy_osc(bool, bool, int, size_t, int*);
cudaError_t occupancy_prodpeak(bool, bool, int, size_t, int*);
cudaError_t occupancy_c0(bool, bool, int, size_t, int*);
cudaError_t occupancy_discont(bool, bool, int, size_t, int*);
cudaError_t occupancy_cosmo6(bool, bool, int, size_t, int*);
cudaError_t occupancy_table(bool, bool, int, size_t, int*);

cudaError_t launch_vsample(int family, bool mixed, bool adjust, const VsArgs& a, int grid, size_t smem,
                           cudaStream_t s)
{
    switch (family) {
    case MCUBES_F_CONST: return launch_vsample_const(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_GAUSS: return launch_vsample_gauss(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_CORNER: return launch_vsample_corner(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_OSC: return launch_vsample_osc(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_PRODPEAK: return launch_vsample_prodpeak(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_C0: return launch_vsample_c0(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_DISCONT: return launch_vsample_discont(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_COSMO6: return launch_vsample_cosmo6(mixed, adjust, a, grid, smem, s);
    case MCUBES_F_TABLE: return launch_vsample_table(mixed, adjust, a, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t vsample_occupancy(int family, bool mixed, bool adjust, int d, size_t smem, int* blocks)
{
    switch (family) {
    case MCUBES_F_CONST: return occupancy_const(mixed, adjust, d, smem, blocks);
    case MCUBES_F_GAUSS: return occupancy_gauss(mixed, adjust, d, smem, blocks);
    case MCUBES_F_CORNER: return occupancy_corner(mixed, adjust, d, smem, blocks);
    case MCUBES_F_OSC: return occupancy_osc(mixed, adjust, d, smem, blocks);
    case MCUBES_F_PRODPEAK: return occupancy_prodpeak(mixed, adjust, d, smem, blocks);
    case MCUBES_F_C0: return occupancy_c0(mixed, adjust, d, smem, blocks);
    case MCUBES_F_DISCONT: return occupancy_discont(mixed, adjust, d, smem, blocks);
    case MCUBES_F_COSMO6: return occupancy_cosmo6(mixed, adjust, d, smem, blocks);
    case MCUBES_F_TABLE: return occupancy_table(mixed, adjust, d, smem, blocks);
    default: return cudaErrorInvalidValue;
    }
}

size_t vsample_smem_bytes(bool mixed, bool adjust, int d, int nb, int hist_d)
{
    const size_t cell = mixed ? 8 : 16;  // float2 or double2 cells
    const size_t h = adjust ? (mixed ? 4 : 8) : 0;
    return (size_t)d * nb * cell + (size_t)hist_d * nb * h;
}

// ---------------------------------------------------------------------------
// integrand registry: parameter validation and the device constant layout
// ---------------------------------------------------------------------------
int family_nparams(int id, int d)
{
    switch (id) {
    case MCUBES_F_CONST: return 1;
    case MCUBES_F_GAUSS: return 1 + 2 * d;
    case MCUBES_F_CORNER: return d;
    case MCUBES_F_OSC: return 1 + d;
    case MCUBES_F_PRODPEAK:
    case MCUBES_F_C0:
    case MCUBES_F_DISCONT: return 2 * d;
    case MCUBES_F_COSMO6: return d == 6 ? 10 : -1;
    default: return -1;
    }
}

// TABLE family: [c, nf, (tab, a, b) x nf] against the tables of the context
// (host copies of their descriptors); fills the factor lists.
static bool table_prepare(const double* p, int np, int d, FamParams* out, const TableDesc* host_tabs, int ntabs,
                          const TableDesc* dev_tabs)
{
    if (np < 2 || ntabs < 1 || !host_tabs || !dev_tabs) return false;
    const int nf = (int)p[1];
    if ((double)nf != p[1] || nf < 1 || nf > kTabFactorsMax || np != 2 + 3 * nf) return false;
    for (int q = 0; q < nf; ++q) {
        const double tq = p[2 + 3 * q], aq = p[3 + 3 * q], bq = p[4 + 3 * q];
        const int t = (int)tq, a = (int)aq, b = (int)bq;
        if ((double)t != tq || (double)a != aq || (double)b != bq) return false;
        if (t < 0 || t >= ntabs || a < 0 || a >= d) return false;
        if (host_tabs[t].ndim == 1 && b != -1) return false;
        if (host_tabs[t].ndim == 2 && (b < 0 || b >= d || b == a)) return false;
        out->tid[q] = t;
        out->ta[q] = a;
        out->tb[q] = b;
    }
    out->nf = nf;
    out->tabs = dev_tabs;
    return true;
}

// Fills the kernel-side constants of one integrand (layout documented in
// mc_device.cuh).  Returns false if the parameters are unusable.  TABLE
// integrands need the context's tables (host descriptors and the device
// array); without them they are rejected.
bool integrand_prepare(int id, const double* p, int np, int d, FamParams* out, const TableDesc* host_tabs,
                       int ntabs, const TableDesc* dev_tabs)
{
    for (int i = 0; i < np; ++i)
        if (!std::isfinite(p[i])) return false;
    out->nf = 0;
    out->tabs = nullptr;
    if (id == MCUBES_F_TABLE) {
        if (!table_prepare(p, np, d, out, host_tabs, ntabs, dev_tabs)) return false;
        for (int i = 0; i < kParMax; ++i) {
            out->c[i] = i == 0 ? p[0] : 0.0;
            out->cf[i] = (float)out->c[i];
        }
        return true;
    }
    if (family_nparams(id, d) < 0 || np != family_nparams(id, d)) return false;
    double c[kParMax];
    std::fill(c, c + kParMax, 0.0);
    const double pi = 3.14159265358979323846;
    switch (id) {
    case MCUBES_F_CONST: c[0] = p[0]; break;
    case MCUBES_F_GAUSS:
        c[0] = p[0];
        for (int j = 0; j < d; ++j) {
            if (!(p[1 + d + j] != 0.0)) return false;
            c[1 + j] = p[1 + j];
            c[13 + j] = 1.0 / (2.0 * p[1 + d + j] * p[1 + d + j]);
        }
        break;
    case MCUBES_F_CORNER:
        for (int j = 0; j < d; ++j) c[j] = p[j];
        break;
    case MCUBES_F_OSC:
        c[0] = 2.0 * pi * p[0];
        for (int j = 0; j < d; ++j) c[1 + j] = p[1 + j];
        break;
    case MCUBES_F_PRODPEAK:
        for (int j = 0; j < d; ++j) {
            if (!(p[j] != 0.0)) return false;
            c[j] = 1.0 / (p[j] * p[j]);
            c[12 + j] = p[d + j];
        }
        break;
    case MCUBES_F_C0:
    case MCUBES_F_DISCONT:
        for (int j = 0; j < d; ++j) {
            c[j] = p[j];
            c[12 + j] = p[d + j];
        }
        break;
    case MCUBES_F_COSMO6:
        if (!(p[7] > 0.0) || !(p[9] > 0.0)) return false;
        for (int j = 0; j < 6; ++j) c[j] = p[j];
        c[2] = p[2] + 1.0;  // the lognormals' 1/x_3, 1/x_4 join the a_3, a_4 powers
        c[3] = p[3] + 1.0;
        c[6] = p[6];
        c[7] = 1.0 / (2.0 * p[7] * p[7]);
        c[8] = p[8];
        c[9] = 1.0 / (2.0 * p[9] * p[9]);
        c[10] = 1.0 / (2.0 * pi * p[7] * p[7]);
        if (!std::isnormal(c[10])) return false;  // the FP64 kernels fold it into the Jacobian's constant
        // the FP64 kernels' expanded lognormal terms: h (L - mu)^2 = h L^2 - 2 h mu L + h mu^2
        c[11] = c[2] - 2.0 * c[7] * c[6];
        c[12] = c[3] - 2.0 * c[7] * c[6];
        c[13] = 2.0 * c[7] * c[6] * c[6];
        break;
    default: return false;
    }
    for (int i = 0; i < kParMax; ++i) {
        out->c[i] = c[i];
        out->cf[i] = (float)c[i];
    }
    return true;
}

bool integrand_prepare(int id, const double* p, int np, int d, FamParams* out)
{
    return integrand_prepare(id, p, np, d, out, nullptr, 0, nullptr);
}

// Geometry of Alg. 2: g = largest integer with g^d <= ncall/2 (>= 1), capped
// so that m = g^d fits a 32-bit counter and nb*g <= 2^31; p = max(ncall/m, 2).
static bool ipow_le(long long g, int d, unsigned long long limit, unsigned long long* out)
{
    unsigned long long v = 1;
    for (int i = 0; i < d; ++i) {
        if (v > limit / (unsigned long long)g) return false;
        v *= (unsigned long long)g;
    }
    *out = v;
    return true;
}

bool geometry(int d, long long ncall, long long g_override, int nb, long long* g, long long* m,
              long long* p)
{
    const unsigned long long mlim = 0xFFFFFFFFull;
    const long long glim = (1ll << 31) / nb;
    unsigned long long mm = 0;
    long long gg;
    if (g_override > 0) {
        gg = g_override;
        if (gg > glim || !ipow_le(gg, d, mlim, &mm)) return false;
    } else {
        const unsigned long long cap = std::min<unsigned long long>((unsigned long long)ncall / 2, mlim);
        long long lo = 1, hi = glim;
        while (lo < hi) {
            const long long mid = lo + (hi - lo + 1) / 2;
            unsigned long long t;
            if (ipow_le(mid, d, cap, &t)) lo = mid; else hi = mid - 1;
        }
        gg = lo;
        ipow_le(gg, d, mlim, &mm);
    }
    long long pp = ncall / (long long)mm;
    if (pp < 2) pp = 2;
    if (pp > 0xFFFFFFFFll) return false;
    *g = gg;
    *m = (long long)mm;
    *p = pp;
    return true;
}

cudaError_t ctx_refresh_cells(mcubes_ctx* c)
{
    const double* g = (const double*)c->grid.ptr;
    return launch_cells(g, g + (size_t)c->d * c->nb, c->cellbox, c->d, c->nb, c->cells.ptr, c->stream);
}

cudaError_t raise_smem_limit(const void* kernel, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> set;  // (kernel, device) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[{kernel, dev}];
    if (smem <= cur && cur > 0) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(smem, cur));
    if (e == cudaSuccess) cur = std::max(smem, cur);
    return e;
}

// Multiplier of the cube order of a range of n cubes (see sample_cubes):
// the integer nearest n times the golden-ratio fraction that is coprime to n.
uint64_t cube_permutation(uint64_t n)
{
    if (n <= 2) return 1;
    uint64_t k = (uint64_t)std::llround(0.6180339887498949 * (double)n);
    if (k < 1) k = 1;
    while (std::gcd(k, n) != 1) k = (k + 1 < n) ? k + 1 : 1;
    return k;
}

// Constant factor of the FP64 kernels' Jacobian: their cells hold the bin
// width over g, and each axis contributes nb * width to J.
// Constant factor an FP64 family returns outside its kernel arithmetic: the
// kernels take it as part of the Jacobian's constant (COSMO6: its
// normalisation c10); 1 for the others.
double family_jac_factor(int id, const FamParams& fp) { return id == MCUBES_F_COSMO6 ? fp.c[10] : 1.0; }

double jacobian_scale(long long g, long long nb, int d)
{
    double j = 1.0;
    for (int i = 0; i < d; ++i) j *= (double)g * (double)nb;
    return j;
}

// 1/p and 1/(p (p-1)) of the cube moments (p >= 2), in both precisions,
// each a correctly rounded IEEE division.
MomentScales moment_scales(long long p)
{
    MomentScales m;
    m.inv_p = 1.0 / (double)p;
    m.inv_var_den = m.inv_p / (double)(p - 1);
    m.inv_p_f = 1.0f / (float)p;
    m.inv_var_den_f = m.inv_p_f / (float)(p - 1);
    return m;
}

void philox_round_keys(uint64_t seed, uint32_t rk[10][2])
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[r][0] = k0;
        rk[r][1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

}  // namespace mc

static mcubes_status cuda_fail(mcubes_ctx* c, cudaError_t e)
{
    if (c) std::snprintf(c->cuda_err, sizeof c->cuda_err, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return MCUBES_ENOMEM;
    return MCUBES_ECUDA;
}

#define MC_CHECK(ctx, expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return cuda_fail((ctx), _e);   \
    } while (0)

static bool opts_valid(const mcubes_opts* o)
{
    if (o->nbins < 2 || o->nbins > MCUBES_NBMAX) return false;
    if (!(o->alpha >= 0.0) || !std::isfinite(o->alpha)) return false;
    if (o->precision != MCUBES_FP64 && o->precision != MCUBES_MIXED) return false;
    if (o->lanes_per_cube < 0 || o->lanes_per_cube > 32 || (o->lanes_per_cube & (o->lanes_per_cube - 1)))
        return false;
    if (o->blocks_per_sm < 0 || o->blocks_per_sm > 32) return false;
    if (o->g_override < 0) return false;
    if (o->one_dim != 0 && o->one_dim != 1) return false;
    return true;
}

static EventPair take_events(mcubes_ctx* c)
{
    if (!c->pool.empty()) {
        EventPair e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    EventPair e;
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
    return e;
}

static void recycle_events(mcubes_ctx* c)
{
    for (auto& e : c->ev_sample) c->pool.push_back(e);
    for (auto& e : c->ev_refine) c->pool.push_back(e);
    c->ev_sample.clear();
    c->ev_refine.clear();
}

extern "C" {

void mcubes_default_opts(mcubes_opts* o)
{
    if (!o) return;
    o->nbins = 500;
    o->ita = -1;
    o->g_override = 0;
    o->alpha = 1.5;
    o->seed = 0;
    o->precision = MCUBES_FP64;
    o->lanes_per_cube = 0;
    o->blocks_per_sm = 0;
    o->one_dim = 0;
}

const char* mcubes_strerror(mcubes_status s)
{
    switch (s) {
    case MCUBES_OK: return "ok";
    case MCUBES_EINVAL: return "invalid argument";
    case MCUBES_ENOMEM: return "out of memory";
    case MCUBES_ECUDA: return "CUDA error";
    case MCUBES_ENONFINITE: return "integrand produced a non-finite value";
    case MCUBES_ENOCONV: return "not converged within itmax";
    case MCUBES_ETIMEOUT: return "device wait timed out";
    case MCUBES_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

const char* mcubes_last_cuda_error(mcubes_ctx* c) { return c ? c->cuda_err : ""; }

static mcubes_status create_impl(mcubes_ctx** out, int device, const mcubes_opts* opts, bool given,
                                 void* stream)
{
    if (!out) return MCUBES_EINVAL;
    *out = nullptr;
    mcubes_opts o;
    mcubes_default_opts(&o);
    if (opts) o = *opts;
    if (!opts_valid(&o)) return MCUBES_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MCUBES_EINVAL;
    mcubes_ctx* c = new (std::nothrow) mcubes_ctx();
    if (!c) return MCUBES_ENOMEM;
    c->device = device;
    c->opts = o;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (given) {
            c->stream = (cudaStream_t)stream;  // may be the legacy default stream (NULL)
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e == cudaSuccess) e = c->state.reserve(sizeof(DevState));
    if (e == cudaSuccess) e = c->range_out.reserve(sizeof(double) * (3 + (size_t)MCUBES_DMAX * MCUBES_NBMAX));
    if (e != cudaSuccess) {
        mcubes_status st = cuda_fail(nullptr, e);
        mcubes_destroy(c);
        return st;
    }
    *out = c;
    return MCUBES_OK;
}

mcubes_status mcubes_create(mcubes_ctx** out, int device, const mcubes_opts* opts)
{
    return create_impl(out, device, opts, false, nullptr);
}

mcubes_status mcubes_create_on_stream(mcubes_ctx** out, int device, const mcubes_opts* opts, void* stream)
{
    return create_impl(out, device, opts, true, stream);
}

mcubes_status mcubes_set_opts(mcubes_ctx* c, const mcubes_opts* o)
{
    if (!c || !o || !opts_valid(o)) return MCUBES_EINVAL;
    c->opts = *o;
    c->ready = false;
    delete c->engine;  // the batched path's buffers depend on the options
    c->engine = nullptr;
    return MCUBES_OK;
}

mcubes_status mcubes_get_opts(mcubes_ctx* c, mcubes_opts* out)
{
    if (!c || !out) return MCUBES_EINVAL;
    *out = c->opts;
    return MCUBES_OK;
}

mcubes_status mcubes_destroy(mcubes_ctx* c)
{
    if (!c) return MCUBES_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->grid.release();
    c->hist.release();
    c->part.release();
    c->hist_acc.release();
    c->cells.release();
    c->state.release();
    c->range_out.release();
    delete c->engine;
    c->engine = nullptr;
    recycle_events(c);
    for (auto& e : c->pool) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return MCUBES_OK;
}

// Chooses how many threads share a cube: enough cube-lanes to cover the
// resident threads several times, and a bounded number of samples per lane.
static int choose_lanes(long long m, long long p, long long resident)
{
    int L = 1;
    while (L < 32 && 2 * L <= p && (m * L < 4 * resident || p / L > 64)) L *= 2;
    return L;
}

mcubes_status mcubes_setup(mcubes_ctx* c, int id, const double* params, int nparams, int d,
                           const double* lo, const double* hi, long long ncall, int itmax,
                           double rel_tol, double abs_tol)
{
    if (!c) return MCUBES_EINVAL;
    c->ready = false;
    if (d < 1 || d > MCUBES_DMAX || ncall < 2 || itmax < 1 || itmax > MCUBES_ITMAX_MAX) return MCUBES_EINVAL;
    if (!lo || !hi || (nparams > 0 && !params)) return MCUBES_EINVAL;
    if (!(rel_tol >= 0.0) || !(abs_tol >= 0.0)) return MCUBES_EINVAL;
    FamParams fp;
    if (!integrand_prepare(id, params, nparams, d, &fp, c->tabs_host.data(), (int)c->tabs_host.size(),
                           (const TableDesc*)c->tab_desc.ptr))
        return MCUBES_EINVAL;
    for (int j = 0; j < d; ++j)
        if (!std::isfinite(lo[j]) || !std::isfinite(hi[j]) || !(lo[j] < hi[j])) return MCUBES_EINVAL;
    const int nb = c->opts.nbins;
    long long g, m, p;
    if (!geometry(d, ncall, c->opts.g_override, nb, &g, &m, &p)) return MCUBES_EINVAL;

    MC_CHECK(c, cudaSetDevice(c->device));
    c->fid = id;
    c->d = d;
    c->nb = nb;
    c->ncall = ncall;
    c->itmax = itmax;
    c->ita = c->opts.ita < 0 ? itmax : std::min(c->opts.ita, itmax);
    c->g = g;
    c->m = m;
    c->p = p;
    c->mixed = c->opts.precision == MCUBES_MIXED;
    c->hist_d = c->opts.one_dim ? 1 : d;
    if (c->opts.one_dim)  // m-Cubes1D: one set of boundaries serves every axis, so the box must be a cube
        for (int j = 1; j < d; ++j)
            if (lo[j] != lo[0] || hi[j] != hi[0]) return MCUBES_EINVAL;

    // launch shapes
    c->smem_adj = vsample_smem_bytes(c->mixed, true, d, nb, c->hist_d);
    c->smem_noadj = vsample_smem_bytes(c->mixed, false, d, nb, c->hist_d);
    int smem_limit = 0;
    MC_CHECK(c, cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (c->smem_adj + 1024 > (size_t)smem_limit) return MCUBES_EINVAL;  // grid + histogram must fit on chip
    int occ_adj = 0, occ_noadj = 0;
    MC_CHECK(c, vsample_occupancy(id, c->mixed, true, d, c->smem_adj, &occ_adj));
    MC_CHECK(c, vsample_occupancy(id, c->mixed, false, d, c->smem_noadj, &occ_noadj));
    if (occ_adj < 1 || occ_noadj < 1) return MCUBES_EINVAL;
    if (c->opts.blocks_per_sm > 0) {
        occ_adj = std::min(occ_adj, c->opts.blocks_per_sm);
        occ_noadj = std::min(occ_noadj, c->opts.blocks_per_sm);
    }
    c->grid_adj = occ_adj * c->num_sms;
    c->grid_noadj = occ_noadj * c->num_sms;
    c->grid_res_adj = c->grid_adj;
    c->grid_res_noadj = c->grid_noadj;
    const int threads = vsample_threads(id, c->mixed, d);
    const long long resident = (long long)std::max(occ_adj, occ_noadj) * c->num_sms * threads;
    c->lanes = c->opts.lanes_per_cube > 0 ? c->opts.lanes_per_cube : choose_lanes(m, p, resident);
    // Cube-split mode: when the cubes cannot keep a quarter of the resident
    // threads busy (few cubes with many samples each), several blocks share
    // one cube, so that about two waves of blocks sample every iteration.
    c->split = 1;
    if (c->opts.lanes_per_cube == 0 && m * c->lanes * 4 < resident && p >= 2 * threads) {
        const long long want = (2LL * std::max(c->grid_adj, c->grid_noadj) + m - 1) / m;
        c->split = (int)std::max(1LL, std::min(want, p / threads));
        if (c->split > 1) c->grid_adj = c->grid_noadj = (int)(m * c->split);
    }
    const int grid_max = std::max(c->grid_adj, c->grid_noadj);

    // device buffers
    MC_CHECK(c, c->grid.reserve(2 * sizeof(double) * d * nb));  // high parts, then low parts
    MC_CHECK(c, c->hist.reserve(sizeof(double) * d * nb));
    MC_CHECK(c, c->part.reserve(sizeof(double) * 3 * grid_max));
    MC_CHECK(c, c->hist_acc.reserve(sizeof(double) * (size_t)c->hist_d * nb));
    MC_CHECK(c, c->cells.reserve((c->mixed ? sizeof(float2) : sizeof(double2)) * (size_t)d * nb));

    // kernel arguments
    VsArgs& a = c->vs;
    std::memset(&a, 0, sizeof a);
    a.grid = (const double*)c->grid.ptr;
    a.grid_lo = (const double*)c->grid.ptr + (size_t)d * nb;
    a.part = (double*)c->part.ptr;
    a.hist_acc = (double*)c->hist_acc.ptr;
    a.cells_g = c->cells.ptr;
    a.st = (DevState*)c->state.ptr;
    a.d = (uint32_t)d;
    a.nb = (uint32_t)nb;
    a.g = (uint32_t)g;
    a.gmagic = (uint32_t)(0xFFFFFFFFu / (uint32_t)g);
    a.p = (uint32_t)p;
    a.lanes = (uint32_t)c->lanes;
    a.hist_d = (uint32_t)c->hist_d;
    a.split = (uint32_t)c->split;
    a.cube_begin = 0;
    a.cube_end = (uint64_t)m;
    a.perm_k = cube_permutation((uint64_t)m);
    philox_round_keys(c->opts.seed, a.rk);
    for (int j = 0; j < d; ++j) {
        a.lo[j] = lo[j];
        a.scale[j] = hi[j] - lo[j];
    }
    a.jac0 = jacobian_scale(g, nb, d) * family_jac_factor(c->fid, fp);
    a.phi_scale_f = (float)(1.0 / ((double)g * nb));
    a.nb_f = (float)nb;
    set_moment_scales(a, p);
    a.want_abs = 0;  // an iteration uses the sums of the cube means and variances only
    a.fam = fp;

    RefineArgs& r = c->rf;
    std::memset(&r, 0, sizeof r);
    r.grid = (double*)c->grid.ptr;
    r.grid_lo = (double*)c->grid.ptr + (size_t)d * nb;
    r.hist = (double*)c->hist.ptr;
    r.part = (const double*)c->part.ptr;
    r.hist_acc = (double*)c->hist_acc.ptr;
    r.cells_g = c->cells.ptr;
    r.g = (uint32_t)g;
    r.mixed = c->mixed ? 1 : 0;
    std::memset(&c->cellbox, 0, sizeof c->cellbox);
    for (int j = 0; j < d; ++j) {
        r.lo[j] = c->cellbox.lo[j] = lo[j];
        r.scale[j] = c->cellbox.scale[j] = hi[j] - lo[j];
    }
    c->cellbox.g = (uint32_t)g;
    c->cellbox.mixed = c->mixed ? 1 : 0;
    r.st = (DevState*)c->state.ptr;
    r.d = d;
    r.nb = nb;
    r.hist_d = c->hist_d;
    r.split = c->split;
    r.p = (double)p;
    r.alpha = c->opts.alpha;
    r.m = (double)m;

    // initial state: uniform grid, empty history
    DevState hst;
    std::memset(&hst, 0, offsetof(DevState, hist_I));
    hst.rel_tol = rel_tol;
    hst.abs_tol = abs_tol;
    MC_CHECK(c, cudaMemcpyAsync(c->state.ptr, &hst, offsetof(DevState, hist_I), cudaMemcpyHostToDevice, c->stream));
    MC_CHECK(c, launch_init_grid((double*)c->grid.ptr, (double*)c->grid.ptr + (size_t)d * nb, d, nb, c->stream));
    MC_CHECK(c, ctx_refresh_cells(c));
    MC_CHECK(c, cudaMemsetAsync(c->hist.ptr, 0, sizeof(double) * d * nb, c->stream));
    MC_CHECK(c, cudaMemsetAsync(c->hist_acc.ptr, 0, sizeof(double) * c->hist_d * nb, c->stream));
    MC_CHECK(c, cudaStreamSynchronize(c->stream));  // hst lives on this stack frame
    c->prob_params.assign(params, params + std::max(nparams, 0));
    c->prob_lo.assign(lo, lo + d);
    c->prob_hi.assign(hi, hi + d);
    c->rel_tol = rel_tol;
    c->abs_tol = abs_tol;
    c->it_enqueued = 0;
    c->shard_open = false;
    c->ready = true;
    return MCUBES_OK;
}

mcubes_status mcubes_iterate(mcubes_ctx* c, int n_iter)
{
    if (!c) return MCUBES_EINVAL;
    if (!c->ready || n_iter < 0 || c->it_enqueued + n_iter > c->itmax || c->shard_open) return MCUBES_ESTATE;
    MC_CHECK(c, cudaSetDevice(c->device));
    for (int i = 0; i < n_iter; ++i) {
        const bool adjust = c->it_enqueued < c->ita;
        const int grid = adjust ? c->grid_adj : c->grid_noadj;
        const size_t smem = adjust ? c->smem_adj : c->smem_noadj;
        EventPair ev;
        if (c->timing) {
            ev = take_events(c);
            MC_CHECK(c, cudaEventRecord(ev.a, c->stream));
        }
        MC_CHECK(c, launch_vsample(c->fid, c->mixed, adjust, c->vs, grid, smem, c->stream));
        if (c->timing) {
            MC_CHECK(c, cudaEventRecord(ev.b, c->stream));
            c->ev_sample.push_back(ev);
        }
        c->rf.nblocks = grid;
        c->rf.adjust = adjust ? 1 : 0;
        EventPair ev2;
        if (c->timing) {
            ev2 = take_events(c);
            MC_CHECK(c, cudaEventRecord(ev2.a, c->stream));
        }
        MC_CHECK(c, launch_refine(c->rf, c->stream));
        if (c->timing) {
            MC_CHECK(c, cudaEventRecord(ev2.b, c->stream));
            c->ev_refine.push_back(ev2);
        }
        ++c->it_enqueued;
    }
    return MCUBES_OK;
}

mcubes_status mcubes_result_get(mcubes_ctx* c, mcubes_result* out)
{
    if (!c || !out) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    MC_CHECK(c, cudaSetDevice(c->device));
    DevState h;
    MC_CHECK(c, cudaMemcpyAsync(&h, c->state.ptr, offsetof(DevState, hist_I), cudaMemcpyDeviceToHost, c->stream));
    MC_CHECK(c, cudaStreamSynchronize(c->stream));
    out->estimate = h.estimate;
    out->sigma = h.sigma;
    out->chi2_dof = h.chi2_dof;
    out->iterations = h.n;
    out->converged = h.converged;
    out->samples_per_iter = c->m * c->p;
    out->g = c->g;
    out->m = c->m;
    out->p = c->p;
    mcubes_status st = h.error ? (mcubes_status)h.error : (h.converged ? MCUBES_OK : MCUBES_ENOCONV);
    out->status = st;
    return st;
}

mcubes_status mcubes_integrate(mcubes_ctx* c, int id, const double* params, int nparams, int d,
                               const double* lo, const double* hi, long long ncall, int itmax,
                               double rel_tol, double abs_tol, mcubes_result* out)
{
    if (!c || !out) return MCUBES_EINVAL;
    mcubes_status st = mcubes_setup(c, id, params, nparams, d, lo, hi, ncall, itmax, rel_tol, abs_tol);
    if (st != MCUBES_OK) return st;
    st = mcubes_iterate(c, itmax);
    if (st != MCUBES_OK) return st;
    return mcubes_result_get(c, out);
}

mcubes_status mcubes_trace_get(mcubes_ctx* c, double* I_it, double* var_it, int cap, int* n)
{
    if (!c || cap < 0) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    MC_CHECK(c, cudaSetDevice(c->device));
    int hn = 0;
    MC_CHECK(c, cudaMemcpyAsync(&hn, (char*)c->state.ptr + offsetof(DevState, n), sizeof(int),
                                cudaMemcpyDeviceToHost, c->stream));
    MC_CHECK(c, cudaStreamSynchronize(c->stream));
    const int k = std::min(hn, cap);
    if (k > 0 && I_it)
        MC_CHECK(c, cudaMemcpy(I_it, (char*)c->state.ptr + offsetof(DevState, hist_I), sizeof(double) * k,
                               cudaMemcpyDeviceToHost));
    if (k > 0 && var_it)
        MC_CHECK(c, cudaMemcpy(var_it, (char*)c->state.ptr + offsetof(DevState, hist_V), sizeof(double) * k,
                               cudaMemcpyDeviceToHost));
    if (n) *n = hn;
    return MCUBES_OK;
}

static mcubes_status copy_dd(mcubes_ctx* c, double* dst, const DevBuf& src, long long count)
{
    if (!c || !dst) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    if (count != (long long)c->d * c->nb) return MCUBES_EINVAL;
    MC_CHECK(c, cudaSetDevice(c->device));
    MC_CHECK(c, cudaMemcpyAsync(dst, src.ptr, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
    MC_CHECK(c, cudaStreamSynchronize(c->stream));
    return MCUBES_OK;
}

mcubes_status mcubes_grid_get(mcubes_ctx* c, double* B, long long count) { return copy_dd(c, B, c->grid, count); }

mcubes_status mcubes_hist_get(mcubes_ctx* c, double* C, long long count) { return copy_dd(c, C, c->hist, count); }

mcubes_status mcubes_grid_set(mcubes_ctx* c, const double* B, long long count)
{
    if (!c || !B) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    if (count != (long long)c->d * c->nb) return MCUBES_EINVAL;
    for (int j = 0; j < c->d; ++j) {
        double prev = 0.0;
        for (int k = 0; k < c->nb; ++k) {
            const double v = B[(size_t)j * c->nb + k];
            if (!(v > prev) || !(v <= 1.0)) return MCUBES_EINVAL;
            prev = v;
        }
        if (prev != 1.0) return MCUBES_EINVAL;
        if (c->hist_d == 1 && j > 0 && std::memcmp(B + (size_t)j * c->nb, B, sizeof(double) * c->nb) != 0)
            return MCUBES_EINVAL;  // m-Cubes1D: every axis has the same boundaries
    }
    MC_CHECK(c, cudaSetDevice(c->device));
    MC_CHECK(c, cudaMemcpyAsync(c->grid.ptr, B, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
    MC_CHECK(c, cudaMemsetAsync((double*)c->grid.ptr + count, 0, sizeof(double) * count, c->stream));
    MC_CHECK(c, ctx_refresh_cells(c));
    MC_CHECK(c, cudaStreamSynchronize(c->stream));
    return MCUBES_OK;
}

mcubes_status mcubes_sample_range(mcubes_ctx* c, unsigned it, int adjust, long long cube_begin,
                                  long long cube_end, double* sums, double* C)
{
    if (!c || !sums) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    if (cube_begin < 0 || cube_end < cube_begin || cube_end > c->m) return MCUBES_EINVAL;
    MC_CHECK(c, cudaSetDevice(c->device));
    VsArgs a = c->vs;
    a.st = nullptr;
    a.it_fixed = it;
    a.split = 1;  // the range pass always uses the cube-stride layout (its partials are sums)
    a.want_abs = 1;  // the pass reports the sum of |cube mean|
    a.cube_begin = (uint64_t)cube_begin;
    a.cube_end = (uint64_t)cube_end;
    a.perm_k = cube_permutation((uint64_t)(cube_end - cube_begin));
    const bool adj = adjust != 0;
    const int grid = adj ? c->grid_adj : c->grid_noadj;
    const size_t smem = adj ? c->smem_adj : c->smem_noadj;
    MC_CHECK(c, launch_vsample(c->fid, c->mixed, adj, a, grid, smem, c->stream));
    double* out = (double*)c->range_out.ptr;
    MC_CHECK(c, launch_reduce_range((const double*)c->part.ptr, (double*)c->hist_acc.ptr, grid, c->hist_d, c->nb,
                                    adj ? 1 : 0, out, out + 3, c->stream));
    MC_CHECK(c, cudaMemcpyAsync(sums, out, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    if (adj && C) {
        const size_t kept = (size_t)c->hist_d * c->nb, all = (size_t)c->d * c->nb;
        MC_CHECK(c, cudaMemcpyAsync(C, out + 3, sizeof(double) * kept, cudaMemcpyDeviceToHost, c->stream));
        std::memset(C + kept, 0, sizeof(double) * (all - kept));  // m-Cubes1D: no histogram on axes 1..d-1
    }
    MC_CHECK(c, cudaStreamSynchronize(c->stream));
    return MCUBES_OK;
}

mcubes_status mcubes_shard_partial_len(mcubes_ctx* c, long long* len)
{
    if (!c || !len) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    *len = MCUBES_SHARD_HEAD + (long long)c->hist_d * c->nb;
    return MCUBES_OK;
}

// A rank's share of the next iteration: the iteration's own sampling launch
// (device state: iteration index, the skip after convergence) over a cube
// range, whose block partials and histogram are then reduced into the
// caller's partial instead of into the iteration.
mcubes_status mcubes_shard_sample(mcubes_ctx* c, long long cube_begin, long long cube_end, double* d_partial)
{
    if (!c || !d_partial) return MCUBES_EINVAL;
    if (!c->ready || c->shard_open || c->it_enqueued >= c->itmax) return MCUBES_ESTATE;
    if (cube_begin < 0 || cube_end < cube_begin || cube_end > c->m) return MCUBES_EINVAL;
    MC_CHECK(c, cudaSetDevice(c->device));
    const bool adjust = c->it_enqueued < c->ita;
    VsArgs a = c->vs;
    a.split = 1;  // a range pass: the partials are sums over whole cubes
    a.cube_begin = (uint64_t)cube_begin;
    a.cube_end = (uint64_t)cube_end;
    a.perm_k = cube_permutation((uint64_t)(cube_end - cube_begin));
    const int grid = adjust ? c->grid_res_adj : c->grid_res_noadj;
    const size_t smem = adjust ? c->smem_adj : c->smem_noadj;
    EventPair ev;
    if (c->timing) {
        ev = take_events(c);
        MC_CHECK(c, cudaEventRecord(ev.a, c->stream));
    }
    MC_CHECK(c, launch_vsample(c->fid, c->mixed, adjust, a, grid, smem, c->stream));
    if (c->timing) {
        MC_CHECK(c, cudaEventRecord(ev.b, c->stream));
        c->ev_sample.push_back(ev);
    }
    if (!adjust)
        MC_CHECK(c, cudaMemsetAsync(d_partial + MCUBES_SHARD_HEAD, 0, sizeof(double) * c->hist_d * c->nb,
                                    c->stream));
    MC_CHECK(c, launch_reduce_range((const double*)c->part.ptr, (double*)c->hist_acc.ptr, grid, c->hist_d, c->nb,
                                    adjust ? 1 : 0, d_partial, d_partial + MCUBES_SHARD_HEAD, c->stream));
    c->shard_open = true;
    c->shard_adjust = adjust;
    return MCUBES_OK;
}

mcubes_status mcubes_shard_finish(mcubes_ctx* c, const double* d_gathered, int nranks)
{
    if (!c || !d_gathered || nranks < 1) return MCUBES_EINVAL;
    if (!c->ready || !c->shard_open) return MCUBES_ESTATE;
    MC_CHECK(c, cudaSetDevice(c->device));
    const int len = MCUBES_SHARD_HEAD + c->hist_d * c->nb;
    MC_CHECK(c, launch_combine_shards(d_gathered, nranks, len, (double*)c->part.ptr, (double*)c->hist_acc.ptr,
                                      c->stream));
    RefineArgs r = c->rf;
    r.nblocks = 1;  // the combined sums, as one block's partial
    r.split = 1;
    r.adjust = c->shard_adjust ? 1 : 0;
    EventPair ev;
    if (c->timing) {
        ev = take_events(c);
        MC_CHECK(c, cudaEventRecord(ev.a, c->stream));
    }
    MC_CHECK(c, launch_refine(r, c->stream));
    if (c->timing) {
        MC_CHECK(c, cudaEventRecord(ev.b, c->stream));
        c->ev_refine.push_back(ev);
    }
    ++c->it_enqueued;
    c->shard_open = false;
    return MCUBES_OK;
}

mcubes_status mcubes_geometry_get(mcubes_ctx* c, long long* g, long long* m, long long* p, int* lanes,
                                  int* blocks)
{
    if (!c) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    if (g) *g = c->g;
    if (m) *m = c->m;
    if (p) *p = c->p;
    if (lanes) *lanes = c->lanes;
    if (blocks) *blocks = c->ita > 0 ? c->grid_adj : c->grid_noadj;
    return MCUBES_OK;
}

mcubes_status mcubes_timing_reset(mcubes_ctx* c, int enable)
{
    if (!c) return MCUBES_EINVAL;
    MC_CHECK(c, cudaSetDevice(c->device));
    MC_CHECK(c, cudaStreamSynchronize(c->stream));
    recycle_events(c);
    c->timing = enable != 0;
    return MCUBES_OK;
}

mcubes_status mcubes_timing_get(mcubes_ctx* c, double* sample_ms, int* sample_launches, double* refine_ms,
                                int* refine_launches)
{
    if (!c) return MCUBES_EINVAL;
    MC_CHECK(c, cudaSetDevice(c->device));
    MC_CHECK(c, cudaStreamSynchronize(c->stream));
    double ts = 0.0, tr = 0.0;
    for (auto& e : c->ev_sample) {
        float ms = 0.f;
        MC_CHECK(c, cudaEventElapsedTime(&ms, e.a, e.b));
        ts += ms;
    }
    for (auto& e : c->ev_refine) {
        float ms = 0.f;
        MC_CHECK(c, cudaEventElapsedTime(&ms, e.a, e.b));
        tr += ms;
    }
    if (sample_ms) *sample_ms = ts;
    if (sample_launches) *sample_launches = (int)c->ev_sample.size();
    if (refine_ms) *refine_ms = tr;
    if (refine_launches) *refine_launches = (int)c->ev_refine.size();
    return MCUBES_OK;
}

mcubes_status mcubes_integrate_batch(mcubes_ctx* c, int n, const mcubes_request* reqs, mcubes_result* outs)
{
    if (!c || n < 0 || (n > 0 && (!reqs || !outs))) return MCUBES_EINVAL;
    if (c->opts.one_dim) return MCUBES_EINVAL;  // the batched kernels keep a histogram per axis
    if (n == 0) return MCUBES_OK;
    if (n > 65535) return MCUBES_EINVAL;
    int itcap = 1;
    for (int i = 0; i < n; ++i) {
        if (reqs[i].itmax < 1 || reqs[i].itmax > MCUBES_ITMAX_MAX) return MCUBES_EINVAL;
        itcap = std::max(itcap, reqs[i].itmax);
    }
    MC_CHECK(c, cudaSetDevice(c->device));
    if (!c->engine) c->engine = new (std::nothrow) BatchEngine(c->device, c->stream, c->num_sms, c->opts);
    if (!c->engine) return MCUBES_ENOMEM;
    BatchEngine& E = *c->engine;
    MC_CHECK(c, E.reserve(std::max(n, E.capacity()), std::max(itcap, E.itcap())));
    c->batch_slots.assign(n, -1);
    c->batch_dims.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        c->batch_dims[i] = reqs[i].d;
        const mcubes_status st = E.admit(reqs[i], i, &c->batch_slots[i]);
        if (st != MCUBES_OK) {
            // nothing has run: drop what was admitted
            std::vector<std::pair<long long, mcubes_result>> none;
            delete c->engine;
            c->engine = nullptr;
            c->batch_slots.clear();
            return st;
        }
    }
    int ran = 1;
    while (ran > 0) MC_CHECK(c, E.step(&ran));
    std::vector<std::pair<long long, mcubes_result>> done;
    E.finished(&done, true);
    for (auto& kv : done) outs[kv.first] = kv.second;
    return MCUBES_OK;
}

mcubes_status mcubes_batch_trace_get(mcubes_ctx* c, int i, double* I_it, double* var_it, int cap, int* n,
                                     double* grid, double* C)
{
    if (!c || cap < 0 || (cap > 0 && (!I_it || !var_it))) return MCUBES_EINVAL;
    if (!c->engine || i < 0 || i >= (int)c->batch_slots.size() || c->batch_slots[i] < 0) return MCUBES_EINVAL;
    MC_CHECK(c, cudaSetDevice(c->device));
    MC_CHECK(c, c->engine->read_slot(c->batch_slots[i], I_it, var_it, cap, n, grid, C));
    return MCUBES_OK;
}

}  // extern "C"
