// checkpoint.cu -- export and import of a context's problem state (C ABI in
// include/mcubes.h).  Everything an iteration reads lives in the context's
// device buffers (the double-double grid and the DevState record), so a
// checkpoint is those bytes plus what mcubes_setup needs to rebuild the
// launch arguments.  Host code only.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ctx_internal.h"

using namespace mc;

namespace {

constexpr char kMagic[8] = {'M', 'C', 'U', 'B', 'E', 'S', 'C', 'K'};
constexpr uint32_t kVersion = 1;

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;    // sizeof(CkptHeader)
    uint64_t total_bytes;     // header + grid + state
    uint32_t state_bytes;     // sizeof(DevState)
    int32_t fid, d, nb, itmax, nparams, it_enqueued;
    long long ncall;
    double rel_tol, abs_tol;
    mcubes_opts opts;
    double params[kParMax];
    double lo[kDMax], hi[kDMax];
};

size_t grid_bytes(int d, int nb) { return 2 * sizeof(double) * (size_t)d * (size_t)nb; }

size_t ckpt_bytes(int d, int nb) { return sizeof(CkptHeader) + grid_bytes(d, nb) + sizeof(DevState); }

mcubes_status fail(mcubes_ctx* c, cudaError_t e)
{
    std::snprintf(c->cuda_err, sizeof c->cuda_err, "%s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MCUBES_ENOMEM : MCUBES_ECUDA;
}

// High parts strictly increasing in (0, 1], the last edge exactly 1 + 0.
bool grid_valid(const double* g, int d, int nb)
{
    const double* lo = g + (size_t)d * nb;
    for (int j = 0; j < d; ++j) {
        double prev = 0.0;
        for (int k = 0; k < nb; ++k) {
            const double v = g[(size_t)j * nb + k];
            if (!(v > prev) || !(v <= 1.0) || !std::isfinite(lo[(size_t)j * nb + k])) return false;
            prev = v;
        }
        if (prev != 1.0 || lo[(size_t)j * nb + nb - 1] != 0.0) return false;
    }
    return true;
}

bool state_valid(const DevState& s, int itmax)
{
    if (s.n < 0 || s.n > itmax || s.it > (uint32_t)itmax) return false;
    if (s.error < MCUBES_OK || s.error > MCUBES_ESTATE) return false;
    return true;
}

}  // namespace

#define CK_CHECK(ctx, expr)                              \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) return fail((ctx), _e);   \
    } while (0)

extern "C" {

mcubes_status mcubes_state_size(mcubes_ctx* c, long long* bytes)
{
    if (!c || !bytes) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    *bytes = (long long)ckpt_bytes(c->d, c->nb);
    return MCUBES_OK;
}

mcubes_status mcubes_problem_get(mcubes_ctx* c, int* integrand_id, int* d, int* nb, int* itmax,
                                 int* iterations_enqueued)
{
    if (!c) return MCUBES_EINVAL;
    if (!c->ready) return MCUBES_ESTATE;
    if (integrand_id) *integrand_id = c->fid;
    if (d) *d = c->d;
    if (nb) *nb = c->nb;
    if (itmax) *itmax = c->itmax;
    if (iterations_enqueued) *iterations_enqueued = c->it_enqueued;
    return MCUBES_OK;
}

mcubes_status mcubes_state_export(mcubes_ctx* c, void* buf, long long cap)
{
    if (!c || !buf) return MCUBES_EINVAL;
    if (!c->ready || c->shard_open) return MCUBES_ESTATE;  // a sharded pass is between sample and finish
    const size_t need = ckpt_bytes(c->d, c->nb);
    if (cap < (long long)need) return MCUBES_EINVAL;
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kMagic, sizeof kMagic);
    h.version = kVersion;
    h.header_bytes = sizeof(CkptHeader);
    h.total_bytes = need;
    h.state_bytes = sizeof(DevState);
    h.fid = c->fid;
    h.d = c->d;
    h.nb = c->nb;
    h.itmax = c->itmax;
    h.nparams = (int32_t)c->prob_params.size();
    h.it_enqueued = c->it_enqueued;
    h.ncall = c->ncall;
    h.rel_tol = c->rel_tol;
    h.abs_tol = c->abs_tol;
    // field by field, so that the struct's padding stays zero and a
    // re-exported checkpoint is byte-identical
    h.opts.nbins = c->opts.nbins;
    h.opts.ita = c->opts.ita;
    h.opts.g_override = c->opts.g_override;
    h.opts.alpha = c->opts.alpha;
    h.opts.seed = c->opts.seed;
    h.opts.precision = c->opts.precision;
    h.opts.lanes_per_cube = c->opts.lanes_per_cube;
    h.opts.blocks_per_sm = c->opts.blocks_per_sm;
    h.opts.one_dim = c->opts.one_dim;
    std::memcpy(h.params, c->prob_params.data(), sizeof(double) * c->prob_params.size());
    std::memcpy(h.lo, c->prob_lo.data(), sizeof(double) * c->d);
    std::memcpy(h.hi, c->prob_hi.data(), sizeof(double) * c->d);
    unsigned char* out = static_cast<unsigned char*>(buf);
    std::memcpy(out, &h, sizeof h);
    CK_CHECK(c, cudaSetDevice(c->device));
    CK_CHECK(c, cudaMemcpyAsync(out + sizeof h, c->grid.ptr, grid_bytes(c->d, c->nb), cudaMemcpyDeviceToHost,
                                c->stream));
    CK_CHECK(c, cudaMemcpyAsync(out + sizeof h + grid_bytes(c->d, c->nb), c->state.ptr, sizeof(DevState),
                                cudaMemcpyDeviceToHost, c->stream));
    CK_CHECK(c, cudaStreamSynchronize(c->stream));
    return MCUBES_OK;
}

mcubes_status mcubes_state_import(mcubes_ctx* c, const void* buf, long long size)
{
    if (!c || !buf || size < (long long)sizeof(CkptHeader)) return MCUBES_EINVAL;
    c->ready = false;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, kMagic, sizeof kMagic) != 0 || h.version != kVersion) return MCUBES_EINVAL;
    if (h.header_bytes != sizeof(CkptHeader) || h.state_bytes != sizeof(DevState)) return MCUBES_EINVAL;
    if (h.d < 1 || h.d > kDMax || h.nparams < 0 || h.nparams > kParMax || h.nb != h.opts.nbins) return MCUBES_EINVAL;
    if (h.nb < 2 || h.nb > MCUBES_NBMAX || h.itmax < 1 || h.itmax > MCUBES_ITMAX_MAX) return MCUBES_EINVAL;
    if (h.total_bytes != ckpt_bytes(h.d, h.nb) || (unsigned long long)size != h.total_bytes) return MCUBES_EINVAL;
    if (h.it_enqueued < 0 || h.it_enqueued > h.itmax) return MCUBES_EINVAL;
    const unsigned char* in = static_cast<const unsigned char*>(buf);
    std::vector<double> grid(2 * (size_t)h.d * h.nb);  // the caller's buffer need not be aligned
    std::memcpy(grid.data(), in + sizeof h, grid_bytes(h.d, h.nb));
    DevState st;
    std::memcpy(&st, in + sizeof h + grid_bytes(h.d, h.nb), sizeof st);
    if (!grid_valid(grid.data(), h.d, h.nb) || !state_valid(st, h.itmax)) return MCUBES_EINVAL;

    mcubes_status s = mcubes_set_opts(c, &h.opts);
    if (s != MCUBES_OK) return s;
    s = mcubes_setup(c, h.fid, h.params, h.nparams, h.d, h.lo, h.hi, h.ncall, h.itmax, h.rel_tol, h.abs_tol);
    if (s != MCUBES_OK) return s;
    c->ready = false;
    CK_CHECK(c, cudaMemcpyAsync(c->grid.ptr, grid.data(), grid_bytes(h.d, h.nb), cudaMemcpyHostToDevice, c->stream));
    CK_CHECK(c, cudaMemcpyAsync(c->state.ptr, &st, sizeof st, cudaMemcpyHostToDevice, c->stream));
    CK_CHECK(c, ctx_refresh_cells(c));
    CK_CHECK(c, cudaStreamSynchronize(c->stream));  // grid and st live on this stack frame
    c->it_enqueued = h.it_enqueued;
    c->ready = true;
    return MCUBES_OK;
}

}  // extern "C"
