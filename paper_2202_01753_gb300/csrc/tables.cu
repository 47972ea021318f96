// tables.cu -- upload of the interpolation tables read by TABLE integrands
// (C ABI in include/mcubes.h; the paper's stateful integrands of Sec. 6.1,
// whose functors read tabulated data).  The tables live in one device
// allocation per precision, read by the kernels through the L1/L2 caches;
// a small device array of descriptors (TableDesc) points into them.  Host
// code only.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ctx_internal.h"

using namespace mc;

namespace {

mcubes_status fail(mcubes_ctx* c, cudaError_t e)
{
    std::snprintf(c->cuda_err, sizeof c->cuda_err, "%s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MCUBES_ENOMEM : MCUBES_ECUDA;
}

// Number of values of a valid table, or 0 if the table is unusable.
size_t table_count(const mcubes_table& t)
{
    if (t.ndim != 1 && t.ndim != 2) return 0;
    if (t.n[0] < 2 || (t.ndim == 2 && t.n[1] < 2) || !t.values) return 0;
    for (int a = 0; a < t.ndim; ++a)
        if (!std::isfinite(t.lo[a]) || !std::isfinite(t.hi[a]) || !(t.lo[a] < t.hi[a])) return 0;
    const size_t n = (size_t)t.n[0] * (size_t)(t.ndim == 2 ? t.n[1] : 1);
    if (n > ((size_t)1 << 31)) return 0;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(t.values[i])) return 0;
    return n;
}

}  // namespace

#define TB_CHECK(ctx, expr)                              \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) return fail((ctx), _e);   \
    } while (0)

extern "C" mcubes_status mcubes_tables_set(mcubes_ctx* c, int n, const mcubes_table* tables)
{
    if (!c || n < 0 || n > MCUBES_TABLES_MAX || (n > 0 && !tables)) return MCUBES_EINVAL;
    std::vector<size_t> count(n), offset(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        count[i] = table_count(tables[i]);
        if (!count[i]) return MCUBES_EINVAL;
        offset[i] = total;
        total += count[i];
    }
    TB_CHECK(c, cudaSetDevice(c->device));
    TB_CHECK(c, cudaStreamSynchronize(c->stream));  // iterations in flight may still read the old tables
    c->ready = false;                                // a problem set up earlier points at them
    c->tabs_host.clear();
    if (n == 0) {
        c->tab_v.release();
        c->tab_vf.release();
        c->tab_desc.release();
        return MCUBES_OK;
    }
    TB_CHECK(c, c->tab_v.reserve(sizeof(double) * total));
    TB_CHECK(c, c->tab_vf.reserve(sizeof(float) * total));
    TB_CHECK(c, c->tab_desc.reserve(sizeof(TableDesc) * n));
    double* dv = static_cast<double*>(c->tab_v.ptr);
    float* dvf = static_cast<float*>(c->tab_vf.ptr);
    std::vector<float> f;
    std::vector<TableDesc> desc(n);
    for (int i = 0; i < n; ++i) {
        const mcubes_table& t = tables[i];
        TB_CHECK(c, cudaMemcpy(dv + offset[i], t.values, sizeof(double) * count[i], cudaMemcpyHostToDevice));
        f.resize(count[i]);
        for (size_t k = 0; k < count[i]; ++k) f[k] = (float)t.values[k];
        TB_CHECK(c, cudaMemcpy(dvf + offset[i], f.data(), sizeof(float) * count[i], cudaMemcpyHostToDevice));
        TableDesc& d = desc[i];
        std::memset(&d, 0, sizeof d);
        d.v = dv + offset[i];
        d.vf = dvf + offset[i];
        d.ndim = t.ndim;
        d.n0 = t.n[0];
        d.n1 = t.ndim == 2 ? t.n[1] : 1;
        d.lo0 = t.lo[0];
        d.hi0 = t.hi[0];
        d.s0 = (double)(t.n[0] - 1) / (t.hi[0] - t.lo[0]);
        d.los0 = d.lo0 * d.s0;
        if (t.ndim == 2) {
            d.lo1 = t.lo[1];
            d.hi1 = t.hi[1];
            d.s1 = (double)(t.n[1] - 1) / (t.hi[1] - t.lo[1]);
            d.los1 = d.lo1 * d.s1;
        }
        d.lo0f = (float)d.lo0;
        d.hi0f = (float)d.hi0;
        d.s0f = (float)d.s0;
        d.lo1f = (float)d.lo1;
        d.hi1f = (float)d.hi1;
        d.s1f = (float)d.s1;
    }
    TB_CHECK(c, cudaMemcpy(c->tab_desc.ptr, desc.data(), sizeof(TableDesc) * n, cudaMemcpyHostToDevice));
    c->tabs_host = desc;
    return MCUBES_OK;
}
