// batch.cu -- the batched engine: a table of resident integrals ("slots"),
// each with its own grid, iteration state and history on the device, that
// are iterated together.  One iteration of every live integral is one
// persistent sampling launch (batch.cuh) plus one refinement launch
// (Adjust-Bin-Bounds per axis, Weighted-Estimates and Check-Convergence per
// integral, Alg. 2); both are captured once as a CUDA graph whose arguments
// live in device memory, and the host rewrites the work partition between
// replays.  Integrals may be admitted and retired between iterations, which
// is what the continuous-batching server (server.cu) builds on.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch_engine.h"
#include "refine_dev.cuh"

namespace mc {
bool integrand_prepare(int id, const double* p, int np, int d, FamParams* out);
bool geometry(int d, long long ncall, long long g_override, int nb, long long* g, long long* m, long long* p);
cudaError_t launch_vsample_batch_const(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_const(bool, int, size_t, int*);
cudaError_t launch_vsample_batch_gauss(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_gauss(bool, int, size_t, int*);
cudaError_t launch_vsample_batch_corner(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_corner(bool, int, size_t, int*);
cudaError_t launch_vsample_batch_osc(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_osc(bool, int, size_t, int*);
cudaError_t launch_vsample_batch_prodpeak(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_prodpeak(bool, int, size_t, int*);
cudaError_t launch_vsample_batch_c0(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_c0(bool, int, size_t, int*);
cudaError_t launch_vsample_batch_discont(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_discont(bool, int, size_t, int*);
cudaError_t launch_vsample_batch_cosmo6(bool, int, const BatchArgs&, int, size_t, cudaStream_t);
cudaError_t vsample_batch_occupancy_cosmo6(bool, int, size_t, int*);

cudaError_t launch_vsample_batch(int cls, bool mixed, const BatchArgs& a, int grid, size_t smem, cudaStream_t s)
{
    const int dcls = cls % kDMax + 1;  // the class's dimension
    switch (cls / kDMax) {
    case MCUBES_F_CONST: return launch_vsample_batch_const(mixed, dcls, a, grid, smem, s);
    case MCUBES_F_GAUSS: return launch_vsample_batch_gauss(mixed, dcls, a, grid, smem, s);
    case MCUBES_F_CORNER: return launch_vsample_batch_corner(mixed, dcls, a, grid, smem, s);
    case MCUBES_F_OSC: return launch_vsample_batch_osc(mixed, dcls, a, grid, smem, s);
    case MCUBES_F_PRODPEAK: return launch_vsample_batch_prodpeak(mixed, dcls, a, grid, smem, s);
    case MCUBES_F_C0: return launch_vsample_batch_c0(mixed, dcls, a, grid, smem, s);
    case MCUBES_F_DISCONT: return launch_vsample_batch_discont(mixed, dcls, a, grid, smem, s);
    case MCUBES_F_COSMO6: return launch_vsample_batch_cosmo6(mixed, dcls, a, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t vsample_batch_occupancy(int cls, bool mixed, size_t smem, int* blocks)
{
    const int dcls = cls % kDMax + 1;  // the class's dimension
    switch (cls / kDMax) {
    case MCUBES_F_CONST: return vsample_batch_occupancy_const(mixed, dcls, smem, blocks);
    case MCUBES_F_GAUSS: return vsample_batch_occupancy_gauss(mixed, dcls, smem, blocks);
    case MCUBES_F_CORNER: return vsample_batch_occupancy_corner(mixed, dcls, smem, blocks);
    case MCUBES_F_OSC: return vsample_batch_occupancy_osc(mixed, dcls, smem, blocks);
    case MCUBES_F_PRODPEAK: return vsample_batch_occupancy_prodpeak(mixed, dcls, smem, blocks);
    case MCUBES_F_C0: return vsample_batch_occupancy_c0(mixed, dcls, smem, blocks);
    case MCUBES_F_DISCONT: return vsample_batch_occupancy_discont(mixed, dcls, smem, blocks);
    case MCUBES_F_COSMO6: return vsample_batch_occupancy_cosmo6(mixed, dcls, smem, blocks);
    default: return cudaErrorInvalidValue;
    }
}

namespace {

using namespace refine_detail;

// Map cells of one axis of a slot from its grid (block-wide).
__device__ void slot_cells_row(const BatchDesc& D, int j)
{
    const int nb = (int)D.nb;
    const double* row = D.grid + (size_t)j * nb;
    const double* row_lo = D.grid + (size_t)D.d * nb + (size_t)j * nb;
    const double inv_g = 1.0 / (double)D.g;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const size_t i = (size_t)j * nb + k;
        if (D.mixed) static_cast<float2*>(D.cells)[i] = map_cell_f32(row, row_lo, k, D.lo[j], D.scale[j], nb);
        else static_cast<double2*>(D.cells)[i] = map_cell_f64(row, row_lo, k, D.lo[j], D.scale[j], inv_g);
    }
}

__device__ void refine_one(const BatchRefineArgs& a, uint32_t j, double* scratch);

// Refinement of one iteration of every live integral: block row y handles
// live integrals y, y + gridDim.y, ...; for integral j, block (axis, row)
// rebins that axis (adjusting iterations) and block (d or 0, row) reduces
// the integral's segment partials in order and weighs the iteration.
__global__ void __launch_bounds__(kRefineThreads) refine_batch_kernel(const __grid_constant__ BatchRefineArgs a)
{
    __shared__ double scratch[33];
    const uint32_t nlive = *a.nlive;
    for (uint32_t j = blockIdx.y; j < nlive; j += gridDim.y) {
        refine_one(a, j, scratch);
        __syncthreads();  // scratch is reused by the next integral
    }
}

__device__ void refine_one(const BatchRefineArgs& a, uint32_t j, double* scratch)
{
    const uint32_t slot = a.live[j];
    const BatchDesc& D = a.desc[slot];
    const uint32_t s0 = a.live_seg[j], s1 = a.live_seg[j + 1];
    const bool adjust = a.segs[s0].adjust != 0;
    const int d = (int)D.d, nb = (int)D.nb;
    const int nrebin = adjust ? d : 0;
    if ((int)blockIdx.x > nrebin) return;
    BatchState* st = a.st + slot;
    // finished in an earlier iteration of this step (its sampling was skipped).
    // The finalising block of this launch may set these while a rebinning
    // block reads them: that block then skips a rebin no iteration will use.
    // One thread reads, so that the whole block takes the same branch.
    __shared__ int skip;
    if (threadIdx.x == 0)
        skip = *(volatile const int*)&st->done || (int)*(volatile const uint32_t*)&st->it >= D.itmax;
    __syncthreads();
    const bool finished = skip != 0;
    __syncthreads();  // skip is rewritten for the next integral
    if (finished) return;
    if ((int)blockIdx.x == nrebin) {
        const IterRecord r{&st->it, &st->done, &st->error, &st->n, &st->converged, &st->estimate, &st->sigma,
                           &st->chi2_dof, D.hist_I, D.hist_V, D.itmax, D.rel_tol, D.abs_tol};
        finalize_iteration(a.seg_part + 3 * (size_t)s0, (int)(s1 - s0), (double)D.m, r);
    } else {
        const int ax = blockIdx.x;
        const size_t off = (size_t)ax * nb;
        const size_t elem = a.hist_is_float ? sizeof(float) : sizeof(double);
        const char* parts = static_cast<const char*>(a.seg_hist) + (a.segs[s0].hist_off + off) * elem;
        rebin_axis(parts, (size_t)d * nb, (int)(s1 - s0), a.hist_is_float != 0, nb, a.alpha, D.grid + off,
                   D.grid + (size_t)d * nb + off, D.hist + off, &st->error, &st->done, scratch);
        __syncthreads();  // the axis's new edges are in global memory: rebuild its map cells
        slot_cells_row(D, ax);
    }
}

// Uniform grid (Init-Bins, Alg. 2, double-double edges), empty histogram and
// a cleared state for every newly admitted slot.
__global__ void init_slots_kernel(const BatchDesc* desc, BatchState* st, const uint32_t* slots, int count)
{
    const uint32_t slot = slots[blockIdx.x];
    const BatchDesc& D = desc[slot];
    const int d = (int)D.d, nb = (int)D.nb;
    for (int i = threadIdx.x; i < d * nb; i += blockDim.x) {
        const int k = i % nb;
        double hi = 1.0, lo = 0.0;
        if (k != nb - 1) {
            hi = __ddiv_rn((double)(k + 1), (double)nb);
            lo = __ddiv_rn(__fma_rn(-hi, (double)nb, (double)(k + 1)), (double)nb);
        }
        D.grid[i] = hi;
        D.grid[(size_t)d * nb + i] = lo;
        D.hist[i] = 0.0;
    }
    __syncthreads();  // the grid is in global memory: build the map cells
    for (int j = 0; j < d; ++j) slot_cells_row(D, j);
    if (threadIdx.x == 0) {
        BatchState z;
        memset(&z, 0, sizeof z);
        st[slot] = z;
    }
}

}  // namespace

cudaError_t launch_refine_batch(const BatchRefineArgs& a, int capacity, int rows, cudaStream_t s)
{
    refine_batch_kernel<<<dim3(kDMax + 1, std::max(1, std::min(capacity, rows))), kRefineThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init_slots(const BatchDesc* desc, BatchState* st, const uint32_t* slots, int count,
                              cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    init_slots_kernel<<<count, 256, 0, s>>>(desc, st, slots, count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------
BatchEngine::BatchEngine(int device, cudaStream_t stream, int num_sms, const mcubes_opts& o)
    : device_(device), stream_(stream), num_sms_(num_sms), opts_(o), mixed_(o.precision == MCUBES_MIXED)
{
}

BatchEngine::~BatchEngine() { release(); }

void BatchEngine::release()
{
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;
    for (DevBuf* b : {&desc_, &st_, &grids_, &cells_, &hists_, &histories_, &segs_, &blk_seg_, &live_, &live_seg_, &nlive_,
                      &seg_part_, &seg_hist_, &admit_slots_})
        b->release();
    if (h_segs_) cudaFreeHost(h_segs_);
    if (h_small_) cudaFreeHost(h_small_);
    if (h_states_) cudaFreeHost(h_states_);
    h_segs_ = nullptr;
    h_small_ = nullptr;
    h_states_ = nullptr;
    for (cudaStream_t s : branch_) cudaStreamDestroy(s);
    for (cudaEvent_t v : join_) cudaEventDestroy(v);
    if (fork_) cudaEventDestroy(fork_);
    branch_.clear();
    join_.clear();
    fork_ = nullptr;
    capacity_ = 0;
}

size_t BatchEngine::smem_bytes(int cls) const
{
    const int dcls = cls % kDMax + 1;  // the class's dimension
    return (size_t)dcls * opts_.nbins * (cell_bytes(mixed_) + hist_bytes(mixed_));
}

int BatchEngine::class_blocks(int cls) const { return std::max(1, std::min(tuned_bps_, occ_[cls])) * num_sms_; }

cudaError_t BatchEngine::reserve(int capacity, int itcap)
{
    if (capacity <= capacity_ && itcap <= itcap_) return cudaSuccess;
    release();
    const int nb = opts_.nbins;
    cudaError_t e;
    int occ_max = 1;
    for (int c = 0; c < kNumClasses; ++c) {
        occ_[c] = 0;
        if (c / kDMax == MCUBES_F_COSMO6 && c % kDMax != 5) continue;  // six axes only
        if ((e = vsample_batch_occupancy(c, mixed_, smem_bytes(c), &occ_[c]))) return e;
        occ_max = std::max(occ_max, occ_[c]);
    }
    bmax_ = occ_max * num_sms_;
    const size_t segmax = (size_t)capacity + (size_t)kNumClasses * bmax_ + 1;
    const size_t grid_stride = 2 * (size_t)kDMax * nb, hist_stride = (size_t)kDMax * nb;
    const size_t elem = mixed_ ? sizeof(float) : sizeof(double);
    const size_t table = (size_t)kNumClasses * (bmax_ + 1);
    // partial histograms: an adjusting segment takes d * nb entries, and a
    // class has at most one segment per integral plus one per boundary
    // between its blocks (at most occ * SMs of them)
    size_t hist_cap = (size_t)capacity * hist_stride;
    for (int c = 0; c < kNumClasses; ++c) hist_cap += (size_t)occ_[c] * num_sms_ * (size_t)(c % kDMax + 1) * nb;
    if ((e = desc_.reserve(sizeof(BatchDesc) * capacity)) || (e = st_.reserve(sizeof(BatchState) * capacity)) ||
        (e = grids_.reserve(sizeof(double) * grid_stride * capacity)) ||
        (e = cells_.reserve(cell_bytes(mixed_) * hist_stride * capacity)) ||
        (e = hists_.reserve(sizeof(double) * hist_stride * capacity)) ||
        (e = histories_.reserve(sizeof(double) * 2 * (size_t)itcap * capacity)) ||
        (e = segs_.reserve(sizeof(BatchSeg) * segmax)) || (e = blk_seg_.reserve(sizeof(uint32_t) * table)) ||
        (e = live_.reserve(sizeof(uint32_t) * capacity)) ||
        (e = live_seg_.reserve(sizeof(uint32_t) * (capacity + 1))) || (e = nlive_.reserve(sizeof(uint32_t))) ||
        (e = seg_part_.reserve(sizeof(double) * 3 * segmax)) ||
        (e = seg_hist_.reserve(elem * hist_cap)) ||
        (e = admit_slots_.reserve(sizeof(uint32_t) * capacity)))
        return e;
    if ((e = cudaHostAlloc((void**)&h_segs_, sizeof(BatchSeg) * segmax, cudaHostAllocDefault)) ||
        (e = cudaHostAlloc((void**)&h_small_, sizeof(uint32_t) * (table + 2 * (size_t)capacity + 8),
                           cudaHostAllocDefault)) ||
        (e = cudaHostAlloc((void**)&h_states_, sizeof(BatchState) * capacity, cudaHostAllocDefault)))
        return e;
    capacity_ = capacity;
    itcap_ = itcap;
    hist_cap_ = hist_cap;
    slots_.assign(capacity, Slot{});
    hdesc_.assign(capacity, BatchDesc{});
    free_.clear();
    for (int i = capacity - 1; i >= 0; --i) free_.push_back(i);
    pending_.clear();
    return cudaSuccess;
}

int BatchEngine::choose_lanes(long long p) const
{
    if (opts_.lanes_per_cube > 0) return (int)std::min<long long>(opts_.lanes_per_cube, std::max<long long>(p, 1));
    int L = 1;
    while (L < 32 && 2 * L <= p && p / L > lanes_cap_) L *= 2;
    return L;
}

size_t BatchEngine::slot_bytes(const mcubes_opts& o, int itcap)
{
    const size_t bins = (size_t)kDMax * o.nbins;
    const size_t elem = o.precision == MCUBES_MIXED ? sizeof(float) : sizeof(double);
    return sizeof(double) * (3 * bins + 2 * (size_t)itcap) + sizeof(BatchDesc) + sizeof(BatchState) +
           bins * elem + bins * cell_bytes(o.precision == MCUBES_MIXED) + sizeof(BatchSeg) + 3 * sizeof(double) +
           3 * sizeof(uint32_t);
}

mcubes_status BatchEngine::validate(const mcubes_request& r) const
{
    const int d = r.d, nb = opts_.nbins;
    if (d < 1 || d > MCUBES_DMAX || r.ncall < 2 || r.itmax < 1 || r.itmax > itcap_ || !r.lo || !r.hi)
        return MCUBES_EINVAL;
    if (!(r.rel_tol >= 0.0) || !(r.abs_tol >= 0.0)) return MCUBES_EINVAL;
    FamParams fp;
    if (!integrand_prepare(r.integrand_id, r.params, r.nparams, d, &fp)) return MCUBES_EINVAL;
    for (int j = 0; j < d; ++j)
        if (!std::isfinite(r.lo[j]) || !std::isfinite(r.hi[j]) || !(r.lo[j] < r.hi[j])) return MCUBES_EINVAL;
    long long g, m, p;
    if (!geometry(d, r.ncall, opts_.g_override, nb, &g, &m, &p)) return MCUBES_EINVAL;
    if (occ_[batch_class(r.integrand_id, d)] < 1) return MCUBES_EINVAL;
    return MCUBES_OK;
}

mcubes_status BatchEngine::admit(const mcubes_request& r, long long tag, int* slot_out)
{
    const mcubes_status vst = validate(r);
    if (vst != MCUBES_OK) return vst;
    const int d = r.d, nb = opts_.nbins;
    FamParams fp;
    integrand_prepare(r.integrand_id, r.params, r.nparams, d, &fp);
    long long g, m, p;
    geometry(d, r.ncall, opts_.g_override, nb, &g, &m, &p);
    if (free_.empty()) return MCUBES_ENOMEM;
    const int slot = free_.back();
    free_.pop_back();
    BatchDesc& D = hdesc_[slot];
    std::memset(&D, 0, sizeof D);
    D.d = (uint32_t)d;
    D.nb = (uint32_t)nb;
    D.g = (uint32_t)g;
    D.gmagic = (uint32_t)(0xFFFFFFFFu / (uint32_t)g);
    D.p = (uint32_t)p;
    D.lanes = (uint32_t)choose_lanes(p);
    D.key0 = (uint32_t)r.seed;
    D.key1 = (uint32_t)(r.seed >> 32);
    D.family = r.integrand_id;
    D.ita = opts_.ita < 0 ? r.itmax : std::min(opts_.ita, r.itmax);
    D.itmax = r.itmax;
    D.m = (uint64_t)m;
    D.jac0 = jacobian_scale(g, nb, d) * family_jac_factor(r.integrand_id, fp);
    D.phi_scale_f = (float)(1.0 / ((double)g * nb));
    set_moment_scales(D, p);
    for (int j = 0; j < d; ++j) {
        D.lo[j] = r.lo[j];
        D.scale[j] = r.hi[j] - r.lo[j];
    }
    D.fam = fp;
    const size_t grid_stride = 2 * (size_t)kDMax * nb, hist_stride = (size_t)kDMax * nb;
    D.grid = (double*)grids_.ptr + grid_stride * slot;
    D.cells = static_cast<unsigned char*>(cells_.ptr) + cell_bytes(mixed_) * hist_stride * slot;
    D.mixed = mixed_ ? 1 : 0;
    D.hist = (double*)hists_.ptr + hist_stride * slot;
    D.hist_I = (double*)histories_.ptr + 2 * (size_t)itcap_ * slot;
    D.hist_V = D.hist_I + itcap_;
    D.rel_tol = r.rel_tol;
    D.abs_tol = r.abs_tol;
    Slot& S = slots_[slot];
    S = Slot{};
    S.used = true;
    S.tag = tag;
    S.work = (double)m * (double)p;
    S.g = g;
    S.m = m;
    S.p = p;
    pending_.push_back(slot);
    if (slot_out) *slot_out = slot;
    return MCUBES_OK;
}

cudaError_t BatchEngine::flush_admissions()
{
    if (pending_.empty()) return cudaSuccess;
    cudaError_t e;
    for (int slot : pending_) {
        if ((e = cudaMemcpyAsync((BatchDesc*)desc_.ptr + slot, &hdesc_[slot], sizeof(BatchDesc),
                                 cudaMemcpyHostToDevice, stream_)))
            return e;
    }
    uint32_t* hs = h_small_;  // staging: slot list
    for (size_t i = 0; i < pending_.size(); ++i) hs[i] = (uint32_t)pending_[i];
    if ((e = cudaMemcpyAsync(admit_slots_.ptr, hs, sizeof(uint32_t) * pending_.size(), cudaMemcpyHostToDevice,
                             stream_)))
        return e;
    if ((e = launch_init_slots((const BatchDesc*)desc_.ptr, (BatchState*)st_.ptr, (const uint32_t*)admit_slots_.ptr,
                               (int)pending_.size(), stream_)))
        return e;
    e = cudaStreamSynchronize(stream_);  // the pinned staging is reused below
    pending_.clear();
    return e;
}

void BatchEngine::live_slots(std::vector<int>* live, ClassMask* class_mask) const
{
    live->clear();
    class_mask->reset();
    std::vector<int> by_class[kNumClasses];
    for (int s = 0; s < capacity_; ++s) {
        const Slot& S = slots_[s];
        if (S.used && !S.finished && S.it < hdesc_[s].itmax)
            by_class[batch_class(hdesc_[s].family, (int)hdesc_[s].d)].push_back(s);
    }
    for (int c = 0; c < kNumClasses; ++c) {
        if (by_class[c].empty()) continue;
        class_mask->set(c);
        live->insert(live->end(), by_class[c].begin(), by_class[c].end());
    }
}

// Fewest samples per chunk of a class's work (measured, mixed precision: the
// 4096-integral batch 1934-1942 integrals/s against 1880-1919 with one chunk
// per block, the serving mix without retries at 2000 requests/s p50 2.6 ms and
// p99 3.9 ms against 15.2 and 21.0; 8192: 3.1 and 4.1 ms, 32768: 7.1 and 8.5).
constexpr double kMinBlockSamples = 2048.0;

// For every class, lays its live integrals' samples end to end and cuts the
// line into equal chunks, at least kMinBlockSamples samples each and at most
// class_blocks(class) of them; cube c of an integral goes to the chunk
// holding its first sample.  Writes the segment list (class by
// class, then block by block), every class's block table (a fixed region of
// bmax_+1 entries per class; classes without work get empty tables) and the
// live integrals' segment offsets.
void BatchEngine::partition(const std::vector<int>& live, int* nseg_out)
{
    uint32_t* table = h_small_;
    const size_t table_n = (size_t)kNumClasses * (bmax_ + 1);
    uint32_t* live_slot = h_small_ + table_n;
    uint32_t* live_seg = live_slot + capacity_;
    std::memset(table, 0, sizeof(uint32_t) * table_n);
    std::fill(class_load_, class_load_ + kNumClasses, 0.0);
    int nseg = 0;
    size_t hist_off = 0;
    size_t j = 0;
    while (j < live.size()) {
        const int cls = batch_class(hdesc_[live[j]].family, (int)hdesc_[live[j]].d);
        size_t j1 = j;
        double total = 0.0;
        while (j1 < live.size() && batch_class(hdesc_[live[j1]].family, (int)hdesc_[live[j1]].d) == cls)
            total += slots_[live[j1++]].work;
        // chunks of at least kMinBlockSamples samples, at most one per block
        // of the class's launch (its full occupancy): a step of small
        // requests is cut into few chunks (each block's fixed work -- staging
        // a segment's grid, writing its partial histogram -- stays small
        // beside its samples, and the refinement merges fewer segments), a
        // large batch fills every block
        const int blocks_max = class_blocks(cls);
        const int blocks = (int)std::max(1.0, std::min((double)blocks_max, std::ceil(total / kMinBlockSamples)));
        class_load_[cls] = total * (4.0 + hdesc_[live[j]].d) / blocks;
        uint32_t* blk_seg = table + (size_t)cls * (bmax_ + 1);
        const double chunk = total / blocks;
        double start = 0.0;  // first sample of the current integral on the class's line
        int b = 0;
        blk_seg[0] = (uint32_t)nseg;
        for (; j < j1; ++j) {
            const int s = live[j];
            const Slot& S = slots_[s];
            live_slot[j] = (uint32_t)s;
            live_seg[j] = (uint32_t)nseg;
            const bool adjust = S.it < hdesc_[s].ita;
            const double p = (double)S.p;
            uint64_t c = 0;
            while (c < (uint64_t)S.m) {
                const double chunk_end = (b + 1 == blocks) ? 1e300 : (b + 1) * chunk;
                const double cend_d = std::ceil((chunk_end - start) / p);
                const uint64_t cend =
                    cend_d >= (double)S.m ? (uint64_t)S.m : (uint64_t)std::max(cend_d, 0.0);
                if (cend > c) {
                    BatchSeg& g = h_segs_[nseg++];
                    g.slot = (uint32_t)s;
                    g.adjust = adjust ? 1u : 0u;
                    g.c0 = c;
                    g.c1 = cend;
                    g.perm_k = cube_permutation(cend - c);
                    g.hist_off = hist_off;
                    if (adjust) hist_off += (size_t)hdesc_[s].d * hdesc_[s].nb;
                    c = cend;
                }
                if (c < (uint64_t)S.m) blk_seg[++b] = (uint32_t)nseg;  // block b is full
            }
            start += S.work;
        }
        while (b < blocks_max) blk_seg[++b] = (uint32_t)nseg;  // blocks past the chunks: empty
    }
    live_seg[live.size()] = (uint32_t)nseg;
    part_hist_ = hist_off;
    *nseg_out = nseg;
}

cudaError_t BatchEngine::upload_partition(const std::vector<int>& live, int nseg)
{
    cudaError_t e;
    if (part_hist_ > hist_cap_) return cudaErrorInvalidValue;  // never: hist_cap_ bounds every partition
    const size_t table_n = (size_t)kNumClasses * (bmax_ + 1);
    const uint32_t* live_slot = h_small_ + table_n;
    const uint32_t* live_seg = live_slot + capacity_;
    uint32_t* nl = h_small_ + table_n + 2 * (size_t)capacity_ + 1;
    *nl = (uint32_t)live.size();
    if ((e = cudaMemcpyAsync(segs_.ptr, h_segs_, sizeof(BatchSeg) * std::max(nseg, 1), cudaMemcpyHostToDevice,
                             stream_)) ||
        (e = cudaMemcpyAsync(blk_seg_.ptr, h_small_, sizeof(uint32_t) * table_n, cudaMemcpyHostToDevice, stream_)) ||
        (e = cudaMemcpyAsync(live_.ptr, live_slot, sizeof(uint32_t) * std::max<size_t>(live.size(), 1),
                             cudaMemcpyHostToDevice, stream_)) ||
        (e = cudaMemcpyAsync(live_seg_.ptr, live_seg, sizeof(uint32_t) * (live.size() + 1),
                             cudaMemcpyHostToDevice, stream_)) ||
        (e = cudaMemcpyAsync(nlive_.ptr, nl, sizeof(uint32_t), cudaMemcpyHostToDevice, stream_)))
        return e;
    return cudaSuccess;
}

BatchArgs BatchEngine::sample_args(int cls) const
{
    BatchArgs a;
    a.desc = (const BatchDesc*)desc_.ptr;
    a.st = (const BatchState*)st_.ptr;
    a.segs = (BatchSeg*)segs_.ptr;
    a.blk_seg = (const uint32_t*)blk_seg_.ptr + (size_t)cls * (bmax_ + 1);
    a.seg_part = (double*)seg_part_.ptr;
    a.seg_hist = seg_hist_.ptr;
    return a;
}

BatchRefineArgs BatchEngine::refine_args() const
{
    BatchRefineArgs r;
    r.desc = (const BatchDesc*)desc_.ptr;
    r.st = (BatchState*)st_.ptr;
    r.live = (const uint32_t*)live_.ptr;
    r.live_seg = (const uint32_t*)live_seg_.ptr;
    r.nlive = (const uint32_t*)nlive_.ptr;
    r.segs = (const BatchSeg*)segs_.ptr;
    r.seg_part = (const double*)seg_part_.ptr;
    r.seg_hist = seg_hist_.ptr;
    r.hist_is_float = mixed_ ? 1 : 0;
    r.alpha = opts_.alpha;
    return r;
}

// The sampling kernels of the classes in the mask, each on its own branch
// stream forked from stream_ and joined back into it: the kernels write
// disjoint segments, and the blocks of one fill the SMs that another's
// last blocks leave idle.
cudaError_t BatchEngine::enqueue_sampling(const ClassMask& mask)
{
    cudaError_t e;
    const size_t n = mask.count();
    if (!fork_ && (e = cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming))) return e;
    while (branch_.size() < n) {
        cudaStream_t s = nullptr;
        cudaEvent_t v = nullptr;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking))) return e;
        branch_.push_back(s);
        if ((e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming))) return e;
        join_.push_back(v);
    }
    // the classes with the longest blocks first: the SMs their last blocks
    // leave idle are filled by the shorter blocks of the classes after them
    int order[kNumClasses];
    int nc = 0;
    for (int c = 0; c < kNumClasses; ++c)
        if (mask.test(c)) order[nc++] = c;
    std::stable_sort(order, order + nc, [&](int x, int y) { return class_load_[x] > class_load_[y]; });
    if ((e = cudaEventRecord(fork_, stream_))) return e;
    size_t k = 0;
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < nc; ++i) {
        const int c = order[i];
        if ((e = cudaStreamWaitEvent(branch_[k], fork_, 0))) return e;
        if (!le) le = launch_vsample_batch(c, mixed_, sample_args(c), class_blocks(c), smem_bytes(c), branch_[k]);
        if ((e = cudaEventRecord(join_[k], branch_[k]))) return e;
        if ((e = cudaStreamWaitEvent(stream_, join_[k], 0))) return e;
        ++k;
    }
    return le;
}

cudaError_t BatchEngine::enqueue_iteration(const ClassMask& mask)
{
    cudaError_t e = enqueue_sampling(mask);
    if (e) return e;
    return launch_refine_batch(refine_args(), capacity_, 2 * num_sms_, stream_);
}

// One iteration as a CUDA graph: the sampling kernels of the classes in the
// mask as parallel branches, then the refinement.  Re-captured only when a class appears that
// the graph does not launch, or the launch shape changes.
cudaError_t BatchEngine::capture(ClassMask mask)
{
    if (exec_ && (mask & ~graph_mask_).none() && graph_bps_ == tuned_bps_) return cudaSuccess;
    mask |= graph_mask_;
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;
    graph_mask_.reset();
    if (stream_ == nullptr) return cudaSuccess;  // the legacy stream cannot be captured: launch directly
    cudaError_t e = cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal);
    if (e) return e;
    cudaError_t le = enqueue_iteration(mask);
    e = cudaStreamEndCapture(stream_, &graph_);
    if (le) return le;
    if (e) return e;
    if ((e = cudaGraphInstantiate(&exec_, graph_, 0))) return e;
    graph_mask_ = mask;
    graph_bps_ = tuned_bps_;
    return cudaSuccess;
}

// Picks the samples-per-thread cap that sets lanes per cube, by timing
// sampling-only launches of a subset of this batch's first iteration; the
// choice is kept for the life of the engine.  Every class kernel launches
// its full occupancy of blocks per SM (opts.blocks_per_sm, when set, caps
// it) and the partition decides how many of them get work (a chunk of at
// least kMinBlockSamples samples each), so the cubes per block follow from
// a class's work in every step: the tuner used to pick the blocks per SM
// as well, on its small subset, where one block per SM (of three) looked
// faster, and kept it for the work that followed -- there full occupancy
// measured 1.4 times the integrals per second at tolerance on the
// 4096-integral batch and 1.25 times the serving mix's capacity.
cudaError_t BatchEngine::autotune(const std::vector<int>& live, const ClassMask& mask)
{
    if (tuned_) return cudaSuccess;
    int occ_hi = 1;
    for (int c = 0; c < kNumClasses; ++c)
        if (mask.test(c)) occ_hi = std::max(occ_hi, occ_[c]);
    // Timing a handful of small integrals tells the launch shapes apart by
    // noise alone, and the choice is kept for the engine's life: until
    // kTuneMinLive integrals are live (a server's first steps), run with the
    // full occupancy and the middle lanes cap, and tune later.
    constexpr size_t kTuneMinLive = 32;
    constexpr int kEachClassOccupancy = 1 << 16;  // no cap: class_blocks takes each class's own occupancy
    if (live.size() < kTuneMinLive && opts_.blocks_per_sm <= 0 && opts_.lanes_per_cube <= 0) {
        tuned_bps_ = kEachClassOccupancy;
        lanes_cap_ = 64;
        return cudaSuccess;
    }
    std::vector<int> bps_list{opts_.blocks_per_sm > 0 ? std::min(opts_.blocks_per_sm, occ_hi) : kEachClassOccupancy};
    std::vector<int> cap_list =
        opts_.lanes_per_cube > 0 ? std::vector<int>{lanes_cap_} : std::vector<int>{64, 16, 256};
    // a subset of the batch (every k-th integral, class order kept) keeps tuning cheap
    std::vector<int> sub;
    const size_t stride = std::max<size_t>(1, live.size() / 256);
    for (size_t i = 0; i < live.size(); i += stride) sub.push_back(live[i]);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_bps = bps_list.front(), best_cap = cap_list.front();
    cudaError_t e = cudaSuccess;
    for (int cap : cap_list) {
        lanes_cap_ = cap;
        for (int s : sub) {
            hdesc_[s].lanes = (uint32_t)choose_lanes(slots_[s].p);
            if ((e = cudaMemcpyAsync((BatchDesc*)desc_.ptr + s, &hdesc_[s], sizeof(BatchDesc),
                                     cudaMemcpyHostToDevice, stream_)))
                break;
        }
        if (e) break;
        for (int bps : bps_list) {
            tuned_bps_ = bps;
            int nseg = 0;
            if ((e = cudaStreamSynchronize(stream_))) break;  // pinned staging reuse
            partition(sub, &nseg);
            if ((e = upload_partition(sub, nseg))) break;
            float ms = 1e30f;
            for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up; the fastest of the rest counts
                cudaEventRecord(e0, stream_);
                if ((e = enqueue_sampling(mask))) break;
                cudaEventRecord(e1, stream_);
                if ((e = cudaEventSynchronize(e1))) break;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, t);
            }
            if (e) break;
            if (ms < 0.97f * best) {  // a clear gain only: ties keep the earlier shape
                best = ms;
                best_bps = bps;
                best_cap = cap;
            }
        }
        if (e) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) return e;
    lanes_cap_ = best_cap;
    tuned_bps_ = best_bps;
    tuned_ = true;
    for (int s = 0; s < capacity_; ++s) {  // final lanes for every resident integral
        if (!slots_[s].used) continue;
        hdesc_[s].lanes = (uint32_t)choose_lanes(slots_[s].p);
        if ((e = cudaMemcpyAsync((BatchDesc*)desc_.ptr + s, &hdesc_[s], sizeof(BatchDesc), cudaMemcpyHostToDevice,
                                 stream_)))
            return e;
    }
    return cudaStreamSynchronize(stream_);
}

cudaError_t BatchEngine::step(int* ran, int iters)
{
    *ran = 0;
    cudaError_t e = flush_admissions();
    if (e) return e;
    std::vector<int> live;
    ClassMask mask;
    live_slots(&live, &mask);
    if (live.empty()) return cudaSuccess;
    if ((e = autotune(live, mask))) return e;
    if ((e = capture(mask))) return e;  // launch order by the class loads of the last partition
    int nseg = 0;
    partition(live, &nseg);
    if ((e = upload_partition(live, nseg))) return e;
    // iters iterations on one partition: an integral that converges or reaches
    // itmax on the way is skipped by the kernels from its next iteration on
    for (int k = 0; k < std::max(iters, 1); ++k) {
        if (exec_) e = cudaGraphLaunch(exec_, stream_);
        else e = enqueue_iteration(mask);
        if (e) return e;
    }
    *ran = (int)live.size();
    // the pinned partition staging is rewritten by the next step: wait here,
    // then read back which integrals have finished
    return refresh();
}

cudaError_t BatchEngine::refresh()
{
    cudaError_t e = cudaMemcpyAsync(h_states_, st_.ptr, sizeof(BatchState) * capacity_, cudaMemcpyDeviceToHost, stream_);
    if (e) return e;
    if ((e = cudaStreamSynchronize(stream_))) return e;
    for (int s = 0; s < capacity_; ++s) {
        Slot& S = slots_[s];
        if (!S.used || S.finished) continue;
        const BatchState& B = h_states_[s];
        S.it = (int)B.it;  // iterations run (the device's count: a step may run several)
        if (B.done || S.it >= hdesc_[s].itmax) {
            S.finished = true;
            mcubes_result& R = S.result;
            R.estimate = B.estimate;
            R.sigma = B.sigma;
            R.chi2_dof = B.chi2_dof;
            R.iterations = B.n;
            R.converged = B.converged;
            R.samples_per_iter = S.m * S.p;
            R.g = S.g;
            R.m = S.m;
            R.p = S.p;
            R.status = B.error ? B.error : (B.converged ? MCUBES_OK : MCUBES_ENOCONV);
        }
    }
    return cudaSuccess;
}

void BatchEngine::finished(std::vector<std::pair<long long, mcubes_result>>* out, bool free_slots)
{
    for (int s = 0; s < capacity_; ++s) {
        Slot& S = slots_[s];
        if (S.used && S.finished && !S.reported) {
            out->emplace_back(S.tag, S.result);
            S.reported = true;
            if (free_slots) {
                S.used = false;
                free_.push_back(s);
            }
        }
    }
}

cudaError_t BatchEngine::read_slot(int slot, double* I, double* V, int cap, int* n, double* grid, double* hist)
{
    const BatchDesc& D = hdesc_[slot];
    const int k = std::min(cap, slots_[slot].result.iterations);
    cudaError_t e = cudaSuccess;
    if (I && k > 0 && (e = cudaMemcpyAsync(I, D.hist_I, sizeof(double) * k, cudaMemcpyDeviceToHost, stream_)))
        return e;
    if (V && k > 0 && (e = cudaMemcpyAsync(V, D.hist_V, sizeof(double) * k, cudaMemcpyDeviceToHost, stream_)))
        return e;
    const size_t bins = (size_t)D.d * D.nb;
    if (grid && (e = cudaMemcpyAsync(grid, D.grid, sizeof(double) * bins, cudaMemcpyDeviceToHost, stream_))) return e;
    if (hist && (e = cudaMemcpyAsync(hist, D.hist, sizeof(double) * bins, cudaMemcpyDeviceToHost, stream_))) return e;
    if (n) *n = slots_[slot].result.iterations;
    return cudaStreamSynchronize(stream_);
}

int BatchEngine::resident() const
{
    int n = 0;
    for (const Slot& S : slots_) n += S.used && !S.finished ? 1 : 0;
    return n;
}

}  // namespace mc
