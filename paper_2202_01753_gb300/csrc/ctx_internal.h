// ctx_internal.h -- the definition of mcubes_ctx (opaque in the public
// header), shared by the translation units that implement the C ABI.
#pragma once

#include <vector>

#include "batch_engine.h"

namespace mc {
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};
}  // namespace mc

struct mcubes_ctx;

namespace mc {
// Rebuilds the context's map cells from its grid (after set-up or after the
// grid is replaced), on the context's stream.
cudaError_t ctx_refresh_cells(mcubes_ctx* c);
}  // namespace mc

struct mcubes_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mcubes_opts opts{};
    int num_sms = 0;
    char cuda_err[256] = {0};

    // current problem (as given to mcubes_setup, kept for checkpoints)
    bool ready = false;
    std::vector<double> prob_params, prob_lo, prob_hi;
    double rel_tol = 0.0, abs_tol = 0.0;
    int fid = 0, d = 0, nb = 0, itmax = 0, ita = 0;
    long long ncall = 0, g = 0, m = 0, p = 0;
    bool mixed = false;
    int hist_d = 0;   // axes with a histogram: d, or 1 in m-Cubes1D
    int split = 1;    // blocks per cube (cube-split mode when > 1)
    int lanes = 1;
    int grid_adj = 0, grid_noadj = 0;
    int grid_res_adj = 0, grid_res_noadj = 0;  // resident blocks x SMs (cube-range passes)
    bool shard_open = false;                    // a shard pass is enqueued and not finished
    bool shard_adjust = false;
    size_t smem_adj = 0, smem_noadj = 0;
    int it_enqueued = 0;
    mc::VsArgs vs{};
    mc::RefineArgs rf{};

    mc::DevBuf grid, hist, part, hist_acc, state, range_out;
    mc::DevBuf cells;     // [d][nb] map cells of the current grid (rebuilt by the refinement)
    mc::CellBox cellbox{};

    // interpolation tables of TABLE integrands (mcubes_tables_set)
    mc::DevBuf tab_v, tab_vf, tab_desc;
    std::vector<mc::TableDesc> tabs_host;  // descriptors as uploaded (device pointers)

    mc::BatchEngine* engine = nullptr;  // batched path, created on first use
    std::vector<int> batch_slots;       // engine slot of each request of the last mcubes_integrate_batch
    std::vector<int> batch_dims;        // and its dimension

    bool timing = false;
    std::vector<mc::EventPair> ev_sample, ev_refine;
    size_t n_sample = 0, n_refine = 0;
    std::vector<mc::EventPair> pool;
};
