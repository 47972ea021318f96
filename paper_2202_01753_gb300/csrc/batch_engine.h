// batch_engine.h -- host side of the batched path: device buffers, the slot
// table of resident integrals, the per-iteration work partition, the CUDA
// graph of one iteration and the launch-shape autotuner (batch.cu).
#pragma once

#include <bitset>
#include <utility>
#include <vector>

#include "mc_internal.h"

namespace mc {

using ClassMask = std::bitset<kNumClasses>;  // kernel classes present (family x dimension)

// A device allocation that only grows.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t n)
    {
        if (n <= bytes) return cudaSuccess;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&ptr, n);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    void release()
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

class BatchEngine {
public:
    BatchEngine(int device, cudaStream_t stream, int num_sms, const mcubes_opts& opts);
    ~BatchEngine();
    BatchEngine(const BatchEngine&) = delete;
    BatchEngine& operator=(const BatchEngine&) = delete;

    // Room for `capacity` resident integrals of up to itcap iterations each
    // (every slot can hold MCUBES_DMAX axes of opts.nbins bins).
    cudaError_t reserve(int capacity, int itcap);
    int capacity() const { return capacity_; }
    int itcap() const { return itcap_; }
    int free_slots() const { return (int)free_.size(); }
    int resident() const;

    // Checks one request against this engine (options, itcap) without
    // admitting it.
    mcubes_status validate(const mcubes_request& r) const;

    // Validates one request and places it in a free slot (its grid and state
    // are initialised on the device at the next step).  tag identifies it in
    // finished().  EINVAL: invalid request; ENOMEM: no free slot.
    mcubes_status admit(const mcubes_request& r, long long tag, int* slot = nullptr);

    // Device bytes one slot occupies (its grid, histogram, history, state
    // and its share of the per-iteration partials), for itcap iterations.
    static size_t slot_bytes(const mcubes_opts& opts, int itcap);

    // iters iterations (graph replays) of every resident, unfinished integral
    // on one partition, then a read-back of which ones have finished (one
    // that finishes on the way is skipped by the kernels from then on).
    // *ran = integrals that were live at the start of the step.
    cudaError_t step(int* ran, int iters = 1);

    // Results of integrals that finished since the last call (tag, result);
    // with free_slots their slots become free for new admissions.
    void finished(std::vector<std::pair<long long, mcubes_result>>* out, bool free_slots);

    // Copies a slot's iteration estimates and variances (up to cap each; *n
    // receives the number recorded), its grid ([d][nb] edge high parts) and
    // the histogram of its last adjusting iteration ([d][nb]) to host arrays
    // (any may be null).  Valid for a finished slot until it is reused.
    cudaError_t read_slot(int slot, double* I, double* V, int cap, int* n, double* grid, double* hist);

    int tuned_blocks_per_sm() const { return tuned_bps_; }  // a cap on each class's occupancy
    int lanes_cap() const { return lanes_cap_; }

private:
    struct Slot {
        bool used = false, finished = false, reported = false;
        long long tag = 0;
        int it = 0;           // iterations run (read back from the device after each step)
        double work = 0.0;    // samples per iteration
        long long g = 0, m = 0, p = 0;
        mcubes_result result{};
    };

    void release();
    size_t smem_bytes(int cls) const;
    int class_blocks(int cls) const;
    int choose_lanes(long long p) const;
    cudaError_t flush_admissions();
    // live slots grouped by class (class order, slot order within a class)
    void live_slots(std::vector<int>* live, ClassMask* class_mask) const;
    void partition(const std::vector<int>& live, int* nseg);
    cudaError_t upload_partition(const std::vector<int>& live, int nseg);
    BatchArgs sample_args(int cls) const;
    BatchRefineArgs refine_args() const;
    cudaError_t enqueue_sampling(const ClassMask& class_mask);
    cudaError_t enqueue_iteration(const ClassMask& class_mask);
    cudaError_t capture(ClassMask class_mask);
    cudaError_t autotune(const std::vector<int>& live, const ClassMask& class_mask);
    cudaError_t refresh();

    int device_;
    cudaStream_t stream_;
    int num_sms_;
    mcubes_opts opts_;
    bool mixed_;
    int capacity_ = 0, itcap_ = 0;
    int occ_[kNumClasses] = {0};   // resident blocks per SM of each class's kernel
    int bmax_ = 0;                 // most blocks any class launches
    size_t hist_cap_ = 0;          // entries of the partial-histogram buffer
    size_t part_hist_ = 0;         // entries the last partition uses
    double class_load_[kNumClasses] = {0};  // a class's work per block in the last partition (launch order)
    bool tuned_ = false;
    int tuned_bps_ = 1, lanes_cap_ = 64;

    std::vector<Slot> slots_;
    std::vector<BatchDesc> hdesc_;
    std::vector<int> free_, pending_;

    DevBuf desc_, st_, grids_, cells_, hists_, histories_, segs_, blk_seg_, live_, live_seg_, nlive_, seg_part_, seg_hist_,
        admit_slots_;
    BatchSeg* h_segs_ = nullptr;     // pinned staging
    uint32_t* h_small_ = nullptr;    // pinned staging: block offsets, live lists, counts
    BatchState* h_states_ = nullptr; // pinned read-back
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    ClassMask graph_mask_;         // classes the captured graph launches
    int graph_bps_ = 0;
    // one branch stream per class kernel of an iteration: forked from and
    // joined back into stream_, so that the class kernels overlap
    std::vector<cudaStream_t> branch_;
    std::vector<cudaEvent_t> join_;
    cudaEvent_t fork_ = nullptr;
};

}  // namespace mc
