// server.cu -- the continuous-batching server (C ABI in include/mcubes.h):
// a FIFO of submitted requests in front of a slot engine (batch.cu).  Every
// step admits queued requests into free slots, advances every resident
// request by one iteration (each at its own iteration index) in one set of
// graph-replayed launches, and retires the finished ones.  Host code only.
#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "ctx_internal.h"

using namespace mc;

namespace {

// A queued request with its own copies of the host arrays.
struct Queued {
    mcubes_request r{};
    std::vector<double> params, lo, hi;
    long long tag = 0;

    Queued(const mcubes_request& src, long long t)
        : r(src), params(src.params, src.params + std::max(src.nparams, 0)), lo(src.lo, src.lo + src.d),
          hi(src.hi, src.hi + src.d), tag(t)
    {
        r.params = params.data();
        r.lo = lo.data();
        r.hi = hi.data();
    }
};

}  // namespace

struct mcubes_server {
    mcubes_ctx* ctx = nullptr;
    BatchEngine* engine = nullptr;
    std::deque<Queued> queue;
    std::vector<std::pair<long long, mcubes_result>> finished;  // not yet polled
    long long completed = 0;
    long long slot_bytes = 0;
    int iters_per_step = 1;
};

static mcubes_status cuda_status(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? MCUBES_ENOMEM : MCUBES_ECUDA;
}

extern "C" {

mcubes_status mcubes_server_create(mcubes_server** out, mcubes_ctx* ctx, long long budget_bytes, int itcap)
{
    if (!out || !ctx || budget_bytes < 0 || itcap < 1 || itcap > MCUBES_ITMAX_MAX) return MCUBES_EINVAL;
    if (ctx->opts.one_dim) return MCUBES_EINVAL;  // the batched kernels keep a histogram per axis
    *out = nullptr;
    const size_t per_slot = BatchEngine::slot_bytes(ctx->opts, itcap);
    long long capacity = budget_bytes > 0 ? budget_bytes / (long long)per_slot : 4096;
    if (capacity < 1) return MCUBES_EINVAL;
    capacity = std::min<long long>(capacity, 65535);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return MCUBES_ECUDA;
    mcubes_server* s = new (std::nothrow) mcubes_server();
    if (!s) return MCUBES_ENOMEM;
    s->ctx = ctx;
    s->slot_bytes = (long long)per_slot;
    s->engine = new (std::nothrow) BatchEngine(ctx->device, ctx->stream, ctx->num_sms, ctx->opts);
    if (!s->engine) {
        delete s;
        return MCUBES_ENOMEM;
    }
    const cudaError_t e = s->engine->reserve((int)capacity, itcap);
    if (e != cudaSuccess) {
        delete s->engine;
        delete s;
        return cuda_status(e);
    }
    *out = s;
    return MCUBES_OK;
}

mcubes_status mcubes_server_destroy(mcubes_server* s)
{
    if (!s) return MCUBES_OK;
    cudaSetDevice(s->ctx->device);
    delete s->engine;
    delete s;
    return MCUBES_OK;
}

mcubes_status mcubes_server_submit(mcubes_server* s, const mcubes_request* req, long long tag)
{
    if (!s || !req || (req->nparams > 0 && !req->params) || !req->lo || !req->hi) return MCUBES_EINVAL;
    const mcubes_status st = s->engine->validate(*req);
    if (st != MCUBES_OK) return st;
    s->queue.emplace_back(*req, tag);
    return MCUBES_OK;
}

// Admission (FIFO, as slots free up), one iteration, retirement.
static mcubes_status server_step(mcubes_server* s, int* ran)
{
    BatchEngine& E = *s->engine;
    while (!s->queue.empty() && E.free_slots() > 0) {
        const Queued& q = s->queue.front();
        const mcubes_status st = E.admit(q.r, q.tag);
        if (st != MCUBES_OK) return st;  // validated at submit: only ENOMEM is possible
        s->queue.pop_front();
    }
    int n = 0;
    const cudaError_t e = E.step(&n, s->iters_per_step);
    if (e != cudaSuccess) return cuda_status(e);
    const size_t before = s->finished.size();
    E.finished(&s->finished, true);
    s->completed += (long long)(s->finished.size() - before);
    if (ran) *ran = n;
    return MCUBES_OK;
}

mcubes_status mcubes_server_step(mcubes_server* s, int* ran)
{
    if (!s) return MCUBES_EINVAL;
    if (cudaSetDevice(s->ctx->device) != cudaSuccess) return MCUBES_ECUDA;
    return server_step(s, ran);
}

mcubes_status mcubes_server_set_step_iterations(mcubes_server* s, int iters)
{
    if (!s || iters < 1 || iters > MCUBES_STEP_ITERS_MAX) return MCUBES_EINVAL;
    s->iters_per_step = iters;
    return MCUBES_OK;
}

mcubes_status mcubes_server_poll(mcubes_server* s, long long* tags, mcubes_result* results, int cap, int* n)
{
    if (!s || cap < 0 || (cap > 0 && (!tags || !results))) return MCUBES_EINVAL;
    const int k = (int)std::min<size_t>((size_t)cap, s->finished.size());
    for (int i = 0; i < k; ++i) {
        tags[i] = s->finished[i].first;
        results[i] = s->finished[i].second;
    }
    s->finished.erase(s->finished.begin(), s->finished.begin() + k);
    if (n) *n = k;
    return MCUBES_OK;
}

mcubes_status mcubes_server_stats(mcubes_server* s, long long* queued, long long* resident, long long* completed,
                                  long long* capacity, long long* slot_bytes)
{
    if (!s) return MCUBES_EINVAL;
    if (queued) *queued = (long long)s->queue.size();
    if (resident) *resident = s->engine->resident();
    if (completed) *completed = s->completed;
    if (capacity) *capacity = s->engine->capacity();
    if (slot_bytes) *slot_bytes = s->slot_bytes;
    return MCUBES_OK;
}

mcubes_status mcubes_server_run_stream(mcubes_server* s, int n, const mcubes_request* reqs, const double* arrival_s,
                                       mcubes_result* results, double* latency_s, double* wall_s)
{
    if (!s || n < 0 || (n > 0 && (!reqs || !arrival_s || !results || !latency_s))) return MCUBES_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!(arrival_s[i] >= 0.0) || (i > 0 && arrival_s[i] < arrival_s[i - 1])) return MCUBES_EINVAL;
        if (!reqs[i].lo || !reqs[i].hi || (reqs[i].nparams > 0 && !reqs[i].params)) return MCUBES_EINVAL;
        const mcubes_status st = s->engine->validate(reqs[i]);
        if (st != MCUBES_OK) return st;
    }
    if (cudaSetDevice(s->ctx->device) != cudaSuccess) return MCUBES_ECUDA;
    using clock = std::chrono::steady_clock;
    const auto t0 = clock::now();
    auto now = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
    // tags of this stream are offset so that earlier polled tags cannot collide
    const long long base = 1ll << 62;
    int next = 0, done = 0;
    std::vector<std::pair<long long, mcubes_result>> fin;
    while (done < n) {
        const double t = now();
        while (next < n && arrival_s[next] <= t) {
            s->queue.emplace_back(reqs[next], base + next);
            ++next;
        }
        if (s->queue.empty() && s->engine->resident() == 0) {
            // idle until the next arrival
            const double wait = arrival_s[next] - now();
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.001)));
            continue;
        }
        int ran = 0;
        const mcubes_status st = server_step(s, &ran);
        if (st != MCUBES_OK) return st;
        const double t_end = now();
        for (auto it = s->finished.begin(); it != s->finished.end();) {
            if (it->first >= base) {
                const long long i = it->first - base;
                results[i] = it->second;
                latency_s[i] = t_end - arrival_s[i];
                ++done;
                it = s->finished.erase(it);
            } else {
                ++it;
            }
        }
    }
    if (wall_s) *wall_s = now();
    return MCUBES_OK;
}

}  // extern "C"
