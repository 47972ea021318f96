// server.cu -- the continuous-batching server (C ABI in include/mcubes.h):
// a FIFO of submitted requests in front of a slot engine (batch.cu).  Every
// step admits queued requests into free slots, advances every resident
// request by one iteration (each at its own iteration index) in one set of
// graph-replayed launches, and retires the finished ones.  Host code only.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>
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
    // copies point r at their own arrays
    Queued(const Queued& o) : Queued(o.r, o.tag) {}
    Queued& operator=(const Queued& o)
    {
        if (this != &o) {
            r = o.r;
            params = o.params;
            lo = o.lo;
            hi = o.hi;
            tag = o.tag;
            r.params = params.data();
            r.lo = lo.data();
            r.hi = hi.data();
        }
        return *this;
    }
};

}  // namespace

struct mcubes_server {
    mcubes_ctx* ctx = nullptr;
    BatchEngine* engine = nullptr;
    // Queued and resident requests carry an internal id (their engine tag);
    // `open` maps it to the caller's tag and keeps the request for a retry.
    std::deque<Queued> queue;
    struct Open {
        long long tag;
        Queued req;
    };
    std::unordered_map<long long, Open> open;
    long long next_id = 0;
    double esc_factor = 1.0;     // calls x factor on a retry (1: no retries)
    double esc_max_factor = 0.0; // > 0: the factor is sized from the attempt's sigma, up to this
    long long esc_ncall_max = 0;
    std::vector<std::pair<long long, mcubes_result>> finished;  // not yet polled
    long long completed = 0;
    long long slot_bytes = 0;
    int iters_per_step = 1;
    long long stream_gen = 0;  // calls of mcubes_server_run_stream so far
};

// Tags from 2^62 up are the server's own: mcubes_server_run_stream tags
// request i of its k-th call 2^62 + (k mod 2^30) 2^31 + i.
constexpr long long kStreamTagBase = 1ll << 62;

// Calls per iteration of a retry.  Fixed rule (max_factor = 0): ncall x
// factor while that stays <= ncall_max (else none: returns ncall).  Sized
// rule: the attempt's sigma against the tolerance tau = max(abs_tol,
// rel_tol |estimate|) predicts the calls that reach it, since sigma falls as
// (calls x iterations)^-1/2 -- ncall x 2 (sigma / tau)^2, the factor clamped
// to [factor, max_factor] (max_factor when tau is not positive), the calls
// to ncall_max.
static long long retry_ncall(const mcubes_request& r, const mcubes_result& res, double factor, double max_factor,
                             long long ncall_max)
{
    if (max_factor <= 0.0) {
        const double more = (double)r.ncall * factor;
        return more <= (double)ncall_max ? (long long)more : r.ncall;
    }
    const double tau = std::max(r.abs_tol, r.rel_tol * std::fabs(res.estimate));
    double k = max_factor;
    if (tau > 0.0 && std::isfinite(res.sigma)) {
        const double q = res.sigma / tau;
        k = std::min(max_factor, std::max(factor, 2.0 * q * q));
    }
    const double more = std::min((double)r.ncall * k, (double)ncall_max);
    return (long long)more;
}

// Queues a caller's request under a new internal id.
static void server_enqueue(mcubes_server* s, const mcubes_request& r, long long tag)
{
    const long long id = s->next_id++;
    s->queue.emplace_back(r, id);
    s->open.emplace(id, mcubes_server::Open{tag, s->queue.back()});
}

// A finished request: reported under its caller's tag, or, when it ran out
// of iterations without converging and the escalation allows, queued again
// (at the front) with factor times the calls per iteration.
static void server_retire(mcubes_server* s, long long id, const mcubes_result& res)
{
    auto it = s->open.find(id);
    if (it == s->open.end()) return;
    mcubes_request& r = it->second.req.r;
    if (res.status == MCUBES_ENOCONV && s->esc_factor > 1.0 && r.ncall < s->esc_ncall_max) {
        const long long more = retry_ncall(r, res, s->esc_factor, s->esc_max_factor, s->esc_ncall_max);
        mcubes_request next = r;
        next.ncall = more;
        if (more > r.ncall && s->engine->validate(next) == MCUBES_OK) {
            r.ncall = next.ncall;
            s->queue.emplace_front(next, id);
            return;
        }
    }
    s->finished.emplace_back(it->second.tag, res);
    ++s->completed;
    s->open.erase(it);
}

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
    if (tag >= kStreamTagBase) return MCUBES_EINVAL;  // reserved for mcubes_server_run_stream
    const mcubes_status st = s->engine->validate(*req);
    if (st != MCUBES_OK) return st;
    server_enqueue(s, *req, tag);
    return MCUBES_OK;
}

mcubes_status mcubes_server_set_escalation(mcubes_server* s, double factor, long long ncall_max)
{
    if (!s || !(factor >= 1.0) || !(factor <= 1024.0) || ncall_max < 0) return MCUBES_EINVAL;
    s->esc_factor = factor;
    s->esc_max_factor = 0.0;
    s->esc_ncall_max = ncall_max;
    return MCUBES_OK;
}

mcubes_status mcubes_server_set_retry_sized(mcubes_server* s, double min_factor, double max_factor,
                                            long long ncall_max)
{
    if (!s || !(min_factor > 1.0) || !(max_factor >= min_factor) || !(max_factor <= 1024.0) || ncall_max < 0)
        return MCUBES_EINVAL;
    s->esc_factor = min_factor;
    s->esc_max_factor = max_factor;
    s->esc_ncall_max = ncall_max;
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
    std::vector<std::pair<long long, mcubes_result>> fin;
    E.finished(&fin, true);
    for (const auto& f : fin) server_retire(s, f.first, f.second);
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
    // Requests left by an earlier call that returned early (ENOMEM, ECUDA):
    // the queued ones are dropped, finished ones discarded; resident ones
    // finish later and are discarded below (their generation differs).
    s->queue.erase(std::remove_if(s->queue.begin(), s->queue.end(),
                                  [s](const Queued& q) {
                                      auto it = s->open.find(q.tag);
                                      if (it == s->open.end() || it->second.tag < kStreamTagBase) return false;
                                      s->open.erase(it);
                                      return true;
                                  }),
                   s->queue.end());
    s->finished.erase(std::remove_if(s->finished.begin(), s->finished.end(),
                                     [](const std::pair<long long, mcubes_result>& f) {
                                         return f.first >= kStreamTagBase;
                                     }),
                      s->finished.end());
    s->stream_gen = (s->stream_gen + 1) & ((1ll << 30) - 1);
    const long long base = kStreamTagBase + (s->stream_gen << 31);
    const auto t0 = clock::now();
    auto now = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
    int next = 0, done = 0;
    while (done < n) {
        const double t = now();
        while (next < n && arrival_s[next] <= t) {
            server_enqueue(s, reqs[next], base + next);
            ++next;
        }
        if (s->queue.empty() && s->engine->resident() == 0) {
            if (next >= n) return MCUBES_ESTATE;  // a request of this call was lost: cannot happen
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
            if (it->first >= kStreamTagBase) {
                const long long i = it->first - base;  // another generation: outside [0, n)
                if (i >= 0 && i < n) {
                    results[i] = it->second;
                    latency_s[i] = t_end - arrival_s[i];
                    ++done;
                }
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
