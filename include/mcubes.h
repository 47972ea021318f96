/*
 * mcubes.h -- C ABI of the GB300 m-Cubes VEGAS integrator.
 *
 * The library implements the per-iteration hot path of m-Cubes (Sakiotis et
 * al., arXiv 2202.01753): the d-cube is split into m = g^d equal sub-cubes
 * (Alg. 2), every sub-cube receives p samples drawn from a counter-based
 * Philox4x32-10 stream keyed by (seed, iteration, cube, sample), the samples
 * are mapped through the adaptive per-axis bin grid (Alg. 1), the integrand
 * is evaluated, per-cube means and variances are reduced into the iteration
 * estimate (Alg. 3), per-axis per-bin sums of f^2 drive the grid refinement
 * (Alg. 2, Adjust-Bin-Bounds), and iterations are combined with inverse-
 * variance weights and chi^2 (Alg. 2, Weighted-Estimates).  Every step runs
 * in CUDA kernels on one GPU; the host only validates arguments and
 * enqueues work.
 *
 * Conventions for every entry point:
 *   - All pointers named host_* or documented as host arrays are host memory
 *     owned by the caller, read (or written) before the call returns.
 *   - A context owns all device memory it uses and one CUDA stream (its own,
 *     or one the caller passes in and keeps alive).  Contexts are not
 *     thread-safe: one host thread at a time per context.
 *   - Every call returns an mcubes_status; no C++ exception crosses the ABI.
 *   - Arrays of bins are laid out [d][nb], axis-major, in unit coordinates
 *     (edges in [0, 1], the right edge of bin k at index k, the left edge of
 *     bin 0 being 0 implicitly).
 */
#ifndef MCUBES_H
#define MCUBES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcubes_ctx mcubes_ctx;

typedef enum {
    MCUBES_OK = 0,
    MCUBES_EINVAL = 1,     /* invalid argument (d, ncall, bounds, params, ids, sizes) */
    MCUBES_ENOMEM = 2,     /* device or host allocation failed */
    MCUBES_ECUDA = 3,      /* a CUDA runtime call failed (see mcubes_last_cuda_error) */
    MCUBES_ENONFINITE = 4, /* the integrand produced a non-finite value */
    MCUBES_ENOCONV = 5,    /* itmax reached before the tolerance: results are still filled */
    MCUBES_ETIMEOUT = 6,   /* a bounded device wait gave up */
    MCUBES_ESTATE = 7      /* call out of order (e.g. iterate before setup) */
} mcubes_status;

typedef enum {
    MCUBES_FP64 = 0,  /* map, integrand and all sums in double precision */
    MCUBES_MIXED = 1  /* map and integrand in single precision; per-cube sums compensated,
                         everything from the thread level up in double precision */
} mcubes_precision;

/* Integrand families (Sec. 5 eqs. 1-6 and Table 1 of the paper in
 * parameterised form, and a stand-in for the six-dimensional integrand of
 * Sec. 6.1).  params layout, d = dimension:
 *   CONST    [v]                      f = v
 *   GAUSS    [A, mu_1..d, sig_1..d]   f = A prod_i exp(-(x_i-mu_i)^2 / (2 sig_i^2))
 *   CORNER   [a_1..d]                 f = (1 + sum_i a_i x_i)^(-(d+1))
 *   OSC      [u, a_1..d]              f = cos(2 pi u + sum_i a_i x_i)
 *   PRODPEAK [c_1..d, w_1..d]         f = prod_i 1 / (c_i^-2 + (x_i - w_i)^2)
 *   C0       [c_1..d, w_1..d]         f = exp(-sum_i c_i |x_i - w_i|)
 *   DISCONT  [c_1..d, w_1..d]         f = exp(sum_i c_i x_i) if x_i < w_i for all i, else 0
 *   COSMO6   [a_1..6, mu, s, r, t]    d = 6 only:
 *            f = prod_i x_i^-a_i * LN(x_3) LN(x_4) * exp(-(x_1 + x_2 - r)^2 / (2 t^2)),
 *            LN(z) = exp(-(ln z - mu)^2 / (2 s^2)) / (z s sqrt(2 pi))
 *   TABLE    [c, nf, (tab, a, b) x nf]  1 <= nf <= 10 factors:
 *            f = c prod_q T_tab_q(x_a_q) (1-D table, b_q = -1) or T_tab_q(x_a_q, x_b_q) (2-D),
 *            T the linear / bilinear interpolant of a table set with mcubes_tables_set
 *            (Sec. 6.1: integrands that read tabulated data); axes a, b are 0-based;
 *            single-integral entry points only (the batched ones reject it)
 * (indices 1-based as written unless stated; x_i > 0 is required for COSMO6). */
enum {
    MCUBES_F_CONST = 0,
    MCUBES_F_GAUSS = 1,
    MCUBES_F_CORNER = 2,
    MCUBES_F_OSC = 3,
    MCUBES_F_PRODPEAK = 4,
    MCUBES_F_C0 = 5,
    MCUBES_F_DISCONT = 6,
    MCUBES_F_COSMO6 = 7,
    MCUBES_F_TABLE = 8,
    MCUBES_F_COUNT = 9
};

#define MCUBES_TABLES_MAX 16  /* interpolation tables per context */

/* One interpolation table of the TABLE family: values at uniformly spaced
 * knots, n[0] knots over [lo[0], hi[0]] (and, for ndim 2, n[1] over
 * [lo[1], hi[1]]; values row-major, values[i0 * n[1] + i1]).  The value at a
 * point is the linear (bilinear) interpolant of the knot values, the point
 * first clamped into the knot range. */
typedef struct {
    int ndim;              /* 1 or 2 */
    int n[2];              /* knots per axis, >= 2 (n[1] unused for ndim 1) */
    double lo[2], hi[2];   /* knot range per axis, lo < hi, finite */
    const double* values;  /* host array of n[0] (x n[1]) finite values, caller-owned */
} mcubes_table;

#define MCUBES_DMAX 12        /* largest dimension */
#define MCUBES_NBMAX 1024     /* largest number of bins per axis */
#define MCUBES_PARAMS_MAX 32  /* largest params blob */
#define MCUBES_ITMAX_MAX 4096 /* largest itmax */

typedef struct {
    int nbins;            /* bins per axis, 2..MCUBES_NBMAX (default 500) */
    int ita;              /* adjusting iterations (Alg. 2); < 0 means all (default -1) */
    long long g_override; /* sub-cubes per axis; 0 = largest g with g^d <= ncall/2 (default 0) */
    double alpha;         /* grid compression exponent of Adjust-Bin-Bounds (default 1.5) */
    uint64_t seed;        /* Philox key (default 0) */
    int precision;        /* mcubes_precision (default MCUBES_FP64) */
    int lanes_per_cube;   /* 0 = automatic; else a power of two 1..32: threads sharing one cube */
    int blocks_per_sm;    /* 0 = automatic (occupancy); else resident sampling blocks per SM */
    int one_dim;          /* 1 = the m-Cubes1D variant (Sec. 3): every axis shares one set of bin
                             boundaries, only axis 0 keeps a histogram and is rebinned, its new edges
                             going to all axes.  Meant for fully symmetric integrands; the box must be
                             a cube (same lo and hi on every axis, else EINVAL), grid_set needs equal
                             rows, hist_get returns zero rows 1..d-1.  The batched entry points and the
                             server reject it (EINVAL).  0 = m-Cubes (default). */
} mcubes_opts;

typedef struct {
    double estimate;            /* weighted estimate over the iterations run */
    double sigma;               /* its standard deviation */
    double chi2_dof;            /* chi^2 per degree of freedom of the iteration estimates */
    int iterations;             /* iterations run */
    int converged;              /* 1 if sigma <= max(abs_tol, rel_tol |estimate|) with >= 2 iterations */
    long long samples_per_iter; /* m * p */
    long long g, m, p;          /* sub-cubes per axis, sub-cubes, samples per sub-cube */
    int status;                 /* mcubes_status of the run */
} mcubes_result;

/* One integral of a batch (mcubes_integrate_batch). */
typedef struct {
    int integrand_id;
    const double* params; /* host, nparams values */
    int nparams;
    int d;
    const double* lo;     /* host, d values */
    const double* hi;     /* host, d values */
    long long ncall;
    int itmax;
    double rel_tol;
    double abs_tol;
    uint64_t seed;        /* this integral's own Philox key */
} mcubes_request;

/* Fills *opts with the defaults listed in mcubes_opts. */
void mcubes_default_opts(mcubes_opts* opts);

/* Creates a context on CUDA device `device` with a stream of its own.
 * opts may be NULL (defaults).  *out receives the context.
 * Errors: EINVAL (bad opts or device), ECUDA, ENOMEM. */
mcubes_status mcubes_create(mcubes_ctx** out, int device, const mcubes_opts* opts);

/* As mcubes_create, but all work is enqueued on `cuda_stream` (a
 * cudaStream_t, e.g. the current PyTorch stream; NULL means the legacy
 * default stream), which the caller keeps alive until mcubes_destroy. */
mcubes_status mcubes_create_on_stream(mcubes_ctx** out, int device, const mcubes_opts* opts,
                                      void* cuda_stream);

/* Replaces the options of an existing context (takes effect at the next setup). */
mcubes_status mcubes_set_opts(mcubes_ctx* ctx, const mcubes_opts* opts);

/* Copies the context's current options to *out.  Errors: EINVAL (null). */
mcubes_status mcubes_get_opts(mcubes_ctx* ctx, mcubes_opts* out);

/* Releases the context and all its device memory. NULL is accepted. */
mcubes_status mcubes_destroy(mcubes_ctx* ctx);

/* Static description of a status code. */
const char* mcubes_strerror(mcubes_status status);

/* Text of the last CUDA error seen by this context (static storage, valid
 * until the next call on the context). */
const char* mcubes_last_cuda_error(mcubes_ctx* ctx);

/* The whole m-Cubes driver (Alg. 2): up to itmax iterations, the first
 * opts.ita of them adjusting the grid, stopping once sigma <= max(abs_tol,
 * rel_tol |estimate|) after at least two iterations.  params, lo and hi are
 * host arrays (nparams and d values).  *out (host) is filled on OK and on
 * ENOCONV.  Blocks until the result is on the host.
 * Errors: EINVAL (d outside 1..MCUBES_DMAX, ncall < 2, lo >= hi, non-finite
 * params or bounds, unknown id, wrong nparams, itmax outside
 * 1..MCUBES_ITMAX_MAX, or a grid too large for one block's shared memory:
 * d * nbins * 24 bytes in FP64, d * nbins * 20 bytes in MIXED, at most the
 * device's opt-in limit less 1 KB, 227 KB on GB300), ENOMEM, ECUDA,
 * ENONFINITE, ENOCONV. */
mcubes_status mcubes_integrate(mcubes_ctx* ctx, int integrand_id, const double* params, int nparams,
                               int d, const double* lo, const double* hi, long long ncall,
                               int itmax, double rel_tol, double abs_tol, mcubes_result* out);

/* n independent integrals, each with its own seed, iterated together: every
 * iteration of all live integrals is one persistent sampling launch per
 * kernel class (integrand family x dimension; the classes run concurrently)
 * and one refinement launch, captured once as a CUDA graph and replayed.  Uses the
 * context's precision, nbins, ita (as a count) and alpha.  outs (host, n
 * entries) receives one result per request, each with its own status.
 * Returns OK if the batch ran (individual statuses are in outs), EINVAL if
 * any request is invalid (nothing runs), ENOMEM, ECUDA. */
mcubes_status mcubes_integrate_batch(mcubes_ctx* ctx, int n, const mcubes_request* reqs,
                                     mcubes_result* outs);

/* Integral i of the last mcubes_integrate_batch call on this context: its
 * per-iteration estimates and variances (host arrays of cap entries; *n
 * receives the number of iterations run), its final grid ([d][nb] right
 * edges, host, may be NULL) and the per-bin sums of f^2 of its last
 * adjusting iteration ([d][nb], host, may be NULL).  Valid until the next
 * batched call on the context.  Errors: EINVAL (no such integral). */
mcubes_status mcubes_batch_trace_get(mcubes_ctx* ctx, int i, double* I_it, double* var_it, int cap, int* n,
                                     double* grid, double* C);

/* ---- continuous-batching server ------------------------------------------
 * A server keeps up to `capacity` integration requests resident on the GPU,
 * each with its own grid, running sums and iteration index, and advances all
 * of them by one iteration per step: one persistent sampling launch per
 * kernel class (integrand family x dimension, run concurrently) and one
 * refinement launch, replayed as a CUDA graph.
 * Requests submitted while others run wait in a FIFO queue and are admitted
 * as slots free up; finished requests (converged, itmax reached, or failed)
 * leave at once.  A request's samples do not depend on what else is
 * resident, so its result equals a solo run up to the grouping of partial
 * sums.  Uses the context's stream, precision, nbins, ita (as a count per
 * request) and alpha.  One host thread at a time per server. */
typedef struct mcubes_server mcubes_server;

/* Capacity is chosen from a device-memory budget: each slot holds a
 * double-double grid and a histogram for MCUBES_DMAX axes and a history of
 * itcap iterations, plus its share of the per-iteration partials
 * (mcubes_server_stats reports the bytes per slot).  budget_bytes = 0 means
 * 4096 slots.  Errors: EINVAL, ENOMEM, ECUDA. */
mcubes_status mcubes_server_create(mcubes_server** out, mcubes_ctx* ctx, long long budget_bytes, int itcap);
mcubes_status mcubes_server_destroy(mcubes_server* srv);

/* Queues one request (host arrays, copied); tag identifies its result.
 * Tags from 2^62 up are reserved for mcubes_server_run_stream.  EINVAL if
 * the request is invalid or the tag reserved (nothing is queued). */
mcubes_status mcubes_server_submit(mcubes_server* srv, const mcubes_request* req, long long tag);

/* Admits queued requests into free slots, runs one iteration (or the number
 * set by mcubes_server_set_step_iterations) of every resident request and
 * retires the finished ones; blocks until the iterations are done.  *ran
 * receives the number of requests iterated. */
mcubes_status mcubes_server_step(mcubes_server* srv, int* ran);

/* Iterations each step runs before it reads back which requests finished
 * (1..MCUBES_STEP_ITERS_MAX, default 1).  More iterations per step spread
 * the step's fixed host work (admission, partition upload, read-back) over
 * more iterations; a request that converges or reaches its itmax inside a
 * step is skipped by the kernels for the rest of it (its result is the same),
 * and new requests are admitted only between steps.  EINVAL outside the
 * range. */
#define MCUBES_STEP_ITERS_MAX 64
mcubes_status mcubes_server_set_step_iterations(mcubes_server* srv, int iters);

/* Retries for requests that reach their itmax without converging (the
 * accuracy protocol of Sec. 5.1 raises the number of samples for tighter
 * tolerances): such a request is queued again, ahead of new arrivals, with
 * factor times its calls per iteration and a fresh start, while that stays
 * at or below ncall_max; its result is that of its last run, and a caller
 * sees only that one.  factor = 1 (the default) disables retries.  Errors:
 * EINVAL (factor outside [1, 1024], ncall_max < 0). */
mcubes_status mcubes_server_set_escalation(mcubes_server* srv, double factor, long long ncall_max);

/* The same retries with the calls sized from the attempt that failed: its
 * sigma against the tolerance tau = max(abs_tol, rel_tol |estimate|)
 * predicts the calls that reach tau, sigma falling as (calls x
 * iterations)^-1/2, so the retry runs ncall x 2 (sigma/tau)^2 calls per
 * iteration, the factor clamped to [min_factor, max_factor] (max_factor when
 * tau is 0) and the calls to ncall_max; a request already at ncall_max is
 * reported.  Replaces the rule of mcubes_server_set_escalation (and the
 * other way round).  Errors: EINVAL (min_factor <= 1, max_factor < min_factor
 * or > 1024, ncall_max < 0). */
mcubes_status mcubes_server_set_retry_sized(mcubes_server* srv, double min_factor, double max_factor,
                                            long long ncall_max);

/* Copies up to cap finished results (and their tags) not yet returned;
 * *n receives how many were copied. */
mcubes_status mcubes_server_poll(mcubes_server* srv, long long* tags, mcubes_result* results, int cap, int* n);

/* queued: waiting for a slot; resident: on the GPU; completed: finished
 * since creation; capacity: slots; slot_bytes: device bytes per slot. */
mcubes_status mcubes_server_stats(mcubes_server* srv, long long* queued, long long* resident,
                                  long long* completed, long long* capacity, long long* slot_bytes);

/* Serves a timed stream in real time: request i (host array reqs) arrives
 * arrival_s[i] seconds after the call starts (non-decreasing); the server
 * queues arrivals, admits, steps and retires until every request is done.
 * results[i] receives request i's result and latency_s[i] the time from its
 * arrival to the end of the step that finished it; *wall_s the duration of
 * the whole call.  The call tags its requests from 2^62 up, a new range per
 * call; requests another call of it left behind (it returned an error) are
 * dropped or, once finished, discarded.  Requests queued by
 * mcubes_server_submit are served alongside and stay pollable.  Errors:
 * EINVAL, ENOMEM, ECUDA. */
mcubes_status mcubes_server_run_stream(mcubes_server* srv, int n, const mcubes_request* reqs,
                                       const double* arrival_s, mcubes_result* results, double* latency_s,
                                       double* wall_s);

/* ---- step-level interface (the pieces of mcubes_integrate) -------------- */

/* Validates one integral, computes its geometry, sizes the device buffers,
 * sets the uniform grid and clears the iteration history.  Host arrays.
 * Errors: as mcubes_integrate. */
mcubes_status mcubes_setup(mcubes_ctx* ctx, int integrand_id, const double* params, int nparams,
                           int d, const double* lo, const double* hi, long long ncall, int itmax,
                           double rel_tol, double abs_tol);

/* Enqueues n_iter further iterations on the context's stream and returns
 * without waiting.  Iterations after convergence (or a device error) are
 * skipped on the device.  Errors: ESTATE (no setup or beyond itmax). */
mcubes_status mcubes_iterate(mcubes_ctx* ctx, int n_iter);

/* Waits for the stream and copies the current result to *out (host). */
mcubes_status mcubes_result_get(mcubes_ctx* ctx, mcubes_result* out);

/* Waits, then copies the per-iteration estimates and variances (host arrays
 * of `cap` entries); *n receives the number of iterations recorded. */
mcubes_status mcubes_trace_get(mcubes_ctx* ctx, double* I_it, double* var_it, int cap, int* n);

/* Waits, then copies the current bin grid ([d][nb] right edges, host).  The
 * library keeps every edge as a double-double number (so that narrow bins
 * keep their width to full precision); this returns the rounded edges. */
mcubes_status mcubes_grid_get(mcubes_ctx* ctx, double* B, long long count);

/* Replaces the current bin grid ([d][nb], host): every axis must have
 * strictly increasing edges in (0, 1] ending at 1; the edges are taken as
 * exact (zero low parts). Errors: EINVAL, ESTATE. */
mcubes_status mcubes_grid_set(mcubes_ctx* ctx, const double* B, long long count);

/* Waits, then copies the per-bin sums of f^2 ([d][nb], host) of the last
 * adjusting iteration. */
mcubes_status mcubes_hist_get(mcubes_ctx* ctx, double* C, long long count);

/* Uploads interpolation tables for TABLE integrands into the context's
 * device memory (global memory, read through the L1/L2 caches), replacing
 * any earlier set; the host arrays are copied before return.  The tables
 * are kept in double precision and, for the mixed-precision path, as a
 * single-precision copy.  The call waits for the context's stream and ends
 * the current problem (ESTATE until the next mcubes_setup): set tables
 * first, then mcubes_setup / mcubes_integrate.  Checkpoints do not hold the
 * tables: set the same ones on a context before importing a TABLE problem.
 * ntables = 0 releases them.  Errors: EINVAL (ntables outside
 * 0..MCUBES_TABLES_MAX, a bad ndim, knot count or range, a non-finite
 * value, more than 2^31 values in one table), ENOMEM, ECUDA. */
mcubes_status mcubes_tables_set(mcubes_ctx* ctx, int ntables, const mcubes_table* tables);

/* ---- checkpoint / resume ------------------------------------------------
 * The paper has no counterpart: these serialise the state of the current
 * problem so that a long run can stop and continue in another process.
 * The checkpoint holds the problem as given to mcubes_setup (integrand id,
 * params, box, ncall, itmax, tolerances), the context's options, the bin
 * grid with the low parts of its double-double edges, the number of
 * iterations enqueued, and the device iteration state (index, flags,
 * weighted result and per-iteration history).  Layout: a fixed header
 * (magic "MCUBESCK", format version, byte sizes) followed by the grid and
 * the iteration state as native-endian doubles and integers; it is meant
 * for the same library build, not as an interchange format.
 *
 * mcubes_state_size: *bytes receives the size of the current problem's
 *   checkpoint.  Errors: EINVAL (null), ESTATE (no setup).
 * mcubes_state_export: waits for the context's stream, then writes the
 *   checkpoint to buf (host, cap bytes; caller-owned).  Errors: EINVAL (null
 *   or cap too small), ESTATE (no setup, or a sharded pass sampled and not
 *   finished), ECUDA.
 * mcubes_state_import: replaces the context's options and problem with the
 *   checkpoint's (as mcubes_set_opts + mcubes_setup would), then restores
 *   its grid and iteration state; mcubes_iterate then continues with the
 *   next iteration.  On the same GPU model, the continued run's results,
 *   trace and grid are bit-identical to those of an uninterrupted run (the
 *   launch shape derives from the options and the SM count).  Errors:
 *   EINVAL (null, wrong magic or version, inconsistent sizes, an invalid
 *   problem or grid), ENOMEM, ECUDA; on error the context has no problem. */
mcubes_status mcubes_state_size(mcubes_ctx* ctx, long long* bytes);
/* The current problem's integrand id, dimension, bins per axis, itmax and
 * the number of iterations enqueued so far (any pointer may be NULL).
 * Errors: EINVAL (null ctx), ESTATE (no setup). */
mcubes_status mcubes_problem_get(mcubes_ctx* ctx, int* integrand_id, int* d, int* nb, int* itmax,
                                 int* iterations_enqueued);
mcubes_status mcubes_state_export(mcubes_ctx* ctx, void* buf, long long cap);
mcubes_status mcubes_state_import(mcubes_ctx* ctx, const void* buf, long long size);

/* One sampling pass (Alg. 3) over sub-cubes [cube_begin, cube_end) of
 * iteration `it` with the current grid, leaving the context's state
 * untouched; blocks.  sums (host, 3 values) receives the sum over those
 * cubes of the cube means, of the variances of the cube means, and of the
 * absolute cube means; C (host, [d][nb], may be NULL) receives the per-bin
 * sums of f^2 when adjust != 0.  The launch is the one mcubes_iterate uses. */
mcubes_status mcubes_sample_range(mcubes_ctx* ctx, unsigned it, int adjust, long long cube_begin,
                                  long long cube_end, double* sums, double* C);

/* ---- one integral over several GPUs: cube-range shards -------------------
 * Alg. 3 reduces every block's results (the cube means and variances, and
 * the bin contributions C) into one iteration result, and Alg. 2's host
 * loop refines the grid from them.  Splitting the sub-cubes [0, m) into
 * contiguous ranges, one per GPU, makes that reduction the only exchange:
 * every rank sets up the same problem with the same options (seed
 * included), samples its range -- the samples are keyed by the global cube
 * index, so the ranges together draw exactly one iteration's samples -- and
 * all ranks combine the gathered partials in rank order, so each runs the
 * identical rebinning and weighting with no broadcast of the grid.
 *
 * A rank's partial is MCUBES_SHARD_HEAD + hist_d * nb doubles: the sum of
 * its cube means, of the variances of those means, of |cube means|, then
 * the per-bin sums of f^2 [hist_d][nb] (zero in non-adjusting iterations;
 * hist_d = d, or 1 in m-Cubes1D).  mcubes_shard_partial_len gives the
 * length for the current problem. */
#define MCUBES_SHARD_HEAD 3
mcubes_status mcubes_shard_partial_len(mcubes_ctx* ctx, long long* len);

/* The sampling pass of the context's next iteration over sub-cubes
 * [cube_begin, cube_end) (any range, empty included), its partial written
 * to the device array d_partial.  Enqueued on the context's stream; returns
 * without waiting.  After an iteration that converged the pass does no
 * work and its partial is not meaningful (mcubes_shard_finish ignores it).
 * Errors: EINVAL (range, null), ESTATE (no setup, or every iteration
 * enqueued), ECUDA. */
mcubes_status mcubes_shard_sample(mcubes_ctx* ctx, long long cube_begin, long long cube_end, double* d_partial);

/* Finishes the iteration sampled by mcubes_shard_sample from nranks
 * partials gathered in rank order (device array [nranks][len]): they are
 * summed element by element in rank order, then the iteration's estimate
 * and variance are recorded, the grid is rebinned (adjusting iterations)
 * and all iterations are weighed and tested for convergence, as
 * mcubes_iterate does after its own pass.  Ranks that pass the same
 * gathered array end with identical state.  Enqueued on the context's
 * stream.  Errors: EINVAL (nranks < 1, null), ESTATE (no sampled
 * iteration to finish), ECUDA. */
mcubes_status mcubes_shard_finish(mcubes_ctx* ctx, const double* d_gathered, int nranks);

/* ---- sampling without device allocation ----------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: hosts whose device memory belongs to
 * another allocator (a framework's caching pool, a fixed arena in an
 * embedded or real-time service), and processes that must not grow their
 * device footprint, or stall on an allocation, once running.
 *
 * The same sampling pass as mcubes_sample_range, over sub-cubes
 * [cube_begin, cube_end) of iteration `it`, but with no context: the
 * problem is given directly (params, lo, hi are host arrays of nparams and d
 * values; nbins, g_override, seed and precision as in mcubes_opts), the grid
 * is read from the caller's device array d_grid ([d][nbins] right edges,
 * taken as exact), and the results go to the caller's device arrays d_sums
 * (3 values: sum of cube means, of their variances, of |cube means|) and,
 * when adjust != 0, d_hist ([d][nbins] per-bin sums of f^2; may be NULL
 * otherwise).  Work is enqueued on cuda_stream (NULL = legacy default
 * stream) and the call returns without waiting.  It launches at most
 * MCUBES_NOALLOC_MAX_BLOCKS blocks, so its sums are grouped differently from
 * mcubes_sample_range's: the two agree to rounding, not bit for bit.
 *
 * It allocates nothing: the per-block partial sums and the histogram
 * accumulator live in one static device array of the library,
 * 3 x MCUBES_NOALLOC_MAX_BLOCKS + 2 x MCUBES_NOALLOC_MAX_BINS doubles (about
 * 56 KiB), which every GPU that loads the library keeps until the process
 * exits.  Limits: d * nbins <=
 * MCUBES_NOALLOC_MAX_BINS, otherwise EINVAL (as for any invalid argument);
 * at most MCUBES_NOALLOC_MAX_BLOCKS sampling blocks are launched.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and must therefore come before any stream capture on that device.  All
 * calls share the array and each overwrites what it uses (the part that must
 * start at zero is cleared on the stream first), so calls whose work
 * overlaps on the GPU -- on different streams, or from different threads --
 * race and corrupt each other's results: serialise them.
 * Errors: EINVAL, ECUDA. */
#define MCUBES_NOALLOC_MAX_BLOCKS 304
#define MCUBES_NOALLOC_MAX_BINS 3072
mcubes_status mcubes_sample_range_noalloc(int device, int integrand_id, const double* params, int nparams,
                                          int d, const double* lo, const double* hi, long long ncall,
                                          int nbins, long long g_override, uint64_t seed, int precision,
                                          unsigned it, int adjust, long long cube_begin, long long cube_end,
                                          const double* d_grid, double* d_sums, double* d_hist,
                                          void* cuda_stream);

/* Diagnostic: evaluates, element-wise over n doubles of the device array
 * d_in into d_out (device), the library's double-precision logarithm
 * (which = 0) or exponential (1) -- table-driven with fixed-point series,
 * used by the FP64 integrands -- or CUDA's log (2) or exp (3), or the
 * library's single-precision cosine of the mixed-precision kernels (4) or
 * CUDA's cosf (5) (both on the value rounded to single precision), or the
 * library's exp(-x) multiplied, before its one rounding, by the fixed factor
 * (0xD3C21BCECCEDA100 / 2^63) 2^40 (6; the FP64 kernels fold their integer
 * Jacobian into the exponential this way), on cuda_stream (NULL = legacy
 * default stream); returns without waiting.
 * The paper has no counterpart; this exists to test accuracy.
 * Errors: EINVAL, ECUDA. */
mcubes_status mcubes_selftest_fxmath(int which, long long n, const double* d_in, double* d_out,
                                     void* cuda_stream);

/* Adjust-Bin-Bounds of one axis (Alg. 2; Lepage 1978) exactly as an
 * iteration's refinement runs it: d_C (device, nb doubles) is the axis's
 * histogram of F^2 sums, d_B / d_Blo (device, nb doubles each) its right
 * edges in the unit interval as double-double numbers (B[nb-1] = 1), updated
 * in place; alpha is the compression exponent.  An all-zero histogram leaves
 * the edges unchanged.  Runs on cuda_stream (NULL = legacy default stream)
 * and waits for it.  The paper has no counterpart; this exists to test the
 * device rebinning against the oracle on chosen histograms.
 * Errors: EINVAL (nb outside 2..MCUBES_NBMAX, alpha <= 0, a NULL pointer),
 * ENONFINITE (a non-finite histogram), ECUDA. */
mcubes_status mcubes_selftest_rebin(int nb, double alpha, double* d_C, double* d_B, double* d_Blo,
                                    void* cuda_stream);

/* Geometry of the current setup: sub-cubes per axis, sub-cubes, samples per
 * sub-cube, lanes per cube and sampling blocks chosen. */
mcubes_status mcubes_geometry_get(mcubes_ctx* ctx, long long* g, long long* m, long long* p,
                                  int* lanes_per_cube, int* blocks);

/* Turns per-launch CUDA-event timing on (enable != 0) or off and clears the
 * counters.  Timing records events on the context's stream around every
 * sampling launch and every refinement launch. */
mcubes_status mcubes_timing_reset(mcubes_ctx* ctx, int enable);

/* Waits, then reports the summed duration (ms) and count of the sampling
 * launches and of the refinement/finalisation launches since the last reset. */
mcubes_status mcubes_timing_get(mcubes_ctx* ctx, double* sample_ms, int* sample_launches,
                                double* refine_ms, int* refine_launches);

#ifdef __cplusplus
}
#endif

#endif /* MCUBES_H */
