/*
 * ifctn.h -- C ABI of the GB300 (sm_103a) iFCTN tensor-completion library.
 *
 * The library runs the proximal alternating minimisation (PAM) solver of
 * iFCTN-TC (Gan & Cui, "iFCTN: an intra-block Fully-Connected Tensor Network
 * Decomposition for Tensor Completion"): Sec. 4.1 eq. (iFCTN-TC) is the model,
 * Sec. 4.2 eq. (updateG) the factor blocks, eq. (updateX) the tensor block,
 * Algorithm 1 the loop.  All arithmetic runs in the library's CUDA kernels.
 *
 * Conventions (every entry point):
 *   - Dense tensors are C order (last index fastest), I_1 x ... x I_N,
 *     2 <= N <= 4.
 *   - Cherry factor G_{k,l} (k != l, Sec. 3 eq. (cherry_factor_set)) is an
 *     R_{k,l} x I_k row-major matrix.  A "packed factor array" holds the
 *     blocks in the order k = 0..N-1, then l = 0..N-1 (l != k), as FP64.
 *   - ranks[k*4+l] is the symmetric iFCTN-rank matrix R (Def. 2); entries
 *     with k,l < N, k != l must satisfy 1 <= R_{k,l} <= 8; others are ignored.
 *     Order-3 problems may use ranks up to 64 (the rank grid of Sec. 5.2
 *     reaches R_{1,2} = 36) as long as every Q_k = prod_{l != k} R_{k,l} is at
 *     most 4096; such problems always run the per-stage sweep graph (never the
 *     persistent launch) and are not tuned by ifctn_tune.
 *   - The observation mask holds one byte per tensor entry, nonzero =
 *     observed (the sample set Omega).
 *   - Tensor buffers are FP64 when the problem's precision is IFCTN_FP64 and
 *     FP32 when it is IFCTN_MIXED.  Factor buffers are always FP64.
 *   - Every pointer argument may be host memory (pageable or pinned) or device
 *     memory of the current device; the library detects which.  It copies
 *     inputs into memory it owns; the caller keeps ownership of its buffers.
 *   - No function throws.  Each returns an ifctn_status and, on failure,
 *     records a message readable with ifctn_last_error() (per thread).
 *   - A context is not thread-safe; a server is (submit/poll from any thread).
 */
#ifndef IFCTN_H
#define IFCTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IFCTN_OK = 0,
    IFCTN_EINVAL = 1,     /* bad argument: shape, rank, rho, null pointer */
    IFCTN_ENOMEM = 2,     /* device allocation failed or budget too small */
    IFCTN_ECUDA = 3,      /* a CUDA call failed */
    IFCTN_ENOTSPD = 4,    /* a proximal normal-equation matrix lost positive definiteness */
    IFCTN_EBUSY = 5,      /* server queue full */
    IFCTN_ENOTREADY = 6,  /* poll: job not finished yet (timeout 0) */
    IFCTN_ETIMEOUT = 7,   /* poll timed out, or a bounded device wait gave up */
    IFCTN_ENOTFOUND = 8   /* unknown ticket */
} ifctn_status;

typedef enum {
    IFCTN_FP64 = 0,   /* tensor, contractions, solves, reductions all FP64 */
    IFCTN_MIXED = 1   /* FP32 tensor, contractions and Gram (FP32 accumulate);
                         FP64 factor master copy, M_k reduction, stop-test,
                         objective and RSE sums.  The small proximal systems
                         are factorised in FP32 (LDL^T) and refined once with
                         a residual formed in two-float arithmetic (about 48
                         significant bits from FP32 instructions): no FP64
                         instruction runs in a solve stage. */
} ifctn_precision;

/* Algorithm 1's inputs (Sec. 4.2): order N, sizes, iFCTN ranks, proximal
   weight rho, t_max, epsilon, plus the arithmetic mode and the seed of the
   default initial factors. */
typedef struct {
    int32_t order;          /* N, 2..4 */
    int64_t dims[4];        /* I_k >= 1 for k < N */
    int32_t ranks[16];      /* R[k*4+l], symmetric, 1..8 off the diagonal (1..64 at order 3) */
    double rho;             /* proximal weight, > 0 (paper default 0.1) */
    int32_t max_sweeps;     /* t_max >= 0 (paper default 1000) */
    double tol;             /* epsilon of the relative-change test; 0 = run all sweeps */
    int32_t precision;      /* ifctn_precision */
    uint64_t seed;          /* seed of G^(0) when no initial factors are given */
} ifctn_problem;

/* Per-sweep record.  rel_change = ||X^{s+1}-X^s||_F / ||X^s||_F (the stop test
   of Algorithm 1); objective = 1/2 ||X^{s+1} - iFCTN(G^{s+1})||_F^2 (Sec. 4.1);
   rse = ||X_true - X||_F / ||X_true||_F and rmse = sqrt(mean over missing
   entries of (X_true - X)^2) (Sec. 5) when a ground truth was registered with
   ifctn_set_truth and metric logging is on, else NaN. */
typedef struct {
    int32_t sweeps_done;
    int32_t converged;
    double rel_change;
    double objective;
    double rse;
    double rmse;
} ifctn_stats;

typedef struct ifctn_ctx ifctn_ctx;
typedef struct ifctn_server ifctn_server;

/* Creates a solver context for one completion problem.
   obs: the observation O (tensor dtype, see conventions); entries outside
   Omega are ignored.  mask: one byte per entry.  X^(0) = P_Omega(O) with zeros
   elsewhere (Algorithm 1, initialisation).  init_factors: packed FP64 G^(0),
   or NULL for the default: seeded U(0,1) entries rescaled by one common
   factor so that ||iFCTN(G^0)||_F = ||P_Omega(O)||_F / sqrt(|Omega|/P).
   cuda_stream: a cudaStream_t to run on, or NULL for a stream owned by the
   context.  On success *out receives the context (free with ifctn_destroy). */
ifctn_status ifctn_create(const ifctn_problem* prob, const void* obs, const uint8_t* mask,
                          const double* init_factors, void* cuda_stream, ifctn_ctx** out);

/* Runs n sweeps of Algorithm 1 (eq. (updateG) for every block in the order
   k = 1..N, i != k ascending, each block with the latest other factors; then
   eq. (updateX)), ignoring tol.  Blocks until done.  out (nullable) receives
   the record of the last sweep. */
ifctn_status ifctn_sweep(ifctn_ctx* ctx, int32_t n, ifctn_stats* out);

/* Enqueues n sweeps (tol ignored) on the context's stream and returns without
   waiting, so that callers can pipeline or time them with their own events on
   that stream.  Device-side failures are reported by the next synchronous call
   (e.g. ifctn_sweep(ctx, 0, &stats)). */
ifctn_status ifctn_sweep_async(ifctn_ctx* ctx, int32_t n);

/* Algorithm 1 from the current state: sweeps until rel_change < tol (tol > 0)
   or until max_sweeps sweeps have run in this call.  out_X (nullable) receives
   the recovered tensor; out (nullable) the last record. */
ifctn_status ifctn_complete(ifctn_ctx* ctx, void* out_X, ifctn_stats* out);

/* Writes iFCTN(G) of the current factors (eq. (iFCTN), Def. 2) into out
   (tensor dtype, P entries). */
ifctn_status ifctn_reconstruct(ifctn_ctx* ctx, void* out);

/* Checkpoint / resume: the PAM state is (G, X) (Sec. 4.2). */
ifctn_status ifctn_get_factors(ifctn_ctx* ctx, double* out);
ifctn_status ifctn_set_factors(ifctn_ctx* ctx, const double* in);
ifctn_status ifctn_get_x(ifctn_ctx* ctx, void* out);
ifctn_status ifctn_set_x(ifctn_ctx* ctx, const void* in);

/* Registers a ground-truth tensor (tensor dtype) for RSE/RMSE and turns
   per-sweep metric logging on (log != 0) or off. */
ifctn_status ifctn_set_truth(ifctn_ctx* ctx, const void* xtrue, int32_t log);

/* Copies up to max per-sweep records (oldest first, of the sweeps run since
   creation, capped at the last 4096) into out; *n receives the count. */
ifctn_status ifctn_get_log(ifctn_ctx* ctx, ifctn_stats* out, int32_t max, int32_t* n);

/* Stage-level access for verification: the mode-k regrouped quantities of
   Prop. 1 at the current state, M_k = X_(k) Z_k (I_k x Q_k, row-major) and
   K_k = Z_k^T Z_k (Q_k x Q_k), Q_k = prod_{m != k} R_{k,m}, rank index in C
   order over the modes m != k ascending.  FP64 host or device buffers. */
ifctn_status ifctn_mode_system(ifctn_ctx* ctx, int32_t k, double* Mk, double* Kk);

/* Enqueues one launch of a single stage of the sweep on the context's stream,
   without waiting (for per-kernel timing with CUDA events).  stage:
     0 = the HBM-streaming mode-k contraction (partials of M_k),
     1 = the mode-k Gram chain (K_k), 2 = the mode-k proximal solves (updates
     the factors), 3 = the fused reconstruct + masked X update (updates X),
     4 = the reduction of the contraction partials into M_k.
   k is ignored by stage 3. */
ifctn_status ifctn_launch_stage(ifctn_ctx* ctx, int32_t stage, int32_t k);

/* Diagnostic of the failure path (no counterpart in the paper; it checks this
   library's error handling).  Every device wait of the library's kernels is
   bounded: on expiry the kernel records a timeout in the context's flag word
   and returns, and the call reports IFCTN_ETIMEOUT.  This runs, on the
   context's stream, one grid barrier that a CTA never joins and one mbarrier
   phase that no copy completes, each with a budget of budget_cycles SM clock
   cycles (1000..4e9), and returns what a real expiry returns: IFCTN_ETIMEOUT.
   The flag word is cleared after it is reported (by this call and by every
   other call that reports a device failure), so the context stays usable;
   this call does not touch the problem's state (G, X).  IFCTN_EINVAL for a
   budget out of range. */
ifctn_status ifctn_wait_selftest(ifctn_ctx* ctx, int64_t budget_cycles);

/* Slab-sharded sweeps: one tensor split along its first mode across several
   processes, one GPU each (the paper's column independence, Sec. 4.2: the
   columns of G_{1,l} are solved independently, and every other quantity a
   mode needs is a sum over tensor entries).
   Each process creates an ordinary context for its slab X[lo:hi, ...]: a
   problem with dims (hi - lo, I_2, ..., I_N) and the full ranks, whose
   factors G_{1,l} are the columns lo..hi-1 of the whole problem's G_{1,l}
   and whose other factors are the whole problem's.  ifctn_sweep_exchange
   then runs n sweeps of Algorithm 1 with the per-stage kernels and calls
   allreduce(user, values, count) on host memory wherever the slabs' results
   must be combined:
     - for every mode k >= 2, before its column solves: the slab's partial
       M_k (I_k x Q_k) followed by its partial K_k (Q_k x Q_k), count =
       I_k Q_k + Q_k^2 doubles;
     - after the X update: the slab's ||X^{s+1} - X^s||^2, ||X^s||^2 and
       ||X^{s+1} - iFCTN(G^{s+1})||^2 (count = 3).
   allreduce must replace every value by its sum over the processes, the same
   bits on every process (e.g. an all-gather summed in process order), and
   return 0; a nonzero return stops the call with IFCTN_EINVAL.  Mode 1 needs
   no exchange: its M_1 rows and its columns are the slab's own, and K_1 does
   not depend on i_1.  The factors G_{k,l} of the modes k >= 2 then come out
   the same on every process and the slab's G_{1,l} columns and X entries are
   those of the whole problem's sweep (up to the order of the partial sums).
   tol is ignored; out (nullable) receives sweeps_done (counted per context),
   rel_change and objective of the last sweep from the combined sums (rse and
   rmse NaN).  No data-path collective runs on the device: the caller's
   allreduce may use any transport. */
typedef int32_t (*ifctn_allreduce_fn)(void* user, double* values, int64_t count);
ifctn_status ifctn_sweep_exchange(ifctn_ctx* ctx, int32_t n, ifctn_allreduce_fn allreduce, void* user,
                                  ifctn_stats* out);

/* Autotuning of the streaming contraction (no counterpart in the paper: it
   picks launch shapes for this GPU).  For every mode whose contraction runs
   the warp-pipelined HBM-streaming kernels, the planner leaves four choices
   open: two rows per lane or one, the ring stages per warp, the task size and
   the grouping of slabs into work units.  This call takes each mode's choice
   from the cache file at cache_path (nullable) when the file holds the key
   (library source digest, dtype, shape, ranks, mode, SM count); otherwise it
   times the distinct candidate plans on the context's stream (CUDA events,
   the median of five runs of the contraction on the context's own
   tensor, together with the reduction of its partials into M_k, which
   depends on the plan too), keeps the fastest by the rule of
   ifctn_tune_choose, and appends
   the choice to the cache.  The results of the sweep do not depend on the
   choice beyond the order of floating-point sums within a mode's partials.
   *timed (nullable) receives the number of candidate plans timed (0 when the
   cache answered every mode).  Contexts created while the environment
   variable IFCTN_TUNE_CACHE names a file tune themselves this way at
   creation.  Such a creation also picks the execution path of a tensor small
   enough for the one-launch persistent path: unless the cache holds the
   choice for the shape, both paths are built, ten sweeps of each are timed
   from the same initial state, the faster context is returned (its state
   restored to the initial one) and the choice is appended to the cache.  The
   contexts of a server's jobs only read that cache (a job never waits for
   timing); shapes it lacks keep the planner's defaults.  Contexts whose sweeps run as one persistent launch have no
   choices to make (*timed = 0). */
ifctn_status ifctn_tune(ifctn_ctx* ctx, const char* cache_path, int32_t* timed);

/* The tuner's selection rule, exposed for callers that time candidates
   themselves: given n > 0 timings with the planner's default first, returns
   the index of the fastest, or 0 unless the fastest beats the default by 2 %
   or more; -1 for n <= 0 or a null array.  Host only. */
int32_t ifctn_tune_choose(int32_t n, const double* seconds);

/* Number of kernel launches one sweep issues when sweeps run as a CUDA graph
   of per-stage kernels (for launch accounting). */
int32_t ifctn_kernels_per_sweep(const ifctn_ctx* ctx);

/* Total number of kernel launches this context has issued for sweeps so far.
   When the device can hold the whole grid co-resident, each sweep call is one
   persistent cooperative launch that runs all its sweeps. */
int64_t ifctn_launch_count(const ifctn_ctx* ctx);

/* Profiling aid for the persistent path: seconds from the start of the first
   sweep of the last persistent launch to the end of each of its phases, in
   order (per mode k: contraction, its barrier, reduction, its barrier, solves,
   their barrier; for k = 0..3; then the X update and its barrier), up to max
   values.  *n receives the count (0 when sweeps run as a graph). */
ifctn_status ifctn_phase_times(ifctn_ctx* ctx, double* out, int32_t max, int32_t* n);

void ifctn_destroy(ifctn_ctx* ctx);

/* Allocation-free reconstruction (an addition of this library; the paper has
   no counterpart).  For callers that cannot call cudaMalloc -- their device
   memory is owned by another allocator, or they must not pay for or
   synchronise on an allocation on their path -- this writes iFCTN(G) (eq.
   (iFCTN)) of the packed FP64 factors into out without allocating anything.
   factors and out must be device memory of the current device (out in the
   tensor dtype of precision: FP64 for IFCTN_FP64, FP32 for IFCTN_MIXED); the
   shape arguments follow ifctn_problem (dims[0..order-1], ranks[16]).
   Scratch: the pair matrices W_{p,q} live in a fixed 8 MiB device array
   inside the library, loaded on every GPU that loads the library and held
   until the process exits; problems whose pair matrices need more
   (sum_{p<q} I_p I_q entries of the tensor dtype) are rejected with
   IFCTN_EINVAL.  The first call on a device looks the array's address up;
   make that first call before any stream capture.  The work is enqueued on
   cuda_stream (NULL = the legacy default stream) and the call returns without
   waiting.  All calls share the one array, and each call overwrites it: calls
   whose work overlaps on the GPU (different streams, or concurrent host
   threads) race. */
ifctn_status ifctn_reconstruct_noalloc(int32_t order, const int64_t* dims, const int32_t* ranks,
                                       int32_t precision, const double* factors, void* out,
                                       void* cuda_stream);

/* ---------------------------------------------------------------------------
   Serving: continuous batching of completion jobs on one GPU.
   A server owns a device-memory budget and up to max_slots resident jobs.
   ifctn_submit copies the job's inputs to pinned host memory and queues it;
   a scheduler thread admits queued jobs in arrival order as slots and budget
   free up and keeps every resident job's sweeps in flight:
     - jobs whose sweeps run as one persistent launch (tensors that stay in
       L2) are batched: one cooperative launch per round runs a few sweeps of
       each such job (one dtype per round), every job on its own slice of the
       grid with its own barriers, stop test and logs;
     - larger jobs run their sweep graphs on separate CUDA streams, so their
       kernels overlap on the device.
   Each result is copied to pinned host memory when its job finishes.  A job
   runs the same kernel code and the same fixed-order reductions alone or in
   a mix (the persistent kernel's results do not depend on its grid), so its
   result does not depend on the mix.
   --------------------------------------------------------------------------- */
ifctn_status ifctn_server_create(size_t hbm_budget_bytes, int32_t max_slots, ifctn_server** out);

/* Queues one job (same inputs as ifctn_create; obs/mask/init are copied
   before return).  *ticket receives the job id.  Fails with IFCTN_ENOMEM if
   the job alone exceeds the budget. */
ifctn_status ifctn_submit(ifctn_server* srv, const ifctn_problem* prob, const void* obs,
                          const uint8_t* mask, const double* init_factors, uint64_t* ticket);

/* Waits up to timeout_us microseconds (0 = do not wait, <0 = forever) for the
   job.  On IFCTN_OK the result was copied to out_X (nullable; tensor dtype)
   and out (nullable), and the ticket is released.  IFCTN_ENOTREADY (timeout 0)
   or IFCTN_ETIMEOUT leave the job untouched. */
ifctn_status ifctn_poll(ifctn_server* srv, uint64_t ticket, void* out_X, ifctn_stats* out,
                        int64_t timeout_us);

/* Server counters: jobs queued, resident and completed; device bytes in use;
   the largest number of jobs resident at once; the shared persistent launches
   run so far and the job rounds they carried (see the serving notes above). */
typedef struct {
    int64_t queued, resident, completed;
    int64_t bytes_in_use;
    int64_t peak_resident;
    int64_t batch_launches, batched_jobs;
} ifctn_server_info;
ifctn_status ifctn_server_info_get(ifctn_server* srv, ifctn_server_info* out);

/* Latency of the job with this ticket, in seconds from its ifctn_submit to the
   end of its last sweep on the device (the result copied to pinned host
   memory).  IFCTN_ENOTFOUND while the job has not finished, or for a ticket
   the server never issued.  Still readable after ifctn_poll has released the
   ticket. */
ifctn_status ifctn_server_latency(ifctn_server* srv, uint64_t ticket, double* seconds);

void ifctn_server_destroy(ifctn_server* srv);

/* Message of the last failure on the calling thread ("" if none). */
const char* ifctn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IFCTN_H */
