/*
 * dgs.h -- C ABI of the GB300 Deep Greedy Switching (DGS) solver for the
 * linear sum assignment problem (LSAP).
 *
 * Problem (paper Section 3): given an n x n benefit matrix a, find a
 * permutation maximising sum_i a[i][tau(i)].  DGS is a heuristic: it starts
 * from a full assignment (Section 3.1) and applies improving 2-exchanges
 * found by the agent/job difference evaluations (Algorithm 2, Section 3.2)
 * until none improves, with the parallel switching rule of Algorithm 3 and
 * the conflict check of Algorithm 4 (Section 5).
 *
 * Conventions shared by every entry point
 *   - benefit: DEVICE pointer to n*n int32, row-major, row i = agent i,
 *     column j = job j (a[i*n + j]).  Caller-owned, never written.  Every
 *     entry must satisfy |a| < 2^29 so that each 2-exchange gain (a sum of
 *     four entries) is exact in int32; otherwise DGS_ERR_RANGE.
 *   - sigma_out[i] = job assigned to agent i (DEVICE pointer, n int32,
 *     caller-owned).  The paper writes this map as tau = M(sigma) and uses
 *     sigma for job -> agent; the output here is the agent -> job map.
 *   - objective_out: pointer to one int64 (exact sum of benefits), in
 *     DEVICE memory or in HOST memory (pageable or pinned).
 *   - stream: a cudaStream_t (the library includes no CUDA header here and
 *     takes it as dgs_stream_t, the same pointer type).
 *   - dgs_solve, dgs_solve_ex and dgs_solve_rect are STREAM-ORDERED: they
 *     enqueue the whole solve on `stream` and return without waiting for it.
 *     The switching loop runs on the device (a CUDA graph whose conditional
 *     loop node repeats until the loop state says the solve has ended), so no
 *     call waits for a sweep.  The outputs -- sigma_out, *objective_out,
 *     dgs_stats and dgs_options.status_out -- are valid once the stream has
 *     reached the end of the solve (for example after
 *     cudaStreamSynchronize); outputs in host memory are written then by a
 *     host callback on the stream, so host memory passed for them must stay
 *     valid until the stream has reached that point.  The return value reports only what is
 *     known when the work is enqueued (invalid arguments, allocation or
 *     launch failures); the outcome of the solve itself (DGS_OK,
 *     DGS_TIMEOUT, DGS_ERR_RANGE, DGS_ERR_INVALID for a USER start that is
 *     not a permutation, DGS_ERR_INTERNAL) arrives in dgs_stats.status and
 *     *dgs_options.status_out.  After an error every sigma_out entry is -1.
 *     Exceptions: options.profile = 1 makes the call wait for its own
 *     timings; dgs_solve_host and the evaluation, greedy-start, autotuning
 *     and batched calls block until their outputs are final.
 *   - The library allocates its own device workspace (about 4*n*n bytes for
 *     the transposed copy of a plus O(n)) with stream-ordered allocation and
 *     frees it, stream-ordered, behind the solve.  Allocation failure ->
 *     DGS_ERR_OOM.
 *   - Results are deterministic: bit-identical across runs, launch shapes
 *     and devices, and equal to the plain CPU oracle's.
 */
#ifndef DGS_H
#define DGS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DGS_API __attribute__((visibility("default")))
#else
#define DGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* dgs_stream_t; /* == cudaStream_t */

typedef enum {
    DGS_OK = 0,
    DGS_ERR_INVALID = 1,  /* n <= 0, null pointer, bad option, invalid USER start */
    DGS_ERR_RANGE = 2,    /* some |a_ij| >= 2^29 */
    DGS_ERR_OOM = 3,      /* device workspace allocation failed */
    DGS_ERR_CUDA = 4,     /* a CUDA call failed (see dgs_last_cuda_error) */
    DGS_TIMEOUT = 5,      /* sweep cap or deadline hit: outputs hold the valid
                             assignment reached so far and its objective */
    DGS_PENDING = 6,      /* dgs_poll / dgs_server_wait: not finished yet */
    DGS_ERR_BUSY = 7,     /* dgs_submit: the request can never fit the budget */
    DGS_ERR_INTERNAL = 8, /* a device-side consistency check failed */
    DGS_CANCELLED = 9     /* dgs_poll / dgs_server_wait: the request was
                             withdrawn by dgs_cancel before it was admitted */
} dgs_status;

typedef enum {
    DGS_INIT_GREEDY = 0,   /* global greedy start (Section 3.1, default) */
    DGS_INIT_RANDOM = 1,   /* random start (Section 3.1, the paper's own): the
                              identity shuffled by Fisher-Yates (Durstenfeld:
                              for i = n-1 .. 1 swap i with next() mod (i+1)),
                              next() = splitmix64 (Steele, Lea, Flood 2014)
                              started at dgs_options.seed */
    DGS_INIT_IDENTITY = 2, /* agent i starts on job i */
    DGS_INIT_USER = 3      /* caller's permutation in dgs_options.init_sigma */
} dgs_init_mode;

/* Which algorithm runs after the start. */
typedef enum {
    DGS_ALG_PARALLEL = 0,   /* Algorithm 3, parallel DGS (Section 5, default) */
    DGS_ALG_SEQUENTIAL = 1  /* Algorithm 1, sequential DGS (Section 3.3): one
                               switch per iteration, the largest delta over all
                               agent and job slots (ties: lowest index; the
                               agent slot only when strictly larger), ADE/JDE
                               of the two agents and jobs after a commit, the
                               outer repeat until a pass leaves f unchanged.
                               dgs_stats.sweeps counts while-loop iterations,
                               max_sweeps caps them. */
} dgs_algorithm;

/* Which slots are re-evaluated after each parallel switch of Algorithm 3. */
typedef enum {
    DGS_REEVAL_BOX = 0,    /* the slots not in the conflict set C (the box of
                              Algorithm 3; slots in C keep their candidates) */
    DGS_REEVAL_ALL = 1     /* every slot (the text of Section 5 read as
                              re-evaluating everything) */
} dgs_reeval_rule;

/* Which kernel runs the full difference evaluations (Algorithm 2 for every
 * slot).  Both give identical candidates: each is the maximum of the same
 * gains with the same tie-breaks. */
typedef enum {
    DGS_EVAL_TILE_PAIRS = 0,  /* unordered pairs of 64 x 64 tiles of the
                                 sigma-permuted benefit rows: every benefit is
                                 read once per evaluation (4 n^2 bytes) */
    DGS_EVAL_ROW_OWNER = 1    /* one CTA per row j of the gain matrix: row
                                 sigma(j) of the benefits plus row j of the
                                 maintained transpose (8 n^2 bytes) */
} dgs_evaluation_kernel;

typedef struct {
    int32_t init;              /* a dgs_init_mode */
    const int32_t* init_sigma; /* DEVICE, n int32 agent -> job; read for USER */
    int32_t max_sweeps;        /* cap on switching sweeps, <= 0: none */
    int64_t deadline_us;       /* wall-clock budget from the call, <= 0: none */
    /* Optional per-sweep trace, DEVICE pointers (any may be NULL): for sweep
     * s < trace_capacity, accepted candidate slots, committed 2-exchanges
     * and the objective after the sweep. */
    int32_t trace_capacity;
    int32_t* trace_accepted;
    int32_t* trace_applied;
    int64_t* trace_objective;
    /* 1: time the whole solve, the first full difference evaluation and the
     * greedy start with CUDA events on the call's stream (dgs_stats.solve_ms,
     * evaluation_ms, greedy_ms); the call then waits for the solve.  0: no
     * timing. */
    int32_t profile;
    uint64_t seed;             /* DGS_INIT_RANDOM: generator start */
    int32_t reeval_rule;       /* a dgs_reeval_rule (default DGS_REEVAL_BOX) */
    int32_t algorithm;         /* a dgs_algorithm (default DGS_ALG_PARALLEL);
                                  dgs_solve_batched and the server take
                                  DGS_ALG_PARALLEL only */
    int32_t evaluation;        /* a dgs_evaluation_kernel (default
                                  DGS_EVAL_TILE_PAIRS); dgs_solve_batched and
                                  the server take DGS_EVAL_TILE_PAIRS only */
    /* Where the outcome of a stream-ordered solve is written when the stream
     * reaches its end (a dgs_status as int32), DEVICE or HOST memory; NULL:
     * not written. */
    int32_t* status_out;
} dgs_options;

typedef struct {
    int32_t sweeps;           /* iterations of the switching loop (Alg. 3) */
    int32_t events;           /* sweeps that committed at least one exchange */
    int64_t swaps_applied;    /* committed 2-exchanges */
    int32_t greedy_rounds;    /* greedy start: the most proposals one agent
                                 made (deferred acceptance; depends on the
                                 order in which the GPU ran them), or the
                                 locally-dominant rounds of the fallback */
    int32_t full_evaluations; /* full difference evaluations (all slots) */
    int32_t row_updates;      /* incremental re-evaluations (row tasks) */
    int64_t rows_recomputed;  /* rows re-evaluated by those row tasks */
    int64_t initial_objective;/* objective of the starting assignment */
    int64_t kernel_launches;  /* kernels this call launched */
    double evaluation_ms;     /* first full evaluation, when options.profile */
    double greedy_ms;         /* greedy start after pass 1, when options.profile */
    int64_t greedy_rescans;   /* rows of a (or its transpose) the greedy start
                                 rescanned (depends on the order of proposals) */
    int32_t status;           /* the solve's outcome (a dgs_status) */
    double solve_ms;          /* everything the call enqueued, when options.profile */
} dgs_stats;

/* Fill *opt with the defaults (GREEDY start, no cap, no deadline, no trace). */
DGS_API void dgs_default_options(dgs_options* opt);

/* Solve one instance with default options (Algorithm 3 from a greedy start
 * to termination: no 2-exchange improves the result).  Stream-ordered (see
 * the conventions above). */
DGS_API dgs_status dgs_solve(const int32_t* benefit, int32_t n, int32_t* sigma_out,
                     int64_t* objective_out, dgs_stream_t stream);

/* Solve with options; stats (HOST) may be NULL.  Stream-ordered; stats are
 * written when the stream reaches the end of the solve. */
DGS_API dgs_status dgs_solve_ex(const int32_t* benefit, int32_t n, int32_t* sigma_out,
                        int64_t* objective_out, const dgs_options* options,
                        dgs_stats* stats, dgs_stream_t stream);

/* Same as dgs_solve_ex but every buffer is in HOST memory (pageable or
 * pinned): benefit (n*n int32), sigma_out (n int32).  The host->device copy
 * of benefit and the device->host copy of sigma_out are part of the call,
 * which BLOCKS until the outputs are final and returns the solve's outcome. */
DGS_API dgs_status dgs_solve_host(const int32_t* benefit_host, int32_t n,
                          int32_t* sigma_out_host, int64_t* objective_out,
                          const dgs_options* options, dgs_stats* stats,
                          dgs_stream_t stream);

/* Rectangular instances: n_agents agents, m_jobs jobs, benefit n_agents x
 * m_jobs (DEVICE, row-major, row = agent, caller-owned).  The switching also
 * moves an agent to a free job (n < m) or off its job (n > m, where an
 * unassigned agent is worth 0): the method runs on the square instance of
 * size max(n, m) padded with zero-benefit dummy agents or dummy jobs,
 * numbered after the real ones, so that such a move is a 2-exchange with a
 * dummy (same gain).  assign_out: DEVICE, n_agents int32, the job of each
 * agent or -1 when it is left without one.  *objective_out: the sum of the
 * real benefits.  options as for dgs_solve_ex, except that USER starts and
 * traces are not taken (DGS_ERR_INVALID).  Workspace: about 8 max(n, m)^2
 * bytes (the padded matrix and its transpose).  Stream-ordered like
 * dgs_solve_ex. */
DGS_API dgs_status dgs_solve_rect(const int32_t* benefit, int32_t n_agents, int32_t m_jobs, int32_t* assign_out,
                                  int64_t* objective_out, const dgs_options* options, dgs_stats* stats,
                                  dgs_stream_t stream);

/* One fresh difference evaluation of every agent and job (Algorithm 2 for
 * all agents, JDE for all jobs; the first parallel block of Algorithm 3)
 * for the assignment sigma_in (DEVICE, agent -> job, must be a permutation).
 * Outputs are DEVICE arrays of n int32:
 *   agent_gain[i] / agent_job[i]: best strictly positive gain of agent i and
 *     the job it would move to (ties: lowest job); 0 / -1 when none improves;
 *   job_gain[j] / job_agent[j]: the same for job j and the agent it would
 *     move to (ties: lowest agent); 0 / -1 when none improves.
 * Blocks until the outputs are final. */
DGS_API dgs_status dgs_evaluate(const int32_t* benefit, int32_t n, const int32_t* sigma_in,
                        int32_t* agent_gain, int32_t* agent_job,
                        int32_t* job_gain, int32_t* job_agent,
                        dgs_stream_t stream);

/* The greedy starting assignment alone (Section 3.1 under the global-greedy
 * reading: repeatedly take the largest remaining benefit, ties to the lowest
 * agent then the lowest job).  sigma_out: DEVICE, agent -> job.  Blocks. */
DGS_API dgs_status dgs_greedy_init(const int32_t* benefit, int32_t n, int32_t* sigma_out,
                           dgs_stream_t stream);

/* ------------------------------------------------------------------------
 * Autotuning of launch shapes.  The paper fixes its block sizes by hand
 * (Section 4); here the shape of the full difference evaluation (Algorithm 2
 * for all slots: rows per thread, column tiles per work item, and whether
 * the sigma-gathered rows arrive by TMA gathers or by per-thread copies) is
 * chosen per size class by timing.  dgs_autotune times every candidate shape on a
 * synthetic n x n instance (values in [0, 10016), a random assignment; it
 * allocates about 4*n*n bytes for it) on `stream`, keeps the fastest for all
 * sizes in the same class (n in (2^(b-1), 2^b]) for the rest of the process,
 * and reports every candidate's time in *result (may be NULL).  The shape
 * never changes a result (every key is a maximum over the same pairs); it
 * only changes the time.  n in [2, 131072]; blocks until done.
 * dgs_get_tuning reports the shape that solves of size n use now. */
#define DGS_TUNE_MAX_CANDIDATES 16
typedef struct {
    int32_t n_lo, n_hi;       /* the size class the result applies to */
    int32_t rows_per_thread;  /* chosen: 4 (1024-thread CTAs), 8 (512) or 16 (256) */
    int32_t strip;            /* chosen: column tiles per work item, 0 = one
                                 contiguous, equal range of tiles per CTA */
    double best_ms;           /* evaluation time of the chosen shape */
    int32_t candidates;       /* shapes timed */
    int32_t cand_rows[DGS_TUNE_MAX_CANDIDATES];
    int32_t cand_strip[DGS_TUNE_MAX_CANDIDATES];
    double cand_ms[DGS_TUNE_MAX_CANDIDATES];  /* best of three launches each */
    int32_t tma;              /* chosen: 1 = rows gathered by TMA (tile::gather4) */
    int32_t cand_tma[DGS_TUNE_MAX_CANDIDATES];
} dgs_tuning;
DGS_API dgs_status dgs_autotune(int32_t n, dgs_tuning* result, dgs_stream_t stream);
DGS_API dgs_status dgs_get_tuning(int32_t n, int32_t* rows_per_thread, int32_t* strip, int32_t* tma);

/* ------------------------------------------------------------------------
 * Batched solves.  The paper solves one instance at a time; its motivating
 * setting (Section 1: a central node that repeatedly assigns peers) solves
 * many.  dgs_solve_batched runs Algorithm 3 (from the start of Section 3.1)
 * on `count` independent instances of different sizes together: every
 * instance keeps its own loop state on the device, and one persistent launch
 * per kernel works on all instances that are in that kernel's phase
 * (greedy rounds, first evaluation, switching sweeps).  The host replays a
 * captured CUDA graph of one step (a fixed number of greedy rounds and
 * switching iterations) until every instance has finished.  Each result is
 * bit-identical to dgs_solve_ex on that instance alone with the same options.
 *
 *   benefits[k]    DEVICE pointer to instance k's ns[k] x ns[k] int32 matrix
 *                  (row-major, caller-owned, not written); the array of
 *                  pointers itself is HOST memory, as are ns[].
 *   ns[k]          1 <= ns[k] <= DGS_BATCH_MAX_N.
 *   sigma_outs[k]  DEVICE pointer to ns[k] int32 (agent -> job); host array.
 *   objectives_out HOST array of count int64.
 *   options        NULL or shared by all instances: init GREEDY, RANDOM
 *                  (every instance from the same seed) or IDENTITY (USER and
 *                  traces are not supported: DGS_ERR_INVALID); max_sweeps,
 *                  deadline_us and reeval_rule apply to each instance.
 *   statuses_out   NULL or HOST array of count statuses (per instance).
 *   stats_out      NULL or HOST array of count dgs_stats.
 * Returns DGS_OK when every instance returned DGS_OK, else the status of the
 * first instance that did not.  Workspace: about 4*n*n + O(n) bytes per
 * instance, allocated stream-ordered for the call.  Blocks until done; the
 * work runs on a private stream ordered after `stream`. */
#define DGS_BATCH_MAX_N 32767
DGS_API dgs_status dgs_solve_batched(const int32_t* const* benefits, const int32_t* ns, int32_t count,
                                     int32_t* const* sigma_outs, int64_t* objectives_out,
                                     const dgs_options* options, dgs_status* statuses_out,
                                     dgs_stats* stats_out, dgs_stream_t stream);

/* ------------------------------------------------------------------------
 * Served solves: a request loop in the spirit of the paper's central
 * peer-assignment node (Section 1).  A server owns one worker thread and a
 * device-memory budget on the device that is current when it is created.
 * Requests are admitted in arrival order as soon as their workspace fits in
 * the budget (continuous batching): the server's upload thread copies an
 * admitted request's matrix to the device while the resident instances keep
 * stepping; the instance then joins the running batch at the next step,
 * keeps its matrix and loop state resident on the device until it finishes,
 * and overlaps on the GPU with every other resident instance.  Results are
 * bit-identical to dgs_solve of the instance alone.
 *
 * dgs_server_create: budget_bytes > 0; max_resident = cap on instances
 *   resident at once (<= 0: 256).  *out receives the server.
 * dgs_submit: benefit is n x n int32 row-major, in HOST memory when flags
 *   has DGS_SUBMIT_HOST, else DEVICE memory of the server's device.  The
 *   buffer must hold the final values when dgs_submit is called and stay
 *   valid until the ticket has finished (it is copied into the server's own
 *   device memory at admission).  1 <= n <= DGS_BATCH_MAX_N.  A request whose
 *   workspace (dgs_server_request_bytes) exceeds the whole budget returns
 *   DGS_ERR_BUSY; otherwise it is queued and *ticket identifies it.
 * dgs_poll: DGS_PENDING while the request is queued or running; otherwise
 *   the request's final status, with sigma_out_host (n int32, agent -> job,
 *   HOST), *objective_out, and (if not NULL) *stats and *times filled; a
 *   finished ticket is forgotten after the poll that returns it.  Unknown
 *   ticket: DGS_ERR_INVALID.
 * dgs_server_wait: as dgs_poll, waiting up to timeout_us (< 0: no limit).
 * dgs_server_destroy: finishes the resident instances, drops queued ones,
 *   stops the worker and frees the server's device memory. */
typedef struct dgs_server dgs_server;
#define DGS_SUBMIT_HOST 1
typedef struct {
    int64_t submit_ns;  /* steady-clock times: submission, */
    int64_t admit_ns;   /* admission (budget and a slot granted), */
    int64_t done_ns;    /* completion (result ready to be taken), */
    int64_t upload_ns;  /* start of the matrix's upload, */
    int64_t ready_ns;   /* matrix on the device, */
    int64_t start_ns;   /* solve started (placed in a slot of the batched */
                        /* engine, or taken by a solo thread) */
} dgs_request_times;
typedef struct {
    int32_t resident;        /* instances on the device now */
    int32_t queued;          /* requests waiting for admission */
    int64_t steps;           /* steps run so far */
    int64_t completed;       /* requests finished so far */
    size_t bytes_in_use;     /* budget taken by resident instances */
    int64_t kernel_launches; /* kernels launched by all steps so far */
    double upload_ms;        /* time the upload thread spent copying matrices */
    double step_ms;          /* time the worker spent in steps (graph replays) */
} dgs_server_info;
DGS_API dgs_status dgs_server_create(size_t budget_bytes, int32_t max_resident, dgs_server** out);
DGS_API size_t dgs_server_request_bytes(int32_t n);
DGS_API dgs_status dgs_submit(dgs_server* server, const int32_t* benefit, int32_t n, int32_t flags,
                              uint64_t* ticket);
/* dgs_submit with per-request options (NULL: defaults): the start (GREEDY,
 * RANDOM with options->seed, IDENTITY, or USER: options->init_sigma, n int32
 * agent -> job in the same memory as benefit, e.g. the previous solution of
 * a periodic re-solve -- a warm start), reeval_rule, max_sweeps and
 * deadline_us (counted from admission).  algorithm must be
 * DGS_ALG_PARALLEL and no trace is taken (DGS_ERR_INVALID otherwise).
 * init_sigma follows the same lifetime rule as benefit. */
DGS_API dgs_status dgs_submit_ex(dgs_server* server, const int32_t* benefit, int32_t n, int32_t flags,
                                 const dgs_options* options, uint64_t* ticket);
DGS_API dgs_status dgs_poll(dgs_server* server, uint64_t ticket, int32_t* sigma_out_host,
                            int64_t* objective_out, dgs_stats* stats, dgs_request_times* times);
DGS_API dgs_status dgs_server_wait(dgs_server* server, uint64_t ticket, int64_t timeout_us,
                                   int32_t* sigma_out_host, int64_t* objective_out, dgs_stats* stats,
                                   dgs_request_times* times);
/* Withdraw a request that has not been admitted yet (it still waits for
 * budget or a slot): DGS_OK, and its ticket then polls DGS_CANCELLED.  A
 * request already admitted runs to its end: DGS_PENDING.  Unknown or
 * finished tickets: DGS_ERR_INVALID. */
DGS_API dgs_status dgs_cancel(dgs_server* server, uint64_t ticket);
DGS_API dgs_status dgs_server_get_info(dgs_server* server, dgs_server_info* info);
DGS_API void dgs_server_destroy(dgs_server* server);

/* ------------------------------------------------------------------------
 * Difference evaluation without any allocation.  The paper has no
 * counterpart to this entry point; it exists for callers that must not
 * allocate device memory while they run -- for example a latency-bound
 * dispatcher (an allocation can take driver locks or wait for the device),
 * a process whose device memory is reserved up front by another allocator,
 * or code that has no way to recover from a failed allocation.
 *
 * dgs_evaluate_static computes exactly what dgs_evaluate computes (same
 * arguments, same outputs) but keeps all of its working memory in one fixed
 * array compiled into the library, about 0.3 MB per GPU, which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocator.  The caller still provides benefit, sigma_in
 * and the four output arrays.
 *
 * Limits: 1 <= n <= DGS_STATIC_MAX_N, n a multiple of 4, benefit 16-byte
 * aligned; otherwise DGS_ERR_INVALID, with the reason in
 * dgs_last_cuda_error().  Results and status codes are those of
 * dgs_evaluate, also on errors (after DGS_ERR_RANGE or DGS_ERR_INVALID from a
 * repeated job in sigma_in every output slot reads gain 0, index -1).
 *
 * The array belongs to the library's device code, which the CUDA runtime
 * loads on a device lazily by default: the first call on each device may be
 * the moment the array is committed, and can then fail with DGS_ERR_CUDA for
 * lack of device memory.  Callers that must not allocate later make one call
 * on each device during their set-up (or set CUDA_MODULE_LOADING=EAGER, which
 * commits it when the context is created).  All calls share the one array and
 * each call clears the parts it needs zeroed; calls that overlap on the GPU
 * (other streams or host threads) race on it and must be serialised by the
 * caller.  Each call synchronises its stream before it returns (the outputs
 * are final then), so it must not be called on a stream that is being
 * captured into a CUDA graph. */
#define DGS_STATIC_MAX_N 8192
DGS_API dgs_status dgs_evaluate_static(const int32_t* benefit, int32_t n, const int32_t* sigma_in,
                                       int32_t* agent_gain, int32_t* agent_job,
                                       int32_t* job_gain, int32_t* job_agent,
                                       dgs_stream_t stream);

/* ------------------------------------------------------------------------
 * Measurement.
 *
 * dgs_read_bandwidth: the rate, in GB/s (1e9 bytes per second), at which the
 * GPU's SMs read `bytes` bytes at `buffer` (DEVICE, 16-byte aligned, `bytes` a
 * multiple of 16), averaged over `repeats` back-to-back reads of the whole
 * buffer after one untimed read; a buffer smaller than L2 is then read from
 * L2.  The roofline of a difference evaluation whose benefit matrix fits in L2
 * is this rate on the matrix itself.  Writes *gbs_out; nothing else is
 * written.  Blocks until the timed reads finish.  Errors: DGS_ERR_INVALID for
 * a null or unaligned buffer, zero or unaligned size, repeats < 1;
 * DGS_ERR_CUDA if a launch or the timing failed. */
DGS_API dgs_status dgs_read_bandwidth(const void* buffer, size_t bytes, int32_t repeats, double* gbs_out,
                                      dgs_stream_t stream);

/* ------------------------------------------------------------------------
 * Device memory.
 *
 * The calls that allocate per call (dgs_solve*, dgs_evaluate, dgs_greedy_init,
 * dgs_autotune, dgs_solve_batched, the server's per-request workspaces) take
 * their device memory from the library's own stream-ordered pool on the
 * current device, which keeps freed memory cached for the next call instead of
 * returning it to the device (back-to-back solves then reuse their workspace
 * instead of mapping it again).  dgs_release_cached_memory returns every
 * cached byte of those pools to the device; memory still in use by a call in
 * flight stays with it.  Errors: DGS_ERR_CUDA if a trim failed. */
DGS_API dgs_status dgs_release_cached_memory(void);

/* Human-readable name of a status code (static string). */
DGS_API const char* dgs_status_string(dgs_status status);

/* Text of the last CUDA error seen by this thread's calls (static buffer). */
DGS_API const char* dgs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DGS_H */
