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
 *   - objective_out: HOST pointer to one int64 (exact sum of benefits).
 *   - stream: a cudaStream_t (the library includes no CUDA header here and
 *     takes it as dgs_stream_t, the same pointer type).  Work is enqueued on
 *     it; every solve entry point BLOCKS until its result is final (it reads
 *     the device-side loop state), so outputs are valid on return.
 *   - The library allocates its own device workspace (about 4*n*n bytes for
 *     the transposed copy of a plus O(n)) with stream-ordered allocation and
 *     frees it before returning.  Allocation failure -> DGS_ERR_OOM.
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
    DGS_PENDING = 6,      /* reserved for asynchronous entry points */
    DGS_ERR_BUSY = 7,     /* reserved for admission control */
    DGS_ERR_INTERNAL = 8  /* a device-side consistency check failed */
} dgs_status;

typedef enum {
    DGS_INIT_GREEDY = 0,   /* global greedy start (Section 3.1, default) */
    DGS_INIT_IDENTITY = 2, /* agent i starts on job i */
    DGS_INIT_USER = 3      /* caller's permutation in dgs_options.init_sigma */
} dgs_init_mode;

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
    /* 1: time the first full difference evaluation and the greedy start with
     * CUDA events on the call's stream (dgs_stats.evaluation_ms, greedy_ms);
     * 0: no timing. */
    int32_t profile;
} dgs_options;

typedef struct {
    int32_t sweeps;           /* iterations of the switching loop (Alg. 3) */
    int32_t events;           /* sweeps that committed at least one exchange */
    int64_t swaps_applied;    /* committed 2-exchanges */
    int32_t greedy_rounds;    /* locally-dominant rounds of the greedy start */
    int32_t full_evaluations; /* full difference evaluations (all slots) */
    int32_t row_updates;      /* incremental re-evaluations (row tasks) */
    int64_t rows_recomputed;  /* rows re-evaluated by those row tasks */
    int64_t initial_objective;/* objective of the starting assignment */
    int64_t kernel_launches;  /* kernels this call launched */
    double evaluation_ms;     /* first full evaluation, when options.profile */
    double greedy_ms;         /* greedy start after pass 1, when options.profile */
    int64_t greedy_rescans;   /* rows of a (or its transpose) the greedy start rescanned */
} dgs_stats;

/* Fill *opt with the defaults (GREEDY start, no cap, no deadline, no trace). */
DGS_API void dgs_default_options(dgs_options* opt);

/* Solve one instance with default options (Algorithm 3 from a greedy start
 * to termination: no 2-exchange improves the result). */
DGS_API dgs_status dgs_solve(const int32_t* benefit, int32_t n, int32_t* sigma_out,
                     int64_t* objective_out, dgs_stream_t stream);

/* Solve with options; stats may be NULL. */
DGS_API dgs_status dgs_solve_ex(const int32_t* benefit, int32_t n, int32_t* sigma_out,
                        int64_t* objective_out, const dgs_options* options,
                        dgs_stats* stats, dgs_stream_t stream);

/* Same as dgs_solve_ex but every buffer is in HOST memory (pageable or
 * pinned): benefit (n*n int32), sigma_out (n int32).  The host->device copy
 * of benefit and the device->host copy of sigma_out are part of the call. */
DGS_API dgs_status dgs_solve_host(const int32_t* benefit_host, int32_t n,
                          int32_t* sigma_out_host, int64_t* objective_out,
                          const dgs_options* options, dgs_stats* stats,
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
 * dgs_last_cuda_error().  The first call on each device looks up the array's
 * device address, so make that first call before any stream capture.  All
 * calls share the one array and each call clears the parts it needs zeroed;
 * calls that overlap on the GPU (other streams or host threads) race on it and
 * must be serialised by the caller.  Blocks until the outputs are final. */
#define DGS_STATIC_MAX_N 8192
DGS_API dgs_status dgs_evaluate_static(const int32_t* benefit, int32_t n, const int32_t* sigma_in,
                                       int32_t* agent_gain, int32_t* agent_job,
                                       int32_t* job_gain, int32_t* job_agent,
                                       dgs_stream_t stream);

/* Human-readable name of a status code (static string). */
DGS_API const char* dgs_status_string(dgs_status status);

/* Text of the last CUDA error seen by this thread's calls (static buffer). */
DGS_API const char* dgs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DGS_H */
