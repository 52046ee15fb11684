// dgs_internal.cuh -- device-side state, key packing and PTX helpers shared
// by the DGS kernels (greedy start, difference evaluation, switching
// control).  Internal to the library; the public interface is include/dgs.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dgs.h"

namespace dgs {

// ----------------------------------------------------------------- limits
constexpr int32_t kMaxN = 1 << 17;           // index fields are 17 bits in places
constexpr int32_t kBenefitLimit = 1 << 29;   // |a| < 2^29 keeps gains exact in int32
constexpr uint32_t kSpinLimit = 1u << 26;    // bound on every device-side wait loop

// Stage of an instance in a batched or served solve (DeviceState::stage);
// every batched kernel acts only on the instances in the stage it serves.
enum : int32_t {
    kStageFree = 0,    // slot unused
    kStageNew = 1,     // workspace initialised, pass 1 (transpose, range check) next
    kStageGreedy = 2,  // locally-dominant greedy rounds
    kStageStart = 3,   // sigma, D, f from the start; first full evaluation
    kStageSwitch = 4,  // switching loop (Algorithm 3)
    kStageDone = 5     // finished; assignment written to the instance's output
};

// Loop status (DeviceState::status).
enum : int32_t { kRunning = 0, kDone = 1, kTimeout = 2, kError = 3 };
// Device-side error codes (DeviceState::error).
enum : int32_t { kErrNone = 0, kErrRange = 1, kErrUserInit = 2, kErrWaitTimeout = 3, kErrInternal = 4 };
// Controller entry phase.
enum : int32_t { kPhaseRefreshAll = 0, kPhaseQuiet = 1 };

// All scalar loop state of one solve, resident in device memory.
struct DeviceState {
    int32_t status;          // kRunning / kDone / kTimeout / kError
    int32_t error;           // kErr*
    int32_t phase;           // controller entry phase
    int32_t need_update;     // 1: the last sweep committed exchanges
    int32_t sweeps;          // switching sweeps done
    int32_t max_sweeps;      // <= 0: none
    int32_t events;          // sweeps with >= 1 committed exchange
    int32_t y_count;         // jobs whose holder changed in the last event sweep
    int32_t rescan_count;    // rows needing a full re-evaluation
    int32_t edge_count;      // live candidate slots in the edge list
    int32_t greedy_remaining;// unmatched agents during the greedy start
    int32_t greedy_rounds;
    int32_t full_evals;
    int32_t row_updates;
    int32_t trace_capacity;
    int32_t greedy_matched;  // the last match kernel matched >= 1 pair
    int32_t update_policy;   // 0: by cost, 1: always full evaluation, 2: always row tasks
    int32_t max_abs;         // max |a| (set by the passes that check the range)
    long long greedy_rescans;  // rows of a / at rescanned by the greedy start
    uint32_t bar_count;      // grid barrier of cooperative launches: arrivals
    uint32_t bar_gen;        //   and generation
    int32_t reeval_all;      // 1: every slot is re-evaluated after a switch (DGS_REEVAL_ALL)
    int32_t pad_state;
    int32_t stage;           // kStage* (batched and served solves only)
    int32_t init_mode;       // batched: DGS_INIT_* of the instance (from Instance::init_mode)
    int64_t f;               // current objective
    int64_t f_initial;
    int64_t swaps;           // committed exchanges
    int64_t rows_recomputed;
    uint64_t deadline_ns;    // %globaltimer deadline, 0: none
    int32_t* trace_accepted;
    int32_t* trace_applied;
    int64_t* trace_objective;
    int32_t loop_iterations; // iterations of the device-side loops (bounded)
    int32_t loop_launches;   // kernels those loops launched
    int32_t seq_inner;       // Algorithm 1: launches of the current pass's switching loop
    int32_t seq_passes;      // Algorithm 1: passes so far
    int64_t f_pass;          // Algorithm 1: objective at the start of the current pass
    int32_t da_next;         // greedy start (deferred acceptance): next agent to take
    int32_t pad_state2;
};

// Pointers to every array of one solve (passed by value to kernels).
struct Workspace {
    const int32_t* a;   // benefit, row pitch lda (elements), lda % 4 == 0, 16-B aligned
    int32_t* at;        // transposed benefit, row pitch ldt, at[j*ldt + i] = a[i*lda + j]
    int32_t n, lda, ldt, pad;
    int32_t* sigma;     // job -> agent
    int32_t* tau;       // agent -> job
    int32_t* diag;      // D[j] = a[sigma[j]][j]
    unsigned long long* key_a;  // row best, agent-slot tie-break (lowest column)
    unsigned long long* key_j;  // row best, job-slot tie-break (lowest partner agent)
    int32_t* ag_gain; int32_t* ag_job;    // agent slot candidates
    int32_t* jb_gain; int32_t* jb_agent;  // job slot candidates
    uint8_t* in_ca; uint8_t* in_cj;       // conflict set C (reading R3: slots)
    uint8_t* in_y; uint8_t* moved;        // jobs changed / agents moved in the last event
    int32_t* y_list;                      // jobs changed in the last event
    int32_t* rescan_list;                 // rows to re-evaluate fully
    // per slot (agent slots 0..n-1, job slots n..2n-1): its edge word (0 when
    // it has no candidate) and its re-evaluated candidate (key, exchange agents)
    unsigned long long* sl_edge;
    int32_t* sl_chunk;  // edges among slots 32c .. 32c + 31 (written with sl_edge)
    unsigned long long* sl_rkey;
    int32_t* sl_ru;
    int32_t* sl_rv;
    int32_t* ctl_slot;  // controller: slot of each edge position (priority order)
    // greedy start
    unsigned long long* g_row;  // best free job per agent   (biased value, ~j)
    unsigned long long* g_col;  // round form: best free agent per job (biased value, ~i);
                                // deferred acceptance: the key (biased value, ~i) of the job's holder
    uint8_t* free_a; uint8_t* free_j;
    unsigned long long* g_list;  // deferred acceptance: per agent, 4 slots: the 2nd-4th jobs of its last scan
    int32_t exact_keys;  // 1: never use the packed 32-bit keys (test knob)
    int32_t row_owner_eval;  // 1: full evaluations by row owners (A-transpose form)
    DeviceState* st;
    unsigned long long* phase_ns;  // optional phase timers (DGS_PHASE_TIMERS=1), else null
};

// Controller scratch in global memory (the parts that do not live in shared
// memory for this n; null otherwise) and its accepted list.
struct CtlGlobal {
    uint32_t* res;
    uint8_t* claimed;
    uint8_t* estate;
    void* edges;
    int32_t* acc;
};

// One instance of a batched or served solve, as the batched kernels see it.
struct Instance {
    Workspace w;
    CtlGlobal ctl;
    int32_t ctl_mode;          // controller scratch placement for this n
    int32_t ctl_cap;           // entries of the controller's accepted list in shared memory
    int32_t fresh;             // 1: the next step initialises this instance
    int32_t max_sweeps;        // options of the instance
    int32_t init_mode;         // DGS_INIT_GREEDY / _IDENTITY / _USER (a random start arrives as USER)
    int32_t reeval_all;        // DGS_REEVAL_ALL
    int64_t deadline_us;
    const int32_t* a_src;      // caller's matrix when w.a is a re-pitched copy, else null
    const int32_t* user_tau;   // DGS_INIT_USER start
    int32_t* sigma_out;        // where the finished assignment goes (device)
    char* zero_begin;          // small arrays to clear at initialisation
    size_t zero_bytes;
    uint8_t* seen;             // start validation flags
};

// One entry of a batched work table: block bid of the nblk blocks that one
// launch gives to instance inst.  Each CTA of a persistent batched launch
// walks the entries blockIdx.x, blockIdx.x + gridDim.x, ...
struct BatchEntry {
    int32_t inst, bid, nblk, pad;
};
struct BatchTable {
    const Instance* inst;
    const BatchEntry* e;
    const int32_t* count;  // device: number of entries
};

// Walk this CTA's entries of a batched table, calling f(instance, bid, nblk)
// for the entries whose instance is in `stage` (stage < 0: every instance
// not free).  The stage is written only by the advance kernel, never during
// another batched launch, so the test is uniform across the CTA.
template <typename F>
__device__ __forceinline__ void for_each_entry(const BatchTable& t, int32_t stage, F&& f) {
    const int32_t count = *t.count;
    for (int32_t g = blockIdx.x; g < count; g += gridDim.x) {
        const BatchEntry e = t.e[g];
        const Instance& in = t.inst[e.inst];
        const int32_t sg = in.w.st->stage;
        if (stage >= 0 ? sg != stage : sg == 0) continue;
        f(in, e.bid, e.nblk);
    }
}

// Work queue of one batched launch: off[k] = first item of slot k, off[cap] =
// total (exclusive prefix of the per-slot item counts, written by the scan
// kernel just before the consumer).  CTA b takes the contiguous items
// [b * per, (b + 1) * per) and calls f(instance, local item, items of that
// slot) for each, the whole CTA together.
template <typename F>
__device__ __forceinline__ void for_each_item(const Instance* inst, const int32_t* off, int32_t cap, F&& f) {
    const int32_t total = off[cap];
    if (total <= 0) return;
    const int32_t per = (total + (int32_t)gridDim.x - 1) / (int32_t)gridDim.x;
    int32_t item = (int32_t)blockIdx.x * per;
    const int32_t end = min(total, item + per);
    if (item >= end) return;
    int32_t lo = 0, hi = cap;  // off[lo] <= item < off[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (off[mid] <= item) lo = mid;
        else hi = mid;
    }
    int32_t k = lo, first = off[k], next = off[k + 1];
    for (; item < end; ++item) {
        while (item >= next) {
            ++k;
            first = next;
            next = off[k + 1];
        }
        f(inst[k], item - first, next - first);
    }
}

// Blocks (work items) of the batched pass 1 and evaluation of an instance of
// size n.  Only the scan kernel uses them; any count is correct (items are
// spread over whatever grid consumes the queue), the caps only bound how
// finely one instance is split.
constexpr int32_t kBatchPass1MaxBlocks = 1216;
constexpr int32_t kBatchEvalMaxBlocks = 152;
__host__ __device__ __forceinline__ int32_t batch_blocks_pass1(int32_t n) {
    const int32_t t = (n + 63) / 64;
    const int32_t b = (t * t + 3) / 4;
    return b < 1 ? 1 : (b > kBatchPass1MaxBlocks ? kBatchPass1MaxBlocks : b);
}
__host__ __device__ __forceinline__ int32_t batch_blocks_eval(int32_t n, int32_t strip) {
    const int32_t nb = (n + 63) / 64, chunks = (nb + strip - 1) / strip;
    const int32_t b = (nb * chunks + 1) / 2;
    return b < 1 ? 1 : (b > kBatchEvalMaxBlocks ? kBatchEvalMaxBlocks : b);
}

// Phases whose work counts the scan kernel computes.
enum : int32_t { kScanPass1 = 0, kScanGreedyDA = 1, kScanStart = 2, kScanSwitch = 3 };

// Phase timer slots.
enum : int32_t {
    kPtDaLastNs = 0, kPtDaSumNs, kPtDaChain, kPtDaGroupScans, kPtCtlLiveSum, kPtCtlListSum, kPtCtlAccSum,
    kPtCtlEntry, kPtCtlTop, kPtCtlPass1, kPtCtlPost, kPtCtlEvent, kPtCtlSweeps, kPtCtlColour, kPtCtlColourPasses,
    kPtCtlColourRounds, kPtCtlColourIters, kPtCtlColourTail, kPtCount
};

// ------------------------------------------------------------- key packing
// A candidate (gain > 0, index) packs into 64 bits so that unsigned max picks
// the larger gain and, among equal gains, the LOWER index.
__device__ __forceinline__ unsigned long long pack_gain(int32_t gain, uint32_t idx) {
    return ((unsigned long long)(uint32_t)gain << 32) | (unsigned long long)(~idx);
}
__device__ __forceinline__ int32_t key_gain(unsigned long long k) { return (int32_t)(k >> 32); }
__device__ __forceinline__ int32_t key_index(unsigned long long k) { return (int32_t)(~(uint32_t)k); }

// Greedy order key: larger benefit first, then lower index.  Benefits are
// biased by 2^29 into [1, 2^30) so that the key is never 0 (0 = "none").
__device__ __forceinline__ unsigned long long pack_benefit(int32_t a, uint32_t idx) {
    return ((unsigned long long)(uint32_t)(a + kBenefitLimit) << 32) | (unsigned long long)(~idx);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long x, unsigned long long y) {
    return x > y ? x : y;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------ mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: returns false when the spin limit is reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// 1-D bulk copy global -> shared (TMA engine), completion on an mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Grid-wide barrier for cooperative launches (every CTA co-resident).  The
// wait is bounded in time; returns false (block-uniform) on timeout.
constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;
__device__ __forceinline__ bool grid_barrier(DeviceState* st) {
    __shared__ int32_t s_bar_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&st->bar_gen) : "memory");
        uint32_t prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&st->bar_count) : "memory");
        int32_t ok = 1;
        if (prev == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&st->bar_count) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&st->bar_gen) : "memory");
        } else {
            const uint64_t t0 = globaltimer_ns();
            for (;;) {
                uint32_t cur;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&st->bar_gen) : "memory");
                if (cur != g) break;
                if (globaltimer_ns() - t0 > kBarrierTimeoutNs) { ok = 0; break; }
                __nanosleep(20);
            }
        }
        s_bar_ok = ok;
    }
    __syncthreads();
    return s_bar_ok != 0;
}

// ------------------------------------------------------ host-side launchers
// Each returns the launch error (cudaSuccess on success).
cudaError_t launch_greedy_pass1(const Workspace& w, cudaStream_t s);
cudaError_t launch_greedy_round(const Workspace& w, cudaStream_t s);
// The greedy start by deferred acceptance (pass 1 must have run without
// column keys, g_col zero); then the assignment is read off the jobs'
// holders.  Returns an error (nothing launched) when the launch is refused
// or DGS_GREEDY_ROUNDS=1; the caller then runs pass 1 with column keys and
// the locally-dominant rounds (launch_greedy_round).
cudaError_t launch_greedy_da(const Workspace& w, cudaStream_t s);
// Pass 1 with (cols = 1) or without (cols = 0) the column keys g_col that the
// locally-dominant rounds need.
cudaError_t launch_greedy_pass1_cols(const Workspace& w, int32_t cols, cudaStream_t s);
cudaError_t launch_range_check(const Workspace& w, cudaStream_t s);
cudaError_t launch_start_from_tau(const Workspace& w, const int32_t* user_tau, int32_t mode, uint8_t* seen,
                                  cudaStream_t s);
cudaError_t launch_full_evaluation(const Workspace& w, int32_t conditional, cudaStream_t s);
// Launch shape of the full evaluation (rows per thread 4 or 8; strip: column
// tiles per work item, 0 = one contiguous balanced range of tiles per CTA;
// tma: X tiles by TMA gathers).
struct EvalShape {
    int32_t rows, strip;
    int32_t tma;  // 1: X tiles by TMA gathers (cp.async.bulk.tensor tile::gather4)
};
EvalShape evaluation_shape(int32_t n);
void set_evaluation_shape(int32_t n, EvalShape shape);
int32_t size_bucket(int32_t n);
cudaError_t launch_full_evaluation_shape(const Workspace& w, int32_t conditional, EvalShape shape, cudaStream_t s);
cudaError_t launch_keys_to_slots(const Workspace& w, int32_t* ag, int32_t* aj, int32_t* jg, int32_t* ja,
                                 cudaStream_t s);
// handle != 0: the controller ends each launch by setting that loop
// condition (1 while the loop state is running) and counts the iteration.
cudaError_t launch_controller_impl(const Workspace& w, const CtlGlobal& g, cudaStream_t s,
                                   unsigned long long handle = 0);
int32_t controller_list_cap(int32_t n, int32_t mode);
// The switching loop in one CTA for small n (see small_loop_kernel), and
// whether a solve of this workspace takes it.
bool use_small_loop(const Workspace& w);
cudaError_t launch_small_loop(const Workspace& w, const CtlGlobal& g, cudaStream_t s);
int32_t controller_smem_mode(int32_t n);
size_t controller_smem_bytes(int32_t n);
size_t full_evaluation_smem_bytes();
int32_t evaluation_strip();
cudaError_t launch_mark_rescan(const Workspace& w, cudaStream_t s);
cudaError_t launch_prepare_edges(const Workspace& w, cudaStream_t s);
cudaError_t launch_row_tasks(const Workspace& w, cudaStream_t s);
cudaError_t launch_row_owner_evaluation(const Workspace& w, int32_t conditional, cudaStream_t s);
cudaError_t launch_finish(const Workspace& w, int32_t* sigma_out, cudaStream_t s);
// The outputs of a solve: sigma_out (every entry -1 after an error), and,
// where not null, the objective and the final dgs_status code (device-
// writable pointers).
cudaError_t launch_finish_outputs(const Workspace& w, int32_t* sigma_out, int64_t* objective, int32_t* status,
                                  cudaStream_t s);
// Loop conditions of the device-side loops (see enqueue_while): the greedy
// rounds' loop (while agents are unmatched), and Algorithm 1's switching loop
// and passes.
cudaError_t launch_greedy_loop_cond(const Workspace& w, unsigned long long handle, cudaStream_t s);
cudaError_t launch_seq_pass_begin(const Workspace& w, unsigned long long inner, cudaStream_t s);
cudaError_t launch_seq_inner_cond(const Workspace& w, unsigned long long inner, cudaStream_t s);
cudaError_t launch_seq_pass_end(const Workspace& w, unsigned long long outer, cudaStream_t s);
// Algorithm 1: slots of a fresh evaluation (from the keys, left as they are),
// and one launch of the single-CTA switching loop (need_update = 1 when the
// launch stopped at its iteration budget before the loop ended).
cudaError_t launch_slots_from_keys(const Workspace& w, cudaStream_t s);
cudaError_t launch_sequential(const Workspace& w, cudaStream_t s);

size_t carve_instance(char* base, int32_t n, bool need_copy, Instance* in);
// One stream-ordered single solve (dgs_solve_ex) for the server's large
// requests; *final_status gets the outcome when the stream reaches it.
dgs_status solve_for_server(const int32_t* benefit, int32_t n, int32_t* sigma_out, int64_t* objective_out,
                            const dgs_options* opt, dgs_stats* stats, cudaStream_t stream, dgs_status* final_status);
// The random start of DGS_INIT_RANDOM (splitmix64 + Fisher-Yates) on the host.
void random_start(int32_t n, uint64_t seed, int32_t* tau);

// Batched launches (one persistent grid each; every kernel acts only on the
// table's instances that are in `stage`).  The tables are described at each
// launcher's definition.
// Queues: q0 / q1 are the two offset arrays (cap + 1 entries) written by
// launch_b_scan for the phase; the consumer launches read them.
struct BatchQueues {
    const Instance* inst;
    int32_t cap;
    int32_t* q0;
    int32_t* q1;
};
cudaError_t launch_b_scan(const BatchQueues& q, int32_t phase, int32_t strip, cudaStream_t s);
cudaError_t launch_b_init(const BatchTable& rows, cudaStream_t s);
cudaError_t launch_b_pass1(const BatchQueues& q, cudaStream_t s);
cudaError_t launch_b_greedy(const BatchTable& rows, const BatchQueues& q, cudaStream_t s);
cudaError_t launch_b_start(const BatchTable& rows, cudaStream_t s);
cudaError_t launch_b_evaluation(const BatchQueues& q, int32_t strip, cudaStream_t s);
cudaError_t launch_b_mark_rescan(const BatchTable& rows, cudaStream_t s);
cudaError_t launch_b_row_tasks(const BatchQueues& q, int32_t max_n, cudaStream_t s);
cudaError_t launch_b_prepare_edges(const BatchTable& rows, cudaStream_t s);
cudaError_t launch_b_controller(const BatchTable& one, cudaStream_t s);
cudaError_t launch_b_finish(const BatchTable& rows, cudaStream_t s);
cudaError_t launch_b_advance(const BatchTable& one, int32_t from_stage, cudaStream_t s);

// ------------------------------------------------------ device-side loops
// Enqueue on stream s a CUDA graph whose one node is a conditional WHILE
// loop; `body` enqueues the loop body on the capture stream it is given and
// passes `handle` to the kernel that decides, at the end of each iteration,
// whether the loop goes on (cudaGraphSetConditional; the condition is 1 when
// the body first runs).  The graph is released as soon as it is launched (an
// executable graph in flight is freed when it completes): the call only
// enqueues work.  `nested` bodies may themselves call capture_while on their
// capture stream to add an inner loop; such a loop's condition is set to 1
// at the start of the graph's launch only, so a body that runs an inner loop
// re-arms it itself: it creates the inner handle first (create_loop_handle on
// its capture stream), sets it from a kernel, and passes it to capture_while.
using LoopBody = dgs_status (*)(void* ctx, cudaStream_t capture, unsigned long long handle);
dgs_status enqueue_while(cudaStream_t s, LoopBody body, void* ctx);
// The same, reusing an executable graph captured earlier on this device with
// the same body and the same `key` bytes (which must cover every value the
// body's launches are captured with); up to 16 are kept.
dgs_status enqueue_while_cached(cudaStream_t s, LoopBody body, void* ctx, const void* key, size_t key_bytes);
dgs_status create_loop_handle(cudaStream_t capturing, unsigned long long* handle);
dgs_status capture_while(cudaStream_t capturing, LoopBody body, void* ctx, unsigned long long handle = 0);
// Pinned host staging blocks from a process-wide cache (never freed while the
// process runs; pinned_put may be called from a stream callback).
void* pinned_get(size_t bytes);
void pinned_put(void* p, size_t bytes);

// Where a result pointer lives: device-writable (device, managed or mapped
// pinned host memory; *alias = the address kernels use) or plain host memory
// (written by a host callback when the stream reaches it).
bool device_writable(const void* p, void** alias);

// Streaming multiprocessors of the current device (queried once per device;
// grids of the persistent and grid-stride kernels are multiples of it).
int32_t device_sms();

// Raise a kernel's dynamic shared memory limit once per device (slot = one
// small integer per kernel).
inline cudaError_t ensure_smem_limit(const void* func, int slot, size_t bytes) {
    static int done[16][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || slot < 0 || slot >= 16) return cudaErrorInvalidValue;
    if (done[slot][dev] >= (int)bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[slot][dev] = (int)bytes;
    return e;
}

// Decision rule shared by the conditional update kernels: re-evaluate all
// rows with the tile-pair sweep when the row tasks would touch more bytes
// (policy 1 / 2 force one path; both give identical keys).
__host__ __device__ __forceinline__ bool use_full_update(int32_t rescans, int32_t n, int32_t policy) {
    if (policy == 1) return true;
    if (policy == 2) return false;
    return (int64_t)rescans * 2 > (int64_t)n;
}

// Test knobs read from the environment once: DGS_UPDATE_POLICY (0/1/2) and
// DGS_CTL_MODE (cap on the controller's shared-memory placement, 0..2).
int32_t env_update_policy();
// Store the text returned by dgs_last_cuda_error() for this thread.
void set_last_error(const char* msg);
// The public status of a finished call for its device loop state (kDone: OK,
// kTimeout: DGS_TIMEOUT, kError: by the device error code; an unknown code is
// DGS_ERR_INTERNAL with its number in dgs_last_cuda_error()).
dgs_status map_device_status(const DeviceState& h);
int32_t env_controller_mode_cap();
// DGS_SHORT_WRAPS=1 shortens the controller's key and stamp periods so that
// tests reach their wrap-around paths.
int32_t env_short_wraps();
int32_t env_phase_timers();
// Stream-ordered allocation from the library's own memory pool on the current
// device.  The pool keeps memory freed by cudaFreeAsync cached for the next
// call (no release threshold); dgs_release_cached_memory returns it.
cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s);
// DGS_CTL_COMPACT_MIN: shortest edge list the controller compacts (default
// 2048; tests lower it so that compaction runs on small instances).
int32_t env_compact_min();
int32_t env_colour_pass();
int32_t small_loop_threads();
// DGS_EXACT_KEYS=1 disables the packed 32-bit keys of the evaluation kernel.
int32_t env_exact_keys();

}  // namespace dgs
