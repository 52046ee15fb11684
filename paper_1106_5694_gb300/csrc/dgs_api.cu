// dgs_api.cu -- the C ABI of include/dgs.h: argument checks, workspace,
// and the host loop that enqueues the kernels of one solve.
//
// Solve flow (Algorithm 3, Section 5, plus the greedy start of Section 3.1):
//   pass 1        transpose a -> at, |a| < 2^29 check, first greedy round keys
//   greedy rounds match mutually-best pairs, rescan rows/columns (device loop,
//                 checked from the host every few rounds)
//   start         sigma, D, f from the starting tau
//   evaluation    full difference evaluation (every slot)
//   switching     controller (quiet sweeps on one CTA) ->
//                 [mark rescan rows -> full evaluation | row tasks] -> controller ...
// The host reads the 100-byte loop state every few launches to learn when the
// loop has ended; everything else stays on the device.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <vector>

#include "../../include/dgs.h"
#include "dgs_internal.cuh"


namespace dgs {
int32_t env_update_policy() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_UPDATE_POLICY");
        const int32_t x = e ? std::atoi(e) : 0;
        return (x >= 0 && x <= 2) ? x : 0;
    }();
    return v;
}
int32_t env_exact_keys() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_EXACT_KEYS");
        return (e && std::atoi(e) == 1) ? 1 : 0;
    }();
    return v;
}
int32_t env_phase_timers() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_PHASE_TIMERS");
        return (e && std::atoi(e) == 1) ? 1 : 0;
    }();
    return v;
}
// One pool per device, created on first use.  Back-to-back solves free and
// allocate workspaces of the same size; with the default pool (release
// threshold 0) the memory is unmapped at every synchronisation and mapped
// again by the next call, which cost about 0.5 ms per n = 10000 solve.
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[64] = {};

cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        if (g_pools[dev] == nullptr) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t created = nullptr;
            e = cudaMemPoolCreate(&created, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(created);
                return e;
            }
            g_pools[dev] = created;
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

int32_t env_compact_min() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_CTL_COMPACT_MIN");
        const int32_t x = e ? std::atoi(e) : 2048;
        return x >= 1 ? x : 2048;
    }();
    return v;
}
int32_t env_short_wraps() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_SHORT_WRAPS");
        return (e && std::atoi(e) == 1) ? 1 : 0;
    }();
    return v;
}
int32_t env_controller_mode_cap() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_CTL_MODE");
        const int32_t x = e ? std::atoi(e) : 2;
        return (x >= 0 && x <= 2) ? x : 2;
    }();
    return v;
}
}  // namespace dgs

namespace {
thread_local char g_last_error[512] = "";
}  // namespace

namespace dgs {
void set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace dgs

namespace {

using namespace dgs;

dgs_status cuda_fail(cudaError_t e, const char* what) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    return DGS_ERR_CUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One stream-ordered allocation carved into every array of a solve.
struct Arena {
    char* base = nullptr;
    size_t size = 0, used = 0;
    template <typename T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base + used);
        used += align_up(count * sizeof(T), 256);
        return p;
    }
};

struct Plan {
    bool need_copy = false;   // a must be re-laid out (n % 4 != 0 or misaligned)
    bool need_at = true;      // transposed copy (greedy start, row tasks)
    int32_t lda = 0, ldt = 0;
    size_t bytes = 0;
};

int32_t round_up32(int32_t x, int32_t m) { return (x + m - 1) / m * m; }

// Carve the workspace; sizes first (base == nullptr), then pointers.
size_t carve(Arena& ar, Workspace& w, const Plan& p, int32_t n, CtlGlobal* ctl, uint8_t** seen,
             int32_t** a_copy) {
    const size_t nb = align_up((size_t)n, 128);
    *a_copy = p.need_copy ? ar.take<int32_t>((size_t)n * p.lda) : nullptr;
    w.at = p.need_at ? ar.take<int32_t>((size_t)n * p.ldt + 64) : nullptr;
    w.sigma = ar.take<int32_t>(nb);
    w.tau = ar.take<int32_t>(nb);
    w.diag = ar.take<int32_t>(nb);
    w.key_a = ar.take<unsigned long long>(nb);
    w.key_j = ar.take<unsigned long long>(nb);
    w.ag_gain = ar.take<int32_t>(nb);
    w.ag_job = ar.take<int32_t>(nb);
    w.jb_gain = ar.take<int32_t>(nb);
    w.jb_agent = ar.take<int32_t>(nb);
    w.in_ca = ar.take<uint8_t>(nb);
    w.in_cj = ar.take<uint8_t>(nb);
    w.in_y = ar.take<uint8_t>(nb);
    w.moved = ar.take<uint8_t>(nb);
    w.y_list = ar.take<int32_t>(nb);
    w.rescan_list = ar.take<int32_t>(nb);
    w.sl_edge = ar.take<unsigned long long>(2 * nb);
    w.sl_rkey = ar.take<unsigned long long>(2 * nb);
    w.sl_ru = ar.take<int32_t>(2 * nb);
    w.sl_rv = ar.take<int32_t>(2 * nb);
    w.ctl_slot = ar.take<int32_t>(2 * nb);
    w.g_row = ar.take<unsigned long long>(nb);
    w.g_col = ar.take<unsigned long long>(nb);
    w.free_a = ar.take<uint8_t>(nb);
    w.free_j = ar.take<uint8_t>(nb);
    w.g_free_a = ar.take<uint32_t>(nb / 32);
    w.g_free_j = ar.take<uint32_t>(nb / 32);
    w.g_dirty = ar.take<uint32_t>(2 * nb / 32);
    w.phase_ns = env_phase_timers() ? ar.take<unsigned long long>(kPtCount) : nullptr;
    w.st = ar.take<DeviceState>(1);
    *seen = ar.take<uint8_t>(4 * nb);
    const int32_t mode = controller_smem_mode(n);
    ctl->edges = mode < 2 ? static_cast<void*>(ar.take<unsigned long long>(2 * nb)) : nullptr;
    ctl->res = mode < 1 ? ar.take<uint32_t>(nb) : nullptr;
    ctl->claimed = mode < 1 ? ar.take<uint8_t>(nb) : nullptr;
    ctl->estate = mode < 1 ? ar.take<uint8_t>(2 * nb) : nullptr;
    ctl->acc = ar.take<int32_t>(2 * nb);
    return ar.used;
}

}  // namespace

namespace dgs {
// DGS_INIT_RANDOM: the identity shuffled by Fisher-Yates in Durstenfeld's
// form (for i = n-1 .. 1, swap i with next() mod (i + 1)), next() being
// splitmix64 (Steele, Lea, Flood 2014) started at seed.
void random_start(int32_t n, uint64_t seed, int32_t* tau) {
    uint64_t state = seed;
    auto next = [&state]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int32_t i = 0; i < n; ++i) tau[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        const int32_t j = (int32_t)(next() % (uint64_t)(i + 1));
        std::swap(tau[i], tau[j]);
    }
}

// Workspace of one batched or served instance inside a caller-provided block
// (base == nullptr: only the size).  need_copy: w.a is a re-pitched copy in
// the block (pitch round_up(n, 4)); otherwise the caller sets w.a.
size_t carve_instance(char* base, int32_t n, bool need_copy, Instance* in) {
    Plan p;
    p.need_copy = need_copy;
    p.need_at = true;
    p.lda = need_copy ? round_up32(n, 4) : n;
    p.ldt = round_up32(n, 64);
    Arena ar;
    ar.base = base;
    Workspace w{};
    CtlGlobal ctl{};
    uint8_t* seen = nullptr;
    int32_t* a_copy = nullptr;
    const size_t bytes = carve(ar, w, p, n, &ctl, &seen, &a_copy);
    if (base == nullptr) return bytes;
    w.n = n;
    w.lda = p.lda;
    w.ldt = p.ldt;
    w.exact_keys = env_exact_keys();
    w.a = a_copy;
    const int32_t mode = controller_smem_mode(n);
    in->w = w;
    in->ctl = ctl;
    in->seen = seen;
    in->ctl_mode = mode;
    in->ctl_cap = controller_list_cap(n, mode);
    in->zero_begin = reinterpret_cast<char*>(w.sigma);
    in->zero_bytes = (size_t)(base + bytes - in->zero_begin);
    return bytes;
}
}  // namespace dgs

namespace {
using namespace dgs;

// Everything one call needs, released in the destructor (stream-ordered).
struct Solve {
    cudaStream_t s;
    Arena ar;
    Workspace w{};
    Plan plan;
    int32_t* a_copy = nullptr;
    CtlGlobal ctl{};
    uint8_t* seen = nullptr;
    int64_t launches = 0;
    explicit Solve(cudaStream_t st) : s(st) {}
    ~Solve() {
        if (ar.base) cudaFreeAsync(ar.base, s);
    }

    // pitched_lda > 0: a is already laid out with that pitch (used in place).
    dgs_status setup(const int32_t* a, int32_t n, bool need_at, int32_t pitched_lda = 0) {
        plan.need_at = need_at;
        plan.need_copy = pitched_lda > 0 ? false : ((n % 4) != 0 || (reinterpret_cast<uintptr_t>(a) % 16) != 0);
        plan.lda = pitched_lda > 0 ? pitched_lda : (plan.need_copy ? round_up32(n, 4) : n);
        plan.ldt = round_up32(n, 64);
        Arena sizing;
        Workspace tmp{};
        carve(sizing, tmp, plan, n, &ctl, &seen, &a_copy);
        plan.bytes = sizing.used;
        cudaError_t e = pool_malloc_async(reinterpret_cast<void**>(&ar.base), plan.bytes, s);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            snprintf(g_last_error, sizeof(g_last_error), "workspace of %zu bytes", plan.bytes);
            ar.base = nullptr;
            return DGS_ERR_OOM;
        }
        if (e != cudaSuccess) return cuda_fail(e, "device allocation");
        ar.size = plan.bytes;
        carve(ar, w, plan, n, &ctl, &seen, &a_copy);
        w.n = n;
        w.lda = plan.lda;
        w.ldt = plan.ldt;
        w.exact_keys = env_exact_keys();
        if (plan.need_copy) {
            e = cudaMemsetAsync(a_copy, 0, (size_t)n * plan.lda * sizeof(int32_t), s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
            e = cudaMemcpy2DAsync(a_copy, (size_t)plan.lda * 4, a, (size_t)n * 4, (size_t)n * 4, n,
                                  cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync");
            w.a = a_copy;
        } else {
            w.a = a;
        }
        // zero every small array in one go (they follow a/at in the arena)
        char* small_begin = reinterpret_cast<char*>(w.sigma);
        const size_t small_bytes = (size_t)(ar.base + ar.used - small_begin);
        e = cudaMemsetAsync(small_begin, 0, small_bytes, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        const size_t nb = align_up((size_t)n, 128);
        e = cudaMemsetAsync(w.free_a, 1, nb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.free_j, 1, nb, s);
        // bitmaps: bits of agents/jobs >= n are never read
        if (e == cudaSuccess) e = cudaMemsetAsync(w.g_free_a, 0xFF, nb / 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.g_free_j, 0xFF, nb / 8, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        return DGS_OK;
    }

    // Workspace for a matrix already laid out with pitch lda (lda % 4 == 0,
    // 16-byte aligned), without the transposed copy.
    dgs_status setup_pitched(const int32_t* a, int32_t n, int32_t lda) { return setup(a, n, false, lda); }

    dgs_status init_state(int32_t max_sweeps, const dgs_options* o) {
        DeviceState h{};
        h.status = kRunning;
        h.phase = kPhaseRefreshAll;
        h.max_sweeps = max_sweeps;
        h.greedy_remaining = w.n;
        h.update_policy = env_update_policy();
        if (o) {
            h.reeval_all = o->reeval_rule == DGS_REEVAL_ALL ? 1 : 0;
            h.trace_capacity = o->trace_capacity > 0 ? o->trace_capacity : 0;
            h.trace_accepted = o->trace_accepted;
            h.trace_applied = o->trace_applied;
            h.trace_objective = o->trace_objective;
        }
        cudaError_t e = cudaMemcpyAsync(w.st, &h, sizeof(h), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(state)");
        return DGS_OK;
    }

    dgs_status read_state(DeviceState* h) {
        cudaError_t e = cudaMemcpyAsync(h, w.st, sizeof(*h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading loop state");
        return DGS_OK;
    }
};

// A stream-ordered device allocation released with the call.
struct DeviceBuffer {
    cudaStream_t s;
    void* p = nullptr;
    explicit DeviceBuffer(cudaStream_t st) : s(st) {}
    ~DeviceBuffer() {
        if (p) cudaFreeAsync(p, s);
    }
    dgs_status alloc(size_t bytes) {
        cudaError_t e = pool_malloc_async(&p, bytes, s);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            p = nullptr;
            return DGS_ERR_OOM;
        }
        return e == cudaSuccess ? DGS_OK : cuda_fail(e, "device allocation");
    }
};

// CUDA events around one launch on the call's stream (options.profile).
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    dgs_status begin(cudaStream_t s) {
        cudaError_t e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        if (e == cudaSuccess) e = cudaEventRecord(a, s);
        return e == cudaSuccess ? DGS_OK : cuda_fail(e, "profile event");
    }
    dgs_status end(cudaStream_t s) {
        cudaError_t e = cudaEventRecord(b, s);
        return e == cudaSuccess ? DGS_OK : cuda_fail(e, "profile event");
    }
    double elapsed_ms() const {
        float ms = 0.f;
        if (a && b && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) return ms;
        return 0.0;
    }
};

__global__ void arm_deadline_kernel(DeviceState* st, int64_t deadline_us) {
    uint64_t now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    st->deadline_ns = now + (uint64_t)deadline_us * 1000ull;
}

__global__ void record_initial_objective_kernel(DeviceState* st) { st->f_initial = st->f; }

// Rectangular instance -> square instance of size s (zero-benefit dummies).
__global__ void pad_square_kernel(const int32_t* a, int32_t n, int32_t m, int32_t s, int32_t* sq) {
    const size_t total = (size_t)s * s;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(q / s), j = (int32_t)(q - (size_t)i * s);
        sq[q] = (i < n && j < m) ? a[(size_t)i * m + j] : 0;
    }
}

// Jobs of the real agents; a dummy job means no job.
__global__ void trim_assignment_kernel(const int32_t* tau, int32_t n, int32_t m, int32_t* out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = tau[i] < m ? tau[i] : -1;
}

// Synthetic benefits for timing launch shapes: values in [0, 10016) from a
// per-element hash (the range of peer-shaped instances, so the packed-key
// path of the evaluation is the one timed).  Pitch lda, padding zero.
__global__ void fill_synthetic_kernel(int32_t* a, int32_t n, int32_t lda, uint64_t seed) {
    const size_t total = (size_t)n * lda;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + q * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        a[q] = (q % (size_t)lda) < (size_t)n ? (int32_t)(z % 10016u) : 0;
    }
}

dgs_status map_device_status(const DeviceState& h) {
    if (h.status == kDone) return DGS_OK;
    if (h.status == kTimeout) return DGS_TIMEOUT;
    if (h.status == kError) {
        if (h.error == kErrRange) return DGS_ERR_RANGE;
        if (h.error == kErrUserInit) return DGS_ERR_INVALID;
        snprintf(g_last_error, sizeof(g_last_error), "device-side error code %d", h.error);
        return DGS_ERR_INTERNAL;
    }
    return DGS_OK;
}

#define DGS_TRY(expr)                          \
    do {                                       \
        dgs_status _st = (expr);               \
        if (_st != DGS_OK) return _st;         \
    } while (0)
#define DGS_CUDA(expr, what)                               \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// Greedy rounds until every agent is matched (or an error).
dgs_status run_greedy(Solve& S, EventPair* timer) {
    DGS_CUDA(launch_greedy_pass1(S.w, S.s), "greedy pass 1");
    S.launches += 1;
    if (timer) DGS_TRY(timer->begin(S.s));
    const cudaError_t pe = launch_greedy_persistent(S.w, S.s);
    if (pe == cudaSuccess) {
        S.launches += 1;
        if (timer) DGS_TRY(timer->end(S.s));
        return DGS_OK;
    }
    // the cooperative launch was refused: one launch per kernel per round
    cudaGetLastError();
    const int32_t batch = 8;
    for (int32_t launched = 0; launched <= S.w.n + batch; launched += batch) {
        for (int32_t r = 0; r < batch; ++r) DGS_CUDA(launch_greedy_round(S.w, S.s), "greedy round");
        S.launches += 3 * batch;
        DeviceState h;
        DGS_TRY(S.read_state(&h));
        if (h.status != kRunning || h.greedy_remaining == 0) {
            if (timer) DGS_TRY(timer->end(S.s));
            return DGS_OK;
        }
    }
    snprintf(g_last_error, sizeof(g_last_error), "greedy start did not finish");
    return DGS_ERR_INTERNAL;
}

// Algorithm 1 after the start: passes of (fresh evaluation of every slot,
// switching loop on one CTA) until a pass leaves f unchanged.
dgs_status run_sequential(Solve& S, int32_t* sigma_out, int64_t* objective_out, const dgs_options& o,
                          dgs_stats* stats, EventPair& gev) {
    cudaStream_t stream = S.s;
    S.launches += 2;
    DeviceState h;
    const int64_t max_passes = 4 * (int64_t)S.w.n + 16;
    bool ended = false;
    for (int64_t pass = 0; pass < max_passes && !ended; ++pass) {
        DGS_TRY(S.read_state(&h));
        if (h.status != kRunning) break;
        const int64_t f_start = h.f;
        DGS_CUDA(launch_full_evaluation(S.w, 0, stream), "evaluation");
        DGS_CUDA(launch_slots_from_keys(S.w, stream), "slots");
        S.launches += 2;
        for (int64_t launch = 0;; ++launch) {
            DGS_CUDA(launch_sequential(S.w, stream), "switching loop");
            S.launches += 1;
            DGS_TRY(S.read_state(&h));
            if (h.status != kRunning || !h.need_update) break;
            if (launch > 64) {
                snprintf(g_last_error, sizeof(g_last_error), "switching loop did not finish");
                return DGS_ERR_INTERNAL;
            }
        }
        if (h.status != kRunning || h.f == f_start) ended = true;
    }
    if (!ended) {
        snprintf(g_last_error, sizeof(g_last_error), "sequential passes did not finish");
        return DGS_ERR_INTERNAL;
    }
    DGS_CUDA(launch_finish(S.w, sigma_out, stream), "finish");
    S.launches += 1;
    DGS_TRY(S.read_state(&h));
    const dgs_status status = h.status == kRunning ? DGS_OK : map_device_status(h);
    *objective_out = h.f;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->sweeps = h.sweeps;
        stats->events = h.events;
        stats->swaps_applied = h.swaps;
        stats->greedy_rounds = h.greedy_rounds;
        stats->initial_objective = h.f_initial;
        stats->kernel_launches = S.launches;
        stats->greedy_ms = (o.profile && o.init == DGS_INIT_GREEDY) ? gev.elapsed_ms() : 0.0;
        stats->greedy_rescans = h.greedy_rescans;
    }
    return status;
}

dgs_status check_common(const int32_t* benefit, int32_t n) {
    if (benefit == nullptr || n <= 0 || n > kMaxN) return DGS_ERR_INVALID;
    return DGS_OK;
}

dgs_status solve_impl(const int32_t* benefit, int32_t n, int32_t* sigma_out, int64_t* objective_out,
                      const dgs_options* opt, dgs_stats* stats, cudaStream_t stream) {
    DGS_TRY(check_common(benefit, n));
    if (sigma_out == nullptr || objective_out == nullptr) return DGS_ERR_INVALID;
    dgs_options o;
    dgs_default_options(&o);
    if (opt) o = *opt;
    if (o.init != DGS_INIT_GREEDY && o.init != DGS_INIT_RANDOM && o.init != DGS_INIT_IDENTITY &&
        o.init != DGS_INIT_USER)
        return DGS_ERR_INVALID;
    if (o.init == DGS_INIT_USER && o.init_sigma == nullptr) return DGS_ERR_INVALID;
    if (o.reeval_rule != DGS_REEVAL_BOX && o.reeval_rule != DGS_REEVAL_ALL) return DGS_ERR_INVALID;
    if (o.algorithm != DGS_ALG_PARALLEL && o.algorithm != DGS_ALG_SEQUENTIAL) return DGS_ERR_INVALID;
    if (o.evaluation != DGS_EVAL_TILE_PAIRS && o.evaluation != DGS_EVAL_ROW_OWNER) return DGS_ERR_INVALID;

    Solve S(stream);
    DGS_TRY(S.setup(benefit, n, true));
    S.w.row_owner_eval = o.evaluation == DGS_EVAL_ROW_OWNER ? 1 : 0;
    // the random start is drawn on the host and enters as the caller's start
    DeviceBuffer rnd(stream);
    if (o.init == DGS_INIT_RANDOM) {
        std::vector<int32_t> perm(n);
        random_start(n, o.seed, perm.data());
        DGS_TRY(rnd.alloc((size_t)n * sizeof(int32_t)));
        DGS_CUDA(cudaMemcpyAsync(rnd.p, perm.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, stream),
                 "copy random start");
        DGS_CUDA(cudaStreamSynchronize(stream), "copy random start");  // perm is released on return
        o.init = DGS_INIT_USER;
        o.init_sigma = static_cast<const int32_t*>(rnd.p);
    }
    DGS_TRY(S.init_state(o.max_sweeps, &o));
    if (o.deadline_us > 0) {
        arm_deadline_kernel<<<1, 1, 0, stream>>>(S.w.st, o.deadline_us);
        DGS_CUDA(cudaGetLastError(), "arm deadline");
        S.launches += 1;
    }
    EventPair gev;
    if (o.init == DGS_INIT_GREEDY) {
        DGS_TRY(run_greedy(S, o.profile ? &gev : nullptr));
    } else {
        DGS_CUDA(launch_greedy_pass1(S.w, stream), "pass 1");  // transpose + range check
        S.launches += 1;
    }
    DGS_CUDA(launch_start_from_tau(S.w, o.init_sigma, o.init, S.seen, stream), "start");
    record_initial_objective_kernel<<<1, 1, 0, stream>>>(S.w.st);
    if (o.algorithm == DGS_ALG_SEQUENTIAL) return run_sequential(S, sigma_out, objective_out, o, stats, gev);
    EventPair ev;
    if (o.profile) DGS_TRY(ev.begin(stream));
    DGS_CUDA(launch_full_evaluation(S.w, 0, stream), "evaluation");
    if (o.profile) DGS_TRY(ev.end(stream));
    DGS_CUDA(launch_prepare_edges(S.w, stream), "prepare");
    DGS_CUDA(launch_controller_impl(S.w, S.ctl, stream), "controller");
    S.launches += 5;
    DeviceState h;
    const int32_t batch = 4;
    const int64_t max_iterations = 16 * (int64_t)n + 4096;
    bool ended = false;
    for (int64_t it = 0; it < max_iterations; it += batch) {
        DGS_TRY(S.read_state(&h));
        if (h.status != kRunning) {
            ended = true;
            break;
        }
        for (int32_t b = 0; b < batch; ++b) {
            DGS_CUDA(launch_mark_rescan(S.w, stream), "mark");
            DGS_CUDA(launch_full_evaluation(S.w, 1, stream), "re-evaluation");
            DGS_CUDA(launch_row_tasks(S.w, stream), "row tasks");
            DGS_CUDA(launch_prepare_edges(S.w, stream), "prepare");
            DGS_CUDA(launch_controller_impl(S.w, S.ctl, stream), "controller");
            S.launches += 5;
        }
    }
    if (!ended) {
        snprintf(g_last_error, sizeof(g_last_error), "switching loop did not finish");
        return DGS_ERR_INTERNAL;
    }
    DGS_CUDA(launch_finish(S.w, sigma_out, stream), "finish");
    S.launches += 1;
    DGS_TRY(S.read_state(&h));
    if (S.w.phase_ns) {  // test/diagnostic output only
        unsigned long long ph[kPtCount];
        if (cudaMemcpy(ph, S.w.phase_ns, sizeof(ph), cudaMemcpyDeviceToHost) == cudaSuccess) {
            fprintf(stderr, "[dgs phases] greedy ns: match %llu bar1 %llu check %llu scan %llu bar2 %llu scanmax %llu | "
                            "controller cycles: entry %llu top %llu conflict check %llu post %llu event %llu sweeps %llu\n",
                    ph[0], ph[1], ph[2], ph[3], ph[4], ph[5], ph[8], ph[9], ph[10], ph[13], ph[14], ph[15]);
        }
    }
    const dgs_status status = map_device_status(h);
    *objective_out = h.f;
    if (stats) {
        stats->sweeps = h.sweeps;
        stats->events = h.events;
        stats->swaps_applied = h.swaps;
        stats->greedy_rounds = h.greedy_rounds;
        stats->full_evaluations = h.full_evals + 1;
        stats->row_updates = h.row_updates;
        stats->rows_recomputed = h.rows_recomputed;
        stats->initial_objective = h.f_initial;
        stats->kernel_launches = S.launches;
        stats->evaluation_ms = o.profile ? ev.elapsed_ms() : 0.0;
        stats->greedy_ms = (o.profile && o.init == DGS_INIT_GREEDY) ? gev.elapsed_ms() : 0.0;
        stats->greedy_rescans = h.greedy_rescans;
    }
    return status;
}

}  // namespace

extern "C" {

void dgs_default_options(dgs_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->init = DGS_INIT_GREEDY;
}

dgs_status dgs_solve(const int32_t* benefit, int32_t n, int32_t* sigma_out, int64_t* objective_out,
                     dgs_stream_t stream) {
    return solve_impl(benefit, n, sigma_out, objective_out, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

dgs_status dgs_solve_ex(const int32_t* benefit, int32_t n, int32_t* sigma_out, int64_t* objective_out,
                        const dgs_options* options, dgs_stats* stats, dgs_stream_t stream) {
    return solve_impl(benefit, n, sigma_out, objective_out, options, stats, reinterpret_cast<cudaStream_t>(stream));
}

dgs_status dgs_solve_host(const int32_t* benefit_host, int32_t n, int32_t* sigma_out_host, int64_t* objective_out,
                          const dgs_options* options, dgs_stats* stats, dgs_stream_t stream) {
    if (benefit_host == nullptr || sigma_out_host == nullptr || objective_out == nullptr || n <= 0 || n > kMaxN)
        return DGS_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t abytes = (size_t)n * n * sizeof(int32_t);
    const size_t obytes = align_up((size_t)n * sizeof(int32_t), 256);
    char* buf = nullptr;
    cudaError_t e = pool_malloc_async(reinterpret_cast<void**>(&buf), abytes + obytes, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return DGS_ERR_OOM;
    }
    if (e != cudaSuccess) return cuda_fail(e, "device allocation");
    int32_t* a_dev = reinterpret_cast<int32_t*>(buf + obytes);
    int32_t* out_dev = reinterpret_cast<int32_t*>(buf);
    dgs_status st = DGS_OK;
    e = cudaMemcpyAsync(a_dev, benefit_host, abytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "copy benefit to device");
    if (st == DGS_OK) st = solve_impl(a_dev, n, out_dev, objective_out, options, stats, s);
    if (st == DGS_OK || st == DGS_TIMEOUT) {
        e = cudaMemcpyAsync(sigma_out_host, out_dev, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy result to host");
    }
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    return st;
}

dgs_status dgs_solve_rect(const int32_t* benefit, int32_t n_agents, int32_t m_jobs, int32_t* assign_out,
                          int64_t* objective_out, const dgs_options* options, dgs_stats* stats, dgs_stream_t stream) {
    if (benefit == nullptr || assign_out == nullptr || objective_out == nullptr || n_agents <= 0 || m_jobs <= 0)
        return DGS_ERR_INVALID;
    const int32_t sz = n_agents > m_jobs ? n_agents : m_jobs;
    if (sz > kMaxN) return DGS_ERR_INVALID;
    dgs_options o;
    dgs_default_options(&o);
    if (options) o = *options;
    if (o.init == DGS_INIT_USER || o.trace_capacity > 0) return DGS_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceBuffer buf(s);
    const size_t sq_bytes = align_up((size_t)sz * sz * sizeof(int32_t), 256);
    DGS_TRY(buf.alloc(sq_bytes + (size_t)sz * sizeof(int32_t)));
    int32_t* sq = static_cast<int32_t*>(buf.p);
    int32_t* tau = reinterpret_cast<int32_t*>(static_cast<char*>(buf.p) + sq_bytes);
    pad_square_kernel<<<152 * 8, 256, 0, s>>>(benefit, n_agents, m_jobs, sz, sq);
    DGS_CUDA(cudaGetLastError(), "pad");
    const dgs_status st = solve_impl(sq, sz, tau, objective_out, &o, stats, s);
    if (st != DGS_OK && st != DGS_TIMEOUT) return st;
    trim_assignment_kernel<<<(n_agents + 255) / 256, 256, 0, s>>>(tau, n_agents, m_jobs, assign_out);
    DGS_CUDA(cudaGetLastError(), "trim");
    DGS_CUDA(cudaStreamSynchronize(s), "trim");
    if (stats) stats->kernel_launches += 2;
    return st;
}

dgs_status dgs_evaluate(const int32_t* benefit, int32_t n, const int32_t* sigma_in, int32_t* agent_gain,
                        int32_t* agent_job, int32_t* job_gain, int32_t* job_agent, dgs_stream_t stream) {
    DGS_TRY(check_common(benefit, n));
    if (!sigma_in || !agent_gain || !agent_job || !job_gain || !job_agent) return DGS_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Solve S(s);
    DGS_TRY(S.setup(benefit, n, false));
    DGS_TRY(S.init_state(0, nullptr));
    DGS_CUDA(launch_range_check(S.w, s), "range check");
    DGS_CUDA(launch_start_from_tau(S.w, sigma_in, DGS_INIT_USER, S.seen, s), "start");
    DGS_CUDA(launch_full_evaluation(S.w, 0, s), "evaluation");
    DGS_CUDA(launch_keys_to_slots(S.w, agent_gain, agent_job, job_gain, job_agent, s), "keys to slots");
    DeviceState h;
    DGS_TRY(S.read_state(&h));
    return map_device_status(h);
}

dgs_status dgs_greedy_init(const int32_t* benefit, int32_t n, int32_t* sigma_out, dgs_stream_t stream) {
    DGS_TRY(check_common(benefit, n));
    if (!sigma_out) return DGS_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Solve S(s);
    DGS_TRY(S.setup(benefit, n, true));
    DGS_TRY(S.init_state(0, nullptr));
    DGS_TRY(run_greedy(S, nullptr));
    DGS_CUDA(launch_finish(S.w, sigma_out, s), "finish");
    DeviceState h;
    DGS_TRY(S.read_state(&h));
    return map_device_status(h);
}

dgs_status dgs_autotune(int32_t n, dgs_tuning* result, dgs_stream_t stream) {
    if (n < 2 || n > kMaxN) return DGS_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int32_t lda = round_up32(n, 4);
    int32_t* buf = nullptr;
    const size_t abytes = (size_t)n * lda * sizeof(int32_t);
    cudaError_t e = pool_malloc_async(reinterpret_cast<void**>(&buf), abytes + align_up((size_t)n * 4, 256), s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return DGS_ERR_OOM;
    }
    if (e != cudaSuccess) return cuda_fail(e, "device allocation");
    int32_t* a = buf;
    int32_t* sigma = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(buf) + abytes);
    dgs_status st = DGS_OK;
    {
        Solve S(s);
        // a synthetic instance of this size with peer-like values, under a
        // random assignment (the evaluation's time does not depend on which)
        fill_synthetic_kernel<<<152 * 8, 256, 0, s>>>(a, n, lda, 0x9E3779B97F4A7C15ull ^ (uint64_t)n);
        std::vector<int32_t> perm(n);
        for (int32_t i = 0; i < n; ++i) perm[i] = i;
        uint64_t x = 0xD1B54A32D192ED03ull ^ (uint64_t)n;
        for (int32_t i = n - 1; i > 0; --i) {  // Fisher-Yates with splitmix64
            x += 0x9E3779B97F4A7C15ull;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            std::swap(perm[i], perm[z % (uint64_t)(i + 1)]);
        }
        e = cudaMemcpyAsync(sigma, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy assignment");
        if (st == DGS_OK) st = S.setup_pitched(a, n, lda);
        if (st == DGS_OK) st = S.init_state(0, nullptr);
        if (st == DGS_OK && (e = launch_range_check(S.w, s)) != cudaSuccess) st = cuda_fail(e, "range check");
        if (st == DGS_OK && (e = launch_start_from_tau(S.w, sigma, DGS_INIT_USER, S.seen, s)) != cudaSuccess)
            st = cuda_fail(e, "start");
        // candidate shapes: 8 and 16 rows per thread with every strip (0:
        // contiguous balanced ranges), 4 rows per thread with two strips, and
        // the TMA-gather variants of 8 and 4 rows with two strips and one
        std::vector<EvalShape> shapes;
        for (int32_t strip : {0, 4, 8, 16, 32, 64}) shapes.push_back(EvalShape{8, strip, 0});
        for (int32_t strip : {0, 8, 16, 32, 64}) shapes.push_back(EvalShape{16, strip, 0});
        for (int32_t strip : {0, 32}) shapes.push_back(EvalShape{4, strip, 0});
        for (int32_t strip : {0, 32}) shapes.push_back(EvalShape{8, strip, 1});
        shapes.push_back(EvalShape{4, 0, 1});
        dgs_tuning r{};
        r.best_ms = 1e30;
        EventPair ev;
        if (st == DGS_OK) st = ev.begin(s);
        for (size_t ci = 0; ci < shapes.size() && ci < DGS_TUNE_MAX_CANDIDATES && st == DGS_OK; ++ci) {
            {
                const EvalShape sh = shapes[ci];
                e = launch_full_evaluation_shape(S.w, 0, sh, s);  // warm-up
                double best = 1e30;
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                    e = cudaEventRecord(ev.a, s);
                    if (e == cudaSuccess) e = launch_full_evaluation_shape(S.w, 0, sh, s);
                    if (e == cudaSuccess) e = cudaEventRecord(ev.b, s);
                    if (e == cudaSuccess) e = cudaEventSynchronize(ev.b);
                    if (e == cudaSuccess) best = std::min(best, ev.elapsed_ms());
                }
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "timing an evaluation shape");
                    break;
                }
                const int32_t c = r.candidates++;
                r.cand_rows[c] = sh.rows;
                r.cand_strip[c] = sh.strip;
                r.cand_tma[c] = sh.tma;
                r.cand_ms[c] = best;
                if (best < r.best_ms) {
                    r.best_ms = best;
                    r.rows_per_thread = sh.rows;
                    r.strip = sh.strip;
                    r.tma = sh.tma;
                }
            }
        }
        if (st == DGS_OK) {
            set_evaluation_shape(n, EvalShape{r.rows_per_thread, r.strip, r.tma});
            const int32_t b = size_bucket(n);
            r.n_lo = b == 0 ? 1 : (1 << (b - 1)) + 1;
            r.n_hi = 1 << b;
            if (result) *result = r;
        }
    }
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    return st;
}

dgs_status dgs_get_tuning(int32_t n, int32_t* rows_per_thread, int32_t* strip, int32_t* tma) {
    if (n <= 0 || n > kMaxN) return DGS_ERR_INVALID;
    const EvalShape sh = evaluation_shape(n);
    if (rows_per_thread) *rows_per_thread = sh.rows;
    if (strip) *strip = sh.strip;
    if (tma) *tma = sh.tma;
    return DGS_OK;
}

const char* dgs_status_string(dgs_status status) {
    switch (status) {
        case DGS_OK: return "DGS_OK";
        case DGS_ERR_INVALID: return "DGS_ERR_INVALID";
        case DGS_ERR_RANGE: return "DGS_ERR_RANGE";
        case DGS_ERR_OOM: return "DGS_ERR_OOM";
        case DGS_ERR_CUDA: return "DGS_ERR_CUDA";
        case DGS_TIMEOUT: return "DGS_TIMEOUT";
        case DGS_PENDING: return "DGS_PENDING";
        case DGS_ERR_BUSY: return "DGS_ERR_BUSY";
        case DGS_ERR_INTERNAL: return "DGS_ERR_INTERNAL";
    }
    return "DGS_UNKNOWN";
}

const char* dgs_last_cuda_error(void) { return g_last_error; }

}  // extern "C"

extern "C" dgs_status dgs_release_cached_memory(void) {
    std::lock_guard<std::mutex> lock(dgs::g_pool_mutex);
    dgs_status st = DGS_OK;
    for (int d = 0; d < 64; ++d) {
        if (dgs::g_pools[d] == nullptr) continue;
        const cudaError_t e = cudaMemPoolTrimTo(dgs::g_pools[d], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemPoolTrimTo");
    }
    return st;
}
