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
// pass 1 over a band of tile rows (k_greedy.cu)
cudaError_t launch_greedy_pass1_rows(const Workspace& w, int32_t cols, int32_t row_tile0, int32_t row_tile1,
                                     cudaStream_t s);
}  // namespace dgs


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
    // DGS_FAKE_OOM_BYTES (tests): requests of at least this many bytes fail
    // as if the device were out of memory, without touching the device
    if (const char* fk = std::getenv("DGS_FAKE_OOM_BYTES")) {
        const long long lim = std::atoll(fk);
        if (lim > 0 && bytes >= (size_t)lim) return cudaErrorMemoryAllocation;
    }
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

// One copy stream per device for host-to-device bands (created once, kept for
// the process; the stream is safe to share between calling threads).
cudaStream_t copy_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (streams[dev] == nullptr && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

int32_t device_sms() {
    static int32_t cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

int32_t env_compact_min() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_CTL_COMPACT_MIN");
        const int32_t x = e ? std::atoi(e) : 2048;
        return x >= 1 ? x : 2048;
    }();
    return v;
}
// DGS_CC_COLOUR: 0 turns the colouring passes over runs of quiet sweeps
// off.  Read on every launch, so that a test can compare both in one process.
int32_t env_colour_pass() {
    const char* e = std::getenv("DGS_CC_COLOUR");
    return (e && std::atoi(e) == 0) ? 0 : 1;
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

// The status a finished solve or evaluation returns for its loop state.
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
    w.sl_chunk = ar.take<int32_t>(2 * nb / 32);
    w.sl_rkey = ar.take<unsigned long long>(2 * nb);
    w.sl_ru = ar.take<int32_t>(2 * nb);
    w.sl_rv = ar.take<int32_t>(2 * nb);
    w.ctl_slot = ar.take<int32_t>(2 * nb);
    w.g_row = ar.take<unsigned long long>(nb);
    w.g_col = ar.take<unsigned long long>(nb);
    w.free_a = ar.take<uint8_t>(nb);
    w.free_j = ar.take<uint8_t>(nb);
    w.g_list = ar.take<unsigned long long>(4 * nb);
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

__global__ void write_state_kernel(DeviceState* st, DeviceState h) { *st = h; }

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
        // by a kernel argument: a copy from pageable host memory would wait
        // for the stream
        write_state_kernel<<<1, 1, 0, s>>>(w.st, h);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "loop state");
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

// ------------------------------------------------ device-side loop bodies
struct LoopCtx {
    Workspace w;
    CtlGlobal ctl;
};

// Everything the loop bodies' launches are captured with: the workspace and
// controller pointers and sizes, and the evaluation's launch shape for n.
struct LoopKey {
    unsigned char w[sizeof(Workspace)];
    unsigned char ctl[sizeof(CtlGlobal)];
    int32_t rows, strip, tma, colour_pass, small_threads, pad;  // launch shapes and knobs the kernels bake in
};

LoopKey loop_key(const LoopCtx& c) {
    LoopKey k;
    memset(&k, 0, sizeof(k));
    memcpy(k.w, &c.w, sizeof(Workspace));
    memcpy(k.ctl, &c.ctl, sizeof(CtlGlobal));
    const EvalShape sh = evaluation_shape(c.w.n);
    k.rows = sh.rows;
    k.strip = sh.strip;
    k.tma = sh.tma;
    k.colour_pass = env_colour_pass();
    k.small_threads = small_loop_threads();
    return k;
}

// DGS_LOOP_ON_HOST=1 (profiling only: per-kernel profilers do not see the
// kernels inside conditional graph nodes): the switching loop's body is
// launched from the host, four iterations between reads of the loop state,
// which makes the call wait for the solve.  Results are the same.
int32_t env_loop_on_host() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_LOOP_ON_HOST");
        return (e && std::atoi(e) == 1) ? 1 : 0;
    }();
    return v;
}

dgs_status switching_body(void* p, cudaStream_t cs, unsigned long long h);

dgs_status enqueue_loop(cudaStream_t s, LoopBody body, LoopCtx* c) {
    if (env_loop_on_host() && body == switching_body) {
        DeviceState* h = static_cast<DeviceState*>(pinned_get(sizeof(DeviceState)));
        if (h == nullptr) return DGS_ERR_OOM;
        dgs_status st = DGS_OK;
        for (int64_t it = 0; st == DGS_OK && it < 16 * (int64_t)c->w.n + 4096; it += 4) {
            for (int r = 0; r < 4 && st == DGS_OK; ++r) st = body(c, s, 0);
            cudaError_t e = cudaMemcpyAsync(h, c->w.st, sizeof(DeviceState), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "reading loop state");
            if (st == DGS_OK && h->status != kRunning) break;
        }
        pinned_put(h, sizeof(DeviceState));
        return st;
    }
    const LoopKey k = loop_key(*c);
    return enqueue_while_cached(s, body, c, &k, sizeof(k));
}

// One locally-dominant greedy round and its loop condition.
dgs_status greedy_round_body(void* p, cudaStream_t cs, unsigned long long h) {
    const LoopCtx* c = static_cast<const LoopCtx*>(p);
    DGS_CUDA(launch_greedy_round(c->w, cs), "greedy round");
    DGS_CUDA(launch_greedy_loop_cond(c->w, h, cs), "greedy loop");
    return DGS_OK;
}

// One iteration of the switching loop of Algorithm 3: re-evaluate what the
// last committing sweep changed (marked rows by row tasks, or all rows by a
// full evaluation), refresh the slots not in C, then the controller's sweeps;
// the controller decides whether the loop goes on.
dgs_status switching_body(void* p, cudaStream_t cs, unsigned long long h) {
    const LoopCtx* c = static_cast<const LoopCtx*>(p);
    DGS_CUDA(launch_mark_rescan(c->w, cs), "mark");
    DGS_CUDA(launch_full_evaluation(c->w, 1, cs), "re-evaluation");
    DGS_CUDA(launch_row_tasks(c->w, cs), "row tasks");
    DGS_CUDA(launch_prepare_edges(c->w, cs), "prepare");
    DGS_CUDA(launch_controller_impl(c->w, c->ctl, cs, h), "controller");
    return DGS_OK;
}

// Algorithm 1: the switching loop of one pass (launches until the loop ends).
dgs_status sequential_inner_body(void* p, cudaStream_t cs, unsigned long long h) {
    const LoopCtx* c = static_cast<const LoopCtx*>(p);
    DGS_CUDA(launch_sequential(c->w, cs), "switching loop");
    DGS_CUDA(launch_seq_inner_cond(c->w, h, cs), "switching loop condition");
    return DGS_OK;
}

// Algorithm 1: one pass of the outer repeat (fresh evaluation of every slot,
// the switching loop), repeated while a pass changes f.
dgs_status sequential_pass_body(void* p, cudaStream_t cs, unsigned long long h) {
    LoopCtx* c = static_cast<LoopCtx*>(p);
    unsigned long long inner = 0;
    DGS_TRY(create_loop_handle(cs, &inner));
    DGS_CUDA(launch_seq_pass_begin(c->w, inner, cs), "pass");
    // the evaluation raises the row keys from zero (slot i reads the key of
    // row tau(i), so the keys cannot be cleared while the slots are read)
    DGS_CUDA(cudaMemsetAsync(c->w.key_a, 0, (size_t)c->w.n * sizeof(unsigned long long), cs), "clear keys");
    DGS_CUDA(cudaMemsetAsync(c->w.key_j, 0, (size_t)c->w.n * sizeof(unsigned long long), cs), "clear keys");
    DGS_CUDA(launch_full_evaluation(c->w, 0, cs), "evaluation");
    DGS_CUDA(launch_slots_from_keys(c->w, cs), "slots");
    DGS_TRY(capture_while(cs, sequential_inner_body, c, inner));
    DGS_CUDA(launch_seq_pass_end(c->w, h, cs), "pass condition");
    return DGS_OK;
}

// The greedy start: pass 1, then deferred acceptance in one cooperative
// launch; where that launch is refused, pass 1 again with the column keys and
// the locally-dominant rounds as a device-side loop (the same assignment).
// A matrix that arrives in row bands (dgs_solve_host): event k is recorded
// once rows [64 k tile_rows, 64 (k + 1) tile_rows) are on the device.
struct HostBands {
    const cudaEvent_t* ev;
    int32_t count;
    int32_t tile_rows;
};

dgs_status run_greedy(Solve& S, EventPair* timer, const HostBands* bands = nullptr) {
    if (bands == nullptr) {
        DGS_CUDA(launch_greedy_pass1_cols(S.w, 0, S.s), "greedy pass 1");
        S.launches += 1;
    } else {  // pass 1 of each band as soon as it has landed, while later ones are still copied
        for (int32_t k = 0; k < bands->count; ++k) {
            DGS_CUDA(cudaStreamWaitEvent(S.s, bands->ev[k], 0), "wait for a band of the matrix");
            DGS_CUDA(launch_greedy_pass1_rows(S.w, 0, k * bands->tile_rows, (k + 1) * bands->tile_rows, S.s),
                     "greedy pass 1");
            S.launches += 1;
        }
    }
    if (timer) DGS_TRY(timer->begin(S.s));
    const cudaError_t pe = launch_greedy_da(S.w, S.s);
    if (pe == cudaSuccess) {
        S.launches += 2;
        if (timer) DGS_TRY(timer->end(S.s));
        return DGS_OK;
    }
    cudaGetLastError();
    DGS_CUDA(launch_greedy_pass1_cols(S.w, 1, S.s), "greedy pass 1");
    S.launches += 1;
    LoopCtx c{S.w, S.ctl};
    DGS_TRY(enqueue_loop(S.s, greedy_round_body, &c));
    if (timer) DGS_TRY(timer->end(S.s));
    return DGS_OK;
}

dgs_status check_common(const int32_t* benefit, int32_t n) {
    if (benefit == nullptr || n <= 0 || n > kMaxN) return DGS_ERR_INVALID;
    return DGS_OK;
}

// The public status of a finished loop state, without touching the calling
// thread's error text (used from stream callbacks).
dgs_status status_of(const DeviceState& h) {
    if (h.status == kTimeout) return DGS_TIMEOUT;
    if (h.status != kError) return DGS_OK;
    if (h.error == kErrRange) return DGS_ERR_RANGE;
    if (h.error == kErrUserInit) return DGS_ERR_INVALID;
    return DGS_ERR_INTERNAL;
}

// What a solve reports on the host once the stream reaches its end: a copy
// of the final loop state in pinned memory is read by a host callback that
// fills the caller's host-side outputs and returns the staging blocks.
struct Completion {
    DeviceState* staged = nullptr;
    void* release = nullptr;  // pinned block of the call (the random start), or null
    size_t release_bytes = 0;
    dgs_stats* stats = nullptr;
    int64_t* objective = nullptr;  // host objective (a device one is written by the finish kernel)
    int32_t* status = nullptr;     // host options.status_out
    dgs_status* status_api = nullptr;
    int64_t launches = 0;          // kernels launched from the host
    int32_t sequential = 0;
    ~Completion() {
        pinned_put(staged, sizeof(DeviceState));
        pinned_put(release, release_bytes);
    }
};

void fill_stats(const DeviceState& h, const Completion& c, dgs_stats* stats) {
    memset(stats, 0, sizeof(*stats));
    stats->sweeps = h.sweeps;
    stats->events = h.events;
    stats->swaps_applied = h.swaps;
    stats->greedy_rounds = h.greedy_rounds;
    stats->full_evaluations = c.sequential ? 0 : h.full_evals + 1;
    stats->row_updates = c.sequential ? 0 : h.row_updates;
    stats->rows_recomputed = c.sequential ? 0 : h.rows_recomputed;
    stats->initial_objective = h.f_initial;
    stats->kernel_launches = c.launches + h.loop_launches;
    stats->greedy_rescans = h.greedy_rescans;
    stats->status = status_of(h);
}

void CUDART_CB completion_callback(void* p) {
    Completion* c = static_cast<Completion*>(p);
    const DeviceState& h = *c->staged;
    const dgs_status st = status_of(h);
    if (c->objective) *c->objective = h.f;
    if (c->status) *c->status = (int32_t)st;
    if (c->status_api) *c->status_api = st;
    if (c->stats) fill_stats(h, *c, c->stats);
    delete c;
}

// The random start's permutation, staged in pinned memory for its copy to
// the device; the block returns to the cache with the call's completion (or
// after the stream drains, on an error path).
struct PinnedStart {
    cudaStream_t s;
    void* p = nullptr;
    size_t bytes = 0;
    bool copied = false;
    explicit PinnedStart(cudaStream_t st) : s(st) {}
    ~PinnedStart() {
        if (p == nullptr) return;
        if (copied) cudaStreamSynchronize(s);
        pinned_put(p, bytes);
    }
    void* release() {
        void* q = p;
        p = nullptr;
        return q;
    }
};

// One solve, enqueued on `stream`.  final_status (host, may be null): set to
// the solve's status when the stream reaches its end.  extra_launches: kernels
// the caller launches around the solve (counted in the stats).
dgs_status solve_impl(const int32_t* benefit, int32_t n, int32_t* sigma_out, int64_t* objective_out,
                      const dgs_options* opt, dgs_stats* stats, cudaStream_t stream,
                      dgs_status* final_status = nullptr, int64_t extra_launches = 0,
                      const HostBands* bands = nullptr) {
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

    // where the objective and the status go: written by the finish kernel when
    // the device can write them, else by the completion callback
    void* obj_dev = nullptr;
    const bool obj_on_device = device_writable(objective_out, &obj_dev);
    void* status_dev = nullptr;
    const bool status_on_device = o.status_out != nullptr && device_writable(o.status_out, &status_dev);

    EventPair whole;
    if (o.profile) DGS_TRY(whole.begin(stream));
    Solve S(stream);
    if (bands != nullptr &&
        (o.init != DGS_INIT_GREEDY || n % 4 != 0 || (reinterpret_cast<uintptr_t>(benefit) % 16) != 0)) {
        // the whole matrix first: the start, or the re-pitched copy, reads it before pass 1
        DGS_CUDA(cudaStreamWaitEvent(stream, bands->ev[bands->count - 1], 0), "wait for the matrix");
        bands = nullptr;
    }
    DGS_TRY(S.setup(benefit, n, true));
    S.w.row_owner_eval = o.evaluation == DGS_EVAL_ROW_OWNER ? 1 : 0;
    // the random start is drawn on the host and enters as the caller's start
    DeviceBuffer rnd(stream);
    PinnedStart pin(stream);
    if (o.init == DGS_INIT_RANDOM) {
        pin.bytes = (size_t)n * sizeof(int32_t);
        pin.p = pinned_get(pin.bytes);
        if (pin.p == nullptr) {
            snprintf(g_last_error, sizeof(g_last_error), "pinned staging of %zu bytes", pin.bytes);
            return DGS_ERR_OOM;
        }
        random_start(n, o.seed, static_cast<int32_t*>(pin.p));
        DGS_TRY(rnd.alloc(pin.bytes));
        DGS_CUDA(cudaMemcpyAsync(rnd.p, pin.p, pin.bytes, cudaMemcpyHostToDevice, stream), "copy random start");
        pin.copied = true;
        o.init = DGS_INIT_USER;
        o.init_sigma = static_cast<const int32_t*>(rnd.p);
    }
    DGS_TRY(S.init_state(o.max_sweeps, &o));
    S.launches += 1;
    if (o.deadline_us > 0) {
        arm_deadline_kernel<<<1, 1, 0, stream>>>(S.w.st, o.deadline_us);
        DGS_CUDA(cudaGetLastError(), "arm deadline");
        S.launches += 1;
    }
    EventPair gev;
    if (o.init == DGS_INIT_GREEDY) {
        DGS_TRY(run_greedy(S, o.profile ? &gev : nullptr, bands));
    } else {
        DGS_CUDA(launch_greedy_pass1(S.w, stream), "pass 1");  // transpose + range check
        S.launches += 1;
    }
    DGS_CUDA(launch_start_from_tau(S.w, o.init_sigma, o.init, S.seen, stream), "start");
    record_initial_objective_kernel<<<1, 1, 0, stream>>>(S.w.st);
    S.launches += 2;
    EventPair ev;
    LoopCtx lc{S.w, S.ctl};
    if (o.algorithm == DGS_ALG_SEQUENTIAL) {
        DGS_TRY(enqueue_loop(stream, sequential_pass_body, &lc));
    } else {
        if (o.profile) DGS_TRY(ev.begin(stream));
        DGS_CUDA(launch_full_evaluation(S.w, 0, stream), "evaluation");
        S.launches += 1;
        if (o.profile) DGS_TRY(ev.end(stream));
        // the single-CTA loop re-evaluates changed rows on one SM: fine after
        // the greedy start (few exchanges per commit), not after a random or
        // given start, whose commits change hundreds of rows (GEOM n = 512,
        // random start: 5.2 ms in one CTA against 1.7 ms on the grid; n = 128:
        // 0.52 against 0.78 ms)
        if (use_small_loop(S.w) && (o.init == DGS_INIT_GREEDY || S.w.n <= 128)) {
            DGS_CUDA(launch_small_loop(S.w, S.ctl, stream), "switching loop");
            S.launches += 1;
        } else {
            DGS_TRY(enqueue_loop(stream, switching_body, &lc));
        }
    }
    DGS_CUDA(launch_finish_outputs(S.w, sigma_out, obj_on_device ? static_cast<int64_t*>(obj_dev) : nullptr,
                                   status_on_device ? static_cast<int32_t*>(status_dev) : nullptr, stream),
             "finish");
    S.launches += 1;
    if (o.profile) DGS_TRY(whole.end(stream));  // the device work of the solve ends here
    const bool host_outputs = stats != nullptr || !obj_on_device || (o.status_out && !status_on_device) ||
                              final_status != nullptr || pin.p != nullptr;
    if (host_outputs) {
        Completion* c = new Completion();
        c->staged = static_cast<DeviceState*>(pinned_get(sizeof(DeviceState)));
        if (c->staged == nullptr) {
            delete c;
            snprintf(g_last_error, sizeof(g_last_error), "pinned staging of the loop state");
            return DGS_ERR_OOM;
        }
        c->stats = stats;
        c->objective = obj_on_device ? nullptr : objective_out;
        c->status = (o.status_out && !status_on_device) ? o.status_out : nullptr;
        c->status_api = final_status;
        c->launches = S.launches + extra_launches;
        c->sequential = o.algorithm == DGS_ALG_SEQUENTIAL ? 1 : 0;
        cudaError_t e = cudaMemcpyAsync(c->staged, S.w.st, sizeof(DeviceState), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(stream, completion_callback, c);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(stream);  // the copy may be in flight
            delete c;
            return cuda_fail(e, "completion");
        }
        c->release_bytes = pin.bytes;
        c->release = pin.release();  // returned by the callback
    }
    if (S.w.phase_ns) {  // test/diagnostic output only: waits for the solve
        unsigned long long ph[kPtCount];
        if (cudaMemcpyAsync(ph, S.w.phase_ns, sizeof(ph), cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
            cudaStreamSynchronize(stream) == cudaSuccess) {
            fprintf(stderr, "[dgs phases] greedy: last group %llu ns, group sum %llu ns, longest chain %llu, "
                            "most scans of a group %llu | controller cycles: entry %llu top %llu conflict check %llu "
                            "post %llu event %llu sweeps %llu | live edges summed over sweeps %llu, listed %llu, "
                            "accepted in quiet sweeps %llu | colouring passes %llu, cycles %llu (reservation "
                            "rounds %llu, after them %llu), sweeps run %llu\n",
                    ph[kPtDaLastNs], ph[kPtDaSumNs], ph[kPtDaChain], ph[kPtDaGroupScans], ph[kPtCtlEntry],
                    ph[kPtCtlTop], ph[kPtCtlPass1], ph[kPtCtlPost], ph[kPtCtlEvent], ph[kPtCtlSweeps],
                    ph[kPtCtlLiveSum], ph[kPtCtlListSum], ph[kPtCtlAccSum], ph[kPtCtlColourPasses], ph[kPtCtlColour],
                    ph[kPtCtlColourIters], ph[kPtCtlColourTail], ph[kPtCtlColourRounds]);
        }
    }
    if (o.profile) {  // the event timings need the solve to have run
        DGS_CUDA(cudaStreamSynchronize(stream), "profile");
        if (stats) {
            stats->solve_ms = whole.elapsed_ms();
            stats->evaluation_ms = o.algorithm == DGS_ALG_SEQUENTIAL ? 0.0 : ev.elapsed_ms();
            stats->greedy_ms = o.init == DGS_INIT_GREEDY ? gev.elapsed_ms() : 0.0;
        }
    }
    return DGS_OK;
}

}  // namespace

namespace dgs {
dgs_status solve_for_server(const int32_t* benefit, int32_t n, int32_t* sigma_out, int64_t* objective_out,
                            const dgs_options* opt, dgs_stats* stats, cudaStream_t stream, dgs_status* final_status) {
    return solve_impl(benefit, n, sigma_out, objective_out, opt, stats, stream, final_status);
}
}  // namespace dgs

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
    dgs_status st = DGS_OK, outcome = DGS_OK;
    // A large matrix from the greedy start is copied in row bands on a copy
    // stream, and greedy pass 1 takes each band as it lands: the copy (bound
    // by the host link) hides pass 1.
    constexpr int32_t kBands = 8;
    cudaEvent_t ev[kBands + 1] = {};
    HostBands bands{ev + 1, 0, 0};
    const bool greedy = options == nullptr || options->init == DGS_INIT_GREEDY;
    cudaStream_t cs = (greedy && n % 4 == 0 && n >= 2048) ? copy_stream() : nullptr;
    if (cs != nullptr) {
        const int32_t tiles = (n + 63) / 64;
        bands.tile_rows = (tiles + kBands - 1) / kBands;
        bands.count = (tiles + bands.tile_rows - 1) / bands.tile_rows;
        for (int32_t k = 0; k <= bands.count && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);  // the buffer exists in the caller's stream order
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
        for (int32_t k = 0; k < bands.count && e == cudaSuccess; ++k) {
            const size_t r0 = (size_t)k * bands.tile_rows * 64;
            const size_t r1 = std::min<size_t>((size_t)n, r0 + (size_t)bands.tile_rows * 64);
            e = cudaMemcpyAsync(a_dev + r0 * n, benefit_host + r0 * n, (r1 - r0) * n * sizeof(int32_t),
                                cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1 + k], cs);
        }
        if (e != cudaSuccess) st = cuda_fail(e, "copy benefit to device");
    } else {
        e = cudaMemcpyAsync(a_dev, benefit_host, abytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy benefit to device");
    }
    if (st == DGS_OK)
        st = solve_impl(a_dev, n, out_dev, objective_out, options, stats, s, &outcome, 0,
                        cs != nullptr ? &bands : nullptr);
    if (st == DGS_OK) {
        e = cudaMemcpyAsync(sigma_out_host, out_dev, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy result to host");
    }
    if (cs != nullptr) {
        // the copy stream's bands precede the free (the caller's stream waited
        // for all of them, or waits now if the solve failed to enqueue)
        if (bands.count > 0 && ev[bands.count] != nullptr) cudaStreamWaitEvent(s, ev[bands.count], 0);
        cudaStreamSynchronize(cs);
    }
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    for (cudaEvent_t x : ev)
        if (x != nullptr) cudaEventDestroy(x);
    return st == DGS_OK ? outcome : st;
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
    pad_square_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(benefit, n_agents, m_jobs, sz, sq);
    DGS_CUDA(cudaGetLastError(), "pad");
    DGS_TRY(solve_impl(sq, sz, tau, objective_out, &o, stats, s, nullptr, 2));
    trim_assignment_kernel<<<(n_agents + 255) / 256, 256, 0, s>>>(tau, n_agents, m_jobs, assign_out);
    DGS_CUDA(cudaGetLastError(), "trim");
    return DGS_OK;
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
        fill_synthetic_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(a, n, lda, 0x9E3779B97F4A7C15ull ^ (uint64_t)n);
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
        case DGS_CANCELLED: return "DGS_CANCELLED";
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
