// dgs_batch.cu -- batched and served solves (include/dgs.h: dgs_solve_batched,
// dgs_server_*).
//
// Many instances of different sizes advance together.  Each instance owns a
// slot: its workspace (the same layout as a single solve) and its loop state
// in one device array of DeviceState, indexed by slot.  An instance moves
// through stages (new -> greedy -> start -> switch -> done) on the device;
// every batched kernel is a persistent grid that walks a table of (instance,
// block) entries and acts only on the instances in the stage it serves, with
// the instance's own n, sigma and loop state.  One step is a fixed sequence
// of launches:
//
//   init (fresh slots) -> pass 1 -> advance(new)
//   -> greedy start (deferred acceptance of every new instance's agents in
//      one launch) -> advance(greedy)
//   -> start, first full evaluation -> advance(start)
//   -> switching iterations x kSwitchPerStep -> finish -> advance(switch)
//   -> copy of every slot's loop state to pinned host memory
//
// captured once as a CUDA graph and replayed; the tables have a fixed
// capacity per slot, so admitting or retiring instances only rewrites the
// tables' contents, never the graph.  Within a stage an instance executes
// exactly the launches of a single solve, in the same order, so its result
// is bit-identical to dgs_solve_ex on that instance alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dgs.h"
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int32_t kSwitchPerStep = 8;   // switching iterations per step

// Static work tables (the per-instance work of these launches is known from
// n alone) and the most entries one instance can take in each: rows =
// ceil(n / 512) blocks of 256 threads over agents, jobs or slots; one = the
// instance itself.  Work that depends on the device state (pass 1 of new
// instances, greedy rescans, evaluations, row tasks) goes through the queues
// of launch_b_scan instead.
enum : int32_t { kTabRows = 0, kTabOne, kTabCount };
constexpr int32_t kMaxPerInstance[kTabCount] = {64, 1};

int32_t ceil_div(int64_t a, int64_t b) { return (int32_t)((a + b - 1) / b); }
int32_t clampi(int32_t x, int32_t lo, int32_t hi) { return x < lo ? lo : (x > hi ? hi : x); }

int32_t blocks_for(int32_t tab, int32_t n) {
    return tab == kTabRows ? clampi(ceil_div(n, 512), 1, kMaxPerInstance[kTabRows]) : 1;
}

thread_local char g_err[512];

dgs_status fail(cudaError_t e, const char* what) {
    snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
    set_last_error(g_err);
    return DGS_ERR_CUDA;
}

#define B_CUDA(expr, what)                              \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return fail(_e, what);   \
    } while (0)

dgs_status status_of(const DeviceState& h) {
    if (h.status == kDone) return DGS_OK;
    if (h.status == kTimeout) return DGS_TIMEOUT;
    if (h.status == kError) {
        if (h.error == kErrRange) return DGS_ERR_RANGE;
        if (h.error == kErrUserInit) return DGS_ERR_INVALID;
        return DGS_ERR_INTERNAL;
    }
    return DGS_ERR_INTERNAL;  // finished without a final status
}

void stats_of(const DeviceState& h, int64_t launches, dgs_stats* out) {
    memset(out, 0, sizeof(*out));
    out->sweeps = h.sweeps;
    out->events = h.events;
    out->swaps_applied = h.swaps;
    out->greedy_rounds = h.greedy_rounds;
    out->full_evaluations = h.full_evals + 1;
    out->row_updates = h.row_updates;
    out->rows_recomputed = h.rows_recomputed;
    out->initial_objective = h.f_initial;
    out->kernel_launches = launches;
    out->greedy_rescans = h.greedy_rescans;
}

// Slots, tables and the step graph of one batch of resident instances.
class Engine {
  public:
    // capacity: slots; max_n: largest n any slot will hold.
    Engine(int32_t capacity, int32_t max_n) : cap_(capacity), max_n_(max_n) {}
    Engine(const Engine&) = delete;
    Engine& operator=(const Engine&) = delete;

    ~Engine() {
        if (exec_) cudaGraphExecDestroy(exec_);
        if (stream_) cudaStreamSynchronize(stream_);
        if (d_inst_) cudaFree(d_inst_);
        if (d_st_) cudaFree(d_st_);
        if (d_ent_) cudaFree(d_ent_);
        if (d_cnt_) cudaFree(d_cnt_);
        if (d_q_) cudaFree(d_q_);
        if (h_inst_) cudaFreeHost(h_inst_);
        if (h_st_) cudaFreeHost(h_st_);
        if (h_ent_) cudaFreeHost(h_ent_);
        if (h_cnt_) cudaFreeHost(h_cnt_);
        if (stream_) cudaStreamDestroy(stream_);
    }

    dgs_status init() {
        // the batched steps carry many small instances: their stream has the
        // highest priority, so that the server's solo solves (lowest
        // priority) yield SMs to them
        int least = 0, greatest = 0;
        B_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
        B_CUDA(cudaStreamCreateWithPriority(&stream_, cudaStreamNonBlocking, greatest), "stream");
        B_CUDA(cudaMalloc(&d_inst_, sizeof(Instance) * cap_), "instance table");
        B_CUDA(cudaMalloc(&d_st_, sizeof(DeviceState) * cap_), "loop states");
        B_CUDA(cudaMemset(d_st_, 0, sizeof(DeviceState) * cap_), "loop states");
        size_t total = 0;
        for (int32_t t = 0; t < kTabCount; ++t) {
            off_[t] = total;
            total += (size_t)kMaxPerInstance[t] * cap_;
        }
        B_CUDA(cudaMalloc(&d_ent_, sizeof(BatchEntry) * total), "work tables");
        B_CUDA(cudaMalloc(&d_cnt_, sizeof(int32_t) * kTabCount), "work table counts");
        B_CUDA(cudaMalloc(&d_q_, sizeof(int32_t) * 2 * (cap_ + 1)), "work queues");
        B_CUDA(cudaMallocHost(&h_inst_, sizeof(Instance) * cap_), "instance table (host)");
        B_CUDA(cudaMallocHost(&h_st_, sizeof(DeviceState) * cap_), "loop states (host)");
        B_CUDA(cudaMallocHost(&h_ent_, sizeof(BatchEntry) * total), "work tables (host)");
        B_CUDA(cudaMallocHost(&h_cnt_, sizeof(int32_t) * kTabCount), "counts (host)");
        memset(h_inst_, 0, sizeof(Instance) * cap_);
        memset(h_st_, 0, sizeof(DeviceState) * cap_);
        used_.assign(cap_, 0);
        return DGS_OK;
    }

    cudaStream_t stream() const { return stream_; }
    int32_t capacity() const { return cap_; }
    bool used(int32_t k) const { return used_[k] != 0; }
    const DeviceState& state(int32_t k) const { return h_st_[k]; }
    int64_t launches_per_step() const { return launches_per_step_; }
    int32_t free_slot() const {
        for (int32_t k = 0; k < cap_; ++k)
            if (!used_[k]) return k;
        return -1;
    }

    // Place an instance in slot k.  mem: carve_instance(nullptr, n, with_copy)
    // bytes of device memory.  Without a copy region the matrix a is used in
    // place; with one, a (if not null) is the caller's unpitched matrix that
    // the init kernel re-pitches into the region, and a == null means the
    // region already holds the pitched matrix.
    void place(int32_t k, char* mem, int32_t n, bool with_copy, const int32_t* a, int32_t* sigma_out,
               int32_t init_mode, int32_t max_sweeps, int64_t deadline_us, const int32_t* user_tau = nullptr,
               bool reeval_all = false) {
        Instance in{};
        carve_instance(mem, n, with_copy, &in);
        if (!with_copy) in.w.a = a;
        else in.a_src = a;
        in.w.st = d_st_ + k;
        in.fresh = 1;
        in.max_sweeps = max_sweeps;
        in.init_mode = init_mode;
        in.user_tau = user_tau;
        in.reeval_all = reeval_all ? 1 : 0;
        in.deadline_us = deadline_us;
        in.sigma_out = sigma_out;
        h_inst_[k] = in;
        h_st_[k] = DeviceState{};
        used_[k] = 1;
        tables_dirty_ = true;
        inst_dirty_ = true;
    }

    void vacate(int32_t k) {
        used_[k] = 0;
        memset(&h_inst_[k], 0, sizeof(Instance));
        tables_dirty_ = true;
        inst_dirty_ = true;
    }

    // One step: upload what changed, replay the step graph, wait for it and
    // read every slot's loop state.
    dgs_status step() {
        if (tables_dirty_) build_tables();
        if (inst_dirty_)
            B_CUDA(cudaMemcpyAsync(d_inst_, h_inst_, sizeof(Instance) * cap_, cudaMemcpyHostToDevice, stream_),
                   "upload instances");
        if (tables_dirty_) {
            size_t total = 0;
            for (int32_t t = 0; t < kTabCount; ++t) total = std::max(total, off_[t] + (size_t)h_cnt_[t]);
            B_CUDA(cudaMemcpyAsync(d_ent_, h_ent_, sizeof(BatchEntry) * total, cudaMemcpyHostToDevice, stream_),
                   "upload tables");
            B_CUDA(cudaMemcpyAsync(d_cnt_, h_cnt_, sizeof(int32_t) * kTabCount, cudaMemcpyHostToDevice, stream_),
                   "upload counts");
        }
        if (!exec_) {
            dgs_status st = capture();
            if (st != DGS_OK) return st;
        }
        B_CUDA(cudaGraphLaunch(exec_, stream_), "step graph");
        B_CUDA(cudaStreamSynchronize(stream_), "step");
        // fresh instances were initialised by this step
        bool cleared = false;
        for (int32_t k = 0; k < cap_; ++k)
            if (used_[k] && h_inst_[k].fresh) {
                h_inst_[k].fresh = 0;
                cleared = true;
            }
        inst_dirty_ = cleared;
        tables_dirty_ = false;
        ++steps_;
        return DGS_OK;
    }

    int64_t steps() const { return steps_; }

  private:
    BatchTable table(int32_t t) const {
        return BatchTable{d_inst_, d_ent_ + off_[t], d_cnt_ + t};
    }

    void build_tables() {
        for (int32_t t = 0; t < kTabCount; ++t) {
            int32_t c = 0;
            BatchEntry* e = h_ent_ + off_[t];
            for (int32_t k = 0; k < cap_; ++k) {
                if (!used_[k]) continue;
                const int32_t nb = blocks_for(t, h_inst_[k].w.n);
                for (int32_t b = 0; b < nb; ++b) e[c++] = BatchEntry{k, b, nb, 0};
            }
            h_cnt_[t] = c;
        }
    }

    dgs_status enqueue_step(cudaStream_t s, int64_t* launches) {
        int64_t L = 0;
#define B_LAUNCH(expr, n_kernels, what)           \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) return fail(_e, what); \
        L += (n_kernels);                         \
    } while (0)
        const BatchTable rows = table(kTabRows), one = table(kTabOne);
        const BatchQueues q{d_inst_, cap_, d_q_, d_q_ + cap_ + 1};
        const int32_t strip = evaluation_strip();
        B_LAUNCH(launch_b_init(rows, s), 1, "init");
        B_LAUNCH(launch_b_scan(q, kScanPass1, strip, s), 1, "scan");
        B_LAUNCH(launch_b_pass1(q, s), 1, "pass 1");
        B_LAUNCH(launch_b_advance(one, kStageNew, s), 1, "advance");
        B_LAUNCH(launch_b_greedy(rows, q, s), 3, "greedy start");
        B_LAUNCH(launch_b_advance(one, kStageGreedy, s), 1, "advance");
        B_LAUNCH(launch_b_start(rows, s), 1, "start");
        B_LAUNCH(launch_b_scan(q, kScanStart, strip, s), 1, "scan");
        B_LAUNCH(launch_b_evaluation(q, strip, s), 1, "evaluation");
        B_LAUNCH(launch_b_advance(one, kStageStart, s), 1, "advance");
        for (int32_t i = 0; i < kSwitchPerStep; ++i) {
            B_LAUNCH(launch_b_mark_rescan(rows, s), 1, "mark");
            B_LAUNCH(launch_b_scan(q, kScanSwitch, strip, s), 1, "scan");
            B_LAUNCH(launch_b_evaluation(q, strip, s), 1, "re-evaluation");
            B_LAUNCH(launch_b_row_tasks(q, max_n_, s), 1, "row tasks");
            B_LAUNCH(launch_b_prepare_edges(rows, s), 1, "prepare");
            B_LAUNCH(launch_b_controller(one, s), 1, "controller");
        }
        B_LAUNCH(launch_b_finish(rows, s), 1, "finish");
        B_LAUNCH(launch_b_advance(one, kStageSwitch, s), 1, "advance");
#undef B_LAUNCH
        B_CUDA(cudaMemcpyAsync(h_st_, d_st_, sizeof(DeviceState) * cap_, cudaMemcpyDeviceToHost, s), "read states");
        *launches = L;
        return DGS_OK;
    }

    dgs_status capture() {
        // kernel attributes are set outside the capture (first launch of each
        // kernel on this device), by one uncaptured pass over empty tables
        {
            const int32_t zero[kTabCount] = {0, 0};
            int32_t* saved = d_cnt_;
            int32_t* d_zero = nullptr;
            B_CUDA(cudaMallocAsync(&d_zero, sizeof(zero), stream_), "counts");
            B_CUDA(cudaMemcpyAsync(d_zero, zero, sizeof(zero), cudaMemcpyHostToDevice, stream_), "counts");
            B_CUDA(cudaStreamSynchronize(stream_), "counts");
            d_cnt_ = d_zero;
            int64_t l = 0;
            const dgs_status st = enqueue_step(stream_, &l);
            d_cnt_ = saved;
            cudaFreeAsync(d_zero, stream_);
            if (st != DGS_OK) return st;
            B_CUDA(cudaStreamSynchronize(stream_), "warm-up step");
        }
        cudaGraph_t g = nullptr;
        B_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal), "begin capture");
        int64_t launches = 0;
        const dgs_status st = enqueue_step(stream_, &launches);
        const cudaError_t e = cudaStreamEndCapture(stream_, &g);
        if (st != DGS_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(e, "end capture");
        const cudaError_t ei = cudaGraphInstantiate(&exec_, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return fail(ei, "instantiate step graph");
        launches_per_step_ = launches;
        return DGS_OK;
    }

    int32_t cap_;
    int32_t max_n_;
    cudaStream_t stream_ = nullptr;
    int32_t* d_q_ = nullptr;  // the two queue offset arrays (cap + 1 each)
    Instance* d_inst_ = nullptr;
    Instance* h_inst_ = nullptr;
    DeviceState* d_st_ = nullptr;
    DeviceState* h_st_ = nullptr;
    BatchEntry* d_ent_ = nullptr;
    BatchEntry* h_ent_ = nullptr;
    int32_t* d_cnt_ = nullptr;
    int32_t* h_cnt_ = nullptr;
    size_t off_[kTabCount] = {};
    std::vector<char> used_;
    bool tables_dirty_ = true, inst_dirty_ = true;
    cudaGraphExec_t exec_ = nullptr;
    int64_t launches_per_step_ = 0;
    int64_t steps_ = 0;
};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Upper bound on the steps of one instance: the greedy start ends within its
// first step, then every step runs kSwitchPerStep switching iterations (at
// most 16 n + 4096 in all, the bound of the single solve).
int64_t max_steps_for(int32_t n) {
    return 5 + ceil_div(16ll * n + 4096, kSwitchPerStep);
}

// Served requests of at least this size are solved alone (the solo
// thread of the server) instead of in the batched engine; DGS_SERVER_SOLO_N
// overrides it (0: every request is batched).
int32_t solo_min_n() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_SERVER_SOLO_N");
        const int32_t x = e ? std::atoi(e) : 4096;
        return x > 0 ? x : (1 << 30);
    }();
    return v;
}
bool solo_request(int32_t n) { return n >= solo_min_n(); }

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace
}  // namespace dgs

using namespace dgs;

// ------------------------------------------------------------- batched solve
extern "C" dgs_status dgs_solve_batched(const int32_t* const* benefits, const int32_t* ns, int32_t count,
                                        int32_t* const* sigma_outs, int64_t* objectives_out,
                                        const dgs_options* options, dgs_status* statuses_out,
                                        dgs_stats* stats_out, dgs_stream_t stream) {
    if (count <= 0 || !benefits || !ns || !sigma_outs || !objectives_out) return DGS_ERR_INVALID;
    dgs_options o;
    dgs_default_options(&o);
    if (options) o = *options;
    if (o.init != DGS_INIT_GREEDY && o.init != DGS_INIT_IDENTITY && o.init != DGS_INIT_RANDOM) return DGS_ERR_INVALID;
    if (o.reeval_rule != DGS_REEVAL_BOX && o.reeval_rule != DGS_REEVAL_ALL) return DGS_ERR_INVALID;
    if (o.trace_capacity > 0 || o.algorithm != DGS_ALG_PARALLEL || o.evaluation != DGS_EVAL_TILE_PAIRS)
        return DGS_ERR_INVALID;
    int32_t max_n = 0;
    for (int32_t k = 0; k < count; ++k) {
        if (!benefits[k] || !sigma_outs[k] || ns[k] <= 0 || ns[k] > DGS_BATCH_MAX_N) return DGS_ERR_INVALID;
        max_n = std::max(max_n, ns[k]);
    }
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    Engine eng(count, max_n);
    dgs_status st = eng.init();
    if (st != DGS_OK) return st;
    cudaStream_t s = eng.stream();
    // the private stream starts after the caller's stream
    cudaEvent_t ev = nullptr;
    B_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(s, ev, 0);
    // one allocation for every instance's workspace
    std::vector<size_t> off(count);
    std::vector<char> copy(count);
    size_t total = 0;
    for (int32_t k = 0; k < count; ++k) {
        copy[k] = (ns[k] % 4) != 0 || !aligned16(benefits[k]);
        off[k] = total;
        total += carve_instance(nullptr, ns[k], copy[k] != 0, nullptr);
    }
    // random starts (drawn on the host, one per instance from the same seed)
    // follow the workspaces in the same allocation
    std::vector<int32_t> starts;
    std::vector<size_t> start_off(count, 0);
    if (o.init == DGS_INIT_RANDOM) {
        size_t sum = 0;
        for (int32_t k = 0; k < count; ++k) {
            start_off[k] = sum;
            sum += (size_t)ns[k];
        }
        starts.resize(sum);
        for (int32_t k = 0; k < count; ++k) random_start(ns[k], o.seed, starts.data() + start_off[k]);
    }
    const size_t ws_total = total;
    total += starts.size() * sizeof(int32_t);
    char* mem = nullptr;
    cudaError_t e = pool_malloc_async(reinterpret_cast<void**>(&mem), total, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        cudaEventDestroy(ev);
        snprintf(g_err, sizeof(g_err), "batched workspace of %zu bytes", total);
        set_last_error(g_err);
        return DGS_ERR_OOM;
    }
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return fail(e, "cudaMallocAsync");
    }
    int32_t* d_starts = reinterpret_cast<int32_t*>(mem + ws_total);
    if (!starts.empty()) {
        e = cudaMemcpyAsync(d_starts, starts.data(), starts.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFreeAsync(mem, s);
            cudaEventDestroy(ev);
            return fail(e, "copy random starts");
        }
    }
    for (int32_t k = 0; k < count; ++k) {
        const bool rnd = o.init == DGS_INIT_RANDOM;
        eng.place(k, mem + off[k], ns[k], copy[k] != 0, benefits[k], sigma_outs[k], rnd ? DGS_INIT_USER : o.init,
                  o.max_sweeps, o.deadline_us, rnd ? d_starts + start_off[k] : nullptr,
                  o.reeval_rule == DGS_REEVAL_ALL);
    }
    const int64_t max_steps = max_steps_for(max_n);
    bool all_done = false;
    for (int64_t it = 0; it < max_steps && st == DGS_OK; ++it) {
        st = eng.step();
        if (st != DGS_OK) break;
        all_done = true;
        for (int32_t k = 0; k < count; ++k)
            if (eng.state(k).stage != kStageDone) {
                all_done = false;
                break;
            }
        if (all_done) break;
    }
    cudaFreeAsync(mem, s);
    cudaEventRecord(ev, s);
    cudaStreamWaitEvent(user, ev, 0);
    cudaStreamSynchronize(s);
    cudaEventDestroy(ev);
    if (st != DGS_OK) return st;
    if (!all_done) {
        set_last_error("batched solve did not finish");
        return DGS_ERR_INTERNAL;
    }
    dgs_status first = DGS_OK;
    const int64_t launches = eng.launches_per_step() * eng.steps();
    for (int32_t k = 0; k < count; ++k) {
        const DeviceState& h = eng.state(k);
        const dgs_status sk = status_of(h);
        objectives_out[k] = h.f;
        if (statuses_out) statuses_out[k] = sk;
        if (stats_out) stats_of(h, launches, &stats_out[k]);
        if (first == DGS_OK && sk != DGS_OK) first = sk;
    }
    return first;
}

// ------------------------------------------------------------------- server
// Two host threads: the worker admits requests by budget, places uploaded
// instances into free slots at step boundaries, runs steps and retires
// finished instances; the uploader copies admitted requests' matrices into
// their device memory on its own stream, so copies overlap the steps.
struct dgs_server {
    struct Request {
        uint64_t ticket;
        const int32_t* a;
        int32_t n;
        int32_t flags;
        size_t bytes;
        int64_t submit_ns;
        int32_t init;              // DGS_INIT_* of the request
        int32_t reeval_all;
        const int32_t* init_tau;   // USER start (same memory space as a), or null
        uint64_t seed;
        int32_t max_sweeps;
        int64_t deadline_us;
        int64_t admit_ns;
    };
    struct Uploaded {
        Request r;
        char* mem;
        int64_t upload_ns, ready_ns;
    };
    struct Resident {
        uint64_t ticket = 0;
        char* mem = nullptr;
        size_t bytes = 0;
        int32_t n = 0;
        int32_t* out = nullptr;
        dgs_request_times times{};
    };
    struct Result {
        dgs_status status;
        int64_t objective;
        std::vector<int32_t> sigma;
        dgs_stats stats;
        dgs_request_times times;
    };

    int device = 0;
    size_t budget = 0;
    Engine eng;
    std::vector<Resident> slots;  // worker only
    // uploads of different requests overlap; small requests are uploaded
    // first, and uploader 0 takes only small ones, so that a small request
    // never waits behind the copies of large matrices
    static constexpr int kUploaders = 4;
    static constexpr int kSolo = 3;       // large requests solved at once, each on its own stream
    std::thread worker, uploader[kUploaders], solo[kSolo];
    cudaStream_t up_stream[kUploaders] = {};
    cudaStream_t solo_stream[kSolo] = {};
    // everything below is guarded by mu
    std::mutex mu;
    std::condition_variable cv_work, cv_up, cv_done;
    std::deque<Request> queue;       // waiting for admission
    std::deque<Request> up_small, up_large;  // admitted, matrix not yet on the device
    std::deque<Uploaded> ready;      // on the device, waiting for a slot
    std::deque<Uploaded> solo_ready; // large requests on the device, waiting for the solo thread
    std::condition_variable cv_solo;
    int32_t solo_count = 0;          // large requests admitted, not finished
    bool solo_stop = false;
    std::unordered_map<uint64_t, Result> results;
    std::unordered_map<uint64_t, int32_t> pending;  // ticket -> 0 queued / 1 admitted
    size_t used = 0;                 // budget taken by admitted requests
    int32_t resident_count = 0;      // instances in slots
    int32_t reserved = 0;            // admitted, not yet in a slot
    uint64_t next_ticket = 1;
    bool stop = false;
    dgs_status fatal = DGS_OK;
    int64_t completed = 0, steps = 0, launches = 0;
    double upload_ms = 0.0, step_ms = 0.0;
    int32_t* h_sigma = nullptr;      // pinned staging for results (worker only)
    size_t h_sigma_cap = 0;

    explicit dgs_server(int32_t cap) : eng(cap, DGS_BATCH_MAX_N), slots(cap) {}

    // Layout of a large request's memory: the n x n matrix, the result,
    // the start.
    static size_t solo_bytes(int32_t n) {
        return ((size_t)n * n * 4 + 255) / 256 * 256 + 2 * (((size_t)n * 4 + 255) / 256 * 256);
    }
    static int32_t* solo_out(char* mem, int32_t n) {
        return reinterpret_cast<int32_t*>(mem + ((size_t)n * n * 4 + 255) / 256 * 256);
    }
    static int32_t* solo_start(char* mem, int32_t n) {
        return reinterpret_cast<int32_t*>(reinterpret_cast<char*>(solo_out(mem, n)) +
                                          ((size_t)n * 4 + 255) / 256 * 256);
    }

    // A request's start (n int32) after its workspace and result.
    static int32_t* start_of(char* mem, int32_t n) {
        return reinterpret_cast<int32_t*>(mem + carve_instance(nullptr, n, true, nullptr) +
                                          ((size_t)n * 4 + 255) / 256 * 256);
    }

    void finish_all_pending(dgs_status why) {  // caller holds mu
        for (auto& kv : pending) {
            Result r{};
            r.status = why;
            results[kv.first] = std::move(r);
        }
        pending.clear();
        queue.clear();
        up_small.clear();
        up_large.clear();
    }

    void record_result(uint64_t ticket, Result&& res, size_t bytes) {  // caller holds mu
        used -= bytes;
        pending.erase(ticket);
        results[ticket] = std::move(res);
        ++completed;
    }

    void run_uploader(int u) {
        cudaSetDevice(device);
        cudaStream_t up = up_stream[u];
        for (;;) {
            Request r;
            {
                std::unique_lock<std::mutex> lk(mu);
                const auto any = [&] { return !up_small.empty() || (u != 0 && !up_large.empty()); };
                cv_up.wait(lk, [&] { return stop || any(); });
                if (!any()) return;  // stopping
                std::deque<Request>& q = up_small.empty() ? up_large : up_small;
                r = q.front();
                q.pop_front();
            }
            const int64_t t0 = now_ns();
            const bool solo_req = solo_request(r.n);
            char* mem = nullptr;
            cudaError_t e = pool_malloc_async(reinterpret_cast<void**>(&mem), solo_req ? solo_bytes(r.n) : r.bytes, up);
            if (e == cudaErrorMemoryAllocation) {  // the device has less free memory than the budget
                cudaGetLastError();
                Result res{};
                res.status = DGS_ERR_OOM;
                res.times.submit_ns = r.submit_ns;
                res.times.admit_ns = r.admit_ns;
                res.times.upload_ns = t0;
                res.times.done_ns = now_ns();
                std::lock_guard<std::mutex> lk(mu);
                if (solo_req) --solo_count;
                else --reserved;
                record_result(r.ticket, std::move(res), r.bytes);
                cv_done.notify_all();
                cv_work.notify_one();
                continue;
            }
            if (e == cudaSuccess && solo_req) {
                // the matrix as it is (n x n), then the result and the start;
                // the single solve re-pitches it itself when n % 4 != 0
                const cudaMemcpyKind kind =
                    (r.flags & DGS_SUBMIT_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
                e = cudaMemcpyAsync(mem, r.a, (size_t)r.n * r.n * 4, kind, up);
                int32_t* start = solo_start(mem, r.n);
                std::vector<int32_t> perm;
                if (e == cudaSuccess && r.init == DGS_INIT_USER)
                    e = cudaMemcpyAsync(start, r.init_tau, (size_t)r.n * 4, kind, up);
                if (e == cudaSuccess && r.init == DGS_INIT_RANDOM) {
                    perm.resize(r.n);
                    random_start(r.n, r.seed, perm.data());
                    e = cudaMemcpyAsync(start, perm.data(), (size_t)r.n * 4, cudaMemcpyHostToDevice, up);
                }
                if (e == cudaSuccess) e = cudaStreamSynchronize(up);
            } else if (e == cudaSuccess) {
                // the matrix, pitched (round_up(n, 4)) at the start of its workspace
                Instance probe{};
                carve_instance(mem, r.n, true, &probe);
                const size_t lda = (size_t)probe.w.lda;
                int32_t* a_dev = const_cast<int32_t*>(probe.w.a);
                if (lda != (size_t)r.n) e = cudaMemsetAsync(a_dev, 0, sizeof(int32_t) * lda * r.n, up);
                const cudaMemcpyKind kind =
                    (r.flags & DGS_SUBMIT_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
                const size_t row_bytes = (size_t)r.n * 4;
                if (e == cudaSuccess && lda == (size_t)r.n) {
                    e = cudaMemcpyAsync(a_dev, r.a, row_bytes * r.n, kind, up);
                } else if (e == cudaSuccess && kind == cudaMemcpyHostToDevice) {
                    // a pitched copy from pageable host memory is slow (the
                    // server's uploads took 14 times longer): copy the rows
                    // contiguously into the region of the transpose (n x ldt
                    // >= n^2 ints, written by pass 1 only later), then
                    // re-pitch on the device
                    e = cudaMemcpyAsync(probe.w.at, r.a, row_bytes * r.n, kind, up);
                    if (e == cudaSuccess)
                        e = cudaMemcpy2DAsync(a_dev, lda * 4, probe.w.at, row_bytes, row_bytes, r.n,
                                              cudaMemcpyDeviceToDevice, up);
                } else if (e == cudaSuccess) {
                    e = cudaMemcpy2DAsync(a_dev, lda * 4, r.a, row_bytes, row_bytes, r.n, kind, up);
                }
                // the start (USER: the caller's; RANDOM: drawn here) after the result
                int32_t* start = start_of(mem, r.n);
                std::vector<int32_t> perm;
                if (e == cudaSuccess && r.init == DGS_INIT_USER)
                    e = cudaMemcpyAsync(start, r.init_tau, (size_t)r.n * 4, kind, up);
                if (e == cudaSuccess && r.init == DGS_INIT_RANDOM) {
                    perm.resize(r.n);
                    random_start(r.n, r.seed, perm.data());
                    e = cudaMemcpyAsync(start, perm.data(), (size_t)r.n * 4, cudaMemcpyHostToDevice, up);
                }
                if (e == cudaSuccess) e = cudaStreamSynchronize(up);
            }
            std::lock_guard<std::mutex> lk(mu);
            upload_ms += (now_ns() - t0) * 1e-6;  // summed over the upload threads
            if (e != cudaSuccess) {
                fail(e, "request upload");
                fatal = DGS_ERR_CUDA;
                finish_all_pending(DGS_ERR_CUDA);
                stop = true;
                cv_done.notify_all();
                cv_work.notify_one();
                return;
            }
            if (solo_req) {
                solo_ready.push_back(Uploaded{r, mem, t0, now_ns()});
                cv_solo.notify_one();
            } else {
                ready.push_back(Uploaded{r, mem, t0, now_ns()});
                cv_work.notify_one();
            }
        }
    }

    // Large requests (n >= solo_min_n()) are solved by kSolo threads, each as
    // a single stream-ordered solve on its thread's stream, beside the
    // batched steps of the small ones: a large instance needs many steps of
    // the batched engine (each also steps every other resident instance),
    // while alone it runs the single solve's kernels at full width.
    void run_solo(int u) {
        cudaSetDevice(device);
        cudaStream_t ss = solo_stream[u];
        int32_t* h_solo = nullptr;  // pinned staging for this thread's results
        size_t h_solo_cap = 0;
        struct Release {
            int32_t*& p;
            ~Release() {
                if (p) cudaFreeHost(p);
            }
        } release{h_solo};
        for (;;) {
            Uploaded u;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_solo.wait(lk, [&] { return solo_stop || !solo_ready.empty(); });
                if (solo_ready.empty()) return;
                u = solo_ready.front();
                solo_ready.pop_front();
            }
            const int64_t start_ns = now_ns();
            const int32_t n = u.r.n;
            int32_t* out = solo_out(u.mem, n);
            dgs_options o;
            dgs_default_options(&o);
            const bool given = u.r.init == DGS_INIT_USER || u.r.init == DGS_INIT_RANDOM;
            o.init = given ? DGS_INIT_USER : u.r.init;
            o.init_sigma = given ? solo_start(u.mem, n) : nullptr;
            o.max_sweeps = u.r.max_sweeps;
            o.deadline_us = u.r.deadline_us;
            o.reeval_rule = u.r.reeval_all ? DGS_REEVAL_ALL : DGS_REEVAL_BOX;
            Result res{};
            dgs_status outcome = DGS_OK;
            dgs_status st = solve_for_server(reinterpret_cast<const int32_t*>(u.mem), n, out, &res.objective, &o,
                                             &res.stats, ss, &outcome);
            if (st == DGS_OK && h_solo_cap < (size_t)n) {
                if (h_solo) cudaFreeHost(h_solo);
                h_solo = nullptr;
                h_solo_cap = 0;
                if (cudaMallocHost(&h_solo, sizeof(int32_t) * n) == cudaSuccess) h_solo_cap = n;
                else st = fail(cudaErrorMemoryAllocation, "result staging");
            }
            cudaError_t e = cudaSuccess;
            if (st == DGS_OK) e = cudaMemcpyAsync(h_solo, out, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ss);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ss);
            if (e != cudaSuccess) st = fail(e, "solo result");
            res.status = st == DGS_OK ? outcome : st;
            if (st == DGS_OK && (outcome == DGS_OK || outcome == DGS_TIMEOUT)) res.sigma.assign(h_solo, h_solo + n);
            res.times.submit_ns = u.r.submit_ns;
            res.times.admit_ns = u.r.admit_ns;
            res.times.upload_ns = u.upload_ns;
            res.times.ready_ns = u.ready_ns;
            res.times.start_ns = start_ns;
            res.times.done_ns = now_ns();
            cudaFreeAsync(u.mem, ss);
            {
                std::lock_guard<std::mutex> lk(mu);
                --solo_count;
                if (pending.count(u.r.ticket)) record_result(u.r.ticket, std::move(res), u.r.bytes);
                else used -= u.r.bytes;  // already answered by a fatal error
            }
            cv_done.notify_all();
            cv_work.notify_one();
        }
    }

    void run() {
        cudaSetDevice(device);
        for (;;) {
            std::vector<Uploaded> place_now;
            {
                std::unique_lock<std::mutex> lk(mu);
                // admission in arrival order while the budget and a slot allow
                while (!stop && !queue.empty() &&
                       (solo_request(queue.front().n) || resident_count + reserved < eng.capacity()) &&
                       used + queue.front().bytes <= budget) {
                    Request r = queue.front();
                    queue.pop_front();
                    r.admit_ns = now_ns();
                    used += r.bytes;
                    if (solo_request(r.n)) ++solo_count;
                    else ++reserved;
                    pending[r.ticket] = 1;
                    (solo_request(r.n) ? up_large : up_small).push_back(r);
                    cv_up.notify_all();
                }
                if (resident_count == 0 && ready.empty()) {
                    if (stop && reserved == 0) break;
                    cv_work.wait(lk, [&] {
                        return !ready.empty() || (stop && reserved == 0) ||
                               (!stop && !queue.empty() &&
                                (solo_request(queue.front().n) || resident_count + reserved < eng.capacity()) &&
                                used + queue.front().bytes <= budget);
                    });
                    continue;
                }
                for (Uploaded& u : ready) place_now.push_back(u);
                ready.clear();
            }
            dgs_status st = DGS_OK;
            for (const Uploaded& u : place_now) place(u);
            if (resident_now() > 0) {
                const int64_t t0 = now_ns();
                st = eng.step();
                std::lock_guard<std::mutex> lk(mu);
                step_ms += (now_ns() - t0) * 1e-6;
                steps = eng.steps();
                launches = eng.launches_per_step() * steps;
            }
            if (st == DGS_OK) st = retire_done();
            if (st != DGS_OK) {
                std::lock_guard<std::mutex> lk(mu);
                fatal = st;
                finish_all_pending(st);
                stop = true;
                cv_done.notify_all();
                cv_up.notify_all();
                break;
            }
        }
    }

    int32_t resident_now() {
        std::lock_guard<std::mutex> lk(mu);
        return resident_count;
    }

    void place(const Uploaded& u) {
        bool drop;
        {
            std::lock_guard<std::mutex> lk(mu);
            drop = stop;
            --reserved;
            if (drop) {
                used -= u.r.bytes;
                pending.erase(u.r.ticket);
            } else {
                ++resident_count;
            }
        }
        if (drop) {  // the server is being destroyed: the request is dropped
            cudaFreeAsync(u.mem, eng.stream());
            return;
        }
        const int32_t k = eng.free_slot();
        Resident& R = slots[k];
        R = Resident{};
        R.ticket = u.r.ticket;
        R.n = u.r.n;
        R.bytes = u.r.bytes;
        R.mem = u.mem;
        R.times.submit_ns = u.r.submit_ns;
        R.times.admit_ns = u.r.admit_ns;
        R.times.upload_ns = u.upload_ns;
        R.times.ready_ns = u.ready_ns;
        R.times.start_ns = now_ns();
        R.out = reinterpret_cast<int32_t*>(u.mem + carve_instance(nullptr, u.r.n, true, nullptr));
        const bool given = u.r.init == DGS_INIT_USER || u.r.init == DGS_INIT_RANDOM;
        eng.place(k, R.mem, R.n, true, nullptr, R.out, given ? DGS_INIT_USER : u.r.init, u.r.max_sweeps,
                  u.r.deadline_us, given ? start_of(u.mem, u.r.n) : nullptr, u.r.reeval_all != 0);
    }

    dgs_status retire_done() {
        cudaStream_t s = eng.stream();
        for (int32_t k = 0; k < eng.capacity(); ++k) {
            if (!eng.used(k) || eng.state(k).stage != kStageDone) continue;
            Resident& R = slots[k];
            const DeviceState& h = eng.state(k);
            Result res{};
            res.status = status_of(h);
            res.objective = h.f;
            stats_of(h, eng.launches_per_step() * eng.steps(), &res.stats);
            if (res.status == DGS_OK || res.status == DGS_TIMEOUT) {
                if (h_sigma_cap < (size_t)R.n) {
                    if (h_sigma) cudaFreeHost(h_sigma);
                    h_sigma = nullptr;
                    B_CUDA(cudaMallocHost(&h_sigma, sizeof(int32_t) * R.n), "result staging");
                    h_sigma_cap = R.n;
                }
                B_CUDA(cudaMemcpyAsync(h_sigma, R.out, sizeof(int32_t) * R.n, cudaMemcpyDeviceToHost, s),
                       "read result");
                B_CUDA(cudaStreamSynchronize(s), "read result");
                res.sigma.assign(h_sigma, h_sigma + R.n);
            }
            res.times = R.times;
            res.times.done_ns = now_ns();
            cudaFreeAsync(R.mem, s);
            eng.vacate(k);
            {
                std::lock_guard<std::mutex> lk(mu);
                --resident_count;
                record_result(R.ticket, std::move(res), R.bytes);
            }
            cv_done.notify_all();
            cv_work.notify_one();
            R = Resident{};
        }
        return DGS_OK;
    }
};

namespace {
size_t request_bytes(int32_t n) {
    // workspace with the pitched matrix, then the result, then the start
    return carve_instance(nullptr, n, true, nullptr) + 2 * (((size_t)n * 4 + 255) / 256 * 256);
}

dgs_status take_result(dgs_server* sv, uint64_t ticket, int32_t* sigma_out_host, int64_t* objective_out,
                       dgs_stats* stats, dgs_request_times* times) {
    auto it = sv->results.find(ticket);
    dgs_server::Result& r = it->second;
    const dgs_status st = r.status;
    if (st == DGS_OK || st == DGS_TIMEOUT) {
        if (sigma_out_host) memcpy(sigma_out_host, r.sigma.data(), sizeof(int32_t) * r.sigma.size());
        if (objective_out) *objective_out = r.objective;
    }
    if (stats) *stats = r.stats;
    if (times) *times = r.times;
    sv->results.erase(it);
    return st;
}
}  // namespace

extern "C" {

size_t dgs_server_request_bytes(int32_t n) {
    if (n <= 0 || n > DGS_BATCH_MAX_N) return 0;
    return request_bytes(n);
}

dgs_status dgs_server_create(size_t budget_bytes, int32_t max_resident, dgs_server** out) {
    if (!out || budget_bytes == 0) return DGS_ERR_INVALID;
    *out = nullptr;
    const int32_t cap = max_resident > 0 ? max_resident : 256;
    dgs_server* sv = new dgs_server(cap);
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e != cudaSuccess) {
        delete sv;
        return fail(e, "cudaGetDevice");
    }
    sv->budget = budget_bytes;
    dgs_status st = sv->eng.init();
    if (st != DGS_OK) {
        delete sv;
        return st;
    }
    for (int u = 0; u < dgs_server::kUploaders && e == cudaSuccess; ++u)
        e = cudaStreamCreateWithFlags(&sv->up_stream[u], cudaStreamNonBlocking);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int u = 0; u < dgs_server::kSolo && e == cudaSuccess; ++u)
        e = cudaStreamCreateWithPriority(&sv->solo_stream[u], cudaStreamNonBlocking, least);
    if (e != cudaSuccess) {
        for (int u = 0; u < dgs_server::kUploaders; ++u)
            if (sv->up_stream[u]) cudaStreamDestroy(sv->up_stream[u]);
        for (int u = 0; u < dgs_server::kSolo; ++u)
            if (sv->solo_stream[u]) cudaStreamDestroy(sv->solo_stream[u]);
        delete sv;
        return fail(e, "upload stream");
    }
    for (int u = 0; u < dgs_server::kSolo; ++u) sv->solo[u] = std::thread([sv, u] { sv->run_solo(u); });
    sv->worker = std::thread([sv] { sv->run(); });
    for (int u = 0; u < dgs_server::kUploaders; ++u) sv->uploader[u] = std::thread([sv, u] { sv->run_uploader(u); });
    *out = sv;
    return DGS_OK;
}

dgs_status dgs_submit(dgs_server* sv, const int32_t* benefit, int32_t n, int32_t flags, uint64_t* ticket) {
    return dgs_submit_ex(sv, benefit, n, flags, nullptr, ticket);
}

dgs_status dgs_submit_ex(dgs_server* sv, const int32_t* benefit, int32_t n, int32_t flags,
                         const dgs_options* options, uint64_t* ticket) {
    if (!sv || !benefit || !ticket || n <= 0 || n > DGS_BATCH_MAX_N) return DGS_ERR_INVALID;
    dgs_options o;
    dgs_default_options(&o);
    if (options) o = *options;
    if (o.init != DGS_INIT_GREEDY && o.init != DGS_INIT_RANDOM && o.init != DGS_INIT_IDENTITY &&
        o.init != DGS_INIT_USER)
        return DGS_ERR_INVALID;
    if (o.init == DGS_INIT_USER && o.init_sigma == nullptr) return DGS_ERR_INVALID;
    if (o.reeval_rule != DGS_REEVAL_BOX && o.reeval_rule != DGS_REEVAL_ALL) return DGS_ERR_INVALID;
    if (o.algorithm != DGS_ALG_PARALLEL || o.trace_capacity > 0 || o.evaluation != DGS_EVAL_TILE_PAIRS)
        return DGS_ERR_INVALID;
    const size_t bytes = request_bytes(n);
    if (bytes > sv->budget) return DGS_ERR_BUSY;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return sv->fatal != DGS_OK ? sv->fatal : DGS_ERR_INVALID;
    const uint64_t t = sv->next_ticket++;
    dgs_server::Request r{t, benefit, n, flags, bytes, now_ns()};
    r.init = o.init;
    r.reeval_all = o.reeval_rule == DGS_REEVAL_ALL ? 1 : 0;
    r.init_tau = o.init == DGS_INIT_USER ? o.init_sigma : nullptr;
    r.seed = o.seed;
    r.max_sweeps = o.max_sweeps;
    r.deadline_us = o.deadline_us;
    sv->queue.push_back(r);
    sv->pending[t] = 0;
    *ticket = t;
    sv->cv_work.notify_one();
    return DGS_OK;
}

dgs_status dgs_poll(dgs_server* sv, uint64_t ticket, int32_t* sigma_out_host, int64_t* objective_out,
                    dgs_stats* stats, dgs_request_times* times) {
    if (!sv) return DGS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->results.count(ticket)) return take_result(sv, ticket, sigma_out_host, objective_out, stats, times);
    return sv->pending.count(ticket) ? DGS_PENDING : DGS_ERR_INVALID;
}

dgs_status dgs_server_wait(dgs_server* sv, uint64_t ticket, int64_t timeout_us, int32_t* sigma_out_host,
                           int64_t* objective_out, dgs_stats* stats, dgs_request_times* times) {
    if (!sv) return DGS_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto ready = [&] { return sv->results.count(ticket) || !sv->pending.count(ticket); };
    if (timeout_us < 0) sv->cv_done.wait(lk, ready);
    else sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (sv->results.count(ticket)) return take_result(sv, ticket, sigma_out_host, objective_out, stats, times);
    return sv->pending.count(ticket) ? DGS_PENDING : DGS_ERR_INVALID;
}

dgs_status dgs_cancel(dgs_server* sv, uint64_t ticket) {
    if (!sv) return DGS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto p = sv->pending.find(ticket);
    if (p == sv->pending.end()) return DGS_ERR_INVALID;  // unknown, or already finished
    if (p->second != 0) return DGS_PENDING;               // admitted: it runs to its end
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        if (it->ticket != ticket) continue;
        dgs_server::Result r{};
        r.status = DGS_CANCELLED;
        r.times.submit_ns = it->submit_ns;
        sv->queue.erase(it);
        sv->pending.erase(p);
        sv->results[ticket] = std::move(r);
        sv->cv_done.notify_all();
        sv->cv_work.notify_one();  // the next request may fit now
        return DGS_OK;
    }
    return DGS_PENDING;
}

dgs_status dgs_server_get_info(dgs_server* sv, dgs_server_info* info) {
    if (!sv || !info) return DGS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    info->resident = sv->resident_count;
    info->queued = (int32_t)sv->queue.size();
    info->steps = sv->steps;
    info->completed = sv->completed;
    info->bytes_in_use = sv->used;
    info->kernel_launches = sv->launches;
    info->upload_ms = sv->upload_ms;
    info->step_ms = sv->step_ms;
    return sv->fatal;
}

void dgs_server_destroy(dgs_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->queue.clear();
        for (auto* q : {&sv->up_small, &sv->up_large}) {  // admitted, never uploaded: dropped
            for (const auto& r : *q) {
                sv->used -= r.bytes;
                if (solo_request(r.n)) --sv->solo_count;
                else --sv->reserved;
            }
            q->clear();
        }
    }
    sv->cv_up.notify_all();
    sv->cv_work.notify_all();
    for (auto& t : sv->uploader)
        if (t.joinable()) t.join();
    {  // no more large requests arrive: the solo thread finishes those it has
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->solo_stop = true;
    }
    sv->cv_solo.notify_all();
    for (auto& t : sv->solo)
        if (t.joinable()) t.join();
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->h_sigma) cudaFreeHost(sv->h_sigma);
    for (int u = 0; u < dgs_server::kSolo; ++u)
        if (sv->solo_stream[u]) cudaStreamDestroy(sv->solo_stream[u]);
    for (int u = 0; u < dgs_server::kUploaders; ++u)
        if (sv->up_stream[u]) cudaStreamDestroy(sv->up_stream[u]);
    delete sv;
}

}  // extern "C"
