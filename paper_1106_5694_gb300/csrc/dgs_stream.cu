// dgs_stream.cu -- what keeps the solve entry points stream-ordered: loops
// that run on the device as CUDA graphs with conditional WHILE nodes (the
// host never waits for a sweep), pinned staging for host-side outputs, and
// the classification of result pointers.
//
// The paper's all-GPU variant avoids host-device crossings inside the
// switching loop (Section 6 attributes the loss of its mixed CPU-GPU variant
// to them); here the loop's continuation is decided by the last kernel of
// each iteration on the device, and a call returns once its work is queued.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/dgs.h"
#include "dgs_internal.cuh"

namespace dgs {
namespace {

// Capture streams, per device, reused across calls (a capture stream holds
// no work: it only records launches into a graph).
std::mutex g_cap_mutex;
std::vector<cudaStream_t> g_cap_free[64];

struct CaptureStream {
    cudaStream_t s = nullptr;
    int dev = -1;
    cudaError_t acquire() {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        {
            std::lock_guard<std::mutex> lock(g_cap_mutex);
            if (!g_cap_free[dev].empty()) {
                s = g_cap_free[dev].back();
                g_cap_free[dev].pop_back();
                return cudaSuccess;
            }
        }
        return cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    }
    ~CaptureStream() {
        if (s == nullptr) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;  // a capture left open by an error path
            if (cudaStreamEndCapture(s, &g) == cudaSuccess && g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
        std::lock_guard<std::mutex> lock(g_cap_mutex);
        g_cap_free[dev].push_back(s);
    }
};

dgs_status fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    set_last_error(buf);
    cudaGetLastError();
    return DGS_ERR_CUDA;
}

// Pinned staging cache: free blocks by size class (powers of two from 4 KB).
std::mutex g_pin_mutex;
std::map<size_t, std::vector<void*>> g_pin_free;

size_t pin_class(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
}

}  // namespace

dgs_status create_loop_handle(cudaStream_t capturing, unsigned long long* handle) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(capturing, &cst, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return fail(e, "capture info");
    if (cst != cudaStreamCaptureStatusActive || g == nullptr) return fail(cudaErrorStreamCaptureInvalidated, "capture");
    cudaGraphConditionalHandle h = 0;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail(e, "loop condition");
    *handle = (unsigned long long)h;
    return DGS_OK;
}

dgs_status capture_while(cudaStream_t capturing, LoopBody body, void* ctx, unsigned long long handle) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(capturing, &cst, nullptr, &g, &deps, &edata, &nd);
    if (e != cudaSuccess) return fail(e, "capture info");
    if (cst != cudaStreamCaptureStatusActive || g == nullptr) return fail(cudaErrorStreamCaptureInvalidated, "capture");
    cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)handle;
    if (h == 0) {
        e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return fail(e, "loop condition");
    }
    // (the struct holds a union without a default constructor: zeroed storage)
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(raw);
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, edata, nd, &p);
    if (e != cudaSuccess) return fail(e, "loop node");
    e = cudaStreamUpdateCaptureDependencies(capturing, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return fail(e, "loop node order");
    CaptureStream cs;
    e = cs.acquire();
    if (e != cudaSuccess) return fail(e, "capture stream");
    cudaGraph_t bg = p.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs.s, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e, "loop body capture");
    const dgs_status st = body(ctx, cs.s, (unsigned long long)h);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs.s, &out);
    if (st != DGS_OK) return st;
    if (e != cudaSuccess) return fail(e, "loop body capture");
    return DGS_OK;
}

namespace {
struct GraphHolder {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    ~GraphHolder() {
        if (x) cudaGraphExecDestroy(x);  // freed when its launches complete
        if (g) cudaGraphDestroy(g);
    }
};

// Executable loop graphs kept for reuse, keyed by the device, the body and
// the bytes of everything its launches were captured with: a call whose
// kernels would get the very same arguments launches the kept graph (its
// launches are ordered behind the previous ones of the same graph).
struct CachedLoop {
    int dev = -1;
    LoopBody body = nullptr;
    std::vector<unsigned char> key;
    GraphHolder* graph = nullptr;
    uint64_t used = 0;
};
constexpr size_t kLoopCacheSize = 16;
std::mutex g_loop_mutex;
std::vector<CachedLoop> g_loop_cache;
uint64_t g_loop_clock = 0;

dgs_status build_loop(LoopBody body, void* ctx, GraphHolder* hd) {
    cudaError_t e = cudaGraphCreate(&hd->g, 0);
    if (e != cudaSuccess) return fail(e, "graph");
    CaptureStream cs;
    e = cs.acquire();
    if (e != cudaSuccess) return fail(e, "capture stream");
    e = cudaStreamBeginCaptureToGraph(cs.s, hd->g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e, "loop capture");
    const dgs_status st = capture_while(cs.s, body, ctx);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs.s, &out);
    if (st != DGS_OK) return st;
    if (e != cudaSuccess) return fail(e, "loop capture");
    e = cudaGraphInstantiate(&hd->x, hd->g, 0);
    if (e != cudaSuccess) return fail(e, "loop graph instantiation");
    return DGS_OK;
}
}  // namespace

dgs_status enqueue_while_cached(cudaStream_t s, LoopBody body, void* ctx, const void* key, size_t key_bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e, "device");
    const unsigned char* kb = static_cast<const unsigned char*>(key);
    {
        std::lock_guard<std::mutex> lock(g_loop_mutex);
        for (CachedLoop& c : g_loop_cache) {
            if (c.dev != dev || c.body != body || c.key.size() != key_bytes ||
                memcmp(c.key.data(), kb, key_bytes) != 0)
                continue;
            c.used = ++g_loop_clock;
            e = cudaGraphLaunch(c.graph->x, s);
            if (e != cudaSuccess) return fail(e, "loop graph launch");
            return DGS_OK;
        }
    }
    GraphHolder* hd = new GraphHolder();
    const dgs_status st = build_loop(body, ctx, hd);
    if (st != DGS_OK) {
        delete hd;
        return st;
    }
    std::lock_guard<std::mutex> lock(g_loop_mutex);
    e = cudaGraphLaunch(hd->x, s);
    if (e != cudaSuccess) {
        delete hd;
        return fail(e, "loop graph launch");
    }
    if (g_loop_cache.size() >= kLoopCacheSize) {  // the least recently used goes (freed when done)
        size_t lru = 0;
        for (size_t i = 1; i < g_loop_cache.size(); ++i)
            if (g_loop_cache[i].used < g_loop_cache[lru].used) lru = i;
        delete g_loop_cache[lru].graph;
        g_loop_cache.erase(g_loop_cache.begin() + (long)lru);
    }
    CachedLoop c;
    c.dev = dev;
    c.body = body;
    c.key.assign(kb, kb + key_bytes);
    c.graph = hd;
    c.used = ++g_loop_clock;
    g_loop_cache.push_back(std::move(c));
    return DGS_OK;
}

dgs_status enqueue_while(cudaStream_t s, LoopBody body, void* ctx) {
    GraphHolder hd;
    cudaError_t e = cudaGraphCreate(&hd.g, 0);
    if (e != cudaSuccess) return fail(e, "graph");
    CaptureStream cs;
    e = cs.acquire();
    if (e != cudaSuccess) return fail(e, "capture stream");
    e = cudaStreamBeginCaptureToGraph(cs.s, hd.g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e, "loop capture");
    const dgs_status st = capture_while(cs.s, body, ctx);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs.s, &out);
    if (st != DGS_OK) return st;
    if (e != cudaSuccess) return fail(e, "loop capture");
    e = cudaGraphInstantiate(&hd.x, hd.g, 0);
    if (e != cudaSuccess) return fail(e, "loop graph instantiation");
    e = cudaGraphLaunch(hd.x, s);
    if (e != cudaSuccess) return fail(e, "loop graph launch");
    return DGS_OK;
}

void* pinned_get(size_t bytes) {
    const size_t c = pin_class(bytes);
    {
        std::lock_guard<std::mutex> lock(g_pin_mutex);
        auto it = g_pin_free.find(c);
        if (it != g_pin_free.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            return p;
        }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_put(void* p, size_t bytes) {
    if (p == nullptr) return;
    std::lock_guard<std::mutex> lock(g_pin_mutex);
    g_pin_free[pin_class(bytes)].push_back(p);
}

bool device_writable(const void* p, void** alias) {
    cudaPointerAttributes at;
    memset(&at, 0, sizeof(at));
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        *alias = const_cast<void*>(p);
        return true;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) {
        *alias = at.devicePointer;
        return true;
    }
    return false;
}

}  // namespace dgs
