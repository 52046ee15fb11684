// dgs_static.cu -- dgs_evaluate_static: the full difference evaluation with
// all of its working memory in one fixed array that is part of the library's
// device image, so that the call allocates nothing.
//
// The array lives at file scope below.  Its name, used in host code, is only
// a host-side stand-in for the device object: handing it to a kernel would
// make the kernel read the wrong memory or fault.  Each call obtains the
// device address with cudaGetSymbolAddress, with the call's device current,
// and passes that address to the kernels.
//
// Every call reuses the same array and leaves its contents behind; the parts
// that must start at zero (row keys, the assignment, the permutation check,
// the loop state) are cleared on each call.  Two calls whose work overlaps on
// the GPU (different streams, different host threads) race on the array and
// must be serialised by the caller.
//
// The array is device memory of this library's module.  With lazy module
// loading (the toolkit's default) the module, and with it the array, is
// loaded and committed on a device the first time the library needs it
// there, which may be inside the first call of this entry point: that first
// call can therefore fail for lack of device memory, and callers that must
// not allocate make it during their set-up (or run with
// CUDA_MODULE_LOADING=EAGER, which commits the array when the library's
// context is created).  The address is looked up on every call (a cheap
// query), so it stays right after a cudaDeviceReset reloads the module.
#include <cstdio>

#include "../../include/dgs.h"
#include "dgs_internal.cuh"

namespace {

using namespace dgs;

constexpr int32_t kStaticMaxN = DGS_STATIC_MAX_N;

// Byte offsets of each array inside the static block (each 256-B aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffSigma = 0;
constexpr size_t kOffTau = kOffSigma + align256(4 * (size_t)kStaticMaxN);
constexpr size_t kOffDiag = kOffTau + align256(4 * (size_t)kStaticMaxN);
constexpr size_t kOffKeyA = kOffDiag + align256(4 * (size_t)kStaticMaxN);
constexpr size_t kOffKeyJ = kOffKeyA + align256(8 * (size_t)kStaticMaxN);
constexpr size_t kOffSeen = kOffKeyJ + align256(8 * (size_t)kStaticMaxN);
constexpr size_t kOffState = kOffSeen + align256(4 * (size_t)kStaticMaxN);
constexpr size_t kStaticBytes = kOffState + align256(sizeof(DeviceState));

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch on the current device.
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

__global__ void static_state_kernel(DeviceState* st) {
    *st = DeviceState{};
    st->status = kRunning;
}


}  // namespace

extern "C" DGS_API dgs_status dgs_evaluate_static(const int32_t* benefit, int32_t n, const int32_t* sigma_in,
                                                  int32_t* agent_gain, int32_t* agent_job, int32_t* job_gain,
                                                  int32_t* job_agent, dgs_stream_t stream) {
    if (!benefit || !sigma_in || !agent_gain || !agent_job || !job_gain || !job_agent || n <= 0)
        return DGS_ERR_INVALID;
    char why[160];
    if (n > kStaticMaxN) {
        snprintf(why, sizeof(why), "dgs_evaluate_static: n=%d exceeds DGS_STATIC_MAX_N=%d", n, kStaticMaxN);
        set_last_error(why);
        return DGS_ERR_INVALID;
    }
    if (n % 4 != 0 || reinterpret_cast<uintptr_t>(benefit) % 16 != 0) {
        snprintf(why, sizeof(why), "dgs_evaluate_static: n=%d must be a multiple of 4 and benefit 16-byte aligned",
                 n);
        set_last_error(why);
        return DGS_ERR_INVALID;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DGS_ERR_CUDA;
    }
    Workspace w{};
    w.a = benefit;
    w.n = n;
    w.lda = n;
    w.ldt = 0;
    w.sigma = reinterpret_cast<int32_t*>(base + kOffSigma);
    w.tau = reinterpret_cast<int32_t*>(base + kOffTau);
    w.diag = reinterpret_cast<int32_t*>(base + kOffDiag);
    w.key_a = reinterpret_cast<unsigned long long*>(base + kOffKeyA);
    w.key_j = reinterpret_cast<unsigned long long*>(base + kOffKeyJ);
    uint8_t* seen = base + kOffSeen;
    w.exact_keys = env_exact_keys();
    w.st = reinterpret_cast<DeviceState*>(base + kOffState);

    // what must start at zero: row keys, the assignment (so that the outputs
    // of a failed call never show another call's keys), the permutation
    // check, the loop state
    e = cudaMemsetAsync(w.key_a, 0, kOffSeen - kOffKeyA, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.tau, 0, 4 * (size_t)kStaticMaxN, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(seen, 0, 4 * (size_t)n, s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DGS_ERR_CUDA;
    }
    static_state_kernel<<<1, 1, 0, s>>>(w.st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_range_check(w, s);
    if (e == cudaSuccess) e = launch_start_from_tau(w, sigma_in, DGS_INIT_USER, seen, s);
    if (e == cudaSuccess) e = launch_full_evaluation(w, 0, s);
    if (e == cudaSuccess) e = launch_keys_to_slots(w, agent_gain, agent_job, job_gain, job_agent, s);
    DeviceState h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, w.st, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DGS_ERR_CUDA;
    }
    return map_device_status(h);
}
