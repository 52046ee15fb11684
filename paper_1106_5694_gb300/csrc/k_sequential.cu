// k_sequential.cu -- Algorithm 1 (sequential DGS, Section 3.3): one switch per
// iteration, chosen as the largest delta over all agent and job slots.
//
// One CTA runs the while loop of one pass on the device.  Every iteration:
//   * i* = argmax_i delta-bar_i, j* = argmax_j delta-underbar_j (ties to the
//     lowest index); the agent slot wins only when its delta is strictly
//     larger; that slot's delta is zeroed;
//   * the exchange switch(i, j, sigma): agent i takes job j from its holder
//     sigma(j) in the current assignment; it is committed when it raises f;
//   * after a commit, ADE of the two agents and JDE of the two jobs are run
//     again.  The two agents now hold the two jobs, so both are rows of G
//     (G[j][k] = a[sigma(j)][k] + a[sigma(k)][j] - D[j] - D[k]): row j gives
//     the ADE of its holder (ties: lowest job k) and the JDE of job j (ties:
//     lowest partner agent sigma(k)).
// The slot deltas live in shared memory (n <= kSeqSmemMaxN) or in the
// workspace's slot arrays.  The outer repeat (a fresh evaluation of every
// slot, then the loop again until a pass leaves f unchanged) runs as a
// device-side loop of passes.
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kSeqThreads = 1024;
constexpr int32_t kSeqSmemMaxN = 25600;  // 2 deltas of 4 bytes per index in shared memory
constexpr int32_t kSeqItersPerLaunch = 1 << 20;

// CTA-wide maximum of one 64-bit key per thread (1024 threads).
__device__ __forceinline__ unsigned long long block_max(unsigned long long x, unsigned long long* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = umax64(x, __shfl_xor_sync(0xffffffffu, x, off));
    __syncthreads();  // red is free again
    if (lane == 0) red[warp] = x;
    __syncthreads();
    x = red[lane];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = umax64(x, __shfl_xor_sync(0xffffffffu, x, off));
    return x;
}

// Full evaluation of row j of G: the packed (gain, ~lowest column) and
// (gain, ~lowest partner agent) keys of its best strictly positive gain.
__device__ __forceinline__ void row_keys(const Workspace& w, int32_t j, unsigned long long* red,
                                         unsigned long long* ka_out, unsigned long long* kj_out) {
    const int32_t n = w.n;
    const int32_t sj = w.sigma[j], dj = w.diag[j];
    const int32_t* arow = w.a + (size_t)sj * w.lda;
    const int32_t* atrow = w.at + (size_t)j * w.ldt;
    int32_t bg = 0, bc = -1, bs = 0x7fffffff;
    for (int32_t k = threadIdx.x; k < n; k += kSeqThreads) {
        const int32_t sk = w.sigma[k];
        const int32_t g = arow[k] + atrow[sk] - dj - w.diag[k];
        const bool gt = g > bg, eq = g == bg;
        bs = gt ? sk : (eq ? min(bs, sk) : bs);
        bc = gt ? k : bc;  // k ascending in this thread: the first maximum is the lowest
        bg = max(bg, g);
    }
    const unsigned long long ka = block_max(bg > 0 ? pack_gain(bg, (uint32_t)bc) : 0ull, red);
    const unsigned long long kj = block_max(bg > 0 ? pack_gain(bg, (uint32_t)bs) : 0ull, red);
    *ka_out = ka;
    *kj_out = kj;
}

__global__ void __launch_bounds__(kSeqThreads, 1) sequential_kernel(Workspace w, int32_t smem_deltas) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    extern __shared__ __align__(16) int32_t s_delta[];  // [0, n): delta-bar, [n, 2n): delta-underbar
    __shared__ unsigned long long red[32];
    __shared__ int32_t s_stop, s_u, s_v, s_target;
    __shared__ long long s_gain;
    const int32_t n = w.n, tid = threadIdx.x;
    int32_t* dbar = smem_deltas ? s_delta : w.ag_gain;
    int32_t* dund = smem_deltas ? s_delta + n : w.jb_gain;
    if (smem_deltas) {
        for (int32_t i = tid; i < n; i += kSeqThreads) {
            dbar[i] = w.ag_gain[i];
            dund[i] = w.jb_gain[i];
        }
    }
    __syncthreads();
    const int32_t max_iters = st->max_sweeps;
    const uint64_t deadline = st->deadline_ns;
    for (int32_t it = 0; it < kSeqItersPerLaunch; ++it) {
        // i* and j*: largest delta, lowest index
        unsigned long long ba = 0ull, bj = 0ull;
        for (int32_t i = tid; i < n; i += kSeqThreads) {
            const int32_t da = dbar[i], dj = dund[i];
            if (da > 0) ba = umax64(ba, pack_gain(da, (uint32_t)i));
            if (dj > 0) bj = umax64(bj, pack_gain(dj, (uint32_t)i));
        }
        ba = block_max(ba, red);
        bj = block_max(bj, red);
        if (tid == 0) {
            int32_t stop = 0;
            if (ba == 0ull && bj == 0ull) {
                stop = 1;  // the while loop of this pass has ended
            } else if ((max_iters > 0 && st->sweeps >= max_iters) ||
                       (deadline != 0 && globaltimer_ns() > deadline)) {
                st->status = kTimeout;
                stop = 1;
            } else {
                const int32_t ga = ba ? key_gain(ba) : 0, gj = bj ? key_gain(bj) : 0;
                if (ga > gj) {
                    const int32_t i = key_index(ba);
                    dbar[i] = 0;
                    s_target = w.ag_job[i];
                    s_u = i;
                    s_v = w.sigma[s_target];
                } else {
                    const int32_t j = key_index(bj);
                    dund[j] = 0;
                    s_target = w.jb_agent[j];
                    s_u = s_target;
                    s_v = w.sigma[j];
                }
                const int32_t u = s_u, v = s_v;
                const int32_t ju = w.tau[u], jv = w.tau[v];
                s_gain = (long long)w.a[(size_t)u * w.lda + jv] + w.a[(size_t)v * w.lda + ju] - w.diag[ju] - w.diag[jv];
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        const int32_t u = s_u, v = s_v;
        const bool applied = s_gain > 0;
        if (applied) {
            if (tid == 0) {
                const int32_t ju = w.tau[u], jv = w.tau[v];
                const int32_t x1 = w.a[(size_t)u * w.lda + jv], x2 = w.a[(size_t)v * w.lda + ju];
                w.tau[u] = jv;
                w.tau[v] = ju;
                w.sigma[jv] = u;
                w.sigma[ju] = v;
                w.diag[jv] = x1;
                w.diag[ju] = x2;
                st->f += s_gain;
                st->swaps += 1;
            }
            __syncthreads();  // the new assignment is visible to the CTA
            // ADE of u and v, JDE of their (new) jobs: rows tau(u), tau(v) of G
            const int32_t rows[2] = {w.tau[u], w.tau[v]};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int32_t j = rows[q];
                unsigned long long ka, kj;
                row_keys(w, j, red, &ka, &kj);
                if (tid == 0) {
                    const int32_t holder = w.sigma[j];
                    dbar[holder] = ka ? key_gain(ka) : 0;
                    w.ag_job[holder] = ka ? key_index(ka) : -1;
                    dund[j] = kj ? key_gain(kj) : 0;
                    w.jb_agent[j] = kj ? key_index(kj) : -1;
                }
            }
        }
        if (tid == 0) {
            const int32_t s = st->sweeps;
            if (s < st->trace_capacity) {
                if (st->trace_accepted) st->trace_accepted[s] = 1;
                if (st->trace_applied) st->trace_applied[s] = applied ? 1 : 0;
                if (st->trace_objective) st->trace_objective[s] = st->f;
            }
            st->sweeps = s + 1;
            if (applied) st->events += 1;
        }
        __syncthreads();
    }
    // the loop ended (or this launch reached its iteration budget: need_update
    // makes the loop condition launch it again)
    if (tid == 0) st->need_update = s_stop ? 0 : 1;
    if (smem_deltas) {
        __syncthreads();
        for (int32_t i = tid; i < n; i += kSeqThreads) {
            w.ag_gain[i] = dbar[i];
            w.jb_gain[i] = dund[i];
        }
    }
}

// Slots of a fresh evaluation: agent slot i <- key_a[tau(i)], job slot j <-
// key_j[j] (gains and targets in the workspace's slot arrays).
__global__ void slots_from_keys_kernel(Workspace w) {
    if (w.st->status != kRunning) return;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < w.n; t += gridDim.x * blockDim.x) {
        const unsigned long long ka = w.key_a[w.tau[t]];
        w.ag_gain[t] = ka ? key_gain(ka) : 0;
        w.ag_job[t] = ka ? key_index(ka) : -1;
        const unsigned long long kj = w.key_j[t];
        w.jb_gain[t] = kj ? key_gain(kj) : 0;
        w.jb_agent[t] = kj ? key_index(kj) : -1;
    }
}

// Device-side passes of Algorithm 1 (conditional WHILE graph nodes): each
// pass begins by recording f and re-arming the switching loop, the loop runs
// while a launch stops at its iteration budget (need_update), and the passes
// go on while a pass changed f (the outer repeat).  Bounds: 4 n + 16 passes,
// 64 launches of the switching loop per pass (internal error beyond).
__global__ void seq_pass_begin_kernel(Workspace w, unsigned long long inner) {
    DeviceState* st = w.st;
    st->f_pass = st->f;
    st->seq_inner = 0;
    st->loop_launches += 3;  // this kernel, the evaluation, the slots
    if (st->status == kRunning && ++st->seq_passes > 4 * w.n + 16) {
        st->error = kErrInternal;
        st->status = kError;
    }
    cudaGraphSetConditional(inner, st->status == kRunning ? 1u : 0u);
}

__global__ void seq_inner_cond_kernel(Workspace w, unsigned long long inner) {
    DeviceState* st = w.st;
    st->loop_launches += 2;  // the switching loop and this kernel
    if (st->status == kRunning && st->need_update && ++st->seq_inner > 64) {
        st->error = kErrInternal;
        st->status = kError;
    }
    cudaGraphSetConditional(inner, (st->status == kRunning && st->need_update) ? 1u : 0u);
}

__global__ void seq_pass_end_kernel(Workspace w, unsigned long long outer) {
    DeviceState* st = w.st;
    st->loop_launches += 1;
    cudaGraphSetConditional(outer, (st->status == kRunning && st->f != st->f_pass) ? 1u : 0u);
}

}  // namespace

cudaError_t launch_seq_pass_begin(const Workspace& w, unsigned long long inner, cudaStream_t s) {
    seq_pass_begin_kernel<<<1, 1, 0, s>>>(w, inner);
    return cudaGetLastError();
}
cudaError_t launch_seq_inner_cond(const Workspace& w, unsigned long long inner, cudaStream_t s) {
    seq_inner_cond_kernel<<<1, 1, 0, s>>>(w, inner);
    return cudaGetLastError();
}
cudaError_t launch_seq_pass_end(const Workspace& w, unsigned long long outer, cudaStream_t s) {
    seq_pass_end_kernel<<<1, 1, 0, s>>>(w, outer);
    return cudaGetLastError();
}

cudaError_t launch_slots_from_keys(const Workspace& w, cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > dgs::device_sms() * 4) grid = dgs::device_sms() * 4;
    slots_from_keys_kernel<<<grid, 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_sequential(const Workspace& w, cudaStream_t s) {
    const int32_t in_smem = w.n <= kSeqSmemMaxN ? 1 : 0;
    const size_t smem = in_smem ? 8 * (size_t)w.n : 0;
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(sequential_kernel), 9, smem);
        if (e != cudaSuccess) return e;
    }
    sequential_kernel<<<1, kSeqThreads, smem, s>>>(w, in_smem);
    return cudaGetLastError();
}

}  // namespace dgs
