// k_control.cu -- the switching loop of Algorithm 3 (Section 5) on the GPU.
//
// Slots.  Agent slot i (priority t = i) holds agent i's candidate (gain,
// job j_i); job slot j (priority t = n + j) holds job j's candidate (gain,
// agent i_j).  A slot with gain > 0 proposes the 2-exchange of the agent
// pair {i, sigma(j_i)} or {sigma(j), i_j} (partners looked up in the current
// sigma); such slots are the edges of the conflict check.
//
// One sweep = CC (Algorithm 4) + parallel switch + re-evaluation:
//   * CC claims agent pairs in priority order.  Its result (the priority
//     greedy matching of the edges) is computed exactly by deterministic
//     reservations: every live edge writes its priority into both agents
//     with atomicMin; an edge holding both agents is accepted; live edges
//     touching a claimed agent are rejected (they form the set C, reading R3);
//     repeat until no edge is live.  An accepted edge has no earlier accepted
//     neighbour and every rejected edge has one, which is exactly the
//     sequential outcome.
//   * Accepted exchanges are agent-disjoint, so each commits independently
//     when its gain under the current sigma is > 0.
//   * Slots not in C are re-evaluated (reading R4) by reading the row-best
//     keys key_a / key_j, which the update kernels keep equal to a fresh
//     evaluation of every row under the current sigma.
//
// The controller is one CTA that keeps running sweeps while they commit
// nothing (sigma, hence every row best, is then unchanged and re-evaluation
// is a read of the keys).  A sweep that commits exchanges stops it: the
// update kernels re-evaluate the affected rows on the whole GPU, then the
// controller is launched again and refreshes every slot not in C.
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kCtlThreads = 1024;
constexpr int32_t kInf = 0x7fffffff;
enum : uint8_t { kDead = 0, kLive = 1, kAcc = 2, kRej = 3 };

__device__ __forceinline__ int32_t exchange_gain(const Workspace& w, int32_t u, int32_t v) {
    if (u == v) return 0;
    const int32_t ju = w.tau[u], jv = w.tau[v];
    return w.a[(size_t)u * w.lda + jv] + w.a[(size_t)v * w.lda + ju] - w.diag[ju] - w.diag[jv];
}

// Edge of slot t under the current sigma; w = current gain of its exchange.
__device__ __forceinline__ int4 make_edge(const Workspace& w, int32_t t) {
    int32_t u, v;
    if (t < w.n) {
        u = t;
        v = w.sigma[w.ag_job[t]];
    } else {
        u = w.sigma[t - w.n];
        v = w.jb_agent[t - w.n];
    }
    return make_int4(t, u, v, exchange_gain(w, u, v));
}

// Block-wide exclusive scan of a 0/1 flag (1024 threads); returns the prefix,
// writes the total to *total (all threads).
__device__ __forceinline__ int32_t block_scan(int32_t flag, int32_t* warp_sums, int32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ballot = __ballot_sync(0xffffffffu, flag);
    const int32_t in_warp = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[warp] = __popc(ballot);
    __syncthreads();
    if (warp == 0) {
        int32_t v = warp_sums[lane];
        int32_t incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        warp_sums[lane] = incl - v;
        if (lane == 31) warp_sums[32] = incl;
    }
    __syncthreads();
    const int32_t r = warp_sums[warp] + in_warp;
    *total = warp_sums[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kCtlThreads, 1) controller_kernel(Workspace w, int32_t use_smem, int32_t* g_res,
                                                                   uint8_t* g_claimed, uint8_t* g_estate) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t warp_sums[33];
    __shared__ int32_t s_L, s_any, s_acc, s_app, s_y;
    __shared__ unsigned long long s_gain;

    const int32_t n = w.n;
    const int tid = threadIdx.x;
    int32_t* res = g_res;
    uint8_t* claimed = g_claimed;
    uint8_t* estate = g_estate;
    if (use_smem) {
        res = reinterpret_cast<int32_t*>(smem_raw);
        claimed = smem_raw + 4 * (size_t)n;
        estate = claimed + n;
    }
    int4* E = w.edges;

    // ---------------------------------------------------------------- entry
    {
        const int32_t yc = st->y_count;
        for (int32_t t = tid; t < yc; t += kCtlThreads) {
            const int32_t j = w.y_list[t];
            w.in_y[j] = 0;
            w.moved[w.sigma[j]] = 0;
        }
        for (int32_t i = tid; i < n; i += kCtlThreads) {
            if (!w.in_ca[i]) {
                const unsigned long long ka = w.key_a[w.tau[i]];
                w.ag_gain[i] = ka ? key_gain(ka) : 0;
                w.ag_job[i] = ka ? key_index(ka) : -1;
            }
            if (!w.in_cj[i]) {
                const unsigned long long kj = w.key_j[i];
                w.jb_gain[i] = kj ? key_gain(kj) : 0;
                w.jb_agent[i] = kj ? key_index(kj) : -1;
            }
            res[i] = kInf;
            claimed[i] = 0;
        }
        if (tid == 0) {
            st->need_update = 0;
            st->y_count = 0;
            s_L = 0;
        }
        __syncthreads();
        // edge list in priority order
        for (int32_t base = 0; base < 2 * n; base += kCtlThreads) {
            const int32_t t = base + tid;
            const int32_t has = (t < 2 * n) ? ((t < n) ? (w.ag_gain[t] > 0) : (w.jb_gain[t - n] > 0)) : 0;
            int32_t total;
            const int32_t pos = block_scan(has, warp_sums, &total);
            if (has) E[s_L + pos] = make_edge(w, t);
            __syncthreads();
            if (tid == 0) s_L += total;
            __syncthreads();
        }
    }

    // ------------------------------------------------------------- sweeps
    // Quiet sweeps turn at least one stale slot into a fresh one each, so one
    // launch runs at most 2n + 1 of them; more means an internal error.
    for (int32_t quiet = 0;; ++quiet) {
        const int32_t L = s_L;
        if (quiet > 2 * n + 1) {
            if (tid == 0) { st->error = kErrInternal; st->status = kError; }
            break;
        }
        if (tid == 0) {
            // loop condition of Algorithm 3 (some slot has delta > 0), sweep
            // cap and deadline; decided by one thread so that all agree
            int32_t stop = 0;
            if (L == 0) {
                st->status = kDone;
                stop = 1;
            } else if ((st->max_sweeps > 0 && st->sweeps >= st->max_sweeps) ||
                       (st->deadline_ns != 0 && globaltimer_ns() > st->deadline_ns)) {
                st->status = kTimeout;
                stop = 1;
            }
            s_any = stop;
            s_acc = 0; s_app = 0; s_y = 0; s_gain = 0ull;
        }
        __syncthreads();
        if (s_any) break;
        for (int32_t e = tid; e < L; e += kCtlThreads) estate[e] = kLive;
        __syncthreads();
        // CC (Algorithm 4) by deterministic reservations
        for (uint32_t round = 0;; ++round) {
            for (int32_t e = tid; e < L; e += kCtlThreads) {
                if (estate[e] != kLive) continue;
                const int4 ed = E[e];
                atomicMin(&res[ed.y], ed.x);
                atomicMin(&res[ed.z], ed.x);
            }
            __syncthreads();
            for (int32_t e = tid; e < L; e += kCtlThreads) {
                if (estate[e] != kLive) continue;
                const int4 ed = E[e];
                if (res[ed.y] == ed.x && res[ed.z] == ed.x) {
                    estate[e] = kAcc;
                    claimed[ed.y] = 1;
                    claimed[ed.z] = 1;
                }
            }
            __syncthreads();
            int32_t any = 0;
            for (int32_t e = tid; e < L; e += kCtlThreads) {
                if (estate[e] != kLive) continue;
                const int4 ed = E[e];
                if (claimed[ed.y] | claimed[ed.z]) {
                    estate[e] = kRej;
                } else {
                    res[ed.y] = kInf;
                    res[ed.z] = kInf;
                    any = 1;
                }
            }
            if (!__syncthreads_or(any)) break;
            if (round > (uint32_t)(2 * n + 2)) {  // cannot happen: each round accepts the first live edge
                if (tid == 0) { st->error = kErrInternal; st->status = kError; }
                return;
            }
        }
        // parallel switch: accepted exchanges are agent-disjoint
        int32_t my_acc = 0, my_app = 0;
        long long my_gain = 0;
        for (int32_t e = tid; e < L; e += kCtlThreads) {
            if (estate[e] != kAcc) continue;
            ++my_acc;
            const int4 ed = E[e];
            if (ed.w > 0) {
                const int32_t u = ed.y, v = ed.z;
                const int32_t ju = w.tau[u], jv = w.tau[v];
                const int32_t x1 = w.a[(size_t)u * w.lda + jv];
                const int32_t x2 = w.a[(size_t)v * w.lda + ju];
                w.tau[u] = jv;
                w.tau[v] = ju;
                w.sigma[jv] = u;
                w.sigma[ju] = v;
                w.diag[jv] = x1;
                w.diag[ju] = x2;
                my_gain += ed.w;
                ++my_app;
                const int32_t p = atomicAdd(&s_y, 2);
                w.y_list[p] = ju;
                w.y_list[p + 1] = jv;
                w.in_y[ju] = 1;
                w.in_y[jv] = 1;
                w.moved[u] = 1;
                w.moved[v] = 1;
            }
        }
        if (my_acc) atomicAdd(&s_acc, my_acc);
        if (my_app) {
            atomicAdd(&s_app, my_app);
            atomicAdd(&s_gain, (unsigned long long)my_gain);
        }
        __syncthreads();
        const int32_t acc = s_acc, app = s_app;
        if (tid == 0) {
            const int32_t sw = st->sweeps;
            st->f += (long long)s_gain;
            st->swaps += app;
            if (sw < st->trace_capacity) {
                if (st->trace_accepted) st->trace_accepted[sw] = acc;
                if (st->trace_applied) st->trace_applied[sw] = app;
                if (st->trace_objective) st->trace_objective[sw] = st->f;
            }
            st->sweeps = sw + 1;
        }
        if (app > 0) {
            // event: record C for the refresh that follows the row update
            for (int32_t i = tid; i < n; i += kCtlThreads) {
                w.in_ca[i] = 0;
                w.in_cj[i] = 0;
            }
            __syncthreads();
            for (int32_t e = tid; e < L; e += kCtlThreads) {
                if (estate[e] != kRej) continue;
                const int32_t t = E[e].x;
                if (t < n) w.in_ca[t] = 1;
                else w.in_cj[t - n] = 1;
            }
            if (tid == 0) {
                st->events += 1;
                st->y_count = s_y;
                st->rescan_count = 0;
                st->need_update = 1;
                st->phase = kPhaseRefreshAll;
            }
            break;
        }
        // quiet sweep: sigma unchanged, so the keys are current; re-evaluate
        // the accepted slots, keep the rejected ones (stale, in C)
        for (int32_t e = tid; e < L; e += kCtlThreads) {
            const int4 ed = E[e];
            res[ed.y] = kInf;
            res[ed.z] = kInf;
            claimed[ed.y] = 0;
            claimed[ed.z] = 0;
        }
        __syncthreads();
        for (int32_t e = tid; e < L; e += kCtlThreads) {
            if (estate[e] != kAcc) continue;
            const int32_t t = E[e].x;
            if (t < n) {
                const unsigned long long ka = w.key_a[w.tau[t]];
                w.ag_gain[t] = ka ? key_gain(ka) : 0;
                w.ag_job[t] = ka ? key_index(ka) : -1;
                if (ka) E[e] = make_int4(t, t, w.sigma[key_index(ka)], key_gain(ka));
                else estate[e] = kDead;
            } else {
                const int32_t j = t - n;
                const unsigned long long kj = w.key_j[j];
                w.jb_gain[j] = kj ? key_gain(kj) : 0;
                w.jb_agent[j] = kj ? key_index(kj) : -1;
                if (kj) E[e] = make_int4(t, w.sigma[j], key_index(kj), key_gain(kj));
                else estate[e] = kDead;
            }
        }
        __syncthreads();
        // compact the edge list (forward, in place, order kept)
        if (tid == 0) s_L = 0;
        __syncthreads();
        for (int32_t base = 0; base < L; base += kCtlThreads) {
            const int32_t e = base + tid;
            const int32_t keep = (e < L) && estate[e] != kDead;
            const int4 ed = keep ? E[e] : make_int4(0, 0, 0, 0);
            int32_t total;
            const int32_t pos = block_scan(keep, warp_sums, &total);
            if (keep) E[s_L + pos] = ed;
            __syncthreads();
            if (tid == 0) s_L += total;
            __syncthreads();
        }
    }
    if (tid == 0) st->edge_count = s_L;
}

// Rows whose best is no longer known: rows of changed jobs, and rows whose
// best partner column changed holder.  Their keys are cleared and listed.
__global__ void mark_rescan_kernel(Workspace w) {
    DeviceState* st = w.st;
    if (st->status != kRunning || !st->need_update) return;
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < w.n; j += gridDim.x * blockDim.x) {
        bool need = w.in_y[j];
        const unsigned long long ka = w.key_a[j];
        const unsigned long long kj = w.key_j[j];
        if (!need && ka) need = w.in_y[key_index(ka)];
        if (!need && kj) need = w.moved[key_index(kj)];
        if (need) {
            w.key_a[j] = 0;
            w.key_j[j] = 0;
            w.rescan_list[atomicAdd(&st->rescan_count, 1)] = j;
        }
    }
}

// Full re-evaluation of the listed rows: row j of G from row sigma(j) of a
// and row j of at (gathered through sigma, staged in shared memory).  Rows
// of changed jobs also push G[k][j] = G[j][k] into every other row k (the
// only entries of row k that changed), through the same atomic keys.
template <bool kStage>
__global__ void __launch_bounds__(512) row_tasks_kernel(Workspace w) {
    DeviceState* st = w.st;
    if (st->status != kRunning || !st->need_update) return;
    const int32_t count = st->rescan_count;
    const int32_t n = w.n;
    if (use_full_update(count, n)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->row_updates += 1;
        st->rows_recomputed += count;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* atrow_s = reinterpret_cast<int32_t*>(smem_raw);
    __shared__ unsigned long long red_a[16], red_j[16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int32_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int32_t j = w.rescan_list[t];
        const int32_t* atrow = w.at + (size_t)j * w.ldt;
        if (kStage) {
            for (int32_t c = tid * 4; c < n; c += blockDim.x * 4)
                *reinterpret_cast<int4*>(atrow_s + c) = *reinterpret_cast<const int4*>(atrow + c);
            __syncthreads();
            atrow = atrow_s;
        }
        const int32_t sjj = w.sigma[j];
        const int32_t dj = w.diag[j];
        const bool scatter = w.in_y[j];
        const int32_t* arow = w.a + (size_t)sjj * w.lda;
        int32_t bg = 0, bc = -1, bs = 0x7fffffff;
        for (int32_t k = tid; k < n; k += blockDim.x) {
            const int32_t sk = w.sigma[k];
            const int32_t g = arow[k] + atrow[sk] - dj - w.diag[k];
            const bool gt = g > bg, eq = g == bg;
            bs = gt ? sk : (eq ? min(bs, sk) : bs);
            bc = gt ? k : bc;
            bg = max(bg, g);
            if (scatter && g > 0 && k != j) {
                if (g >= key_gain(w.key_a[k])) {
                    atomicMax(&w.key_a[k], pack_gain(g, (uint32_t)j));
                    atomicMax(&w.key_j[k], pack_gain(g, (uint32_t)sjj));
                }
            }
        }
        unsigned long long ka = bg > 0 ? pack_gain(bg, (uint32_t)bc) : 0ull;
        unsigned long long kj = bg > 0 ? pack_gain(bg, (uint32_t)bs) : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ka = umax64(ka, __shfl_xor_sync(0xffffffffu, ka, off));
            kj = umax64(kj, __shfl_xor_sync(0xffffffffu, kj, off));
        }
        if (lane == 0) { red_a[warp] = ka; red_j[warp] = kj; }
        __syncthreads();
        if (tid == 0) {
            unsigned long long ma = 0, mj = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { ma = umax64(ma, red_a[q]); mj = umax64(mj, red_j[q]); }
            if (ma) {
                atomicMax(&w.key_a[j], ma);
                atomicMax(&w.key_j[j], mj);
            }
        }
        __syncthreads();
    }
}

// tau given (greedy result, identity or the caller's permutation): build
// sigma, D and f; validate a caller's permutation.
__global__ void start_from_tau_kernel(Workspace w, const int32_t* user_tau, int32_t mode, uint8_t* seen) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x) {
        int32_t j;
        if (mode == 2) j = i;                 // identity
        else if (mode == 3) j = user_tau[i];  // caller's permutation
        else j = w.tau[i];                    // greedy result
        if (j < 0 || j >= w.n || atomicExch(reinterpret_cast<unsigned int*>(seen) + j, 1u) != 0u) {
            st->error = kErrUserInit;
            st->status = kError;
            continue;
        }
        w.tau[i] = j;
        w.sigma[j] = i;
        const int32_t d = w.a[(size_t)i * w.lda + j];
        w.diag[j] = d;
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->f), (unsigned long long)(long long)d);
    }
}

__global__ void finish_kernel(Workspace w, int32_t* sigma_out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x)
        sigma_out[i] = w.tau[i];
}

}  // namespace

// controller scratch lives in shared memory up to this size
constexpr int32_t kCtlSmemMaxN = 28000;

size_t controller_smem_bytes(int32_t n) {
    if (n > kCtlSmemMaxN) return 0;
    return 4 * (size_t)n + (size_t)n + 2 * (size_t)n + 16;
}

cudaError_t launch_controller_impl(const Workspace& w, int32_t* g_res, uint8_t* g_claimed, uint8_t* g_estate,
                                   cudaStream_t s) {
    const size_t smem = controller_smem_bytes(w.n);
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(controller_kernel), 1, smem);
        if (e != cudaSuccess) return e;
    }
    controller_kernel<<<1, kCtlThreads, smem, s>>>(w, smem ? 1 : 0, g_res, g_claimed, g_estate);
    return cudaGetLastError();
}

cudaError_t launch_mark_rescan(const Workspace& w, cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > 152 * 4) grid = 152 * 4;
    mark_rescan_kernel<<<grid, 256, 0, s>>>(w);
    return cudaGetLastError();
}

constexpr int32_t kRowStageMaxN = 56 * 1024;

cudaError_t launch_row_tasks(const Workspace& w, cudaStream_t s) {
    const int grid = 152 * 2;
    if (w.n <= kRowStageMaxN) {
        const size_t smem = 4 * (size_t)w.ldt;
        if (smem > 48 * 1024) {
            cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(row_tasks_kernel<true>), 2, smem);
            if (e != cudaSuccess) return e;
        }
        row_tasks_kernel<true><<<grid, 512, smem, s>>>(w);
    } else {
        row_tasks_kernel<false><<<grid, 512, 0, s>>>(w);
    }
    return cudaGetLastError();
}

cudaError_t launch_start_from_tau(const Workspace& w, const int32_t* user_tau, int32_t mode, uint8_t* seen,
                                  cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > 152 * 4) grid = 152 * 4;
    start_from_tau_kernel<<<grid, 256, 0, s>>>(w, user_tau, mode, seen);
    return cudaGetLastError();
}

cudaError_t launch_finish(const Workspace& w, int32_t* sigma_out, cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > 152 * 4) grid = 152 * 4;
    finish_kernel<<<grid, 256, 0, s>>>(w, sigma_out);
    return cudaGetLastError();
}

}  // namespace dgs
