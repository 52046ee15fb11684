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
constexpr int32_t kClaimed = -1;  // reservation value of an agent claimed this sweep
enum : uint8_t { kDead = 0, kLive = 1, kAcc = 2, kRej = 3 };

// Edge word: agent u (bits 0..16), agent v (17..33), applies (34): its
// exchange raises f under the current sigma, fresh (35): re-evaluated in this
// launch.  Edge positions follow slot priority, so a position is a priority.
constexpr unsigned long long kApplies = 1ull << 34;
constexpr unsigned long long kFresh = 1ull << 35;
__device__ __forceinline__ unsigned long long edge_word(int32_t u, int32_t v) {
    return (unsigned long long)(uint32_t)u | ((unsigned long long)(uint32_t)v << 17);
}
__device__ __forceinline__ int32_t edge_u(unsigned long long e) { return (int32_t)(e & 0x1FFFFu); }
__device__ __forceinline__ int32_t edge_v(unsigned long long e) { return (int32_t)((e >> 17) & 0x1FFFFu); }

__device__ __forceinline__ int32_t exchange_gain(const Workspace& w, int32_t u, int32_t v) {
    if (u == v) return 0;
    const int32_t ju = w.tau[u], jv = w.tau[v];
    return w.a[(size_t)u * w.lda + jv] + w.a[(size_t)v * w.lda + ju] - w.diag[ju] - w.diag[jv];
}

// Block-wide exclusive scan of one int per thread (1024 threads).
__device__ __forceinline__ int32_t block_scan(int32_t x, int32_t* warp_sums, int32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int32_t v = warp_sums[lane];
        int32_t wi = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += o;
        }
        warp_sums[lane] = wi - v;
        if (lane == 31) warp_sums[32] = wi;
    }
    __syncthreads();
    const int32_t r = warp_sums[warp] + incl - x;
    *total = warp_sums[32];
    __syncthreads();
    return r;
}

struct CtlScratch {
    int32_t* res;               // per agent: reservation (lowest live priority) or kClaimed
    uint8_t* estate;            // per edge position
    unsigned long long* edges;  // per edge position
};

// Switching loop (see the file comment).  smem_mode 2: edges, reservations
// and edge states in shared memory; 1: edges in global memory; 0: all global.
__global__ void __launch_bounds__(kCtlThreads, 1) controller_kernel(Workspace w, int32_t smem_mode, CtlScratch g) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int32_t warp_sums[33];
    __shared__ int32_t s_L, s_live, s_stop, s_acc, s_app, s_y, s_sweeps, s_event;
    __shared__ unsigned long long s_gain;

    const int32_t n = w.n;
    const int tid = threadIdx.x;
    CtlScratch c = g;
    if (smem_mode >= 1) {
        c.res = reinterpret_cast<int32_t*>(smem_raw);
        c.estate = smem_raw + 4 * (size_t)n;
        if (smem_mode == 2)
            c.edges = reinterpret_cast<unsigned long long*>(smem_raw + ((4 * (size_t)n + 2 * (size_t)n + 15) & ~(size_t)15));
    }
    int32_t* res = c.res;
    uint8_t* estate = c.estate;
    unsigned long long* E = c.edges;

    // ---------------------------------------------------------------- entry
    {
        const int32_t yc = st->y_count;
        for (int32_t t = tid; t < yc; t += kCtlThreads) {
            const int32_t j = w.y_list[t];
            w.in_y[j] = 0;
            w.moved[w.sigma[j]] = 0;
        }
        // re-evaluation of the slots not in C: read the current row keys
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
        }
        if (tid == 0) {
            st->need_update = 0;
            st->y_count = 0;
            s_sweeps = st->sweeps;
        }
        __syncthreads();
        // edge list in priority order: each thread owns a contiguous slot range
        const int32_t per = (2 * n + kCtlThreads - 1) / kCtlThreads;
        const int32_t t0 = min(2 * n, tid * per), t1 = min(2 * n, t0 + per);
        int32_t cnt = 0;
        for (int32_t t = t0; t < t1; ++t) cnt += (t < n) ? (w.ag_gain[t] > 0) : (w.jb_gain[t - n] > 0);
        int32_t total;
        int32_t pos = block_scan(cnt, warp_sums, &total);
        for (int32_t t = t0; t < t1; ++t) {
            int32_t u, v;
            if (t < n) {
                if (w.ag_gain[t] <= 0) continue;
                u = t;
                v = w.sigma[w.ag_job[t]];
            } else {
                if (w.jb_gain[t - n] <= 0) continue;
                u = w.sigma[t - n];
                v = w.jb_agent[t - n];
            }
            w.ctl_slot[pos] = t;
            E[pos] = edge_word(u, v);
            ++pos;
        }
        if (tid == 0) { s_L = total; s_live = total; }
        __syncthreads();
        const int32_t L = s_L;
        // current gains and the re-evaluation outcome of every edge's slot
        // (keys do not change while no exchange is committed)
#pragma unroll 4
        for (int32_t p = tid; p < L; p += kCtlThreads) {
            const unsigned long long e = E[p];
            const int32_t t = w.ctl_slot[p];
            unsigned long long key;
            int32_t ru, rv;
            if (t < n) {
                key = w.key_a[w.tau[t]];
                ru = t;
                rv = key ? w.sigma[key_index(key)] : t;
            } else {
                key = w.key_j[t - n];
                ru = w.sigma[t - n];
                rv = key ? key_index(key) : ru;
            }
            w.ctl_rkey[p] = key;
            w.ctl_ru[p] = ru;
            w.ctl_rv[p] = rv;
            E[p] = e | (exchange_gain(w, edge_u(e), edge_v(e)) > 0 ? kApplies : 0ull);
            estate[p] = kLive;
        }
        __syncthreads();
    }

    // ------------------------------------------------------------- sweeps
    // Quiet sweeps turn at least one stale slot into a fresh one each, so one
    // launch runs at most 2n + 1 of them; more means an internal error.
    const int32_t L = s_L;
    for (int32_t quiet = 0;; ++quiet) {
        if (tid == 0) {
            // loop condition of Algorithm 3 (some slot has delta > 0), sweep
            // cap and deadline; decided by one thread so that all agree
            int32_t stop = 0;
            if (s_live == 0) {
                st->status = kDone;
                stop = 1;
            } else if ((st->max_sweeps > 0 && s_sweeps >= st->max_sweeps) ||
                       (st->deadline_ns != 0 && globaltimer_ns() > st->deadline_ns)) {
                st->status = kTimeout;
                stop = 1;
            } else if (quiet > 2 * n + 1) {
                st->error = kErrInternal;
                st->status = kError;
                stop = 1;
            }
            s_stop = stop;
            s_acc = 0; s_app = 0; s_y = 0; s_gain = 0ull; s_event = 0;
        }
        __syncthreads();
        if (s_stop) break;
        // CC (Algorithm 4) by deterministic reservations
        for (uint32_t round = 0;; ++round) {
            for (int32_t p = tid; p < L; p += kCtlThreads) {
                if (estate[p] != kLive) continue;
                const unsigned long long e = E[p];
                const int32_t u = edge_u(e), v = edge_v(e);
                if (p < res[u]) atomicMin(&res[u], p);
                if (p < res[v]) atomicMin(&res[v], p);
            }
            __syncthreads();
            int32_t acc = 0, ev = 0;
            for (int32_t p = tid; p < L; p += kCtlThreads) {
                if (estate[p] != kLive) continue;
                const unsigned long long e = E[p];
                const int32_t u = edge_u(e), v = edge_v(e);
                if (res[u] == p && res[v] == p) {
                    estate[p] = kAcc;
                    res[u] = kClaimed;
                    res[v] = kClaimed;
                    ++acc;
                    ev |= (e & kApplies) ? 1 : 0;
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(w.ctl_rkey + p));
                }
            }
            if (acc) atomicAdd(&s_acc, acc);
            if (ev) s_event = 1;
            __syncthreads();
            int32_t any = 0;
            for (int32_t p = tid; p < L; p += kCtlThreads) {
                if (estate[p] != kLive) continue;
                const unsigned long long e = E[p];
                const int32_t u = edge_u(e), v = edge_v(e);
                if (res[u] == kClaimed || res[v] == kClaimed) {
                    estate[p] = kRej;
                } else {
                    res[u] = kInf;
                    res[v] = kInf;
                    any = 1;
                }
            }
            if (!__syncthreads_or(any)) break;
            if (round > (uint32_t)(L + 2)) {  // each round accepts the first live edge
                if (tid == 0) { st->error = kErrInternal; st->status = kError; }
                return;
            }
        }
        if (s_event) {
            // parallel switch: accepted exchanges are agent-disjoint; those
            // that raise f under the current sigma commit
            int32_t my_app = 0;
            long long my_gain = 0;
            for (int32_t p = tid; p < L; p += kCtlThreads) {
                if (estate[p] != kAcc) continue;
                const unsigned long long e = E[p];
                if (!(e & kApplies)) continue;
                const int32_t u = edge_u(e), v = edge_v(e);
                const int32_t ju = w.tau[u], jv = w.tau[v];
                const int32_t x1 = w.a[(size_t)u * w.lda + jv];
                const int32_t x2 = w.a[(size_t)v * w.lda + ju];
                my_gain += (long long)x1 + x2 - w.diag[ju] - w.diag[jv];
                w.tau[u] = jv;
                w.tau[v] = ju;
                w.sigma[jv] = u;
                w.sigma[ju] = v;
                w.diag[jv] = x1;
                w.diag[ju] = x2;
                ++my_app;
                const int32_t q = atomicAdd(&s_y, 2);
                w.y_list[q] = ju;
                w.y_list[q + 1] = jv;
                w.in_y[ju] = 1;
                w.in_y[jv] = 1;
                w.moved[u] = 1;
                w.moved[v] = 1;
            }
            if (my_app) {
                atomicAdd(&s_app, my_app);
                atomicAdd(&s_gain, (unsigned long long)my_gain);
            }
            for (int32_t i = tid; i < n; i += kCtlThreads) {
                w.in_ca[i] = 0;
                w.in_cj[i] = 0;
            }
            __syncthreads();
            // record C (the rejected slots keep their candidates, reading R4)
            for (int32_t p = tid; p < L; p += kCtlThreads) {
                if (estate[p] != kRej) continue;
                const int32_t t = w.ctl_slot[p];
                if (t < n) w.in_ca[t] = 1;
                else w.in_cj[t - n] = 1;
            }
            if (tid == 0) {
                const int32_t sw = s_sweeps;
                st->f += (long long)s_gain;
                st->swaps += s_app;
                if (sw < st->trace_capacity) {
                    if (st->trace_accepted) st->trace_accepted[sw] = s_acc;
                    if (st->trace_applied) st->trace_applied[sw] = s_app;
                    if (st->trace_objective) st->trace_objective[sw] = st->f;
                }
                s_sweeps = sw + 1;
                st->events += 1;
                st->y_count = s_y;
                st->rescan_count = 0;
                st->need_update = 1;
                st->phase = kPhaseRefreshAll;
            }
            break;
        }
        // quiet sweep: sigma unchanged, so the keys are current.  Accepted
        // slots are re-evaluated (their precomputed outcome); rejected slots
        // stay in C with their candidates for the next sweep.
        int32_t died = 0;
        for (int32_t p = tid; p < L; p += kCtlThreads) {
            const uint8_t es = estate[p];
            if (es == kDead) continue;
            const unsigned long long e = E[p];
            res[edge_u(e)] = kInf;
            res[edge_v(e)] = kInf;
            if (es == kRej) {
                estate[p] = kLive;
            } else if (es == kAcc) {
                const int32_t t = w.ctl_slot[p];
                const unsigned long long key = w.ctl_rkey[p];
                const int32_t gain = key ? key_gain(key) : 0;
                const int32_t target = key ? key_index(key) : -1;
                if (t < n) { w.ag_gain[t] = gain; w.ag_job[t] = target; }
                else { w.jb_gain[t - n] = gain; w.jb_agent[t - n] = target; }
                if (key) {
                    E[p] = edge_word(w.ctl_ru[p], w.ctl_rv[p]) | kApplies | kFresh;
                    estate[p] = kLive;
                } else {
                    estate[p] = kDead;
                    ++died;
                }
            }
        }
        if (died) atomicSub(&s_live, died);
        if (tid == 0) {
            const int32_t sw = s_sweeps;
            if (sw < st->trace_capacity) {
                if (st->trace_accepted) st->trace_accepted[sw] = s_acc;
                if (st->trace_applied) st->trace_applied[sw] = 0;
                if (st->trace_objective) st->trace_objective[sw] = st->f;
            }
            s_sweeps = sw + 1;
        }
        __syncthreads();
    }
    if (tid == 0) {
        st->sweeps = s_sweeps;
        st->edge_count = s_live;
    }
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
// and row j of at (gathered through sigma; staged in shared memory by one TMA
// bulk copy).  Rows of changed jobs also push G[k][j] = G[j][k] into every
// other row k (the only entries of row k that changed), through the same
// atomic keys.
template <bool kStage>
__global__ void __launch_bounds__(512) row_tasks_kernel(Workspace w) {
    DeviceState* st = w.st;
    if (st->status != kRunning || !st->need_update) return;
    const int32_t count = st->rescan_count;
    const int32_t n = w.n;
    if (use_full_update(count, n, st->update_policy)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->row_updates += 1;
        st->rows_recomputed += count;
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int32_t* atrow_s = reinterpret_cast<int32_t*>(smem_raw);
    __shared__ unsigned long long red_a[16], red_j[16];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int32_t s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (kStage && tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_fail = 0;
    }
    __syncthreads();
    uint32_t phase = 0;
    const int32_t n4 = (n + 3) / 4;
    for (int32_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int32_t j = w.rescan_list[t];
        const int32_t* atrow = w.at + (size_t)j * w.ldt;
        if (kStage) {
            if (tid == 0) {
                const uint32_t bytes = 16u * (uint32_t)n4;
                mbar_arrive_expect_tx(&bar, bytes);
                bulk_g2s(atrow_s, atrow, bytes, &bar);
            }
            const bool ok = mbar_wait_bounded(&bar, phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) { st->error = kErrWaitTimeout; st->status = kError; }
                return;
            }
            atrow = atrow_s;
        }
        const int32_t sjj = w.sigma[j];
        const int32_t dj = w.diag[j];
        const bool scatter = w.in_y[j];
        const int32_t* arow = w.a + (size_t)sjj * w.lda;
        int32_t bg = 0, bc = -1, bs = 0x7fffffff;
#pragma unroll 2
        for (int32_t q = tid; q < n4; q += blockDim.x) {
            const int32_t k0 = 4 * q;
            const int4 x4 = *reinterpret_cast<const int4*>(arow + k0);
            const int4 s4 = *reinterpret_cast<const int4*>(w.sigma + k0);
            const int4 d4 = *reinterpret_cast<const int4*>(w.diag + k0);
            const int32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
            const int32_t ss[4] = {s4.x, s4.y, s4.z, s4.w};
            const int32_t ds[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int32_t k = k0 + e;
                if (k >= n) break;
                const int32_t sk = ss[e];
                const int32_t g = xs[e] + atrow[sk] - dj - ds[e];
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
        __syncthreads();  // red_* and the staged row are reused by the next row
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

// Controller scratch placement (bytes of dynamic shared memory per mode).
constexpr size_t kCtlSmemLimit = 227 * 1024 - 1024;

int32_t controller_smem_mode(int32_t n) {
    const size_t all = ((6 * (size_t)n + 15) & ~(size_t)15) + 16 * (size_t)n;
    int32_t mode = 0;
    if (all <= kCtlSmemLimit) mode = 2;
    else if (6 * (size_t)n <= kCtlSmemLimit) mode = 1;
    return min(mode, env_controller_mode_cap());
}

size_t controller_smem_bytes(int32_t n) {
    const int32_t mode = controller_smem_mode(n);
    if (mode == 2) return ((6 * (size_t)n + 15) & ~(size_t)15) + 16 * (size_t)n;
    if (mode == 1) return 6 * (size_t)n;
    return 0;
}

cudaError_t launch_controller_impl(const Workspace& w, int32_t* g_res, uint8_t* g_estate, unsigned long long* g_edges,
                                   cudaStream_t s) {
    const int32_t mode = controller_smem_mode(w.n);
    const size_t smem = controller_smem_bytes(w.n);
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(controller_kernel), 1, smem);
        if (e != cudaSuccess) return e;
    }
    CtlScratch c{g_res, g_estate, g_edges};
    controller_kernel<<<1, kCtlThreads, smem, s>>>(w, mode, c);
    return cudaGetLastError();
}

cudaError_t launch_mark_rescan(const Workspace& w, cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > 152 * 4) grid = 152 * 4;
    mark_rescan_kernel<<<grid, 256, 0, s>>>(w);
    return cudaGetLastError();
}

constexpr int32_t kRowStageMaxN = 54 * 1024;

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
