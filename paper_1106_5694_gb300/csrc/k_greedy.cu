// k_greedy.cu -- greedy starting assignment (Section 3.1, read as the global
// greedy: repeatedly take the largest remaining benefit, ties to the lowest
// agent, then the lowest job).
//
// Parallel form: locally-dominant rounds.  Under the strict total order on
// pairs (benefit desc, agent asc, job asc), every free agent finds its best
// free job and every free job its best free agent; mutually-best pairs are
// matched.  The globally largest remaining pair is always mutually best and
// the matched pairs are disjoint, so the rounds produce exactly the
// sequential global-greedy assignment.
//
// Pass 1 reads a once in 64x64 tiles and, in the same pass, writes the
// transposed copy at (used later for column scans), checks |a| < 2^29 and
// computes every agent's and job's best pair.  Later rounds rescan only the
// agents (rows of a) and jobs (rows of at) whose best partner was taken.
#include <cstdlib>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kT = 64;  // tile edge

// a_src (batched instances only): the caller's matrix with row pitch n when w.a
// is the workspace's pitched copy still to be filled; this pass reads a_src
// and writes the copy as it goes.  Null: w.a is read.
__device__ __forceinline__ void greedy_pass1_body(const Workspace& w, int32_t tiles_x, int32_t tiles_total,
                                                  int32_t bid, int32_t nblk, const int32_t* a_src = nullptr,
                                                  bool cols = true) {
    __shared__ int32_t s[kT][kT + 1];
    __shared__ unsigned long long colpart[4][kT];
    const int32_t n = w.n;
    const int t = threadIdx.x;
    const int lane16 = t & 15;
    bool bad = false;
    int32_t amax = 0;
    for (int32_t tile = bid; tile < tiles_total; tile += nblk) {
        const int32_t I0 = (tile / tiles_x) * kT;
        const int32_t J0 = (tile % tiles_x) * kT;
        // load 64 rows x 64 cols with int4, 16 threads per row, 4 passes
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int r = (t >> 4) + 16 * p;
            const int c = lane16 * 4;
            const int32_t i = I0 + r, j = J0 + c;
            int4 v = make_int4(0, 0, 0, 0);
            if (a_src == nullptr) {
                if (i < n && j < w.lda) v = *reinterpret_cast<const int4*>(w.a + (size_t)i * w.lda + j);
            } else if (i < n && j < w.lda) {  // re-pitch: unaligned reads, padding columns 0
                const int32_t* src = a_src + (size_t)i * n + j;
                v.x = j < n ? src[0] : 0;
                v.y = j + 1 < n ? src[1] : 0;
                v.z = j + 2 < n ? src[2] : 0;
                v.w = j + 3 < n ? src[3] : 0;
                *reinterpret_cast<int4*>(const_cast<int32_t*>(w.a) + (size_t)i * w.lda + j) = v;
            }
            s[r][c + 0] = v.x; s[r][c + 1] = v.y; s[r][c + 2] = v.z; s[r][c + 3] = v.w;
            // row best over this tile's 4 columns of this thread
            unsigned long long best = 0;
            const int32_t vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (i < n && j + e < n) {
                    const int32_t x = vals[e];
                    bad |= (x >= kBenefitLimit) || (x <= -kBenefitLimit);
                    amax = max(amax, x == INT32_MIN ? INT32_MAX : abs(x));
                    best = umax64(best, pack_benefit(x, (uint32_t)(j + e)));
                }
            }
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, off));
            if (lane16 == 0 && i < n && best != 0) atomicMax(&w.g_row[i], best);
        }
        __syncthreads();
        // column best: thread (group g = t/64, column c = t%64) scans 16 rows
        if (cols) {
            const int c = t & 63, g = t >> 6;
            const int32_t j = J0 + c;
            unsigned long long best = 0;
            if (j < n) {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int32_t i = I0 + g * 16 + r;
                    if (i < n) best = umax64(best, pack_benefit(s[g * 16 + r][c], (uint32_t)i));
                }
            }
            colpart[g][c] = best;
        }
        // transposed store: at row j = J0 + jr, 4 agents per thread
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int jr = (t >> 4) + 16 * p;
            const int i4 = lane16 * 4;
            const int32_t j = J0 + jr;
            if (j < n) {
                int4 v;
                v.x = s[i4 + 0][jr]; v.y = s[i4 + 1][jr]; v.z = s[i4 + 2][jr]; v.w = s[i4 + 3][jr];
                *reinterpret_cast<int4*>(w.at + (size_t)j * w.ldt + I0 + i4) = v;
            }
        }
        __syncthreads();
        if (cols && t < kT) {
            const int32_t j = J0 + t;
            unsigned long long best = umax64(umax64(colpart[0][t], colpart[1][t]), umax64(colpart[2][t], colpart[3][t]));
            if (j < n && best != 0) atomicMax(&w.g_col[j], best);
        }
        __syncthreads();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    if ((t & 31) == 0 && amax) atomicMax(&w.st->max_abs, amax);
    if (bad) {
        atomicExch(&w.st->error, kErrRange);
        atomicExch(&w.st->status, kError);
    }
}

// tiles tile0 .. tiles_total - 1 (row-major: a band of whole tile rows)
__global__ void __launch_bounds__(256) greedy_pass1_kernel(Workspace w, int32_t tiles_x, int32_t tiles_total,
                                                           int32_t cols, int32_t tile0) {
    greedy_pass1_body(w, tiles_x, tiles_total, tile0 + blockIdx.x, gridDim.x, nullptr, cols != 0);
}

// Match every mutually-best (agent, job) pair.
__device__ __forceinline__ void greedy_match_body(const Workspace& w, int32_t bid, int32_t nblk) {
    DeviceState* st = w.st;
    if (st->status != kRunning || st->greedy_remaining == 0) return;
    for (int32_t i = bid * blockDim.x + threadIdx.x; i < w.n; i += nblk * blockDim.x) {
        if (!w.free_a[i]) continue;
        const int32_t j = key_index(w.g_row[i]);
        if (j < 0 || j >= w.n) {  // every free agent has a free best job
            st->error = kErrInternal;
            st->status = kError;
            continue;
        }
        if (key_index(w.g_col[j]) == i) {
            w.tau[i] = j;
            w.sigma[j] = i;
            w.free_a[i] = 0;
            w.free_j[j] = 0;
            atomicSub(&st->greedy_remaining, 1);
            st->greedy_matched = 1;
        }
    }
}

__global__ void greedy_match_kernel(Workspace w) { greedy_match_body(w, blockIdx.x, gridDim.x); }

// Rescan: for each free "owner" whose best partner was taken, find the best
// free partner in its row of mat (a for agents over jobs, at for jobs over
// agents).  One CTA per owner; 16-byte loads, several in flight per thread.
__global__ void __launch_bounds__(256) greedy_rescan_kernel(Workspace w, const int32_t* mat, int32_t ld,
                                                            unsigned long long* keys, const uint8_t* owner_free,
                                                            const uint8_t* partner_free, int32_t count_round) {
    DeviceState* st = w.st;
    if (count_round && blockIdx.x == 0 && threadIdx.x == 0 && st->greedy_matched) {
        st->greedy_rounds += 1;  // the match kernel before this one matched pairs
        st->greedy_matched = 0;
    }
    if (st->status != kRunning || st->greedy_remaining == 0) return;
    __shared__ unsigned long long red[8];
    const int32_t n = w.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int32_t o = blockIdx.x; o < n; o += gridDim.x) {
        if (!owner_free[o]) continue;
        const int32_t b = key_index(keys[o]);
        if (b >= 0 && b < n && partner_free[b]) continue;  // best partner still free
        const int32_t* row = mat + (size_t)o * ld;
        if (tid == 0) atomicAdd((unsigned long long*)&st->greedy_rescans, 1ull);
        unsigned long long best = 0;
#pragma unroll 4
        for (int32_t c = tid * 4; c < n; c += 1024) {
            const int4 v = *reinterpret_cast<const int4*>(row + c);
            const uint32_t fr = *reinterpret_cast<const uint32_t*>(partner_free + c);
            const int32_t vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c + e < n && ((fr >> (8 * e)) & 0xffu)) best = umax64(best, pack_benefit(vals[e], (uint32_t)(c + e)));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, off));
        if (lane == 0) red[warp] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long m = 0;
            for (int q = 0; q < 8; ++q) m = umax64(m, red[q]);
            keys[o] = m;
        }
        __syncthreads();
    }
}

// Deferred acceptance (Gale and Shapley 1962, agents proposing).  Every
// agent ranks the jobs by (benefit desc, job asc) and every job ranks the
// agents by (benefit desc, agent asc); both rankings are induced by the one
// strict total order on pairs (benefit desc, agent asc, job asc), so the
// stable matching is unique and equals the global greedy assignment: the
// greedy matching is stable, and in any other perfect matching the first
// pair, in that order, where the two differ is a greedy pair, which blocks
// the other matching.  Deferred acceptance in any order of proposals reaches
// it.
//
// Form: g_col[j] holds the key (biased benefit, ~agent) of the job's holder
// and only grows (64-bit atomicMax).  Agent i beats the holder of job j iff
// its own key (a[i][j] biased, ~i) is larger.  A free agent proposes to its
// best job among those whose holder it beats; a proposal that raises the
// key displaces the holder.  The first proposal of every agent is its best
// job overall, found by pass 1 (g_row).  A later proposal takes the first
// job of the agent's list that it still beats; the list (g_list, three
// keys) holds the second to fourth jobs of the agent's last scan.  Holders'
// keys only grow, so every job ranked above a list entry and left out of
// the list was already lost at the scan and is lost still: the first list
// entry the agent beats is its best job.  With no such entry the agent
// rescans its row of a against the holders' keys (a stale key is lower and
// only admits a job whose atomicMax then fails) and keeps the top four.  A
// failed proposal tries the list, else rescans.  A group of threads takes
// the next agent from a global counter and follows the chain of
// displacements: the agent it displaced proposes next, by the same group,
// until a proposal lands on a job nobody held.  Every free agent is thus in
// exactly one group's hands, no group waits for another, and the launch
// ends when the counter is exhausted and every chain has ended.
constexpr int kDaThreads = 1024;
constexpr uint64_t kDaTimeoutNs = 16000000000ull;  // bound on one group's work (internal error beyond)
constexpr int kDaList = 3;                         // list entries per agent (g_list has 4 slots)

template <int kGroup>
__device__ __forceinline__ void group_bar(int grp) {
    if (kGroup == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(kGroup) : "memory");
}

// 64-bit atomic max with acquire-release order at GPU scope: the proposal
// publishes the proposer's list, and the displacer then reads the displaced
// agent's list.
__device__ __forceinline__ unsigned long long atomic_max_acq_rel(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.max.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

// Insert key k into the descending t[0..3] (keys are distinct: the low word
// is the job).
__device__ __forceinline__ void top4_insert(unsigned long long (&t)[4], unsigned long long k) {
    if (k <= t[3]) return;
    t[3] = k;
    if (t[3] > t[2]) { const unsigned long long x = t[2]; t[2] = t[3]; t[3] = x; }
    if (t[2] > t[1]) { const unsigned long long x = t[1]; t[1] = t[2]; t[2] = x; }
    if (t[1] > t[0]) { const unsigned long long x = t[0]; t[0] = t[1]; t[1] = x; }
}

// The four largest keys of the warp, in every lane's out[0..3].
__device__ __forceinline__ void warp_top4(unsigned long long (&t)[4], unsigned long long (&out)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        unsigned long long m = t[0];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = umax64(m, __shfl_xor_sync(0xffffffffu, m, off));
        out[r] = m;
        if (m != 0 && t[0] == m) {  // the owner drops it
            t[0] = t[1];
            t[1] = t[2];
            t[2] = t[3];
            t[3] = 0;
        }
    }
}

// One proposal of agent i (and its retries after failed ones), by the whole
// group.  first: i has not proposed yet (its best job overall, from pass 1).
// s_red: 4 keys per warp of the block; s_top: 4 keys per group.  Returns the
// displaced agent, -1 when the job was free, -2 on an error.
template <int kGroup>
__device__ __forceinline__ int32_t da_propose(const Workspace& w, int32_t i, bool first, int grp, int gt,
                                              unsigned long long* s_red, unsigned long long* s_top,
                                              int32_t* s_out, int32_t& scans) {
    constexpr int kWarps = kGroup / 32;
    constexpr unsigned long long kHi = 0xFFFFFFFF00000000ull;
    DeviceState* st = w.st;
    const int32_t n = w.n;
    const int glane = gt & 31, gwarp = gt >> 5;
    const int32_t* row = w.a + (size_t)i * w.lda;
    const uint32_t me_lo = ~(uint32_t)i;
    unsigned long long* list = w.g_list + 4 * (size_t)i;
    for (int32_t attempt = 0;; ++attempt) {
        unsigned long long best = 0;
        if (gt == 0) {
            int32_t need_scan = 0;
            if (attempt == 0 && first) {
                best = w.g_row[i];
            } else {  // the first list entry whose holder this agent beats
                unsigned long long l[kDaList], h[kDaList];
#pragma unroll
                for (int m = 0; m < kDaList; ++m) l[m] = list[m];
#pragma unroll
                for (int m = 0; m < kDaList; ++m) h[m] = l[m] ? __ldcg(w.g_col + key_index(l[m])) : ~0ull;
                int32_t used = kDaList;
#pragma unroll
                for (int m = kDaList - 1; m >= 0; --m)
                    if (l[m] != 0 && ((l[m] & kHi) | me_lo) > h[m]) {
                        best = l[m];
                        used = m + 1;
                    }
                if (best == 0) need_scan = 1;
#pragma unroll
                for (int m = 0; m < kDaList; ++m)
                    if (m < used) list[m] = 0ull;  // consumed
            }
            *s_out = need_scan;
        }
        group_bar<kGroup>(grp);
        const bool need_scan = *s_out != 0;
        group_bar<kGroup>(grp);
        if (need_scan) {
            // the four best jobs whose holders this agent beats
            ++scans;
            unsigned long long t[4] = {0ull, 0ull, 0ull, 0ull};
            // the whole row is requested into L2 at once (prefetches hold no
            // registers), so that the batches below wait for L2, not DRAM
            for (int32_t c = gt * 32; c < n; c += 32 * kGroup)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(row + c));
            constexpr int kB = 2;  // 16-byte loads of the row (and 32 bytes of holder keys each) in flight
            for (int32_t c0 = gt * 4; c0 < n; c0 += 4 * kGroup * kB) {
                int4 v[kB];
                ulonglong2 h[kB][2];
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int32_t c = c0 + b * 4 * kGroup;
                    if (c < n) {
                        v[b] = __ldcs(reinterpret_cast<const int4*>(row + c));
                        h[b][0] = __ldcg(reinterpret_cast<const ulonglong2*>(w.g_col + c));
                        h[b][1] = __ldcg(reinterpret_cast<const ulonglong2*>(w.g_col + c + 2));
                    }
                }
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int32_t c = c0 + b * 4 * kGroup;
                    if (c >= n) continue;
                    const int32_t vals[4] = {v[b].x, v[b].y, v[b].z, v[b].w};
                    const unsigned long long hs[4] = {h[b][0].x, h[b][0].y, h[b][1].x, h[b][1].y};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const unsigned long long x = (uint32_t)(vals[e] + kBenefitLimit);
                        if (c + e < n && ((x << 32) | me_lo) > hs[e])
                            top4_insert(t, (x << 32) | (unsigned long long)(~(uint32_t)(c + e)));
                    }
                }
            }
            unsigned long long wt[4];
            warp_top4(t, wt);
            if (kWarps == 1) {
                if (gt == 0) {
                    best = wt[0];
#pragma unroll
                    for (int m = 0; m < kDaList; ++m) list[m] = wt[1 + m];
                }
            } else {
            if (glane == 0) {
#pragma unroll
                for (int r = 0; r < 4; ++r) s_red[(grp * kWarps + gwarp) * 4 + r] = wt[r];
            }
            group_bar<kGroup>(grp);
            if (gwarp == 0) {  // the group's first warp merges its warps' candidates
                unsigned long long c4[4] = {0ull, 0ull, 0ull, 0ull};
                for (int q = glane; q < kWarps * 4; q += 32) top4_insert(c4, s_red[grp * kWarps * 4 + q]);
                unsigned long long gt4[4];
                warp_top4(c4, gt4);
                if (glane == 0) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) s_top[grp * 4 + r] = gt4[r];
                }
            }
            group_bar<kGroup>(grp);
            if (gt == 0) {
                best = s_top[grp * 4];
#pragma unroll
                for (int m = 0; m < kDaList; ++m) list[m] = s_top[grp * 4 + 1 + m];
            }
            }
        }
        if (gt == 0) {
            int32_t out = -1;
            const int32_t j = key_index(best);
            // some job always accepts a free agent, and every failed proposal
            // or rejected list entry rules a job out, so an agent needs at
            // most 2 n + 2 attempts
            if (best == 0 || j < 0 || j >= n || attempt > 2 * n + 2) {
                st->error = kErrInternal;
                st->status = kError;
                out = -2;
            } else {
                const unsigned long long mine = (best & kHi) | me_lo;
                const unsigned long long old = atomic_max_acq_rel(w.g_col + j, mine);
                if (old < mine) {
                    out = old == 0 ? -1 : key_index(old);
                } else {
                    out = -3;  // the job was taken meanwhile: the list, else a rescan
                }
            }
            *s_out = out;
        }
        group_bar<kGroup>(grp);
        const int32_t out = *s_out;
        group_bar<kGroup>(grp);
        if (out != -3) return out;
    }
}

template <int kGroup>
__global__ void __launch_bounds__(kDaThreads, 1) greedy_da_kernel(Workspace w) {
    constexpr int kGroups = kDaThreads / kGroup;
    DeviceState* st = w.st;
    __shared__ unsigned long long s_red[kDaThreads / 32 * 4];
    __shared__ unsigned long long s_top[kGroups * 4];
    __shared__ int32_t s_out[kGroups];
    __shared__ int32_t s_status;
    if (threadIdx.x == 0) s_status = *(volatile int32_t*)&st->status;
    __syncthreads();
    if (s_status != kRunning) return;
    const int32_t n = w.n;
    const int tid = threadIdx.x, grp = tid / kGroup, gt = tid % kGroup;
    int32_t scans = 0, longest = 0;
    bool worked = false;
    const uint64_t t_start = globaltimer_ns();
    for (;;) {
        if (gt == 0) s_out[grp] = atomicAdd(&st->da_next, 1);
        group_bar<kGroup>(grp);
        int32_t a = s_out[grp];
        group_bar<kGroup>(grp);
        if (a >= n) break;
        bool first = true;
        int32_t d, steps = 0;
        worked = true;
        // the chain of displacements that starts with agent a
        while ((d = da_propose<kGroup>(w, a, first, grp, gt, s_red, s_top, &s_out[grp], scans)) >= 0) {
            a = d;
            first = false;
            ++steps;
            longest = max(longest, steps);
            if (gt == 0 && globaltimer_ns() - t_start > kDaTimeoutNs) {
                st->error = kErrWaitTimeout;
                st->status = kError;
                s_out[grp] = 1;
            } else if (gt == 0) {
                s_out[grp] = 0;
            }
            group_bar<kGroup>(grp);
            const bool late = s_out[grp] != 0;
            group_bar<kGroup>(grp);
            if (late) {
                d = -2;
                break;
            }
        }
        if (d == -2) break;
    }
    if (gt == 0 && scans) atomicAdd((unsigned long long*)&st->greedy_rescans, (unsigned long long)scans);
    if (gt == 0 && worked) atomicMax(&st->greedy_rounds, longest + 1);  // proposals along the longest chain
    if (gt == 0 && w.phase_ns) {  // diagnostics (DGS_PHASE_TIMERS=1)
        const uint64_t t = globaltimer_ns() - t_start;
        atomicMax(w.phase_ns + kPtDaLastNs, (unsigned long long)t);
        atomicAdd(w.phase_ns + kPtDaSumNs, (unsigned long long)t);
        atomicMax(w.phase_ns + kPtDaChain, (unsigned long long)longest);
        atomicMax(w.phase_ns + kPtDaGroupScans, (unsigned long long)scans);
    }
}

// Loop condition of the locally-dominant rounds run as a device-side loop
// (three kernels and this one per iteration): go on while agents are
// unmatched; more than n + 8 rounds is an internal error.
__global__ void greedy_loop_cond_kernel(Workspace w, unsigned long long cond) {
    DeviceState* st = w.st;
    const int32_t it = ++st->loop_iterations;
    st->loop_launches += 4;
    if (st->status == kRunning && st->greedy_remaining > 0 && it > w.n + 8) {
        st->error = kErrInternal;
        st->status = kError;
    }
    cudaGraphSetConditional(cond, (st->status == kRunning && st->greedy_remaining > 0) ? 1u : 0u);
}

// The assignment from the jobs' holders.
__global__ void greedy_da_finish_kernel(Workspace w) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->greedy_remaining = 0;
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < w.n; j += gridDim.x * blockDim.x) {
        const int32_t i = key_index(w.g_col[j]);
        if (i < 0 || i >= w.n) {
            st->error = kErrInternal;
            st->status = kError;
            continue;
        }
        w.sigma[j] = i;
        w.tau[i] = j;
    }
}

// |a| < 2^29 check alone (for entry points that do not run pass 1).
__global__ void range_check_kernel(Workspace w) {
    bool bad = false;
    int32_t amax = 0;
    const size_t total4 = (size_t)w.n * (size_t)(w.lda / 4);
    const int32_t row4 = w.lda / 4;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total4; q += (size_t)gridDim.x * blockDim.x) {
        const int32_t c = (int32_t)(q % row4) * 4;
        const int4 v = reinterpret_cast<const int4*>(w.a)[q];
        const int32_t vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (c + e < w.n) {
                bad |= (vals[e] >= kBenefitLimit) || (vals[e] <= -kBenefitLimit);
                amax = max(amax, vals[e] == INT32_MIN ? INT32_MAX : abs(vals[e]));
            }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    if ((threadIdx.x & 31) == 0 && amax) atomicMax(&w.st->max_abs, amax);
    if (bad) {
        atomicExch(&w.st->error, kErrRange);
        atomicExch(&w.st->status, kError);
    }
}

__global__ void __launch_bounds__(256) greedy_pass1_batched_kernel(BatchQueues q) {
    for_each_item(q.inst, q.q0, q.cap, [&](const Instance& in, int32_t bid, int32_t nblk) {
        const int32_t tx = (in.w.n + kT - 1) / kT;
        greedy_pass1_body(in.w, tx, tx * tx, bid, nblk, in.a_src, false);
    });
}

// Deferred acceptance of every instance in kStageGreedy in one launch: the
// agents of all those instances form one index space (prefix offsets q0 of
// the kScanGreedyDA scan, which also zeroes q1[0], the shared counter); a
// group takes the next agent of that space and follows its chain of
// displacements inside its instance, exactly as greedy_da_kernel does for a
// single solve.
template <int kGroup>
__global__ void __launch_bounds__(kDaThreads, 1) greedy_da_batched_kernel(BatchQueues q) {
    constexpr int kGroups = kDaThreads / kGroup;
    __shared__ unsigned long long s_red[kDaThreads / 32 * 4];
    __shared__ unsigned long long s_top[kGroups * 4];
    __shared__ int32_t s_out[kGroups];
    const int32_t total = q.q0[q.cap];
    if (total <= 0) return;
    const int tid = threadIdx.x, grp = tid / kGroup, gt = tid % kGroup;
    int32_t scans = 0, k_last = -1;
    for (;;) {
        if (gt == 0) s_out[grp] = atomicAdd(q.q1, 1);
        group_bar<kGroup>(grp);
        const int32_t g = s_out[grp];
        group_bar<kGroup>(grp);
        if (g >= total) break;
        int32_t lo = 0, hi = q.cap;  // q0[lo] <= g < q0[hi]
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (q.q0[mid] <= g) lo = mid;
            else hi = mid;
        }
        const Instance& in = q.inst[lo];
        if (k_last != lo && k_last >= 0 && gt == 0 && scans)  // rescans are counted per instance
            atomicAdd((unsigned long long*)&q.inst[k_last].w.st->greedy_rescans, (unsigned long long)scans);
        if (k_last != lo) scans = 0;
        k_last = lo;
        int32_t a = g - q.q0[lo];
        bool first = true;
        int32_t d, steps = 1;
        while ((d = da_propose<kGroup>(in.w, a, first, grp, gt, s_red, s_top, &s_out[grp], scans)) >= 0) {
            a = d;
            first = false;
            ++steps;
        }
        if (gt == 0 && d == -1) atomicMax(&in.w.st->greedy_rounds, steps);
    }
    if (k_last >= 0 && gt == 0 && scans)
        atomicAdd((unsigned long long*)&q.inst[k_last].w.st->greedy_rescans, (unsigned long long)scans);
}

// The assignment of every instance in kStageGreedy from its jobs' holders
// (greedy_da_finish_kernel per instance).
__global__ void greedy_da_finish_batched_kernel(BatchTable t) {
    for_each_entry(t, kStageGreedy, [&](const Instance& in, int32_t bid, int32_t nblk) {
        const Workspace& w = in.w;
        DeviceState* st = w.st;
        // every queued agent of the instance was placed by the launch before
        // (the instance's blocks must not test greedy_remaining, which block
        // 0 clears here for the advance kernel)
        if (st->status != kRunning) return;
        if (bid == 0 && threadIdx.x == 0) st->greedy_remaining = 0;
        for (int32_t j = bid * blockDim.x + threadIdx.x; j < w.n; j += nblk * blockDim.x) {
            const int32_t i = key_index(w.g_col[j]);
            if (i < 0 || i >= w.n) {
                st->error = kErrInternal;
                st->status = kError;
                continue;
            }
            w.sigma[j] = i;
            w.tau[i] = j;
        }
    });
}

}  // namespace

cudaError_t launch_range_check(const Workspace& w, cudaStream_t s) {
    range_check_kernel<<<dgs::device_sms() * 4, 256, 0, s>>>(w);
    return cudaGetLastError();
}

// Pass 1 over the rows of tile rows [row_tile0, row_tile1) (64 rows each):
// the bands of a matrix that arrives in pieces can be processed as they land.
cudaError_t launch_greedy_pass1_rows(const Workspace& w, int32_t cols, int32_t row_tile0, int32_t row_tile1,
                                     cudaStream_t s) {
    const int32_t tx = (w.n + kT - 1) / kT;
    const int32_t t0 = row_tile0 * tx, t1 = (row_tile1 < tx ? row_tile1 : tx) * tx;
    const int32_t count = t1 - t0;
    if (count <= 0) return cudaSuccess;
    const int32_t grid = count < dgs::device_sms() * 8 ? count : dgs::device_sms() * 8;
    greedy_pass1_kernel<<<grid, 256, 0, s>>>(w, tx, t1, cols, t0);
    return cudaGetLastError();
}

cudaError_t launch_greedy_pass1_cols(const Workspace& w, int32_t cols, cudaStream_t s) {
    return launch_greedy_pass1_rows(w, cols, 0, (w.n + kT - 1) / kT, s);
}

cudaError_t launch_greedy_pass1(const Workspace& w, cudaStream_t s) { return launch_greedy_pass1_cols(w, 1, s); }

cudaError_t launch_greedy_loop_cond(const Workspace& w, unsigned long long handle, cudaStream_t s) {
    greedy_loop_cond_kernel<<<1, 1, 0, s>>>(w, handle);
    return cudaGetLastError();
}

cudaError_t launch_greedy_round(const Workspace& w, cudaStream_t s) {
    const int32_t nb = (w.n + 255) / 256;
    greedy_match_kernel<<<nb < dgs::device_sms() * 4 ? nb : dgs::device_sms() * 4, 256, 0, s>>>(w);
    const int32_t g = w.n < dgs::device_sms() * 8 ? w.n : dgs::device_sms() * 8;  // one owner per CTA at a time
    greedy_rescan_kernel<<<g, 256, 0, s>>>(w, w.a, w.lda, w.g_row, w.free_a, w.free_j, 1);
    greedy_rescan_kernel<<<g, 256, 0, s>>>(w, w.at, w.ldt, w.g_col, w.free_j, w.free_a, 0);
    return cudaGetLastError();
}

// Pass 1 of the instances queued by the kScanPass1 scan (blocks over the
// 64x64 tiles of a).
cudaError_t launch_b_pass1(const BatchQueues& q, cudaStream_t s) {
    greedy_pass1_batched_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(q);
    return cudaGetLastError();
}

// Threads per proposal of the deferred acceptance (DGS_DA_GROUP = 32, 128,
// 256 or 512; results do not depend on it).  Groups of more than one warp
// synchronise on named barriers 1..15, one per group of the block.
int32_t da_group_env() {
    static const int32_t v = [] {
        const char* e = std::getenv("DGS_DA_GROUP");
        const int32_t x = e ? std::atoi(e) : 256;
        return (x == 32 || x == 128 || x == 512) ? x : 256;
    }();
    return v;
}

template <template <int> class K>
const void* da_kernel_for(int32_t g) {
    return g == 32 ? reinterpret_cast<const void*>(K<32>::fn)
         : g == 128 ? reinterpret_cast<const void*>(K<128>::fn)
         : g == 512 ? reinterpret_cast<const void*>(K<512>::fn)
                    : reinterpret_cast<const void*>(K<256>::fn);
}
template <int G> struct SingleDa { static constexpr auto fn = greedy_da_kernel<G>; };
template <int G> struct BatchedDa { static constexpr auto fn = greedy_da_batched_kernel<G>; };

// The greedy start of every instance in kStageGreedy (deferred acceptance:
// queue the agents, one launch, then the assignments; the advance kernel
// moves the instances on once greedy_remaining is 0).
cudaError_t launch_b_greedy(const BatchTable& rows, const BatchQueues& q, cudaStream_t s) {
    cudaError_t e = launch_b_scan(q, kScanGreedyDA, 0, s);
    if (e != cudaSuccess) return e;
    BatchQueues arg = q;
    void* args[] = {&arg};
    e = cudaLaunchKernel(da_kernel_for<BatchedDa>(da_group_env()), dim3(dgs::device_sms()), dim3(kDaThreads), args,
                         0, s);
    if (e != cudaSuccess) return e;
    greedy_da_finish_batched_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(rows);
    return cudaGetLastError();
}



// DGS_GREEDY_ROUNDS=1: the locally-dominant rounds instead of deferred
// acceptance (tests; the same assignment).  Read at every call.
int32_t greedy_rounds_env() {
    const char* e = std::getenv("DGS_GREEDY_ROUNDS");
    return (e && std::atoi(e) == 1) ? 1 : 0;
}

cudaError_t launch_greedy_da(const Workspace& w, cudaStream_t s) {
    if (greedy_rounds_env() || w.g_list == nullptr) return cudaErrorNotSupported;
    const void* kernel = da_kernel_for<SingleDa>(da_group_env());
    Workspace arg = w;
    void* args[] = {&arg};
    cudaError_t e = cudaLaunchKernel(kernel, dim3(dgs::device_sms()), dim3(kDaThreads), args, 0, s);
    if (e != cudaSuccess) return e;
    const int32_t nb = (w.n + 255) / 256;
    greedy_da_finish_kernel<<<nb < dgs::device_sms() * 4 ? nb : dgs::device_sms() * 4, 256, 0, s>>>(w);
    return cudaGetLastError();
}

}  // namespace dgs
