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
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kT = 64;  // tile edge

// a_src (batched instances only): the caller's matrix with row pitch n when w.a
// is the workspace's pitched copy still to be filled; this pass reads a_src
// and writes the copy as it goes.  Null: w.a is read.
__device__ __forceinline__ void greedy_pass1_body(const Workspace& w, int32_t tiles_x, int32_t tiles_total,
                                                  int32_t bid, int32_t nblk, const int32_t* a_src = nullptr) {
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
        {
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
        if (t < kT) {
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

__global__ void __launch_bounds__(256) greedy_pass1_kernel(Workspace w, int32_t tiles_x, int32_t tiles_total) {
    greedy_pass1_body(w, tiles_x, tiles_total, blockIdx.x, gridDim.x);
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

// All rounds in one cooperative launch, one grid barrier per round.  Every
// CTA keeps its own copy of the free-agent and free-job sets as bitmaps in
// shared memory and computes the round's matches redundantly from the keys
// (all CTAs reach the same result), then the full list of owners to rescan;
// CTA b rescans the entries of rank b, b + G, ... of that list, so the work
// is balanced without further synchronisation.  Round r equals round r of
// the launch-per-round path.
constexpr int kPThreads = 1024;
constexpr int kPGroups = 8;          // rescans run in groups of 128 threads
constexpr int kPMaxBitWords = 2048;  // n <= 65536 (larger n: one launch per round)
constexpr int kPMaxMine = 512;       // rescans per CTA per round held in shared memory

__device__ __forceinline__ bool bit_get(const uint32_t* bm, int32_t i) { return (bm[i >> 5] >> (i & 31)) & 1u; }

// Flags and keys written by other CTAs during the launch are read with
// __ldcg (from L2): L1 is not coherent across SMs.
__global__ void __launch_bounds__(kPThreads, 1) greedy_persistent_kernel(Workspace w) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    __shared__ uint32_t s_free_a[kPMaxBitWords], s_free_j[kPMaxBitWords], s_dirty[2 * kPMaxBitWords];
    __shared__ int32_t s_mine[kPMaxMine];
    __shared__ int32_t s_nmine, s_rem, s_warp[33];
    __shared__ unsigned long long s_red[kPThreads / 32];
    const int32_t n = w.n, G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int32_t words = (n + 31) >> 5;
    for (int32_t q = tid; q < words; q += kPThreads) {
        const int32_t hi = min(32, n - 32 * q);
        const uint32_t m = hi == 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u);
        s_free_a[q] = m;
        s_free_j[q] = m;
    }
    // the global copies start full (set by the host); every CTA reads them
    // only after the first barrier
    __syncthreads();
    unsigned long long* pt = w.phase_ns;
    const bool timing = pt != nullptr && tid == 0;
    uint64_t tp = timing ? globaltimer_ns() : 0, scan_total = 0;
#define DGS_PT(slot)                                   \
    if (timing && b == 0) {                            \
        const uint64_t now = globaltimer_ns();         \
        atomicAdd(pt + (slot), now - tp);              \
        tp = now;                                      \
    } else if (timing) {                               \
        tp = globaltimer_ns();                         \
    }
    int32_t rounds = 0;
    for (int32_t round = 0; round <= n; ++round) {
        // ---- every CTA copied last round's dirty bitmap before the round's
        // final barrier: clear it (the new flags are set after the next one)
        for (int32_t q = b * kPThreads + tid; q < (2 * n + 31) >> 5; q += G * kPThreads) w.g_dirty[q] = 0u;
        // ---- match every mutually-best pair: each CTA its slice of agents,
        // recorded in the global free bitmaps; then every CTA copies them
        for (int32_t i0 = b * kPThreads + tid; i0 < n; i0 += 4 * G * kPThreads) {
            int32_t jj[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t i = i0 + k * G * kPThreads;
                jj[k] = (i < n && bit_get(s_free_a, i)) ? key_index(__ldcg(w.g_row + i)) : -1;
            }
            int32_t back[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) back[k] = (jj[k] >= 0 && jj[k] < n) ? key_index(__ldcg(w.g_col + jj[k])) : -2;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t i = i0 + k * G * kPThreads, j = jj[k];
                if (back[k] != i) continue;
                atomicAnd(w.g_free_a + (i >> 5), ~(1u << (i & 31)));
                atomicAnd(w.g_free_j + (j >> 5), ~(1u << (j & 31)));
                w.tau[i] = j;
                w.sigma[j] = i;
            }
        }
        if (!grid_barrier(st)) {
            if (tid == 0) { st->error = kErrWaitTimeout; st->status = kError; }
            return;
        }
        for (int32_t q = tid; q < words; q += kPThreads) {
            s_free_a[q] = __ldcg(w.g_free_a + q);
            s_free_j[q] = __ldcg(w.g_free_j + q);
        }
        __syncthreads();
        ++rounds;
        // ---- remaining free agents, and the owners to rescan (rows: free
        // agents whose best job was taken; columns: the converse)
        if (tid == 0) { s_rem = 0; s_nmine = 0; }
        __syncthreads();
        {
            int32_t rem = 0;
            for (int32_t q = tid; q < words; q += kPThreads) {
                const int32_t hi = min(32, n - 32 * q);  // bits of agents >= n are not counted
                rem += __popc(s_free_a[q] & (hi == 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) rem += __shfl_xor_sync(0xffffffffu, rem, off);
            if ((tid & 31) == 0 && rem) atomicAdd(&s_rem, rem);
        }
        __syncthreads();
        if (b == 0 && tid == 0) st->greedy_remaining = s_rem;
        DGS_PT(kPtGreedyMatch)
        if (s_rem == 0 || *(volatile int32_t*)&st->status != kRunning) break;
        // owners are numbered 0..2n-1 (rows, then columns): each CTA flags
        // the dirty owners of its slice in the global bitmap (cleared by the
        // previous round), then every CTA copies the bitmap and ranks it
        const int32_t owner_words = (2 * n + 31) >> 5;
        for (int32_t o0 = b * kPThreads + tid; o0 < 2 * n; o0 += 4 * G * kPThreads) {
            int32_t best[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t o = o0 + k * G * kPThreads;
                best[k] = -3;
                if (o < 2 * n) {
                    const bool is_row = o < n;
                    const int32_t x = is_row ? o : o - n;
                    if (bit_get(is_row ? s_free_a : s_free_j, x))
                        best[k] = key_index(__ldcg(is_row ? w.g_row + x : w.g_col + x));
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (best[k] == -3) continue;
                const int32_t o = o0 + k * G * kPThreads;
                const bool is_row = o < n;
                const bool taken = best[k] < 0 || best[k] >= n || !bit_get(is_row ? s_free_j : s_free_a, best[k]);
                if (taken) atomicOr(w.g_dirty + (o >> 5), 1u << (o & 31));
            }
        }
        if (!grid_barrier(st)) {
            if (tid == 0) { st->error = kErrWaitTimeout; st->status = kError; }
            return;
        }
        for (int32_t q = tid; q < owner_words; q += kPThreads) s_dirty[q] = __ldcg(w.g_dirty + q);
        __syncthreads();
        int32_t base_rank = 0;
        for (int32_t w0 = 0; w0 < owner_words; w0 += kPThreads) {
            const int32_t q = w0 + tid;
            uint32_t dirty = q < owner_words ? s_dirty[q] : 0u;
            const int32_t c = __popc(dirty);
            int32_t total;
            // exclusive block scan of c
            int32_t incl = c;
            const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int32_t o = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += o;
            }
            if (lane == 31) s_warp[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const int32_t v = s_warp[lane];
                int32_t wi = v;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int32_t o = __shfl_up_sync(0xffffffffu, wi, off);
                    if (lane >= off) wi += o;
                }
                s_warp[lane] = wi - v;
                if (lane == 31) s_warp[32] = wi;
            }
            __syncthreads();
            const int32_t rank = base_rank + s_warp[warp] + incl - c;
            total = s_warp[32];
            // this word's owners take ranks rank .. rank + c - 1; the ones this
            // CTA rescans are the set bits of index i = (b - rank) mod G,
            // i + G, ... below c
            for (int32_t i = ((b - rank) % G + G) % G; i < c; i += G) {
                uint32_t d = dirty;
                for (int32_t skip = 0; skip < i; ++skip) d &= d - 1u;  // drop the i lowest set bits
                const int32_t slot = atomicAdd(&s_nmine, 1);
                if (slot < kPMaxMine) s_mine[slot] = 32 * q + (__ffs(d) - 1);
            }
            base_rank += total;
            __syncthreads();
        }
        if (s_nmine > kPMaxMine) {  // cannot happen for n <= 131072 with G >= 152
            if (tid == 0) { st->error = kErrInternal; st->status = kError; }
            break;
        }
        DGS_PT(kPtGreedyCheck)
        if (tid == 0 && s_nmine) atomicAdd((unsigned long long*)&st->greedy_rescans, (unsigned long long)s_nmine);
        // ---- rescan this CTA's owners: eight 128-thread groups
        const int32_t cnt = s_nmine;
        const int grp = tid >> 7, gt = tid & 127, glane = tid & 31, gwarp = (tid >> 5) & 3;
        for (int32_t t = grp; t < cnt; t += kPGroups) {
            const int32_t o2 = s_mine[t];
            const bool is_row = o2 < n;
            const int32_t o = is_row ? o2 : o2 - n;
            const int32_t* row = is_row ? w.a + (size_t)o * w.lda : w.at + (size_t)o * w.ldt;
            const uint32_t* pfree = is_row ? s_free_j : s_free_a;
            unsigned long long best = 0;
#pragma unroll 8
            for (int32_t c = gt * 4; c < n; c += 4 * 128) {
                const int4 v = *reinterpret_cast<const int4*>(row + c);
                const uint32_t fr = (pfree[c >> 5] >> (c & 31)) & 0xFu;
                const int32_t vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (c + e < n && ((fr >> e) & 1u)) best = umax64(best, pack_benefit(vals[e], (uint32_t)(c + e)));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, off));
            if (glane == 0) s_red[grp * 4 + gwarp] = best;
            asm volatile("bar.sync %0, 128;" ::"r"(grp + 1) : "memory");
            if (gt == 0) {
                const unsigned long long m = umax64(umax64(s_red[grp * 4], s_red[grp * 4 + 1]),
                                                    umax64(s_red[grp * 4 + 2], s_red[grp * 4 + 3]));
                (is_row ? w.g_row : w.g_col)[o] = m;
            }
            asm volatile("bar.sync %0, 128;" ::"r"(grp + 1) : "memory");
        }
        __syncthreads();
        if (timing) scan_total += globaltimer_ns() - tp;
        DGS_PT(kPtGreedyScan)
        if (!grid_barrier(st)) {
            if (tid == 0) { st->error = kErrWaitTimeout; st->status = kError; }
            return;
        }
        DGS_PT(kPtGreedyBar2)
    }
    if (timing) atomicMax(pt + kPtGreedyScanMax, (unsigned long long)scan_total);
#undef DGS_PT
    if (b == 0 && tid == 0) st->greedy_rounds = rounds;
    // the free flags of the round-based path are not used after this kernel
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
        greedy_pass1_body(in.w, tx, tx * tx, bid, nblk, in.a_src);
    });
}

__global__ void __launch_bounds__(256) greedy_match_batched_kernel(BatchTable t) {
    for_each_entry(t, kStageGreedy, [&](const Instance& in, int32_t bid, int32_t nblk) {
        greedy_match_body(in.w, bid, nblk);
    });
}

// After a match: list the owners to rescan (owners 0..n-1 are agents, rows of
// a; n..2n-1 are jobs, rows of at): free owners whose best partner was just
// taken.  The list lives in ctl_slot (unused until the switching loop) and
// its length in rescan_count (the scan kernel reads and clears it).
__global__ void __launch_bounds__(256) greedy_dirty_batched_kernel(BatchTable t) {
    for_each_entry(t, kStageGreedy, [&](const Instance& in, int32_t bid, int32_t nblk) {
        const Workspace& w = in.w;
        DeviceState* st = w.st;
        if (st->status != kRunning || st->greedy_remaining == 0) return;
        const int32_t n = w.n;
        for (int32_t o = bid * blockDim.x + threadIdx.x; o < 2 * n; o += nblk * blockDim.x) {
            const bool is_row = o < n;
            const int32_t x = is_row ? o : o - n;
            if (!(is_row ? w.free_a[x] : w.free_j[x])) continue;
            const int32_t b = key_index(is_row ? w.g_row[x] : w.g_col[x]);
            if (b >= 0 && b < n && (is_row ? w.free_j[b] : w.free_a[b])) continue;
            w.ctl_slot[atomicAdd(&st->rescan_count, 1)] = o;
        }
    });
}

// One listed owner per item: its best free partner over its whole row, with
// the CTA (the same scan as greedy_rescan_kernel).
__global__ void __launch_bounds__(256) greedy_rescan_batched_kernel(BatchQueues q) {
    __shared__ unsigned long long red[8];
    for_each_item(q.inst, q.q0, q.cap, [&](const Instance& in, int32_t t, int32_t) {
        const Workspace& w = in.w;
        const int32_t n = w.n;
        const int32_t o2 = w.ctl_slot[t];
        const bool is_row = o2 < n;
        const int32_t o = is_row ? o2 : o2 - n;
        const int32_t* row = is_row ? w.a + (size_t)o * w.lda : w.at + (size_t)o * w.ldt;
        const uint8_t* partner_free = is_row ? w.free_j : w.free_a;
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
            for (int k = 0; k < 8; ++k) m = umax64(m, red[k]);
            (is_row ? w.g_row : w.g_col)[o] = m;
        }
        __syncthreads();
    });
}

}  // namespace

cudaError_t launch_range_check(const Workspace& w, cudaStream_t s) {
    range_check_kernel<<<152 * 4, 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_greedy_pass1(const Workspace& w, cudaStream_t s) {
    const int32_t tx = (w.n + kT - 1) / kT;
    const int32_t total = tx * tx;
    const int32_t grid = total < 152 * 8 ? total : 152 * 8;
    greedy_pass1_kernel<<<grid, 256, 0, s>>>(w, tx, total);
    return cudaGetLastError();
}

cudaError_t launch_greedy_round(const Workspace& w, cudaStream_t s) {
    const int32_t nb = (w.n + 255) / 256;
    greedy_match_kernel<<<nb < 152 * 4 ? nb : 152 * 4, 256, 0, s>>>(w);
    const int32_t g = w.n < 152 * 8 ? w.n : 152 * 8;  // one owner per CTA at a time
    greedy_rescan_kernel<<<g, 256, 0, s>>>(w, w.a, w.lda, w.g_row, w.free_a, w.free_j, 1);
    greedy_rescan_kernel<<<g, 256, 0, s>>>(w, w.at, w.ldt, w.g_col, w.free_j, w.free_a, 0);
    return cudaGetLastError();
}

// Pass 1 of the instances queued by the kScanPass1 scan (blocks over the
// 64x64 tiles of a).
cudaError_t launch_b_pass1(const BatchQueues& q, cudaStream_t s) {
    greedy_pass1_batched_kernel<<<152 * 8, 256, 0, s>>>(q);
    return cudaGetLastError();
}

// One locally-dominant round of the instances in kStageGreedy: match (rows:
// entries over agents and jobs), list the owners to rescan, queue them
// (scan), rescan each with one CTA.
cudaError_t launch_b_greedy_round(const BatchTable& rows, const BatchQueues& q, cudaStream_t s) {
    greedy_match_batched_kernel<<<152 * 8, 256, 0, s>>>(rows);
    greedy_dirty_batched_kernel<<<152 * 8, 256, 0, s>>>(rows);
    cudaError_t e = launch_b_scan(q, kScanGreedy, 0, s);
    if (e != cudaSuccess) return e;
    greedy_rescan_batched_kernel<<<152 * 8, 256, 0, s>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_greedy_persistent(const Workspace& w, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, greedy_persistent_kernel, kPThreads, 0);
    if (e != cudaSuccess) return e;
    int grid = sms * (per_sm < 1 ? per_sm : 1);
    if (w.g_free_a == nullptr || w.g_free_j == nullptr || w.g_dirty == nullptr) return cudaErrorNotSupported;
    if (grid < 1) return cudaErrorNotSupported;
    if (w.n > 32 * kPMaxBitWords || (int64_t)2 * w.n > (int64_t)kPMaxMine * grid) return cudaErrorNotSupported;
    Workspace arg = w;
    void* args[] = {&arg};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(greedy_persistent_kernel), dim3(grid),
                                       dim3(kPThreads), args, 0, s);
}

}  // namespace dgs
