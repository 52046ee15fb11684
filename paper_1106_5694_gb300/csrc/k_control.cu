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
//     greedy matching of the edges) is computed exactly, chunk by chunk of
//     the priority order: edges touching an agent claimed by an earlier chunk
//     are rejected at once; the chunk's other edges run deterministic
//     reservations among themselves (each writes its priority into both
//     agents with atomicMin; an edge holding both agents is accepted and
//     claims them; edges touching a claimed agent are rejected; repeat).
//     Rejected edges form the set C (reading R3).  An accepted edge has no
//     earlier accepted neighbour and every rejected edge has one, which is
//     exactly the sequential outcome.
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
#include <algorithm>
#include <cstdlib>

#include "../../include/dgs.h"
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kCtlThreads = 1024;

// Slot edge word: agent u (bits 0..16), agent v (17..33), applies (34): its
// exchange raises f under the current sigma, valid (36): set on every edge
// (0 means "no candidate").  Edge positions follow slot priority, so a position is a priority.
constexpr unsigned long long kApplies = 1ull << 34;
constexpr unsigned long long kValid = 1ull << 36;  // a slot's edge word is never 0
__device__ __forceinline__ unsigned long long edge_word(int32_t u, int32_t v) {
    return (unsigned long long)(uint32_t)u | ((unsigned long long)(uint32_t)v << 17) | kValid;
}
__device__ __forceinline__ int32_t edge_u(unsigned long long e) { return (int32_t)(e & 0x1FFFFu); }
__device__ __forceinline__ int32_t edge_v(unsigned long long e) { return (int32_t)((e >> 17) & 0x1FFFFu); }

__device__ __forceinline__ int32_t exchange_gain(const Workspace& w, int32_t u, int32_t v) {
    if (u == v) return 0;
    const int32_t ju = w.tau[u], jv = w.tau[v];
    return w.a[(size_t)u * w.lda + jv] + w.a[(size_t)v * w.lda + ju] - w.diag[ju] - w.diag[jv];
}

// Block-wide exclusive scan of one int per thread (1024 threads).
// (kT threads, at most 1024; warp_sums holds 33 entries)
template <int kT = 1024>
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
        const int32_t v = lane < kT / 32 ? warp_sums[lane] : 0;
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

// Controller scratch.  res: per agent, the reservation key of the current DR
// round; claimed: per agent, the stamp of the sweep that claimed it; estate:
// per edge position (alive / applies / fresh bits); E: per edge position, the
// two agents of its exchange.  The list of accepted positions is two-tier:
// the first `cap` entries in shared memory (16-bit positions), the rest in
// global memory.
struct CtlScratch {
    uint32_t* res;
    uint8_t* claimed;
    uint8_t* estate;
    void* edges;
    int32_t* acc_g;  // accepted positions beyond the shared-memory part
};

enum : uint8_t { kAlive = 1, kAppl = 2, kFreshBit = 4, kAccBit = 8 };

struct TwoTier {
    uint16_t* s;
    int32_t cap;
    int32_t* g;
    __device__ __forceinline__ void put(int32_t i, int32_t v) const {
        if (i < cap) s[i] = (uint16_t)v;
        else g[i - cap] = v;
    }
    __device__ __forceinline__ int32_t get(int32_t i) const { return i < cap ? (int32_t)s[i] : g[i - cap]; }
};

// Reservation key of edge position p in DR round r: each round's keys are
// smaller than every earlier round's, so reservations never need clearing
// (the array is reset once per key period).
constexpr uint32_t kPosBits = 18, kRoundSpanMax = 1u << 14;
__device__ __forceinline__ uint32_t round_base(uint32_t r, uint32_t span) {
    return (span - 1u - (r & (span - 1u))) << kPosBits;
}

template <typename EdgeT>
struct Codec;
template <>
struct Codec<uint32_t> {  // n <= 65535
    static __device__ __forceinline__ uint32_t make(int32_t u, int32_t v) { return (uint32_t)u | ((uint32_t)v << 16); }
    static __device__ __forceinline__ int32_t u(uint32_t e) { return (int32_t)(e & 0xFFFFu); }
    static __device__ __forceinline__ int32_t v(uint32_t e) { return (int32_t)(e >> 16); }
};
template <>
struct Codec<unsigned long long> {
    static __device__ __forceinline__ unsigned long long make(int32_t u, int32_t v) {
        return (unsigned long long)(uint32_t)u | ((unsigned long long)(uint32_t)v << 32);
    }
    static __device__ __forceinline__ int32_t u(unsigned long long e) { return (int32_t)(uint32_t)e; }
    static __device__ __forceinline__ int32_t v(unsigned long long e) { return (int32_t)(e >> 32); }
};


// Re-evaluation records of the first kRecCap accepted edges of a sweep are
// copied into shared memory while the sweep's conflict check still runs
// (asynchronous copies, awaited before its last barrier), so that a quiet
// sweep's refresh reads no global memory; later ones are only prefetched.
constexpr int32_t kRecCap = 64, kRecBytes = 16 * kRecCap;
__device__ __forceinline__ void fetch_record(unsigned char* rec, int32_t idx, const Workspace& w, int32_t t) {
    if (rec != nullptr && idx < kRecCap) {
        const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(rec + 16 * idx));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(w.sl_rkey + t) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + 8), "l"(w.sl_ru + t) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + 12), "l"(w.sl_rv + t) : "memory");
    } else {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(w.sl_rkey + t));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(w.sl_ru + t));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(w.sl_rv + t));
    }
}

// Colouring pass.  In a sweep in which no accepted exchange applies (a quiet
// sweep) sigma does not change, so every accepted edge is stale and is only
// re-evaluated: it dies or comes back, applicable, at its position.  Round k
// of a run of such sweeps accepts the greedy set of the edges left after the
// rounds before it, so a stale edge is accepted exactly in the round that
// first-fit edge colouring in position order gives it (the smallest colour
// that no earlier stale edge sharing one of its agents has), and an
// applicable edge in the first round from its birth on that no earlier stale
// edge sharing an agent holds; the first such round ends the run with an
// event.  The pass colours the stale edges with colours below kColourCap by
// reservation rounds (an edge is coloured once it is the first pending edge
// at both its agents, from the colour masks of those agents, which then hold
// exactly its earlier neighbours' colours), finds the first round E in which
// an applicable edge is accepted and the first round R in which a re-
// evaluated edge that lives on is born (its colour + 1), and re-evaluates the
// edges of the F = min(E, R, kColourCap, sweeps left) rounds before both at
// once, as F quiet sweeps would; each round's count is left in s_hist.
// Colour masks use the claim array (cleared afterwards), colours the high
// half of the edge states.  Rounds past the last one with an accepted edge
// are not counted: with no edge left the run ends.  Returns F, or -1 on an
// internal error.
constexpr int32_t kColourCap = 8, kColourMinList = 1024;

template <typename EdgeT, int kT>
__device__ __forceinline__ int32_t colour_pass_rounds(const Workspace& w, EdgeT* E, uint8_t* estate,
                                                      const uint16_t* slot_s, uint32_t* res, uint8_t* mask,
                                                      int32_t L, uint32_t span, uint32_t& s_round, int32_t& s_pE,
                                                      int32_t& s_pR, int32_t& s_pF, int32_t* s_hist,
                                                      int32_t max_sweeps, int32_t sweeps, int32_t& s_live,
                                                      unsigned long long* s_pt) {
    using C = Codec<EdgeT>;
    const int tid = threadIdx.x;
    const int32_t n = w.n;
    for (int32_t i = tid; i < n; i += kT) mask[i] = 0;
    if (tid == 0) {
        s_pE = kColourCap;
        s_pR = kColourCap;
        for (int k = 0; k < kColourCap; ++k) s_hist[k] = 0;
    }
    __syncthreads();
    // The edges of the thread's first kHeld positions (tid + k kT)
    // and their states are held in registers for the whole pass: bit k of pm
    // says pending, of am applicable; nibble k of cols is the outcome (c + 1
    // coloured c, 15 closed).  Positions past them keep theirs in the high
    // half of the edge states.
    constexpr int kHeld = 8;
    EdgeT he[kHeld];
    uint32_t pm = 0, am = 0, cols = 0;
#pragma unroll
    for (int k = 0; k < kHeld; ++k) {
        const int32_t p = tid + k * kT;
        const uint8_t es = p < L ? estate[p] : (uint8_t)0;
        he[k] = (es & kAlive) ? E[p] : (EdgeT)0;
        if (es & kAlive) pm |= 1u << k;
        if (es & kAppl) am |= 1u << k;
    }
    const int32_t tail0 = kHeld * kT;
    // one pending edge, first half of a round: false if it closes (masks only
    // grow: a full one leaves no colour, or round, below the cap), else it
    // reserves both agents
    auto reserve = [&](int32_t p, EdgeT e, bool appl, uint32_t base) -> bool {
        const int32_t u = C::u(e), v = C::v(e);
        const uint32_t mu = mask[u], mv = mask[v];
        if (appl ? (mu | mv) == 0xFFu : (mu == 0xFFu || mv == 0xFFu)) return false;
        const uint32_t key = base | (uint32_t)p;
        if (key < res[u]) atomicMin(&res[u], key);
        if (key < res[v]) atomicMin(&res[v], key);
        return true;
    };
    // second half: -1 while an earlier edge at u or v is pending, else the
    // outcome; the edge is then the only one holding u and v, so its mask
    // updates are plain stores
    auto settle = [&](int32_t p, EdgeT e, bool appl, uint32_t base) -> int32_t {
        const int32_t u = C::u(e), v = C::v(e);
        const uint32_t key = base | (uint32_t)p;
        if (res[u] != key || res[v] != key) return -1;
        const uint32_t fr = ~((uint32_t)mask[u] | (uint32_t)mask[v]) & 0xFFu;
        if (appl) {
            if (fr) atomicMin(&s_pE, __ffs(fr) - 1);
            return 15;
        }
        if (!fr) return 15;
        const int32_t c = __ffs(fr) - 1;
        mask[u] |= (uint8_t)(1u << c);
        mask[v] |= (uint8_t)(1u << c);
        return c + 1;
    };
    for (int32_t r = 0;; ++r) {
        if (r > L + 1) return -1;  // every round colours or closes the first pending edge
        if ((s_round & (span - 1u)) == 0u && s_round != 0u) {  // reservation keys wrap
            for (int32_t i = tid; i < n; i += kT) res[i] = 0xFFFFFFFFu;
            __syncthreads();
        }
        const uint32_t base = round_base(s_round, span);
        bool pend = false;
#pragma unroll
        for (int k = 0; k < kHeld; ++k) {
            if (!((pm >> k) & 1u)) continue;
            if (reserve(tid + k * kT, he[k], (am >> k) & 1u, base)) {
                pend = true;
            } else {
                pm &= ~(1u << k);
                cols |= 15u << (4 * k);
            }
        }
        for (int32_t p = tail0 + tid; p < L; p += kT) {
            const uint8_t es = estate[p];
            if (!(es & kAlive) || (es >> 4)) continue;
            if (reserve(p, E[p], (es & kAppl) != 0, base)) pend = true;
            else estate[p] = es | 0xF0;
        }
        if (s_pt && tid == 0) s_pt[kPtCtlColourIters] += 1;
        if (!__syncthreads_or(pend)) break;
#pragma unroll
        for (int k = 0; k < kHeld; ++k) {
            if (!((pm >> k) & 1u)) continue;
            const int32_t nib = settle(tid + k * kT, he[k], (am >> k) & 1u, base);
            if (nib >= 0) {
                pm &= ~(1u << k);
                cols |= (uint32_t)nib << (4 * k);
            }
        }
        for (int32_t p = tail0 + tid; p < L; p += kT) {
            const uint8_t es = estate[p];
            if (!(es & kAlive) || (es >> 4)) continue;
            const int32_t nib = settle(p, E[p], (es & kAppl) != 0, base);
            if (nib >= 0) estate[p] = es | (uint8_t)(nib << 4);
        }
        if (tid == 0) s_round = s_round + 1u;
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kHeld; ++k) {  // outcomes back to the edge states (the same thread reads them next)
        const uint32_t nib = (cols >> (4 * k)) & 15u;
        if (nib) estate[tid + k * kT] |= (uint8_t)(nib << 4);
    }
    const long long t_tail = clock64();
    for (int32_t p = tid; p < L; p += kT) {
        const int32_t nib = estate[p] >> 4;
        if (nib < 1 || nib > kColourCap) continue;
        atomicAdd(&s_hist[nib - 1], 1);
        const int32_t t = slot_s ? (int32_t)slot_s[p] : w.ctl_slot[p];
        const unsigned long long key = w.sl_rkey[t];
        if (key && key_gain(key) > 0) atomicMin(&s_pR, nib);  // born in round colour + 1 = nib
    }
    __syncthreads();
    if (tid == 0) {
        int32_t F = min(s_pE, s_pR);
        if (max_sweeps > 0) F = min(F, max_sweeps - sweeps);
        F = max(F, 0);
        // a round with live edges accepts at least one (and an edge of colour c
        // has neighbours of every colour below c): an empty round means that
        // no edge is left, and the run ends before it
        while (F > 0 && s_hist[F - 1] == 0) --F;
        s_pF = F;
    }
    __syncthreads();
    const int32_t F = s_pF;
    int32_t died = 0;
    for (int32_t p = tid; p < L; p += kT) {
        uint8_t es = estate[p];
        const int32_t nib = es >> 4;
        if (!nib) continue;
        es &= 0x0F;
        if (nib <= F) {  // accepted in round nib - 1 < F: re-evaluated
            const int32_t t = slot_s ? (int32_t)slot_s[p] : w.ctl_slot[p];
            const unsigned long long key = w.sl_rkey[t];
            const int32_t gain = key ? key_gain(key) : 0;
            const int32_t target = key ? key_index(key) : -1;
            if (t < n) { w.ag_gain[t] = gain; w.ag_job[t] = target; }
            else { w.jb_gain[t - n] = gain; w.jb_agent[t - n] = target; }
            if (gain > 0) {
                E[p] = C::make(w.sl_ru[t], w.sl_rv[t]);
                es = kAlive | kAppl | kFreshBit;
            } else {
                es = 0;
                ++died;
            }
        }
        estate[p] = es;
    }
    if (died) atomicSub(&s_live, died);
    for (int32_t i = tid; i < n; i += kT) mask[i] = 0;  // claim stamps start clean
    __syncthreads();
    if (s_pt && tid == 0) s_pt[kPtCtlColourTail] += (unsigned long long)(clock64() - t_tail);
    return F;
}

// Switching loop (see the file comment).
// span: reservation-key period (power of two <= kRoundSpanMax); stamp_wrap:
// claim-stamp period (<= 255).  Both are shortened only by a test knob.
// list_cap: entries of the accepted list held in shared memory.
// colour_pass: runs of quiet sweeps go through colouring passes (only
// while the edges are in shared memory); 0 turns them off.
template <typename EdgeT, int kT = kCtlThreads, bool kEdgesToShared = true>
__device__ __forceinline__ void controller_body(const Workspace& w, int32_t smem_mode, const CtlScratch& g,
                                                uint32_t span, uint32_t stamp_wrap, int32_t list_cap,
                                                int32_t compact_min, int32_t colour_pass) {
    using C = Codec<EdgeT>;
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int32_t warp_sums[33];
    __shared__ int32_t s_L, s_live, s_stop, s_acc, s_app, s_y, s_sweeps, s_event;
    __shared__ int32_t s_max_sweeps, s_trace_cap;
    __shared__ int32_t s_pass_ok, s_pE, s_pR, s_pF, s_hist[kColourCap];
    __shared__ uint32_t s_round;
    __shared__ uint32_t s_stamp;
    __shared__ unsigned long long s_gain, s_deadline;
    __shared__ long long s_f;

    const int32_t n = w.n;
    const int tid = threadIdx.x;
    uint32_t* res = g.res;
    uint8_t* claimed = g.claimed;
    uint8_t* estate = g.estate;
    EdgeT* E = static_cast<EdgeT*>(g.edges);
    uint16_t* lists_s = nullptr;
    uint16_t* slot_s = nullptr;  // slot of each edge position (shared-memory modes)
    unsigned char* rec = nullptr;  // re-evaluation records (shared-memory modes)
    if (smem_mode >= 1) {
        size_t off = 0;
        rec = smem_raw;
        off += kRecBytes;
        res = reinterpret_cast<uint32_t*>(smem_raw + off);
        off += 4 * (size_t)n;
        if (smem_mode == 2) {
            E = reinterpret_cast<EdgeT*>(smem_raw + off);
            off += sizeof(EdgeT) * 2 * (size_t)n;
        }
        lists_s = reinterpret_cast<uint16_t*>(smem_raw + off);
        off += 2 * (size_t)list_cap;
        slot_s = reinterpret_cast<uint16_t*>(smem_raw + off);
        off += 2 * 2 * (size_t)n;
        claimed = smem_raw + off;
        off += (size_t)n;
        estate = smem_raw + off;
    }
    // Mode 1 keeps the edge array in global memory, but a list of at most
    // edges_s_cap() (about n / 2) positions fits in the upper half of slot_s
    // (positions below n use only its lower half): a launch whose list is
    // that short, or is compacted to that length, moves its edges there.
    // kEdgesToShared = false (the batched controller, which otherwise spills
    // more registers, and the single-CTA loop, which runs in mode 2 only)
    // leaves them in global memory.
    const bool es_mode = kEdgesToShared && smem_mode == 1 && sizeof(EdgeT) == 4;
    auto edges_s = [&]() -> EdgeT* {
        return reinterpret_cast<EdgeT*>((reinterpret_cast<uintptr_t>(slot_s + n) + 3u) & ~static_cast<uintptr_t>(3u));
    };
    auto edges_s_cap = [&]() -> int32_t {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(edges_s());
        const uintptr_t hi = reinterpret_cast<uintptr_t>(slot_s + 2 * (size_t)n);
        return hi > lo ? (int32_t)((hi - lo) / sizeof(EdgeT)) : 0;
    };
    const int32_t cap = lists_s ? list_cap : 0;
    TwoTier accl{lists_s, cap, g.acc_g};
    unsigned long long* pt = (tid == 0) ? w.phase_ns : nullptr;
    long long tp = clock64();
    // diagnostics (DGS_PHASE_TIMERS=1): thread 0 sums into shared memory and
    // adds the sums to global memory once per launch, so that the counters
    // add no global round trips to the loops they time
    __shared__ unsigned long long s_pt[kPtCount];
    if (pt)
        for (int k = 0; k < kPtCount; ++k) s_pt[k] = 0ull;
#define DGS_PT(slot, v) \
    if (pt) s_pt[slot] += (unsigned long long)(v);
#define DGS_CT(slot)                     \
    if (pt) {                            \
        const long long now = clock64(); \
        s_pt[slot] += (unsigned long long)(now - tp); \
        tp = now;                        \
    }

    // ---------------------------------------------------------------- entry
    // The slot refresh and the per-slot edge data were prepared by the grid
    // (prepare_edges_kernel); here the edges are listed in priority order.
    {
        for (int32_t i = tid; i < n; i += kT) {
            res[i] = 0xFFFFFFFFu;
            claimed[i] = 0;
        }
        if (tid == 0) {
            st->need_update = 0;
            st->y_count = 0;
            s_sweeps = st->sweeps;
            s_max_sweeps = st->max_sweeps;
            s_deadline = st->deadline_ns;
            s_trace_cap = st->trace_capacity;
            s_f = st->f;
            s_round = 0;
            s_stamp = 0;
            s_pass_ok = 0;  // a colouring pass follows a quiet sweep
        }
        // Warp wp lists the slots of its own range [lo, hi) (ranges are
        // multiples of 32 long and ascend with wp): it sums the edge counts
        // of its 32-slot chunks (written by the grid beside the edge words),
        // the 32 warp counts are scanned once, and it writes the edges of
        // its chunks that have any at its offset, so positions follow slot
        // order (the priority order).
        constexpr int kWarps = kT / 32;
        const int32_t lane = tid & 31, wp = tid >> 5;
        const int32_t per = (2 * n + 32 * kWarps - 1) / (32 * kWarps) * 32;
        const int32_t lo = min(2 * n, wp * per), hi = min(2 * n, lo + per);
        const int32_t c_lo = lo >> 5, c_hi = lo < hi ? (hi + 31) >> 5 : c_lo;  // lo is a multiple of 32
        int32_t cnt = 0;
        for (int32_t c = c_lo + lane; c < c_hi; c += 32) cnt += w.sl_chunk[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (lane == 0) warp_sums[wp] = cnt;
        __syncthreads();
        if (wp == 0) {
            const int32_t v = lane < kWarps ? warp_sums[lane] : 0;
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
        if (es_mode && warp_sums[32] <= edges_s_cap()) E = edges_s();  // the whole list fits in shared memory
        int32_t pos0 = warp_sums[wp];
        const uint32_t below = (1u << lane) - 1u;
        for (int32_t cb = c_lo; cb < c_hi; cb += 32) {
            uint32_t nz = __ballot_sync(0xffffffffu, cb + lane < c_hi && w.sl_chunk[cb + lane] > 0);
            while (nz) {  // four chunks with edges at a time, their loads in flight together
                int32_t ck[4];
                unsigned long long ew[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    ck[k] = nz ? cb + __ffs(nz) - 1 : -1;
                    nz &= nz - 1u;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int32_t t = ck[k] * 32 + lane;
                    ew[k] = (ck[k] >= 0 && t < hi) ? w.sl_edge[t] : 0ull;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int32_t t = ck[k] * 32 + lane;
                    const bool has = ew[k] != 0ull;
                    const uint32_t m = __ballot_sync(0xffffffffu, has);
                    if (has) {
                        const int32_t pos = pos0 + __popc(m & below);
                        w.ctl_slot[pos] = t;
                        if (slot_s) slot_s[pos] = (uint16_t)t;
                        E[pos] = C::make(edge_u(ew[k]), edge_v(ew[k]));
                        estate[pos] = kAlive | ((ew[k] & kApplies) ? kAppl : 0);
                    }
                    pos0 += __popc(m);
                }
            }
        }
        if (tid == 0) { s_L = warp_sums[32]; s_live = warp_sums[32]; }
        __syncthreads();
    }
    DGS_CT(kPtCtlEntry)

    // ------------------------------------------------------------- sweeps
    // Quiet sweeps turn at least one stale slot into a fresh one each, so one
    // launch runs at most 2n + 1 of them; more means an internal error.
    int32_t L = s_L;
    for (int32_t quiet = 0;; ++quiet) {
        if (tid == 0) {
            // loop condition of Algorithm 3 (some slot has delta > 0), sweep
            // cap and deadline; decided by one thread so that all agree
            int32_t stop = 0;
            if (s_live == 0) {
                st->status = kDone;
                stop = 1;
            } else if ((s_max_sweeps > 0 && s_sweeps >= s_max_sweeps) ||
                       (s_deadline != 0 && globaltimer_ns() > s_deadline)) {
                st->status = kTimeout;
                stop = 1;
            } else if (quiet > 2 * n + 1) {
                st->error = kErrInternal;
                st->status = kError;
                stop = 1;
            }
            s_stop = stop;
            s_acc = 0; s_app = 0; s_y = 0; s_gain = 0ull; s_event = 0;
            s_stamp = s_stamp + 1u;
        }
        __syncthreads();
        DGS_CT(kPtCtlTop)
        if (s_stop) break;
        DGS_PT(kPtCtlSweeps, 1)
        DGS_PT(kPtCtlLiveSum, s_live)
        DGS_PT(kPtCtlListSum, L)
        // An edge that dies in a quiet sweep never lives again in this launch.
        // Once fewer than half of the L listed positions are live, compact the
        // list in place, keeping the priority order (positions are
        // priorities, and deterministic reservations depend only on their
        // order), so that later sweeps scan live edges only; the reservation
        // keys restart with the new positions.
        if (s_live * 2 < L && L >= compact_min) {
            // (mode 1: into shared memory when the live edges fit there)
            const int32_t es_cap = es_mode ? edges_s_cap() : 0;
            const bool to_s = es_mode && E != edges_s();  // edges still in global memory
            EdgeT* const Ed = (to_s && s_live <= es_cap) ? edges_s() : E;
            const bool bounded = es_mode && Ed == edges_s();
            int32_t base = 0;
            for (int32_t c0 = 0; c0 < L; c0 += kT) {
                const int32_t p = c0 + tid;
                const uint8_t es = p < L ? estate[p] : (uint8_t)0;
                const bool alive = (es & kAlive) != 0;
                const EdgeT e = alive ? E[p] : (EdgeT)0;
                const int32_t slot = alive ? w.ctl_slot[p] : 0;
                int32_t total;
                const int32_t pos = base + block_scan<kT>(alive ? 1 : 0, warp_sums, &total);  // every read is done
                if (alive) {
                    if (!bounded || pos < es_cap) Ed[pos] = e;
                    estate[pos] = es;
                    w.ctl_slot[pos] = slot;
                    if (slot_s) slot_s[pos] = (uint16_t)slot;
                }
                base += total;
            }
            for (int32_t i = tid; i < n; i += kT) res[i] = 0xFFFFFFFFu;
            __syncthreads();
            if (tid == 0) {
                s_L = base;
                s_round = 0u;
                if (bounded && base > es_cap) {  // the live count disagreed with the list
                    st->error = kErrInternal;
                    st->status = kError;
                    s_stop = 1;
                }
            }
            __syncthreads();
            if (s_stop) break;
            L = s_L;
            E = Ed;
        }
        if (s_stamp >= stamp_wrap) {  // claim stamps wrap: clear them once
            for (int32_t i = tid; i < n; i += kT) claimed[i] = 0;
            __syncthreads();
            if (tid == 0) s_stamp = 1;
            __syncthreads();
        }
        if ((s_round & (span - 1u)) == 0u && s_round != 0u) {  // reservation keys wrap
            for (int32_t i = tid; i < n; i += kT) res[i] = 0xFFFFFFFFu;
            __syncthreads();
        }
        const uint8_t stamp = (uint8_t)s_stamp;
        // Colouring pass (after a quiet sweep; see colour_pass_rounds).  It
        // runs F >= 1 sweeps at once, or none when an applicable edge is
        // accepted in this very sweep; then this sweep goes on as usual.
        // (modes 1 and 2 hold n <= 32767, so only 32-bit edges take this path)
        // (short lists: a pass costs more than the sweeps it saves)
        if (sizeof(EdgeT) == 4 && colour_pass && (smem_mode == 2 || (es_mode && E == edges_s())) && s_pass_ok &&
            L > kColourMinList) {
            const int32_t F = colour_pass_rounds<EdgeT, kT>(w, E, estate, slot_s, res, claimed, L, span, s_round, s_pE,
                                                        s_pR, s_pF, s_hist, s_max_sweeps, s_sweeps, s_live,
                                                        pt ? s_pt : nullptr);
            if (F < 0) {  // internal error
                if (tid == 0) {
                    st->error = kErrInternal;
                    st->status = kError;
                }
                break;
            }
            if (tid == 0) {
                for (int32_t k = 0; k < F; ++k) {
                    const int32_t sw = s_sweeps + k;
                    if (sw < s_trace_cap) {
                        if (st->trace_accepted) st->trace_accepted[sw] = s_hist[k];
                        if (st->trace_applied) st->trace_applied[sw] = 0;
                        if (st->trace_objective) st->trace_objective[sw] = s_f;
                    }
                }
                s_sweeps = s_sweeps + F;
                DGS_PT(kPtCtlColourPasses, 1)
                DGS_PT(kPtCtlColourRounds, F)
                // another pass may follow at once only if this one met no
                // bound inside its window
                s_pass_ok = (F == kColourCap && s_pE >= kColourCap && s_pR >= kColourCap) ? 1 : 0;
            }
            __syncthreads();
            DGS_CT(kPtCtlColour)
            if (F > 0) continue;
        }
        // CC (Algorithm 4): the accepted set is the greedy one in priority
        // order (a slot is accepted when neither agent of its exchange was
        // claimed by an earlier accepted slot).  The list is taken in chunks
        // of one edge per thread, in order: an edge touching an agent claimed
        // by an earlier chunk is rejected at once; the chunk's other edges
        // are decided among themselves by deterministic reservations (each
        // round, the remaining candidates reserve both agents with a key that
        // orders them by position; an edge holding both reservations is
        // accepted and claims its agents; an edge touching a newly claimed
        // agent is rejected; the first remaining candidate always wins, so
        // every round accepts at least one edge).  Claims of a chunk reach
        // the next through a barrier, so the result is the greedy one.
        {
            int32_t ev = 0;
            // edges per thread and chunk (a chunk is kPer * kT
            // positions); four per thread crossed fewer barriers but was
            // slower (uniform n = 10000: 22.2 ms against 18.8 ms), so one
            constexpr int kPer = 1;
            for (int32_t c0 = 0; c0 < L; c0 += kPer * kT) {
                int32_t p[kPer], u[kPer], v[kPer];
                uint8_t es[kPer];
                bool cand[kPer];
                bool any = false;
#pragma unroll
                for (int k = 0; k < kPer; ++k) {
                    p[k] = c0 + k * kT + tid;
                    es[k] = p[k] < L ? estate[p[k]] : (uint8_t)0;
                    u[k] = 0;
                    v[k] = 0;
                    cand[k] = false;
                    if (es[k] & kAlive) {
                        const EdgeT e = E[p[k]];
                        u[k] = C::u(e);
                        v[k] = C::v(e);
                        cand[k] = claimed[u[k]] != stamp && claimed[v[k]] != stamp;
                    }
                    any |= cand[k];
                }
                for (int32_t r = 0; __syncthreads_or(any); ++r) {
                    if (r > kPer * kT) {  // every round accepts the first candidate
                        if (tid == 0) {
                            st->error = kErrInternal;
                            st->status = kError;
                            s_stop = 1;
                        }
#pragma unroll
                        for (int k = 0; k < kPer; ++k) cand[k] = false;
                        any = false;
                        continue;
                    }
                    if ((s_round & (span - 1u)) == 0u && s_round != 0u) {  // reservation keys wrap
                        for (int32_t i = tid; i < n; i += kT) res[i] = 0xFFFFFFFFu;
                        __syncthreads();
                    }
                    const uint32_t base = round_base(s_round, span);
#pragma unroll
                    for (int k = 0; k < kPer; ++k) {
                        if (!cand[k]) continue;
                        // (lanes of a warp that reserve the same agent were
                        // first made to agree on their smallest key with
                        // __match_any_sync / __reduce_min_sync: 3.7 times
                        // slower on uniform n = 10000, so every candidate
                        // issues its own atomics)
                        const uint32_t key = base | (uint32_t)p[k];
                        if (key < res[u[k]]) atomicMin(&res[u[k]], key);
                        if (key < res[v[k]]) atomicMin(&res[v[k]], key);
                    }
                    __syncthreads();
#pragma unroll
                    for (int k = 0; k < kPer; ++k) {
                        const uint32_t key = base | (uint32_t)p[k];
                        if (cand[k] && res[u[k]] == key && res[v[k]] == key) {
                            claimed[u[k]] = stamp;
                            claimed[v[k]] = stamp;
                            const int32_t idx = atomicAdd(&s_acc, 1);
                            accl.put(idx, p[k]);
                            if (slot_s) fetch_record(rec, idx, w, slot_s[p[k]]);  // its slot's re-evaluation
                            ev |= (es[k] & kAppl) ? 1 : 0;
                            cand[k] = false;
                        }
                    }
                    __syncthreads();  // this round's claims are visible
                    any = false;
#pragma unroll
                    for (int k = 0; k < kPer; ++k) {
                        if (cand[k] && (claimed[u[k]] == stamp || claimed[v[k]] == stamp)) cand[k] = false;  // rejected
                        any |= cand[k];
                    }
                    if (tid == 0) s_round = s_round + 1u;
                }
            }
            if (ev) s_event = 1;
            if (rec) asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
        }
        DGS_CT(kPtCtlPass1)
        if (s_stop) break;  // an internal error of the conflict check
        const int32_t nacc = s_acc;
        if (s_event) {
            // parallel switch: accepted exchanges are agent-disjoint; those
            // that raise f under the current sigma commit
            int32_t my_app = 0;
            long long my_gain = 0;
            for (int32_t q = tid; q < nacc; q += kT) {
                const int32_t p = accl.get(q);
                estate[p] |= kAccBit;
                if (!(estate[p] & kAppl)) continue;
                const EdgeT e = E[p];
                const int32_t u = C::u(e), v = C::v(e);
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
                const int32_t qy = atomicAdd(&s_y, 2);
                w.y_list[qy] = ju;
                w.y_list[qy + 1] = jv;
                w.in_y[ju] = 1;
                w.in_y[jv] = 1;
                w.moved[u] = 1;
                w.moved[v] = 1;
            }
            if (my_app) {
                atomicAdd(&s_app, my_app);
                atomicAdd(&s_gain, (unsigned long long)my_gain);
            }
            if (((reinterpret_cast<uintptr_t>(w.in_ca) | reinterpret_cast<uintptr_t>(w.in_cj)) & 15) == 0) {
                // both arrays hold round_up(n, 128) bytes: clear them in 16-byte words
                const int32_t n16 = (n + 15) / 16;
                for (int32_t i = tid; i < n16; i += kT) {
                    reinterpret_cast<uint4*>(w.in_ca)[i] = make_uint4(0, 0, 0, 0);
                    reinterpret_cast<uint4*>(w.in_cj)[i] = make_uint4(0, 0, 0, 0);
                }
            } else {
                for (int32_t i = tid; i < n; i += kT) {
                    w.in_ca[i] = 0;
                    w.in_cj[i] = 0;
                }
            }
            __syncthreads();
            // record C: every live slot that was not accepted keeps its
            // candidate (reading R4)
            for (int32_t p = tid; p < L; p += kT) {
                const uint8_t es = estate[p];
                if (!(es & kAlive) || (es & kAccBit)) continue;
                const int32_t t = slot_s ? (int32_t)slot_s[p] : w.ctl_slot[p];
                if (t < n) w.in_ca[t] = 1;
                else w.in_cj[t - n] = 1;
            }
            if (tid == 0) {
                const int32_t sw = s_sweeps;
                s_f += (long long)s_gain;
                st->swaps += s_app;
                if (sw < s_trace_cap) {
                    if (st->trace_accepted) st->trace_accepted[sw] = nacc;
                    if (st->trace_applied) st->trace_applied[sw] = s_app;
                    if (st->trace_objective) st->trace_objective[sw] = s_f;
                }
                s_sweeps = sw + 1;
                st->events += 1;
                st->y_count = s_y;
                st->rescan_count = 0;
                st->need_update = 1;
                st->phase = kPhaseRefreshAll;
            }
            DGS_CT(kPtCtlEvent)
            break;
        }
        // quiet sweep: sigma unchanged, so the keys are current.  Accepted
        // slots are re-evaluated (their precomputed outcome); the others stay
        // in C with their candidates for the next sweep.
        int32_t died = 0;
        for (int32_t q = tid; q < nacc; q += kT) {
            const int32_t p = accl.get(q);
            const int32_t t = slot_s ? (int32_t)slot_s[p] : w.ctl_slot[p];
            const bool held = rec != nullptr && q < kRecCap;
            const unsigned long long key =
                held ? *reinterpret_cast<const unsigned long long*>(rec + 16 * q) : w.sl_rkey[t];
            const int32_t gain = key ? key_gain(key) : 0;
            const int32_t target = key ? key_index(key) : -1;
            if (t < n) { w.ag_gain[t] = gain; w.ag_job[t] = target; }
            else { w.jb_gain[t - n] = gain; w.jb_agent[t - n] = target; }
            if (gain > 0) {
                const int32_t ru = held ? *reinterpret_cast<const int32_t*>(rec + 16 * q + 8) : w.sl_ru[t];
                const int32_t rv = held ? *reinterpret_cast<const int32_t*>(rec + 16 * q + 12) : w.sl_rv[t];
                E[p] = C::make(ru, rv);
                estate[p] = kAlive | kAppl | kFreshBit;
            } else {
                estate[p] = 0;
                ++died;
            }
        }
        if (died) atomicSub(&s_live, died);
        if (tid == 0) s_pass_ok = 1;
        DGS_PT(kPtCtlAccSum, nacc)
        if (tid == 0 && s_sweeps < s_trace_cap) {
            const int32_t sw = s_sweeps;
            if (st->trace_accepted) st->trace_accepted[sw] = nacc;
            if (st->trace_applied) st->trace_applied[sw] = 0;
            if (st->trace_objective) st->trace_objective[sw] = s_f;
        }
        if (tid == 0) s_sweeps = s_sweeps + 1;
        __syncthreads();
        DGS_CT(kPtCtlPost)
    }
#undef DGS_CT
#undef DGS_PT
    if (pt)
        for (int k = 0; k < kPtCount; ++k)
            if (s_pt[k]) atomicAdd(pt + k, s_pt[k]);
    if (tid == 0) {
        st->sweeps = s_sweeps;
        st->edge_count = s_live;
        st->f = s_f;
    }
    __syncthreads();  // shared memory is reused by the caller's next call
}

// cond != 0: the launch is the last kernel of an iteration of the device-
// side switching loop (a conditional WHILE graph node, five kernels per
// iteration); it sets the loop condition from the loop state.  The loop is
// bounded: more than 16 n + 4096 iterations is an internal error.
template <typename EdgeT>
__global__ void __launch_bounds__(kCtlThreads, 1) controller_kernel(Workspace w, int32_t smem_mode, CtlScratch g,
                                                                   uint32_t span, uint32_t stamp_wrap,
                                                                   int32_t list_cap, int32_t compact_min,
                                                                   int32_t colour_pass, unsigned long long cond) {
    controller_body<EdgeT>(w, smem_mode, g, span, stamp_wrap, list_cap, compact_min, colour_pass);
    if (cond != 0 && threadIdx.x == 0) {
        DeviceState* st = w.st;
        const int32_t it = ++st->loop_iterations;
        st->loop_launches += 5;
        if (st->status == kRunning && it > 16 * w.n + 4096) {
            st->error = kErrInternal;
            st->status = kError;
        }
        cudaGraphSetConditional(cond, st->status == kRunning ? 1u : 0u);
    }
}

// Before each controller launch: clear the marks of the last event, re-
// evaluate every slot not in C from the current row keys (reading R4), and
// for every slot with a candidate (delta > 0) record its edge (the agents of
// its exchange under the current sigma, and whether that exchange raises f
// now).  Also record each slot's re-evaluated candidate, which stays valid
// for as long as no exchange is committed.  One thread per slot.
__device__ __forceinline__ void prepare_edges_body(const Workspace& w, int32_t bid, int32_t nblk) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    const int32_t n = w.n;
    const int32_t stride = nblk * blockDim.x;
    const int32_t yc = st->y_count;
    for (int32_t t = bid * blockDim.x + threadIdx.x; t < yc; t += stride) {
        const int32_t j = w.y_list[t];
        w.in_y[j] = 0;
        w.moved[w.sigma[j]] = 0;
    }
    for (int32_t t = bid * blockDim.x + threadIdx.x; t < 2 * n; t += stride) {
        unsigned long long key;
        int32_t ru, rv, gain, target;
        bool in_c;
        if (t < n) {
            key = w.key_a[w.tau[t]];
            ru = t;
            rv = key ? w.sigma[key_index(key)] : t;
            in_c = w.in_ca[t] && !st->reeval_all;
            if (!in_c) {
                w.ag_gain[t] = key ? key_gain(key) : 0;
                w.ag_job[t] = key ? key_index(key) : -1;
            }
            gain = in_c ? w.ag_gain[t] : (key ? key_gain(key) : 0);
            target = in_c ? w.ag_job[t] : (key ? key_index(key) : -1);
        } else {
            const int32_t j = t - n;
            key = w.key_j[j];
            ru = w.sigma[j];
            rv = key ? key_index(key) : ru;
            in_c = w.in_cj[j] && !st->reeval_all;
            if (!in_c) {
                w.jb_gain[j] = key ? key_gain(key) : 0;
                w.jb_agent[j] = key ? key_index(key) : -1;
            }
            gain = in_c ? w.jb_gain[j] : (key ? key_gain(key) : 0);
            target = in_c ? w.jb_agent[j] : (key ? key_index(key) : -1);
        }
        w.sl_rkey[t] = key;
        w.sl_ru[t] = ru;
        w.sl_rv[t] = rv;
        unsigned long long e = 0ull;
        if (gain > 0) {
            const int32_t u = (t < n) ? t : w.sigma[t - n];
            const int32_t v = (t < n) ? w.sigma[target] : target;
            e = edge_word(u, v) | (exchange_gain(w, u, v) > 0 ? kApplies : 0ull);
        }
        w.sl_edge[t] = e;
        // the warp's 32 consecutive slots form one chunk: its edge count
        // lets the controller skip chunks without edges
        const uint32_t am = __activemask();
        const uint32_t bm = __ballot_sync(am, e != 0ull);
        if ((int)(threadIdx.x & 31) == __ffs(am) - 1) w.sl_chunk[t >> 5] = __popc(bm);
    }
}

__global__ void prepare_edges_kernel(Workspace w) { prepare_edges_body(w, blockIdx.x, gridDim.x); }

// Rows whose best is no longer known: rows of changed jobs, and rows whose
// best partner column changed holder.  Their keys are cleared and listed.
__device__ __forceinline__ void mark_rescan_body(const Workspace& w, int32_t bid, int32_t nblk) {
    DeviceState* st = w.st;
    if (st->status != kRunning || !st->need_update) return;
    for (int32_t j = bid * blockDim.x + threadIdx.x; j < w.n; j += nblk * blockDim.x) {
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

__global__ void mark_rescan_kernel(Workspace w) { mark_rescan_body(w, blockIdx.x, gridDim.x); }

// Row j of G recomputed in full by the CTA from row sigma(j) of a (read
// directly) and row j of at (`atrow`: global memory, or its copy staged in
// shared memory), gathered through sigma; its two keys are raised to the row's
// best.  With `scatter` and j a changed job, the row also pushes G[k][j] =
// G[j][k] into every other row k (the only entries of row k that changed),
// through the same atomic keys.  red_a / red_j: 16 entries each.  Ends with
// a CTA barrier (red_* and the staged row may be reused).
__device__ __forceinline__ void row_task_compute(const Workspace& w, int32_t j, const int32_t* atrow, bool scatter_ok,
                                                 unsigned long long* red_a, unsigned long long* red_j) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t n = w.n;
    const int32_t n4 = (n + 3) / 4;
    const int32_t sjj = w.sigma[j];
    const int32_t dj = w.diag[j];
    const bool scatter = scatter_ok && w.in_y[j];
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
    __syncthreads();
}

// Full re-evaluation of one listed row (row tasks): row j of at staged in
// shared memory by one TMA bulk copy when kStage.  Returns false (CTA-uniform)
// if the staged copy did not arrive within the wait limit.
template <bool kStage>
__device__ __forceinline__ bool row_task_row(const Workspace& w, int32_t j, int32_t* atrow_s, uint64_t* bar,
                                             uint32_t& phase, unsigned long long* red_a,
                                             unsigned long long* red_j) {
    const int32_t* atrow = w.at + (size_t)j * w.ldt;
    if (kStage) {
        if (threadIdx.x == 0) {
            const uint32_t bytes = 16u * (uint32_t)((w.n + 3) / 4);
            mbar_arrive_expect_tx(bar, bytes);
            bulk_g2s(atrow_s, atrow, bytes, bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) mbar_wait_bounded(bar, phase);  // the copy may still land: wait once more
            return false;
        }
        phase ^= 1u;
        atrow = atrow_s;
    }
    row_task_compute(w, j, atrow, true, red_a, red_j);
    return true;
}

template <bool kStage>
__device__ __forceinline__ void row_tasks_body(const Workspace& w, int32_t bid, int32_t nblk) {
    DeviceState* st = w.st;
    if (st->status != kRunning || !st->need_update) return;
    const int32_t count = st->rescan_count;
    const int32_t n = w.n;
    if (use_full_update(count, n, st->update_policy)) return;
    if (bid == 0 && threadIdx.x == 0) {
        st->row_updates += 1;
        st->rows_recomputed += count;
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int32_t* atrow_s = reinterpret_cast<int32_t*>(smem_raw);
    __shared__ unsigned long long red_a[16], red_j[16];
    __shared__ __align__(8) uint64_t bar;
    if (kStage && threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int32_t t = bid; t < count; t += nblk) {
        if (!row_task_row<kStage>(w, w.rescan_list[t], atrow_s, &bar, phase, red_a, red_j)) {
            if (threadIdx.x == 0) { st->error = kErrWaitTimeout; st->status = kError; }
            return;
        }
    }
}

template <bool kStage>
__global__ void __launch_bounds__(512) row_tasks_kernel(Workspace w) {
    row_tasks_body<kStage>(w, blockIdx.x, gridDim.x);
}

// Row j of G re-evaluated in full by one warp (the row task of the
// single-CTA switching loop): the same gains, tie-breaks and scatter into
// the other rows' keys as row_task_compute, with lane-strided columns (each
// lane sees its columns in ascending order, so its first maximum is its
// lowest column, and the packed keys combine across lanes).
__device__ __forceinline__ void row_task_warp(const Workspace& w, int32_t j) {
    const int lane = threadIdx.x & 31;
    const int32_t n = w.n;
    const int32_t sjj = w.sigma[j];
    const int32_t dj = w.diag[j];
    const bool scatter = w.in_y[j];
    const int32_t* arow = w.a + (size_t)sjj * w.lda;
    const int32_t* atrow = w.at + (size_t)j * w.ldt;
    int32_t bg = 0, bc = -1, bs = 0x7fffffff;
    for (int32_t k = lane; k < n; k += 32) {
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
    if (lane == 0 && ka) {
        atomicMax(&w.key_a[j], ka);
        atomicMax(&w.key_j[j], kj);
    }
}

// The whole switching loop of Algorithm 3 in one CTA, for small n (the
// per-launch cost of the five kernels of an iteration would dominate): per
// iteration the rows marked by the last committing sweep are re-evaluated
// (row tasks, one warp per row; identical keys to a full evaluation, see the
// update kernels), the slots refreshed, then the controller's sweeps; until
// the loop state stops running.  Bounded like the graph loop.
template <typename EdgeT, int kT>
__global__ void __launch_bounds__(kT, 1) small_loop_kernel(Workspace w, int32_t smem_mode, CtlScratch g,
                                                                   uint32_t span, uint32_t stamp_wrap,
                                                                   int32_t list_cap, int32_t compact_min,
                                                                   int32_t colour_pass) {
    __shared__ int32_t s_go, s_count;
    DeviceState* st = w.st;
    const int32_t n = w.n;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (;;) {
        mark_rescan_body(w, 0, 1);
        __syncthreads();
        if (tid == 0) {
            const bool rows = st->status == kRunning && st->need_update;
            s_count = rows ? st->rescan_count : 0;
            if (rows) {
                st->row_updates += 1;
                st->rows_recomputed += s_count;
            }
        }
        __syncthreads();
        for (int32_t t = warp; t < s_count; t += kT / 32) row_task_warp(w, w.rescan_list[t]);
        __syncthreads();
        prepare_edges_body(w, 0, 1);
        __syncthreads();
        controller_body<EdgeT, kT, false>(w, smem_mode, g, span, stamp_wrap, list_cap, compact_min, colour_pass);
        if (tid == 0) {
            const int32_t it = ++st->loop_iterations;
            if (st->status == kRunning && it > 16 * n + 4096) {
                st->error = kErrInternal;
                st->status = kError;
            }
            s_go = st->status == kRunning;
        }
        __syncthreads();
        if (!s_go) break;
    }
}

// The row-owner form of the full difference evaluation (Algorithm 2 for every
// slot, the A-transpose variant): CTA b owns rows j = b, b + nblk, ... of G and
// recomputes each from row sigma(j) of a and row j of the maintained at, with
// the next row of at already in flight to the second shared-memory stage
// (TMA bulk copies) while the current row is evaluated.  It touches 8n^2 bytes
// per evaluation (the tile-pair kernel reads each benefit once, 4n^2) but needs
// only one key update per row.  Keys are raised with atomicMax, so the result
// is the tile-pair kernel's: the same maxima with the same tie-breaks.
template <bool kStage>
__global__ void __launch_bounds__(512) row_owner_evaluation_kernel(Workspace w, int32_t conditional) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    if (conditional && !(st->need_update && use_full_update(st->rescan_count, w.n, st->update_policy))) return;
    if (conditional && blockIdx.x == 0 && threadIdx.x == 0) st->full_evals += 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ unsigned long long red_a[16], red_j[16];
    __shared__ __align__(8) uint64_t bar[2];
    const int32_t n = w.n;
    const uint32_t bytes = 16u * (uint32_t)((n + 3) / 4);
    int32_t* const stage0 = reinterpret_cast<int32_t*>(smem_raw);  // stage b at stage0 + b * ldt
    if (kStage && threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int32_t j = blockIdx.x;
    if (kStage && threadIdx.x == 0 && j < n) {
        mbar_arrive_expect_tx(&bar[0], bytes);
        bulk_g2s(stage0, w.at + (size_t)j * w.ldt, bytes, &bar[0]);
    }
    uint32_t phase = 0;  // bit b: parity of stage b's next completion
    for (int32_t it = 0; j < n; ++it, j += gridDim.x) {
        const int b = it & 1;
        const int32_t* atrow = w.at + (size_t)j * w.ldt;
        if (kStage) {
            // the other stage was last read by the previous row, which ended
            // with a CTA barrier: it is free for the next row's copy
            const int32_t jn = j + (int32_t)gridDim.x;
            if (threadIdx.x == 0 && jn < n) {
                mbar_arrive_expect_tx(&bar[b ^ 1], bytes);
                bulk_g2s(stage0 + (b ^ 1) * w.ldt, w.at + (size_t)jn * w.ldt, bytes, &bar[b ^ 1]);
            }
            const uint32_t pb = (phase >> b) & 1u;
            const bool ok = mbar_wait_bounded(&bar[b], pb);
            phase ^= 1u << b;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    st->error = kErrWaitTimeout;
                    st->status = kError;
                    // this row's copy and the next one may still be in flight
                    // into this CTA's shared memory: wait for them (bounded)
                    // before leaving
                    mbar_wait_bounded(&bar[b], pb);
                    if (jn < n) mbar_wait_bounded(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u);
                }
                return;
            }
            atrow = stage0 + b * w.ldt;
        }
        row_task_compute(w, j, atrow, false, red_a, red_j);
    }
}

// tau given (greedy result, identity or the caller's permutation): build
// sigma, D and f; validate a caller's permutation.
__device__ __forceinline__ void start_from_tau_body(const Workspace& w, const int32_t* user_tau, int32_t mode,
                                                    uint8_t* seen, int32_t bid, int32_t nblk) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    for (int32_t i = bid * blockDim.x + threadIdx.x; i < w.n; i += nblk * blockDim.x) {
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

__global__ void start_from_tau_kernel(Workspace w, const int32_t* user_tau, int32_t mode, uint8_t* seen) {
    start_from_tau_body(w, user_tau, mode, seen, blockIdx.x, gridDim.x);
}

__global__ void finish_kernel(Workspace w, int32_t* sigma_out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x)
        sigma_out[i] = w.tau[i];
}

// The dgs_status code of a finished loop state (the device side of
// map_device_status).
__device__ __forceinline__ int32_t device_status_code(const DeviceState* st) {
    if (st->status == kTimeout) return DGS_TIMEOUT;
    if (st->status != kError) return DGS_OK;
    if (st->error == kErrRange) return DGS_ERR_RANGE;
    if (st->error == kErrUserInit) return DGS_ERR_INVALID;
    return DGS_ERR_INTERNAL;
}

__global__ void finish_outputs_kernel(Workspace w, int32_t* sigma_out, int64_t* objective, int32_t* status) {
    const DeviceState* st = w.st;
    const bool failed = st->status == kError;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x)
        sigma_out[i] = failed ? -1 : w.tau[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (objective) *objective = st->f;
        if (status) *status = device_status_code(st);
    }
}

// ------------------------------------------------------- batched launches
// Initialise the fresh instances of the table: clear their small arrays, mark
// every agent and job free, re-pitch the caller's matrix where needed, and
// write the loop state (stage kStageNew).  Entries walk 16-byte chunks.
__global__ void init_batched_kernel(BatchTable t, int32_t update_policy) {
    const int32_t count = *t.count;
    for (int32_t g = blockIdx.x; g < count; g += gridDim.x) {
        const BatchEntry e = t.e[g];
        const Instance& in = t.inst[e.inst];
        if (!in.fresh) continue;
        const Workspace& w = in.w;
        const size_t nb = ((size_t)w.n + 127) / 128 * 128;
        const char* fa = reinterpret_cast<const char*>(w.free_a);
        const char* fj = reinterpret_cast<const char*>(w.free_j);
        const size_t chunks = in.zero_bytes / 16;
        const size_t stride = (size_t)e.nblk * blockDim.x;
        for (size_t q = (size_t)e.bid * blockDim.x + threadIdx.x; q < chunks; q += stride) {
            char* p = in.zero_begin + 16 * q;
            const bool ones = (p >= fa && p < fa + nb) || (p >= fj && p < fj + nb);
            const uint32_t v = ones ? 0x01010101u : 0u;
            *reinterpret_cast<uint4*>(p) = make_uint4(v, v, v, v);
        }
        // a caller's matrix that needs re-pitching (n % 4 != 0 or misaligned) is
        // copied into the workspace by pass 1, which reads it anyway
        if (e.bid == 0 && threadIdx.x == 0) {
            DeviceState h{};
            h.status = kRunning;
            h.phase = kPhaseRefreshAll;
            h.max_sweeps = in.max_sweeps;
            h.greedy_remaining = w.n;
            h.update_policy = update_policy;
            h.stage = kStageNew;
            h.init_mode = in.init_mode;
            h.reeval_all = in.reeval_all;
            if (in.deadline_us > 0) h.deadline_ns = globaltimer_ns() + (uint64_t)in.deadline_us * 1000ull;
            *w.st = h;
        }
    }
}

__global__ void start_batched_kernel(BatchTable t) {
    for_each_entry(t, kStageStart, [&](const Instance& in, int32_t bid, int32_t nblk) {
        start_from_tau_body(in.w, in.user_tau, in.w.st->init_mode, in.seen, bid, nblk);
    });
}

__global__ void mark_rescan_batched_kernel(BatchTable t) {
    for_each_entry(t, kStageSwitch, [&](const Instance& in, int32_t bid, int32_t nblk) {
        mark_rescan_body(in.w, bid, nblk);
    });
}

// The rows queued by the kScanSwitch scan (q1): one row task per item, the
// at row staged by TMA; one mbarrier for the CTA's whole sequence of rows.
__global__ void __launch_bounds__(512) row_tasks_batched_kernel(BatchQueues q) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int32_t* atrow_s = reinterpret_cast<int32_t*>(smem_raw);
    __shared__ unsigned long long red_a[16], red_j[16];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    bool dead = false;
    for_each_item(q.inst, q.q1, q.cap, [&](const Instance& in, int32_t t, int32_t) {
        if (dead) return;
        const Workspace& w = in.w;
        if (!row_task_row<true>(w, w.rescan_list[t], atrow_s, &bar, phase, red_a, red_j)) {
            if (threadIdx.x == 0) { w.st->error = kErrWaitTimeout; w.st->status = kError; }
            dead = true;  // the buffer may still be written: no further copies into it
        }
    });
}

// Per-slot work counts of one phase as exclusive prefix offsets (q0, q1; cap
// + 1 entries each), with the counters a single solve updates at the same
// point.  One CTA of 1024 threads.
//   kScanPass1:  q0 = pass-1 blocks of instances in kStageNew
//   kScanGreedyDA: q0 = agents of the instances in kStageGreedy (every q1
//                entry is 0: q1[0] is the deferred acceptance's shared counter)
//   kScanStart:  q0 = evaluation blocks of instances in kStageStart
//   kScanSwitch: q0 = evaluation blocks of the updates that re-evaluate every
//                row, q1 = rows of the updates that use row tasks
__global__ void __launch_bounds__(1024) scan_batched_kernel(BatchQueues q, int32_t phase, int32_t strip) {
    __shared__ int32_t warp_sums[33];
    int32_t carry0 = 0, carry1 = 0;
    for (int32_t c0 = 0; c0 < q.cap; c0 += 1024) {
        const int32_t k = c0 + (int32_t)threadIdx.x;
        int32_t x0 = 0, x1 = 0;
        if (k < q.cap) {
            const Instance& in = q.inst[k];
            DeviceState* st = in.w.st;
            const int32_t n = in.w.n;
            if (st != nullptr && n > 0) {
                const int32_t stage = st->stage;
                const bool running = st->status == kRunning;
                if (phase == kScanPass1) {
                    if (stage == kStageNew) x0 = batch_blocks_pass1(n);
                } else if (phase == kScanGreedyDA) {
                    if (stage == kStageGreedy && running && st->greedy_remaining > 0) x0 = n;
                } else if (phase == kScanStart) {
                    if (stage == kStageStart && running) x0 = batch_blocks_eval(n, strip);
                } else if (phase == kScanSwitch) {
                    if (stage == kStageSwitch && running && st->need_update) {
                        const int32_t count = st->rescan_count;
                        if (use_full_update(count, n, st->update_policy)) {
                            x0 = batch_blocks_eval(n, strip);
                            st->full_evals += 1;
                        } else {
                            x1 = count;
                            st->row_updates += 1;
                            st->rows_recomputed += count;
                        }
                    }
                }
            }
        }
        int32_t t0, t1;
        const int32_t p0 = block_scan(x0, warp_sums, &t0);
        const int32_t p1 = block_scan(x1, warp_sums, &t1);
        if (k < q.cap) {
            q.q0[k] = carry0 + p0;
            q.q1[k] = carry1 + p1;
        }
        carry0 += t0;
        carry1 += t1;
    }
    if (threadIdx.x == 0) {
        q.q0[q.cap] = carry0;
        q.q1[q.cap] = carry1;
    }
}

__global__ void prepare_edges_batched_kernel(BatchTable t) {
    for_each_entry(t, kStageSwitch, [&](const Instance& in, int32_t bid, int32_t nblk) {
        prepare_edges_body(in.w, bid, nblk);
    });
}

__global__ void __launch_bounds__(kCtlThreads, 1) controller_batched_kernel(BatchTable t, uint32_t span,
                                                                           uint32_t stamp_wrap, int32_t compact_min,
                                                                           int32_t colour_pass) {
    for_each_entry(t, kStageSwitch, [&](const Instance& in, int32_t, int32_t) {
        const CtlScratch c{in.ctl.res, in.ctl.claimed, in.ctl.estate, in.ctl.edges, in.ctl.acc};
        controller_body<uint32_t, kCtlThreads, false>(in.w, in.ctl_mode, c, span, stamp_wrap, in.ctl_cap, compact_min,
                                                      colour_pass);
    });
}

// The switching loop of an instance has ended: write its assignment.
__global__ void finish_batched_kernel(BatchTable t) {
    for_each_entry(t, kStageSwitch, [&](const Instance& in, int32_t bid, int32_t nblk) {
        const DeviceState* st = in.w.st;
        if (st->status != kDone && st->status != kTimeout) return;
        for (int32_t i = bid * blockDim.x + threadIdx.x; i < in.w.n; i += nblk * blockDim.x)
            in.sigma_out[i] = in.w.tau[i];
    });
}

// Stage transitions of the instances in from_stage (one thread each).
__global__ void advance_batched_kernel(BatchTable t, int32_t from_stage) {
    const int32_t count = *t.count;
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < count; g += gridDim.x * blockDim.x) {
        const Instance& in = t.inst[t.e[g].inst];
        DeviceState* st = in.w.st;
        if (st->stage != from_stage) continue;
        const bool running = st->status == kRunning;
        int32_t next = from_stage;
        if (from_stage == kStageNew) {
            next = !running ? kStageDone : (st->init_mode == 0 ? kStageGreedy : kStageStart);
        } else if (from_stage == kStageGreedy) {
            next = !running ? kStageDone : (st->greedy_remaining == 0 ? kStageStart : kStageGreedy);
        } else if (from_stage == kStageStart) {
            st->f_initial = st->f;
            next = running ? kStageSwitch : kStageDone;
        } else if (from_stage == kStageSwitch) {
            next = running ? kStageSwitch : kStageDone;
        }
        st->stage = next;
    }
}

}  // namespace

// Controller scratch placement.  Mode 2: reservations, 32-bit edges, list
// heads, claims and edge states in shared memory; mode 1: edges in global
// memory (the controller kernel of a single solve moves a list of up to
// about n / 2 positions into the spare half of the slot array); mode 0:
// everything in global memory.
constexpr size_t kCtlSmemLimit = 227 * 1024 - 1024;

static size_t ctl_fixed_bytes(int32_t n, int32_t mode) {
    // records + res (4n) + slot of each position (4n) + claimed (n) + estate (2n) [+ 32-bit edges (8n)]
    return kRecBytes + 11 * (size_t)n + (mode == 2 ? 8 * (size_t)n : 0);
}

int32_t controller_smem_mode(int32_t n) {
    int32_t mode = 0;
    if (n <= 32767 && ctl_fixed_bytes(n, 2) + 2 * 256 + 16 <= kCtlSmemLimit) mode = 2;
    else if (n <= 32767 && ctl_fixed_bytes(n, 1) + 2 * 256 + 16 <= kCtlSmemLimit) mode = 1;
    return min(mode, env_controller_mode_cap());
}

int32_t controller_list_cap(int32_t n, int32_t mode) {
    if (mode == 0) return 0;
    const size_t room = kCtlSmemLimit - ctl_fixed_bytes(n, mode) - 16;
    const size_t cap = room / 2;  // one 16-bit list
    return (int32_t)(cap < 2 * (size_t)n ? cap : 2 * (size_t)n);
}

size_t controller_smem_bytes(int32_t n) {
    const int32_t mode = controller_smem_mode(n);
    if (mode == 0) return 0;
    return ctl_fixed_bytes(n, mode) + 2 * (size_t)controller_list_cap(n, mode) + 16;
}

// DGS_SMALL_LOOP_N: the largest n whose switching loop runs in one CTA
// (small_loop_kernel); 0 turns it off (read on every call).  Only with the
// default update policy (the test knob that forces an update path keeps the
// grid kernels).
int32_t small_loop_max_n() {
    const char* e = std::getenv("DGS_SMALL_LOOP_N");
    return e ? std::atoi(e) : 768;  // measured: faster up to n = 512, slower from n = 1024
}

bool use_small_loop(const Workspace& w) {
    return w.n <= small_loop_max_n() && controller_smem_mode(w.n) == 2 && env_update_policy() == 0 &&
           w.row_owner_eval == 0;
}

template <int kT>
static cudaError_t launch_small_loop_t(const Workspace& w, const CtlGlobal& gs, cudaStream_t s, int slot) {
    const int32_t mode = controller_smem_mode(w.n);
    const size_t smem = controller_smem_bytes(w.n);
    const int32_t cap = controller_list_cap(w.n, mode);
    CtlScratch c{gs.res, gs.claimed, gs.estate, gs.edges, gs.acc};
    const void* fn = reinterpret_cast<const void*>(small_loop_kernel<uint32_t, kT>);
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_smem_limit(fn, slot, smem);
        if (e != cudaSuccess) return e;
    }
    const bool short_wrap = env_short_wraps() != 0;
    small_loop_kernel<uint32_t, kT><<<1, kT, smem, s>>>(w, mode, c, short_wrap ? 4u : kRoundSpanMax,
                                                         short_wrap ? 5u : 250u, cap, env_compact_min(),
                                                         env_colour_pass());
    return cudaGetLastError();
}

// DGS_SMALL_LOOP_THREADS (256, 512 or 1024; read on every launch): the CTA
// width of the single-CTA loop.  Measured at n = 256 (uniform [0, 1000), 52
// sweeps): 0.32 / 0.29 / 0.30 ms; peer-shaped: 0.150 / 0.144 / 0.143 ms.
int32_t small_loop_threads() {
    const char* e = std::getenv("DGS_SMALL_LOOP_THREADS");
    const int32_t x = e ? std::atoi(e) : 512;
    return (x == 256 || x == 1024) ? x : 512;
}

cudaError_t launch_small_loop(const Workspace& w, const CtlGlobal& gs, cudaStream_t s) {
    switch (small_loop_threads()) {
        case 1024: return launch_small_loop_t<1024>(w, gs, s, 14);
        case 512: return launch_small_loop_t<512>(w, gs, s, 15);
        default: return launch_small_loop_t<256>(w, gs, s, 8);
    }
}

cudaError_t launch_controller_impl(const Workspace& w, const CtlGlobal& gs, cudaStream_t s, unsigned long long handle) {
    const int32_t mode = controller_smem_mode(w.n);
    const size_t smem = controller_smem_bytes(w.n);
    const int32_t cap = controller_list_cap(w.n, mode);
    CtlScratch c{gs.res, gs.claimed, gs.estate, gs.edges, gs.acc};
    const bool narrow = w.n <= 65535;
    const void* fn = narrow ? reinterpret_cast<const void*>(controller_kernel<uint32_t>)
                            : reinterpret_cast<const void*>(controller_kernel<unsigned long long>);
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_smem_limit(fn, narrow ? 1 : 3, smem);
        if (e != cudaSuccess) return e;
    }
    const bool short_wrap = env_short_wraps() != 0;
    const uint32_t span = short_wrap ? 4u : kRoundSpanMax;
    const uint32_t stamp_wrap = short_wrap ? 5u : 250u;
    const int32_t cmin = env_compact_min();
    const int32_t cp = env_colour_pass();
    if (narrow)
        controller_kernel<uint32_t><<<1, kCtlThreads, smem, s>>>(w, mode, c, span, stamp_wrap, cap, cmin, cp, handle);
    else
        controller_kernel<unsigned long long><<<1, kCtlThreads, smem, s>>>(w, mode, c, span, stamp_wrap, cap, cmin,
                                                                          cp, handle);
    return cudaGetLastError();
}

cudaError_t launch_prepare_edges(const Workspace& w, cudaStream_t s) {
    int grid = (2 * w.n + 255) / 256;
    if (grid > dgs::device_sms() * 8) grid = dgs::device_sms() * 8;
    prepare_edges_kernel<<<grid, 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_mark_rescan(const Workspace& w, cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > dgs::device_sms() * 4) grid = dgs::device_sms() * 4;
    mark_rescan_kernel<<<grid, 256, 0, s>>>(w);
    return cudaGetLastError();
}

constexpr int32_t kRowStageMaxN = 54 * 1024;

cudaError_t launch_row_tasks(const Workspace& w, cudaStream_t s) {
    const int grid = dgs::device_sms() * 2;
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

// Two stages of one row of at each: up to 27 * 1024 columns (216 KB).
constexpr int32_t kRowOwnerStageMaxN = 27 * 1024;

cudaError_t launch_row_owner_evaluation(const Workspace& w, int32_t conditional, cudaStream_t s) {
    if (w.n <= kRowOwnerStageMaxN) {
        const size_t smem = 2 * 4 * (size_t)w.ldt;
        if (smem > 48 * 1024) {
            cudaError_t e =
                ensure_smem_limit(reinterpret_cast<const void*>(row_owner_evaluation_kernel<true>), 12, smem);
            if (e != cudaSuccess) return e;
        }
        const int per_sm = smem <= 110 * 1024 ? 2 : 1;
        row_owner_evaluation_kernel<true><<<dgs::device_sms() * per_sm, 512, smem, s>>>(w, conditional);
    } else {
        row_owner_evaluation_kernel<false><<<dgs::device_sms() * 2, 512, 0, s>>>(w, conditional);
    }
    return cudaGetLastError();
}

cudaError_t launch_start_from_tau(const Workspace& w, const int32_t* user_tau, int32_t mode, uint8_t* seen,
                                  cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > dgs::device_sms() * 4) grid = dgs::device_sms() * 4;
    start_from_tau_kernel<<<grid, 256, 0, s>>>(w, user_tau, mode, seen);
    return cudaGetLastError();
}

// ---------------------------------------------------- batched launchers
// rows: entries over the agents/slots of each instance (256 threads per
// block); one: one entry per instance.

cudaError_t launch_b_init(const BatchTable& rows, cudaStream_t s) {
    init_batched_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(rows, env_update_policy());
    return cudaGetLastError();
}

cudaError_t launch_b_start(const BatchTable& rows, cudaStream_t s) {
    start_batched_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(rows);
    return cudaGetLastError();
}

cudaError_t launch_b_mark_rescan(const BatchTable& rows, cudaStream_t s) {
    mark_rescan_batched_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(rows);
    return cudaGetLastError();
}

// The row tasks queued in q.q1; max_n bounds every queued instance's n.
cudaError_t launch_b_row_tasks(const BatchQueues& q, int32_t max_n, cudaStream_t s) {
    const size_t smem = 4 * (size_t)((max_n + 63) / 64 * 64);
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(row_tasks_batched_kernel), 6, smem);
        if (e != cudaSuccess) return e;
    }
    const int per_sm = (int)std::min<size_t>(4, (227 * 1024) / (smem + 1024));  // 512 threads, 2048 per SM
    row_tasks_batched_kernel<<<dgs::device_sms() * (per_sm < 1 ? 1 : per_sm), 512, smem, s>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_b_scan(const BatchQueues& q, int32_t phase, int32_t strip, cudaStream_t s) {
    scan_batched_kernel<<<1, 1024, 0, s>>>(q, phase, strip);
    return cudaGetLastError();
}

cudaError_t launch_b_prepare_edges(const BatchTable& rows, cudaStream_t s) {
    prepare_edges_batched_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(rows);
    return cudaGetLastError();
}

// Instances of a batched launch have n <= 32767 (16-bit edge positions and
// 32-bit edge words); each CTA lays out its shared memory for its own n.
cudaError_t launch_b_controller(const BatchTable& one, cudaStream_t s) {
    const size_t smem = kCtlSmemLimit;
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(controller_batched_kernel), 5, smem);
    if (e != cudaSuccess) return e;
    const bool short_wrap = env_short_wraps() != 0;
    controller_batched_kernel<<<dgs::device_sms(), kCtlThreads, smem, s>>>(one, short_wrap ? 4u : kRoundSpanMax,
                                                            short_wrap ? 5u : 250u, env_compact_min(),
                                                            env_colour_pass());
    return cudaGetLastError();
}

cudaError_t launch_b_finish(const BatchTable& rows, cudaStream_t s) {
    finish_batched_kernel<<<dgs::device_sms() * 8, 256, 0, s>>>(rows);
    return cudaGetLastError();
}

cudaError_t launch_b_advance(const BatchTable& one, int32_t from_stage, cudaStream_t s) {
    advance_batched_kernel<<<8, 256, 0, s>>>(one, from_stage);
    return cudaGetLastError();
}

cudaError_t launch_finish_outputs(const Workspace& w, int32_t* sigma_out, int64_t* objective, int32_t* status,
                                  cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > dgs::device_sms() * 4) grid = dgs::device_sms() * 4;
    finish_outputs_kernel<<<grid, 256, 0, s>>>(w, sigma_out, objective, status);
    return cudaGetLastError();
}

cudaError_t launch_finish(const Workspace& w, int32_t* sigma_out, cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > dgs::device_sms() * 4) grid = dgs::device_sms() * 4;
    finish_kernel<<<grid, 256, 0, s>>>(w, sigma_out);
    return cudaGetLastError();
}

}  // namespace dgs
