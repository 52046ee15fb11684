// k_evaluate.cu -- full difference evaluation (Algorithm 2 for every agent,
// JDE for every job: the first parallel block of Algorithm 3, Section 5).
//
// Notation: R[j][k] = a[sigma(j)][k] (a with rows permuted by sigma, read
// through sigma; never copied), D[j] = R[j][j].  Exchanging the holders of
// jobs j and k changes the objective by
//     G[j][k] = R[j][k] + R[k][j] - D[j] - D[k]          (G symmetric, G[j][j] = 0).
// ADE of agent sigma(j) and JDE of job j both maximise row j of G: the agent
// slot breaks ties by the lowest partner job k, the job slot by the lowest
// partner agent sigma(k).  The kernel produces, for every row j, the two
// packed keys key_a[j] = (gain, ~k) and key_j[j] = (gain, ~sigma(k)) of the
// best strictly positive gain (0 when none).
//
// Design (HBM-bound, no tensor cores): G is symmetric, so one 64x64 block
// G[J][K] (J <= K) serves the rows of J (over columns K) and the rows of K
// (over columns J).  The block needs the tiles X = R[J,K] and Y = R[K,J]:
// 64 row segments of 256 B each, gathered through sigma.  All 512 threads
// stage them into shared memory with 16-byte cp.async copies in a 5-deep
// pipeline (one barrier per tile).  Every element of a is read exactly once
// per evaluation.  (One-dimensional TMA bulk copies of the same 256-byte
// segments were measured request-rate bound at about 1.5 TB/s on GB300, which
// is why the copies are issued by the threads.)  A CTA walks a strip of tiles
// with the same J, keeping the row-side maxima of its 64 rows in registers;
// column-side maxima of each tile are combined across the CTA in shared
// memory at the next barrier and committed with 64-bit atomicMax, which is
// order independent and therefore deterministic.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kT = 64;         // tile edge
constexpr int kYP = kT + 4;    // Y row pitch (ints): 16-B aligned and int4-conflict-free
// Pipeline depth: 5 stages of 34 KB (a sixth, which fits beside the column
// buffers of 8 or 16 rows per thread, measured no faster: the kernel is
// bound by instruction issue before it is by bytes in flight).
constexpr int stages_for(int) { return 5; }

// Thread geometry for kRows rows per thread: kThreads = 64 columns x
// (64 / kRows) row groups; each thread copies kCopies row segments of X and
// of Y per tile.
template <int kRows>
struct Geo {
    static constexpr int kThreads = kT * kT / kRows;
    static constexpr int kGroups = kThreads / kT;
    static constexpr int kCopies = 1024 / kThreads;
    static constexpr int kRowStep = kThreads / 16;
};

struct Stage {
    int32_t x[kT * kT];
    int32_t y[kT * kYP];
    int32_t sk[kT];  // sigma of the tile's columns
    int32_t dk[kT];  // D of the tile's columns
    int32_t sj[kT];  // sigma of the tile's rows (the row block J)
    int32_t dj[kT];  // D of the tile's rows
};

struct TileCursor {
    int32_t j;      // row block of the current tile
    int32_t k;      // column tile of the current tile
    int32_t kend;   // one past the last column tile of the current row run
    int32_t item;   // strided schedule: index of the current item
    int32_t lin;    // contiguous schedule: linear index of the current tile
    int32_t lend;   //   and one past the last tile of this block's range (< 2^31: nb <= 2048)
};

// Two schedules of the upper-triangle tiles (J <= K) over the nblk blocks of
// one instance.
//  strip > 0 (strided items): item (J, c) = tiles J + strip*c .. + strip - 1
//    of row block J, numbered J * chunks + c; block b walks items b, b +
//    nblk, ...; items past the last tile are empty and skipped.
//  strip == 0 (contiguous): the tiles in row-major order, split into nblk
//    equal contiguous ranges; block b walks range b, one row run per row
//    block it touches.
// Either way every tile is visited by exactly one block.
__device__ __forceinline__ bool cursor_strided(TileCursor& c, int32_t item, int32_t nb, int32_t strip,
                                               int32_t nblk) {
    const int32_t chunks = (nb + strip - 1) / strip;
    const int32_t total = nb * chunks;
    for (; item < total; item += nblk) {
        const int32_t j = item / chunks;
        const int32_t k0 = j + strip * (item - j * chunks);
        if (k0 < nb) {
            c.item = item;
            c.j = j;
            c.k = k0;
            c.kend = min(k0 + strip, nb);
            return true;
        }
    }
    c.item = item;
    return false;
}

// first tile of row block J in row-major upper-triangle order
__device__ __forceinline__ int32_t tri_offset(int32_t J, int32_t nb) { return J * nb - J * (J - 1) / 2; }

__device__ __forceinline__ bool cursor_first(TileCursor& c, int32_t nb, int32_t strip, int32_t bid, int32_t nblk) {
    if (strip > 0) return cursor_strided(c, bid, nb, strip, nblk);
    const int64_t total = tri_offset(nb, nb);
    c.lin = (int32_t)(total * bid / nblk);
    c.lend = (int32_t)(total * (bid + 1) / nblk);
    if (c.lin >= c.lend) return false;
    int32_t lo = 0, hi = nb;  // tri_offset(lo) <= lin < tri_offset(hi)
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (tri_offset(mid, nb) <= c.lin) lo = mid;
        else hi = mid;
    }
    c.j = lo;
    c.k = lo + (c.lin - tri_offset(lo, nb));
    c.kend = min(nb, c.k + (c.lend - c.lin));
    return true;
}

__device__ __forceinline__ bool cursor_next(TileCursor& c, int32_t nb, int32_t strip, int32_t nblk) {
    if (strip > 0) {
        if (++c.k < c.kend) return true;
        return cursor_strided(c, c.item + nblk, nb, strip, nblk);
    }
    if (++c.lin >= c.lend) return false;
    if (++c.k >= nb) {
        ++c.j;
        c.k = c.j;
        c.kend = min(nb, c.k + (c.lend - c.lin));
    }
    return true;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// sigma of the rows this thread copies for tile (J, K): X rows J0 + rq + c *
// kRowStep and Y rows K0 + rq + c * kRowStep (rq = threadIdx.x / 16).
template <int kRows>
struct CopyRows {
    int32_t x[Geo<kRows>::kCopies], y[Geo<kRows>::kCopies];
};

template <int kRows, bool kTma = false>
__device__ __forceinline__ CopyRows<kRows> copy_rows(const Workspace& w, int32_t J, int32_t K) {
    const int32_t rq = threadIdx.x >> 4;
    const int32_t K0 = K * kT, n = w.n;
    CopyRows<kRows> c;
#pragma unroll
    for (int q = 0; q < Geo<kRows>::kCopies; ++q) {
        const int32_t r = rq + q * Geo<kRows>::kRowStep;
        c.x[q] = -1;  // X rows come from the producer's per-run sources (or TMA)
        c.y[q] = (K0 + r < n) ? w.sigma[K0 + r] : -1;
    }
    return c;
}

template <int kRows>
__device__ __forceinline__ CopyRows<kRows> no_rows() {
    CopyRows<kRows> c;
#pragma unroll
    for (int q = 0; q < Geo<kRows>::kCopies; ++q) c.x[q] = c.y[q] = -1;
    return c;
}

// This thread's X source rows for row block J (the rows of a at sigma(J0 +
// r), at this thread's chunk; null past n).  They do not change along a row
// run, so the producer computes them once per run.
template <int kRows>
struct XRows {
    const int32_t* p[Geo<kRows>::kCopies];
};

template <int kRows>
__device__ __forceinline__ void x_sources(const Workspace& w, int32_t J, XRows<kRows>& xr) {
    const int32_t chunk = (threadIdx.x & 15) * 4;
    const int32_t rq = threadIdx.x >> 4;
#pragma unroll
    for (int q = 0; q < Geo<kRows>::kCopies; ++q) {
        const int32_t r = J * kT + rq + q * Geo<kRows>::kRowStep;
        xr.p[q] = r < w.n ? w.a + (size_t)w.sigma[r] * w.lda + chunk : nullptr;
    }
}

// Issue this thread's 16-byte copies of tile (J, K) into stage: the X rows
// from xr (skipped when xr is null, as under the TMA path), the Y rows of
// sigma c.y, sigma and D of the tile's columns and rows.
template <int kRows>
__device__ __forceinline__ void issue_tile(const Workspace& w, Stage* stage, int32_t J, int32_t K,
                                           const CopyRows<kRows>& c, const XRows<kRows>* xr) {
    const int32_t chunk = (threadIdx.x & 15) * 4;  // first int of the 16-byte chunk
    const int32_t rq = threadIdx.x >> 4;
    const int32_t J0 = J * kT, K0 = K * kT;
    const bool in_x = chunk < w.lda - K0;  // X rows hold columns K0.. (row pitch lda)
    const bool in_y = chunk < w.lda - J0;  // Y rows hold columns J0..
#pragma unroll
    for (int q = 0; q < Geo<kRows>::kCopies; ++q) {
        const int32_t r = rq + q * Geo<kRows>::kRowStep;
        if (xr != nullptr && in_x && xr->p[q] != nullptr) cp_async16(stage->x + r * kT + chunk, xr->p[q] + K0);
        if (in_y && c.y[q] >= 0) cp_async16(stage->y + r * kYP + chunk, w.a + (size_t)c.y[q] * w.lda + J0 + chunk);
    }
    // sigma and D of the columns (arrays hold at least round_up(n, 64) entries)
    if (threadIdx.x < 16) cp_async16(stage->sk + chunk, w.sigma + K0 + chunk);
    else if (threadIdx.x < 32) cp_async16(stage->dk + chunk, w.diag + K0 + chunk);
    else if (threadIdx.x < 48) cp_async16(stage->sj + chunk, w.sigma + J0 + chunk);
    else if (threadIdx.x < 64) cp_async16(stage->dj + chunk, w.diag + J0 + chunk);
}

// TMA path: the X tile of (J, K) (rows sigma(J0 .. J0 + 63), columns K0 ..
// K0 + 63 of a) as 16 four-row gathers (cp.async.bulk.tensor tile::gather4,
// box 64 x 1 of the tensor map over a), issued by lanes 0..15 of warp 0 and
// completing on the stage's mbarrier (16 KB per tile).  xs: the four rows'
// sigma of this lane (rows past n read row 0; their pairs are never used).
__device__ __forceinline__ void gather_x(Stage* stage, const CUtensorMap* tm, int32_t K0, const int32_t (&xs)[4],
                                         uint64_t* bar) {
    const int lane = threadIdx.x;  // warp 0 only
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(kT * kT * sizeof(int32_t)));
    __syncwarp();
    if (lane < 16) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(stage->x + lane * 4 * kT)),
            "l"(reinterpret_cast<uint64_t>(tm)), "r"(K0), "r"(xs[0]), "r"(xs[1]), "r"(xs[2]), "r"(xs[3]),
            "r"(smem_u32(bar))
            : "memory");
    }
}

// This lane's four X rows of row block J (warp 0, lanes 0..15).
__device__ __forceinline__ void x_rows(const Workspace& w, int32_t J, int32_t (&xs)[4]) {
    const int32_t r0 = J * kT + 4 * (int32_t)(threadIdx.x & 15);
#pragma unroll
    for (int q = 0; q < 4; ++q) xs[q] = (r0 + q < w.n) ? w.sigma[r0 + q] : 0;
}

// Packed-key geometry for this n and value range; pw = 0 means "exact path".
struct Packing {
    int32_t pw;    // 2^s
    int32_t mask;  // 2^s - 1
};

__device__ __forceinline__ Packing packing_for(int32_t n, int32_t max_abs) {
    const int32_t s = 32 - __clz(max(n - 1, 1));
    const int64_t gmax = 4ll * (int64_t)max_abs + 1;
    Packing p{0, 0};
    if (s <= 24 && gmax < ((int64_t)1 << (30 - s))) {
        p.pw = 1 << s;
        p.mask = p.pw - 1;
    }
    return p;
}

__device__ __forceinline__ unsigned long long unpack_key(int32_t key, const Packing& pk) {
    if (key <= pk.mask) return 0ull;  // gain <= 0
    return pack_gain(key >> __popc(pk.mask), (uint32_t)(pk.mask - (key & pk.mask)));
}

// Per-thread state of its kRows rows across a strip (tiles with the same row
// block J).  Packed path (when |gain| * 2^s fits in int32, s = index bits):
// two int32 keys per row, (gain << s) + (mask - column) in g and (gain << s) +
// (mask - partner agent) in s, whose max picks the larger gain, then the lower
// index; ca / cj: mask - row and mask - sigma(row), the column-side tie
// offsets.  Exact path: best gain g, its lowest column c, lowest partner
// agent s among the columns reaching it; sj = sigma of the rows.
template <int kRows, bool kPacked>
struct Rows {
    int32_t g[kRows], s[kRows], d[kRows];
    int32_t c[kPacked ? 1 : kRows];
    int32_t ca[kPacked ? kRows : 1], cj[kPacked ? kRows : 1];
    int32_t sj[kPacked ? 1 : kRows];
};

template <int kRows, bool kPacked>
__device__ __forceinline__ void rows_start(Rows<kRows, kPacked>& rs, const Stage* stage, int32_t J0,
                                           const Packing& pk) {
    const int ty = threadIdx.x >> 6;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        rs.d[r] = stage->dj[ty * kRows + r];
        if (kPacked) {
            rs.g[r] = pk.mask;
            rs.s[r] = pk.mask;
            rs.ca[r] = pk.mask - (J0 + ty * kRows + r);
            rs.cj[r] = pk.mask - stage->sj[ty * kRows + r];
        } else {
            rs.g[r] = 0;
            rs.c[r] = -1;
            rs.s[r] = 0x7fffffff;
            rs.sj[r] = stage->sj[ty * kRows + r];
        }
    }
}

// One tile: thread (ty, tx) covers column k = K0 + tx and rows J0 + ty*kRows
// .. + kRows - 1.  Column-side partial keys go to the tile's column buffer cb
// (combined at the next barrier): packed 32-bit keys when kPacked (unpacked
// once per column by commit_columns), else 64-bit keys.
template <int kRows, bool kRagged, bool kPacked>
__device__ __forceinline__ void compute_tile(const Stage* stage, Rows<kRows, kPacked>& rs, int32_t J0, int32_t K0,
                                             int32_t n, const Packing& pk, void* cb) {
    constexpr int kGroups = Geo<kRows>::kGroups;
    const int tx = threadIdx.x & 63;
    const int ty = threadIdx.x >> 6;
    const int32_t k = K0 + tx;
    unsigned long long ka = 0ull, kj = 0ull;
    int32_t ca = pk.mask, cj = pk.mask;  // packed column-side keys ("none")
    if (!kRagged || k < n) {
        const int32_t sk = stage->sk[tx];
        const int32_t dk = stage->dk[tx];
        const int32_t* xrow = stage->x + (ty * kRows) * kT + tx;
        const int4* yrow = reinterpret_cast<const int4*>(stage->y + tx * kYP + ty * kRows);
        if (kPacked) {
            // With h = X + Y - D[jr] (so g = h - D[k]) every key is h * 2^s
            // plus a constant: the row-side constants fold -D[k] * 2^s in
            // once per tile, and the column side subtracts it once after its
            // maximum over the rows (a common shift commutes with max).  The
            // products and sums are formed modulo 2^32; every key compared is
            // exactly g * 2^s + offset, which fits in int32 by the packing
            // bound, and the column-side partial maxima exceed it by at most
            // D[k] * 2^s < 2^28.  The rows' column-side terms are reduced as a
            // tree (depth log2 kRows instead of a kRows-long chain).
            const uint32_t pw = (uint32_t)pk.pw;
            const uint32_t dks = (uint32_t)dk * pw;
            const uint32_t cka = (uint32_t)(pk.mask - k) - dks, ckj = (uint32_t)(pk.mask - sk) - dks;
            int32_t ta[kRows], tj[kRows];
#pragma unroll
            for (int q = 0; q < kRows / 4; ++q) {
                const int4 y4 = yrow[q];
                const int32_t yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = q * 4 + e;
                    if (kRagged && J0 + ty * kRows + r >= n) {
                        ta[r] = tj[r] = INT32_MIN;
                        continue;
                    }
                    const uint32_t hs = (uint32_t)(xrow[r * kT] + yv[e] - rs.d[r]) * pw;
                    rs.g[r] = max(rs.g[r], (int32_t)(hs + cka));  // row jr, lowest column
                    rs.s[r] = max(rs.s[r], (int32_t)(hs + ckj));  // row jr, lowest partner agent
                    ta[r] = (int32_t)(hs + (uint32_t)rs.ca[r]);   // row k, lowest column (+ D[k] 2^s)
                    tj[r] = (int32_t)(hs + (uint32_t)rs.cj[r]);   // row k, lowest partner agent (+ D[k] 2^s)
                }
            }
#pragma unroll
            for (int h = kRows / 2; h >= 1; h /= 2) {
#pragma unroll
                for (int r = 0; r < h; ++r) {
                    ta[r] = max(ta[r], ta[r + h]);
                    tj[r] = max(tj[r], tj[r + h]);
                }
            }
            if (!kRagged || ta[0] != INT32_MIN) {
                ca = max(ca, (int32_t)((uint32_t)ta[0] - dks));
                cj = max(cj, (int32_t)((uint32_t)tj[0] - dks));
            }
        } else {
            int32_t cg = 0, cc = -1, cs = 0x7fffffff;
#pragma unroll
            for (int q = 0; q < kRows / 4; ++q) {
                const int4 y4 = yrow[q];
                const int32_t yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = q * 4 + e;
                    const int32_t jr = J0 + ty * kRows + r;
                    if (kRagged && jr >= n) continue;
                    const int32_t g = xrow[r * kT] + yv[e] - rs.d[r] - dk;
                    // row side: row jr, partner column k (ascending in this thread)
                    {
                        const bool gt = g > rs.g[r];
                        const bool eq = g == rs.g[r];
                        rs.s[r] = gt ? sk : (eq ? min(rs.s[r], sk) : rs.s[r]);
                        rs.c[r] = gt ? k : rs.c[r];
                        rs.g[r] = max(rs.g[r], g);
                    }
                    // column side: row k, partner column jr (ascending in this loop)
                    {
                        const bool gt = g > cg;
                        const bool eq = g == cg;
                        cs = gt ? rs.sj[r] : (eq ? min(cs, rs.sj[r]) : cs);
                        cc = gt ? jr : cc;
                        cg = max(cg, g);
                    }
                }
            }
            if (cg > 0) {
                ka = pack_gain(cg, (uint32_t)cc);
                kj = pack_gain(cg, (uint32_t)cs);
            }
        }
    }
    if (kPacked) {
        int32_t* c32 = static_cast<int32_t*>(cb);
        c32[ty * kT + tx] = ca;
        c32[kGroups * kT + ty * kT + tx] = cj;
    } else {
        unsigned long long* c64 = static_cast<unsigned long long*>(cb);
        c64[ty * kT + tx] = ka;
        c64[kGroups * kT + ty * kT + tx] = kj;
    }
}

// Combine the row-group partials of the previous tile's columns.
template <int kRows, bool kPacked>
__device__ __forceinline__ void commit_columns(const void* cb, int32_t K0, int32_t n, const Workspace& w,
                                               const Packing& pk) {
    constexpr int kGroups = Geo<kRows>::kGroups;
    const int t = threadIdx.x;
    if (t >= 2 * kT) return;
    const int q = t & 63;
    const int half = t < kT ? 0 : 1;  // 0: agent keys, 1: job keys
    unsigned long long m = 0ull;
    if (kPacked) {
        const int32_t* src = static_cast<const int32_t*>(cb) + half * kGroups * kT;
        int32_t p = src[q];
#pragma unroll
        for (int g = 1; g < kGroups; ++g) p = max(p, src[g * kT + q]);
        m = unpack_key(p, pk);
    } else {
        const unsigned long long* src = static_cast<const unsigned long long*>(cb) + half * kGroups * kT;
#pragma unroll
        for (int g = 0; g < kGroups; ++g) m = umax64(m, src[g * kT + q]);
    }
    const int32_t k = K0 + q;
    if (m != 0ull && k < n) atomicMax(half == 0 ? &w.key_a[k] : &w.key_j[k], m);
}

template <int kRows, bool kPacked>
__device__ __forceinline__ void commit_rows(const Rows<kRows, kPacked>& rs, int32_t J0, int32_t n,
                                            const Workspace& w, const Packing& pk) {
    const int lane = threadIdx.x & 31;
    const int ty = threadIdx.x >> 6;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        unsigned long long ka, kj;
        if (kPacked) {
            int32_t a = rs.g[r], j = rs.s[r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                a = max(a, __shfl_xor_sync(0xffffffffu, a, off));
                j = max(j, __shfl_xor_sync(0xffffffffu, j, off));
            }
            ka = unpack_key(a, pk);
            kj = unpack_key(j, pk);
        } else {
            ka = rs.g[r] > 0 ? pack_gain(rs.g[r], (uint32_t)rs.c[r]) : 0ull;
            kj = rs.g[r] > 0 ? pack_gain(rs.g[r], (uint32_t)rs.s[r]) : 0ull;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                ka = umax64(ka, __shfl_xor_sync(0xffffffffu, ka, off));
                kj = umax64(kj, __shfl_xor_sync(0xffffffffu, kj, off));
            }
        }
        const int32_t jr = J0 + ty * kRows + r;
        if (lane == 0 && jr < n && ka != 0) {
            atomicMax(&w.key_a[jr], ka);
            atomicMax(&w.key_j[jr], kj);
        }
    }
}

template <int kRows>
constexpr size_t eval_smem_bytes() {
    return sizeof(Stage) * stages_for(kRows) + 2 * 2 * Geo<kRows>::kGroups * kT * sizeof(unsigned long long);
}

// The tile loop of one block of one instance's evaluation.  kTma: the X
// tiles arrive by TMA gathers (tm: tensor map over a) tracked by one mbarrier
// per stage; the Y tiles and the sigma / D rows by 16-byte cp.async.
template <int kRows, bool kPacked, bool kTma>
__device__ __forceinline__ void evaluation_loop(const Workspace& w, int32_t strip, int32_t bid, int32_t nblk,
                                                const Packing& pk, const CUtensorMap* tm) {
    constexpr int kGroups = Geo<kRows>::kGroups;
    constexpr int kStages = stages_for(kRows);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Stage* stages = reinterpret_cast<Stage*>(smem_raw);
    unsigned long long* colbuf = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(Stage) * kStages);
    // colbuf[b][0: agent keys kGroups x 64 | 1: job keys kGroups x 64], b = tile parity
    __shared__ __align__(8) uint64_t s_bar[kStages];
    if (kTma) {
        if (threadIdx.x == 0) {
            for (int q = 0; q < kStages; ++q) mbar_init(&s_bar[q], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }

    const int32_t n = w.n;
    const int32_t nb = (n + kT - 1) / kT;
    int32_t xs[4] = {0, 0, 0, 0};  // warp 0 under kTma: sigma of this lane's X rows of row block xs_j
    int32_t xs_j = -1;
    XRows<kRows> xr;  // without kTma: this thread's X source rows for row block xr_j
    int32_t xr_j = -1;

    // producer cursor: kStages - 1 tiles ahead of the consumer; the rows
    // (sigma) it will copy are loaded two tiles before they are needed
    TileCursor prod;
    bool prod_ok = cursor_first(prod, nb, strip, bid, nblk);
    for (int s = 0; s < kStages - 1; ++s) {
        if (prod_ok) {
            if (!kTma && prod.j != xr_j) {
                x_sources<kRows>(w, prod.j, xr);
                xr_j = prod.j;
            }
            issue_tile<kRows>(w, &stages[s], prod.j, prod.k, copy_rows<kRows, kTma>(w, prod.j, prod.k),
                              kTma ? nullptr : &xr);
            if (kTma && threadIdx.x < 32) {
                if (prod.j != xs_j) {
                    x_rows(w, prod.j, xs);
                    xs_j = prod.j;
                }
                gather_x(&stages[s], tm, prod.k * kT, xs, &s_bar[s]);
            }
            prod_ok = cursor_next(prod, nb, strip, nblk);
        }
        cp_async_commit();
    }
    TileCursor ahead = prod;  // one tile after prod
    bool ahead_ok = prod_ok && cursor_next(ahead, nb, strip, nblk);
    CopyRows<kRows> rows_now = prod_ok ? copy_rows<kRows, kTma>(w, prod.j, prod.k) : no_rows<kRows>();
    CopyRows<kRows> rows_next = ahead_ok ? copy_rows<kRows, kTma>(w, ahead.j, ahead.k) : no_rows<kRows>();

    TileCursor cons;
    bool cons_ok = cursor_first(cons, nb, strip, bid, nblk);
    Rows<kRows, kPacked> rs;
    bool item_start = true;
    int32_t t = 0, prev_k0 = -1;
    int32_t cs = 0;       // consumer stage (t mod kStages)
    uint32_t cph = 0;     // its mbarrier phase
    while (cons_ok) {
        const int32_t J0 = cons.j * kT;
        cp_async_wait<kStages - 2>();
        if (kTma) {
            const bool ok = mbar_wait_bounded(&s_bar[cs], cph);
            if (__syncthreads_or(!ok)) {  // a gather never arrived: stop with an error
                if (threadIdx.x == 0) {
                    w.st->error = kErrWaitTimeout;
                    w.st->status = kError;
                    // gathers may still be in flight into any stage: wait for
                    // each stage's next completion (bounded) before leaving;
                    // stages before cs in this cycle complete next with the
                    // other parity
                    for (int q = 0; q < kStages; ++q) mbar_wait_bounded(&s_bar[q], q < cs ? cph ^ 1u : cph);
                }
                break;
            }
        } else {
            __syncthreads();  // tile t landed for every thread; tile t-1 fully consumed
        }
        const Stage* stage = &stages[cs];
        if (item_start) {
            rows_start<kRows, kPacked>(rs, stage, J0, pk);
            item_start = false;
        }
        if (prev_k0 >= 0) commit_columns<kRows, kPacked>(colbuf + ((t - 1) & 1) * 2 * kGroups * kT, prev_k0, n, w, pk);
        if (prod_ok) {
            const int32_t ps = cs == 0 ? kStages - 1 : cs - 1;  // the stage of tile t - 1, free now
            if (!kTma && prod.j != xr_j) {
                x_sources<kRows>(w, prod.j, xr);
                xr_j = prod.j;
            }
            issue_tile<kRows>(w, &stages[ps], prod.j, prod.k, rows_now, kTma ? nullptr : &xr);
            if (kTma && threadIdx.x < 32) {
                if (prod.j != xs_j) {
                    x_rows(w, prod.j, xs);
                    xs_j = prod.j;
                }
                gather_x(&stages[ps], tm, prod.k * kT, xs, &s_bar[ps]);
            }
            prod = ahead;
            prod_ok = ahead_ok;
            rows_now = rows_next;
            if (ahead_ok) {
                ahead_ok = cursor_next(ahead, nb, strip, nblk);
                if (ahead_ok) rows_next = copy_rows<kRows, kTma>(w, ahead.j, ahead.k);
            }
        }
        cp_async_commit();
        const int32_t K0 = cons.k * kT;
        unsigned long long* cb = colbuf + (t & 1) * 2 * kGroups * kT;
        if ((J0 + kT > n) || (K0 + kT > n)) compute_tile<kRows, true, kPacked>(stage, rs, J0, K0, n, pk, cb);
        else compute_tile<kRows, false, kPacked>(stage, rs, J0, K0, n, pk, cb);
        const bool run_end = cons.k + 1 >= cons.kend;  // last tile of this row run
        if (run_end) commit_rows<kRows, kPacked>(rs, J0, n, w, pk);
        prev_k0 = K0;
        ++t;
        if (++cs == kStages) {
            cs = 0;
            cph ^= 1u;
        }
        cons_ok = cursor_next(cons, nb, strip, nblk);
        item_start = run_end;
    }
    cp_async_wait<0>();
    __syncthreads();
    if (prev_k0 >= 0 && w.st->status == kRunning)
        commit_columns<kRows, kPacked>(colbuf + ((t - 1) & 1) * 2 * kGroups * kT, prev_k0, n, w, pk);
    __syncthreads();  // the stages and colbuf may be reused by the caller's next call
}

// The evaluation of one instance by block bid of the nblk blocks assigned to
// it (a CTA of the single-instance launch, or one item of a batched queue).
// All threads of the CTA call it together.
template <int kRows, bool kTma = false>
__device__ __forceinline__ void full_evaluation_body(const Workspace& w, int32_t conditional, int32_t strip,
                                                     int32_t bid, int32_t nblk, const CUtensorMap* tm = nullptr) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    if (conditional && !(st->need_update && use_full_update(st->rescan_count, w.n, st->update_policy))) return;
    if (conditional && bid == 0 && threadIdx.x == 0) st->full_evals += 1;
    const Packing pk = packing_for(w.n, st->max_abs);
    if (pk.pw != 0 && !w.exact_keys) evaluation_loop<kRows, true, kTma>(w, strip, bid, nblk, pk, tm);
    else evaluation_loop<kRows, false, kTma>(w, strip, bid, nblk, pk, tm);
}

template <int kRows, bool kTma>
__global__ void __launch_bounds__(Geo<kRows>::kThreads, 1) full_evaluation_kernel(Workspace w, int32_t conditional,
                                                                                  int32_t strip,
                                                                                  const __grid_constant__ CUtensorMap tm) {
    full_evaluation_body<kRows, kTma>(w, conditional, strip, blockIdx.x, gridDim.x, &tm);
}

// Batched: each queue item is one block of one instance's evaluation (the
// scan kernel queued exactly the instances that need one).
template <int kRows>
__global__ void __launch_bounds__(Geo<kRows>::kThreads, 1) full_evaluation_batched_kernel(BatchQueues q,
                                                                                          int32_t strip) {
    for_each_item(q.inst, q.q0, q.cap, [&](const Instance& in, int32_t bid, int32_t nblk) {
        full_evaluation_body<kRows>(in.w, 0, strip, bid, nblk);
    });
}

// agent slot i <- key_a[tau(i)], job slot j <- key_j[j]  (public evaluation
// API); after a range or start error every slot reads "no candidate"
__global__ void keys_to_slots_kernel(Workspace w, int32_t* ag, int32_t* aj, int32_t* jg, int32_t* ja) {
    const bool failed = w.st->status == kError;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < w.n; t += gridDim.x * blockDim.x) {
        if (failed) {
            ag[t] = 0;
            aj[t] = -1;
            jg[t] = 0;
            ja[t] = -1;
            continue;
        }
        const unsigned long long ka = w.key_a[w.tau[t]];
        ag[t] = ka ? key_gain(ka) : 0;
        aj[t] = ka ? key_index(ka) : -1;
        const unsigned long long kj = w.key_j[t];
        jg[t] = kj ? key_gain(kj) : 0;
        ja[t] = kj ? key_index(kj) : -1;
    }
}

}  // namespace

// Launch shape of the single-instance evaluation: rows per thread (4: 1024
// threads per CTA; 8: 512) and strip (column tiles per work item; 0: one
// contiguous balanced range of tiles per CTA), per size
// class (bucket = bit length of n - 1).  Defaults until an autotune sets a
// class; DGS_EVAL_ROWS / DGS_EVAL_STRIP override every class (tests).  The
// shape never changes a result: every key is a maximum over the same pairs.
constexpr int kStrip = 8;
constexpr int32_t kBuckets = 18;
std::atomic<int32_t> g_shape[kBuckets];  // 0: default, else tma << 16 | rows << 8 | strip

int32_t size_bucket(int32_t n) { return n <= 1 ? 0 : std::min<int32_t>(kBuckets - 1, 32 - __builtin_clz((uint32_t)(n - 1))); }

int32_t env_int(const char* name, int32_t fallback) {
    const char* e = std::getenv(name);
    return e ? std::atoi(e) : fallback;
}

EvalShape evaluation_shape(int32_t n) {
    static const int32_t env_rows = env_int("DGS_EVAL_ROWS", 0);
    static const int32_t env_strip = env_int("DGS_EVAL_STRIP", -1);
    static const int32_t env_tma = env_int("DGS_EVAL_TMA", -1);
    EvalShape sh{8, kStrip, 0};
    const int32_t v = g_shape[size_bucket(n)].load(std::memory_order_relaxed);
    if (v != 0) sh = EvalShape{(v >> 8) & 255, v & 255, v >> 16};
    if (env_rows == 4 || env_rows == 8 || env_rows == 16) sh.rows = env_rows;
    if (env_strip >= 0 && env_strip <= 255) sh.strip = env_strip;
    if (env_tma == 0 || env_tma == 1) sh.tma = env_tma;
    if (sh.rows == 16) sh.tma = 0;  // 16 rows per thread: per-thread copies only
    return sh;
}

void set_evaluation_shape(int32_t n, EvalShape sh) {
    g_shape[size_bucket(n)].store((sh.tma ? 1 << 16 : 0) | sh.rows << 8 | sh.strip, std::memory_order_relaxed);
}

size_t full_evaluation_smem_bytes() { return eval_smem_bytes<8>(); }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return static_cast<EncodeTiledFn>(nullptr);
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Tensor map over a (n rows of lda int32, row pitch lda) with 64 x 1 boxes,
// the shape the gathers of the TMA path read.
bool make_gather_map(const Workspace& w, CUtensorMap* tm) {
    EncodeTiledFn fn = encode_tiled();
    if (fn == nullptr) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)w.lda, (cuuint64_t)w.n};
    const cuuint64_t strides[1] = {(cuuint64_t)w.lda * sizeof(int32_t)};
    const cuuint32_t box[2] = {(cuuint32_t)kT, 1};
    const cuuint32_t estr[2] = {1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, const_cast<int32_t*>(w.a), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int kRows, bool kTma>
static cudaError_t launch_eval(const Workspace& w, int32_t conditional, int32_t strip, const CUtensorMap& tm,
                               cudaStream_t s) {
    constexpr size_t smem = eval_smem_bytes<kRows>();
    const int slot = kRows == 16 ? 13 : kRows == 8 ? (kTma ? 11 : 0) : (kTma ? 10 : 7);  // attribute cache slots
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(full_evaluation_kernel<kRows, kTma>), slot, smem);
    if (e != cudaSuccess) return e;
    full_evaluation_kernel<kRows, kTma><<<dgs::device_sms(), Geo<kRows>::kThreads, smem, s>>>(w, conditional, strip, tm);
    return cudaGetLastError();
}

cudaError_t launch_full_evaluation_shape(const Workspace& w, int32_t conditional, EvalShape sh, cudaStream_t s) {
    alignas(64) CUtensorMap tm{};
    const bool tma = sh.tma && make_gather_map(w, &tm);
    if (sh.rows == 16) return launch_eval<16, false>(w, conditional, sh.strip, tm, s);
    if (sh.rows == 4) return tma ? launch_eval<4, true>(w, conditional, sh.strip, tm, s)
                                 : launch_eval<4, false>(w, conditional, sh.strip, tm, s);
    return tma ? launch_eval<8, true>(w, conditional, sh.strip, tm, s)
               : launch_eval<8, false>(w, conditional, sh.strip, tm, s);
}

cudaError_t launch_full_evaluation(const Workspace& w, int32_t conditional, cudaStream_t s) {
    if (w.row_owner_eval) return launch_row_owner_evaluation(w, conditional, s);
    return launch_full_evaluation_shape(w, conditional, evaluation_shape(w.n), s);
}

int32_t evaluation_strip() { return kStrip; }

// The evaluations queued in q.q0 (batch_blocks_eval(n, strip) blocks each),
// 512 threads per CTA (the 1024-thread variant would spill the instance's
// workspace pointers it reads from global memory).
cudaError_t launch_b_evaluation(const BatchQueues& q, int32_t strip, cudaStream_t s) {
    constexpr size_t smem = eval_smem_bytes<8>();
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(full_evaluation_batched_kernel<8>), 4, smem);
    if (e != cudaSuccess) return e;
    full_evaluation_batched_kernel<8><<<dgs::device_sms(), Geo<8>::kThreads, smem, s>>>(q, strip);
    return cudaGetLastError();
}

cudaError_t launch_keys_to_slots(const Workspace& w, int32_t* ag, int32_t* aj, int32_t* jg, int32_t* ja,
                                 cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > 1024) grid = 1024;
    keys_to_slots_kernel<<<grid, 256, 0, s>>>(w, ag, aj, jg, ja);
    return cudaGetLastError();
}

}  // namespace dgs
