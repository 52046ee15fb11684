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
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kT = 64;         // tile edge
constexpr int kYP = kT + 4;    // Y row pitch (ints): 16-B aligned and int4-conflict-free
constexpr int kStages = 5;
constexpr int kThreads = 512;  // 8 row groups x 64 columns
constexpr int kRows = 8;       // rows per thread
constexpr int kGroups = kThreads / kT;

struct Stage {
    int32_t x[kT * kT];
    int32_t y[kT * kYP];
    int32_t sk[kT];  // sigma of the tile's columns
    int32_t dk[kT];  // D of the tile's columns
    int32_t sj[kT];  // sigma of the tile's rows (the row block J)
    int32_t dj[kT];  // D of the tile's rows
};

struct TileCursor {
    int32_t item;   // index into the item table
    int32_t k;      // current column tile
    int32_t kend;   // one past the last column tile of the item
    int32_t j;      // row block
};

// Work items (row block J, first column tile J + strip * c) are numbered
// J * chunks + c; items whose first tile lies past the last block are empty
// and skipped.  Block b of the nblk blocks working on one instance walks
// items b, b + nblk, b + 2 nblk, ...
__device__ __forceinline__ bool cursor_load(TileCursor& c, int32_t item, int32_t nb, int32_t strip, int32_t nblk) {
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

__device__ __forceinline__ bool cursor_next(TileCursor& c, int32_t nb, int32_t strip, int32_t nblk) {
    if (++c.k < c.kend) return true;
    return cursor_load(c, c.item + nblk, nb, strip, nblk);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// sigma of the rows this thread copies for tile (J, K): X rows J0+rq, J0+rq+32
// and Y rows K0+rq, K0+rq+32 (row rq = threadIdx.x / 16).
struct CopyRows {
    int32_t x0, x1, y0, y1;
};

__device__ __forceinline__ CopyRows copy_rows(const Workspace& w, int32_t J, int32_t K) {
    const int32_t rq = threadIdx.x >> 4;
    const int32_t J0 = J * kT, K0 = K * kT, n = w.n;
    CopyRows c;
    c.x0 = (J0 + rq < n) ? w.sigma[J0 + rq] : -1;
    c.x1 = (J0 + rq + 32 < n) ? w.sigma[J0 + rq + 32] : -1;
    c.y0 = (K0 + rq < n) ? w.sigma[K0 + rq] : -1;
    c.y1 = (K0 + rq + 32 < n) ? w.sigma[K0 + rq + 32] : -1;
    return c;
}

// Issue this thread's four 16-byte copies of tile (J, K) into stage.
__device__ __forceinline__ void issue_tile(const Workspace& w, Stage* stage, int32_t J, int32_t K,
                                           const CopyRows& c) {
    const int32_t chunk = (threadIdx.x & 15) * 4;  // first int of the 16-byte chunk
    const int32_t rq = threadIdx.x >> 4;
    const int32_t J0 = J * kT, K0 = K * kT;
    const bool in_x = chunk < w.lda - K0;  // X rows hold columns K0.. (row pitch lda)
    const bool in_y = chunk < w.lda - J0;  // Y rows hold columns J0..
    if (in_x && c.x0 >= 0) cp_async16(stage->x + rq * kT + chunk, w.a + (size_t)c.x0 * w.lda + K0 + chunk);
    if (in_x && c.x1 >= 0) cp_async16(stage->x + (rq + 32) * kT + chunk, w.a + (size_t)c.x1 * w.lda + K0 + chunk);
    if (in_y && c.y0 >= 0) cp_async16(stage->y + rq * kYP + chunk, w.a + (size_t)c.y0 * w.lda + J0 + chunk);
    if (in_y && c.y1 >= 0) cp_async16(stage->y + (rq + 32) * kYP + chunk, w.a + (size_t)c.y1 * w.lda + J0 + chunk);
    // sigma and D of the columns (arrays hold at least round_up(n, 64) entries)
    if (threadIdx.x < 16) cp_async16(stage->sk + chunk, w.sigma + K0 + chunk);
    else if (threadIdx.x < 32) cp_async16(stage->dk + chunk, w.diag + K0 + chunk);
    else if (threadIdx.x < 48) cp_async16(stage->sj + chunk, w.sigma + J0 + chunk);
    else if (threadIdx.x < 64) cp_async16(stage->dj + chunk, w.diag + J0 + chunk);
}

// Row-side state of a thread's 8 rows across a strip.  Exact path: best gain,
// its lowest column, lowest partner agent among columns reaching it.  Packed
// path (when |gain| * 2^s fits in int32, s = index bits): two int32 keys per
// row, (gain << s) + (mask - column) and (gain << s) + (mask - partner agent),
// where max picks the larger gain, then the lower index.
struct RowState {
    int32_t g[kRows];
    int32_t c[kRows];
    int32_t s[kRows];
};

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

// One tile: thread (ty, tx) covers column k = K0 + tx and rows J0 + ty*8 .. +7.
// Column-side partial keys go to colbuf (combined at the next barrier).
template <bool kRagged, bool kPacked>
__device__ __forceinline__ void compute_tile(const Stage* stage, RowState& rs, const int32_t (&dj)[kRows],
                                             const int32_t (&sj)[kRows], int32_t J0, int32_t K0, int32_t n,
                                             const Packing& pk, unsigned long long* col_a,
                                             unsigned long long* col_j) {
    const int tx = threadIdx.x & 63;
    const int ty = threadIdx.x >> 6;
    const int32_t k = K0 + tx;
    unsigned long long ka = 0ull, kj = 0ull;
    if (!kRagged || k < n) {
        const int32_t sk = stage->sk[tx];
        const int32_t dk = stage->dk[tx];
        const int32_t* xrow = stage->x + (ty * kRows) * kT + tx;
        const int4* yrow = reinterpret_cast<const int4*>(stage->y + tx * kYP + ty * kRows);
        if (kPacked) {
            const int32_t cka = pk.mask - k, ckj = pk.mask - sk;
            int32_t ca = pk.mask, cj = pk.mask;
#pragma unroll
            for (int q = 0; q < kRows / 4; ++q) {
                const int4 y4 = yrow[q];
                const int32_t yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = q * 4 + e;
                    const int32_t jr = J0 + ty * kRows + r;
                    if (kRagged && jr >= n) continue;
                    const int32_t g = xrow[r * kT] + yv[e] - dj[r] - dk;
                    rs.g[r] = max(rs.g[r], g * pk.pw + cka);          // row jr, lowest column
                    rs.s[r] = max(rs.s[r], g * pk.pw + ckj);          // row jr, lowest partner agent
                    ca = max(ca, g * pk.pw + (pk.mask - jr));          // row k, lowest column
                    cj = max(cj, g * pk.pw + (pk.mask - sj[r]));       // row k, lowest partner agent
                }
            }
            ka = unpack_key(ca, pk);
            kj = unpack_key(cj, pk);
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
                    const int32_t g = xrow[r * kT] + yv[e] - dj[r] - dk;
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
                        cs = gt ? sj[r] : (eq ? min(cs, sj[r]) : cs);
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
    col_a[ty * kT + tx] = ka;
    col_j[ty * kT + tx] = kj;
}

// Combine the 8 row-group partials of the previous tile's columns.
__device__ __forceinline__ void commit_columns(const unsigned long long* col_a, const unsigned long long* col_j,
                                               int32_t K0, int32_t n, const Workspace& w) {
    const int t = threadIdx.x;
    if (t >= 2 * kT) return;
    const int q = t & 63;
    const unsigned long long* src = (t < kT) ? col_a : col_j;
    unsigned long long m = 0ull;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) m = umax64(m, src[g * kT + q]);
    const int32_t k = K0 + q;
    if (m != 0ull && k < n) atomicMax((t < kT) ? &w.key_a[k] : &w.key_j[k], m);
}

template <bool kPacked>
__device__ __forceinline__ void commit_rows(const RowState& rs, int32_t J0, int32_t n, const Workspace& w,
                                            const Packing& pk) {
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

// The evaluation of one instance by block bid of the nblk blocks assigned to
// it (a CTA of the single-instance launch, or one entry of a batched work
// table).  All threads of the CTA call it together.
__device__ __forceinline__ void full_evaluation_body(const Workspace& w, int32_t conditional, int32_t strip,
                                                     int32_t bid, int32_t nblk) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    if (conditional && !(st->need_update && use_full_update(st->rescan_count, w.n, st->update_policy))) return;
    if (conditional && bid == 0 && threadIdx.x == 0) st->full_evals += 1;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    Stage* stages = reinterpret_cast<Stage*>(smem_raw);
    unsigned long long* colbuf = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(Stage) * kStages);
    // colbuf[b][0: agent keys 8x64 | 1: job keys 8x64], b = tile parity

    const int32_t n = w.n;
    const int32_t nb = (n + kT - 1) / kT;
    const Packing pk = packing_for(n, st->max_abs);
    const bool packed = pk.pw != 0 && !w.exact_keys;

    // producer cursor: kStages - 1 tiles ahead of the consumer; the rows
    // (sigma) it will copy are loaded two tiles before they are needed
    TileCursor prod;
    bool prod_ok = cursor_load(prod, bid, nb, strip, nblk);
    for (int s = 0; s < kStages - 1; ++s) {
        if (prod_ok) {
            issue_tile(w, &stages[s], prod.j, prod.k, copy_rows(w, prod.j, prod.k));
            prod_ok = cursor_next(prod, nb, strip, nblk);
        }
        cp_async_commit();
    }
    TileCursor ahead = prod;  // one tile after prod
    bool ahead_ok = prod_ok && cursor_next(ahead, nb, strip, nblk);
    CopyRows rows_now = prod_ok ? copy_rows(w, prod.j, prod.k) : CopyRows{-1, -1, -1, -1};
    CopyRows rows_next = ahead_ok ? copy_rows(w, ahead.j, ahead.k) : CopyRows{-1, -1, -1, -1};

    TileCursor cons;
    bool cons_ok = cursor_load(cons, bid, nb, strip, nblk);
    RowState rs;
    int32_t dj[kRows], sj[kRows];
    bool item_start = true;
    int32_t t = 0, prev_k0 = -1;
    while (cons_ok) {
        const int32_t J0 = cons.j * kT;
        cp_async_wait<kStages - 2>();
        __syncthreads();  // tile t landed for every thread; tile t-1 fully consumed
        const Stage* stage = &stages[t % kStages];
        if (item_start) {
            const int ty = threadIdx.x >> 6;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                dj[r] = stage->dj[ty * kRows + r];
                sj[r] = stage->sj[ty * kRows + r];
                rs.g[r] = packed ? pk.mask : 0;
                rs.c[r] = -1;
                rs.s[r] = packed ? pk.mask : 0x7fffffff;
            }
            item_start = false;
        }
        if (prev_k0 >= 0) {
            const unsigned long long* cb = colbuf + ((t - 1) & 1) * 2 * kGroups * kT;
            commit_columns(cb, cb + kGroups * kT, prev_k0, n, w);
        }
        if (prod_ok) {
            issue_tile(w, &stages[(t + kStages - 1) % kStages], prod.j, prod.k, rows_now);
            prod = ahead;
            prod_ok = ahead_ok;
            rows_now = rows_next;
            if (ahead_ok) {
                ahead_ok = cursor_next(ahead, nb, strip, nblk);
                if (ahead_ok) rows_next = copy_rows(w, ahead.j, ahead.k);
            }
        }
        cp_async_commit();
        const int32_t K0 = cons.k * kT;
        unsigned long long* cb = colbuf + (t & 1) * 2 * kGroups * kT;
        const bool ragged = (J0 + kT > n) || (K0 + kT > n);
        if (packed) {
            if (ragged) compute_tile<true, true>(stage, rs, dj, sj, J0, K0, n, pk, cb, cb + kGroups * kT);
            else compute_tile<false, true>(stage, rs, dj, sj, J0, K0, n, pk, cb, cb + kGroups * kT);
        } else {
            if (ragged) compute_tile<true, false>(stage, rs, dj, sj, J0, K0, n, pk, cb, cb + kGroups * kT);
            else compute_tile<false, false>(stage, rs, dj, sj, J0, K0, n, pk, cb, cb + kGroups * kT);
        }
        if (cons.k + 1 >= cons.kend) {
            if (packed) commit_rows<true>(rs, J0, n, w, pk);
            else commit_rows<false>(rs, J0, n, w, pk);
        }
        prev_k0 = K0;
        ++t;
        if (++cons.k >= cons.kend) {
            cons_ok = cursor_load(cons, cons.item + nblk, nb, strip, nblk);
            item_start = true;
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    if (prev_k0 >= 0) {
        const unsigned long long* cb = colbuf + ((t - 1) & 1) * 2 * kGroups * kT;
        commit_columns(cb, cb + kGroups * kT, prev_k0, n, w);
    }
    __syncthreads();  // the stages and colbuf may be reused by the caller's next call
}

__global__ void __launch_bounds__(kThreads, 1) full_evaluation_kernel(Workspace w, int32_t conditional,
                                                                      int32_t strip) {
    full_evaluation_body(w, conditional, strip, blockIdx.x, gridDim.x);
}

// Batched: each queue item is one block of one instance's evaluation (the
// scan kernel queued exactly the instances that need one).
__global__ void __launch_bounds__(kThreads, 1) full_evaluation_batched_kernel(BatchQueues q, int32_t strip) {
    for_each_item(q.inst, q.q0, q.cap, [&](const Instance& in, int32_t bid, int32_t nblk) {
        full_evaluation_body(in.w, 0, strip, bid, nblk);
    });
}

// agent slot i <- key_a[tau(i)], job slot j <- key_j[j]  (public evaluation API)
__global__ void keys_to_slots_kernel(Workspace w, int32_t* ag, int32_t* aj, int32_t* jg, int32_t* ja) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < w.n; t += gridDim.x * blockDim.x) {
        const unsigned long long ka = w.key_a[w.tau[t]];
        ag[t] = ka ? key_gain(ka) : 0;
        aj[t] = ka ? key_index(ka) : -1;
        const unsigned long long kj = w.key_j[t];
        jg[t] = kj ? key_gain(kj) : 0;
        ja[t] = kj ? key_index(kj) : -1;
    }
}

}  // namespace

constexpr int kStrip = 8;

size_t full_evaluation_smem_bytes() { return sizeof(Stage) * kStages + 2 * 2 * kGroups * kT * sizeof(unsigned long long); }

cudaError_t launch_full_evaluation(const Workspace& w, int32_t conditional, cudaStream_t s) {
    const size_t smem = full_evaluation_smem_bytes();
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(full_evaluation_kernel), 0, smem);
    if (e != cudaSuccess) return e;
    int grid = 152;
    if (grid < 1) grid = 1;
    full_evaluation_kernel<<<grid, kThreads, smem, s>>>(w, conditional, kStrip);
    return cudaGetLastError();
}

int32_t evaluation_strip() { return kStrip; }

// The evaluations queued in q.q0 (batch_blocks_eval(n, strip) blocks each).
cudaError_t launch_b_evaluation(const BatchQueues& q, int32_t strip, cudaStream_t s) {
    const size_t smem = full_evaluation_smem_bytes();
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(full_evaluation_batched_kernel), 4, smem);
    if (e != cudaSuccess) return e;
    full_evaluation_batched_kernel<<<152, kThreads, smem, s>>>(q, strip);
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
