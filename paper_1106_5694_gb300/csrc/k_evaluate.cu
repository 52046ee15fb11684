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
// 64 row segments of 256 B each, gathered through sigma and copied into
// shared memory by the TMA engine (1-D cp.async.bulk, mbarrier completion).
// Every element of a is read exactly once per evaluation.  A CTA walks a
// strip of tiles with the same J, keeping the row-side maxima of its 64 rows
// in registers; column-side maxima are committed per tile with 64-bit
// atomicMax, which is order independent and therefore deterministic.
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kT = 64;        // tile edge
constexpr int kYP = kT + 4;   // Y row pitch (ints): 16-B aligned and int4-conflict-free
constexpr int kStages = 3;
constexpr int kThreads = 256; // 4 row groups x 64 columns
constexpr int kRows = 16;     // rows per thread

struct Stage {
    int32_t x[kT * kT];
    int32_t y[kT * kYP];
};

struct TileCursor {
    int32_t item;   // index into the item table
    int32_t k;      // current column tile
    int32_t kend;   // one past the last column tile of the item
    int32_t j;      // row block
};

__device__ __forceinline__ bool cursor_load(TileCursor& c, const Workspace& w, int32_t item, int32_t nb,
                                            int32_t strip) {
    c.item = item;
    if (item >= w.item_count) return false;
    const int2 it = w.items[item];
    c.j = it.x;
    c.k = it.y;
    c.kend = min(it.y + strip, nb);
    return true;
}

// Issue the bulk copies of tile (J, K) into stage s (warp 0, all lanes).
__device__ __forceinline__ void issue_tile(const Workspace& w, Stage* stage, uint64_t* bar, int32_t J, int32_t K) {
    const int lane = threadIdx.x & 31;
    const int32_t n = w.n;
    const int32_t J0 = J * kT, K0 = K * kT;
    const int32_t rows_x = min(kT, n - J0), rows_y = min(kT, n - K0);
    const uint32_t bytes_x = 4u * (uint32_t)min(kT, w.lda - K0);  // row segment of X (columns K)
    const uint32_t bytes_y = 4u * (uint32_t)min(kT, w.lda - J0);  // row segment of Y (columns J)
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)rows_x * bytes_x + (uint32_t)rows_y * bytes_y);
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        if (r < rows_x) {
            const int32_t src_row = w.sigma[J0 + r];
            bulk_g2s(stage->x + r * kT, w.a + (size_t)src_row * w.lda + K0, bytes_x, bar);
        }
        if (r < rows_y) {
            const int32_t src_row = w.sigma[K0 + r];
            bulk_g2s(stage->y + r * kYP, w.a + (size_t)src_row * w.lda + J0, bytes_y, bar);
        }
    }
}

struct RowState {
    int32_t g[kRows];  // best gain (starts at 0: only strictly positive gains count)
    int32_t c[kRows];  // its lowest partner column
    int32_t s[kRows];  // lowest partner agent among the columns reaching g
};

template <bool kRagged>
__device__ __forceinline__ void compute_tile(const Stage* stage, RowState& rs, const int32_t (&dj)[kRows],
                                             const int32_t (&sj)[kRows], int32_t J0, int32_t K0, int32_t n,
                                             const Workspace& w) {
    const int tx = threadIdx.x & 63;
    const int ty = threadIdx.x >> 6;
    const int32_t k = K0 + tx;
    if (kRagged && k >= n) return;
    const int32_t sk = w.sigma[k];
    const int32_t dk = w.diag[k];
    int32_t cg = 0, cc = -1, cs = 0x7fffffff;
    const int32_t* xrow = stage->x + (ty * kRows) * kT + tx;
    const int4* yrow = reinterpret_cast<const int4*>(stage->y + tx * kYP + ty * kRows);
#pragma unroll
    for (int q = 0; q < kRows / 4; ++q) {
        const int4 y4 = yrow[q];
        const int32_t yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = q * 4 + e;
            const int32_t jr = J0 + ty * kRows + r;
            if (kRagged && jr >= n) continue;
            const int32_t x = xrow[r * kT];
            const int32_t g = x + yv[e] - dj[r] - dk;
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
        atomicMax(&w.key_a[k], pack_gain(cg, (uint32_t)cc));
        atomicMax(&w.key_j[k], pack_gain(cg, (uint32_t)cs));
    }
}

__device__ __forceinline__ void commit_rows(const RowState& rs, int32_t J0, int32_t n, const Workspace& w) {
    const int lane = threadIdx.x & 31;
    const int ty = threadIdx.x >> 6;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        unsigned long long ka = rs.g[r] > 0 ? pack_gain(rs.g[r], (uint32_t)rs.c[r]) : 0ull;
        unsigned long long kj = rs.g[r] > 0 ? pack_gain(rs.g[r], (uint32_t)rs.s[r]) : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ka = umax64(ka, __shfl_xor_sync(0xffffffffu, ka, off));
            kj = umax64(kj, __shfl_xor_sync(0xffffffffu, kj, off));
        }
        const int32_t jr = J0 + ty * kRows + r;
        if (lane == 0 && jr < n && ka != 0) {
            atomicMax(&w.key_a[jr], ka);
            atomicMax(&w.key_j[jr], kj);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2) full_evaluation_kernel(Workspace w, int32_t conditional,
                                                                      int32_t strip) {
    DeviceState* st = w.st;
    if (st->status != kRunning) return;
    if (conditional && !(st->need_update && use_full_update(st->rescan_count, w.n))) return;
    if (conditional && blockIdx.x == 0 && threadIdx.x == 0) st->full_evals += 1;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    Stage* stages = reinterpret_cast<Stage*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(Stage) * kStages);

    const int32_t n = w.n;
    const int32_t nb = (n + kT - 1) / kT;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // producer cursor (warp 0) runs kStages tiles ahead of the consumer
    TileCursor prod;
    bool prod_ok = cursor_load(prod, w, blockIdx.x, nb, strip);
    int32_t issued = 0;
    if (warp == 0) {
        for (int s = 0; s < kStages && prod_ok; ++s) {
            issue_tile(w, &stages[s], &bars[s], prod.j, prod.k);
            ++issued;
            if (++prod.k >= prod.kend) prod_ok = cursor_load(prod, w, prod.item + gridDim.x, nb, strip);
        }
    }

    TileCursor cons;
    bool cons_ok = cursor_load(cons, w, blockIdx.x, nb, strip);
    int32_t consumed = 0;
    bool failed = false;
    RowState rs;
    int32_t dj[kRows], sj[kRows];
    bool item_start = true;
    while (cons_ok) {
        const int32_t J0 = cons.j * kT;
        if (item_start) {
            const int ty = threadIdx.x >> 6;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const int32_t jr = J0 + ty * kRows + r;
                dj[r] = jr < n ? w.diag[jr] : 0;
                sj[r] = jr < n ? w.sigma[jr] : 0;
                rs.g[r] = 0;
                rs.c[r] = -1;
                rs.s[r] = 0x7fffffff;
            }
            item_start = false;
        }
        const int s = consumed % kStages;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((consumed / kStages) & 1));
        if (__syncthreads_or(!ok)) {  // block-uniform decision
            failed = true;
            break;
        }
        const int32_t K0 = cons.k * kT;
        const bool ragged = (J0 + kT > n) || (K0 + kT > n);
        if (ragged) compute_tile<true>(&stages[s], rs, dj, sj, J0, K0, n, w);
        else compute_tile<false>(&stages[s], rs, dj, sj, J0, K0, n, w);
        ++consumed;
        const bool last_of_item = (cons.k + 1 >= cons.kend);
        if (last_of_item) commit_rows(rs, J0, n, w);
        __syncthreads();  // stage s fully read
        if (warp == 0 && prod_ok) {
            issue_tile(w, &stages[s], &bars[s], prod.j, prod.k);
            ++issued;
            if (++prod.k >= prod.kend) prod_ok = cursor_load(prod, w, prod.item + gridDim.x, nb, strip);
        }
        if (++cons.k >= cons.kend) {
            cons_ok = cursor_load(cons, w, cons.item + gridDim.x, nb, strip);
            item_start = true;
        }
    }
    if (failed) {
        // drain this CTA's own copies still in flight (bounded), then report
        if (threadIdx.x == 0) {
            for (int32_t t = consumed; t < issued; ++t)
                (void)mbar_wait_bounded(&bars[t % kStages], (uint32_t)((t / kStages) & 1));
            atomicExch(&st->error, kErrWaitTimeout);
            atomicExch(&st->status, kError);
        }
        __syncthreads();
    }
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

size_t full_evaluation_smem_bytes() { return sizeof(Stage) * kStages + 64; }

cudaError_t launch_full_evaluation(const Workspace& w, int32_t conditional, cudaStream_t s) {
    const size_t smem = full_evaluation_smem_bytes();
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(full_evaluation_kernel), 0, smem);
    if (e != cudaSuccess) return e;
    int grid = w.item_count < 152 * 2 ? w.item_count : 152 * 2;
    if (grid < 1) grid = 1;
    full_evaluation_kernel<<<grid, kThreads, smem, s>>>(w, conditional, kStrip);
    return cudaGetLastError();
}

int32_t evaluation_strip() { return kStrip; }

cudaError_t launch_keys_to_slots(const Workspace& w, int32_t* ag, int32_t* aj, int32_t* jg, int32_t* ja,
                                 cudaStream_t s) {
    int grid = (w.n + 255) / 256;
    if (grid > 1024) grid = 1024;
    keys_to_slots_kernel<<<grid, 256, 0, s>>>(w, ag, aj, jg, ja);
    return cudaGetLastError();
}

}  // namespace dgs
