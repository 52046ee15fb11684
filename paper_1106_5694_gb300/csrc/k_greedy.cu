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

__global__ void __launch_bounds__(256) greedy_pass1_kernel(Workspace w, int32_t tiles_x, int32_t tiles_total) {
    __shared__ int32_t s[kT][kT + 1];
    __shared__ unsigned long long colpart[4][kT];
    const int32_t n = w.n;
    const int t = threadIdx.x;
    const int lane16 = t & 15;
    bool bad = false;
    for (int32_t tile = blockIdx.x; tile < tiles_total; tile += gridDim.x) {
        const int32_t I0 = (tile / tiles_x) * kT;
        const int32_t J0 = (tile % tiles_x) * kT;
        // load 64 rows x 64 cols with int4, 16 threads per row, 4 passes
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int r = (t >> 4) + 16 * p;
            const int c = lane16 * 4;
            const int32_t i = I0 + r, j = J0 + c;
            int4 v = make_int4(0, 0, 0, 0);
            if (i < n && j < w.lda) v = *reinterpret_cast<const int4*>(w.a + (size_t)i * w.lda + j);
            s[r][c + 0] = v.x; s[r][c + 1] = v.y; s[r][c + 2] = v.z; s[r][c + 3] = v.w;
            // row best over this tile's 4 columns of this thread
            unsigned long long best = 0;
            const int32_t vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (i < n && j + e < n) {
                    const int32_t x = vals[e];
                    bad |= (x >= kBenefitLimit) || (x <= -kBenefitLimit);
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
    if (bad) {
        atomicExch(&w.st->error, kErrRange);
        atomicExch(&w.st->status, kError);
    }
}

// Match every mutually-best (agent, job) pair.
__global__ void greedy_match_kernel(Workspace w) {
    DeviceState* st = w.st;
    if (st->status != kRunning || st->greedy_remaining == 0) return;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x) {
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

// |a| < 2^29 check alone (for entry points that do not run pass 1).
__global__ void range_check_kernel(Workspace w) {
    bool bad = false;
    const size_t total4 = (size_t)w.n * (size_t)(w.lda / 4);
    const int32_t row4 = w.lda / 4;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total4; q += (size_t)gridDim.x * blockDim.x) {
        const int32_t c = (int32_t)(q % row4) * 4;
        const int4 v = reinterpret_cast<const int4*>(w.a)[q];
        const int32_t vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (c + e < w.n) bad |= (vals[e] >= kBenefitLimit) || (vals[e] <= -kBenefitLimit);
    }
    if (bad) {
        atomicExch(&w.st->error, kErrRange);
        atomicExch(&w.st->status, kError);
    }
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

}  // namespace dgs
