// Evaluation tooling: Kendall's tau-b of tau against kappa (Section 5.2,
// Fig. 7: how similar the order of the r-cliques by an early-stopped tau is
// to the order by kappa).
//
// The values are small integers, so the pair count runs over a dense 2D
// histogram instead of sorting.  H[a][b] counts the r-cliques with
// (x - min x, y - min y) = (a, b).  After two suffix scans, in place,
// Q[a][b] = #{i : x_i >= a, y_i >= b} (in shifted coordinates).  A pair
// with a < a' is concordant if b < b' and discordant if b > b'; so the
// cell (a, b) contributes
//     H[a][b] * (Q[a+1][b+1] - (Q[a+1][0] - Q[a+1][b]))
// to S = concordant - discordant, and pairs tied in x or in y contribute 0.
// Ties: t_a = Q[a][0] - Q[a+1][0] values share x = a, giving t_a (t_a - 1) / 2
// pairs; likewise per column.  tau_b = S / sqrt((n0 - ties_x) (n0 - ties_y)).
// Work and memory are (Vx + 1) (Vy + 1) cells, Vx and Vy the value ranges.
#include "nd_internal.cuh"

#include <math.h>

namespace {

constexpr int kThreads = 256;
constexpr int64_t kMaxCells = int64_t(1) << 28;  // 2 GB of 8-byte counters

__global__ void k_minmax(const int32_t* __restrict__ x, const int32_t* __restrict__ y, int64_t n,
                         int* __restrict__ mm /* min x, max x, min y, max y */) {
    int lo_x = INT32_MAX, hi_x = INT32_MIN, lo_y = INT32_MAX, hi_y = INT32_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int a = x[i], b = y[i];
        lo_x = min(lo_x, a);
        hi_x = max(hi_x, a);
        lo_y = min(lo_y, b);
        hi_y = max(hi_y, b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo_x = min(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, o));
        hi_x = max(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, o));
        lo_y = min(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, o));
        hi_y = max(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm, lo_x);
        atomicMax(mm + 1, hi_x);
        atomicMin(mm + 2, lo_y);
        atomicMax(mm + 3, hi_y);
    }
}

__global__ void k_hist2d(const int32_t* __restrict__ x, const int32_t* __restrict__ y, int64_t n, int min_x,
                         int min_y, int64_t W, unsigned long long* __restrict__ Q) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(Q + (int64_t)(x[i] - min_x) * W + (y[i] - min_y), 1ull);
}

// Q[a][b] = sum over b' >= b of H[a][b'], one warp per row a (W - 1 = Vy
// cells; the last column stays 0)
__global__ void k_row_suffix(unsigned long long* __restrict__ Q, int64_t Vx, int64_t W) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < Vx; a += warps) {
        unsigned long long* row = Q + a * W;
        unsigned long long carry = 0;
        for (int64_t c0 = W - 2; c0 >= 0; c0 -= 32) {
            const int64_t b = c0 - lane;  // lane 0 holds the highest column of the chunk
            unsigned long long v = b >= 0 ? row[b] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            if (b >= 0) row[b] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// Q[a][b] += Q[a+1][b] from the last row up, one thread per column (row Vx
// stays 0)
__global__ void k_col_suffix(unsigned long long* __restrict__ Q, int64_t Vx, int64_t W) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < W; b += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long run = 0;
        for (int64_t a = Vx - 1; a >= 0; --a) {
            run += Q[a * W + b];
            Q[a * W + b] = run;
        }
    }
}

// out[0] += S, out[1] += ties in x, out[2] += ties in y (signed S in two's
// complement)
__global__ void k_kendall_terms(const unsigned long long* __restrict__ Q, int64_t Vx, int64_t Vy,
                                unsigned long long* __restrict__ out) {
    const int64_t W = Vy + 1;
    long long s = 0;
    unsigned long long tx = 0, ty = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < Vx * Vy;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = c / Vy, b = c % Vy;
        const unsigned long long q00 = Q[a * W + b], q10 = Q[(a + 1) * W + b];
        const unsigned long long q01 = Q[a * W + b + 1], q11 = Q[(a + 1) * W + b + 1];
        const unsigned long long h = q00 - q10 - q01 + q11;
        if (h) {
            const long long conc = (long long)q11;
            const long long disc = (long long)(Q[(a + 1) * W] - q10);
            s += (long long)h * (conc - disc);
        }
        if (b == 0) {
            const unsigned long long t = Q[a * W] - Q[(a + 1) * W];
            tx += t * (t - (t > 0)) / 2;
        }
        if (a == 0) {
            const unsigned long long u = Q[b] - Q[b + 1];
            ty += u * (u - (u > 0)) / 2;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        tx += __shfl_xor_sync(0xffffffffu, tx, o);
        ty += __shfl_xor_sync(0xffffffffu, ty, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (s) atomicAdd(out, (unsigned long long)s);
        if (tx) atomicAdd(out + 1, tx);
        if (ty) atomicAdd(out + 2, ty);
    }
}

}  // namespace

nd_status nd_kendall_dev(const int32_t* x, const int32_t* y, int64_t n, int sm_count, double* tau_out,
                         int64_t* counts_out, cudaStream_t st) {
    *tau_out = NAN;
    if (counts_out) counts_out[0] = counts_out[1] = counts_out[2] = 0;
    if (n < 2) return ND_OK;
    const int cap = (sm_count > 0 ? sm_count : 152) * 8;
    nd_tmp<int> mm(st);
    ND_TRY(mm.alloc(4));
    const int init[4] = {INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN};
    ND_CUDA(cudaMemcpyAsync(mm.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
    {
        nd_prof_scope ps("kendall", st);
        k_minmax<<<nd_blocks_for(n, kThreads, cap), kThreads, 0, st>>>(x, y, n, mm);
        ND_CUDA(cudaGetLastError());
    }
    int h_mm[4];
    ND_CUDA(cudaMemcpyAsync(h_mm, mm.p, sizeof(h_mm), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    const int64_t Vx = (int64_t)h_mm[1] - h_mm[0] + 1, Vy = (int64_t)h_mm[3] - h_mm[2] + 1;
    const int64_t W = Vy + 1;
    if ((double)(Vx + 1) * (double)W > (double)kMaxCells) {
        nd_set_error("value ranges too wide for the 2D histogram (more than 2^28 cells)");
        return ND_E_TOO_LARGE;
    }
    nd_tmp<unsigned long long> Q(st), out(st);
    ND_TRY(Q.alloc((Vx + 1) * W));
    ND_TRY(out.alloc(3));
    ND_CUDA(cudaMemsetAsync(Q.p, 0, sizeof(unsigned long long) * (size_t)((Vx + 1) * W), st));
    ND_CUDA(cudaMemsetAsync(out.p, 0, sizeof(unsigned long long) * 3, st));
    {
        nd_prof_scope ps("kendall", st, 4);
        k_hist2d<<<nd_blocks_for(n, kThreads, cap), kThreads, 0, st>>>(x, y, n, h_mm[0], h_mm[2], W, Q);
        ND_CUDA(cudaGetLastError());
        k_row_suffix<<<nd_blocks_for(Vx * 32, kThreads, cap), kThreads, 0, st>>>(Q, Vx, W);
        ND_CUDA(cudaGetLastError());
        k_col_suffix<<<nd_blocks_for(W, kThreads, cap), kThreads, 0, st>>>(Q, Vx, W);
        ND_CUDA(cudaGetLastError());
        k_kendall_terms<<<nd_blocks_for(Vx * Vy, kThreads, cap), kThreads, 0, st>>>(Q, Vx, Vy, out);
        ND_CUDA(cudaGetLastError());
    }
    unsigned long long h_out[3];
    ND_CUDA(cudaMemcpyAsync(h_out, out.p, sizeof(h_out), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    const long long S = (long long)h_out[0];
    if (counts_out) {
        counts_out[0] = S;
        counts_out[1] = (int64_t)h_out[1];
        counts_out[2] = (int64_t)h_out[2];
    }
    const double n0 = (double)n * (double)(n - 1) / 2.0;
    const double den = (n0 - (double)h_out[1]) * (n0 - (double)h_out[2]);
    *tau_out = den > 0.0 ? (double)S / sqrt(den) : NAN;
    return ND_OK;
}
