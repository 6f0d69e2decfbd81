// Exclusive prefix sums over int64 (offsets of every CSR this library builds).
//
// Three-phase scan: each 256-thread block reduces a tile of 2048 elements,
// the tile sums are scanned (recursively), then each tile is scanned and
// offset.  HBM-bound: two reads and one write of the array.
#include "nd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread across the block; returns the
// block total through *total
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t w = (lane < kThreads / 32) ? warp_sums[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < kThreads / 32) warp_sums[lane] = wi - w;  // exclusive prefix of warp sums
        if (lane == kThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = warp_sums[wid] + incl - v;
    __syncthreads();
    return r;
}

__global__ void k_tile_sums(const int64_t* __restrict__ a, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (base + i < n) s += a[base + i];
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_tile_scan(int64_t* __restrict__ a, int64_t n, const int64_t* __restrict__ offs) {
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        v[i] = (base + i < n) ? a[base + i] : 0;
        s += v[i];
    }
    int64_t run = block_excl_scan(s, &tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (base + i < n) {
            int64_t x = v[i];
            a[base + i] = run;
            run += x;
        }
}

nd_status scan_rec(int64_t* data, int64_t count, cudaStream_t st) {
    const int64_t n = count + 1;  // the trailing slot receives the total
    const int64_t tiles = (n + kTile - 1) / kTile;
    if (tiles == 1) {
        k_tile_scan<<<1, kThreads, 0, st>>>(data, n, nullptr);
        ND_CUDA(cudaGetLastError());
        return ND_OK;
    }
    int64_t* sums = nullptr;
    ND_CUDA(cudaMallocAsync((void**)&sums, sizeof(int64_t) * (tiles + 1), st));
    ND_CUDA(cudaMemsetAsync(sums + tiles, 0, sizeof(int64_t), st));
    k_tile_sums<<<(unsigned)tiles, kThreads, 0, st>>>(data, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { cudaFreeAsync(sums, st); return nd_cuda_fail(e, "k_tile_sums", __FILE__, __LINE__); }
    nd_status s = scan_rec(sums, tiles, st);  // sums[tiles] = grand total (unused)
    if (s != ND_OK) { cudaFreeAsync(sums, st); return s; }
    k_tile_scan<<<(unsigned)tiles, kThreads, 0, st>>>(data, n, sums);
    e = cudaGetLastError();
    cudaFreeAsync(sums, st);
    if (e != cudaSuccess) return nd_cuda_fail(e, "k_tile_scan", __FILE__, __LINE__);
    return ND_OK;
}

}  // namespace

nd_status nd_scan_i64(int64_t* data, int64_t count, cudaStream_t st) {
    nd_prof_scope ps("scan", st);
    return scan_rec(data, count, st);
}
