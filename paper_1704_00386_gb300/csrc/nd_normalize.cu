// Edge list -> simple undirected CSR, the input form of Section 2 (a simple
// undirected graph: no self-loop, no repeated edge, every edge seen from both
// endpoints, rows sorted).
//
// Every pair (a, b) with a != b emits its two directed keys (a, b) and (b, a),
// packed as (u << B) | v with B = bits of n - 1.  A stable LSD radix sort
// (8-bit digits) orders the keys; equal neighbours are adjacent after the sort,
// so the CSR is the first copy of every key: col = its low B bits, and row_ptr
// [u] = the first unique key whose row is >= u (a binary search per vertex).
//
// Radix pass, tile of kTile keys per block:
//   k_radix_hist   : 256-bin digit histogram of the tile -> hist[d * tiles + t];
//   scan           : exclusive prefix over (digit, tile) gives every tile's
//                    first output slot per digit (stable: tiles in order);
//   k_radix_scatter: stable rank of each key inside its tile (warps walk their
//                    keys in order, peers with the same digit found by
//                    __match_any_sync), keys reordered by digit in shared
//                    memory, then written out as contiguous runs.
// HBM-bound: each pass reads the keys twice and writes them once.
#include "nd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                   // keys per thread per tile
constexpr int kTile = kThreads * kItems;     // 4096 keys per block
constexpr int kPerWarp = kTile / kWarps;     // 512 keys per warp, in rounds of 32
constexpr int kBins = 256;

// both directed keys of every non-loop pair; ids out of [0, n) raise *err.
// Keys are appended through a warp-aggregated counter (their order is
// irrelevant: the sort below fixes it).
__global__ void k_emit_keys(const int64_t* __restrict__ src, const int64_t* __restrict__ dst, int64_t m, int64_t n,
                            int bits, unsigned long long* __restrict__ keys, unsigned long long* __restrict__ count,
                            int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every lane runs the same number of trips so the warp stays converged
    const int64_t trips = (m + stride - 1) / stride;
    for (int64_t k = 0; k < trips; ++k) {
        const int64_t i = first + k * stride;
        bool emit = false;
        unsigned long long ka = 0, kb = 0;
        if (i < m) {
            const int64_t a = src[i], b = dst[i];
            if (a < 0 || a >= n || b < 0 || b >= n) {
                atomicOr(err, 1);
            } else if (a != b) {
                emit = true;
                ka = ((unsigned long long)a << bits) | (unsigned long long)b;
                kb = ((unsigned long long)b << bits) | (unsigned long long)a;
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, emit);
        if (!mask) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(count, 2ull * (unsigned long long)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (emit) {
            const unsigned long long at = base + 2ull * (unsigned long long)__popc(mask & ((1u << lane) - 1u));
            keys[at] = ka;
            keys[at + 1] = kb;
        }
    }
}

__device__ __forceinline__ unsigned digit_of(unsigned long long k, int shift) {
    return (unsigned)(k >> shift) & (kBins - 1);
}

// 256-bin histogram of one tile's digits: hist[d * tiles + t]
__global__ void __launch_bounds__(kThreads) k_radix_hist(const unsigned long long* __restrict__ keys, int64_t count,
                                                         int shift, int64_t tiles, int64_t* __restrict__ hist) {
    __shared__ unsigned h[kBins];
    for (int i = threadIdx.x; i < kBins; i += kThreads) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;  // coalesced
        if (i < count) atomicAdd(&h[digit_of(keys[i], shift)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kThreads) hist[(int64_t)d * tiles + blockIdx.x] = h[d];
}

// stable scatter of one tile to its digit slots
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const unsigned long long* __restrict__ in,
                                                            unsigned long long* __restrict__ out, int64_t count,
                                                            int shift, int64_t tiles,
                                                            const int64_t* __restrict__ offs) {
    __shared__ unsigned wcount[kWarps][kBins];  // keys of each digit per warp; then the warp's offset
    __shared__ unsigned dstart[kBins];          // first position of each digit inside the tile
    __shared__ unsigned long long stage[kTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * kTile;
    const int64_t wbase = tbase + (int64_t)w * kPerWarp;
    // 1. stable rank of every key among the earlier keys of its warp with
    //    the same digit: rounds in order, lanes in order inside a round
    unsigned long long key[kPerWarp / 32];
    unsigned rank[kPerWarp / 32];
#pragma unroll
    for (int k = 0; k < kPerWarp / 32; ++k) {
        const int64_t i = wbase + (int64_t)k * 32 + lane;
        const bool ok = i < count;
        key[k] = ok ? in[i] : 0ull;
        // padding keys take digit kBins (never counted, never written)
        const unsigned d = ok ? digit_of(key[k], shift) : (unsigned)kBins;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned before = __popc(peers & ((1u << lane) - 1u));
        const unsigned run = ok ? wcount[w][d] : 0u;
        rank[k] = run + before;
        __syncwarp();
        if (ok && before == 0) wcount[w][d] = run + (unsigned)__popc(peers);  // the lowest peer updates
        __syncwarp();
    }
    __syncthreads();
    // 2. per digit: the warps' offsets inside the digit (in warp order), and
    //    the digit's start inside the tile (exclusive scan over digits)
    {
        const int d = threadIdx.x;  // kThreads == kBins
        unsigned run = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const unsigned c = wcount[ww][d];
            wcount[ww][d] = run;
            run += c;
        }
        // block-wide exclusive scan of the digit totals
        unsigned incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        __shared__ unsigned wsum[kWarps];
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        unsigned before = 0;
        for (int ww = 0; ww < w; ++ww) before += wsum[ww];
        dstart[d] = before + incl - run;
    }
    __syncthreads();
    // 3. reorder the tile by digit in shared memory
#pragma unroll
    for (int k = 0; k < kPerWarp / 32; ++k) {
        const int64_t i = wbase + (int64_t)k * 32 + lane;
        if (i < count) {
            const unsigned d = digit_of(key[k], shift);
            stage[dstart[d] + wcount[w][d] + rank[k]] = key[k];
        }
    }
    __syncthreads();
    // 4. write the runs out: consecutive threads, consecutive slots
    const int64_t valid = min((int64_t)kTile, count - tbase);
    for (int p = threadIdx.x; p < valid; p += kThreads) {
        const unsigned long long k = stage[p];
        const unsigned d = digit_of(k, shift);
        out[offs[(int64_t)d * tiles + blockIdx.x] + (p - dstart[d])] = k;
    }
}

// 1 where a key differs from its predecessor (the first copy of each key)
__global__ void k_first_copy(const unsigned long long* __restrict__ keys, int64_t count, int64_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// the first copies, compacted: their keys and their column ids
__global__ void k_compact(const unsigned long long* __restrict__ keys, int64_t count, const int64_t* __restrict__ pos,
                          int bits, unsigned long long* __restrict__ ukeys, int32_t* __restrict__ col) {
    const unsigned long long vmask = (1ull << bits) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        if (pos[i + 1] != pos[i]) {
            const unsigned long long k = keys[i];
            ukeys[pos[i]] = k;
            col[pos[i]] = (int32_t)(k & vmask);
        }
}

// row_ptr[u] = number of unique keys whose row is < u (lower bound of u << bits)
__global__ void k_row_ptr(const unsigned long long* __restrict__ ukeys, int64_t nnz, int64_t n, int bits,
                          int64_t* __restrict__ row_ptr) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= n; u += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long x = (unsigned long long)u << bits;
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (ukeys[mid] < x) lo = mid + 1; else hi = mid;
        }
        row_ptr[u] = lo;
    }
}

}  // namespace

int nd_id_bits(int64_t n) {
    int b = 1;
    while (b < 63 && ((int64_t)1 << b) < n) ++b;
    return b;
}

// stable LSD radix sort of keys[0, count) over their low `bits` bits; the
// result is in *result (keys or alt)
nd_status nd_sort_u64(unsigned long long* keys, unsigned long long* alt, int64_t count, int bits,
                      unsigned long long** result, cudaStream_t st) {
    *result = keys;
    if (count <= 1) return ND_OK;
    const int64_t tiles = (count + kTile - 1) / kTile;
    if (tiles > INT32_MAX) { nd_set_error("too many keys for one sort"); return ND_E_TOO_LARGE; }
    nd_tmp<int64_t> hist(st);
    ND_TRY(hist.alloc((int64_t)kBins * tiles + 1));
    unsigned long long *a = keys, *b = alt;
    for (int shift = 0; shift < bits; shift += 8) {
        {
            nd_prof_scope ps("radix_hist", st);
            k_radix_hist<<<(unsigned)tiles, kThreads, 0, st>>>(a, count, shift, tiles, hist);
            ND_CUDA(cudaGetLastError());
        }
        ND_TRY(nd_scan_i64(hist, (int64_t)kBins * tiles, st));
        {
            nd_prof_scope ps("radix_scatter", st);
            k_radix_scatter<<<(unsigned)tiles, kThreads, 0, st>>>(a, b, count, shift, tiles, hist);
            ND_CUDA(cudaGetLastError());
        }
        unsigned long long* t = a;
        a = b;
        b = t;
    }
    *result = a;
    return ND_OK;
}

extern "C" nd_status nd_normalize(const int64_t* src, const int64_t* dst, int64_t m, int64_t n, int on_device,
                                  int64_t* row_ptr_out, int32_t* col_out, int64_t col_capacity, int64_t* nnz_out,
                                  void* stream) {
    if (m < 0 || n < 0 || col_capacity < 0) { nd_set_error("negative size"); return ND_E_INVAL; }
    if (n >= INT32_MAX) { nd_set_error("more than 2^31-1 vertices"); return ND_E_TOO_LARGE; }
    if (!nnz_out || !row_ptr_out || (m > 0 && (!src || !dst))) { nd_set_error("NULL argument"); return ND_E_INVAL; }
    if (m > 0 && n == 0) { nd_set_error("edges given for an empty vertex set"); return ND_E_INVAL; }
    *nnz_out = 0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    ND_CUDA(cudaGetDevice(&dev));
    ND_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int bits = nd_id_bits(n);  // ids need `bits` bits; keys 2 * bits
    // device copies of host input
    const int64_t *dsrc = src, *ddst = dst;
    nd_tmp<int64_t> hsrc(st), hdst(st);
    if (!on_device && m > 0) {
        ND_TRY(hsrc.alloc(m));
        ND_TRY(hdst.alloc(m));
        ND_CUDA(cudaMemcpyAsync(hsrc, src, sizeof(int64_t) * m, cudaMemcpyHostToDevice, st));
        ND_CUDA(cudaMemcpyAsync(hdst, dst, sizeof(int64_t) * m, cudaMemcpyHostToDevice, st));
        dsrc = hsrc;
        ddst = hdst;
    }
    const int64_t cap = 2 * m;
    nd_tmp<unsigned long long> keys(st), alt(st), cnt(st);
    nd_tmp<int> err(st);
    ND_TRY(keys.alloc(cap));
    ND_TRY(alt.alloc(cap));
    ND_TRY(cnt.alloc(1));
    ND_TRY(err.alloc(1));
    ND_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    ND_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (m > 0) {
        nd_prof_scope ps("emit_keys", st);
        k_emit_keys<<<nd_blocks_for(m, kThreads, sms * 8), kThreads, 0, st>>>(dsrc, ddst, m, n, bits, keys, cnt, err);
        ND_CUDA(cudaGetLastError());
    }
    unsigned long long hcount = 0;
    int herr = 0;
    ND_CUDA(cudaMemcpyAsync(&hcount, cnt, sizeof(hcount), cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    if (herr) { nd_set_error("a vertex id is outside [0, n)"); return ND_E_INVAL; }
    const int64_t count = (int64_t)hcount;
    unsigned long long* sorted = keys;
    ND_TRY(nd_sort_u64(keys, alt, count, 2 * bits, &sorted, st));
    unsigned long long* ukeys = (sorted == keys) ? (unsigned long long*)alt : (unsigned long long*)keys;
    // first copies -> positions (exclusive scan; pos[count] = number of unique keys)
    nd_tmp<int64_t> pos(st);
    ND_TRY(pos.alloc(count + 1));
    if (count > 0) {
        nd_prof_scope ps("first_copy", st);
        k_first_copy<<<nd_blocks_for(count, kThreads, sms * 8), kThreads, 0, st>>>(sorted, count, pos);
        ND_CUDA(cudaGetLastError());
    }
    ND_CUDA(cudaMemsetAsync(pos + count, 0, sizeof(int64_t), st));
    ND_TRY(nd_scan_i64(pos, count, st));
    int64_t nnz = 0;
    ND_CUDA(cudaMemcpyAsync(&nnz, pos + count, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    *nnz_out = nnz;
    if (nnz > col_capacity) {
        nd_set_error("col_out holds fewer entries than the normalised graph (*nnz_out gives the size needed)");
        return ND_E_INVAL;
    }
    if (nnz > 0 && !col_out) { nd_set_error("col_out is NULL"); return ND_E_INVAL; }
    // outputs: straight into device buffers, or staged for host buffers
    int32_t* dcol = col_out;
    int64_t* drp = row_ptr_out;
    nd_tmp<int32_t> scol(st);
    nd_tmp<int64_t> srp(st);
    if (!on_device) {
        ND_TRY(scol.alloc(nnz));
        ND_TRY(srp.alloc(n + 1));
        dcol = scol;
        drp = srp;
    }
    if (count > 0) {
        nd_prof_scope ps("compact", st);
        k_compact<<<nd_blocks_for(count, kThreads, sms * 8), kThreads, 0, st>>>(sorted, count, pos, bits, ukeys, dcol);
        ND_CUDA(cudaGetLastError());
    }
    {
        nd_prof_scope ps("row_ptr", st);
        k_row_ptr<<<nd_blocks_for(n + 1, kThreads, sms * 8), kThreads, 0, st>>>(ukeys, nnz, n, bits, drp);
        ND_CUDA(cudaGetLastError());
    }
    if (!on_device) {
        ND_CUDA(cudaMemcpyAsync(row_ptr_out, drp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
        if (nnz > 0) ND_CUDA(cudaMemcpyAsync(col_out, dcol, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st));
    }
    return nd_wait(st);
}
