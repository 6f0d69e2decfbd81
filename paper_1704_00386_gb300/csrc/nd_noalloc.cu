// Core numbers by SND with no device allocation at all.
//
// Some callers cannot allocate device memory when they call us: their
// process hands the whole GPU memory to another allocator up front (a
// framework that pre-reserves the device pool), or they run where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// nd_core_snd_noalloc serves them.  It computes the same core numbers as
// nd_build_incidence(g, 1, 2) followed by nd_snd, straight from a device
// CSR, and its only scratch is the file-scope array below (one previous-pass
// tau buffer and a ring of per-pass counters).
//
// The array belongs to this file's device code, which CUDA loads onto a GPU
// lazily (by default): the first call on a device that looks up the array,
// or launches one of the kernels below, loads the code and creates the array
// there, and that step itself takes device memory.  A call with n = 0 does
// exactly that and nothing else, so a caller whose allocator reserves the
// device up front makes that call first.  From then on the device holds the
// array until the process exits, and no call allocates.
#include <mutex>

#include "nd_internal.cuh"

namespace {

constexpr int64_t kMaxVertices = 1 << 20;   // largest graph this entry point accepts
constexpr int kRing = 64;                   // per-pass counter slots
constexpr int kBatch = 16;                  // passes enqueued between host reads
constexpr int kThreads = 256;
constexpr size_t kTauBytes = sizeof(int32_t) * kMaxVertices;
constexpr size_t kScratchBytes = kTauBytes + sizeof(unsigned long long) * 2 * kRing;

// [0, kTauBytes): tau of the previous pass; then kRing x {changed, error}
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Per-device address of g_scratch as seen by kernels.  In host code the name
// g_scratch is only a host-side stand-in, so the address must be fetched
// with cudaGetSymbolAddress, once per device, with that device current.  A
// failed set-up is not remembered: the next call tries again.
std::mutex g_mu;
void* g_addr[64];

__global__ void k_core_init(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, int32_t* __restrict__ a,
                            int32_t* __restrict__ b, unsigned long long* __restrict__ err) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = rp[u], hi = rp[u + 1];
        int32_t d = 0;
        if (lo < 0 || hi < lo || hi > nnz) atomicOr(err, 1ull);
        else d = (int32_t)(hi - lo);
        a[u] = d;
        b[u] = d;
    }
}

// One SND pass (Alg. 2) for (r,s) = (1,2): tau_out(u) = H({tau_in(v) : v in
// N(u)}) clipped to tau_in(u), one warp per vertex.  Rows and neighbour ids
// are bounds-checked; a bad entry is skipped and reported.
__global__ void __launch_bounds__(kThreads) k_core_pass(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                                        const int32_t* __restrict__ col,
                                                        const int32_t* __restrict__ tin, int32_t* __restrict__ tout,
                                                        unsigned long long* __restrict__ ctr,
                                                        const unsigned long long* __restrict__ prev) {
    if (prev != nullptr && *(volatile const unsigned long long*)prev == 0ull) return;  // converged
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long changed = 0, bad = 0;
    for (int64_t u = warp; u < n; u += warps) {
        const int64_t lo_p = rp[u], hi_p = rp[u + 1];
        const int32_t t = tin[u];
        if (lo_p < 0 || hi_p < lo_p || hi_p > nnz) {
            if (lane == 0) { tout[u] = t; bad = 1; }
            continue;
        }
        // count neighbours whose tau reaches x
        auto count_ge = [&](int32_t x) {
            int c = 0;
            for (int64_t p = lo_p + lane; p < hi_p; p += 32) {
                const int32_t v = col[p];
                if (v >= 0 && v < n) c += (tin[v] >= x);
                else bad = 1;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            return c;
        };
        int32_t h = 0;
        if (t > 0) {
            const int cnt = count_ge(t);
            if (cnt >= t) {
                h = t;  // preserve-tau exit (Section 4.4)
            } else {
                int lo = cnt, hi = t;  // #{tau >= lo} >= lo holds; at hi it fails (Def. 3)
                while (hi - lo > 1) {
                    const int mid = lo + ((hi - lo) >> 1);
                    if (count_ge(mid) >= mid) lo = mid; else hi = mid;
                }
                h = lo;
            }
        }
        if (lane == 0) {
            tout[u] = h;
            changed += (h != t);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_xor_sync(0xffffffffu, changed, o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
        if (changed) atomicAdd(ctr, changed);
        if (bad) atomicOr(ctr + 1, 1ull);
    }
}

// Set-up on the current device, once: the array's address, and the two
// kernels loaded (cudaFuncGetAttributes loads a lazily loaded kernel), so
// that no later call loads code or data onto the device.
nd_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    ND_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { nd_set_error("device ordinal out of range"); return ND_E_INVAL; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* addr = nullptr;
        ND_CUDA(cudaGetSymbolAddress(&addr, g_scratch));
        cudaFuncAttributes fa;
        ND_CUDA(cudaFuncGetAttributes(&fa, k_core_init));
        ND_CUDA(cudaFuncGetAttributes(&fa, k_core_pass));
        g_addr[dev] = addr;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return ND_OK;
}

}  // namespace

extern "C" nd_status nd_core_snd_noalloc(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz,
                                         int32_t* core_out, int32_t max_iters, int32_t* iters_out,
                                         void* stream) {
    if (n < 0 || nnz < 0 || max_iters < 0) { nd_set_error("negative size"); return ND_E_INVAL; }
    if (n > kMaxVertices) {
        nd_set_error("nd_core_snd_noalloc accepts at most 1048576 vertices; use nd_build_incidence + nd_snd");
        return ND_E_TOO_LARGE;
    }
    if (iters_out) *iters_out = 0;
    unsigned char* scratch = nullptr;
    ND_TRY(scratch_for_current_device(&scratch));  // the set-up; all a call with n = 0 does
    if (n == 0) return ND_OK;
    if (!row_ptr || !core_out || (nnz > 0 && !col)) { nd_set_error("NULL pointer"); return ND_E_INVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t* tprev = reinterpret_cast<int32_t*>(scratch);
    unsigned long long* ring = reinterpret_cast<unsigned long long*>(scratch + kTauBytes);
    int sms = 152;
    int dev = 0;
    ND_CUDA(cudaGetDevice(&dev));
    ND_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nd_blocks_for(n * 32, kThreads, sms * 8);
    // the array keeps the previous call's contents: clear every counter first
    ND_CUDA(cudaMemsetAsync(ring, 0, sizeof(unsigned long long) * 2 * kRing, st));
    k_core_init<<<nd_blocks_for(n, kThreads, sms * 8), kThreads, 0, st>>>(n, nnz, row_ptr, core_out, tprev, ring + 1);
    ND_CUDA(cudaGetLastError());
    // pass p reads buf[p % 2] and writes buf[(p + 1) % 2]; buf[0] = scratch, buf[1] = core_out
    int32_t* buf[2] = {tprev, core_out};
    int32_t pass = 0, updating = 0, newest = 0;
    bool done = false, bad = false;
    while (!done && pass < max_iters) {
        const int32_t start = pass;
        int nb = kBatch;
        if (nb > max_iters - pass) nb = max_iters - pass;
        const int slot0 = start % kRing;
        if (slot0 + nb > kRing) nb = kRing - slot0;
        if (start > 0)
            ND_CUDA(cudaMemsetAsync(ring + 2 * slot0, 0, sizeof(unsigned long long) * 2 * nb, st));
        for (int k = 0; k < nb; ++k, ++pass) {
            const unsigned long long* prev = pass == 0 ? nullptr : ring + 2 * ((pass - 1) % kRing);
            k_core_pass<<<grid, kThreads, 0, st>>>(n, nnz, row_ptr, col, buf[pass & 1], buf[(pass & 1) ^ 1],
                                                   ring + 2 * (pass % kRing), prev);
            ND_CUDA(cudaGetLastError());
        }
        unsigned long long host[2 * kBatch];
        ND_CUDA(cudaMemcpyAsync(host, ring + 2 * slot0, sizeof(unsigned long long) * 2 * nb,
                                cudaMemcpyDeviceToHost, st));
        ND_TRY(nd_wait(st));
        for (int k = 0; k < nb; ++k) {
            if (host[2 * k + 1]) bad = true;
            newest = ((start + k) & 1) ^ 1;
            if (host[2 * k] == 0) { done = true; break; }
            ++updating;
        }
        if (bad) break;
    }
    // the error flag of the initialisation lives in slot 0
    unsigned long long init_bad = 0;
    ND_CUDA(cudaMemcpyAsync(&init_bad, ring + 1, sizeof(init_bad), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    if (bad || init_bad) { nd_set_error("row_ptr / col out of range"); return ND_E_INVAL; }
    if (pass > 0 && buf[newest] != core_out)
        ND_CUDA(cudaMemcpyAsync(core_out, buf[newest], sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
    ND_TRY(nd_wait(st));
    if (iters_out) *iters_out = updating;
    if (!done) { nd_set_error("iteration cap reached before a pass without change"); return ND_E_NOT_CONVERGED; }
    return ND_OK;
}
