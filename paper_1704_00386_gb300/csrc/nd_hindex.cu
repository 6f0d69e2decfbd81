// The iterated h-index update (Def. 4) as GPU passes: SND (Alg. 2) and AND
// with or without notification (Alg. 3, Section 4.3).
//
// One pass = one launch.  Blocks are dispatched to four degree buckets of
// r-cliques (d_s in [1,8], [9,64], [65,1024], >1024) and each r-clique is
// evaluated by a group of 4, 8, 32 or 32 lanes.  A group:
//   1. streams the r-clique's incidence row (coalesced, q ids per s-clique),
//      gathers the q tau values of each s-clique and keeps
//      rho = min(...) in registers (Def. 4, step 1);
//   2. counts rho >= tau(R).  If at least tau(R) of them are, H = tau(R):
//      the preserve-tau early exit of Section 4.4, valid because the update
//      never raises tau (Thm. 1);
//   3. otherwise H lies in [count, tau(R)) and is found by binary search on
//      h over the register-resident rho values, testing
//      #{rho >= h} >= h (Def. 3).  No histogram, no sort.
// The paper's linear-time hashmap h-index (Section 4.4) is replaced by this
// tau-bounded count; both compute Def. 3 exactly.
//
// SND reads tau_p and writes tau (ping-pong buffers, no copy).  AND reads and
// writes one tau array in place; tau only decreases, so a stale read is a
// larger value and at worst delays convergence.  With notification, an
// r-clique is evaluated only if its bit is set in the current frontier; when
// its tau drops to h it sets the next-frontier bit of every neighbour R' with
// h <= tau(R') (Alg. 3, the orange lines).  It does not re-activate itself.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "nd_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kThreads = 256;

struct SweepParams {
    const int64_t* __restrict__ inc_ptr;
    const uint32_t* __restrict__ inc;
    const int32_t* tin;   // SND: tau of the previous pass; AND: same array as tout
    int32_t* tout;
    const uint32_t* __restrict__ perm;
    int64_t lo[ND_NB], hi[ND_NB];
    int blk[ND_NB + 1];
    const uint32_t* cur;  // AND + notification: frontier read in this pass
    uint32_t* next;       // and the frontier written for the next pass
    unsigned long long* ctr;         // this pass: [0] changed, [1] evaluated
    const unsigned long long* prev;  // previous pass (null on the first)
};

template <bool RO>
__device__ __forceinline__ int32_t ld_tau(const int32_t* p) {
    if (RO) return __ldg(p);
    return *(volatile const int32_t*)p;
}

// rho(S,R) for the s-clique at incidence j: min of the other r-cliques' tau
template <int Q, bool RO>
__device__ __forceinline__ int32_t rho_at(const uint32_t* __restrict__ inc, const int32_t* tau, int64_t j) {
    if (Q == 1) {
        return ld_tau<RO>(tau + __ldg(inc + j));
    } else if (Q == 2) {
        uint2 id = __ldg(reinterpret_cast<const uint2*>(inc) + j);
        return min(ld_tau<RO>(tau + id.x), ld_tau<RO>(tau + id.y));
    } else {
        const uint32_t* p = inc + 3 * j;
        uint32_t a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
        return min(min(ld_tau<RO>(tau + a), ld_tau<RO>(tau + b)), ld_tau<RO>(tau + c));
    }
}

// H({rho_j}) clipped to t, for one r-clique, by a group of G lanes.
// C > 0: the row fits in G*C registers.  C == 0: stream the row per probe.
template <int Q, int G, int C, bool RO>
__device__ __forceinline__ int32_t group_hindex(const cg::thread_block_tile<G>& g,
                                                const uint32_t* __restrict__ inc, const int32_t* tau,
                                                int64_t jb, int64_t je, int32_t t) {
    const int lane = g.thread_rank();
    if (t <= 0) return 0;
    if (C > 0) {
        int32_t rho[C > 0 ? C : 1];
        int cnt = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            int64_t j = jb + lane + (int64_t)c * G;
            rho[c] = (j < je) ? rho_at<Q, RO>(inc, tau, j) : -1;
            cnt += (rho[c] >= t);
        }
        cnt = cg::reduce(g, cnt, cg::plus<int>());
        if (cnt >= t) return t;
        int lo = cnt, hi = t;  // #{rho >= lo} >= lo holds; at hi it fails
        while (hi - lo > 1) {
            int mid = lo + ((hi - lo) >> 1);
            int c2 = 0;
#pragma unroll
            for (int c = 0; c < C; ++c) c2 += (rho[c] >= mid);
            c2 = cg::reduce(g, c2, cg::plus<int>());
            if (c2 >= mid) lo = mid; else hi = mid;
        }
        return lo;
    } else {
        int cnt = 0;
        for (int64_t j = jb + lane; j < je; j += G) cnt += (rho_at<Q, RO>(inc, tau, j) >= t);
        cnt = cg::reduce(g, cnt, cg::plus<int>());
        if (cnt >= t) return t;
        int lo = cnt, hi = t;
        while (hi - lo > 1) {
            int mid = lo + ((hi - lo) >> 1);
            int c2 = 0;
            for (int64_t j = jb + lane; j < je; j += G) c2 += (rho_at<Q, RO>(inc, tau, j) >= mid);
            c2 = cg::reduce(g, c2, cg::plus<int>());
            if (c2 >= mid) lo = mid; else hi = mid;
        }
        return lo;
    }
}

template <int Q, int G, int C, bool AND, bool NOTIFY>
__device__ __forceinline__ void run_bucket(const SweepParams& P, int b, unsigned long long& changed,
                                           unsigned long long& evals) {
    auto g = cg::tiled_partition<G>(cg::this_thread_block());
    const int64_t groups_per_block = kThreads / G;
    const int64_t nblk = P.blk[b + 1] - P.blk[b];
    const int64_t gid = (int64_t)(blockIdx.x - P.blk[b]) * groups_per_block + g.meta_group_rank();
    const int64_t stride = nblk * groups_per_block;
    const int lane = g.thread_rank();
    for (int64_t i = P.lo[b] + gid; i < P.hi[b]; i += stride) {
        const uint32_t R = __ldg(P.perm + i);
        if (AND && NOTIFY) {
            if (!((__ldg(P.cur + (R >> 5)) >> (R & 31)) & 1u)) continue;
        }
        const int32_t t = ld_tau<!AND>(P.tin + R);
        const int64_t jb = __ldg(P.inc_ptr + R), je = __ldg(P.inc_ptr + R + 1);
        const int32_t h = group_hindex<Q, G, C, !AND>(g, P.inc, P.tin, jb, je, t);
        if (lane == 0) {
            evals++;
            if (h != t) changed++;
            if (!AND || h != t) P.tout[R] = h;
        }
        if (AND && NOTIFY && h != t) {
            // notify every neighbour whose tau could still depend on R: h <= tau(R')
            for (int64_t j = jb + lane; j < je; j += G) {
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    uint32_t Rp = __ldg(P.inc + Q * j + k);
                    if (h <= ld_tau<false>(P.tin + Rp)) {
                        uint32_t bit = 1u << (Rp & 31);
                        uint32_t* w = P.next + (Rp >> 5);
                        if (!(*(volatile uint32_t*)w & bit)) atomicOr(w, bit);
                    }
                }
            }
        }
    }
}

template <int Q, bool AND, bool NOTIFY>
__global__ void __launch_bounds__(kThreads) k_pass(SweepParams P) {
    if (P.prev != nullptr && *(volatile const unsigned long long*)P.prev == 0ull) return;  // converged
    unsigned long long changed = 0, evals = 0;
    int b = 0;
    while (b < ND_NB - 1 && (int)blockIdx.x >= P.blk[b + 1]) ++b;
    switch (b) {
        case 0: run_bucket<Q, 4, 2, AND, NOTIFY>(P, 0, changed, evals); break;
        case 1: run_bucket<Q, 8, 8, AND, NOTIFY>(P, 1, changed, evals); break;
        case 2: run_bucket<Q, 32, 32, AND, NOTIFY>(P, 2, changed, evals); break;
        default: run_bucket<Q, 32, 0, AND, NOTIFY>(P, 3, changed, evals); break;
    }
    __shared__ unsigned long long s_ch[kThreads / 32], s_ev[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_xor_sync(0xffffffffu, changed, o);
        evals += __shfl_xor_sync(0xffffffffu, evals, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { s_ch[wid] = changed; s_ev[wid] = evals; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, e = 0;
        for (int w = 0; w < kThreads / 32; ++w) { a += s_ch[w]; e += s_ev[w]; }
        if (a) atomicAdd(P.ctr, a);
        if (e) atomicAdd(P.ctr + 1, e);
    }
}

__global__ void k_init_tau(int64_t N, const int64_t* __restrict__ inc_ptr, int32_t* __restrict__ a,
                           int32_t* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = (int32_t)(inc_ptr[i + 1] - inc_ptr[i]);
        a[i] = d;
        if (b) b[i] = d;
    }
}

__global__ void k_fill_front(int64_t N, uint32_t* __restrict__ f) {
    const int64_t words = (N + 31) / 32;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = N - w * 32;
        f[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
}

__global__ void k_add_const(const int32_t* __restrict__ in, int64_t n, int32_t c, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] + c;
}

typedef void (*pass_fn)(SweepParams);

pass_fn pick(int q, int mode) {
    // mode: ND_SND, ND_AND (notify), ND_AND_NN
    if (q == 1) return mode == ND_SND ? k_pass<1, false, false> : (mode == ND_AND ? k_pass<1, true, true> : k_pass<1, true, false>);
    if (q == 2) return mode == ND_SND ? k_pass<2, false, false> : (mode == ND_AND ? k_pass<2, true, true> : k_pass<2, true, false>);
    return mode == ND_SND ? k_pass<3, false, false> : (mode == ND_AND ? k_pass<3, true, true> : k_pass<3, true, false>);
}

// blocks per bucket in proportion to its incidences (its share of the work),
// never more than its groups need, at least one if it is non-empty
void plan_blocks(const nd_incidence* h, SweepParams& P) {
    const int group[ND_NB] = {4, 8, 32, 32};
    const int64_t total_blocks = (int64_t)(h->sm_count > 0 ? h->sm_count : 152) * 8;
    int64_t tot_inc = 0;
    for (int b = 0; b < ND_NB; ++b) tot_inc += h->bucket_inc[b];
    int acc = 0;
    for (int b = 0; b < ND_NB; ++b) {
        P.blk[b] = acc;
        int64_t cnt = h->bucket_lo[b + 1] - h->bucket_lo[b];
        P.lo[b] = h->bucket_lo[b];
        P.hi[b] = h->bucket_lo[b + 1];
        if (cnt == 0) continue;
        int64_t need = (cnt * group[b] + kThreads - 1) / kThreads;
        int64_t share = tot_inc > 0 ? (total_blocks * h->bucket_inc[b] + tot_inc - 1) / tot_inc : 1;
        int64_t nb = share < need ? share : need;
        if (nb < 1) nb = 1;
        acc += (int)nb;
    }
    P.blk[ND_NB] = acc;
}

nd_status ensure_state(nd_incidence* h, bool and_mode, cudaStream_t st) {
    const int64_t N = h->num_r > 0 ? h->num_r : 1;
    if (!h->tau[0]) ND_TRY(nd_alloc((void**)&h->tau[0], sizeof(int32_t) * N, st, h));
    if (!and_mode && !h->tau[1]) ND_TRY(nd_alloc((void**)&h->tau[1], sizeof(int32_t) * N, st, h));
    const int64_t words = (N + 31) / 32;
    if (and_mode && !h->front[0]) {
        ND_TRY(nd_alloc((void**)&h->front[0], sizeof(uint32_t) * words, st, h));
        ND_TRY(nd_alloc((void**)&h->front[1], sizeof(uint32_t) * words, st, h));
    }
    if (!h->counters) {
        ND_TRY(nd_alloc((void**)&h->counters, sizeof(unsigned long long) * 2 * ND_RING, st, h));
        ND_CUDA(cudaMallocHost((void**)&h->h_counters, sizeof(unsigned long long) * 2 * ND_RING));
    }
    return ND_OK;
}

}  // namespace

nd_status nd_init_tau(nd_incidence* h, int32_t* tau, cudaStream_t st) {
    if (h->num_r == 0) return ND_OK;
    int blocks = nd_blocks_for(h->num_r, kThreads, h->sm_count * 8);
    nd_prof_scope ps("init_tau", st);
    k_init_tau<<<blocks, kThreads, 0, st>>>(h->num_r, h->inc_ptr, tau, nullptr);
    ND_CUDA(cudaGetLastError());
    return ND_OK;
}

nd_status nd_classic_truss(const int32_t* in, int64_t n, int32_t* out, cudaStream_t st) {
    if (n == 0) return ND_OK;
    int blocks = nd_blocks_for(n, kThreads, 152 * 8);
    nd_prof_scope ps("classic_truss", st);
    k_add_const<<<blocks, kThreads, 0, st>>>(in, n, 2, out);
    ND_CUDA(cudaGetLastError());
    return ND_OK;
}

// Runs passes of `mode` until a pass changes nothing or max_passes passes ran.
// Passes are enqueued in batches; each pass reads the previous pass's counter
// on the device and returns at once if it was zero, so the host only reads
// the counters back once per batch.
nd_status nd_run(nd_incidence* h, int mode, int32_t max_passes, const int32_t* tau_in_dev,
                 int32_t** tau_result, int32_t* updating, int64_t* evals, bool* converged,
                 cudaStream_t st) {
    const bool and_mode = (mode != ND_SND);
    const int64_t N = h->num_r;
    ND_TRY(ensure_state(h, and_mode, st));
    h->last_changed.clear();
    h->last_evals.clear();
    *updating = 0;
    *evals = 0;
    *converged = false;
    int blocks = nd_blocks_for(N, kThreads, h->sm_count * 8);
    if (N > 0) {
        if (tau_in_dev) {
            ND_CUDA(cudaMemcpyAsync(h->tau[0], tau_in_dev, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
            if (!and_mode)
                ND_CUDA(cudaMemcpyAsync(h->tau[1], tau_in_dev, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
        } else {
            nd_prof_scope ps("init_tau", st);
            k_init_tau<<<blocks, kThreads, 0, st>>>(N, h->inc_ptr, h->tau[0], and_mode ? nullptr : h->tau[1]);
            ND_CUDA(cudaGetLastError());
        }
    }
    *tau_result = h->tau[0];
    if (N == 0 || max_passes <= 0) {
        *converged = (N == 0);
        return ND_OK;
    }
    const int64_t words = (N + 31) / 32;
    int fc = 0;  // index of the current frontier
    if (mode == ND_AND) {
        nd_prof_scope ps("fill_front", st);
        k_fill_front<<<nd_blocks_for(words, kThreads, h->sm_count * 8), kThreads, 0, st>>>(N, h->front[0]);
        ND_CUDA(cudaGetLastError());
    }
    SweepParams P;
    P.inc_ptr = h->inc_ptr;
    P.inc = h->inc;
    P.perm = h->perm;
    plan_blocks(h, P);
    const int grid = P.blk[ND_NB];
    pass_fn fn = pick(h->q, mode);
    const int kBatch = 16;
    int32_t pass = 0;
    bool done = false;
    int32_t last_written = 0;  // SND: index of the buffer holding the newest tau
    while (!done && pass < max_passes) {
        const int32_t start = pass;
        const int slot0 = start % ND_RING;
        int nb = kBatch;
        if (nb > max_passes - pass) nb = max_passes - pass;
        if (slot0 + nb > ND_RING) nb = ND_RING - slot0;
        ND_CUDA(cudaMemsetAsync(h->counters + 2 * slot0, 0, sizeof(unsigned long long) * 2 * nb, st));
        for (int k = 0; k < nb; ++k, ++pass) {
            const int slot = pass % ND_RING;
            P.ctr = h->counters + 2 * slot;
            P.prev = (pass == 0) ? nullptr : h->counters + 2 * ((pass - 1) % ND_RING);
            if (and_mode) {
                P.tin = h->tau[0];
                P.tout = h->tau[0];
                P.cur = h->front[fc];
                P.next = h->front[fc ^ 1];
                if (mode == ND_AND)
                    ND_CUDA(cudaMemsetAsync(h->front[fc ^ 1], 0, sizeof(uint32_t) * words, st));
                fc ^= 1;
            } else {
                P.tin = h->tau[pass & 1];
                P.tout = h->tau[(pass & 1) ^ 1];
                P.cur = nullptr;
                P.next = nullptr;
            }
            if (grid > 0) {
                nd_prof_scope ps(mode == ND_SND ? "snd_pass" : (mode == ND_AND ? "and_pass" : "and_nn_pass"), st);
                fn<<<grid, kThreads, 0, st>>>(P);
                ND_CUDA(cudaGetLastError());
            }
        }
        ND_CUDA(cudaMemcpyAsync(h->h_counters + 2 * slot0, h->counters + 2 * slot0,
                                sizeof(unsigned long long) * 2 * nb, cudaMemcpyDeviceToHost, st));
        ND_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < nb; ++k) {
            const int32_t p = start + k;
            unsigned long long ch = h->h_counters[2 * (slot0 + k)];
            unsigned long long ev = h->h_counters[2 * (slot0 + k) + 1];
            // r-cliques with d_s = 0 are never launched: tau = H(empty) = 0 = d_s.
            // They count as evaluated in every SND / AND-nn pass and in the first
            // AND pass, as in the paper's sequential loops.
            if (mode != ND_AND || p == 0) ev += (unsigned long long)h->num_zero;
            h->last_changed.push_back((int64_t)ch);
            h->last_evals.push_back((int64_t)ev);
            *evals += (int64_t)ev;
            if (!and_mode) last_written = (p & 1) ^ 1;
            if (ch == 0) { done = true; break; }
            (*updating)++;
        }
    }
    *converged = done;
    *tau_result = and_mode ? h->tau[0] : h->tau[last_written];
    return ND_OK;
}
