// The iterated h-index update (Def. 4) as GPU passes: SND (Alg. 2) and AND
// with or without notification (Alg. 3, Section 4.3).
//
// One pass = one launch of a persistent grid.  R-cliques are grouped into
// four degree buckets (by default d_s in [1,8], [9,64], [65,2048], >2048)
// and evaluated by a group of 4 or 8 lanes, a warp, or a whole CTA.  The CTA
// rows are taken one per block from a per-pass counter; the rest are warp
// tasks, taken in chunks of consecutive tasks per warp from a second
// counter.  A group of 4 or 8:
//   1. streams the r-clique's incidence row (coalesced, q ids per s-clique),
//      gathers the q tau values of each s-clique and keeps
//      rho = min(...) in registers (Def. 4, step 1);
//   2. counts rho >= tau(R).  If at least tau(R) of them are, H = tau(R):
//      the preserve-tau early exit of Section 4.4, valid because the update
//      never raises tau (Thm. 1);
//   3. otherwise H lies in [count, tau(R)) and is found by binary search on
//      h over the register-resident rho values, testing
//      #{rho >= h} >= h (Def. 3).  No histogram, no sort.
// A warp or a CTA (longer rows) streams its row instead: one pass counts
// rho >= tau(R); if that fails, each further pass bins rho into at most 256
// shared-memory counters over the interval [lo, hi) that holds H, and the
// suffix sums at the bin edges cut the interval 256-fold, so H is exact after
// 1-2 more streaming passes whatever the row length.
// The paper's linear-time hashmap h-index (Section 4.4) is replaced by this
// tau-bounded count; both compute Def. 3 exactly.
//
// SND reads tau_p and writes tau (ping-pong buffers, no copy).  AND reads and
// writes one tau array in place; tau only decreases, so a stale read is a
// larger value and at worst delays a decrease by a pass.  With notification, an
// r-clique is evaluated only if its bit is set in the current frontier; when
// its tau drops to h it sets the next-frontier bit of every neighbour R' with
// h <= tau(R') (Alg. 3, the orange lines).  It does not re-activate itself.
//
// (2,3) uses the adjacency layout: incidence entries are the CSR slots of
// the other two edges, the gathers read a 16-bit copy of tau indexed by CSR
// slot, and the frontier has one bit per slot.  k_pass_otf is the same update
// with no stored incidence: it finds each edge's triangles again by
// intersecting adjacency lists on every pass.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "nd_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kThreads = 256;
#ifndef ND_WARP_UNROLL
#define ND_WARP_UNROLL 4  // streamed incidences in flight per lane (warp / CTA rows)
#endif
constexpr int kWarpUnroll = ND_WARP_UNROLL;
#ifndef ND_WARP_CHUNK
#define ND_WARP_CHUNK 16  // consecutive warp tasks per counter grab
#endif
constexpr int kWarpChunk = ND_WARP_CHUNK;
#ifndef ND_NOTIFY_UNROLL
#define ND_NOTIFY_UNROLL 4  // notification entries in flight per lane ((2,3))
#endif
constexpr int kNotifyUnroll = ND_NOTIFY_UNROLL;
#ifndef ND_FRONT_L1
#define ND_FRONT_L1 1  // 0: read the next frontier's words from L2 only
#endif

// a word of the next frontier, which this pass only sets bits in: read
// through L1, where a stale clear bit only costs a redundant, idempotent
// atomic (a set bit is never stale).  Measured against L2-only reads: the
// k-core AND of R-MAT scale 24 took 73.8 against 89.9 ms, where the frontier
// words of the hub vertices are read again and again; the truss and (3,4)
// AND did not change.
__device__ __forceinline__ uint32_t ld_front(const uint32_t* p) {
#if ND_FRONT_L1
    return __ldca(p);
#else
    return __ldcg(p);
#endif
}
#ifndef ND_CORE_AND_CTA_FIRST
#define ND_CORE_AND_CTA_FIRST 1  // (1,2) AND: the CTA rows (hub vertices) before the warp tasks
#endif
#ifndef ND_RHO_CACHE
#define ND_RHO_CACHE 1024  // rho values a warp keeps in shared memory for the search passes (0 = none)
#endif
constexpr int kRhoCache = ND_RHO_CACHE;

// Work of one pass: rows longer than the CTA threshold are taken one per
// block from a per-pass counter; all other rows form warp tasks that warps
// take in chunks from a second counter.

struct SweepParams {
    const int64_t* __restrict__ inc_ptr;
    const uint32_t* __restrict__ inc;
    const int32_t* tin;   // SND: tau of the previous pass; AND: same array as tout
    int32_t* tout;
    // gathers: a copy of tau in 16 bits saturated at 65535, exact for every
    // row with tau(R) <= 65535 (the row only looks at min(rho, tau(R))); a
    // row above that (a CTA row) gathers tin.  Indexed by CSR position for
    // (2,3), where an updated edge writes both of its entries (e_pos), and by
    // vertex for (1,2); (3,4) gathers tin.
    const uint16_t* gin;
    uint16_t* gout;
    const uint2* __restrict__ epos;
    const uint32_t* __restrict__ eid;  // CSR position -> edge id (notification)
    // (2,3) without a stored incidence: the graph and the edge endpoints
    const int64_t* __restrict__ rp;
    const int32_t* __restrict__ col;
    const int32_t* __restrict__ eu;
    const int32_t* __restrict__ ev;
    const nd_item* __restrict__ items;
    int64_t lo[ND_NB], hi[ND_NB];  // bucket ranges in items
    const uint32_t* cur;  // AND + notification: frontier read in this pass
    uint32_t* next;       // and the frontier written for the next pass
    const uint32_t* members;  // PartialAnd: only members are notified (null = everyone)
    // batches, SND and AND-nn: graph of every r-clique, the graphs that changed
    // in the previous pass (gact_in) and those changing in this one (gact_out);
    // null for a single graph
    const uint32_t* __restrict__ gid;
    const uint8_t* gact_in;
    uint8_t* gact_out;
    unsigned long long* ctr;         // this pass: [0] changed, [1] evaluated, [2] next CTA row,
                                     // [3] incidences of the evaluated rows, [4] next warp chunk
    const unsigned long long* prev;  // previous pass (null on the first)
};

// tau loads.  SND reads last pass's array through the read-only path.  AND
// reads the array it is updating with plain (L1-cacheable) loads: a value
// seen early or from another SM's stale line is never smaller than the true
// one, because tau only decreases, so it can only delay a decrease to a later
// pass (the writer notifies) or over-notify; every pass is a new launch, which
// starts from fresh caches.
template <bool RO>
__device__ __forceinline__ int32_t ld_tau(const int32_t* p) {
    if (RO) return __ldg(p);
    return *p;
}

template <bool RO>
__device__ __forceinline__ int32_t ld_tau(const uint16_t* p) {
    if (RO) return (int32_t)__ldg(p);
    return (int32_t)*p;
}

// rho(S,R) for the s-clique at incidence j: min of the other r-cliques' tau
// (for (2,3) the entries index the CSR-position copy of tau).
// SND reads each row once per pass, so its ids are loaded evict-first and do
// not push the gathered tau values out of L2.  AND re-reads the row of a
// changed r-clique to notify its neighbours, so its ids are cached normally.
template <bool RO>
__device__ __forceinline__ uint32_t ld_id(const uint32_t* p) {
    return RO ? __ldcs(p) : __ldg(p);
}

template <int Q, bool RO, typename T>
__device__ __forceinline__ int32_t rho_at(const uint32_t* __restrict__ inc, const T* tau, int64_t j) {
    if (Q == 1) {
        return ld_tau<RO>(tau + ld_id<RO>(inc + j));
    } else if (Q == 2) {
        const uint2* p = reinterpret_cast<const uint2*>(inc) + j;
        uint2 id = RO ? __ldcs(p) : __ldg(p);
        return min(ld_tau<RO>(tau + id.x), ld_tau<RO>(tau + id.y));
    } else {
        const uint32_t* p = inc + 3 * j;
        uint32_t a = ld_id<RO>(p), b = ld_id<RO>(p + 1), c = ld_id<RO>(p + 2);
        return min(min(ld_tau<RO>(tau + a), ld_tau<RO>(tau + b)), ld_tau<RO>(tau + c));
    }
}

// rho of incidence j, as a functor for the h-index routines below
template <int Q, bool RO, typename T>
struct Rho {
    const uint32_t* __restrict__ inc;
    const T* tau;
    __device__ __forceinline__ int32_t operator()(int64_t j) const { return rho_at<Q, RO>(inc, tau, j); }
};

// (2,3) rows with tau(R) > 65535 (so d_s > 65535, CTA rows): exact values,
// CSR position -> edge id -> tau
template <bool RO>
struct RhoExact2 {
    const uint32_t* __restrict__ inc;
    const uint32_t* __restrict__ eid;
    const int32_t* tau;
    __device__ __forceinline__ int32_t operator()(int64_t j) const {
        const uint2 id = __ldg(reinterpret_cast<const uint2*>(inc) + j);
        return min(ld_tau<RO>(tau + __ldg(eid + id.x)), ld_tau<RO>(tau + __ldg(eid + id.y)));
    }
};

constexpr int32_t kTau16Max = 65535;

// the gather of a row whose tau is at most 65535: the 16-bit copy for (1,2)
// and (2,3).  (3,4) gathers int32 tau directly: its rows are not ordered, and
// the 16-bit copy measured 3% slower there (Chung-Lu 100K (3,4) with planted
// cliques) against 6% faster for a scale-24 k-core.
template <int Q, bool RO>
__device__ __forceinline__ auto make_rho(const SweepParams& P) {
    if constexpr (Q == 3) return Rho<3, RO, int32_t>{P.inc, P.tin};
    else return Rho<Q, RO, uint16_t>{P.inc, P.gin};
}

// H({rho_j}) clipped to t, for one r-clique, by a group of G lanes; the row
// (at most G*C <= 1024 incidences, so t <= 1024) is held in registers as
// min(rho, t), two 16-bit values per register.
template <int G, int C, typename F>
__device__ __forceinline__ int32_t group_hindex(const cg::thread_block_tile<G>& g, const F& rho,
                                                int64_t jb, int64_t je, int32_t t) {
    static_assert(C % 2 == 0, "values are packed in pairs");
    const int lane = g.thread_rank();
    if (t <= 0) return 0;
    uint32_t pk[C / 2];
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < C; c += 2) {
        const int64_t j0 = jb + lane + (int64_t)c * G, j1 = j0 + G;
        const int32_t r0 = (j0 < je) ? rho(j0) : 0;
        const int32_t r1 = (j1 < je) ? rho(j1) : 0;
        cnt += (r0 >= t) + (r1 >= t);
        pk[c / 2] = (uint32_t)min(r0, t) | ((uint32_t)min(r1, t) << 16);
    }
    cnt = cg::reduce(g, cnt, cg::plus<int>());
    if (cnt >= t) return t;
    int lo = cnt, hi = t;  // #{rho >= lo} >= lo holds; at hi it fails
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        int c2 = 0;
#pragma unroll
        for (int c = 0; c < C / 2; ++c)
            c2 += ((int)(pk[c] & 0xffffu) >= mid) + ((int)(pk[c] >> 16) >= mid);
        c2 = cg::reduce(g, c2, cg::plus<int>());
        if (c2 >= mid) lo = mid; else hi = mid;
    }
    return lo;
}

// Bin selection of one k-ary search step, by one full warp.  bins[0..255]
// count rho in [lo + b*width, lo + (b+1)*width), bins[256] counts rho >= hi.
// #{rho >= lo + b*width} is the suffix sum from b; the answer H lies in
// [k, next edge) for the largest bin edge k whose suffix is >= k (bin 0
// always qualifies, because #{rho >= lo} >= lo).  Each lane owns 8 bins.
// P16: the counters are 16 bits, two to a word (bin b in word b/2), for
// rows of fewer than 65,536 entries; 129 words instead of 257.
template <bool P16>
__device__ __forceinline__ unsigned bin_count(const unsigned* bins, int b) {
    if constexpr (P16) return (bins[b >> 1] >> ((b & 1) << 4)) & 0xffffu;
    return bins[b];
}

template <bool P16>
__device__ __forceinline__ void select_bin(const unsigned* bins, int lo, int hi, int width, int nb,
                                           int* nlo, int* nhi) {
    const int lane = threadIdx.x & 31;
    unsigned own = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) own += bin_count<P16>(bins, 8 * lane + k);
    unsigned incl = own;  // inclusive prefix over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    int64_t run = (int64_t)bin_count<P16>(bins, 256) + (total - incl);  // rho at or above this lane's bins
    int best = -1;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const int b = 8 * lane + k;
        run += bin_count<P16>(bins, b);
        if (best < 0 && run >= (int64_t)lo + (int64_t)b * width) best = b;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, best >= 0);
    const int b = __shfl_sync(0xffffffffu, best, 31 - __clz(hit));
    *nlo = lo + b * width;
    const int e = (b + 1 < nb) ? lo + (b + 1) * width : hi;
    *nhi = e < hi ? e : hi;
}

template <bool P16>
__device__ __forceinline__ void kary_bin(unsigned* bins, int32_t r, int lo, int hi, int width) {
    if (r < lo) return;
    const int b = r >= hi ? 256 : (r - lo) / width;
    if constexpr (P16) atomicAdd(&bins[b >> 1], 1u << ((b & 1) << 4));
    else atomicAdd(&bins[b], 1u);
}

// words of one set of bins: 257 counters, packed or not
template <bool P16>
__device__ __forceinline__ int bin_words() { return P16 ? 129 : 257; }

// H({rho_j}) clipped to t by one warp, streaming the row: one pass counts
// rho >= t; if that fails, k-ary search with 256 shared-memory bins per
// streaming pass (at most 2 passes for t <= 65536).  The counting pass keeps
// min(rho, t) of the row's first ncache entries in `cache` (16 bits: a warp
// row has t <= d_s < 65536), so the search passes read them from shared
// memory instead of gathering them again; only entries past ncache are
// streamed again.
// P16: packed 16-bit bins, for rows of fewer than 65,536 entries
template <bool P16 = false, typename F>
__device__ __forceinline__ int32_t warp_hindex(const F& rho, int64_t jb, int64_t je, int32_t t, unsigned* bins,
                                               uint16_t* cache = nullptr, int ncache = 0) {
    const int lane = threadIdx.x & 31;
    if (t <= 0) return 0;
    int cnt = 0;
    if (!cache || t > 65535) ncache = 0;
    const int64_t jc = jb + ncache;  // entries [jb, jc) go to the cache
#pragma unroll kWarpUnroll
    for (int64_t j = jb + lane; j < je; j += 32) {
        const int32_t r = rho(j);
        cnt += (r >= t);
        if (j < jc) cache[j - jb] = (uint16_t)min(r, t);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (cnt >= t) return t;
    __syncwarp();  // the cache is complete
    int lo = cnt, hi = t;
    while (hi - lo > 1) {
        const int span = hi - lo;
        const int nb = span < 256 ? span : 256;
        const int width = (span + nb - 1) / nb;
        for (int i = lane; i < bin_words<P16>(); i += 32) bins[i] = 0;
        __syncwarp();
        for (int64_t j = jb + lane; j < jc && j < je; j += 32)
            kary_bin<P16>(bins, (int32_t)cache[j - jb], lo, hi, width);
        for (int64_t j = jc + lane; j < je; j += 32) kary_bin<P16>(bins, rho(j), lo, hi, width);
        __syncwarp();
        int nlo, nhi;
        select_bin<P16>(bins, lo, hi, width, nb, &nlo, &nhi);
        lo = nlo;
        hi = nhi;
        __syncwarp();
    }
    return lo;
}

// The same by the whole CTA (the longest rows); warp 0 selects the bin.
// The first ncache entries are kept in `cache` as for a warp.
template <typename F>
__device__ __forceinline__ int32_t cta_hindex(const F& rho, int64_t jb, int64_t je, int32_t t,
                                              unsigned* bins /* 257 */, int* bounds /* 2 */,
                                              uint16_t* cache = nullptr, int ncache = 0) {
    if (t <= 0) return 0;
    int cnt = 0;
    if (!cache || t > 65535) ncache = 0;
    const int64_t jc = jb + ncache;
#pragma unroll kWarpUnroll
    for (int64_t j = jb + threadIdx.x; j < je; j += kThreads) {
        const int32_t r = rho(j);
        cnt += (r >= t);
        if (j < jc) cache[j - jb] = (uint16_t)min(r, t);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) bins[threadIdx.x >> 5] = (unsigned)cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int w = 0; w < kThreads / 32; ++w) tot += bins[w];
        bounds[0] = (int)tot;
    }
    __syncthreads();
    cnt = bounds[0];
    __syncthreads();
    if (cnt >= t) return t;
    int lo = cnt, hi = t;  // #{rho >= lo} >= lo holds; at hi it fails
    while (hi - lo > 1) {
        const int span = hi - lo;
        const int nb = span < 256 ? span : 256;
        const int width = (span + nb - 1) / nb;
        for (int i = threadIdx.x; i <= 256; i += kThreads) bins[i] = 0;
        __syncthreads();
        for (int64_t j = jb + threadIdx.x; j < jc && j < je; j += kThreads)
            kary_bin<false>(bins, (int32_t)cache[j - jb], lo, hi, width);
        for (int64_t j = jc + threadIdx.x; j < je; j += kThreads)
            kary_bin<false>(bins, rho(j), lo, hi, width);
        __syncthreads();
        if (threadIdx.x < 32) {
            int nlo, nhi;
            select_bin<false>(bins, lo, hi, width, nb, &nlo, &nhi);
            if (threadIdx.x == 0) { bounds[0] = nlo; bounds[1] = nhi; }
        }
        __syncthreads();
        lo = bounds[0];
        hi = bounds[1];
        __syncthreads();
    }
    return lo;
}

// the new tau of R; (2,3) also writes it to both CSR entries of the edge
template <int Q>
__device__ __forceinline__ void store_tau(const SweepParams& P, uint32_t R, int32_t h) {
    P.tout[R] = h;
    const uint16_t v = (uint16_t)min(h, kTau16Max);
    if (Q == 2) {
        const uint2 ep = __ldg(P.epos + R);
        P.gout[ep.x] = v;
        P.gout[ep.y] = v;
    } else if (Q == 1) {
        P.gout[R] = v;
    }
}

// (2,3): notify the edge at CSR position pos, whose tau read from the
// 16-bit copy is tv, if h <= tau (the exact int32 value when h > 65535).
// The caller has just seen its frontier bit clear, with a relaxed L2 read:
// a bit set meanwhile only costs a redundant atomic, and a set bit is never
// cleared within a pass.
__device__ __forceinline__ void notify_clear(const SweepParams& P, uint32_t pos, int32_t h, int32_t tv) {
    if (h > kTau16Max) tv = ld_tau<false>(P.tin + __ldg(P.eid + pos));
    if (h > tv) return;
    if (P.members) {  // PartialAnd: members only
        const uint32_t Rp = __ldg(P.eid + pos);
        if (!((__ldg(P.members + (Rp >> 5)) >> (Rp & 31)) & 1u)) return;
    }
    atomicOr(P.next + (pos >> 5), 1u << (pos & 31));
}

// the same, testing the bit first and reading tau only if it is clear
__device__ __forceinline__ void notify_pos(const SweepParams& P, uint32_t pos, int32_t h) {
    if ((ld_front(P.next + (pos >> 5)) >> (pos & 31)) & 1u) return;
    notify_clear(P, pos, h, ld_tau<false>(P.gin + pos));
}

// is R in the current frontier?  (2,3): either bit of its two CSR positions
template <int Q>
__device__ __forceinline__ bool in_frontier(const SweepParams& P, uint32_t R) {
    if constexpr (Q == 2) {
        const uint2 ep = __ldg(P.epos + R);
        return ((__ldg(P.cur + (ep.x >> 5)) >> (ep.x & 31)) & 1u) | ((__ldg(P.cur + (ep.y >> 5)) >> (ep.y & 31)) & 1u);
    } else {
        return (__ldg(P.cur + (R >> 5)) >> (R & 31)) & 1u;
    }
}

// notify every neighbour whose tau could still depend on R (Alg. 3, orange
// lines): set its next-frontier bit if h <= tau(R').  A neighbour whose bit
// is already set needs nothing, so the bitmap word (2 MB for 16M r-cliques,
// cache-resident) is read before the neighbour's tau, and an atomic is only
// issued for a bit that is still clear.  (Warp-wide merging of bits that
// share a word was measured slower: the match runs for every neighbour,
// while most neighbours need no write.)
template <int Q>
__device__ __forceinline__ void notify_row(const SweepParams& P, int64_t jb, int64_t je, int32_t h,
                                           int first, int step) {
    if constexpr (Q == 2) {
        // (2,3): the entries are CSR positions; the frontier has one bit per
        // position, so the test reads the 16-bit copy and the bit sits next
        // to it (no edge id on this path).  kNotifyUnroll entries per lane
        // are loaded before any is tested, so their latencies overlap.
        const uint2* pairs = reinterpret_cast<const uint2*>(P.inc);
        for (int64_t j0 = jb + first; j0 < je; j0 += (int64_t)kNotifyUnroll * step) {
            uint2 id[kNotifyUnroll];
            uint32_t wx[kNotifyUnroll], wy[kNotifyUnroll];
#pragma unroll
            for (int u = 0; u < kNotifyUnroll; ++u) {
                const int64_t j = j0 + (int64_t)u * step;
                id[u] = j < je ? __ldg(pairs + j) : make_uint2(0u, 0u);
            }
            // the frontier words first: a neighbour whose bit is already set
            // needs neither its tau nor an atomic
#pragma unroll
            for (int u = 0; u < kNotifyUnroll; ++u) {
                const bool ok = j0 + (int64_t)u * step < je;
                wx[u] = ok ? ld_front(P.next + (id[u].x >> 5)) : 0xffffffffu;
                wy[u] = ok ? ld_front(P.next + (id[u].y >> 5)) : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < kNotifyUnroll; ++u) {
                if (!((wx[u] >> (id[u].x & 31)) & 1u)) notify_clear(P, id[u].x, h, ld_tau<false>(P.gin + id[u].x));
                if (!((wy[u] >> (id[u].y & 31)) & 1u)) notify_clear(P, id[u].y, h, ld_tau<false>(P.gin + id[u].y));
            }
        }
    } else {
        // (1,2), (3,4): ids of r-cliques; the same overlap, kNotifyUnroll
        // entries (Q ids each) and their bit words loaded before any test
        constexpr int U = Q == 1 ? kNotifyUnroll : 2;
        for (int64_t j0 = jb + first; j0 < je; j0 += (int64_t)U * step) {
            uint32_t id[U][Q], wd[U][Q];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t j = j0 + (int64_t)u * step;
#pragma unroll
                for (int k = 0; k < Q; ++k) id[u][k] = j < je ? __ldg(P.inc + Q * j + k) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = j0 + (int64_t)u * step < je;
#pragma unroll
                for (int k = 0; k < Q; ++k) wd[u][k] = ok ? ld_front(P.next + (id[u][k] >> 5)) : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const uint32_t Rp = id[u][k];
                    const uint32_t bit = 1u << (Rp & 31);
                    if (wd[u][k] & bit) continue;  // already active (or past the row's end)
                    if (P.members && !(__ldg(P.members + (Rp >> 5)) & bit)) continue;  // PartialAnd
                    if (h <= ld_tau<false>(P.tin + Rp)) atomicOr(P.next + (Rp >> 5), bit);
                }
            }
        }
    }
}

// notification for one incidence entry j of a row whose tau dropped to h:
// the same test as notify_row, for a single entry (the merged walk of group
// rows below gives each lane entries of different rows)
template <int Q>
__device__ __forceinline__ void notify_entry(const SweepParams& P, int64_t j, int32_t h) {
    if constexpr (Q == 2) {
        const uint2 id = __ldg(reinterpret_cast<const uint2*>(P.inc) + j);
        const uint32_t wx = ld_front(P.next + (id.x >> 5)), wy = ld_front(P.next + (id.y >> 5));
        if (!((wx >> (id.x & 31)) & 1u)) notify_clear(P, id.x, h, ld_tau<false>(P.gin + id.x));
        if (!((wy >> (id.y & 31)) & 1u)) notify_clear(P, id.y, h, ld_tau<false>(P.gin + id.y));
    } else {
        uint32_t id[Q], wd[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) id[k] = __ldg(P.inc + Q * j + k);
#pragma unroll
        for (int k = 0; k < Q; ++k) wd[k] = ld_front(P.next + (id[k] >> 5));
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const uint32_t Rp = id[k];
            const uint32_t bit = 1u << (Rp & 31);
            if (wd[k] & bit) continue;
            if (P.members && !(__ldg(P.members + (Rp >> 5)) & bit)) continue;  // PartialAnd
            if (h <= ld_tau<false>(P.tin + Rp)) atomicOr(P.next + (Rp >> 5), bit);
        }
    }
}

// batches (GB): has R's graph converged (no change in its previous pass)?
// Its rows then keep their tau, as the graph's own run would have stopped.
// The single-graph kernels (GB = false) carry no test at all.
template <bool GB>
__device__ __forceinline__ bool graph_done(const SweepParams& P, uint32_t R) {
    if constexpr (GB) return !P.gact_in[__ldg(P.gid + R)];
    return false;
}

// batches: R changed, so its graph is still changing
template <bool GB>
__device__ __forceinline__ void graph_changed(const SweepParams& P, uint32_t R) {
    if constexpr (GB) P.gact_out[__ldg(P.gid + R)] = 1;
}

__device__ __forceinline__ nd_item load_item(const nd_item* __restrict__ items, int64_t i) {
    longlong2 v = __ldg(reinterpret_cast<const longlong2*>(items) + i);
    nd_item it;
    it.jb = v.x;
    it.R = (uint32_t)(unsigned long long)v.y;
    it.d = (uint32_t)((unsigned long long)v.y >> 32);
    return it;
}

// work items [first, first + 32/G): one r-clique per group of G lanes of the
// calling warp
template <int Q, int G, int C, bool AND, bool NOTIFY, bool GB = false>
__device__ __forceinline__ void run_groups(const SweepParams& P, int64_t first, int64_t last,
                                           unsigned long long& changed, unsigned long long& evals,
                                           unsigned long long& incs) {
    auto g = cg::tiled_partition<G>(cg::this_thread_block());
    const int lane = g.thread_rank();
    // the group's index inside its warp, from the lane id (G divides 32)
    const int64_t i = first + (int64_t)((threadIdx.x & 31) / G);
    if (i >= last) return;
    const nd_item it = load_item(P.items, i);
    const uint32_t R = it.R;
    const int64_t jb = it.jb, je = it.jb + it.d;
    if (AND && NOTIFY && !in_frontier<Q>(P, R)) return;
    if (graph_done<GB>(P, R)) return;
    const int32_t t0 = ld_tau<!AND>(P.tin + R);
    // H <= d_s, so tau is clipped at d_s for the search (a no-op for every
    // valid tau, which is <= d_s); changes are detected against the stored value
    const int32_t t = min(t0, (int32_t)it.d);
    const int32_t h = group_hindex<G, C>(g, make_rho<Q, !AND>(P), jb, je, t);
    if (lane == 0) {
        evals++;
        incs += it.d;
        if (h != t0) {
            changed++;
            graph_changed<GB>(P, R);
        }
        if (!AND || h != t0) store_tau<Q>(P, R, h);
    }
    if (AND && NOTIFY && h != t0) notify_row<Q>(P, jb, je, h, lane, G);
}

// one r-clique per warp (rows of the warp bucket), streamed.  CHECK: test
// the frontier here (false when the caller has already selected active rows)
template <int Q, bool AND, bool NOTIFY, bool CHECK = true, bool GB = false, bool PK = true>
__device__ __forceinline__ void run_warp_row(const SweepParams& P, const nd_item& it, unsigned* bins,
                                             uint16_t* cache, unsigned long long& changed, unsigned long long& evals,
                                             unsigned long long& incs) {
    const int lane = threadIdx.x & 31;
    const uint32_t R = it.R;
    if (CHECK && AND && NOTIFY && !in_frontier<Q>(P, R)) return;
    if (graph_done<GB>(P, R)) return;
    const int32_t t0 = ld_tau<!AND>(P.tin + R);
    // H <= d_s, so tau is clipped at d_s for the search (a no-op for every
    // valid tau, which is <= d_s); changes are detected against the stored value
    const int32_t t = min(t0, (int32_t)it.d);
    const int64_t jb = it.jb, je = it.jb + it.d;
    // a warp row has d_s <= the warp threshold (at most 8,192), so 16-bit bins hold its counts
    const int32_t h = warp_hindex<PK>(make_rho<Q, !AND>(P), jb, je, t, bins, cache, kRhoCache);
    if (lane == 0) {
        evals++;
        incs += it.d;
        if (h != t0) {
            changed++;
            graph_changed<GB>(P, R);
        }
        if (!AND || h != t0) store_tau<Q>(P, R, h);
    }
    if (AND && NOTIFY && h != t0) notify_row<Q>(P, jb, je, h, lane, 32);
}

// one r-clique per CTA (rows longer than 2048 incidences)
template <int Q, bool AND, bool NOTIFY, bool GB = false>
__device__ __forceinline__ void run_cta(const SweepParams& P, int64_t first, int64_t last,
                                        unsigned* bins, int* bounds, uint16_t* cache, int ncache,
                                        unsigned long long& changed,
                                        unsigned long long& evals, unsigned long long& incs) {
    for (int64_t i = first; i < last; ++i) {
        const nd_item it = load_item(P.items, i);
        const uint32_t R = it.R;
        if (AND && NOTIFY && !in_frontier<Q>(P, R)) continue;
        if (graph_done<GB>(P, R)) continue;  // the same R for the whole block
        const int32_t t0 = ld_tau<!AND>(P.tin + R);
        // H <= d_s, so tau is clipped at d_s for the search (a no-op for every
        // valid tau, which is <= d_s); changes are detected against the stored value
        const int32_t t = min(t0, (int32_t)it.d);
        const int64_t jb = it.jb, je = it.jb + it.d;
        int32_t h;
        if (Q == 2 && t > kTau16Max)  // only then can a saturated value matter
            h = cta_hindex(RhoExact2<!AND>{P.inc, P.eid, P.tin}, jb, je, t, bins, bounds);
        else if (Q == 1 && t > kTau16Max)
            h = cta_hindex(Rho<Q, !AND, int32_t>{P.inc, P.tin}, jb, je, t, bins, bounds);
        else
            h = cta_hindex(make_rho<Q, !AND>(P), jb, je, t, bins, bounds, cache, ncache);
        if (threadIdx.x == 0) {
            evals++;
            incs += it.d;
            if (h != t0) {
                changed++;
                graph_changed<GB>(P, R);
            }
            if (!AND || h != t0) store_tau<Q>(P, R, h);
        }
        if (AND && NOTIFY && h != t0) notify_row<Q>(P, jb, je, h, threadIdx.x, kThreads);
        __syncthreads();
    }
}

// AND with notification: the frontier bits of the rows [a, b) of a warp
// chunk (at most 32 * W rows), tested by all lanes at once (one row per lane
// per word, every load issued before any test) and returned as W ballots.
template <int Q, int W>
__device__ __forceinline__ void active_masks(const SweepParams& P, int64_t a, int64_t b, unsigned (&mask)[W]) {
    const int lane = threadIdx.x & 31;
    uint32_t R[W];
    bool ok[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int64_t i = a + (int64_t)w * 32 + lane;
        ok[w] = i < b;
        R[w] = ok[w] ? __ldg(reinterpret_cast<const uint32_t*>(P.items + i) + 2) : 0u;  // nd_item::R
    }
    if constexpr (Q == 2) {
        uint2 ep[W];
#pragma unroll
        for (int w = 0; w < W; ++w) ep[w] = ok[w] ? __ldg(P.epos + R[w]) : make_uint2(0u, 0u);
        uint32_t bx[W], by[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            bx[w] = __ldg(P.cur + (ep[w].x >> 5));
            by[w] = __ldg(P.cur + (ep[w].y >> 5));
        }
#pragma unroll
        for (int w = 0; w < W; ++w)
            mask[w] = __ballot_sync(0xffffffffu, ok[w] && (((bx[w] >> (ep[w].x & 31)) | (by[w] >> (ep[w].y & 31))) & 1u));
    } else {
        uint32_t bw[W];
#pragma unroll
        for (int w = 0; w < W; ++w) bw[w] = __ldg(P.cur + (R[w] >> 5));
#pragma unroll
        for (int w = 0; w < W; ++w) mask[w] = __ballot_sync(0xffffffffu, ok[w] && ((bw[w] >> (R[w] & 31)) & 1u));
    }
}

// position of the k-th (0-based) set bit of m, for k < popc(m): halves by popcount
__device__ __forceinline__ int nth_set_bit(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const unsigned low = m & ((1u << w) - 1u);
        const int c = __popc(low);
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        } else {
            m = low;
        }
    }
    return pos;
}

// AND with notification, group rows: the active rows among the 32 rows
// a + {bits of mask}, packed densely onto the 32/G groups of the warp (no
// group idles on an inactive row).  After each round the entries of every
// row that changed are walked by all 32 lanes together (the merged
// notification), instead of by each row's own G lanes while the groups whose
// rows did not change wait.
template <int Q, int G, int C>
__device__ __forceinline__ void run_groups_active(const SweepParams& P, int64_t a, unsigned mask,
                                                  unsigned long long& changed, unsigned long long& evals,
                                                  unsigned long long& incs) {
    constexpr int NG = 32 / G;
    auto g = cg::tiled_partition<G>(cg::this_thread_block());
    const int lane = threadIdx.x & 31;
    const int grp = lane / G;
    const int cnt = __popc(mask);
    for (int base = 0; base < cnt; base += NG) {
        const int k = base + grp;  // this group's k-th active row
        int64_t jb = 0;
        int32_t h = 0, dn = 0;
        if (k < cnt) {  // uniform inside the group
            const int64_t i = a + nth_set_bit(mask, k);
            const nd_item it = load_item(P.items, i);
            const int32_t t0 = ld_tau<false>(P.tin + it.R);
            const int32_t t = min(t0, (int32_t)it.d);
            jb = it.jb;
            h = group_hindex<G, C>(g, make_rho<Q, false>(P), jb, jb + it.d, t);
            if (g.thread_rank() == 0) {
                evals++;
                incs += it.d;
                if (h != t0) {
                    changed++;
                    store_tau<Q>(P, it.R, h);
                }
            }
            dn = (h != t0) ? (int32_t)it.d : 0;
        }
        // merged notification over the changed rows of this round
        int tot = 0;
#pragma unroll
        for (int q = 0; q < NG; ++q) tot += __shfl_sync(0xffffffffu, dn, q * G);
        for (int e0 = 0; e0 < tot; e0 += 32) {
            const int e = e0 + lane;
            int64_t j = 0;
            int32_t hh = 0;
            int run = 0;
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                const int v = __shfl_sync(0xffffffffu, dn, q * G);
                const int64_t jq = __shfl_sync(0xffffffffu, jb, q * G);
                const int32_t hq = __shfl_sync(0xffffffffu, h, q * G);
                if (e >= run && e < run + v) { j = jq + (e - run); hh = hq; }
                run += v;
            }
            if (e < tot) notify_entry<Q>(P, j, hh);
        }
    }
}

#ifndef ND_PASS_MIN_BLOCKS
#define ND_PASS_MIN_BLOCKS 6  // resident blocks per SM the register budget targets (6 measured best)
#endif
#ifndef ND_PACKED_BINS_Q2
#define ND_PACKED_BINS_Q2 0  // (2,3) passes with the packed bins too (measured slower on the R-MAT k-truss)
#endif
#ifndef ND_CARVEOUT_FN0
#define ND_CARVEOUT_FN0 1  // request the carve-out for the first batch's kernel too
#endif
#ifndef ND_NC_CARVEOUT
#define ND_NC_CARVEOUT 1  // the late-pass kernel asks for the carve-out it needs (0: the driver's choice)
#endif
#ifndef ND_NC_MIN_BLOCKS
#define ND_NC_MIN_BLOCKS 6  // the late-pass kernel without the rho cache
#endif
#ifndef ND_AND_MIN_BLOCKS
#define ND_AND_MIN_BLOCKS 6   // the same for the AND pass with notification
#endif
// GB: a batch handle's SND / AND-nn pass, which skips the rows of graphs
// that have converged
// NC: no rho cache, for the late passes of a run, where few rows search:
// without its 16 KB per block the SM keeps more of its memory as L1 for the
// gathers
template <int Q, bool AND, bool NOTIFY, bool GB = false, bool NC = false>
__global__ void __launch_bounds__(kThreads, NC ? ND_NC_MIN_BLOCKS
                                               : ((AND && NOTIFY) ? ND_AND_MIN_BLOCKS : ND_PASS_MIN_BLOCKS))
    k_pass(SweepParams P) {
    if (P.prev != nullptr && *(volatile const unsigned long long*)P.prev == 0ull) return;  // converged
    constexpr int kRC = NC ? 0 : kRhoCache;
    // k-ary search bins.  (1,2) and (3,4): one packed set per warp (16-bit
    // counters), and a 32-bit set for the CTA rows in the last 1,040 bytes of
    // the block's rho cache, which a CTA row then does not use for values;
    // that keeps six blocks within a 132 KB shared-memory carve-out, and the
    // rest of the SM's memory serves as L1 (R-MAT scale-26 k-core: 794 against
    // 825 ms per step; Chung-Lu 100K (3,4): 121.9 against 126.8 ms).  (2,3): one
    // 32-bit set per warp, the CTA rows using warp 0's (the packed layout
    // measured 262.8 against 258.9 ms per step on the R-MAT scale-20 k-truss).
    // PK: packed warp bins and the CTA bins in the cache (ND_PACKED_BINS_Q2
    // selects it for (2,3))
    constexpr bool PK = Q != 2 || ND_PACKED_BINS_Q2;
    constexpr int kCtaBinWords = 260;
    constexpr int kCtaCache = kRC > 0 ? (kThreads / 32) * kRC - (PK ? 2 * kCtaBinWords : 0) : 0;
    static_assert(kRC == 0 || kCtaCache > 0, "the rho cache holds the CTA bins");
    __shared__ unsigned bins[kThreads / 32][PK ? 132 : 260];
    __shared__ __align__(16) uint16_t rho_cache[kThreads / 32][kRC > 0 ? kRC : 1];  // per warp; a CTA row uses all
    __shared__ unsigned cta_bins_own[(kRC > 0 && PK) ? 1 : kCtaBinWords];
    uint16_t* const wcache = kRC > 0 ? rho_cache[threadIdx.x >> 5] : nullptr;
    uint16_t* const bcache = kRC > 0 ? &rho_cache[0][0] : nullptr;
    unsigned* const cta_bins =
        (kRC > 0 && PK) ? reinterpret_cast<unsigned*>(&rho_cache[0][0] + kCtaCache) : (PK ? cta_bins_own : bins[0]);
    __shared__ int bounds[2];
    __shared__ unsigned long long s_chunk;
    unsigned long long changed = 0, evals = 0, incs = 0;
    // phase 1: rows longer than the CTA threshold, one per block at a time,
    // taken from a per-pass counter (longest rows first)
    const int64_t n3 = P.hi[3] - P.lo[3];
    auto cta_phase = [&]() {
        if (n3 <= 0) return;
        for (;;) {
            if (threadIdx.x == 0) s_chunk = atomicAdd(P.ctr + 2, 1ull);
            __syncthreads();
            const int64_t c = (int64_t)s_chunk;
            __syncthreads();
            if (c >= n3) break;
            run_cta<Q, AND, NOTIFY, GB>(P, P.lo[3] + c, P.lo[3] + c + 1, cta_bins, bounds, bcache, kCtaCache,
                                        changed, evals, incs);
        }
    };
    // AND updates in place, so a row evaluated later in a pass already sees
    // what earlier rows lowered: AND takes the shortest rows first and the
    // CTA rows last (measured 3% faster than longest first on R-MAT scale 20
    // k-truss).  SND, whose pass reads only the previous pass, takes the
    // longest rows first, for balance.  A k-core's CTA rows are the hub
    // vertices, up to hundreds of thousands of entries each, and one block
    // streams a row: taken last, they kept a few blocks busy long after the
    // rest of the pass had finished (18% of the AND time of an R-MAT scale
    // 26 k-core in ncu), so (1,2) AND takes them first.
    constexpr bool kShortFirst = AND;
    constexpr bool kCtaFirst = !AND || (Q == 1 && ND_CORE_AND_CTA_FIRST);
    if (kCtaFirst) cta_phase();
    // phase 2: warp tasks (one warp row, four 8-lane rows or eight 4-lane
    // rows), longest first (SND) or shortest first (AND).  Each warp takes
    // chunks of kWarpChunk
    // consecutive tasks from a per-pass counter (one atomic per chunk, no
    // barrier): consecutive r-cliques share a vertex and gather from the
    // same part of tau, and dynamic chunks keep the warps balanced even when
    // only a scattered subset of r-cliques is active (AND).
    const int64_t n2 = P.hi[2] - P.lo[2];
    const int64_t t1 = (P.hi[1] - P.lo[1] + 3) / 4;
    const int64_t t0 = (P.hi[0] - P.lo[0] + 7) / 8;
    const int64_t tasks = n2 + t1 + t0;
    const int lane32 = threadIdx.x & 31;
    for (;;) {
        unsigned long long c = 0;
        if (lane32 == 0) c = atomicAdd(P.ctr + 4, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        const int64_t nchunks = (tasks + kWarpChunk - 1) / kWarpChunk;
        if ((int64_t)c >= nchunks) break;
        const int64_t cc = kShortFirst ? nchunks - 1 - (int64_t)c : (int64_t)c;
        int64_t t = cc * kWarpChunk;
        const int64_t te = min(t + (int64_t)kWarpChunk, tasks);
        if constexpr (AND && NOTIFY) {
            // the chunk's rows per bucket, their frontier bits tested up front;
            // only active rows are evaluated
            static_assert(kWarpChunk <= 32, "one mask word of warp rows per chunk");
            const int64_t w_hi = min(te, n2);
            if (t < w_hi) {
                unsigned m2[1];
                active_masks<Q, 1>(P, P.lo[2] + t, P.lo[2] + w_hi, m2);
                unsigned mm = m2[0];
                while (mm) {
                    const int b = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const nd_item it = load_item(P.items, P.lo[2] + t + b);
                    run_warp_row<Q, AND, NOTIFY, false, false, PK>(P, it, bins[threadIdx.x >> 5], wcache, changed,
                                                                   evals, incs);
                }
            }
            const int64_t t1_lo = max(t, n2), t1_hi = min(te, n2 + t1);
            if (t1_lo < t1_hi) {
                constexpr int W1 = (kWarpChunk * 4 + 31) / 32;
                const int64_t a = P.lo[1] + 4 * (t1_lo - n2), b = min(P.lo[1] + 4 * (t1_hi - n2), P.hi[1]);
                unsigned mk[W1];
                active_masks<Q, W1>(P, a, b, mk);
#pragma unroll
                for (int w = 0; w < W1; ++w)
                    if (mk[w]) run_groups_active<Q, 8, 8>(P, a + 32 * w, mk[w], changed, evals, incs);
            }
            const int64_t t0_lo = max(t, n2 + t1);
            if (t0_lo < te) {
                constexpr int W0 = (kWarpChunk * 8 + 31) / 32;
                const int64_t a = P.lo[0] + 8 * (t0_lo - n2 - t1), b = min(P.lo[0] + 8 * (te - n2 - t1), P.hi[0]);
                unsigned mk[W0];
                active_masks<Q, W0>(P, a, b, mk);
#pragma unroll
                for (int w = 0; w < W0; ++w)
                    if (mk[w]) run_groups_active<Q, 4, 2>(P, a + 32 * w, mk[w], changed, evals, incs);
            }
            continue;
        }
        const int64_t e2 = min(te, n2);
        if (t < e2) {
            // warp rows: the next row's work item is loaded before this one runs
            nd_item it = load_item(P.items, P.lo[2] + t);
            while (t < e2) {
                nd_item nx;
                if (t + 1 < e2) nx = load_item(P.items, P.lo[2] + t + 1);
                run_warp_row<Q, AND, NOTIFY, true, GB, PK>(P, it, bins[threadIdx.x >> 5], wcache, changed, evals,
                                                           incs);
                it = nx;
                ++t;
            }
        }
        for (; t < te; ++t) {
            if (t < n2 + t1) {
                const int64_t first = P.lo[1] + 4 * (t - n2);
                run_groups<Q, 8, 8, AND, NOTIFY, GB>(P, first, min(first + 4, P.hi[1]), changed, evals, incs);
            } else {
                const int64_t first = P.lo[0] + 8 * (t - n2 - t1);
                run_groups<Q, 4, 2, AND, NOTIFY, GB>(P, first, min(first + 8, P.hi[0]), changed, evals, incs);
            }
        }
    }
    if (!kCtaFirst) cta_phase();
    __shared__ unsigned long long s_ch[kThreads / 32], s_ev[kThreads / 32], s_in[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_xor_sync(0xffffffffu, changed, o);
        evals += __shfl_xor_sync(0xffffffffu, evals, o);
        incs += __shfl_xor_sync(0xffffffffu, incs, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { s_ch[wid] = changed; s_ev[wid] = evals; s_in[wid] = incs; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, e = 0, c = 0;
        for (int w = 0; w < kThreads / 32; ++w) { a += s_ch[w]; e += s_ev[w]; c += s_in[w]; }
        if (a) atomicAdd(P.ctr, a);
        if (e) atomicAdd(P.ctr + 1, e);
        if (c) atomicAdd(P.ctr + 3, c);
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

// tau -> its CSR-position copies: both entries of every edge
__global__ void k_tau_to_adj(int64_t N, const uint2* __restrict__ epos, const int32_t* __restrict__ tau,
                             uint16_t* __restrict__ a, uint16_t* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 ep = epos[i];
        const uint16_t v = (uint16_t)min(max(tau[i], 0), kTau16Max);
        a[ep.x] = v;
        a[ep.y] = v;
        if (b) {
            b[ep.x] = v;
            b[ep.y] = v;
        }
    }
}

// tau -> its 16-bit gather copies indexed by r-clique id ((1,2), (3,4))
__global__ void k_tau_to_16(int64_t N, const int32_t* __restrict__ tau, uint16_t* __restrict__ a,
                            uint16_t* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t v = (uint16_t)min(max(tau[i], 0), kTau16Max);
        a[i] = v;
        if (b) b[i] = v;
    }
}

// PartialAnd with the (2,3) layout: both CSR positions of every member
__global__ void k_member_pos(int64_t N, const uint32_t* __restrict__ members, const uint2* __restrict__ epos,
                             uint32_t* __restrict__ f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!((members[i >> 5] >> (i & 31)) & 1u)) continue;
        const uint2 ep = epos[i];
        atomicOr(f + (ep.x >> 5), 1u << (ep.x & 31));
        atomicOr(f + (ep.y >> 5), 1u << (ep.y & 31));
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

__global__ void k_member_mask(const uint32_t* __restrict__ ids, int64_t count, int64_t N,
                              uint32_t* __restrict__ mask, int* __restrict__ err, const int32_t* __restrict__ to_new) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t R = ids[i];
        if ((int64_t)R >= N) { atomicOr(err, 1); continue; }
        if (to_new) R = (uint32_t)to_new[R];  // relabelled (1,2) handle
        atomicOr(mask + (R >> 5), 1u << (R & 31));
    }
}

__global__ void k_count_equal(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t n,
                              unsigned long long* __restrict__ out) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (a[i] == b[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_add_const(const int32_t* __restrict__ in, int64_t n, int32_t c, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] + c;
}

// ---- (2,3) without a stored incidence ----------------------------------------
// The paper's own mode (its s-cliques are not stored but found again on every
// pass, Section 4.1 "Time complexity" and Section 5): for row R = edge (x,y)
// the triangles are the w in both N(x) and N(y).  Its entries are indexed by
// the slots of the shorter list N(s): entry j is w = N(s)[j], present if w is
// in the longer list N(l) (binary search).  A present entry has
// rho = min(tau at P(s,w), tau at P(l,w)), two slots of the CSR-position copy
// (the same slots the stored layout lists); a missing one returns -1, which
// no h-index step counts (every bound is >= 0).  One warp per row, longest
// rows first, in chunks from a counter.
template <bool RO, bool EXACT>
struct RhoOtf {
    const int32_t* __restrict__ col;
    int64_t sb, lb;  // first slots of N(s) and N(l)
    int ln;          // |N(l)|
    const uint16_t* tau16;
    const uint32_t* __restrict__ eid;
    const int32_t* tau32;
    __device__ __forceinline__ int32_t operator()(int64_t j) const {
        const int32_t w = __ldg(col + sb + j);
        const int k = nd_lower_bound_n(col + lb, ln, w);
        if (k >= ln || __ldg(col + lb + k) != w) return -1;
        const int64_t ps = sb + j, pl = lb + k;
        if (EXACT) return min(ld_tau<RO>(tau32 + __ldg(eid + ps)), ld_tau<RO>(tau32 + __ldg(eid + pl)));
        return min(ld_tau<RO>(tau16 + ps), ld_tau<RO>(tau16 + pl));
    }
};

constexpr int kOtfChunk = 4;  // rows per counter grab

template <bool AND, bool NOTIFY>
__global__ void __launch_bounds__(kThreads, ND_PASS_MIN_BLOCKS) k_pass_otf(SweepParams P) {
    if (P.prev != nullptr && *(volatile const unsigned long long*)P.prev == 0ull) return;  // converged
    __shared__ unsigned bins[kThreads / 32][260];
    unsigned long long changed = 0, evals = 0, incs = 0;
    const int lane = threadIdx.x & 31;
    unsigned* wb = bins[threadIdx.x >> 5];
    const int64_t first = P.lo[0], rows = P.hi[ND_NB - 1] - P.lo[0];
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(P.ctr + 4, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        const int64_t t0 = (int64_t)c * kOtfChunk;
        if (t0 >= rows) break;
        const int64_t t1 = min(t0 + (int64_t)kOtfChunk, rows);
        for (int64_t t = t0; t < t1; ++t) {
            const nd_item it = load_item(P.items, first + rows - 1 - t);  // longest first
            const uint32_t R = it.R;
            if (AND && NOTIFY && !in_frontier<2>(P, R)) continue;
            const int32_t tr = ld_tau<!AND>(P.tin + R);
            const int32_t tc = min(tr, (int32_t)it.d);
            const int32_t x = __ldg(P.eu + R), y = __ldg(P.ev + R);
            const int64_t xb = __ldg(P.rp + x), xe = __ldg(P.rp + x + 1);
            const int64_t yb = __ldg(P.rp + y), ye = __ldg(P.rp + y + 1);
            const bool xs = (xe - xb) <= (ye - yb);
            const int64_t sb = xs ? xb : yb, se = xs ? xe : ye;
            const int64_t lb = xs ? yb : xb, le = xs ? ye : xe;
            int32_t h;
            if (tc > kTau16Max)
                h = warp_hindex(RhoOtf<!AND, true>{P.col, sb, lb, (int)(le - lb), P.gin, P.eid, P.tin}, 0, se - sb,
                                tc, wb);
            else
                h = warp_hindex(RhoOtf<!AND, false>{P.col, sb, lb, (int)(le - lb), P.gin, P.eid, P.tin}, 0, se - sb,
                                tc, wb);
            if (lane == 0) {
                evals++;
                incs += it.d;
                if (h != tr) changed++;
                if (!AND || h != tr) store_tau<2>(P, R, h);
            }
            if (AND && NOTIFY && h != tr) {
                // notify the other two edges of every triangle, found again
                for (int64_t j = lane; j < se - sb; j += 32) {
                    const int32_t w = __ldg(P.col + sb + j);
                    const int k = nd_lower_bound_n(P.col + lb, (int)(le - lb), w);
                    if (k >= (int)(le - lb) || __ldg(P.col + lb + k) != w) continue;
                    const uint32_t ps = (uint32_t)(sb + j), pl = (uint32_t)(lb + k);
                    notify_pos(P, ps, h);
                    notify_pos(P, pl, h);
                }
            }
        }
    }
    __shared__ unsigned long long s_ch[kThreads / 32], s_ev[kThreads / 32], s_in[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_xor_sync(0xffffffffu, changed, o);
        evals += __shfl_xor_sync(0xffffffffu, evals, o);
        incs += __shfl_xor_sync(0xffffffffu, incs, o);
    }
    const int wid = threadIdx.x >> 5;
    if (lane == 0) { s_ch[wid] = changed; s_ev[wid] = evals; s_in[wid] = incs; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, e = 0, c2 = 0;
        for (int w = 0; w < kThreads / 32; ++w) { a += s_ch[w]; e += s_ev[w]; c2 += s_in[w]; }
        if (a) atomicAdd(P.ctr, a);
        if (e) atomicAdd(P.ctr + 1, e);
        if (c2) atomicAdd(P.ctr + 3, c2);
    }
}

typedef void (*pass_fn)(SweepParams);

#ifndef ND_LATE_FROM
#define ND_LATE_FROM 16  // the first pass (0-based) of a run that takes the late-pass kernel
#endif
#ifndef ND_AND_LATE_FROM
#define ND_AND_LATE_FROM 16  // the same for AND with notification
#endif
static_assert(ND_LATE_FROM >= 0 && ND_LATE_FROM <= ND_BATCH, "the late kernel starts within the first batch");
static_assert(ND_AND_LATE_FROM >= 0 && ND_AND_LATE_FROM <= ND_BATCH, "the late kernel starts within the first batch");
#ifndef ND_LATE_NOCACHE
#define ND_LATE_NOCACHE 2  // passes after the first batch without the rho cache: 0 none, 1 SND, 2 SND and AND
#endif
pass_fn pick(const nd_incidence* h, int mode, bool late = false) {
    // mode: ND_SND, ND_AND (notify), ND_AND_NN
    const int q = h->q;
    if (late && !h->otf) {
        const bool gb = h->gid && mode != ND_AND;  // a batch's SND / AND-nn pass
        if (mode == ND_SND && ND_LATE_NOCACHE >= 1) {
            if (gb)
                return q == 1 ? k_pass<1, false, false, true, true>
                              : (q == 2 ? k_pass<2, false, false, true, true> : k_pass<3, false, false, true, true>);
            return q == 1 ? k_pass<1, false, false, false, true>
                          : (q == 2 ? k_pass<2, false, false, false, true> : k_pass<3, false, false, false, true>);
        }
        if (mode == ND_AND && ND_LATE_NOCACHE >= 2)
            return q == 1 ? k_pass<1, true, true, false, true>
                          : (q == 2 ? k_pass<2, true, true, false, true> : k_pass<3, true, true, false, true>);
        if (mode == ND_AND_NN && ND_LATE_NOCACHE >= 2) {
            if (gb)
                return q == 1 ? k_pass<1, true, false, true, true>
                              : (q == 2 ? k_pass<2, true, false, true, true> : k_pass<3, true, false, true, true>);
            return q == 1 ? k_pass<1, true, false, false, true>
                          : (q == 2 ? k_pass<2, true, false, false, true> : k_pass<3, true, false, false, true>);
        }
    }
    if (h->otf) return mode == ND_SND ? k_pass_otf<false, false> : (mode == ND_AND ? k_pass_otf<true, true> : k_pass_otf<true, false>);
    if (h->gid && mode != ND_AND) {  // a batch: converged graphs are skipped
        if (q == 1) return mode == ND_SND ? k_pass<1, false, false, true> : k_pass<1, true, false, true>;
        if (q == 2) return mode == ND_SND ? k_pass<2, false, false, true> : k_pass<2, true, false, true>;
        return mode == ND_SND ? k_pass<3, false, false, true> : k_pass<3, true, false, true>;
    }
    if (q == 1) return mode == ND_SND ? k_pass<1, false, false> : (mode == ND_AND ? k_pass<1, true, true> : k_pass<1, true, false>);
    if (q == 2) return mode == ND_SND ? k_pass<2, false, false> : (mode == ND_AND ? k_pass<2, true, true> : k_pass<2, true, false>);
    return mode == ND_SND ? k_pass<3, false, false> : (mode == ND_AND ? k_pass<3, true, true> : k_pass<3, true, false>);
}

// bucket ranges of a pass
void plan_buckets(const nd_incidence* h, SweepParams& P) {
    for (int b = 0; b < ND_NB; ++b) {
        P.lo[b] = h->bucket_lo[b];
        P.hi[b] = h->bucket_lo[b + 1];
    }
}

// work units of a pass: CTA rows + warp tasks (see k_pass); the grid never
// exceeds what the work needs
int64_t pass_units(const nd_incidence* h, const SweepParams& P) {
    if (h->otf) return P.hi[ND_NB - 1] - P.lo[0];  // one warp per row
    return (P.hi[3] - P.lo[3]) + (P.hi[2] - P.lo[2]) + (P.hi[1] - P.lo[1] + 3) / 4 + (P.hi[0] - P.lo[0] + 7) / 8;
}

// persistent grid: as many blocks as fit on the GPU at once (never more than
// the work needs)
int pass_grid(const nd_incidence* h, const void* fn, int64_t units) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t g = (int64_t)per_sm * (h->sm_count > 0 ? h->sm_count : 152);
    const int64_t need = (units + kThreads / 32 - 1) / (kThreads / 32);
    if (g > need) g = need;
    return (int)(g < 1 ? 1 : g);
}

nd_status ensure_state(nd_incidence* h, bool and_mode, cudaStream_t st) {
    const int64_t N = h->num_r > 0 ? h->num_r : 1;
    if (!h->tau[0]) ND_TRY(nd_alloc((void**)&h->tau[0], sizeof(int32_t) * N, st, h));
    if (!and_mode && !h->tau[1]) ND_TRY(nd_alloc((void**)&h->tau[1], sizeof(int32_t) * N, st, h));
    if (h->q != 3) {
        // 16-bit gather copies: one per CSR slot for (2,3), per vertex for (1,2)
        const int64_t E = h->adj ? (h->nnz > 0 ? h->nnz : 1) : N;
        if (!h->tg[0]) ND_TRY(nd_alloc((void**)&h->tg[0], sizeof(uint16_t) * E, st, h));
        if (!and_mode && !h->tg[1]) ND_TRY(nd_alloc((void**)&h->tg[1], sizeof(uint16_t) * E, st, h));
    }
    // (2,3): one frontier bit per CSR position (notification sets the bit of
    // the slot it has just read); otherwise one per r-clique
    const int64_t words = ((h->adj ? h->nnz : N) + 31) / 32;
    if (and_mode && !h->front[0]) {
        ND_TRY(nd_alloc((void**)&h->front[0], sizeof(uint32_t) * words, st, h));
        ND_TRY(nd_alloc((void**)&h->front[1], sizeof(uint32_t) * words, st, h));
    }
    if (!h->counters) {
        ND_TRY(nd_alloc((void**)&h->counters, sizeof(unsigned long long) * ND_SLOT * ND_RING, st, h));
        ND_CUDA(cudaMallocHost((void**)&h->h_counters, sizeof(unsigned long long) * ND_SLOT * ND_RING));
    }
    return ND_OK;
}


// the smallest shared-memory carve-out (percent of the SM's maximum) that
// holds the resident blocks of a pass kernel (all are built for 6 per SM)
nd_status request_carveout(const void* fn) {
    static_assert(ND_PASS_MIN_BLOCKS == 6 && ND_AND_MIN_BLOCKS == 6 && ND_NC_MIN_BLOCKS == 6,
                  "the carve-out is sized for six blocks per SM");
    cudaFuncAttributes fa;
    int dev = 0, max_sm = 0;
    ND_CUDA(cudaFuncGetAttributes(&fa, fn));
    ND_CUDA(cudaGetDevice(&dev));
    ND_CUDA(cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    if (max_sm <= 0) return ND_OK;
    const int64_t need = 6 * ((int64_t)fa.sharedSizeBytes + 1024);
    int pct = (int)((100 * need + max_sm - 1) / max_sm);  // rounded up to a supported carve-out
    if (pct > 100) pct = 100;
    ND_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    return ND_OK;
}

// parameters of one pass: its counter slot, the slot of the pass before it
// (-1: none), and the parity of its index in the run (SND reads tau[parity]
// and writes the other buffer; AND reads the frontier front[parity])
SweepParams pass_params(const nd_incidence* h, int mode, const SweepParams& P0, int slot, int prev_slot,
                        int parity) {
    SweepParams P = P0;
    P.ctr = h->counters + ND_SLOT * slot;
    P.prev = prev_slot < 0 ? nullptr : h->counters + ND_SLOT * prev_slot;
    if (P.gid) {
        P.gact_in = h->gact[parity];
        P.gact_out = h->gact[parity ^ 1];
    }
    if (mode != ND_SND) {
        P.tin = h->tau[0];
        P.tout = h->tau[0];
        P.gin = h->tg[0];
        P.gout = h->tg[0];
        P.cur = h->front[parity];
        P.next = h->front[parity ^ 1];
    } else {
        P.tin = h->tau[parity];
        P.tout = h->tau[parity ^ 1];
        P.gin = h->tg[parity];
        P.gout = h->tg[parity ^ 1];
        P.cur = nullptr;
        P.next = nullptr;
    }
    return P;
}

// A full batch of passes as one CUDA graph: clear the batch's counters, then
// for each pass (AND: clear the next frontier) the pass kernel, then copy
// the counters to the pinned host mirror.  Built explicitly (not by stream
// capture) so that it also serves the legacy default stream.  On any
// failure the handle falls back to ordinary launches for this kind.
void make_batch_graph(nd_incidence* h, int mode, int kind, const SweepParams& P0, int grid0, pass_fn fn0,
                      int grid1, pass_fn fn1, int late_from, int64_t words) {
    const int base = (kind == 2) ? ND_BATCH : 0;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphNode_t last = nullptr;
    if (ok) {
        cudaMemsetParams ms = {};
        ms.dst = h->counters + ND_SLOT * base;
        ms.value = 0;
        ms.elementSize = 4;
        ms.width = (size_t)ND_SLOT * ND_BATCH * 2;
        ms.height = 1;
        ok = cudaGraphAddMemsetNode(&last, g, nullptr, 0, &ms) == cudaSuccess;
    }
    for (int k = 0; ok && k < ND_BATCH; ++k) {
        // a batch starts at an even pass; its first pass reads the last slot
        // of the other half (the caller puts the previous pass's counters there)
        const int prev_slot = k > 0 ? base + k - 1 : (kind == 0 ? -1 : (base ^ ND_BATCH) + ND_BATCH - 1);
        SweepParams P = pass_params(h, mode, P0, base + k, prev_slot, k & 1);
        if (mode == ND_AND) {
            cudaMemsetParams ms = {};
            ms.dst = P.next;
            ms.value = 0;
            ms.elementSize = 4;
            ms.width = (size_t)words;
            ms.height = 1;
            cudaGraphNode_t n = nullptr;
            ok = cudaGraphAddMemsetNode(&n, g, &last, 1, &ms) == cudaSuccess;
            last = n;
        }
        if (ok && P.gid) {  // batches: the graphs changing in this pass, from none
            cudaMemsetParams ms = {};
            ms.dst = P.gact_out;
            ms.value = 0;
            ms.elementSize = 1;
            ms.width = (size_t)h->ngraphs;
            ms.height = 1;
            cudaGraphNode_t n = nullptr;
            ok = cudaGraphAddMemsetNode(&n, g, &last, 1, &ms) == cudaSuccess;
            last = n;
        }
        if (!ok) break;
        cudaKernelNodeParams kp = {};
        void* args[] = {&P};
        // passes from late_from on (in the run) take the late-pass kernel
        const bool late = (kind == 0 ? k : ND_BATCH + k) >= late_from;
        kp.func = (void*)(late ? fn1 : fn0);
        kp.gridDim = dim3(late ? grid1 : grid0);
        kp.blockDim = dim3(kThreads);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t n = nullptr;
        ok = cudaGraphAddKernelNode(&n, g, &last, 1, &kp) == cudaSuccess;
        last = n;
    }
    if (ok) {
        cudaGraphNode_t n = nullptr;
        ok = cudaGraphAddMemcpyNode1D(&n, g, &last, 1, h->h_counters + ND_SLOT * base, h->counters + ND_SLOT * base,
                                      sizeof(unsigned long long) * ND_SLOT * ND_BATCH,
                                      cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();  // clear, and use ordinary launches instead
        h->pass_graph_failed[mode][kind] = true;
        return;
    }
    h->pass_graph[mode][kind] = ex;
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

nd_status nd_member_mask(const uint32_t* ids, int64_t count, int64_t N, uint32_t* mask, int* err, cudaStream_t st,
                         const int32_t* to_new) {
    if (count == 0) return ND_OK;
    nd_prof_scope ps("member_mask", st);
    k_member_mask<<<nd_blocks_for(count, kThreads, 152 * 8), kThreads, 0, st>>>(ids, count, N, mask, err, to_new);
    ND_CUDA(cudaGetLastError());
    return ND_OK;
}

nd_status nd_count_equal_dev(const int32_t* a, const int32_t* b, int64_t n, unsigned long long* out_dev,
                             cudaStream_t st) {
    ND_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(unsigned long long), st));
    if (n == 0) return ND_OK;
    nd_prof_scope ps("count_equal", st);
    k_count_equal<<<nd_blocks_for(n, kThreads, 152 * 8), kThreads, 0, st>>>(a, b, n, out_dev);
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
                 cudaStream_t st, nd_run_opts* opts) {
    const uint32_t* members = (opts && mode != ND_SND) ? opts->members : nullptr;
    const double stop_active = (opts && mode != ND_SND) ? opts->stop_active : 0.0;
    if (opts) opts->stopped = false;
    const bool and_mode = (mode != ND_SND);
    const int64_t N = h->num_r;
    ND_TRY(ensure_state(h, and_mode, st));
    h->last_changed.clear();
    h->last_evals.clear();
    h->last_incs.clear();
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
        if (h->q != 3) {
            nd_prof_scope ps("init_tau", st);
            if (h->adj)
                k_tau_to_adj<<<blocks, kThreads, 0, st>>>(N, h->e_pos, h->tau[0], h->tg[0],
                                                          and_mode ? nullptr : h->tg[1]);
            else
                k_tau_to_16<<<blocks, kThreads, 0, st>>>(N, h->tau[0], h->tg[0], and_mode ? nullptr : h->tg[1]);
            ND_CUDA(cudaGetLastError());
        }
    }
    *tau_result = h->tau[0];
    if (N == 0 || max_passes <= 0) {
        *converged = (N == 0);
        return ND_OK;
    }
    const int64_t fbits = h->adj ? h->nnz : N;  // frontier bits (see ensure_state)
    const int64_t words = (fbits + 31) / 32;
    if (mode == ND_AND && members) {
        // PartialAnd: the members start active (end of Section 4.3)
        if (h->adj) {
            ND_CUDA(cudaMemsetAsync(h->front[0], 0, sizeof(uint32_t) * words, st));
            nd_prof_scope ps("fill_front", st);
            k_member_pos<<<blocks, kThreads, 0, st>>>(N, members, h->e_pos, h->front[0]);
            ND_CUDA(cudaGetLastError());
        } else {
            ND_CUDA(cudaMemcpyAsync(h->front[0], members, sizeof(uint32_t) * words, cudaMemcpyDeviceToDevice, st));
        }
    } else if (mode == ND_AND) {
        nd_prof_scope ps("fill_front", st);
        k_fill_front<<<nd_blocks_for(words, kThreads, h->sm_count * 8), kThreads, 0, st>>>(fbits, h->front[0]);
        ND_CUDA(cudaGetLastError());
    }
    SweepParams P;
    P.inc_ptr = h->inc_ptr;
    P.inc = h->inc;
    P.epos = h->e_pos;
    P.eid = h->eid;
    P.rp = h->rp;
    P.col = h->col;
    P.eu = h->e_u;
    P.ev = h->e_v;
    P.items = h->items;
    P.members = members;
    // batches, SND and AND-nn: every graph starts active (AND with
    // notification needs nothing more: a converged graph notifies no one)
    P.gid = nullptr;
    P.gact_in = nullptr;
    P.gact_out = nullptr;
    if (h->gid && mode != ND_AND) {
        for (int b = 0; b < 2; ++b)
            if (!h->gact[b]) ND_TRY(nd_alloc((void**)&h->gact[b], (size_t)h->ngraphs, st, h));
        ND_CUDA(cudaMemsetAsync(h->gact[0], 1, (size_t)h->ngraphs, st));
        P.gid = h->gid;
    }
    plan_buckets(h, P);
    // the first batch of passes, where rows still search, keeps the rho
    // cache; later batches may run a kernel without it
    pass_fn fn0 = pick(h, mode), fn1 = pick(h, mode, true);
    const int late_from = mode == ND_SND ? ND_LATE_FROM : ND_AND_LATE_FROM;
    // ask for a shared-memory carve-out that just holds each kernel's six
    // resident blocks (plus the 1 KB each block reserves), leaving the rest
    // of the SM's memory as L1 for the gathers.  Left to itself the driver
    // chose 132 KB for the late-pass kernel, where 64 KB suffice.
    if (ND_NC_CARVEOUT && !h->otf) {
        if (ND_CARVEOUT_FN0) ND_TRY(request_carveout((const void*)fn0));
        if (fn1 != fn0) ND_TRY(request_carveout((const void*)fn1));
    }
    const int64_t units = pass_units(h, P);
    const int grid0 = units > 0 ? pass_grid(h, (const void*)fn0, units) : 0;
    const int grid1 = units > 0 ? pass_grid(h, (const void*)fn1, units) : 0;
    const int kBatch = ND_BATCH;
    // Thm. 3 / Lemma 2: SND settles within the number of degree levels, at
    // most N_R, and AND never needs more passes than SND.  A run longer than
    // N_R + 1 passes (including the pass that detects convergence) can only
    // be a fault, and is reported instead of looping on.
    const int64_t bound = N + 1;
    bool over_bound = false;
    if ((int64_t)max_passes > bound) { max_passes = (int32_t)bound; over_bound = true; }
    const char* pname = mode == ND_SND ? "snd_pass" : (mode == ND_AND ? "and_pass" : "and_nn_pass");
    int32_t pass = 0;
    int64_t batch = 0;
    int last_slot = -1;  // counter slot of the last pass enqueued
    bool done = false;
    int32_t last_written = 0;  // SND: index of the buffer holding the newest tau
    while (!done && pass < max_passes) {
        // batch b uses counter slots [base, base + nb) of one half of the
        // ring; its first pass reads the counters of the pass enqueued before
        // it, and every pass takes its buffers by the parity of its index in
        // the run (batches of one pass, for the stopping rule, included)
        const int32_t start = pass;
        const int base = (int)(batch & 1) * kBatch;
        int nb = kBatch;
        if (nb > max_passes - pass) nb = max_passes - pass;
        if (stop_active > 0.0) nb = 1;  // the stopping rule looks at every pass
        const int kind = batch == 0 ? 0 : ((batch & 1) ? 2 : 1);
        bool launched = false;
        // graphs hold the plain parameters; runs with members or a stopping rule launch directly
        if (nb == kBatch && grid0 > 0 && !members && (start & 1) == 0 && !h->pass_graph_failed[mode][kind]) {
            if (!h->pass_graph[mode][kind])
                make_batch_graph(h, mode, kind, P, grid0, fn0, grid1, fn1, late_from, words);
            if (h->pass_graph[mode][kind]) {
                // the graph's first pass reads the last slot of the other half
                const int want = (base ^ ND_BATCH) + ND_BATCH - 1;
                if (kind != 0 && last_slot != want)
                    ND_CUDA(cudaMemcpyAsync(h->counters + ND_SLOT * want, h->counters + ND_SLOT * last_slot,
                                            sizeof(unsigned long long) * ND_SLOT, cudaMemcpyDeviceToDevice, st));
                nd_prof_scope ps(pname, st, kBatch);
                ND_CUDA(cudaGraphLaunch(h->pass_graph[mode][kind], st));
                launched = true;
                pass += kBatch;
            }
        }
        if (!launched) {
            ND_CUDA(cudaMemsetAsync(h->counters + ND_SLOT * base, 0, sizeof(unsigned long long) * ND_SLOT * nb, st));
            for (int k = 0; k < nb; ++k, ++pass) {
                SweepParams Pk = pass_params(h, mode, P, base + k, k > 0 ? base + k - 1 : last_slot, pass & 1);
                if (mode == ND_AND)
                    ND_CUDA(cudaMemsetAsync(Pk.next, 0, sizeof(uint32_t) * words, st));
                if (Pk.gid) ND_CUDA(cudaMemsetAsync(Pk.gact_out, 0, (size_t)h->ngraphs, st));
                if (grid0 > 0) {
                    const bool late = pass >= late_from;
                    nd_prof_scope ps(pname, st);
                    (late ? fn1 : fn0)<<<late ? grid1 : grid0, kThreads, 0, st>>>(Pk);
                    ND_CUDA(cudaGetLastError());
                }
            }
            ND_CUDA(cudaMemcpyAsync(h->h_counters + ND_SLOT * base, h->counters + ND_SLOT * base,
                                    sizeof(unsigned long long) * ND_SLOT * nb, cudaMemcpyDeviceToHost, st));
        }
        last_slot = base + nb - 1;
        ND_TRY(nd_wait(st));
        for (int k = 0; k < nb; ++k) {
            const int32_t p = start + k;
            unsigned long long ch = h->h_counters[ND_SLOT * (base + k)];
            unsigned long long ev = h->h_counters[ND_SLOT * (base + k) + 1];
            // r-cliques with d_s = 0 are never launched: tau = H(empty) = 0 = d_s.
            // They count as evaluated in every SND / AND-nn pass and in the first
            // AND pass, as in the paper's sequential loops (in a batch, whose
            // graphs stop at different passes, once per run).
            if ((mode != ND_AND && !h->gid) || p == 0) ev += (unsigned long long)h->num_zero;
            h->last_changed.push_back((int64_t)ch);
            h->last_evals.push_back((int64_t)ev);
            h->last_incs.push_back((int64_t)h->h_counters[ND_SLOT * (base + k) + 3]);
            *evals += (int64_t)ev;
            if (!and_mode) last_written = (p & 1) ^ 1;
            if (ch == 0) { done = true; break; }
            (*updating)++;
            // active-ratio rule (Section 5.2, Fig. 9): the fraction of r-cliques
            // evaluated in this pass predicts how close tau is to kappa
            const double active = (double)h->h_counters[ND_SLOT * (base + k) + 1] / (double)N;
            if (stop_active > 0.0 && active < stop_active) {
                opts->stopped = true;
                done = true;
                break;
            }
        }
        ++batch;
    }
    *converged = done && !(opts && opts->stopped);
    *tau_result = and_mode ? h->tau[0] : h->tau[last_written];
    if (!done && over_bound) {
        nd_set_error("no convergence within N_R + 1 passes, the bound of Thm. 3 (internal fault)");
        return ND_E_NOT_CONVERGED;
    }
    return ND_OK;
}
