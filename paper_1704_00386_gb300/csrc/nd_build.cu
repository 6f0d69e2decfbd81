// Incidence construction: r-clique -> s-clique incidence as CSR (Def. 1).
//
// The paper discovers the s-cliques of an r-clique through the
// neighbourhoods of its vertices (Section 4.1, "Time complexity": all
// (s-r)-tuples of a neighbourhood), and recomputes them on every pass.  Here
// they are found once, by sorted-list intersection, and stored:
//   (1,2)  the CSR itself is the incidence (q = 1), under ids ordered by
//          degree class for graphs of 65,536 vertices or more;
//   (2,3)  triangle {u,v,w} -> one pair per edge: the CSR slots of its other
//          two edges at the edge's endpoints (found once each, by degree
//          orientation), each row then ordered by the third vertex;
//   (3,4)  triangle (u,v,w): x in N(u) /\ N(v) /\ N(w) -> the ids of the
//          triangles {u,v,x}, {u,w,x}, {v,w,x}.
// Every step is a count pass, an exclusive scan and a fill pass over the same
// enumeration.  Intersections: one warp per list pair; the lanes walk the
// shorter list in order and binary-search each element in the other list(s)
// (read-only path).
#include "nd_internal.cuh"

#include <vector>

namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t lo,
                                                   int64_t hi, int32_t x) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

__device__ __forceinline__ int64_t warp_id_global() {
    return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

__device__ __forceinline__ int64_t warp_count_global() {
    return ((int64_t)gridDim.x * blockDim.x) >> 5;
}

// ---- validation and degree split (one warp per vertex) -------------------
// A row must lie inside [0, nnz], be strictly increasing and hold ids in
// [0, n) other than its own, and every entry v of row u needs u in row v.
// Writes nlow[u] = #neighbours < u and upcnt[u] = #neighbours > u.  Reads
// only inside the bounds it has checked, so a malformed graph cannot fault.
//
// Symmetry: vertices are ordered by the key (row length, id).  An entry
// (u, v) whose row u has the larger key searches the shorter row v for u;
// the others are not searched.  The reverse of a searching entry is a
// non-searching one, and distinct entries have distinct reverses, so if
// every searching entry finds its reverse and the searching entries are
// exactly half of nnz (counted in *searched, checked by the host), the two
// halves are in one-to-one correspondence: the graph is symmetric.  A hub
// row is thus never binary-searched, whatever the order of the caller's ids.
// BY_LENGTH = false: the key is the id alone, so the entries above the
// diagonal search (the same argument holds).  That is for graphs whose ids
// the build itself assigned by degree class, high degree first, where the
// entry above the diagonal already points at the shorter row (or one of its
// class) and nothing needs gathering to decide it.
// With mirror (builds with r >= 2), it also records for both entries of
// every pair the position of the other: the reverse entry, found by the same
// search.

// FP (k-core builds, which need no reverse entries): symmetry by
// fingerprint instead of searches.  Every entry (u, v) adds
// f(u, v) - f(v, u) to two 64-bit sums, each with its own mixing function f
// (the splitmix64 finalizer, after Steele, Lea and Flood, on different
// inputs).  A symmetric graph sums to zero exactly.  Otherwise the sums are
// those of f over the entries without a reverse minus f over the missing
// reverses, and both are zero only by a coincidence of two 64-bit hashes.
// It streams col once and gathers nothing.
__device__ __forceinline__ unsigned long long fp_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ void fp_add(unsigned long long (&fp)[2], int64_t u, int32_t v) {
    const unsigned long long k = ((unsigned long long)u << 32) | (uint32_t)v;
    const unsigned long long r = ((unsigned long long)(uint32_t)v << 32) | (unsigned long long)u;
    fp[0] += fp_mix(k ^ 0x9e3779b97f4a7c15ull) - fp_mix(r ^ 0x9e3779b97f4a7c15ull);
    fp[1] += fp_mix(fp_mix(k) + 0x632be59bd9b4e019ull) - fp_mix(fp_mix(r) + 0x632be59bd9b4e019ull);
}

// the checks of entries [pb, pe) of row u (which spans [b, e)), one entry
// per lane: the count of entries below the diagonal, of searching entries,
// and whether any check failed (FP: fp collects this lane's fingerprint
// terms, summed over the warp by the caller)
template <bool BY_LENGTH, bool FP = false>
__device__ __forceinline__ void validate_entries(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                                 const int32_t* __restrict__ col, int64_t u, int64_t b, int64_t e,
                                                 int64_t pb, int64_t pe, uint32_t* __restrict__ mirror, int& low,
                                                 int& found, bool& rowbad, unsigned long long (&fp)[2]) {
    const int lane = threadIdx.x & 31;
    for (int64_t p = pb + lane; p < pe; p += 32) {
        int32_t v = col[p];
        if (v < 0 || v >= n || v == u) { rowbad = true; continue; }
        if (p > b && col[p - 1] >= v) rowbad = true;
        low += (v < u);
        if constexpr (FP) {
            fp_add(fp, u, v);
            continue;
        }
        if (!BY_LENGTH && v < u) continue;
        int64_t vb = rp[v], ve = rp[v + 1];
        // a row longer than n - 1 cannot be simple (and would not fit the 32-bit search)
        if (vb < 0 || ve < vb || ve > nnz || ve - vb >= n) { rowbad = true; continue; }
        if (BY_LENGTH && (e - b < ve - vb || (e - b == ve - vb && u < v))) continue;
        const int64_t pos = vb + nd_lower_bound_n(col + vb, (int)(ve - vb), (int32_t)u);
        if (pos >= ve || col[pos] != (int32_t)u) { rowbad = true; continue; }
        ++found;
        if (mirror) {
            mirror[p] = (uint32_t)pos;
            mirror[pos] = (uint32_t)p;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        low += __shfl_xor_sync(kFull, low, o);
        found += __shfl_xor_sync(kFull, found, o);
    }
    rowbad = __any_sync(kFull, rowbad);
}

// Rows longer than kLongRow entries are not walked by one warp (a hub row of
// a million entries would take a single warp tens of thousands of dependent
// steps): the per-vertex kernels skip them, and a second launch spreads
// their kLongSeg-entry segments over the whole grid.
constexpr int64_t kLongRow = 4096;
constexpr int64_t kLongSeg = 1024;

__device__ __forceinline__ bool is_long_row(int64_t b, int64_t e) { return e - b > kLongRow; }

// the rows (with valid bounds) longer than kLongRow, and their lengths.  It
// runs before validation: the rows of a valid offset array are disjoint, so
// fewer than cap of them are long, and a count above cap (rows that overlap)
// is written nowhere and reported by the caller.
__global__ void k_long_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, int32_t* __restrict__ rows,
                            int64_t* __restrict__ len, unsigned long long cap,
                            unsigned long long* __restrict__ count) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[u], e = rp[u + 1];
        if (b < 0 || e < b || e > nnz || !is_long_row(b, e)) continue;
        const unsigned long long i = atomicAdd(count, 1ull);
        if (i >= cap) continue;
        rows[i] = (int32_t)u;
        len[i] = e - b;
    }
}

// segment s of the long rows: row index i (seg_off[i] <= s < seg_off[i+1])
// and the entry range [pb, pe)
__device__ __forceinline__ void long_segment(int64_t s, const int32_t* __restrict__ rows,
                                             const int64_t* __restrict__ seg_off, int64_t count,
                                             const int64_t* __restrict__ rp, int64_t& u, int64_t& b, int64_t& pb,
                                             int64_t& pe) {
    int64_t lo = 0, hi = count;  // last i with seg_off[i] <= s
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (seg_off[mid] <= s) lo = mid; else hi = mid;
    }
    u = rows[lo];
    b = rp[u];
    const int64_t e = rp[u + 1];
    pb = b + (s - seg_off[lo]) * kLongSeg;
    pe = min(pb + kLongSeg, e);
}

// the two fingerprint sums of a warp's lanes, added to fp_out[0..1]
__device__ __forceinline__ void fp_flush(unsigned long long (&fp)[2], unsigned long long* fp_out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fp[0] += __shfl_xor_sync(kFull, fp[0], o);
        fp[1] += __shfl_xor_sync(kFull, fp[1], o);
    }
    if ((threadIdx.x & 31) == 0 && (fp[0] | fp[1])) {
        atomicAdd(fp_out, fp[0]);
        atomicAdd(fp_out + 1, fp[1]);
    }
}

template <bool BY_LENGTH, bool FP = false>
__global__ void k_validate_split(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                 const int32_t* __restrict__ col, int32_t* __restrict__ nlow,
                                 int64_t* __restrict__ upcnt, int* __restrict__ err,
                                 unsigned long long* __restrict__ searched, uint32_t* __restrict__ mirror,
                                 unsigned long long* __restrict__ fp_out) {
    const int lane = threadIdx.x & 31;
    unsigned long long fp[2] = {0ull, 0ull};
    for (int64_t u = warp_id_global(); u < n; u += warp_count_global()) {
        int64_t b = rp[u], e = rp[u + 1];
        bool bad = (b < 0) || (e < b) || (e > nnz) || (u == 0 && b != 0) || (u == n - 1 && e != nnz);
        if (bad) {
            if (lane == 0) { atomicOr(err, 1); nlow[u] = 0; upcnt[u] = 0; }
            continue;
        }
        if (is_long_row(b, e)) {  // counted by k_validate_long
            if (lane == 0) { nlow[u] = 0; upcnt[u] = 0; }
            continue;
        }
        int low = 0, found = 0;
        bool rowbad = false;
        validate_entries<BY_LENGTH, FP>(n, nnz, rp, col, u, b, e, b, e, mirror, low, found, rowbad, fp);
        if (lane == 0) {
            nlow[u] = low;
            upcnt[u] = (e - b) - low;
            if (found) atomicAdd(searched, (unsigned long long)found);
            if (rowbad) atomicOr(err, 2);
        }
    }
    if constexpr (FP) fp_flush(fp, fp_out);
}

// the long rows, one warp per segment; the counts add up per row
template <bool BY_LENGTH, bool FP = false>
__global__ void k_validate_long(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const int32_t* __restrict__ rows,
                                const int64_t* __restrict__ seg_off, int64_t count, int64_t segs,
                                int32_t* __restrict__ nlow, int64_t* __restrict__ upcnt, int* __restrict__ err,
                                unsigned long long* __restrict__ searched, uint32_t* __restrict__ mirror,
                                unsigned long long* __restrict__ fp_out) {
    const int lane = threadIdx.x & 31;
    unsigned long long fp[2] = {0ull, 0ull};
    for (int64_t sg = warp_id_global(); sg < segs; sg += warp_count_global()) {
        int64_t u, b, pb, pe;
        long_segment(sg, rows, seg_off, count, rp, u, b, pb, pe);
        int low = 0, found = 0;
        bool rowbad = false;
        validate_entries<BY_LENGTH, FP>(n, nnz, rp, col, u, b, rp[u + 1], pb, pe, mirror, low, found, rowbad, fp);
        if (lane == 0) {
            atomicAdd(nlow + u, low);
            atomicAdd(reinterpret_cast<unsigned long long*>(upcnt + u), (unsigned long long)((pe - pb) - low));
            if (found) atomicAdd(searched, (unsigned long long)found);
            if (rowbad) atomicOr(err, 2);
        }
    }
    if constexpr (FP) fp_flush(fp, fp_out);
}

// ---- (1,2): vertices relabelled by degree class ----------------------------
// The k-core pass gathers tau at the neighbour ids of every row.  With ids in
// no particular order (a scrambled R-MAT), the gathers of a large graph go to
// DRAM; most of them hit the few high-degree vertices, but those are spread
// over the whole tau array, one value per line.  The build therefore gives
// the vertices new ids by degree class, floor(log2 d) descending, stable
// within a class, so that the values most gathered share lines.  Results
// are permuted back at the boundary (nd_api.cu).
constexpr int kClasses = 34;         // 0..31 by degree, 32: degree 0, 33: past n
constexpr int kRelabelTile = 4096;   // vertices per block (16 rounds of 256)

__device__ __forceinline__ int degree_class(int64_t d) {
    return d == 0 ? 32 : 31 - (63 - __clzll((unsigned long long)d));  // high degree first
}

__global__ void k_class_count(int64_t n, const int64_t* __restrict__ rp, int64_t* __restrict__ cnt,
                              int64_t nblocks) {
    __shared__ unsigned c[kClasses];
    for (int i = threadIdx.x; i < kClasses; i += blockDim.x) c[i] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kRelabelTile;
    for (int64_t v = t0 + threadIdx.x; v < min(t0 + kRelabelTile, n); v += blockDim.x)
        atomicAdd(&c[degree_class(rp[v + 1] - rp[v])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kClasses - 1; i += blockDim.x) cnt[(int64_t)i * nblocks + blockIdx.x] = c[i];
}

// new id = start of (class, block) + earlier vertices of the class in the block
__global__ void k_class_scatter(int64_t n, const int64_t* __restrict__ rp, const int64_t* __restrict__ off,
                                int64_t nblocks, int32_t* __restrict__ to_new, int32_t* __restrict__ to_old) {
    __shared__ unsigned wcnt[kThreads / 32][kClasses];
    __shared__ unsigned run[kClasses];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kClasses; i += blockDim.x) run[i] = 0;
    const int64_t t0 = (int64_t)blockIdx.x * kRelabelTile;
    for (int64_t r0 = t0; r0 < t0 + kRelabelTile; r0 += kThreads) {
        const int64_t v = r0 + threadIdx.x;
        const bool ok = v < n && v < t0 + kRelabelTile;
        const int k = ok ? degree_class(rp[v + 1] - rp[v]) : kClasses - 1;
        for (int i = lane; i < kClasses; i += 32) wcnt[warp][i] = 0;
        __syncthreads();
        const unsigned same = __match_any_sync(0xffffffffu, k);
        const unsigned rank = __popc(same & ((1u << lane) - 1u));
        if (rank == 0) wcnt[warp][k] = __popc(same);
        __syncthreads();
        if (ok) {
            unsigned before = run[k];
            for (int w = 0; w < warp; ++w) before += wcnt[w][k];
            const int64_t id = off[(int64_t)k * nblocks + blockIdx.x] + before + rank;
            to_new[v] = (int32_t)id;
            to_old[id] = (int32_t)v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kClasses; i += blockDim.x) {
            unsigned tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) tot += wcnt[w][i];
            run[i] += tot;
        }
        __syncthreads();
    }
}

__global__ void k_new_degrees(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ to_new,
                              int64_t* __restrict__ len) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        len[to_new[v]] = rp[v + 1] - rp[v];
}

__device__ __forceinline__ void relabel_entries(const int32_t* __restrict__ col, const int32_t* __restrict__ to_new,
                                                int32_t* __restrict__ ncol, int64_t b, int64_t nb, int64_t pb,
                                                int64_t pe) {
    for (int64_t p = pb + (threadIdx.x & 31); p < pe; p += 32) ncol[nb + (p - b)] = to_new[col[p]];
}

__global__ void k_relabel_rows(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ to_new, const int64_t* __restrict__ nrp,
                               int32_t* __restrict__ ncol) {
    for (int64_t u = warp_id_global(); u < n; u += warp_count_global()) {
        const int64_t b = rp[u], e = rp[u + 1];
        if (is_long_row(b, e)) continue;  // k_relabel_long
        relabel_entries(col, to_new, ncol, b, nrp[to_new[u]], b, e);
    }
}

__global__ void k_relabel_long(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ to_new, const int64_t* __restrict__ nrp,
                               int32_t* __restrict__ ncol, const int32_t* __restrict__ rows,
                               const int64_t* __restrict__ seg_off, int64_t count, int64_t segs) {
    for (int64_t sg = warp_id_global(); sg < segs; sg += warp_count_global()) {
        int64_t u, b, pb, pe;
        long_segment(sg, rows, seg_off, count, rp, u, b, pb, pe);
        relabel_entries(col, to_new, ncol, b, nrp[to_new[u]], pb, pe);
    }
}

__global__ void k_permute_i32(int64_t n, const int32_t* __restrict__ idx, const int32_t* __restrict__ in,
                              int32_t* __restrict__ out, int scatter) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (scatter) out[idx[i]] = in[i];
        else out[i] = in[idx[i]];
    }
}

// (2,3) relabelling: the key (new u, new v) of every entry, at its own
// position (the sort that follows fixes the order)
__device__ __forceinline__ void relabel_key_entries(const int32_t* __restrict__ col, const int32_t* __restrict__ to_new,
                                                    int bits, unsigned long long* __restrict__ keys, int64_t u,
                                                    int64_t pb, int64_t pe) {
    const unsigned long long hi = (unsigned long long)to_new[u] << bits;
    for (int64_t p = pb + (threadIdx.x & 31); p < pe; p += 32) keys[p] = hi | (unsigned long long)to_new[col[p]];
}

__global__ void k_relabel_keys(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ to_new, int bits, unsigned long long* __restrict__ keys) {
    for (int64_t u = warp_id_global(); u < n; u += warp_count_global()) {
        const int64_t b = rp[u], e = rp[u + 1];
        if (is_long_row(b, e)) continue;  // k_relabel_keys_long
        relabel_key_entries(col, to_new, bits, keys, u, b, e);
    }
}

__global__ void k_relabel_keys_long(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const int32_t* __restrict__ to_new, int bits, unsigned long long* __restrict__ keys,
                                    const int32_t* __restrict__ rows, const int64_t* __restrict__ seg_off,
                                    int64_t count, int64_t segs) {
    for (int64_t sg = warp_id_global(); sg < segs; sg += warp_count_global()) {
        int64_t u, b, pb, pe;
        long_segment(sg, rows, seg_off, count, rp, u, b, pb, pe);
        relabel_key_entries(col, to_new, bits, keys, u, pb, pe);
    }
}

__global__ void k_keys_to_col(int64_t nnz, const unsigned long long* __restrict__ keys, int bits,
                              int32_t* __restrict__ col) {
    const unsigned long long mask = (1ull << bits) - 1ull;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x)
        col[j] = (int32_t)(keys[j] & mask);
}

// new edge e = (e_u[e], e_v[e]) -> the caller's edge id: its endpoints in
// caller ids, smaller first, and the rank of the larger among the smaller
// one's larger neighbours in the caller's CSR
__global__ void k_edge_map(int64_t m, const int32_t* __restrict__ e_u, const int32_t* __restrict__ e_v,
                           const int32_t* __restrict__ vto_old, const int64_t* __restrict__ c_rp,
                           const int32_t* __restrict__ c_col, const int32_t* __restrict__ c_nlow,
                           const int64_t* __restrict__ c_up, int32_t* __restrict__ to_new,
                           int32_t* __restrict__ to_old, int* __restrict__ err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = vto_old[e_u[e]], b = vto_old[e_v[e]];
        const int32_t x = a < b ? a : b, y = a < b ? b : a;
        const int64_t first = c_rp[x] + c_nlow[x], end = c_rp[x + 1];
        const int64_t pos = lower_bound_i32(c_col, first, end, y);
        if (pos >= end || c_col[pos] != y) { atomicOr(err, 1); continue; }
        const int64_t cid = c_up[x] + (pos - first);
        to_old[e] = (int32_t)cid;
        to_new[cid] = (int32_t)e;
    }
}

// r-clique tuples of a relabelled (2,3) handle: caller vertex ids, at the
// caller's edge ids
__global__ void k_r_cliques_mapped(int64_t N, const int32_t* __restrict__ e_u, const int32_t* __restrict__ e_v,
                                   const int32_t* __restrict__ vto_old, const int32_t* __restrict__ to_old,
                                   int32_t* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = vto_old[e_u[e]], b = vto_old[e_v[e]];
        const int64_t c = to_old[e];
        out[2 * c] = a < b ? a : b;
        out[2 * c + 1] = a < b ? b : a;
    }
}

// ---- canonical edge ids (one warp per vertex) ------------------------------
// Edge (u,v), u < v, gets id up_start[u] + (rank of v among u's larger
// neighbours): lexicographic order.  eid[p] is the id of the edge at CSR
// position p, for both directions (the reverse entry comes from mirror,
// written by the validation, when there is one).  For the (2,3) adjacency
// layout it also writes, per edge (x,y) with x < y, e_pos = (P(x,y), P(y,x)).
__device__ __forceinline__ void edge_id_entries(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                const int32_t* __restrict__ nlow,
                                                const int64_t* __restrict__ up_start, uint32_t* __restrict__ eid,
                                                int32_t* __restrict__ e_u, int32_t* __restrict__ e_v,
                                                const uint32_t* __restrict__ mirror, uint2* __restrict__ e_pos,
                                                int64_t u, int64_t b, int64_t pb, int64_t pe) {
    const int lane = threadIdx.x & 31;
    const int64_t first_up = b + nlow[u];
    const int64_t base = up_start[u];
    for (int64_t p = pb + lane; p < pe; p += 32) {
        int32_t v = col[p];
        if (p >= first_up) {
            int64_t id = base + (p - first_up);
            eid[p] = (uint32_t)id;
            e_u[id] = (int32_t)u;
            e_v[id] = v;
        } else {
            const int64_t vfirst = rp[v] + nlow[v];
            // the reverse entry: recorded by the validation when available
            const int64_t pos = mirror ? (int64_t)mirror[p]
                                       : lower_bound_i32(col, vfirst, rp[v + 1], (int32_t)u);
            const int64_t id = up_start[v] + (pos - vfirst);
            eid[p] = (uint32_t)id;
            // edge (v,u), v < u: entry pos = P(v,u), entry p = P(u,v)
            if (e_pos) e_pos[id] = make_uint2((uint32_t)pos, (uint32_t)p);
        }
    }
}

__global__ void k_edge_ids(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ nlow, const int64_t* __restrict__ up_start,
                           uint32_t* __restrict__ eid, int32_t* __restrict__ e_u,
                           int32_t* __restrict__ e_v, const uint32_t* __restrict__ mirror,
                           uint2* __restrict__ e_pos) {
    for (int64_t u = warp_id_global(); u < n; u += warp_count_global()) {
        const int64_t b = rp[u], e = rp[u + 1];
        if (is_long_row(b, e)) continue;  // k_edge_ids_long
        edge_id_entries(rp, col, nlow, up_start, eid, e_u, e_v, mirror, e_pos, u, b, b, e);
    }
}

__global__ void k_edge_ids_long(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ nlow, const int64_t* __restrict__ up_start,
                                uint32_t* __restrict__ eid, int32_t* __restrict__ e_u, int32_t* __restrict__ e_v,
                                const uint32_t* __restrict__ mirror, uint2* __restrict__ e_pos,
                                const int32_t* __restrict__ rows, const int64_t* __restrict__ seg_off,
                                int64_t count, int64_t segs) {
    for (int64_t sg = warp_id_global(); sg < segs; sg += warp_count_global()) {
        int64_t u, b, pb, pe;
        long_segment(sg, rows, seg_off, count, rp, u, b, pb, pe);
        edge_id_entries(rp, col, nlow, up_start, eid, e_u, e_v, mirror, e_pos, u, b, pb, pe);
    }
}

// ---- (2,3): triangles by degree orientation --------------------------------
// Vertex u precedes v iff (d_u, u) < (d_v, v).  Orienting every edge from the
// earlier to the later endpoint, each triangle {u,v,w} (u before v before w)
// is found exactly once, as w in out(u) /\ out(v) for the oriented edge
// u -> v; out-lists are at most sqrt(2m) long.  The triangle then adds one
// incidence to each of its three edges, at slots taken from per-edge counters
// (count pass) and cursors (fill pass).  Row order inside an edge's incidence
// row is therefore unspecified; the h-index of a row does not depend on it.
__device__ __forceinline__ bool precedes(int64_t du, int32_t u, int64_t dv, int32_t v) {
    return du < dv || (du == dv && u < v);
}

// one warp per vertex: count / list the out-neighbours of u in id order
// (with out_pos: also the CSR positions of the entry and of its reverse)
template <bool FILL>
__global__ void k_orient(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const uint32_t* __restrict__ eid, int64_t* __restrict__ out_ptr,
                         int32_t* __restrict__ out_col, uint32_t* __restrict__ out_eid,
                         int32_t* __restrict__ out_src, const uint32_t* __restrict__ mirror,
                         uint32_t* __restrict__ out_pos, uint32_t* __restrict__ out_mir) {
    const int lane = threadIdx.x & 31;
    for (int64_t u = warp_id_global(); u < n; u += warp_count_global()) {
        const int64_t b = rp[u], e = rp[u + 1], du = e - b;
        const int64_t base = FILL ? out_ptr[u] : 0;
        int64_t cnt = 0;
        for (int64_t p0 = b; p0 < e; p0 += 32) {
            const int64_t p = p0 + lane;
            bool keep = false;
            int32_t v = 0;
            if (p < e) {
                v = __ldg(col + p);
                keep = precedes(du, (int32_t)u, __ldg(rp + v + 1) - __ldg(rp + v), v);
            }
            const unsigned bal = __ballot_sync(kFull, keep);
            if (FILL && keep) {
                const int64_t slot = base + cnt + __popc(bal & lanemask_lt());
                out_col[slot] = v;
                out_eid[slot] = __ldg(eid + p);
                out_src[slot] = (int32_t)u;
                if (out_pos) {
                    out_pos[slot] = (uint32_t)p;
                    out_mir[slot] = __ldg(mirror + p);
                }
            }
            cnt += __popc(bal);
        }
        if (!FILL && lane == 0) out_ptr[u] = cnt;
    }
}

// one warp per oriented edge u -> v: the triangles {u, v, w}, w in out(u) /\ out(v).
// ADJ: the entries are CSR positions, each pair ordered by its edge's
// canonical endpoints (the entry of the smaller endpoint first).
#ifndef ND_TRI_COUNT_MIN_BLOCKS
#define ND_TRI_COUNT_MIN_BLOCKS 8  // the count pass (with its records) at full occupancy
#endif
#ifndef ND_TRI_MIN_BLOCKS
#define ND_TRI_MIN_BLOCKS 6  // resident blocks per SM for the searching fill (used when the records do not fit)
#endif
// REC (count pass): also record every triangle found from edge k, as the
// offsets of w in the shorter and in the longer out-list (16 bits each: an
// out-list holds at most sqrt(2m) < 65536 entries, since each of its
// vertices has at least the owner's degree and nnz < 2^32), at
// rec[rec_ptr[k] + i]; rec_ptr[k] reserves min(|out(u)|, |out(v)|) slots,
// the most edge k can find.  rec_cnt[k] = triangles found.
template <bool FILL, bool ADJ, typename C = unsigned long long, bool REC = false>
__global__ void __launch_bounds__(kThreads, FILL ? ND_TRI_MIN_BLOCKS : ND_TRI_COUNT_MIN_BLOCKS) k_tri_oriented(int64_t m, const int64_t* __restrict__ out_ptr,
                               const int32_t* __restrict__ out_col, const uint32_t* __restrict__ out_eid,
                               const int32_t* __restrict__ out_src, const uint32_t* __restrict__ out_pos,
                               const uint32_t* __restrict__ out_mir, C* __restrict__ ctr,
                               uint2* __restrict__ inc, const int64_t* __restrict__ rec_ptr = nullptr,
                               uint32_t* __restrict__ rec = nullptr, uint32_t* __restrict__ rec_cnt = nullptr) {
    const int lane = threadIdx.x & 31;
    for (int64_t k = warp_id_global(); k < m; k += warp_count_global()) {
        uint32_t nrec = 0;  // REC: triangles recorded so far for edge k
        const int32_t u = out_src[k], v = out_col[k];
        const uint32_t e_uv = out_eid[k];
        uint32_t Puv = 0, Pvu = 0;
        if (ADJ) { Puv = __ldg(out_pos + k); Pvu = __ldg(out_mir + k); }
        int64_t ab = out_ptr[u], ae = out_ptr[u + 1], bb = out_ptr[v], be = out_ptr[v + 1];
        bool a_is_u = true;
        if (ae - ab > be - bb) {
            int64_t t = ab; ab = bb; bb = t; t = ae; ae = be; be = t;
            a_is_u = false;
        }
        int64_t lo = bb;
        for (int64_t base = ab; base < ae; base += 32) {
            const int64_t p = base + lane;
            bool found = false;
            int64_t pb = 0;
            int32_t x = 0;
            // FILL: the values at p are loaded with x, ahead of the search
            // (coalesced), so only the loads at pb wait for it
            uint32_t ea = 0, pa = 0, ma = 0;
            if (p < ae) {
                x = __ldg(out_col + p);
                if (FILL) {
                    ea = __ldg(out_eid + p);
                    if (ADJ) {
                        pa = __ldg(out_pos + p);
                        ma = __ldg(out_mir + p);
                    }
                }
                pb = lo + nd_lower_bound_n(out_col + lo, (int)(be - lo), x);
                found = (pb < be) && (__ldg(out_col + pb) == x);
            }
            const unsigned bal = __ballot_sync(kFull, found);
            const int nf = __popc(bal);
            if (nf) {
                uint32_t e_uw = 0, e_vw = 0;
                if (!FILL) {
                    if (found) {
                        const uint32_t ea0 = __ldg(out_eid + p), eb = __ldg(out_eid + pb);
                        e_uw = a_is_u ? ea0 : eb;
                        e_vw = a_is_u ? eb : ea0;
                    }
                    if (lane == 0) atomicAdd(ctr + e_uv, (C)nf);
                    if (found) {
                        atomicAdd(ctr + e_uw, (C)1);
                        atomicAdd(ctr + e_vw, (C)1);
                    }
                    if (REC) {
                        if (found)
                            rec[rec_ptr[k] + nrec + __popc(bal & lanemask_lt())] =
                                (uint32_t)(p - ab) | ((uint32_t)(pb - bb) << 16);
                        nrec += (uint32_t)nf;
                    }
                } else {
                    uint32_t pbp = 0, mb = 0;
                    if (found) {
                        const uint32_t eb = __ldg(out_eid + pb);
                        if (ADJ) {
                            pbp = __ldg(out_pos + pb);
                            mb = __ldg(out_mir + pb);
                        }
                        e_uw = a_is_u ? ea : eb;
                        e_vw = a_is_u ? eb : ea;
                    }
                    // the three slot reservations are independent: issue them together
                    C s0 = 0, s_uw = 0, s_vw = 0;
                    if (lane == 0) s0 = atomicAdd(ctr + e_uv, (C)nf);
                    if (found) {
                        s_uw = atomicAdd(ctr + e_uw, (C)1);
                        s_vw = atomicAdd(ctr + e_vw, (C)1);
                    }
                    s0 = __shfl_sync(kFull, s0, 0);
                    if (found) {
                        uint2 r_uv, r_uw, r_vw;
                        if (ADJ) {
                            // third vertex w = x; positions P(.,.) of the six entries
                            const uint32_t Puw = a_is_u ? pa : pbp, Pwu = a_is_u ? ma : mb;
                            const uint32_t Pvw = a_is_u ? pbp : pa, Pwv = a_is_u ? mb : ma;
                            r_uv = u < v ? make_uint2(Puw, Pvw) : make_uint2(Pvw, Puw);
                            r_uw = u < x ? make_uint2(Puv, Pwv) : make_uint2(Pwv, Puv);
                            r_vw = v < x ? make_uint2(Pvu, Pwu) : make_uint2(Pwu, Pvu);
                        } else {
                            r_uv = make_uint2(e_uw, e_vw);
                            r_uw = make_uint2(e_uv, e_vw);
                            r_vw = make_uint2(e_uv, e_uw);
                        }
                        inc[s0 + __popc(bal & lanemask_lt())] = r_uv;
                        inc[s_uw] = r_uw;
                        inc[s_vw] = r_vw;
                    }
                }
            }
            const int64_t last_pb = __shfl_sync(kFull, pb, 31);
            if (base + 32 <= ae) lo = last_pb;
        }
        if (REC && lane == 0) rec_cnt[k] = nrec;
    }
}

// the fill from the count pass's records: one warp per oriented edge k, one
// recorded triangle per lane, so no search is repeated.  The six positions
// of a triangle are read at the recorded offsets of w in the two out-lists
// (the shorter list's reads coalesce, as in the searching fill); slots and
// entries are as in k_tri_oriented<true, true>.
#ifndef ND_FILL_MIN_BLOCKS
#define ND_FILL_MIN_BLOCKS 5  // the fill from records: 48 registers, no spills (24.1 against 25.0 ms at 6 blocks)
#endif
template <typename C>
__global__ void __launch_bounds__(kThreads, ND_FILL_MIN_BLOCKS)
    k_tri_fill_rec(int64_t m, const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ out_col,
                   const uint32_t* __restrict__ out_eid, const int32_t* __restrict__ out_src,
                   const uint32_t* __restrict__ out_pos, const uint32_t* __restrict__ out_mir, C* __restrict__ ctr,
                   uint2* __restrict__ inc, const int64_t* __restrict__ rec_ptr, const uint32_t* __restrict__ rec,
                   const uint32_t* __restrict__ rec_cnt) {
    const int lane = threadIdx.x & 31;
    for (int64_t k = warp_id_global(); k < m; k += warp_count_global()) {
        const uint32_t c = __ldg(rec_cnt + k);
        if (c == 0) continue;
        const int32_t u = out_src[k], v = out_col[k];
        const uint32_t e_uv = out_eid[k];
        const uint32_t Puv = __ldg(out_pos + k), Pvu = __ldg(out_mir + k);
        int64_t ab = out_ptr[u], ae = out_ptr[u + 1], bb = out_ptr[v], be = out_ptr[v + 1];
        bool a_is_u = true;
        if (ae - ab > be - bb) {  // the same choice of the shorter list as the count pass
            int64_t t = ab; ab = bb; bb = t; t = ae; ae = be; be = t;
            a_is_u = false;
        }
        const int64_t r0 = rec_ptr[k];
        for (uint32_t base = 0; base < c; base += 32) {
            const uint32_t i = base + lane;
            const bool found = i < c;
            uint32_t ea = 0, pa = 0, ma = 0, eb = 0, pbp = 0, mb = 0;
            int32_t x = 0;
            if (found) {
                const uint32_t r = __ldg(rec + r0 + i);
                const int64_t p = ab + (r & 0xffffu), pb = bb + (r >> 16);
                x = __ldg(out_col + p);
                ea = __ldg(out_eid + p);
                pa = __ldg(out_pos + p);
                ma = __ldg(out_mir + p);
                eb = __ldg(out_eid + pb);
                pbp = __ldg(out_pos + pb);
                mb = __ldg(out_mir + pb);
            }
            const unsigned bal = __ballot_sync(kFull, found);
            const int nf = __popc(bal);
            const uint32_t e_uw = a_is_u ? ea : eb, e_vw = a_is_u ? eb : ea;
            C s0 = 0, s_uw = 0, s_vw = 0;
            if (lane == 0) s0 = atomicAdd(ctr + e_uv, (C)nf);
            if (found) {
                s_uw = atomicAdd(ctr + e_uw, (C)1);
                s_vw = atomicAdd(ctr + e_vw, (C)1);
            }
            s0 = __shfl_sync(kFull, s0, 0);
            if (found) {
                const uint32_t Puw = a_is_u ? pa : pbp, Pwu = a_is_u ? ma : mb;
                const uint32_t Pvw = a_is_u ? pbp : pa, Pwv = a_is_u ? mb : ma;
                inc[s0 + __popc(bal & lanemask_lt())] = u < v ? make_uint2(Puw, Pvw) : make_uint2(Pvw, Puw);
                inc[s_uw] = u < x ? make_uint2(Puv, Pwv) : make_uint2(Pwv, Puv);
                inc[s_vw] = v < x ? make_uint2(Pvu, Pwu) : make_uint2(Pwu, Pvu);
            }
        }
    }
}

// the record slots of each oriented edge: min(|out(u)|, |out(v)|)
__global__ void k_rec_bound(int64_t m, const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ out_src,
                            const int32_t* __restrict__ out_col, int64_t* __restrict__ rec_ptr) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = out_src[k], v = out_col[k];
        const int64_t a = out_ptr[u + 1] - out_ptr[u], b = out_ptr[v + 1] - out_ptr[v];
        rec_ptr[k] = a < b ? a : b;
    }
}

__global__ void k_widen_u32(int64_t m, const unsigned* __restrict__ in, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)in[i];
}

__global__ void k_narrow_u32(int64_t m, const int64_t* __restrict__ in, unsigned* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (unsigned)in[i];
}

// ---- (2,3) adjacency layout: order each row by its third vertex -----------
// The entries of the row of edge (x,y) are pairs (P(x,w), P(y,w)) over the
// triangles {x,y,w}, in fill order.  Both components grow with w, so the
// rank of an entry is the rank of its component in the shorter of the two
// adjacency lists, N(s): one bit per position of N(s) marks the row's
// entries, and rank = (bits set in earlier words) + (bits below it in its
// word).  O(d + deg(s)/32) per row, no comparison sort.  Rows up to 32
// entries are ranked by comparing keys across the warp instead.  One warp
// per row; the bit and prefix words sit in shared memory (kRankWords per
// warp); a row whose shorter list needs more words is left to the overflow
// pass, which uses global scratch.
constexpr int kRankWarps = 8;
#ifndef ND_RANK_WORDS
#define ND_RANK_WORDS 512  // 16,384 positions per warp; 32 KB per block
#endif
constexpr int kRankWords = ND_RANK_WORDS;

__device__ __forceinline__ void rank_row(const uint2* __restrict__ src, uint2* __restrict__ dst, int64_t jb,
                                         int64_t d, int comp, uint32_t base, int64_t nw,
                                         uint32_t* __restrict__ bm, uint32_t* __restrict__ pre) {
    const int lane = threadIdx.x & 31;
    if (d <= 32) {
        uint2 e = make_uint2(0u, 0u);
        uint32_t key = 0xffffffffu;
        if (lane < d) {
            e = src[jb + lane];
            key = comp ? e.y : e.x;
        }
        int rank = 0;
        for (int o = 0; o < d; ++o) rank += (__shfl_sync(kFull, key, o) < key);
        if (lane < d) dst[jb + rank] = e;
        return;
    }
    for (int64_t w = lane; w < nw; w += 32) bm[w] = 0u;
    __syncwarp();
    for (int64_t j = jb + lane; j < jb + d; j += 32) {
        const uint2 e = src[j];
        const uint32_t k = (comp ? e.y : e.x) - base;
        atomicOr(bm + (k >> 5), 1u << (k & 31));
    }
    __syncwarp();
    uint32_t run = 0;
    for (int64_t w0 = 0; w0 < nw; w0 += 32) {
        const int64_t w = w0 + lane;
        const uint32_t c = w < nw ? (uint32_t)__popc(bm[w]) : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (w < nw) pre[w] = run + incl - c;
        run += __shfl_sync(kFull, incl, 31);
    }
    __syncwarp();
    for (int64_t j = jb + lane; j < jb + d; j += 32) {
        const uint2 e = src[j];
        const uint32_t k = (comp ? e.y : e.x) - base;
        const uint32_t rank = pre[k >> 5] + (uint32_t)__popc(bm[k >> 5] & ((1u << (k & 31)) - 1u));
        dst[jb + rank] = e;
    }
    __syncwarp();
}

// BIG = false: every row, bits in shared memory; rows that need more than
// kRankWords words are appended to `over` (count in over_ctr[0], largest
// word count in over_ctr[1]).  BIG = true: the rows in `over`, bits in
// global scratch of 2 * scratch_words words per warp.
template <bool BIG>
__global__ void __launch_bounds__(32 * kRankWarps)
k_row_rank(int64_t N, const int64_t* __restrict__ inc_ptr, const int32_t* __restrict__ e_u,
           const int32_t* __restrict__ e_v, const int64_t* __restrict__ rp, const uint2* __restrict__ src,
           uint2* __restrict__ dst, uint32_t* __restrict__ over, unsigned long long* __restrict__ over_ctr,
           uint32_t* __restrict__ scratch, int64_t scratch_words) {
    extern __shared__ uint32_t rank_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *bm, *pre;
    if (BIG) {
        bm = scratch + (size_t)2 * scratch_words * warp_id_global();
        pre = bm + scratch_words;
    } else {
        bm = rank_smem + (size_t)2 * kRankWords * wib;
        pre = bm + kRankWords;
    }
    const int64_t rows = BIG ? (int64_t)over_ctr[0] : N;
    for (int64_t i = warp_id_global(); i < rows; i += warp_count_global()) {
        const int64_t R = BIG ? (int64_t)over[i] : i;
        const int64_t jb = inc_ptr[R], d = inc_ptr[R + 1] - jb;
        if (d <= 1) {
            if (d == 1 && lane == 0) dst[jb] = src[jb];
            continue;
        }
        const int32_t x = e_u[R], y = e_v[R];
        const int64_t dx = rp[x + 1] - rp[x], dy = rp[y + 1] - rp[y];
        const int comp = dx <= dy ? 0 : 1;
        const uint32_t base = (uint32_t)rp[comp ? y : x];
        const int64_t nw = ((comp ? dy : dx) + 31) / 32;
        if (!BIG && d > 32 && nw > kRankWords) {
            if (lane == 0) {
                over[atomicAdd(over_ctr, 1ull)] = (uint32_t)R;
                atomicMax(over_ctr + 1, (unsigned long long)nw);
            }
            continue;
        }
        rank_row(src, dst, jb, d, comp, base, nw, bm, pre);
    }
}

// ---- (3,4) step 1: canonical triangle list (one warp per edge) -------------
// Edge (u,v), u<v, owns the triangles (u,v,w) with w > v: w in the parts of
// N(u) and N(v) above v.  COUNT: ptr[e] = number owned.  FILL: tri_w, tri_e.
template <bool FILL>
__global__ void k_triangle_list(int64_t m, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const int32_t* __restrict__ nlow,
                                const int64_t* __restrict__ up_start, const int32_t* __restrict__ e_u,
                                const int32_t* __restrict__ e_v, int64_t* __restrict__ ptr,
                                int32_t* __restrict__ tri_w, uint32_t* __restrict__ tri_e) {
    const int lane = threadIdx.x & 31;
    for (int64_t e = warp_id_global(); e < m; e += warp_count_global()) {
        const int32_t u = e_u[e], v = e_v[e];
        // position of v in row u follows from the edge id; entries after it are > v
        int64_t ab = rp[u] + nlow[u] + (e - up_start[u]) + 1, ae = rp[u + 1];
        int64_t bb = rp[v] + nlow[v], be = rp[v + 1];
        if (ae - ab > be - bb) { int64_t t = ab; ab = bb; bb = t; t = ae; ae = be; be = t; }
        int64_t out = FILL ? ptr[e] : 0;
        int64_t cnt = 0;
        int64_t lo = bb;
        for (int64_t base = ab; base < ae; base += 32) {
            int64_t p = base + lane;
            bool found = false;
            int64_t pb = 0;
            int32_t x = 0;
            if (p < ae) {
                x = __ldg(col + p);
                pb = lower_bound_i32(col, lo, be, x);
                found = (pb < be) && (__ldg(col + pb) == x);
            }
            unsigned bal = __ballot_sync(kFull, found);
            if (FILL && found) {
                int64_t slot = out + cnt + __popc(bal & lanemask_lt());
                tri_w[slot] = x;
                tri_e[slot] = (uint32_t)e;
            }
            cnt += __popc(bal);
            int64_t last_pb = __shfl_sync(kFull, pb, 31);
            if (base + 32 <= ae) lo = last_pb;
        }
        if (!FILL && lane == 0) ptr[e] = cnt;
    }
}

// ---- (3,4): 4-cliques by degree orientation ---------------------------------
// Every 4-clique {a,b,w,x} with a before b before w before x (degree order) is
// found exactly once, as x in out(a) /\ out(b) /\ out(w) for the oriented
// triangle (a,b,w).  Its four triangles get their canonical ids (lexicographic
// u<v<w, grouped by edge (u,v) in tri_ptr / tri_w) from one binary search
// each, because the six edge ids are known from the out-lists.  The 4-cliques
// are listed once (4 triangle ids each), then scattered into the incidence
// rows through per-triangle cursors; row order is therefore unspecified.

struct otri {  // oriented triangle a -> b -> w and its edge ids
    int32_t a, b, w;
    uint32_t e_ab, e_aw, e_bw;
};

// one warp per oriented edge a -> b: the oriented triangles (a, b, w)
template <bool FILL>
__global__ void k_otri(int64_t m, const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ out_col,
                       const uint32_t* __restrict__ out_eid, const int32_t* __restrict__ out_src,
                       int64_t* __restrict__ ptr, otri* __restrict__ tris) {
    const int lane = threadIdx.x & 31;
    for (int64_t k = warp_id_global(); k < m; k += warp_count_global()) {
        const int32_t a = out_src[k], b = out_col[k];
        const uint32_t e_ab = out_eid[k];
        int64_t ab = out_ptr[a], ae = out_ptr[a + 1], bb = out_ptr[b], be = out_ptr[b + 1];
        bool a_is_a = true;
        if (ae - ab > be - bb) {
            int64_t t = ab; ab = bb; bb = t; t = ae; ae = be; be = t;
            a_is_a = false;
        }
        const int64_t out = FILL ? ptr[k] : 0;
        int64_t cnt = 0, lo = bb;
        for (int64_t base = ab; base < ae; base += 32) {
            const int64_t p = base + lane;
            bool found = false;
            int64_t pb = 0;
            int32_t x = 0;
            if (p < ae) {
                x = __ldg(out_col + p);
                pb = lower_bound_i32(out_col, lo, be, x);
                found = (pb < be) && (__ldg(out_col + pb) == x);
            }
            const unsigned bal = __ballot_sync(kFull, found);
            if (FILL && found) {
                const uint32_t e1 = __ldg(out_eid + p), e2 = __ldg(out_eid + pb);
                otri t;
                t.a = a; t.b = b; t.w = x; t.e_ab = e_ab;
                t.e_aw = a_is_a ? e1 : e2;
                t.e_bw = a_is_a ? e2 : e1;
                tris[out + cnt + __popc(bal & lanemask_lt())] = t;
            }
            cnt += __popc(bal);
            const int64_t last_pb = __shfl_sync(kFull, pb, 31);
            if (base + 32 <= ae) lo = last_pb;
        }
        if (!FILL && lane == 0) ptr[k] = cnt;
    }
}

// canonical id of the triangle on vertices p, q, r with edge ids epq, epr, eqr
__device__ __forceinline__ uint32_t canon_tri(int32_t p, int32_t q, int32_t r, uint32_t epq, uint32_t epr,
                                              uint32_t eqr, const int64_t* __restrict__ tri_ptr,
                                              const int32_t* __restrict__ tri_w, bool* ok) {
    // the smallest two vertex ids own the triangle; the largest is its third vertex
    uint32_t edge;
    int32_t third;
    if (p > q && p > r) { edge = eqr; third = p; }
    else if (q > r) { edge = epr; third = q; }
    else { edge = epq; third = r; }
    const int64_t lo = __ldg(tri_ptr + edge), hi = __ldg(tri_ptr + edge + 1);
    const int64_t pos = lower_bound_i32(tri_w, lo, hi, third);
    if (pos >= hi || __ldg(tri_w + pos) != third) { *ok = false; return 0; }
    return (uint32_t)pos;
}

// one warp per oriented triangle: x in out(a) /\ out(b) /\ out(w).
// MODE 0 counts the 4-cliques of the triangle into ptr[t]; MODE 1 writes
// their four canonical triangle ids at ptr[t] (scanned) and counts the
// incidences of each triangle in rowcnt.
template <int MODE>
__global__ void k_k4(int64_t T, const otri* __restrict__ tris, const int64_t* __restrict__ out_ptr,
                     const int32_t* __restrict__ out_col, const uint32_t* __restrict__ out_eid,
                     const int64_t* __restrict__ tri_ptr, const int32_t* __restrict__ tri_w,
                     int64_t* __restrict__ ptr, uint4* __restrict__ k4, unsigned long long* __restrict__ rowcnt,
                     int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    for (int64_t t = warp_id_global(); t < T; t += warp_count_global()) {
        const otri tr = tris[t];
        const int32_t vtx[3] = {tr.a, tr.b, tr.w};
        int64_t rb[3], re[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) { rb[i] = out_ptr[vtx[i]]; re[i] = out_ptr[vtx[i] + 1]; }
        int A = 0;
        if (re[1] - rb[1] < re[A] - rb[A]) A = 1;
        if (re[2] - rb[2] < re[A] - rb[A]) A = 2;
        const int B1 = (A == 0) ? 1 : 0, B2 = (A == 2) ? 1 : 2;
        const int64_t out = MODE ? ptr[t] : 0;
        int64_t cnt = 0;
        bool ok = true;
        uint32_t id0 = 0;  // MODE 1: the triangle (a,b,w) itself, shared by all its 4-cliques
        if (MODE == 1) {
            if (ptr[t + 1] == out) continue;  // no 4-clique here
            id0 = canon_tri(tr.a, tr.b, tr.w, tr.e_ab, tr.e_aw, tr.e_bw, tri_ptr, tri_w, &ok);
        }
        for (int64_t base = rb[A]; base < re[A]; base += 32) {
            const int64_t p = base + lane;
            bool found = false;
            int64_t pos[3] = {0, 0, 0};
            int32_t x = 0;
            if (p < re[A]) {
                x = __ldg(out_col + p);
                pos[A] = p;
                pos[B1] = lower_bound_i32(out_col, rb[B1], re[B1], x);
                if (pos[B1] < re[B1] && __ldg(out_col + pos[B1]) == x) {
                    pos[B2] = lower_bound_i32(out_col, rb[B2], re[B2], x);
                    found = (pos[B2] < re[B2]) && (__ldg(out_col + pos[B2]) == x);
                }
            }
            const unsigned bal = __ballot_sync(kFull, found);
            if (MODE == 1 && found) {
                const uint32_t e_ax = __ldg(out_eid + pos[0]), e_bx = __ldg(out_eid + pos[1]),
                               e_wx = __ldg(out_eid + pos[2]);
                uint4 ids;
                ids.x = id0;
                ids.y = canon_tri(tr.a, tr.b, x, tr.e_ab, e_ax, e_bx, tri_ptr, tri_w, &ok);
                ids.z = canon_tri(tr.a, tr.w, x, tr.e_aw, e_ax, e_wx, tri_ptr, tri_w, &ok);
                ids.w = canon_tri(tr.b, tr.w, x, tr.e_bw, e_bx, e_wx, tri_ptr, tri_w, &ok);
                k4[out + cnt + __popc(bal & lanemask_lt())] = ids;
                atomicAdd(rowcnt + ids.y, 1ull);
                atomicAdd(rowcnt + ids.z, 1ull);
                atomicAdd(rowcnt + ids.w, 1ull);
            }
            cnt += __popc(bal);
        }
        if (MODE == 1 && cnt > 0 && lane == 0) atomicAdd(rowcnt + id0, (unsigned long long)cnt);
        if (MODE == 1 && !__all_sync(kFull, ok) && lane == 0) atomicOr(err, 4);
        if (MODE == 0 && lane == 0) ptr[t] = cnt;
    }
}

// one thread per 4-clique: add it to the rows of its four triangles
template <typename C>
__global__ void k_k4_scatter(int64_t K, const uint4* __restrict__ k4, C* __restrict__ cursor,
                             uint32_t* __restrict__ inc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 q = k4[i];
        const uint32_t id[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t* d = inc + 3 * (int64_t)atomicAdd(cursor + id[k], (C)1);
            int o = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j != k) d[o++] = id[j];
        }
    }
}

// ---- degree buckets --------------------------------------------------------
// bucket of a row of length d under thresholds t = (t0, t1, t2):
// [1,t0] -> 4 lanes, (t0,t1] -> 8 lanes, (t1,t2] -> a warp, > t2 -> a CTA
__device__ __forceinline__ int bucket_of(int64_t d, int3 t) {
    return d == 0 ? -1 : (d <= t.x ? 0 : (d <= t.y ? 1 : (d <= t.z ? 2 : 3)));
}

__global__ void k_bucket_flags(int64_t N, const int64_t* __restrict__ inc_ptr, int b, int3 thr,
                               int64_t* __restrict__ flags, unsigned long long* __restrict__ inc_sum) {
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = inc_ptr[i + 1] - inc_ptr[i];
        bool in = bucket_of(d, thr) == b;
        flags[i] = in;
        if (in) local += (unsigned long long)d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(inc_sum, local);
}

__global__ void k_bucket_scatter(int64_t N, const int64_t* __restrict__ inc_ptr, int b, int3 thr,
                                 const int64_t* __restrict__ pos, nd_item* __restrict__ items) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = inc_ptr[i + 1] - inc_ptr[i];
        if (bucket_of(d, thr) == b) {
            nd_item it;
            it.jb = inc_ptr[i];
            it.R = (uint32_t)i;
            it.d = (uint32_t)d;
            items[pos[i]] = it;
        }
    }
}

// graph index of r-clique R (caller's order): the i with off[i] <= R < off[i+1]
__global__ void k_graph_ids(int64_t N, const int64_t* __restrict__ off, int count, const int32_t* __restrict__ to_new,
                            uint32_t* __restrict__ gid) {
    for (int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; R < N; R += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = count;  // last i with off[i] <= R
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= R) lo = mid; else hi = mid;
        }
        gid[to_new ? to_new[R] : R] = (uint32_t)lo;
    }
}

__global__ void k_r_cliques(int r, int64_t N, const int32_t* __restrict__ e_u,
                            const int32_t* __restrict__ e_v, const int32_t* __restrict__ tri_w,
                            const uint32_t* __restrict__ tri_e, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (r == 1) {
            out[i] = (int32_t)i;
        } else if (r == 2) {
            out[2 * i] = e_u[i];
            out[2 * i + 1] = e_v[i];
        } else {
            uint32_t e = tri_e[i];
            out[3 * i] = e_u[e];
            out[3 * i + 1] = e_v[e];
            out[3 * i + 2] = tri_w[i];
        }
    }
}

// ---- batches: the disjoint union of many graphs (one block per graph) ------
// Vertex ids of graph i are shifted by n_off; its CSR slots by nnz_off.  A
// graph whose offsets or ids fall outside its own range is reported.
__global__ void k_union(const nd_union_part* __restrict__ parts, int count, int64_t* __restrict__ urp,
                        int32_t* __restrict__ ucol, int* __restrict__ err) {
    for (int gi = blockIdx.x; gi < count; gi += gridDim.x) {
        const nd_union_part p = parts[gi];
        if (threadIdx.x == 0 && (p.rp[0] != 0 || p.rp[p.n] != p.nnz)) atomicOr(err, 1);
        for (int64_t i = threadIdx.x; i < p.n; i += blockDim.x) {
            int64_t x = p.rp[i];
            if (x < 0 || x > p.nnz) { atomicOr(err, 1); x = 0; }
            urp[p.n_off + i] = p.nnz_off + x;
        }
        for (int64_t j = threadIdx.x; j < p.nnz; j += blockDim.x) {
            int32_t v = p.col[j];
            if (v < 0 || v >= p.n) { atomicOr(err, 2); v = 0; }
            ucol[p.nnz_off + j] = v + (int32_t)p.n_off;
        }
    }
}

// out[i] = src[idx[i]] for the r-clique offsets of a batch
__global__ void k_gather_i64(const int64_t* __restrict__ src, const int64_t* __restrict__ idx, int count,
                             int64_t* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = src[idx[i]];
}

int grid_cap(const nd_incidence* h) { return (h->sm_count > 0 ? h->sm_count : 152) * 8; }

nd_status read_flag(int* dflag, int* hval, cudaStream_t st) {
    ND_CUDA(cudaMemcpyAsync(hval, dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    return ND_OK;
}

nd_status read_i64(const int64_t* d, int64_t* hv, cudaStream_t st) {
    ND_CUDA(cudaMemcpyAsync(hv, d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    return ND_OK;
}

}  // namespace

// Copy the caller's CSR into owned device buffers, validate it, split each
// row at its own vertex and derive the canonical edge numbering offsets.
// the rows longer than kLongRow and the offsets of their kLongSeg segments
// (a host scan over the few such rows); kept on the handle for the edge ids
static nd_status find_long_rows(nd_incidence* h, cudaStream_t st) {
    h->long_count = h->long_segs = 0;
    if (h->n == 0 || h->nnz <= kLongRow) return ND_OK;
    const int64_t cap = h->nnz / kLongRow + 1;
    ND_TRY(nd_alloc((void**)&h->long_rows, sizeof(int32_t) * cap, st, h));
    nd_tmp<int64_t> len(st);
    nd_tmp<unsigned long long> cnt(st);
    ND_TRY(len.alloc(cap));
    ND_TRY(cnt.alloc(1));
    ND_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    k_long_rows<<<nd_blocks_for(h->n, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
        h->n, h->nnz, h->rp, h->long_rows, len, (unsigned long long)cap, cnt);
    ND_CUDA(cudaGetLastError());
    unsigned long long c = 0;
    ND_CUDA(cudaMemcpyAsync(&c, cnt.p, sizeof(c), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    if (c > (unsigned long long)cap) {  // overlapping rows: not an offset array
        nd_set_error("row_ptr is not a valid offset array");
        return ND_E_INVAL;
    }
    if (c == 0) return ND_OK;
    std::vector<int64_t> hl(c), off(c + 1, 0);
    ND_CUDA(cudaMemcpyAsync(hl.data(), len.p, sizeof(int64_t) * c, cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    for (unsigned long long i = 0; i < c; ++i) off[i + 1] = off[i] + (hl[i] + kLongSeg - 1) / kLongSeg;
    ND_TRY(nd_alloc((void**)&h->long_seg, sizeof(int64_t) * (c + 1), st, h));
    ND_CUDA(cudaMemcpyAsync(h->long_seg, off.data(), sizeof(int64_t) * (c + 1), cudaMemcpyHostToDevice, st));
    ND_TRY(nd_wait(st));  // off is a host temporary
    h->long_count = (int64_t)c;
    h->long_segs = off[c];
    return ND_OK;
}

static void release_long_rows(nd_incidence* h, cudaStream_t st) {
    nd_release(h->long_rows, st);
    nd_release(h->long_seg, st);
    h->long_rows = nullptr;
    h->long_seg = nullptr;
    h->long_count = h->long_segs = 0;
}

// validation and degree split of the handle's CSR (h->rp, h->col): nlow,
// up_start, the long rows, for r >= 2 the reverse entries, and h->m
// by_length: the symmetry key of k_validate_split (false only for ids that
// the build assigned by degree class); mirror: record the reverse entries
static nd_status validate_split(nd_incidence* h, cudaStream_t st, bool by_length, bool mirror) {
    const nd_csr gg{h->n, h->nnz, h->rp, h->col, 1};
    const nd_csr* g = &gg;
    ND_TRY(nd_alloc((void**)&h->nlow, sizeof(int32_t) * (g->n > 0 ? g->n : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->up_start, sizeof(int64_t) * (g->n + 1), st, h));
    // reverse entries for the edge ids and the (2,3) adjacency layout (build only)
    if (mirror && h->r >= 2 && g->nnz > 0 && g->nnz < (int64_t)UINT32_MAX)
        ND_TRY(nd_alloc((void**)&h->mirror, sizeof(uint32_t) * g->nnz, st, h));
    nd_tmp<int> derr(st);
    ND_TRY(derr.alloc(1));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    // k-core builds (no reverse entries needed) decide symmetry by fingerprint
    const bool fp = h->r == 1;
    nd_tmp<unsigned long long> dsearched(st);
    ND_TRY(dsearched.alloc(3));  // [0] searching entries found, [1..2] fingerprint sums
    ND_CUDA(cudaMemsetAsync(dsearched, 0, 3 * sizeof(unsigned long long), st));
    ND_CUDA(cudaMemsetAsync(h->up_start, 0, sizeof(int64_t) * (g->n + 1), st));
    ND_TRY(find_long_rows(h, st));
    if (g->n > 0) {
        nd_prof_scope ps("validate_split", st);
        int blocks = nd_blocks_for(g->n * 32, kThreads, grid_cap(h) * 4);
        auto split = fp ? k_validate_split<true, true> : (by_length ? k_validate_split<true> : k_validate_split<false>);
        split<<<blocks, kThreads, 0, st>>>(g->n, g->nnz, h->rp, h->col, h->nlow, h->up_start, derr, dsearched,
                                           h->mirror, dsearched.p + 1);
        ND_CUDA(cudaGetLastError());
        if (h->long_segs > 0) {
            auto lng = fp ? k_validate_long<true, true> : (by_length ? k_validate_long<true> : k_validate_long<false>);
            lng<<<nd_blocks_for(h->long_segs * 32, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
                g->n, g->nnz, h->rp, h->col, h->long_rows, h->long_seg, h->long_count, h->long_segs, h->nlow,
                h->up_start, derr, dsearched, h->mirror, dsearched.p + 1);
            ND_CUDA(cudaGetLastError());
        }
    }
    int herr = 0;
    ND_TRY(read_flag(derr, &herr, st));
    if (herr) {
        nd_set_error(herr & 1 ? "row_ptr is not a valid offset array"
                              : "col is not simple, sorted and symmetric");
        return ND_E_INVAL;
    }
    ND_TRY(nd_scan_i64(h->up_start, g->n, st));
    int64_t m = 0, found = 0;
    unsigned long long hs[3] = {0, 0, 0};
    ND_TRY(read_i64(h->up_start + g->n, &m, st));
    ND_CUDA(cudaMemcpyAsync(hs, dsearched.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    found = (int64_t)hs[0];
    if (fp ? (hs[1] != 0 || hs[2] != 0 || 2 * m != g->nnz) : (2 * found != g->nnz || 2 * m != g->nnz)) {
        // every searching entry has its reverse; a surplus of the others is
        // an entry without one
        nd_set_error("col is not symmetric (an entry without its reverse)");
        return ND_E_INVAL;
    }
    h->m = m;
    return ND_OK;
}

// graphs smaller than this keep their ids: their tau fits in cache anyway,
// and the few launches of a relabelling would dominate their build
constexpr int64_t kRelabelMinVertices = 1 << 16;

nd_status nd_build_graph(nd_incidence* h, const nd_csr* g, cudaStream_t st, bool truss_relabel) {
    h->n = g->n;
    h->nnz = g->nnz;
    ND_TRY(nd_alloc((void**)&h->rp, sizeof(int64_t) * (g->n + 1), st, h));
    ND_TRY(nd_alloc((void**)&h->col, sizeof(int32_t) * (g->nnz > 0 ? g->nnz : 1), st, h));
    cudaMemcpyKind kind = g->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ND_CUDA(cudaMemcpyAsync(h->rp, g->row_ptr, sizeof(int64_t) * (g->n + 1), kind, st));
    if (g->nnz > 0) ND_CUDA(cudaMemcpyAsync(h->col, g->col, sizeof(int32_t) * g->nnz, kind, st));
    // a (2,3) graph that the relabelling will rewrite is validated again
    // under its new ids, and only that second pass records reverse entries
    const bool rewritten = truss_relabel && h->r == 2 && g->n >= kRelabelMinVertices;
    return validate_split(h, st, true, !rewritten);
}

// vertex ids by degree class (k_class_count / k_class_scatter) for the graph
// in h->rp: to_new[caller id] = new id, to_old[new id] = caller id
static nd_status class_ids(nd_incidence* h, int32_t* to_new, int32_t* to_old, cudaStream_t st) {
    const int64_t n = h->n;
    const int64_t nblocks = (n + kRelabelTile - 1) / kRelabelTile;
    const int64_t cells = (int64_t)(kClasses - 1) * nblocks;
    nd_tmp<int64_t> cnt(st);
    ND_TRY(cnt.alloc(cells + 1));
    ND_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (cells + 1), st));
    k_class_count<<<nblocks, kThreads, 0, st>>>(n, h->rp, cnt, nblocks);
    ND_CUDA(cudaGetLastError());
    ND_TRY(nd_scan_i64(cnt, cells, st));
    k_class_scatter<<<nblocks, kThreads, 0, st>>>(n, h->rp, cnt, nblocks, to_new, to_old);
    ND_CUDA(cudaGetLastError());
    return ND_OK;
}

// (2,3), step 1 of the relabelling (after validation, before the edge ids):
// vertices renumbered by degree class, the graph rewritten under the new ids
// with every row sorted again (a radix sort of the keys (new u, new v) of
// all entries, which is the new CSR in row order), then validated and split
// again.  The caller's CSR and its split are kept until step 2 has mapped
// the edges.  Graphs below kRelabelMinVertices keep their ids.
nd_status nd_relabel_truss_graph(nd_incidence* h, cudaStream_t st) {
    const int64_t n = h->n, nnz = h->nnz;
    if (n < kRelabelMinVertices || h->r != 2) return ND_OK;
    nd_prof_scope ps("relabel", st);
    int32_t* vto_new = nullptr;
    ND_TRY(nd_alloc((void**)&vto_new, sizeof(int32_t) * n, st, h));
    ND_TRY(nd_alloc((void**)&h->vto_old, sizeof(int32_t) * n, st, h));
    nd_status rc = class_ids(h, vto_new, h->vto_old, st);
    int64_t* nrp = nullptr;
    int32_t* ncol = nullptr;
    if (rc == ND_OK) rc = nd_alloc((void**)&nrp, sizeof(int64_t) * (n + 1), st, h);
    if (rc == ND_OK) rc = nd_alloc((void**)&ncol, sizeof(int32_t) * (nnz > 0 ? nnz : 1), st, h);
    if (rc == ND_OK && nnz > 0) {
        nd_tmp<unsigned long long> keys(st), alt(st);
        rc = keys.alloc(nnz);
        if (rc == ND_OK) rc = alt.alloc(nnz);
        const int bits = nd_id_bits(n);
        if (rc == ND_OK) {
            k_relabel_keys<<<nd_blocks_for(n * 32, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
                n, h->rp, h->col, vto_new, bits, keys);
            if (h->long_segs > 0)
                k_relabel_keys_long<<<nd_blocks_for(h->long_segs * 32, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
                    h->rp, h->col, vto_new, bits, keys, h->long_rows, h->long_seg, h->long_count, h->long_segs);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = nd_cuda_fail(e, "k_relabel_keys", __FILE__, __LINE__);
        }
        unsigned long long* sorted = nullptr;
        if (rc == ND_OK) rc = nd_sort_u64(keys, alt, nnz, 2 * bits, &sorted, st);
        if (rc == ND_OK) {
            k_keys_to_col<<<nd_blocks_for(nnz, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(nnz, sorted, bits, ncol);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = nd_cuda_fail(e, "k_keys_to_col", __FILE__, __LINE__);
        }
    }
    if (rc == ND_OK) {
        ND_CUDA(cudaMemsetAsync(nrp + n, 0, sizeof(int64_t), st));
        k_new_degrees<<<nd_blocks_for(n, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(n, h->rp, vto_new, nrp);
        ND_CUDA(cudaGetLastError());
        rc = nd_scan_i64(nrp, n, st);
    }
    nd_release(vto_new, st);
    if (rc != ND_OK) {
        nd_release(nrp, st);
        nd_release(ncol, st);
        return rc;
    }
    // keep the caller's graph and split for the edge map; the new graph
    // takes their place and is split again
    h->c_rp = h->rp;
    h->c_col = h->col;
    h->c_nlow = h->nlow;
    h->c_up = h->up_start;
    h->rp = nrp;
    h->col = ncol;
    h->nlow = nullptr;
    h->up_start = nullptr;
    nd_release(h->mirror, st);
    h->mirror = nullptr;
    release_long_rows(h, st);
    const int64_t m = h->m;
    ND_TRY(validate_split(h, st, false, true));
    if (h->m != m) { nd_set_error("relabelled graph lost edges (internal fault)"); return ND_E_CUDA; }
    return ND_OK;
}

// (2,3), step 2 (after the edge ids of the new graph): the map between the
// new canonical edge ids and the caller's, by searching each new edge's
// caller endpoints in the caller's rows; then the caller's arrays go
nd_status nd_relabel_truss_edges(nd_incidence* h, cudaStream_t st) {
    if (!h->c_rp) return ND_OK;
    const int64_t m = h->m;
    ND_TRY(nd_alloc((void**)&h->to_new, sizeof(int32_t) * (m > 0 ? m : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->to_old, sizeof(int32_t) * (m > 0 ? m : 1), st, h));
    nd_tmp<int> derr(st);
    ND_TRY(derr.alloc(1));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    if (m > 0) {
        nd_prof_scope ps("relabel", st);
        k_edge_map<<<nd_blocks_for(m, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
            m, h->e_u, h->e_v, h->vto_old, h->c_rp, h->c_col, h->c_nlow, h->c_up, h->to_new, h->to_old, derr);
        ND_CUDA(cudaGetLastError());
    }
    int herr = 0;
    ND_TRY(read_flag(derr, &herr, st));
    if (herr) { nd_set_error("an edge of the relabelled graph is missing from the caller's (internal fault)"); return ND_E_CUDA; }
    nd_release(h->c_rp, st);
    nd_release(h->c_col, st);
    nd_release(h->c_nlow, st);
    nd_release(h->c_up, st);
    h->c_rp = h->c_up = nullptr;
    h->c_col = h->c_nlow = nullptr;
    return ND_OK;
}

nd_status nd_relabel_by_degree(nd_incidence* h, cudaStream_t st) {
    const int64_t n = h->n, nnz = h->nnz;
    if (n >= kRelabelMinVertices) {
        nd_prof_scope ps("relabel", st);
        const int64_t nblocks = (n + kRelabelTile - 1) / kRelabelTile;
        const int64_t cells = (int64_t)(kClasses - 1) * nblocks;
        nd_tmp<int64_t> cnt(st);
        ND_TRY(cnt.alloc(cells + 1));
        ND_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (cells + 1), st));
        k_class_count<<<nblocks, kThreads, 0, st>>>(n, h->rp, cnt, nblocks);
        ND_CUDA(cudaGetLastError());
        ND_TRY(nd_scan_i64(cnt, cells, st));
        ND_TRY(nd_alloc((void**)&h->to_new, sizeof(int32_t) * n, st, h));
        ND_TRY(nd_alloc((void**)&h->to_old, sizeof(int32_t) * n, st, h));
        k_class_scatter<<<nblocks, kThreads, 0, st>>>(n, h->rp, cnt, nblocks, h->to_new, h->to_old);
        ND_CUDA(cudaGetLastError());
        int64_t* nrp = nullptr;
        int32_t* ncol = nullptr;
        ND_TRY(nd_alloc((void**)&nrp, sizeof(int64_t) * (n + 1), st, h));
        ND_CUDA(cudaMemsetAsync(nrp + n, 0, sizeof(int64_t), st));
        k_new_degrees<<<nd_blocks_for(n, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(n, h->rp, h->to_new, nrp);
        ND_CUDA(cudaGetLastError());
        ND_TRY(nd_scan_i64(nrp, n, st));
        ND_TRY(nd_alloc((void**)&ncol, sizeof(int32_t) * (nnz > 0 ? nnz : 1), st, h));
        if (nnz > 0) {
            k_relabel_rows<<<nd_blocks_for(n * 32, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
                n, h->rp, h->col, h->to_new, nrp, ncol);
            ND_CUDA(cudaGetLastError());
            if (h->long_segs > 0) {
                k_relabel_long<<<nd_blocks_for(h->long_segs * 32, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
                    h->rp, h->col, h->to_new, nrp, ncol, h->long_rows, h->long_seg, h->long_count, h->long_segs);
                ND_CUDA(cudaGetLastError());
            }
        }
        nd_release(h->rp, st);
        nd_release(h->col, st);
        h->rp = nrp;
        h->col = ncol;
    }
    release_long_rows(h, st);
    return ND_OK;
}

nd_status nd_permute_i32(const int32_t* idx, const int32_t* in, int32_t* out, int64_t n, bool scatter,
                         cudaStream_t st) {
    if (n == 0) return ND_OK;
    k_permute_i32<<<nd_blocks_for(n, kThreads, 152 * 8), kThreads, 0, st>>>(n, idx, in, out, scatter ? 1 : 0);
    ND_CUDA(cudaGetLastError());
    return ND_OK;
}

nd_status nd_build_edges(nd_incidence* h, cudaStream_t st) {
    if (h->m >= (int64_t)UINT32_MAX) { nd_set_error("more than 2^32-1 edges"); return ND_E_TOO_LARGE; }
    ND_TRY(nd_alloc((void**)&h->eid, sizeof(uint32_t) * (h->nnz > 0 ? h->nnz : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->e_u, sizeof(int32_t) * (h->m > 0 ? h->m : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->e_v, sizeof(int32_t) * (h->m > 0 ? h->m : 1), st, h));
    if (h->r == 2) {
        // (2,3) incidence entries are CSR positions (uint32)
        if (h->nnz >= (int64_t)UINT32_MAX) {
            nd_set_error("(2,3) needs fewer than 2^32-1 CSR entries");
            return ND_E_TOO_LARGE;
        }
        h->adj = true;
        ND_TRY(nd_alloc((void**)&h->e_pos, sizeof(uint2) * (h->m > 0 ? h->m : 1), st, h));
    }
    if (h->n > 0 && h->nnz > 0) {
        nd_prof_scope ps("edge_ids", st);
        int blocks = nd_blocks_for(h->n * 32, kThreads, grid_cap(h) * 4);
        k_edge_ids<<<blocks, kThreads, 0, st>>>(h->n, h->rp, h->col, h->nlow, h->up_start, h->eid,
                                                h->e_u, h->e_v, h->mirror, h->e_pos);
        ND_CUDA(cudaGetLastError());
        if (h->long_segs > 0) {
            k_edge_ids_long<<<nd_blocks_for(h->long_segs * 32, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(
                h->rp, h->col, h->nlow, h->up_start, h->eid, h->e_u, h->e_v, h->mirror, h->e_pos, h->long_rows,
                h->long_seg, h->long_count, h->long_segs);
            ND_CUDA(cudaGetLastError());
        }
    }
    release_long_rows(h, st);
    if (!h->adj && h->mirror) {  // only the (2,3) build needs it further
        nd_release(h->mirror, st);
        h->mirror = nullptr;
    }
    return ND_OK;
}

// oriented out-lists (degree order), used by the (2,3) and (3,4) builds
struct nd_oriented {
    nd_tmp<int64_t> out_ptr;
    nd_tmp<int32_t> out_col, out_src;
    nd_tmp<uint32_t> out_eid, out_pos, out_mir;
    explicit nd_oriented(cudaStream_t st)
        : out_ptr(st), out_col(st), out_src(st), out_eid(st), out_pos(st), out_mir(st) {}
};

static nd_status orient_graph(nd_incidence* h, nd_oriented* o, cudaStream_t st) {
    const int64_t n = h->n, m = h->m;
    ND_TRY(o->out_ptr.alloc(n + 1));
    ND_TRY(o->out_col.alloc(m));
    ND_TRY(o->out_src.alloc(m));
    ND_TRY(o->out_eid.alloc(m));
    const bool positions = h->adj && !h->otf;  // only the stored (2,3) fill uses them
    if (positions) {
        ND_TRY(o->out_pos.alloc(m));
        ND_TRY(o->out_mir.alloc(m));
    }
    ND_CUDA(cudaMemsetAsync(o->out_ptr.p + n, 0, sizeof(int64_t), st));
    const int vblocks = nd_blocks_for(n * 32, kThreads, grid_cap(h) * 4);
    if (n > 0) {
        nd_prof_scope ps("orient", st);
        k_orient<false><<<vblocks, kThreads, 0, st>>>(n, h->rp, h->col, h->eid, o->out_ptr, nullptr, nullptr, nullptr,
                                                      nullptr, nullptr, nullptr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(o->out_ptr, n, st));
    if (n > 0) {
        nd_prof_scope ps("orient", st);
        k_orient<true><<<vblocks, kThreads, 0, st>>>(n, h->rp, h->col, h->eid, o->out_ptr, o->out_col, o->out_eid,
                                                     o->out_src, h->mirror, positions ? o->out_pos.p : nullptr,
                                                     o->out_mir);
        ND_CUDA(cudaGetLastError());
    }
    return ND_OK;
}

// order the rows of the (2,3) adjacency layout by w (see k_row_rank); if
// the second buffer does not fit, the rows stay in fill order (the h-index
// does not depend on it; the gathers are only less local)
static nd_status sort_tri_rows(nd_incidence* h, cudaStream_t st) {
    const int64_t N = h->num_r, M = h->num_inc;
    uint2* dst = nullptr;
    if (cudaMallocAsync((void**)&dst, sizeof(uint2) * (size_t)M, st) != cudaSuccess) {
        cudaGetLastError();
        return ND_OK;
    }
    nd_tmp<uint32_t> over(st);
    nd_tmp<unsigned long long> over_ctr(st);
    nd_status rc = over.alloc(N);
    if (rc == ND_OK) rc = over_ctr.alloc(2);
    if (rc != ND_OK) { cudaFreeAsync(dst, st); return rc; }
    ND_CUDA(cudaMemsetAsync(over_ctr, 0, sizeof(unsigned long long) * 2, st));
    const size_t smem = sizeof(uint32_t) * 2 * kRankWords * kRankWarps;
    ND_CUDA(cudaFuncSetAttribute(k_row_rank<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        nd_prof_scope ps("row_rank", st);
        const int blocks = nd_blocks_for(N * 32, 32 * kRankWarps, grid_cap(h) * 8);
        k_row_rank<false><<<blocks, 32 * kRankWarps, smem, st>>>(N, h->inc_ptr, h->e_u, h->e_v, h->rp,
                                                                  (const uint2*)h->inc, dst, over, over_ctr,
                                                                  nullptr, 0);
        ND_CUDA(cudaGetLastError());
    }
    unsigned long long hc[2] = {0, 0};
    ND_CUDA(cudaMemcpyAsync(hc, over_ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    if (hc[0] > 0) {
        // rows whose shorter adjacency list needs more than kRankWords words
        const int warps = 64;
        nd_tmp<uint32_t> scratch(st);
        ND_TRY(scratch.alloc((int64_t)2 * (int64_t)hc[1] * warps));
        nd_prof_scope ps("row_rank", st);
        k_row_rank<true><<<warps / kRankWarps, 32 * kRankWarps, 0, st>>>(
            N, h->inc_ptr, h->e_u, h->e_v, h->rp, (const uint2*)h->inc, dst, over, over_ctr, scratch,
            (int64_t)hc[1]);
        ND_CUDA(cudaGetLastError());
    }
    nd_release(h->inc, st);
    h->inc = reinterpret_cast<uint32_t*>(dst);
    h->rows_sorted = true;
    return ND_OK;
}

nd_status nd_build_tri_incidence(nd_incidence* h, cudaStream_t st) {
    const int64_t m = h->m;
    h->num_r = m;
    ND_TRY(nd_alloc((void**)&h->inc_ptr, sizeof(int64_t) * (m + 1), st, h));
    ND_CUDA(cudaMemsetAsync(h->inc_ptr, 0, sizeof(int64_t) * (m + 1), st));
    if (m == 0) { h->num_inc = 0; ND_TRY(nd_alloc((void**)&h->inc, 16, st, h)); return ND_OK; }
    nd_oriented o(st);
    ND_TRY(orient_graph(h, &o, st));
    const int eblocks = nd_blocks_for(m * 32, kThreads, grid_cap(h) * 4);
    // the stored adjacency layout keeps the count pass's triangles as records
    // (4 B each, min(|out(u)|, |out(v)|) slots reserved per oriented edge), so
    // that the fill does not search again; without the memory for them the
    // fill searches as the count pass does
    nd_tmp<int64_t> rec_ptr(st);
    nd_tmp<uint32_t> rec(st), rec_cnt(st);
    bool use_rec = false;
    if (h->adj && !h->otf && rec_ptr.alloc(m + 1) == ND_OK) {
        k_rec_bound<<<nd_blocks_for(m, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(m, o.out_ptr, o.out_src,
                                                                                     o.out_col, rec_ptr);
        ND_CUDA(cudaGetLastError());
        ND_CUDA(cudaMemsetAsync(rec_ptr.p + m, 0, sizeof(int64_t), st));
        ND_TRY(nd_scan_i64(rec_ptr, m, st));
        int64_t slots = 0;
        ND_TRY(read_i64(rec_ptr.p + m, &slots, st));
        use_rec = rec.alloc(slots) == ND_OK && rec_cnt.alloc(m) == ND_OK;
        if (!use_rec) nd_set_error("");
    }
    {
        // per-edge counts fit 32 bits (d_s < n); 32-bit atomics, widened for the scan
        nd_tmp<unsigned> cnt32(st);
        ND_TRY(cnt32.alloc(m));
        ND_CUDA(cudaMemsetAsync(cnt32, 0, sizeof(unsigned) * m, st));
        nd_prof_scope ps("tri_count", st, 2);
        if (use_rec)
            k_tri_oriented<false, false, unsigned, true><<<eblocks, kThreads, 0, st>>>(
                m, o.out_ptr, o.out_col, o.out_eid, o.out_src, nullptr, nullptr, cnt32.p, nullptr, rec_ptr, rec,
                rec_cnt);
        else
            k_tri_oriented<false, false, unsigned><<<eblocks, kThreads, 0, st>>>(m, o.out_ptr, o.out_col, o.out_eid,
                                                                                 o.out_src, nullptr, nullptr, cnt32.p,
                                                                                 nullptr);
        ND_CUDA(cudaGetLastError());
        k_widen_u32<<<nd_blocks_for(m, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(m, cnt32, h->inc_ptr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(h->inc_ptr, m, st));
    ND_TRY(read_i64(h->inc_ptr + m, &h->num_inc, st));
    if (h->otf) {
        // no stored incidence: the counts (d_s, tau_0 and the buckets) are all
        // that is kept; every pass finds the triangles again
        nd_release(h->mirror, st);
        h->mirror = nullptr;
        return nd_alloc((void**)&h->inc, 16, st, h);
    }
    ND_TRY(nd_alloc((void**)&h->inc, sizeof(uint32_t) * 2 * (h->num_inc > 0 ? h->num_inc : 1), st, h));
    if (h->num_inc > 0) {
        nd_tmp<unsigned long long> cursor(st);
        nd_tmp<unsigned> cursor32(st);
        const bool narrow = h->adj && h->num_inc < (int64_t)UINT32_MAX;  // 32-bit slot atomics
        if (narrow) {
            ND_TRY(cursor32.alloc(m));
            k_narrow_u32<<<nd_blocks_for(m, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(m, h->inc_ptr, cursor32);
            ND_CUDA(cudaGetLastError());
        } else {
            ND_TRY(cursor.alloc(m));
            ND_CUDA(cudaMemcpyAsync(cursor, h->inc_ptr, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, st));
        }
        nd_prof_scope ps("tri_fill", st);
        if (use_rec && narrow)
            k_tri_fill_rec<unsigned><<<eblocks, kThreads, 0, st>>>(m, o.out_ptr, o.out_col, o.out_eid, o.out_src,
                                                                   o.out_pos, o.out_mir, cursor32.p, (uint2*)h->inc,
                                                                   rec_ptr, rec, rec_cnt);
        else if (use_rec)
            k_tri_fill_rec<unsigned long long><<<eblocks, kThreads, 0, st>>>(
                m, o.out_ptr, o.out_col, o.out_eid, o.out_src, o.out_pos, o.out_mir, cursor.p, (uint2*)h->inc, rec_ptr,
                rec, rec_cnt);
        else if (narrow)
            k_tri_oriented<true, true, unsigned><<<eblocks, kThreads, 0, st>>>(
                m, o.out_ptr, o.out_col, o.out_eid, o.out_src, o.out_pos, o.out_mir, cursor32.p, (uint2*)h->inc);
        else if (h->adj)
            k_tri_oriented<true, true><<<eblocks, kThreads, 0, st>>>(m, o.out_ptr, o.out_col, o.out_eid, o.out_src,
                                                                     o.out_pos, o.out_mir, cursor.p, (uint2*)h->inc);
        else
            k_tri_oriented<true, false><<<eblocks, kThreads, 0, st>>>(m, o.out_ptr, o.out_col, o.out_eid,
                                                                      o.out_src, nullptr, nullptr, cursor.p,
                                                                      (uint2*)h->inc);
        ND_CUDA(cudaGetLastError());
    }
    // the records are no longer needed: free them before the row ranking
    // takes its second incidence buffer
    nd_release(rec.p, st);
    rec.p = nullptr;
    if (h->adj) {
        nd_release(h->mirror, st);  // build only
        h->mirror = nullptr;
        if (h->num_inc > 0) ND_TRY(sort_tri_rows(h, st));
    }
    return ND_OK;
}

nd_status nd_build_triangles(nd_incidence* h, cudaStream_t st) {
    ND_TRY(nd_alloc((void**)&h->tri_ptr, sizeof(int64_t) * (h->m + 1), st, h));
    ND_CUDA(cudaMemsetAsync(h->tri_ptr, 0, sizeof(int64_t) * (h->m + 1), st));
    int blocks = nd_blocks_for(h->m * 32, kThreads, grid_cap(h) * 4);
    if (h->m > 0) {
        nd_prof_scope ps("tri_list_count", st);
        k_triangle_list<false><<<blocks, kThreads, 0, st>>>(h->m, h->rp, h->col, h->nlow, h->up_start,
                                                            h->e_u, h->e_v, h->tri_ptr, nullptr,
                                                            nullptr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(h->tri_ptr, h->m, st));
    ND_TRY(read_i64(h->tri_ptr + h->m, &h->num_tri, st));
    if (h->num_tri >= (int64_t)UINT32_MAX) { nd_set_error("more than 2^32-1 triangles"); return ND_E_TOO_LARGE; }
    ND_TRY(nd_alloc((void**)&h->tri_w, sizeof(int32_t) * (h->num_tri > 0 ? h->num_tri : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->tri_e, sizeof(uint32_t) * (h->num_tri > 0 ? h->num_tri : 1), st, h));
    if (h->num_tri > 0) {
        nd_prof_scope ps("tri_list_fill", st);
        k_triangle_list<true><<<blocks, kThreads, 0, st>>>(h->m, h->rp, h->col, h->nlow, h->up_start,
                                                           h->e_u, h->e_v, h->tri_ptr, h->tri_w,
                                                           h->tri_e);
        ND_CUDA(cudaGetLastError());
    }
    return ND_OK;
}

nd_status nd_build_k4_incidence(nd_incidence* h, cudaStream_t st) {
    const int64_t T = h->num_tri, m = h->m;
    h->num_r = T;
    ND_TRY(nd_alloc((void**)&h->inc_ptr, sizeof(int64_t) * (T + 1), st, h));
    ND_CUDA(cudaMemsetAsync(h->inc_ptr, 0, sizeof(int64_t) * (T + 1), st));
    if (T == 0) { h->num_inc = 0; ND_TRY(nd_alloc((void**)&h->inc, 16, st, h)); return ND_OK; }
    nd_oriented o(st);
    ND_TRY(orient_graph(h, &o, st));
    nd_tmp<int64_t> optr(st), kptr(st);  // oriented triangles per oriented edge; 4-cliques per triangle
    nd_tmp<otri> tris(st);
    nd_tmp<int> derr(st);
    ND_TRY(optr.alloc(m + 1));
    ND_TRY(kptr.alloc(T + 1));
    ND_TRY(tris.alloc(T));
    ND_TRY(derr.alloc(1));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    ND_CUDA(cudaMemsetAsync(optr.p + m, 0, sizeof(int64_t), st));
    ND_CUDA(cudaMemsetAsync(kptr.p + T, 0, sizeof(int64_t), st));
    const int eblocks = nd_blocks_for(m * 32, kThreads, grid_cap(h) * 4);
    const int tblocks = nd_blocks_for(T * 32, kThreads, grid_cap(h) * 4);
    {
        nd_prof_scope ps("otri", st);
        k_otri<false><<<eblocks, kThreads, 0, st>>>(m, o.out_ptr, o.out_col, o.out_eid, o.out_src, optr, nullptr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(optr, m, st));
    {
        nd_prof_scope ps("otri", st);
        k_otri<true><<<eblocks, kThreads, 0, st>>>(m, o.out_ptr, o.out_col, o.out_eid, o.out_src, optr, tris);
        ND_CUDA(cudaGetLastError());
    }
    {
        nd_prof_scope ps("k4_count", st);
        k_k4<0><<<tblocks, kThreads, 0, st>>>(T, tris, o.out_ptr, o.out_col, o.out_eid, h->tri_ptr, h->tri_w,
                                              kptr, nullptr, nullptr, derr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(kptr, T, st));
    int64_t K = 0;
    ND_TRY(read_i64(kptr.p + T, &K, st));
    nd_tmp<uint4> k4(st);
    ND_TRY(k4.alloc(K));
    if (K > 0) {
        nd_prof_scope ps("k4_list", st);
        k_k4<1><<<tblocks, kThreads, 0, st>>>(T, tris, o.out_ptr, o.out_col, o.out_eid, h->tri_ptr, h->tri_w,
                                              kptr, k4, (unsigned long long*)h->inc_ptr, derr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(h->inc_ptr, T, st));
    ND_TRY(read_i64(h->inc_ptr + T, &h->num_inc, st));
    ND_TRY(nd_alloc((void**)&h->inc, sizeof(uint32_t) * 3 * (h->num_inc > 0 ? h->num_inc : 1), st, h));
    if (K > 0) {
        nd_prof_scope ps("k4_fill", st);
        const int kb = nd_blocks_for(K, kThreads, grid_cap(h) * 4);
        if (h->num_inc < (int64_t)UINT32_MAX) {  // 32-bit slot atomics
            nd_tmp<unsigned> cursor(st);
            ND_TRY(cursor.alloc(T));
            k_narrow_u32<<<nd_blocks_for(T, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(T, h->inc_ptr, cursor);
            ND_CUDA(cudaGetLastError());
            k_k4_scatter<unsigned><<<kb, kThreads, 0, st>>>(K, k4, cursor.p, h->inc);
        } else {
            nd_tmp<unsigned long long> cursor(st);
            ND_TRY(cursor.alloc(T));
            ND_CUDA(cudaMemcpyAsync(cursor, h->inc_ptr, sizeof(int64_t) * T, cudaMemcpyDeviceToDevice, st));
            k_k4_scatter<unsigned long long><<<kb, kThreads, 0, st>>>(K, k4, cursor.p, h->inc);
        }
        ND_CUDA(cudaGetLastError());
    }
    int herr = 0;
    ND_TRY(read_flag(derr, &herr, st));
    if (herr) { nd_set_error("internal: a triangle of a 4-clique was not found"); return ND_E_INVAL; }
    return ND_OK;
}

nd_status nd_build_buckets(nd_incidence* h, cudaStream_t st) {
    const int64_t N = h->num_r;
    // pass graphs hold the bucket ranges of the old buckets
    for (auto& row : h->pass_graph)
        for (auto& ex : row)
            if (ex) { cudaGraphExecDestroy(ex); ex = nullptr; }
    const int3 thr = make_int3(h->thr[0], h->thr[1], h->thr[2]);
    nd_tmp<int64_t> flags(st);
    nd_tmp<unsigned long long> sums(st);
    ND_TRY(flags.alloc(N + 1));
    ND_TRY(sums.alloc(ND_NB));
    ND_CUDA(cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * ND_NB, st));
    if (!h->items) ND_TRY(nd_alloc((void**)&h->items, sizeof(nd_item) * (N > 0 ? N : 1), st, h));
    int blocks = nd_blocks_for(N, kThreads, grid_cap(h) * 2);
    int64_t lo = 0;
    for (int b = 0; b < ND_NB; ++b) {
        h->bucket_lo[b] = lo;
        if (N == 0) continue;
        ND_CUDA(cudaMemsetAsync(flags.p + N, 0, sizeof(int64_t), st));
        {
            nd_prof_scope ps("buckets", st);
            k_bucket_flags<<<blocks, kThreads, 0, st>>>(N, h->inc_ptr, b, thr, flags, sums.p + b);
            ND_CUDA(cudaGetLastError());
        }
        ND_TRY(nd_scan_i64(flags, N, st));
        {
            nd_prof_scope ps("buckets", st);
            k_bucket_scatter<<<blocks, kThreads, 0, st>>>(N, h->inc_ptr, b, thr, flags, h->items + lo);
            ND_CUDA(cudaGetLastError());
        }
        int64_t cnt = 0;
        ND_TRY(read_i64(flags.p + N, &cnt, st));
        lo += cnt;
    }
    h->bucket_lo[ND_NB] = lo;
    unsigned long long hs[ND_NB] = {0, 0, 0, 0};
    ND_CUDA(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    for (int b = 0; b < ND_NB; ++b) h->bucket_inc[b] = (int64_t)hs[b];
    h->num_zero = N - lo;
    return ND_OK;
}

nd_status nd_write_r_cliques(const nd_incidence* h, int32_t* out_dev, cudaStream_t st) {
    if (h->num_r == 0) return ND_OK;
    int blocks = nd_blocks_for(h->num_r, kThreads, grid_cap(h) * 2);
    nd_prof_scope ps("r_cliques", st);
    if (h->r == 2 && h->vto_old)
        k_r_cliques_mapped<<<blocks, kThreads, 0, st>>>(h->num_r, h->e_u, h->e_v, h->vto_old, h->to_old, out_dev);
    else
        k_r_cliques<<<blocks, kThreads, 0, st>>>(h->r, h->num_r, h->e_u, h->e_v, h->tri_w, h->tri_e, out_dev);
    ND_CUDA(cudaGetLastError());
    return ND_OK;
}

nd_status nd_union_device(const nd_union_part* parts_host, int count, int64_t n, int64_t nnz, int64_t* urp,
                          int32_t* ucol, cudaStream_t st) {
    nd_tmp<nd_union_part> dparts(st);
    nd_tmp<int> derr(st);
    ND_TRY(dparts.alloc(count));
    ND_TRY(derr.alloc(1));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    if (count > 0)
        ND_CUDA(cudaMemcpyAsync(dparts, parts_host, sizeof(nd_union_part) * count, cudaMemcpyHostToDevice, st));
    if (count > 0) {
        nd_prof_scope ps("union", st);
        k_union<<<count < 152 * 16 ? count : 152 * 16, kThreads, 0, st>>>(dparts, count, urp, ucol, derr);
        ND_CUDA(cudaGetLastError());
    }
    ND_CUDA(cudaMemcpyAsync(urp + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    int herr = 0;
    ND_TRY(read_flag(derr, &herr, st));
    if (herr) {
        nd_set_error(herr & 1 ? "a graph of the batch has an invalid row_ptr"
                              : "a graph of the batch has a neighbour id outside its own vertex range");
        return ND_E_INVAL;
    }
    return ND_OK;
}

// r-clique offsets of the graphs of a batch: the union's canonical order
// lists graph 0's r-cliques first, then graph 1's, and so on.
nd_status nd_batch_offsets(const nd_incidence* h, const int64_t* vertex_off /* count+1, host */, int count,
                           int64_t* r_off /* count+1, host */, cudaStream_t st) {
    if (h->r == 1) {
        for (int i = 0; i <= count; ++i) r_off[i] = vertex_off[i];
        return ND_OK;
    }
    nd_tmp<int64_t> didx(st), dout(st);
    ND_TRY(didx.alloc(count + 1));
    ND_TRY(dout.alloc(count + 1));
    ND_CUDA(cudaMemcpyAsync(didx, vertex_off, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
    // edges owned by vertices below the graph's first vertex
    k_gather_i64<<<nd_blocks_for(count + 1, kThreads, 64), kThreads, 0, st>>>(h->up_start, didx, count + 1, dout);
    ND_CUDA(cudaGetLastError());
    const int64_t* res = dout;
    if (h->r == 3) {
        // triangles owned by those edges
        k_gather_i64<<<nd_blocks_for(count + 1, kThreads, 64), kThreads, 0, st>>>(h->tri_ptr, dout, count + 1, didx);
        ND_CUDA(cudaGetLastError());
        res = didx;
    }
    ND_CUDA(cudaMemcpyAsync(r_off, res, sizeof(int64_t) * (count + 1), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    return ND_OK;
}

nd_status nd_batch_graph_ids(nd_incidence* h, const int64_t* r_off, int count, cudaStream_t st) {
    if (count < 2 || h->num_r == 0) return ND_OK;  // one graph: nothing to skip
    nd_tmp<int64_t> doff(st);
    ND_TRY(doff.alloc(count + 1));
    ND_CUDA(cudaMemcpyAsync(doff, r_off, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
    ND_TRY(nd_alloc((void**)&h->gid, sizeof(uint32_t) * h->num_r, st, h));
    k_graph_ids<<<nd_blocks_for(h->num_r, kThreads, grid_cap(h) * 4), kThreads, 0, st>>>(h->num_r, doff, count,
                                                                                         h->to_new, h->gid);
    ND_CUDA(cudaGetLastError());
    h->ngraphs = count;
    return nd_wait(st);  // the offsets are a host array
}
