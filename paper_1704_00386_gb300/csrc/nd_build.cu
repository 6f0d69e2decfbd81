// Incidence construction: r-clique -> s-clique incidence as CSR (Def. 1).
//
// The paper discovers the s-cliques of an r-clique through the
// neighbourhoods of its vertices (Section 4.1, "Time complexity": all
// (s-r)-tuples of a neighbourhood), and recomputes them on every pass.  Here
// they are found once, by sorted-list intersection, and stored:
//   (1,2)  the CSR itself is the incidence (q = 1);
//   (2,3)  triangle {u,v,w} -> one pair per edge: the ids of its other two
//          edges (found once each, by degree orientation);
//   (3,4)  triangle (u,v,w): x in N(u) /\ N(v) /\ N(w) -> the ids of the
//          triangles {u,v,x}, {u,w,x}, {v,w,x}.
// Every step is a count pass, an exclusive scan and a fill pass over the same
// enumeration.  Intersections: one warp per list pair; the lanes walk the
// shorter list in order and binary-search each element in the other list(s)
// (read-only path).
#include "nd_internal.cuh"

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
// A row must lie inside [0, nnz], be strictly increasing, hold ids in [0, n)
// other than its own, and every entry v of row u needs u in row v.  Writes
// nlow[u] = #neighbours < u and upcnt[u] = #neighbours > u.  Reads only
// inside the bounds it has checked, so a malformed graph cannot fault.
__global__ void k_validate_split(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                 const int32_t* __restrict__ col, int32_t* __restrict__ nlow,
                                 int64_t* __restrict__ upcnt, int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    for (int64_t u = warp_id_global(); u < n; u += warp_count_global()) {
        int64_t b = rp[u], e = rp[u + 1];
        bool bad = (b < 0) || (e < b) || (e > nnz) || (u == 0 && b != 0) || (u == n - 1 && e != nnz);
        if (bad) {
            if (lane == 0) { atomicOr(err, 1); nlow[u] = 0; upcnt[u] = 0; }
            continue;
        }
        int low = 0;
        bool rowbad = false;
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t v = col[p];
            if (v < 0 || v >= n || v == u) { rowbad = true; continue; }
            if (p > b && col[p - 1] >= v) rowbad = true;
            low += (v < u);
            int64_t vb = rp[v], ve = rp[v + 1];
            if (vb < 0 || ve < vb || ve > nnz) { rowbad = true; continue; }
            int64_t pos = lower_bound_i32(col, vb, ve, (int32_t)u);
            if (pos >= ve || col[pos] != (int32_t)u) rowbad = true;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) low += __shfl_xor_sync(kFull, low, o);
        rowbad = __any_sync(kFull, rowbad);
        if (lane == 0) {
            nlow[u] = low;
            upcnt[u] = (e - b) - low;
            if (rowbad) atomicOr(err, 2);
        }
    }
}

// ---- canonical edge ids (one warp per vertex) ------------------------------
// Edge (u,v), u < v, gets id up_start[u] + (rank of v among u's larger
// neighbours): lexicographic order.  eid[p] is the id of the edge at CSR
// position p, for both directions.
__global__ void k_edge_ids(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ nlow, const int64_t* __restrict__ up_start,
                           uint32_t* __restrict__ eid, int32_t* __restrict__ e_u,
                           int32_t* __restrict__ e_v) {
    const int lane = threadIdx.x & 31;
    for (int64_t u = warp_id_global(); u < n; u += warp_count_global()) {
        const int64_t b = rp[u], e = rp[u + 1];
        const int64_t first_up = b + nlow[u];
        const int64_t base = up_start[u];
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t v = col[p];
            if (p >= first_up) {
                int64_t id = base + (p - first_up);
                eid[p] = (uint32_t)id;
                e_u[id] = (int32_t)u;
                e_v[id] = v;
            } else {
                int64_t vfirst = rp[v] + nlow[v];
                int64_t pos = lower_bound_i32(col, vfirst, rp[v + 1], (int32_t)u);
                eid[p] = (uint32_t)(up_start[v] + (pos - vfirst));
            }
        }
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
template <bool FILL>
__global__ void k_orient(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const uint32_t* __restrict__ eid, int64_t* __restrict__ out_ptr,
                         int32_t* __restrict__ out_col, uint32_t* __restrict__ out_eid,
                         int32_t* __restrict__ out_src) {
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
            }
            cnt += __popc(bal);
        }
        if (!FILL && lane == 0) out_ptr[u] = cnt;
    }
}

// one warp per oriented edge u -> v: the triangles {u, v, w}, w in out(u) /\ out(v)
template <bool FILL>
__global__ void k_tri_oriented(int64_t m, const int64_t* __restrict__ out_ptr,
                               const int32_t* __restrict__ out_col, const uint32_t* __restrict__ out_eid,
                               const int32_t* __restrict__ out_src, unsigned long long* __restrict__ ctr,
                               uint2* __restrict__ inc) {
    const int lane = threadIdx.x & 31;
    for (int64_t k = warp_id_global(); k < m; k += warp_count_global()) {
        const int32_t u = out_src[k], v = out_col[k];
        const uint32_t e_uv = out_eid[k];
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
            if (p < ae) {
                const int32_t x = __ldg(out_col + p);
                pb = lower_bound_i32(out_col, lo, be, x);
                found = (pb < be) && (__ldg(out_col + pb) == x);
            }
            const unsigned bal = __ballot_sync(kFull, found);
            const int nf = __popc(bal);
            if (nf) {
                uint32_t e_uw = 0, e_vw = 0;
                if (found) {
                    const uint32_t ea = __ldg(out_eid + p), eb = __ldg(out_eid + pb);
                    e_uw = a_is_u ? ea : eb;
                    e_vw = a_is_u ? eb : ea;
                }
                if (!FILL) {
                    if (lane == 0) atomicAdd(ctr + e_uv, (unsigned long long)nf);
                    if (found) {
                        atomicAdd(ctr + e_uw, 1ull);
                        atomicAdd(ctr + e_vw, 1ull);
                    }
                } else {
                    unsigned long long s0 = 0;
                    if (lane == 0) s0 = atomicAdd(ctr + e_uv, (unsigned long long)nf);
                    s0 = __shfl_sync(kFull, s0, 0);
                    if (found) {
                        inc[s0 + __popc(bal & lanemask_lt())] = make_uint2(e_uw, e_vw);
                        inc[atomicAdd(ctr + e_uw, 1ull)] = make_uint2(e_uv, e_vw);
                        inc[atomicAdd(ctr + e_vw, 1ull)] = make_uint2(e_uv, e_uw);
                    }
                }
            }
            const int64_t last_pb = __shfl_sync(kFull, pb, 31);
            if (base + 32 <= ae) lo = last_pb;
        }
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

// id of triangle {a, b, x} where a < b are two vertices of the current
// triangle, pa / pb the positions of x in rows a / b and e_ab the id of edge
// (a,b).  Sorted, the triangle's smallest edge is (x,a) if x < a, (a,x) if
// a < x < b, and (a,b) if x > b; its third vertex is b, b, x.
__device__ __forceinline__ uint32_t tri_lookup(int32_t a, int32_t b, int32_t x, int64_t pa,
                                               uint32_t e_ab, const uint32_t* __restrict__ eid,
                                               const int64_t* __restrict__ tri_ptr,
                                               const int32_t* __restrict__ tri_w, bool* ok) {
    uint32_t edge;
    int32_t third;
    if (x < b) { edge = __ldg(eid + pa); third = b; }
    else { edge = e_ab; third = x; }
    (void)a;
    int64_t lo = __ldg(tri_ptr + edge), hi = __ldg(tri_ptr + edge + 1);
    int64_t pos = lower_bound_i32(tri_w, lo, hi, third);
    if (pos >= hi || __ldg(tri_w + pos) != third) { *ok = false; return 0; }
    return (uint32_t)pos;
}

// ---- (3,4) step 2: 4-cliques of every triangle (one warp per triangle) -----
template <bool FILL>
__global__ void k_triangle_k4(int64_t T, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const uint32_t* __restrict__ eid, const int32_t* __restrict__ e_u,
                              const int32_t* __restrict__ e_v, const int64_t* __restrict__ tri_ptr,
                              const int32_t* __restrict__ tri_w, const uint32_t* __restrict__ tri_e,
                              int64_t* __restrict__ ptr, uint32_t* __restrict__ inc,
                              int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    for (int64_t t = warp_id_global(); t < T; t += warp_count_global()) {
        const uint32_t e = tri_e[t];
        const int32_t vtx[3] = {e_u[e], e_v[e], tri_w[t]};  // u < v < w
        int64_t rb[3], re[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) { rb[i] = rp[vtx[i]]; re[i] = rp[vtx[i] + 1]; }
        int A = 0;
        if (re[1] - rb[1] < re[A] - rb[A]) A = 1;
        if (re[2] - rb[2] < re[A] - rb[A]) A = 2;
        const int B1 = (A == 0) ? 1 : 0, B2 = (A == 2) ? 1 : 2;
        uint32_t e_uw = 0, e_vw = 0;
        if (FILL) {  // ids of edges (u,w) and (v,w): positions of w in rows u and v
            int64_t p1 = lower_bound_i32(col, rb[0], re[0], vtx[2]);
            int64_t p2 = lower_bound_i32(col, rb[1], re[1], vtx[2]);
            e_uw = __ldg(eid + p1);
            e_vw = __ldg(eid + p2);
        }
        int64_t out = FILL ? ptr[t] : 0;
        int64_t cnt = 0;
        bool ok = true;
        for (int64_t base = rb[A]; base < re[A]; base += 32) {
            int64_t p = base + lane;
            bool found = false;
            int64_t pos[3] = {0, 0, 0};
            int32_t x = 0;
            if (p < re[A]) {
                x = __ldg(col + p);
                pos[A] = p;
                pos[B1] = lower_bound_i32(col, rb[B1], re[B1], x);
                if (pos[B1] < re[B1] && __ldg(col + pos[B1]) == x) {
                    pos[B2] = lower_bound_i32(col, rb[B2], re[B2], x);
                    found = (pos[B2] < re[B2]) && (__ldg(col + pos[B2]) == x);
                }
            }
            unsigned bal = __ballot_sync(kFull, found);
            if (FILL && found) {
                int64_t slot = out + cnt + __popc(bal & lanemask_lt());
                uint32_t* dst = inc + 3 * slot;
                dst[0] = tri_lookup(vtx[0], vtx[1], x, pos[0], e, eid, tri_ptr, tri_w, &ok);
                dst[1] = tri_lookup(vtx[0], vtx[2], x, pos[0], e_uw, eid, tri_ptr, tri_w, &ok);
                dst[2] = tri_lookup(vtx[1], vtx[2], x, pos[1], e_vw, eid, tri_ptr, tri_w, &ok);
            }
            cnt += __popc(bal);
        }
        if (FILL && !ok) atomicOr(err, 4);
        if (!FILL && lane == 0) ptr[t] = cnt;
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
    ND_CUDA(cudaStreamSynchronize(st));
    return ND_OK;
}

nd_status read_i64(const int64_t* d, int64_t* hv, cudaStream_t st) {
    ND_CUDA(cudaMemcpyAsync(hv, d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    return ND_OK;
}

}  // namespace

// Copy the caller's CSR into owned device buffers, validate it, split each
// row at its own vertex and derive the canonical edge numbering offsets.
nd_status nd_build_graph(nd_incidence* h, const nd_csr* g, cudaStream_t st) {
    h->n = g->n;
    h->nnz = g->nnz;
    ND_TRY(nd_alloc((void**)&h->rp, sizeof(int64_t) * (g->n + 1), st, h));
    ND_TRY(nd_alloc((void**)&h->col, sizeof(int32_t) * (g->nnz > 0 ? g->nnz : 1), st, h));
    cudaMemcpyKind kind = g->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ND_CUDA(cudaMemcpyAsync(h->rp, g->row_ptr, sizeof(int64_t) * (g->n + 1), kind, st));
    if (g->nnz > 0) ND_CUDA(cudaMemcpyAsync(h->col, g->col, sizeof(int32_t) * g->nnz, kind, st));
    ND_TRY(nd_alloc((void**)&h->nlow, sizeof(int32_t) * (g->n > 0 ? g->n : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->up_start, sizeof(int64_t) * (g->n + 1), st, h));
    int* derr = nullptr;
    ND_CUDA(cudaMallocAsync((void**)&derr, sizeof(int), st));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    ND_CUDA(cudaMemsetAsync(h->up_start, 0, sizeof(int64_t) * (g->n + 1), st));
    if (g->n > 0) {
        nd_prof_scope ps("validate_split", st);
        int blocks = nd_blocks_for(g->n * 32, kThreads, grid_cap(h) * 4);
        k_validate_split<<<blocks, kThreads, 0, st>>>(g->n, g->nnz, h->rp, h->col, h->nlow,
                                                      h->up_start, derr);
        ND_CUDA(cudaGetLastError());
    }
    int herr = 0;
    nd_status s = read_flag(derr, &herr, st);
    cudaFreeAsync(derr, st);
    if (s != ND_OK) return s;
    if (herr) {
        nd_set_error(herr & 1 ? "row_ptr is not a valid offset array"
                              : "col is not simple, sorted and symmetric");
        return ND_E_INVAL;
    }
    ND_TRY(nd_scan_i64(h->up_start, g->n, st));
    int64_t m = 0;
    ND_TRY(read_i64(h->up_start + g->n, &m, st));
    if (2 * m != g->nnz) {
        nd_set_error("edge count is inconsistent with nnz");
        return ND_E_INVAL;
    }
    h->m = m;
    return ND_OK;
}

nd_status nd_build_edges(nd_incidence* h, cudaStream_t st) {
    if (h->m >= (int64_t)UINT32_MAX) { nd_set_error("more than 2^32-1 edges"); return ND_E_TOO_LARGE; }
    ND_TRY(nd_alloc((void**)&h->eid, sizeof(uint32_t) * (h->nnz > 0 ? h->nnz : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->e_u, sizeof(int32_t) * (h->m > 0 ? h->m : 1), st, h));
    ND_TRY(nd_alloc((void**)&h->e_v, sizeof(int32_t) * (h->m > 0 ? h->m : 1), st, h));
    if (h->n > 0 && h->nnz > 0) {
        nd_prof_scope ps("edge_ids", st);
        int blocks = nd_blocks_for(h->n * 32, kThreads, grid_cap(h) * 4);
        k_edge_ids<<<blocks, kThreads, 0, st>>>(h->n, h->rp, h->col, h->nlow, h->up_start, h->eid,
                                                h->e_u, h->e_v);
        ND_CUDA(cudaGetLastError());
    }
    return ND_OK;
}

nd_status nd_build_tri_incidence(nd_incidence* h, cudaStream_t st) {
    const int64_t m = h->m, n = h->n;
    h->num_r = m;
    ND_TRY(nd_alloc((void**)&h->inc_ptr, sizeof(int64_t) * (m + 1), st, h));
    ND_CUDA(cudaMemsetAsync(h->inc_ptr, 0, sizeof(int64_t) * (m + 1), st));
    if (m == 0) { h->num_inc = 0; ND_TRY(nd_alloc((void**)&h->inc, 16, st, h)); return ND_OK; }
    // oriented out-lists (temporary)
    int64_t* out_ptr = nullptr;
    int32_t *out_col = nullptr, *out_src = nullptr;
    uint32_t* out_eid = nullptr;
    unsigned long long* cursor = nullptr;
    ND_CUDA(cudaMallocAsync((void**)&out_ptr, sizeof(int64_t) * (n + 1), st));
    ND_CUDA(cudaMallocAsync((void**)&out_col, sizeof(int32_t) * m, st));
    ND_CUDA(cudaMallocAsync((void**)&out_src, sizeof(int32_t) * m, st));
    ND_CUDA(cudaMallocAsync((void**)&out_eid, sizeof(uint32_t) * m, st));
    ND_CUDA(cudaMemsetAsync(out_ptr + n, 0, sizeof(int64_t), st));
    const int vblocks = nd_blocks_for(n * 32, kThreads, grid_cap(h) * 4);
    {
        nd_prof_scope ps("orient", st);
        k_orient<false><<<vblocks, kThreads, 0, st>>>(n, h->rp, h->col, h->eid, out_ptr, nullptr, nullptr, nullptr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(out_ptr, n, st));
    {
        nd_prof_scope ps("orient", st);
        k_orient<true><<<vblocks, kThreads, 0, st>>>(n, h->rp, h->col, h->eid, out_ptr, out_col, out_eid, out_src);
        ND_CUDA(cudaGetLastError());
    }
    const int eblocks = nd_blocks_for(m * 32, kThreads, grid_cap(h) * 4);
    {
        nd_prof_scope ps("tri_count", st);
        k_tri_oriented<false><<<eblocks, kThreads, 0, st>>>(m, out_ptr, out_col, out_eid, out_src,
                                                            (unsigned long long*)h->inc_ptr, nullptr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(h->inc_ptr, m, st));
    ND_TRY(read_i64(h->inc_ptr + m, &h->num_inc, st));
    ND_TRY(nd_alloc((void**)&h->inc, sizeof(uint32_t) * 2 * (h->num_inc > 0 ? h->num_inc : 1), st, h));
    if (h->num_inc > 0) {
        ND_CUDA(cudaMallocAsync((void**)&cursor, sizeof(unsigned long long) * m, st));
        ND_CUDA(cudaMemcpyAsync(cursor, h->inc_ptr, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, st));
        nd_prof_scope ps("tri_fill", st);
        k_tri_oriented<true><<<eblocks, kThreads, 0, st>>>(m, out_ptr, out_col, out_eid, out_src, cursor,
                                                           (uint2*)h->inc);
        ND_CUDA(cudaGetLastError());
    }
    cudaFreeAsync(out_ptr, st);
    cudaFreeAsync(out_col, st);
    cudaFreeAsync(out_src, st);
    cudaFreeAsync(out_eid, st);
    if (cursor) cudaFreeAsync(cursor, st);
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
    const int64_t T = h->num_tri;
    h->num_r = T;
    ND_TRY(nd_alloc((void**)&h->inc_ptr, sizeof(int64_t) * (T + 1), st, h));
    ND_CUDA(cudaMemsetAsync(h->inc_ptr, 0, sizeof(int64_t) * (T + 1), st));
    int blocks = nd_blocks_for(T * 32, kThreads, grid_cap(h) * 4);
    int* derr = nullptr;
    ND_CUDA(cudaMallocAsync((void**)&derr, sizeof(int), st));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    if (T > 0) {
        nd_prof_scope ps("k4_count", st);
        k_triangle_k4<false><<<blocks, kThreads, 0, st>>>(T, h->rp, h->col, h->eid, h->e_u, h->e_v,
                                                          h->tri_ptr, h->tri_w, h->tri_e, h->inc_ptr,
                                                          nullptr, derr);
        ND_CUDA(cudaGetLastError());
    }
    ND_TRY(nd_scan_i64(h->inc_ptr, T, st));
    ND_TRY(read_i64(h->inc_ptr + T, &h->num_inc, st));
    ND_TRY(nd_alloc((void**)&h->inc, sizeof(uint32_t) * 3 * (h->num_inc > 0 ? h->num_inc : 1), st, h));
    if (h->num_inc > 0) {
        nd_prof_scope ps("k4_fill", st);
        k_triangle_k4<true><<<blocks, kThreads, 0, st>>>(T, h->rp, h->col, h->eid, h->e_u, h->e_v,
                                                         h->tri_ptr, h->tri_w, h->tri_e, h->inc_ptr,
                                                         h->inc, derr);
        ND_CUDA(cudaGetLastError());
    }
    int herr = 0;
    nd_status s = read_flag(derr, &herr, st);
    cudaFreeAsync(derr, st);
    if (s != ND_OK) return s;
    if (herr) { nd_set_error("internal: a triangle of a 4-clique was not found"); return ND_E_INVAL; }
    return ND_OK;
}

nd_status nd_build_buckets(nd_incidence* h, cudaStream_t st) {
    const int64_t N = h->num_r;
    // pass graphs hold the chunk table of the old buckets
    for (auto& row : h->pass_graph)
        for (auto& ex : row)
            if (ex) { cudaGraphExecDestroy(ex); ex = nullptr; }
    const int3 thr = make_int3(h->thr[0], h->thr[1], h->thr[2]);
    int64_t* flags = nullptr;
    unsigned long long* sums = nullptr;
    ND_CUDA(cudaMallocAsync((void**)&flags, sizeof(int64_t) * (N + 1), st));
    ND_CUDA(cudaMallocAsync((void**)&sums, sizeof(unsigned long long) * ND_NB, st));
    ND_CUDA(cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * ND_NB, st));
    if (!h->items) ND_TRY(nd_alloc((void**)&h->items, sizeof(nd_item) * (N > 0 ? N : 1), st, h));
    int blocks = nd_blocks_for(N, kThreads, grid_cap(h) * 2);
    int64_t lo = 0;
    for (int b = 0; b < ND_NB; ++b) {
        h->bucket_lo[b] = lo;
        if (N == 0) continue;
        ND_CUDA(cudaMemsetAsync(flags + N, 0, sizeof(int64_t), st));
        {
            nd_prof_scope ps("buckets", st);
            k_bucket_flags<<<blocks, kThreads, 0, st>>>(N, h->inc_ptr, b, thr, flags, sums + b);
            ND_CUDA(cudaGetLastError());
        }
        ND_TRY(nd_scan_i64(flags, N, st));
        {
            nd_prof_scope ps("buckets", st);
            k_bucket_scatter<<<blocks, kThreads, 0, st>>>(N, h->inc_ptr, b, thr, flags, h->items + lo);
            ND_CUDA(cudaGetLastError());
        }
        int64_t cnt = 0;
        ND_TRY(read_i64(flags + N, &cnt, st));
        lo += cnt;
    }
    h->bucket_lo[ND_NB] = lo;
    unsigned long long hs[ND_NB] = {0, 0, 0, 0};
    ND_CUDA(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < ND_NB; ++b) h->bucket_inc[b] = (int64_t)hs[b];
    h->num_zero = N - lo;
    cudaFreeAsync(flags, st);
    cudaFreeAsync(sums, st);
    return ND_OK;
}

nd_status nd_write_r_cliques(const nd_incidence* h, int32_t* out_dev, cudaStream_t st) {
    if (h->num_r == 0) return ND_OK;
    int blocks = nd_blocks_for(h->num_r, kThreads, grid_cap(h) * 2);
    nd_prof_scope ps("r_cliques", st);
    k_r_cliques<<<blocks, kThreads, 0, st>>>(h->r, h->num_r, h->e_u, h->e_v, h->tri_w, h->tri_e, out_dev);
    ND_CUDA(cudaGetLastError());
    return ND_OK;
}

nd_status nd_union_device(const nd_union_part* parts_host, int count, int64_t n, int64_t nnz, int64_t* urp,
                          int32_t* ucol, cudaStream_t st) {
    nd_union_part* dparts = nullptr;
    int* derr = nullptr;
    ND_CUDA(cudaMallocAsync((void**)&dparts, sizeof(nd_union_part) * (count > 0 ? count : 1), st));
    ND_CUDA(cudaMallocAsync((void**)&derr, sizeof(int), st));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    ND_CUDA(cudaMemcpyAsync(dparts, parts_host, sizeof(nd_union_part) * count, cudaMemcpyHostToDevice, st));
    if (count > 0) {
        nd_prof_scope ps("union", st);
        k_union<<<count < 152 * 16 ? count : 152 * 16, kThreads, 0, st>>>(dparts, count, urp, ucol, derr);
        ND_CUDA(cudaGetLastError());
    }
    ND_CUDA(cudaMemcpyAsync(urp + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    int herr = 0;
    nd_status s = read_flag(derr, &herr, st);
    cudaFreeAsync(dparts, st);
    cudaFreeAsync(derr, st);
    if (s != ND_OK) return s;
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
    int64_t* didx = nullptr;
    int64_t* dout = nullptr;
    ND_CUDA(cudaMallocAsync((void**)&didx, sizeof(int64_t) * (count + 1), st));
    ND_CUDA(cudaMallocAsync((void**)&dout, sizeof(int64_t) * (count + 1), st));
    ND_CUDA(cudaMemcpyAsync(didx, vertex_off, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
    // edges owned by vertices below the graph's first vertex
    k_gather_i64<<<nd_blocks_for(count + 1, kThreads, 64), kThreads, 0, st>>>(h->up_start, didx, count + 1, dout);
    ND_CUDA(cudaGetLastError());
    if (h->r == 3) {
        // triangles owned by those edges
        k_gather_i64<<<nd_blocks_for(count + 1, kThreads, 64), kThreads, 0, st>>>(h->tri_ptr, dout, count + 1, didx);
        ND_CUDA(cudaGetLastError());
        ND_CUDA(cudaMemcpyAsync(r_off, didx, sizeof(int64_t) * (count + 1), cudaMemcpyDeviceToHost, st));
    } else {
        ND_CUDA(cudaMemcpyAsync(r_off, dout, sizeof(int64_t) * (count + 1), cudaMemcpyDeviceToHost, st));
    }
    ND_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(didx, st);
    cudaFreeAsync(dout, st);
    return ND_OK;
}
