// Internal declarations shared by the libnd translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "nd.h"

// ----------------------------------------------------------------------------
// error handling: every CUDA call is checked; failures become ND_E_CUDA with a
// thread-local message, never an abort.
// ----------------------------------------------------------------------------
void nd_set_error(const std::string& msg);
nd_status nd_cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define ND_CUDA(call)                                                         \
    do {                                                                      \
        cudaError_t nd_e_ = (call);                                           \
        if (nd_e_ != cudaSuccess) return nd_cuda_fail(nd_e_, #call, __FILE__, __LINE__); \
    } while (0)

#define ND_TRY(expr)                                                          \
    do {                                                                      \
        nd_status nd_s_ = (expr);                                             \
        if (nd_s_ != ND_OK) return nd_s_;                                     \
    } while (0)

// ----------------------------------------------------------------------------
// per-kernel timing (CUDA events on the launching stream), see nd_prof_*
// ----------------------------------------------------------------------------
struct nd_prof_scope {
    int kid;
    cudaStream_t st;
    cudaEvent_t a, b;
    bool on;
    int count;  // kernel launches the scope covers (a graph of passes covers several)
    nd_prof_scope(const char* name, cudaStream_t s, int launches = 1);
    ~nd_prof_scope();
};

// ----------------------------------------------------------------------------
// degree buckets for the h-index sweeps: r-cliques are grouped by d_s so that
// each group of lanes that evaluates one r-clique is sized to its work.
// ----------------------------------------------------------------------------
// buckets (thresholds t0 <= 8, t1 <= 64 fit the register caches of the
// 4- and 8-lane groups; defaults 8 / 64 / 2048, tunable per handle):
// 0: d_s in [1,t0] (4 lanes), 1: (t0,t1] (8 lanes), 2: (t1,t2] (a warp), 3: > t2 (a CTA)
enum { ND_NB = 4, ND_T0_MAX = 8, ND_T1_MAX = 64 };

// one unit of h-index work: the r-clique and its incidence row, so that a
// pass reaches the row with one 16-byte load instead of two dependent ones
struct __align__(16) nd_item {
    int64_t jb;   // first incidence of the row
    uint32_t R;   // r-clique id
    uint32_t d;   // row length d_s(R)
};

struct nd_incidence {
    int r = 0, s = 0, q = 0;
    int64_t n = 0, nnz = 0, m = 0;  // m = number of edges (nnz / 2)
    int64_t num_r = 0, num_inc = 0, num_tri = 0;
    int sm_count = 0;
    // graph on the device (owned copies)
    int64_t* rp = nullptr;
    int32_t* col = nullptr;
    int32_t* nlow = nullptr;       // [n] number of neighbours smaller than u
    int64_t* up_start = nullptr;   // [n+1] first edge id owned by u (edges u<v)
    uint32_t* eid = nullptr;       // [nnz] edge id of every CSR entry
    int32_t* e_u = nullptr;        // [m] canonical edges (u<v), lexicographic
    int32_t* e_v = nullptr;
    int64_t* tri_ptr = nullptr;    // [m+1] triangles (u<v<w) grouped by edge (u,v)
    int32_t* tri_w = nullptr;      // [T] third vertex w, ascending inside a group
    uint32_t* tri_e = nullptr;     // [T] owning edge (u,v)
    // incidence (r-clique -> other r-cliques of each s-clique)
    int64_t* inc_ptr = nullptr;    // [num_r+1]
    uint32_t* inc = nullptr;       // [num_inc*q]
    // (2,3) adjacency layout: an incidence entry of edge (x,y), x<y, for the
    // triangle {x,y,w} is the pair of CSR positions (P(x,w), P(y,w)), rows
    // sorted by w, and the passes gather tau from a 16-bit copy indexed by
    // CSR position (each edge's value at both of its entries, saturated at
    // 65535)
    // build only: rows longer than a few thousand entries, split into
    // segments for the per-vertex build kernels (rows, segment offsets)
    int32_t* long_rows = nullptr;
    int64_t* long_seg = nullptr;
    int64_t long_count = 0, long_segs = 0;
    // (1,2): vertices relabelled by degree class (nd_relabel_by_degree); rp and
    // col hold the relabelled graph, and results are permuted back at the
    // boundary.  Null when the handle keeps the caller's ids.
    // (2,3): edges relabelled the same way (nd_relabel_truss_graph); to_new /
    // to_old then map the caller's edge ids to the internal ones and back
    // (num_r each), and vto_old maps internal vertex ids to the caller's.
    // c_*: the caller's CSR and split, kept during the build only.
    int32_t* to_new = nullptr;  // [num_r] caller's r-clique id -> internal id
    int32_t* to_old = nullptr;  // [num_r] internal r-clique id -> caller's id
    int32_t* vto_old = nullptr;
    int64_t *c_rp = nullptr, *c_up = nullptr;
    int32_t *c_col = nullptr, *c_nlow = nullptr;
    bool adj = false;
    uint32_t* mirror = nullptr;    // [nnz] build only: P(v,u) for the entry P(u,v)
    uint2* e_pos = nullptr;        // [m] (P(x,y), P(y,x)) of edge (x,y), x<y
    uint16_t* tg[2] = {nullptr, nullptr};  // [nnz] gather copies of tau by CSR position
    bool rows_sorted = false;      // rows ordered by w (else in fill order)
    // (2,3) with no stored incidence (ND_BUILD_ON_THE_FLY): inc is empty and
    // every pass finds the triangles of each edge again
    bool otf = false;
    bool inc_aliases_graph = false;  // r = 1: inc_ptr/inc are rp/col
    // batches (nd_build_incidence_batch): the graph of every r-clique
    // (internal ids) and, per pass, which graphs are still changing (two byte
    // arrays by pass parity).  A graph whose pass changed nothing has
    // converged: its later SND / AND-nn passes are skipped, as its own run
    // would have stopped there.
    int64_t ngraphs = 0;
    uint32_t* gid = nullptr;
    uint8_t* gact[2] = {nullptr, nullptr};
    // degree-bucketed processing order
    nd_item* items = nullptr;      // [num_r - num_zero], bucket by bucket
    int64_t bucket_lo[ND_NB + 1] = {0, 0, 0, 0, 0};
    int64_t bucket_inc[ND_NB] = {0, 0, 0, 0};
    int64_t num_zero = 0;          // r-cliques with d_s = 0 (kappa = 0, never updated)
    int32_t thr[3] = {8, 64, 2048};  // bucket thresholds t0, t1, t2
    // iteration state
    int32_t* tau[2] = {nullptr, nullptr};
    uint32_t* front[2] = {nullptr, nullptr};
    unsigned long long* counters = nullptr;  // ring of per-pass counters
    unsigned long long* h_counters = nullptr;  // pinned host mirror
    std::vector<int64_t> last_changed, last_evals, last_incs;
    int64_t bytes = 0;
    cudaStream_t last_stream = 0;  // stream of the latest call on this handle
    // instantiated CUDA graphs of a full batch of passes, per mode (SND, AND,
    // AND-nn) and batch kind (first, even, odd); built on first use
    cudaGraphExec_t pass_graph[3][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr},
                                        {nullptr, nullptr, nullptr}};
    bool pass_graph_failed[3][3] = {{false, false, false}, {false, false, false}, {false, false, false}};
    // set while a call uses the iteration state (nd_claim); a second call
    // meanwhile gets ND_E_BUSY
    std::atomic<int> busy{0};
};

// marks a handle in use for the lifetime of the object; ok == false if
// another call holds it (the caller then returns ND_E_BUSY)
struct nd_claim {
    nd_incidence* h;
    bool ok;
    explicit nd_claim(nd_incidence* hh) : h(hh), ok(false) {
        int expect = 0;
        ok = h != nullptr && h->busy.compare_exchange_strong(expect, 1);
    }
    ~nd_claim() {
        if (ok) h->busy.store(0);
    }
    nd_claim(const nd_claim&) = delete;
    nd_claim& operator=(const nd_claim&) = delete;
};

#define ND_CLAIM(handle)                                                      \
    nd_claim nd_claim_((handle));                                             \
    if (!nd_claim_.ok) {                                                      \
        nd_set_error("another call is using this handle");                    \
        return ND_E_BUSY;                                                     \
    }

// passes are enqueued in batches of ND_BATCH; the per-pass counters (ND_SLOT
// u64 each) live in two halves of ND_BATCH slots used by alternate batches
enum { ND_BATCH = 16, ND_RING = 2 * ND_BATCH, ND_SLOT = 6 };

// wait for a stream with a time limit (ND_E_TIMEOUT past it)
nd_status nd_wait(cudaStream_t st);

// a stream-ordered device temporary, released when it goes out of scope
// (also on every early error return)
template <typename T>
struct nd_tmp {
    T* p = nullptr;
    cudaStream_t st = 0;
    explicit nd_tmp(cudaStream_t s) : st(s) {}
    nd_tmp(const nd_tmp&) = delete;
    nd_tmp& operator=(const nd_tmp&) = delete;
    ~nd_tmp() {
        if (p) cudaFreeAsync(p, st);
    }
    nd_status alloc(int64_t count) {
        if (count < 1) count = 1;
        if (cudaMallocAsync((void**)&p, sizeof(T) * (size_t)count, st) != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            nd_set_error("device allocation of a temporary failed");
            return ND_E_NOMEM;
        }
        return ND_OK;
    }
    operator T*() const { return p; }
};

// device memory helpers (stream-ordered)
nd_status nd_alloc(void** p, size_t bytes, cudaStream_t st, nd_incidence* owner);
void nd_release(void* p, cudaStream_t st);

// exclusive scan of data[0..count] in place (count+1 entries; data[count]
// becomes the total).  Uses stream-ordered scratch.
nd_status nd_scan_i64(int64_t* data, int64_t count, cudaStream_t st);

// stable LSD radix sort (8-bit digits) of keys[0, count) over their low
// `bits` bits, ping-ponging with alt; *result is whichever holds the sorted
// keys (nd_normalize.cu).  nd_id_bits(n): bits of the ids 0..n-1 (at least 1).
nd_status nd_sort_u64(unsigned long long* keys, unsigned long long* alt, int64_t count, int bits,
                      unsigned long long** result, cudaStream_t st);
int nd_id_bits(int64_t n);

// build steps (nd_build.cu)
// the handle's CSR copy, validated and split; truss_relabel: a (2,3) build
// that will renumber the graph (nd_relabel_truss_graph) next
nd_status nd_build_graph(nd_incidence* h, const nd_csr* g, cudaStream_t st, bool truss_relabel);
nd_status nd_build_edges(nd_incidence* h, cudaStream_t st);
nd_status nd_build_tri_incidence(nd_incidence* h, cudaStream_t st);
nd_status nd_build_triangles(nd_incidence* h, cudaStream_t st);
nd_status nd_build_k4_incidence(nd_incidence* h, cudaStream_t st);
nd_status nd_build_buckets(nd_incidence* h, cudaStream_t st);
nd_status nd_relabel_by_degree(nd_incidence* h, cudaStream_t st);
nd_status nd_relabel_truss_graph(nd_incidence* h, cudaStream_t st);
nd_status nd_relabel_truss_edges(nd_incidence* h, cudaStream_t st);
// out[idx[i]] = in[i] (scatter) or out[i] = in[idx[i]] (gather), n int32 values on st
nd_status nd_permute_i32(const int32_t* idx, const int32_t* in, int32_t* out, int64_t n, bool scatter,
                         cudaStream_t st);
nd_status nd_write_r_cliques(const nd_incidence* h, int32_t* out_dev, cudaStream_t st);

// batches (disjoint unions of independent graphs)
struct nd_union_part {
    const int64_t* rp;
    const int32_t* col;
    int64_t n, nnz, n_off, nnz_off;
};
nd_status nd_union_device(const nd_union_part* parts_host, int count, int64_t n, int64_t nnz, int64_t* urp,
                          int32_t* ucol, cudaStream_t st);
nd_status nd_batch_offsets(const nd_incidence* h, const int64_t* vertex_off, int count, int64_t* r_off,
                           cudaStream_t st);
// the graph index of every r-clique of a batch handle (h->gid, internal ids)
nd_status nd_batch_graph_ids(nd_incidence* h, const int64_t* r_off /* count+1, host */, int count, cudaStream_t st);

// iteration (nd_hindex.cu)
nd_status nd_init_tau(nd_incidence* h, int32_t* tau, cudaStream_t st);
// options of a run beyond the paper's plain SND / AND
struct nd_run_opts {
    const uint32_t* members = nullptr;  // PartialAnd: member bitmap (device), AND modes only
    double stop_active = 0.0;           // AND: stop after a pass that evaluated < this fraction of N_R
    bool stopped = false;               // out: the active-ratio rule ended the run
};
nd_status nd_run(nd_incidence* h, int mode, int32_t max_passes, const int32_t* tau_in_dev,
                 int32_t** tau_result, int32_t* updating, int64_t* evals, bool* converged,
                 cudaStream_t st, nd_run_opts* opts = nullptr);
nd_status nd_member_mask(const uint32_t* ids, int64_t count, int64_t N, uint32_t* mask, int* err, cudaStream_t st,
                         const int32_t* to_new = nullptr);
nd_status nd_count_equal_dev(const int32_t* a, const int32_t* b, int64_t n, unsigned long long* out_dev,
                             cudaStream_t st);
nd_status nd_classic_truss(const int32_t* in, int64_t n, int32_t* out, cudaStream_t st);
// evaluation (nd_eval.cu): Kendall's tau-b of two device sequences; waits on st
nd_status nd_kendall_dev(const int32_t* x, const int32_t* y, int64_t n, int sm_count, double* tau_out,
                         int64_t* counts_out, cudaStream_t st);

// lower bound of x in the sorted list a[0, n), n < 2^31 (32-bit offsets)
static __device__ __forceinline__ int nd_lower_bound_n(const int32_t* __restrict__ a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// launch geometry
static inline int nd_blocks_for(int64_t work_items, int per_block, int cap) {
    int64_t b = (work_items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}
