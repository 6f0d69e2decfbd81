/*
 * nd.h -- C ABI of the GB300 local nucleus decomposition library (libnd).
 *
 * The library computes, for every r-clique R of a simple undirected graph,
 * its kappa_s index (core number for (r,s) = (1,2), truss number for (2,3),
 * (3,4)-nucleus number for (3,4)) by the iterated h-index update of
 * Sariyuce, Seshadhri and Pinar, "Local Algorithms for Hierarchical Dense
 * Subgraph Discovery" (PVLDB 12(1), 2019):
 *   - the problem statement is the input/output of Alg. 1, Alg. 2, Alg. 3
 *     (Input: graph G, integers r < s; Output: kappa_s of every r-clique);
 *   - r-cliques, s-cliques and the S-degree d_s are Def. 1; kappa_s is Def. 2;
 *   - the update operator U (rho(S,R) = min over the other r-cliques of S,
 *     then the h-index H of Def. 3) is Def. 4;
 *   - SND (synchronous, Jacobi-like) is Alg. 2, Section 4.1;
 *   - AND (asynchronous, in place, Gauss-Seidel-like) is Alg. 3, Section 4.2,
 *     and its notification mechanism is Section 4.3.
 *
 * Conventions shared by every call:
 *   - Status codes are returned, never thrown; no call aborts the process.
 *     nd_last_error() gives a message for the calling thread's last failure.
 *   - Integers: vertex ids int32; r-clique ids fit uint32; offsets int64;
 *     tau / kappa int32.  The arithmetic is exact integer throughout.
 *   - Pointers flagged "host or device" are host memory when the call's
 *     on_device argument is 0 and device memory (this GPU) when it is 1.
 *     The caller owns every buffer it passes; the library owns the
 *     nd_incidence handle and everything inside it until nd_free().
 *   - Calls are stream-ordered on the given cudaStream_t (passed as void*;
 *     NULL = the legacy default stream).  A call that returns results into
 *     host memory synchronises that stream before returning; a call that
 *     writes device memory returns once the work is enqueued, except where
 *     it must read a count back (each such call says so).
 *   - Canonical r-clique order: lexicographic order of the sorted vertex
 *     tuple.  Vertex v for r = 1; edge (u,v), u < v, for r = 2; triangle
 *     (u,v,w), u < v < w, for r = 3.  tau arrays are indexed in this order.
 *   - Truss numbers follow the paper's convention (Section 2.1): an edge in
 *     a k-truss lies in at least k triangles; the classic k-truss of Cohen
 *     is kappa_3 + 2 (see nd_truss_classic).
 */
#ifndef ND_H
#define ND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ND_OK = 0,
    ND_E_INVAL = 1,           /* bad argument or malformed graph (not simple, sorted, symmetric) */
    ND_E_UNSUPPORTED_RS = 2,  /* (r,s) not one of (1,2), (2,3), (3,4) */
    ND_E_NOMEM = 3,           /* a device or host allocation failed */
    ND_E_CUDA = 4,            /* a CUDA runtime call failed (message in nd_last_error) */
    ND_E_NOT_CONVERGED = 5,   /* the iteration cap was reached; tau is still a valid upper bound */
    ND_E_TIMEOUT = 6,         /* a host-side wait exceeded its limit */
    ND_E_TOO_LARGE = 7,       /* more r-cliques than the 32-bit id space, or a size limit */
    ND_E_BUSY = 8             /* another call is using the same handle (calls on one handle
                                 must not overlap; the refused call did nothing) */
} nd_status;

typedef enum { ND_SND = 0, ND_AND = 1, ND_AND_NN = 2 } nd_mode;

/* Simple undirected graph in CSR form: row_ptr[n+1] (int64), col[nnz]
 * (int32), every row strictly increasing, no self-loops, symmetric
 * (v in row u iff u in row v), so nnz = 2|E|.  Host or device per on_device. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    int on_device;
} nd_csr;

typedef struct nd_incidence nd_incidence; /* opaque; owned by the library */

/* Edge list -> the simple undirected graph of Section 2, as the CSR that
 * nd_build_incidence takes.  src[m], dst[m] (int64; host or device per
 * on_device) are arbitrary vertex pairs in [0, n): each pair (a, b) with
 * a != b is the undirected edge {a, b}; self-loops (a == b) are dropped and
 * a pair given more than once, in either direction, is one edge.
 * Output (caller-owned, the same kind of memory as the input):
 *   row_ptr_out[n+1] int64; col_out[col_capacity] int32, where 2m always
 *   suffices; *nnz_out = entries written = 2|E|.  Every row is strictly
 *   increasing and the adjacency is symmetric.
 * An id outside [0, n) gives ND_E_INVAL.  If col_capacity is below the
 * result's size, the call returns ND_E_INVAL with the size needed in
 * *nnz_out and writes no output.  Runs on this GPU (a stable radix sort of
 * the 2m directed pairs); temporary device memory is about 40 B per pair
 * (plus 16 B per pair for host input).  Synchronises `stream`. */
nd_status nd_normalize(const int64_t* src, const int64_t* dst, int64_t m, int64_t n, int on_device,
                       int64_t* row_ptr_out, int32_t* col_out, int64_t col_capacity, int64_t* nnz_out,
                       void* stream);

/* Build the r-clique -> s-clique incidence of g (Def. 1) on this GPU:
 * degree split and canonical edge ids, then triangle enumeration for r = 2
 * and r = 3 and 4-clique enumeration for r = 3, by sorted-list intersection
 * (the paper finds s-cliques through vertex neighbourhoods, Section 4.1,
 * "Time complexity"; here they are materialised once as CSR).
 * For each r-clique R the incidence lists, per s-clique S containing R, the
 * q = C(s,r) - 1 other r-cliques of S; row lengths are d_s(R).  How they are
 * named inside the handle (edge ids, CSR slots, relabelled vertex ids) is
 * internal: every call takes and returns r-cliques in the canonical order
 * of nd_r_cliques.
 * The graph is validated first; a malformed graph returns ND_E_INVAL and
 * builds nothing.  Bounds, ids, self-loops and row order are checked
 * exactly.  Symmetry is checked exactly for r >= 2, where the build finds
 * every entry's reverse anyway.  For r = 1 it is checked by a fingerprint:
 * two 64-bit sums, over all entries (u, v), of a hash of (u, v) minus the
 * same hash of (v, u).  A symmetric graph always passes.  An asymmetric one
 * passes only if both sums vanish by coincidence, about 2^-128 for inputs
 * not built to collide.  A k-core of such an input reads only inside its
 * arrays.  Synchronises `stream` (sizes are read back to allocate).
 * On success *out owns device memory until nd_free(*out). */
nd_status nd_build_incidence(const nd_csr* g, int r, int s, void* stream, nd_incidence** out);

/* nd_build_incidence with options.  flags = 0 is nd_build_incidence.
 * ND_BUILD_ON_THE_FLY: store no r-clique -> s-clique incidence.  The paper's
 * own implementation does not store the s-cliques but finds them again
 * through the neighbourhoods on every update (Section 4.1, "Time
 * complexity"; Section 5); this mode does the same for memory-bound inputs.
 * Only the counts d_s are kept (tau_0 and the work buckets); every SND / AND
 * pass then finds the triangles of edge (x,y) by searching each entry of the
 * shorter of N(x), N(y) in the longer.  Results are identical to the stored
 * mode; a pass costs about sum over edges of min(deg) binary searches
 * instead of a stream of 8 B per incidence.  For (1,2) the CSR already is the
 * incidence and the flag changes nothing; (3,4) gives ND_E_UNSUPPORTED_RS.
 * Unknown flags give ND_E_INVAL. */
#define ND_BUILD_ON_THE_FLY 1u
nd_status nd_build_incidence_ex(const nd_csr* g, int r, int s, unsigned flags, void* stream, nd_incidence** out);

/* Batched build: the incidence of many independent graphs at once, as the
 * incidence of their disjoint union (graph i's vertex ids are shifted past
 * those of graphs 0..i-1).  kappa_s of a disjoint union is kappa_s of each
 * part (Lemma 1: a subgraph around R only gains from R's own component), so
 * every later call (nd_snd, nd_and, nd_iterate_k, ...) processes all graphs
 * in one launch per pass.  In the union's canonical order the r-cliques of
 * graph i are the contiguous slice [r_offsets[i], r_offsets[i+1]), in graph
 * i's own canonical order.  graphs[count]: all on the host or all on the
 * device; each must be a valid CSR whose ids stay inside its own range.
 * r_offsets: host int64[count+1] (may be NULL).  Synchronises `stream`. */
nd_status nd_build_incidence_batch(const nd_csr* graphs, int count, int r, int s, void* stream,
                                   nd_incidence** out, int64_t* r_offsets);

/* Sizes of a built incidence: number of r-clique (N_R), number of
 * (R, S) incidences (M = sum of d_s), and q.  Any output may be NULL. */
nd_status nd_incidence_info(const nd_incidence* inc, int64_t* num_r, int64_t* num_incidences,
                            int* q);

/* Vertex tuples of the r-cliques in canonical order: num_r * r int32,
 * host or device per on_device. */
nd_status nd_r_cliques(const nd_incidence* inc, int32_t* verts_out, int on_device, void* stream);

/* d_s(R) for every r-clique (tau_0 of Alg. 2 and Alg. 3): num_r int32. */
nd_status nd_s_degree(const nd_incidence* inc, int32_t* ds_out, int on_device, void* stream);

/* SND, Alg. 2: tau_0 = d_s, tau_{t+1} = U tau_t, until a pass changes no
 * tau or max_iters passes ran.  tau_out: num_r int32 (host or device).
 * *iters_out (may be NULL) = number of passes that changed at least one
 * tau (the pass that detects convergence is not counted).  Synchronises
 * `stream`.  Returns ND_E_NOT_CONVERGED if the cap was reached first. */
nd_status nd_snd(nd_incidence* inc, int32_t* tau_out, int on_device, int32_t max_iters,
                 int32_t* iters_out, void* stream);

/* AND, Alg. 3: tau updated in place from the latest values.  notify = 1
 * enables the notification mechanism of Section 4.3 (only r-cliques whose
 * neighbours changed are recomputed); notify = 0 is "AND-nn".  Processing
 * order inside a pass is not fixed (any order reaches the same kappa_s).
 * *iters_out = passes that changed a tau; *evals_out = h-index evaluations
 * performed over all passes (either may be NULL).  Synchronises `stream`. */
nd_status nd_and(nd_incidence* inc, int32_t* tau_out, int on_device, int notify,
                 int32_t max_iters, int32_t* iters_out, int64_t* evals_out, void* stream);

/* Early-stopped iteration (Section 5.2.3's runtime/accuracy trade-off):
 * run at most k passes of `mode` starting from tau_inout (tau_init_given = 1;
 * any tau with kappa_s <= tau <= d_s is a valid start, Lemma 2) or from d_s
 * (tau_init_given = 0), and write the result back into tau_inout.  Stops
 * early if a pass changes nothing.  *updating_out = passes that changed a
 * tau.  SND results are deterministic; AND results depend on the schedule
 * but always satisfy kappa_s <= tau_AND_k <= tau_SND_k.  Synchronises. */
nd_status nd_iterate_k(nd_incidence* inc, int mode, int32_t k, int32_t* tau_inout,
                       int tau_init_given, int on_device, int32_t* updating_out, void* stream);

/* PartialAnd (end of Section 4.3; the ego-network queries of Section 5.4):
 * AND with notification restricted to the member set P, given as `count`
 * r-clique ids (host or device per on_device).  Only members start active
 * and only members are ever notified; every other r-clique keeps d_s.  The
 * result is the greatest fixed point of the restricted update below d_s, the
 * same for any processing order, with kappa_s <= tau (equal to kappa_s when P
 * holds every r-clique).  An id >= num_r gives ND_E_INVAL.  tau_out: num_r
 * int32.  Synchronises `stream`. */
nd_status nd_and_partial(nd_incidence* inc, const uint32_t* members, int64_t count, int on_device,
                         int32_t* tau_out, int32_t max_iters, int32_t* iters_out, int64_t* evals_out,
                         void* stream);

/* AND with notification and the active-ratio stopping rule of Section 5.2
 * (Fig. 9): stop after the first pass that evaluated fewer than
 * active_ratio * num_r r-cliques (the paper's 40% and 10% settings are 0.4
 * and 0.1), or at convergence.  *stopped_out = 1 if the rule ended the run.
 * tau_out then holds kappa_s <= tau <= d_s.  Synchronises `stream`. */
nd_status nd_and_until(nd_incidence* inc, double active_ratio, int32_t* tau_out, int on_device,
                       int32_t max_iters, int32_t* iters_out, int64_t* evals_out, int* stopped_out,
                       void* stream);

/* Number of positions where a[i] == b[i] over n int32 values (host or device
 * per on_device): the accuracy of an early-stopped tau against kappa_s
 * (Section 5.2, "accuracy").  Synchronises `stream`. */
nd_status nd_count_equal(const int32_t* a, const int32_t* b, int64_t n, int on_device, int64_t* equal_out,
                         void* stream);

/* Kendall's tau-b of x against y over n int32 values (host or device per
 * on_device): the similarity of the order of the r-cliques by an
 * early-stopped tau with the order by kappa_s (Section 5.2, Fig. 7; the
 * paper does not name the variant, and tau-b corrects for the many ties of
 * integer indices).  tau_b = S / sqrt((n0 - tx) (n0 - ty)), S = concordant
 * minus discordant pairs, tx / ty = pairs tied in x / in y, n0 = n(n-1)/2.
 * *tau_out is NaN when either sequence is constant or n < 2.  counts_out
 * (optional, 3 int64) receives S, tx, ty.  Uses (max x - min x + 2) *
 * (max y - min y + 2) 8-byte counters of device memory; more than 2^28
 * gives ND_E_TOO_LARGE.  Synchronises `stream`. */
nd_status nd_kendall_tau_b(const int32_t* x, const int32_t* y, int64_t n, int on_device, double* tau_out,
                           int64_t* counts_out, void* stream);

/* Classic truss numbers (Cohen's k-2 convention) from kappa_3: out = in + 2
 * for every edge.  Host or device per on_device (host buffers are copied
 * through the device).  Synchronises `stream` for host buffers. */
nd_status nd_truss_classic(const int32_t* kappa3, int64_t num_edges, int32_t* out, int on_device,
                           void* stream);

/* Per-kernel timing with CUDA events recorded on the launching stream.
 * nd_prof_enable(1) starts recording (and clears the totals); with 0 it
 * stops.  nd_prof_read synchronises and returns, for kernel index i, its
 * name, launch count and total milliseconds; it returns ND_E_INVAL past the
 * last kernel.  Profiling is off by default. */
nd_status nd_prof_enable(int on);
nd_status nd_prof_read(int i, const char** name, int64_t* launches, double* total_ms);

/* Autotune the degree buckets of this handle: for each candidate threshold
 * set (t0 in {4,8}, t1 in {32,64}, t2 in {256,1024,2048,8192}; rows of
 * length [1,t0] go to 4-lane groups, (t0,t1] to 8-lane groups, (t1,t2] to
 * warps, longer ones to whole CTAs) time `passes` SND passes from d_s, keep
 * the fastest, and remember it for this device, (r,s) and size class
 * (floor(log2 of the incidence count)): later nd_build_incidence calls of the
 * same class start with it.  Results never depend on the thresholds.
 * thr_out[3] and best_ms_out may be NULL.  Synchronises `stream`. */
nd_status nd_autotune(nd_incidence* inc, int32_t passes, void* stream, int32_t* thr_out, double* best_ms_out);

/* Counters of the last nd_snd / nd_and / nd_iterate_k call on this handle,
 * pass by pass: changed[i] = r-cliques whose tau changed in pass i,
 * evaluated[i] = h-index evaluations in pass i (active r-cliques for AND),
 * incidences[i] = incidences (s-cliques) streamed by those evaluations.
 * Any array may be NULL.  Fills at most cap entries and returns the number
 * of passes in *passes. */
nd_status nd_last_passes(const nd_incidence* inc, int64_t* changed, int64_t* evaluated, int64_t* incidences,
                         int32_t cap, int32_t* passes);

/* Device memory held by the handle, in bytes. */
nd_status nd_incidence_bytes(const nd_incidence* inc, int64_t* bytes);

/* Core numbers ((r,s) = (1,2)) by SND without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they call in -- their process has
 * handed all GPU memory to another allocator up front, or they cannot
 * afford the implicit device synchronisation of cudaMalloc / cudaFree.
 * It returns the same core numbers and pass count as nd_build_incidence
 * (g, 1, 2) + nd_snd, computed straight from a device CSR.
 *   row_ptr[n+1], col[nnz]: device pointers to a simple, sorted, symmetric
 *     CSR (rows and ids are bounds-checked: a violation gives ND_E_INVAL;
 *     sortedness and symmetry are not checked).
 *   core_out[n]: device pointer; receives the core numbers.
 *   n must be at most 1,048,576; larger graphs get ND_E_TOO_LARGE.
 *   max_iters caps the passes as for nd_snd; *iters_out (may be NULL) =
 *   passes that changed a value.  Synchronises `stream` before returning.
 * Scratch: one file-scope device array of 4 MiB + 1 KiB (a previous-pass
 * tau buffer and per-pass counters).
 * Set-up: CUDA loads this entry point's device code and array onto a GPU
 * lazily, and that load takes device memory.  The first call on a device
 * (with that device current) does the load and looks up the array's device
 * address (cudaGetSymbolAddress); a call with n = 0 does only that (row_ptr,
 * col and core_out may be NULL) and returns its status.  A caller whose
 * allocator reserves the device's memory makes that n = 0 call first,
 * before the reservation, and before any stream capture.  A failed set-up
 * is not remembered: the next call tries again.  After it the device holds
 * the array until the process exits, and no call allocates device memory.
 * All calls share the array and it keeps the last call's contents (the
 * counters are cleared at the start of each call): calls that overlap on
 * the GPU -- on two streams, or from two threads -- race and must be
 * serialised by the caller. */
nd_status nd_core_snd_noalloc(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz,
                              int32_t* core_out, int32_t max_iters, int32_t* iters_out, void* stream);

/* Limit of every host-side wait (default 600 s; process-wide).  A call that
 * waits for its stream polls it and returns ND_E_TIMEOUT once the limit has
 * passed; the work it enqueued keeps running, and the handle is usable again
 * once the stream has drained.  seconds must be > 0. */
nd_status nd_set_wait_limit(double seconds);

/* Limit on the device memory one handle may hold (nd_incidence_bytes;
 * process-wide; 0 = none, the default).  A build or iteration call that
 * would take a handle past it returns ND_E_NOMEM; a failed build frees what
 * it took.  Lets a server that admits work by memory footprint enforce its
 * budget per request.  bytes must be >= 0. */
nd_status nd_set_handle_memory_limit(int64_t bytes);

/* Calls on one handle must not overlap (a handle holds one iteration state).
 * Every call that uses a handle's state (nd_snd, nd_and, nd_iterate_k,
 * nd_and_partial, nd_and_until, nd_autotune, nd_last_passes) marks the
 * handle in use while it runs; a second such call that comes in meanwhile,
 * from another thread, returns ND_E_BUSY at once and does nothing.  Calls on
 * different handles may run concurrently on different streams. */

void nd_free(nd_incidence* inc);
const char* nd_strerror(nd_status st);
const char* nd_last_error(void);
int nd_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ND_H */
