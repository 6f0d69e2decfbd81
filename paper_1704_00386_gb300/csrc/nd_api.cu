// C ABI of libnd (declared and documented in include/nd.h).
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <map>
#include <tuple>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <thread>

#include "nd_internal.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void nd_set_error(const std::string& msg) { g_last_error = msg; }

nd_status nd_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
    if (e == cudaErrorMemoryAllocation) return ND_E_NOMEM;
    return ND_E_CUDA;
}

// ---------------------------------------------------------------------------
// profiling: per-kernel CUDA events on the launching stream
// ---------------------------------------------------------------------------
namespace {
struct ProfEntry {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfEntry> g_prof;

int prof_id(const char* name) {
    for (size_t i = 0; i < g_prof.size(); ++i)
        if (g_prof[i].name == name) return (int)i;
    g_prof.push_back(ProfEntry());
    g_prof.back().name = name;
    return (int)g_prof.size() - 1;
}

void prof_drain() {
    for (auto& e : g_prof) {
        for (auto& pr : e.pending) {
            cudaEventSynchronize(pr.second);
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) e.ms += ms;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        e.pending.clear();
    }
}
}  // namespace

nd_prof_scope::nd_prof_scope(const char* name, cudaStream_t s, int launches)
    : kid(-1), st(s), a(nullptr), b(nullptr), on(false), count(launches) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    kid = prof_id(name);
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
    cudaEventRecord(a, st);
    on = true;
}

nd_prof_scope::~nd_prof_scope() {
    if (!on) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof[kid].launches += count;
    g_prof[kid].pending.push_back({a, b});
}

// ---------------------------------------------------------------------------
// device memory (stream-ordered; the pool keeps freed blocks for reuse)
// ---------------------------------------------------------------------------
// per-handle device memory limit (nd_set_handle_memory_limit; 0 = none)
static std::atomic<int64_t> g_handle_limit{0};

nd_status nd_alloc(void** p, size_t bytes, cudaStream_t st, nd_incidence* owner) {
    if (bytes == 0) bytes = 16;
    const int64_t limit = g_handle_limit.load();
    if (owner && limit > 0 && owner->bytes + (int64_t)bytes > limit) {
        *p = nullptr;
        char buf[200];
        snprintf(buf, sizeof(buf), "the handle would hold %lld bytes of device memory, above its limit of %lld",
                 (long long)(owner->bytes + (int64_t)bytes), (long long)limit);
        nd_set_error(buf);
        return ND_E_NOMEM;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed", bytes);
        nd_set_error(buf);
        return ND_E_NOMEM;
    }
    if (owner) owner->bytes += (int64_t)bytes;
    return ND_OK;
}

void nd_release(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

static void keep_pool(int dev) {
    static std::once_flag once[64];
    if (dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// bounded wait: poll the stream instead of blocking forever
static std::atomic<double> g_wait_limit{600.0};

nd_status nd_wait(cudaStream_t st) {
    const double seconds = g_wait_limit.load();
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return ND_OK;
        if (e != cudaErrorNotReady) return nd_cuda_fail(e, "cudaStreamQuery", __FILE__, __LINE__);
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > seconds) {
            char buf[96];
            snprintf(buf, sizeof(buf), "stream did not finish within %g s", seconds);
            nd_set_error(buf);
            return ND_E_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int nd_abi_version(void) { return 1; }

const char* nd_strerror(nd_status st) {
    switch (st) {
        case ND_OK: return "ok";
        case ND_E_INVAL: return "invalid argument or malformed graph";
        case ND_E_UNSUPPORTED_RS: return "unsupported (r,s): use (1,2), (2,3) or (3,4)";
        case ND_E_NOMEM: return "out of memory";
        case ND_E_CUDA: return "CUDA runtime error";
        case ND_E_NOT_CONVERGED: return "iteration cap reached before convergence";
        case ND_E_TIMEOUT: return "timed out";
        case ND_E_TOO_LARGE: return "problem exceeds the 32-bit id space or a size limit";
        case ND_E_BUSY: return "another call is using this handle";
    }
    return "unknown status";
}

const char* nd_last_error(void) { return g_last_error.c_str(); }

nd_status nd_set_wait_limit(double seconds) {
    if (!(seconds > 0.0)) { nd_set_error("the wait limit must be > 0 seconds"); return ND_E_INVAL; }
    g_wait_limit.store(seconds);
    return ND_OK;
}

nd_status nd_set_handle_memory_limit(int64_t bytes) {
    if (bytes < 0) { nd_set_error("negative memory limit"); return ND_E_INVAL; }
    g_handle_limit.store(bytes);
    return ND_OK;
}

void nd_free(nd_incidence* h) {
    if (!h) return;
    // every call on a handle is ordered on its stream; wait for the latest
    // one, then release on it (other streams keep running)
    cudaStream_t st = h->last_stream;
    cudaStreamSynchronize(st);
    void* ptrs[] = {h->nlow, h->up_start, h->eid, h->e_u, h->e_v, h->tri_ptr, h->tri_w, h->tri_e,
                    h->items, h->tau[0], h->tau[1], h->front[0], h->front[1], h->counters,
                    h->mirror, h->e_pos, h->tg[0], h->tg[1], h->long_rows, h->long_seg, h->to_new, h->to_old,
                    h->vto_old, h->c_rp, h->c_up, h->c_col, h->c_nlow, h->gid, h->gact[0], h->gact[1]};
    for (void* p : ptrs) nd_release(p, st);
    for (auto& row : h->pass_graph)
        for (auto& ex : row)
            if (ex) cudaGraphExecDestroy(ex);
    if (!h->inc_aliases_graph) {
        nd_release(h->inc_ptr, st);
        nd_release(h->inc, st);
    }
    nd_release(h->rp, st);
    nd_release(h->col, st);
    if (h->h_counters) cudaFreeHost(h->h_counters);
    cudaStreamSynchronize(st);
    delete h;
}

// ---------------------------------------------------------------------------
// bucket autotuning: thresholds picked by timing, cached per (device, r, s,
// size class = floor(log2(incidences)))
// ---------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, std::array<int32_t, 3>> g_tune;

static int size_class(const nd_incidence* h) {
    return (int)std::floor(std::log2((double)(h->num_inc > 0 ? h->num_inc : 1)));
}

static void apply_tuned(nd_incidence* h, int dev) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, h->r, h->s, size_class(h)));
    if (it != g_tune.end())
        for (int i = 0; i < 3; ++i) h->thr[i] = it->second[i];
}

static nd_status check_rs(int r, int s) {
    if (r < 1 || s <= r) { nd_set_error("need 1 <= r < s"); return ND_E_INVAL; }
    if (!((r == 1 && s == 2) || (r == 2 && s == 3) || (r == 3 && s == 4))) {
        nd_set_error("only (1,2), (2,3) and (3,4) are implemented");
        return ND_E_UNSUPPORTED_RS;
    }
    return ND_OK;
}

static nd_status check_csr(const nd_csr* g) {
    if (!g) { nd_set_error("graph is NULL"); return ND_E_INVAL; }
    if (g->n < 0 || g->nnz < 0 || !g->row_ptr || (g->nnz > 0 && !g->col)) {
        nd_set_error("bad CSR header");
        return ND_E_INVAL;
    }
    if (g->n >= INT32_MAX) { nd_set_error("more than 2^31-1 vertices"); return ND_E_TOO_LARGE; }
    if (g->n == 0 && g->nnz != 0) { nd_set_error("nnz > 0 with no vertices"); return ND_E_INVAL; }
    return ND_OK;
}

// the whole build on one (validated-header) CSR
// size limits that can be told from the header, checked before any copy:
// (2,3) keeps CSR positions and edge ids in 32 bits
static nd_status check_limits(const nd_csr* g, int r) {
    if (r >= 2 && g->nnz / 2 >= (int64_t)UINT32_MAX) {
        nd_set_error("more than 2^32-1 edges");
        return ND_E_TOO_LARGE;
    }
    if (r == 2 && g->nnz >= (int64_t)UINT32_MAX) {
        nd_set_error("(2,3) needs fewer than 2^32-1 CSR entries");
        return ND_E_TOO_LARGE;
    }
    return ND_OK;
}

// relabel: single-graph builds may renumber a large (2,3) graph by degree
// class; a batch keeps its ids (each graph's vertices stay contiguous)
static nd_status build_common(const nd_csr* g, int r, int s, cudaStream_t st, nd_incidence** out,
                              unsigned flags = 0, bool relabel = true) {
    int dev = 0;
    ND_CUDA(cudaGetDevice(&dev));
    keep_pool(dev);
    nd_incidence* h = new (std::nothrow) nd_incidence();
    if (!h) { nd_set_error("host allocation failed"); return ND_E_NOMEM; }
    h->r = r;
    h->s = s;
    h->q = (r == 1) ? 1 : (r == 2 ? 2 : 3);
    h->otf = (flags & ND_BUILD_ON_THE_FLY) && r == 2;
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        h->sm_count = 152;
    h->last_stream = st;
    nd_status rc = nd_build_graph(h, g, st, r == 2 && !h->otf && relabel);
    if (rc == ND_OK && r == 2 && !h->otf && relabel) rc = nd_relabel_truss_graph(h, st);
    if (rc == ND_OK && r >= 2) rc = nd_build_edges(h, st);
    if (rc == ND_OK && r == 2) rc = nd_relabel_truss_edges(h, st);
    if (rc == ND_OK) {
        if (r == 1) {
            rc = nd_relabel_by_degree(h, st);
            h->num_r = h->n;
            h->num_inc = h->nnz;
            h->inc_ptr = h->rp;
            h->inc = reinterpret_cast<uint32_t*>(h->col);
            h->inc_aliases_graph = true;
        } else if (r == 2) {
            rc = nd_build_tri_incidence(h, st);
        } else {
            rc = nd_build_triangles(h, st);
            if (rc == ND_OK) rc = nd_build_k4_incidence(h, st);
        }
    }
    if (rc == ND_OK) apply_tuned(h, dev);
    if (rc == ND_OK) rc = nd_build_buckets(h, st);
    if (rc == ND_OK) rc = nd_wait(st);
    if (rc != ND_OK) {
        std::string keep = g_last_error;
        cudaStreamSynchronize(st);
        nd_free(h);
        g_last_error = keep;
        return rc;
    }
    *out = h;
    return ND_OK;
}

nd_status nd_build_incidence(const nd_csr* g, int r, int s, void* stream, nd_incidence** out) {
    if (!out) { nd_set_error("out is NULL"); return ND_E_INVAL; }
    *out = nullptr;
    ND_TRY(check_rs(r, s));
    ND_TRY(check_csr(g));
    ND_TRY(check_limits(g, r));
    return build_common(g, r, s, (cudaStream_t)stream, out);
}

nd_status nd_build_incidence_ex(const nd_csr* g, int r, int s, unsigned flags, void* stream, nd_incidence** out) {
    if (!out) { nd_set_error("out is NULL"); return ND_E_INVAL; }
    *out = nullptr;
    ND_TRY(check_rs(r, s));
    if (flags & ~(unsigned)ND_BUILD_ON_THE_FLY) { nd_set_error("unknown build flag"); return ND_E_INVAL; }
    if ((flags & ND_BUILD_ON_THE_FLY) && r == 3) {
        nd_set_error("the on-the-fly mode covers (1,2) and (2,3)");
        return ND_E_UNSUPPORTED_RS;
    }
    ND_TRY(check_csr(g));
    ND_TRY(check_limits(g, r));
    return build_common(g, r, s, (cudaStream_t)stream, out, flags);
}

nd_status nd_build_incidence_batch(const nd_csr* graphs, int count, int r, int s, void* stream,
                                   nd_incidence** out, int64_t* r_offsets) {
    if (!out) { nd_set_error("out is NULL"); return ND_E_INVAL; }
    *out = nullptr;
    ND_TRY(check_rs(r, s));
    if (count < 0 || (count > 0 && !graphs)) { nd_set_error("bad graph list"); return ND_E_INVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> voff(count + 1, 0);
    std::vector<nd_union_part> parts(count);
    int64_t n = 0, nnz = 0;
    const int on_device = count > 0 ? graphs[0].on_device : 1;
    for (int i = 0; i < count; ++i) {
        ND_TRY(check_csr(&graphs[i]));
        if (graphs[i].on_device != on_device) {
            nd_set_error("all graphs of a batch must be on the host or all on the device");
            return ND_E_INVAL;
        }
        parts[i] = {graphs[i].row_ptr, graphs[i].col, graphs[i].n, graphs[i].nnz, n, nnz};
        n += graphs[i].n;
        nnz += graphs[i].nnz;
        voff[i + 1] = n;
    }
    if (n >= INT32_MAX) { nd_set_error("batch has more than 2^31-1 vertices"); return ND_E_TOO_LARGE; }
    {
        const nd_csr whole{n, nnz, nullptr, nullptr, on_device};
        ND_TRY(check_limits(&whole, r));
    }
    nd_tmp<int64_t> urp(st);
    nd_tmp<int32_t> ucol(st);
    nd_status rc = ND_OK;
    if (on_device) {
        ND_TRY(urp.alloc(n + 1));
        ND_TRY(ucol.alloc(nnz));
        rc = nd_union_device(parts.data(), count, n, nnz, urp, ucol, st);
        if (rc == ND_OK) {
            nd_csr u{n, nnz, urp, ucol, 1};
            rc = build_common(&u, r, s, st, out, 0, false);
        }
    } else {
        // host graphs: assemble the union on the host and copy it once
        std::vector<int64_t> hrp(n + 1);
        std::vector<int32_t> hcol(nnz > 0 ? nnz : 1);
        for (int i = 0; i < count && rc == ND_OK; ++i) {
            const nd_union_part& p = parts[i];
            if (p.rp[0] != 0 || p.rp[p.n] != p.nnz) { nd_set_error("a graph of the batch has an invalid row_ptr"); rc = ND_E_INVAL; break; }
            for (int64_t u = 0; u < p.n; ++u) hrp[p.n_off + u] = p.nnz_off + p.rp[u];
            for (int64_t j = 0; j < p.nnz; ++j) {
                const int32_t v = p.col[j];
                if (v < 0 || v >= p.n) { nd_set_error("a graph of the batch has a neighbour id outside its own vertex range"); rc = ND_E_INVAL; break; }
                hcol[p.nnz_off + j] = v + (int32_t)p.n_off;
            }
        }
        hrp[n] = nnz;
        if (rc == ND_OK) {
            nd_csr u{n, nnz, hrp.data(), hcol.data(), 0};
            rc = build_common(&u, r, s, st, out, 0, false);
        }
    }
    // the r-clique slice of every graph, and the graph of every r-clique
    std::vector<int64_t> roff(count + 1, 0);
    if (rc == ND_OK && count > 0) rc = nd_batch_offsets(*out, voff.data(), count, roff.data(), st);
    if (rc == ND_OK) rc = nd_batch_graph_ids(*out, roff.data(), count, st);
    if (rc == ND_OK && r_offsets) std::memcpy(r_offsets, roff.data(), sizeof(int64_t) * (count + 1));
    if (rc != ND_OK && *out) { nd_free(*out); *out = nullptr; }
    return rc;
}

nd_status nd_incidence_info(const nd_incidence* h, int64_t* num_r, int64_t* num_inc, int* q) {
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    if (num_r) *num_r = h->num_r;
    if (num_inc) *num_inc = h->num_inc;
    if (q) *q = h->q;
    return ND_OK;
}

nd_status nd_incidence_bytes(const nd_incidence* h, int64_t* bytes) {
    if (!h || !bytes) { nd_set_error("NULL argument"); return ND_E_INVAL; }
    *bytes = h->bytes;
    return ND_OK;
}

static nd_status deliver(const int32_t* src_dev, int64_t count, int32_t* dst, int on_device, cudaStream_t st) {
    if (count == 0) return ND_OK;
    if (on_device) {
        ND_CUDA(cudaMemcpyAsync(dst, src_dev, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, st));
        return ND_OK;
    }
    ND_CUDA(cudaMemcpyAsync(dst, src_dev, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
    return nd_wait(st);
}

nd_status nd_r_cliques(const nd_incidence* h, int32_t* out, int on_device, void* stream) {
    if (!h || (!out && h->num_r > 0)) { nd_set_error("NULL argument"); return ND_E_INVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const_cast<nd_incidence*>(h)->last_stream = st;
    const int64_t count = h->num_r * h->r;
    if (count == 0) return ND_OK;
    if (on_device) return nd_write_r_cliques(h, out, st);
    nd_tmp<int32_t> tmp(st);
    ND_TRY(tmp.alloc(count));
    ND_TRY(nd_write_r_cliques(h, tmp, st));
    return deliver(tmp, count, out, 0, st);
}

nd_status nd_s_degree(const nd_incidence* h, int32_t* out, int on_device, void* stream) {
    if (!h || (!out && h->num_r > 0)) { nd_set_error("NULL argument"); return ND_E_INVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const_cast<nd_incidence*>(h)->last_stream = st;
    if (h->num_r == 0) return ND_OK;
    if (on_device && !h->to_new) return nd_init_tau(const_cast<nd_incidence*>(h), out, st);
    nd_tmp<int32_t> tmp(st), tmp_old(st);
    ND_TRY(tmp.alloc(h->num_r));
    ND_TRY(nd_init_tau(const_cast<nd_incidence*>(h), tmp, st));
    const int32_t* res = tmp;
    if (h->to_new) {  // internal ids -> caller's ids
        ND_TRY(tmp_old.alloc(h->num_r));
        ND_TRY(nd_permute_i32(h->to_new, tmp, tmp_old, h->num_r, false, st));
        res = tmp_old;
    }
    if (on_device) {
        ND_CUDA(cudaMemcpyAsync(out, res, sizeof(int32_t) * h->num_r, cudaMemcpyDeviceToDevice, st));
        return nd_wait(st);  // the temporaries are released on return
    }
    return deliver(res, h->num_r, out, 0, st);
}

static nd_status run_and_deliver(nd_incidence* h, int mode, int32_t max_passes, const int32_t* tau_in,
                                 int tau_in_on_device, int32_t* tau_out, int on_device,
                                 int32_t* iters_out, int64_t* evals_out, bool require_convergence,
                                 cudaStream_t st, nd_run_opts* opts = nullptr) {
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    if (!tau_out && h->num_r > 0) { nd_set_error("tau_out is NULL"); return ND_E_INVAL; }
    if (mode != ND_SND && mode != ND_AND && mode != ND_AND_NN) { nd_set_error("bad mode"); return ND_E_INVAL; }
    if (max_passes < 0) { nd_set_error("negative iteration cap"); return ND_E_INVAL; }
    h->last_stream = st;
    const int32_t* tin_dev = nullptr;
    nd_tmp<int32_t> staged(st);
    if (tau_in && h->num_r > 0) {
        if (tau_in_on_device) {
            tin_dev = tau_in;
        } else {
            ND_TRY(staged.alloc(h->num_r));
            ND_CUDA(cudaMemcpyAsync(staged, tau_in, sizeof(int32_t) * h->num_r, cudaMemcpyHostToDevice, st));
            tin_dev = staged;
        }
    }
    nd_tmp<int32_t> tin_new(st), res_old(st);
    if (tin_dev && h->to_new) {  // caller's ids -> internal ids
        ND_TRY(tin_new.alloc(h->num_r));
        ND_TRY(nd_permute_i32(h->to_new, tin_dev, tin_new, h->num_r, true, st));
        tin_dev = tin_new;
    }
    int32_t* result = nullptr;
    int32_t updating = 0;
    int64_t evals = 0;
    bool converged = false;
    nd_status s = nd_run(h, mode, max_passes, tin_dev, &result, &updating, &evals, &converged, st, opts);
    if (s != ND_OK) return s;
    if (h->to_new && h->num_r > 0) {  // internal ids -> caller's ids
        ND_TRY(res_old.alloc(h->num_r));
        ND_TRY(nd_permute_i32(h->to_new, result, res_old, h->num_r, false, st));
        result = res_old;
    }
    s = deliver(result, h->num_r, tau_out, on_device, st);
    if (s != ND_OK) return s;
    if (on_device) ND_TRY(nd_wait(st));
    if (iters_out) *iters_out = updating;
    if (evals_out) *evals_out = evals;
    if (require_convergence && !converged && !(opts && opts->stopped)) {
        nd_set_error("iteration cap reached before a pass without change");
        return ND_E_NOT_CONVERGED;
    }
    return ND_OK;
}

nd_status nd_snd(nd_incidence* h, int32_t* tau_out, int on_device, int32_t max_iters,
                 int32_t* iters_out, void* stream) {
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    ND_CLAIM(h);
    return run_and_deliver(h, ND_SND, max_iters, nullptr, 0, tau_out, on_device, iters_out, nullptr, true,
                           (cudaStream_t)stream);
}

nd_status nd_and(nd_incidence* h, int32_t* tau_out, int on_device, int notify, int32_t max_iters,
                 int32_t* iters_out, int64_t* evals_out, void* stream) {
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    ND_CLAIM(h);
    return run_and_deliver(h, notify ? ND_AND : ND_AND_NN, max_iters, nullptr, 0, tau_out, on_device,
                           iters_out, evals_out, true, (cudaStream_t)stream);
}

nd_status nd_iterate_k(nd_incidence* h, int mode, int32_t k, int32_t* tau_inout, int tau_init_given,
                       int on_device, int32_t* updating_out, void* stream) {
    if (k < 0) { nd_set_error("negative k"); return ND_E_INVAL; }
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    ND_CLAIM(h);
    return run_and_deliver(h, mode, k, tau_init_given ? tau_inout : nullptr, on_device, tau_inout,
                           on_device, updating_out, nullptr, false, (cudaStream_t)stream);
}

nd_status nd_and_partial(nd_incidence* h, const uint32_t* members, int64_t count, int on_device,
                         int32_t* tau_out, int32_t max_iters, int32_t* iters_out, int64_t* evals_out,
                         void* stream) {
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    if (count < 0 || (count > 0 && !members)) { nd_set_error("bad member list"); return ND_E_INVAL; }
    ND_CLAIM(h);
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    const int64_t words = (h->num_r + 31) / 32;
    nd_tmp<uint32_t> mask(st), staged(st);
    nd_tmp<int> derr(st);
    ND_TRY(mask.alloc(words));
    ND_TRY(derr.alloc(1));
    ND_CUDA(cudaMemsetAsync(mask, 0, sizeof(uint32_t) * (words > 0 ? words : 1), st));
    ND_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    const uint32_t* ids = members;
    if (count > 0 && !on_device) {
        ND_TRY(staged.alloc(count));
        ND_CUDA(cudaMemcpyAsync(staged, members, sizeof(uint32_t) * count, cudaMemcpyHostToDevice, st));
        ids = staged;
    }
    ND_TRY(nd_member_mask(ids, count, h->num_r, mask, derr, st, h->to_new));
    int herr = 0;
    ND_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    if (herr) { nd_set_error("a member id is not an r-clique id"); return ND_E_INVAL; }
    nd_run_opts opts;
    opts.members = mask;
    return run_and_deliver(h, ND_AND, max_iters, nullptr, 0, tau_out, on_device, iters_out, evals_out, true, st,
                           &opts);
}

nd_status nd_and_until(nd_incidence* h, double active_ratio, int32_t* tau_out, int on_device, int32_t max_iters,
                       int32_t* iters_out, int64_t* evals_out, int* stopped_out, void* stream) {
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    if (!(active_ratio >= 0.0 && active_ratio <= 1.0)) { nd_set_error("active_ratio must be in [0,1]"); return ND_E_INVAL; }
    ND_CLAIM(h);
    nd_run_opts opts;
    opts.stop_active = active_ratio;
    nd_status rc = run_and_deliver(h, ND_AND, max_iters, nullptr, 0, tau_out, on_device, iters_out, evals_out,
                                   true, (cudaStream_t)stream, &opts);
    if (stopped_out) *stopped_out = opts.stopped ? 1 : 0;
    return rc;
}

nd_status nd_count_equal(const int32_t* a, const int32_t* b, int64_t n, int on_device, int64_t* equal_out,
                         void* stream) {
    if (n < 0 || !equal_out || (n > 0 && (!a || !b))) { nd_set_error("bad arguments"); return ND_E_INVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t *da = a, *db = b;
    nd_tmp<int32_t> sa(st), sb(st);
    nd_tmp<unsigned long long> dout(st);
    ND_TRY(dout.alloc(1));
    if (!on_device && n > 0) {
        ND_TRY(sa.alloc(n));
        ND_TRY(sb.alloc(n));
        ND_CUDA(cudaMemcpyAsync(sa, a, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        ND_CUDA(cudaMemcpyAsync(sb, b, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        da = sa;
        db = sb;
    }
    ND_TRY(nd_count_equal_dev(da, db, n, dout, st));
    unsigned long long hv = 0;
    ND_CUDA(cudaMemcpyAsync(&hv, dout, sizeof(hv), cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    *equal_out = (int64_t)hv;
    return ND_OK;
}

nd_status nd_truss_classic(const int32_t* kappa3, int64_t num_edges, int32_t* out, int on_device,
                           void* stream) {
    if (num_edges < 0 || (num_edges > 0 && (!kappa3 || !out))) { nd_set_error("bad arguments"); return ND_E_INVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (on_device || num_edges == 0) return nd_classic_truss(kappa3, num_edges, out, st);
    // host buffers: through the device like every other call
    nd_tmp<int32_t> din(st), dout(st);
    ND_TRY(din.alloc(num_edges));
    ND_TRY(dout.alloc(num_edges));
    ND_CUDA(cudaMemcpyAsync(din, kappa3, sizeof(int32_t) * num_edges, cudaMemcpyHostToDevice, st));
    ND_TRY(nd_classic_truss(din, num_edges, dout, st));
    ND_CUDA(cudaMemcpyAsync(out, dout, sizeof(int32_t) * num_edges, cudaMemcpyDeviceToHost, st));
    ND_TRY(nd_wait(st));
    return ND_OK;
}

nd_status nd_kendall_tau_b(const int32_t* x, const int32_t* y, int64_t n, int on_device, double* tau_out,
                           int64_t* counts_out, void* stream) {
    if (n < 0 || !tau_out || (n > 0 && (!x || !y))) { nd_set_error("bad arguments"); return ND_E_INVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    ND_CUDA(cudaGetDevice(&dev));
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    const int32_t *dx = x, *dy = y;
    nd_tmp<int32_t> sx(st), sy(st);
    if (!on_device && n > 0) {
        ND_TRY(sx.alloc(n));
        ND_TRY(sy.alloc(n));
        ND_CUDA(cudaMemcpyAsync(sx, x, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        ND_CUDA(cudaMemcpyAsync(sy, y, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        dx = sx;
        dy = sy;
    }
    return nd_kendall_dev(dx, dy, n, sms, tau_out, counts_out, st);
}

nd_status nd_autotune(nd_incidence* h, int32_t passes, void* stream, int32_t* thr_out, double* best_ms_out) {
    if (!h) { nd_set_error("handle is NULL"); return ND_E_INVAL; }
    if (passes < 1) passes = 2;
    ND_CLAIM(h);
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    int dev = 0;
    ND_CUDA(cudaGetDevice(&dev));
    static const int32_t T0[] = {4, 8}, T1[] = {32, 64}, T2[] = {256, 1024, 2048, 8192};
    std::array<int32_t, 3> best = {h->thr[0], h->thr[1], h->thr[2]};
    double best_ms = -1.0;
    cudaEvent_t a = nullptr, b = nullptr;
    ND_CUDA(cudaEventCreate(&a));
    ND_CUDA(cudaEventCreate(&b));
    nd_status rc = ND_OK;
    for (int32_t t0 : T0)
        for (int32_t t1 : T1)
            for (int32_t t2 : T2) {
                if (rc != ND_OK) break;
                h->thr[0] = t0;
                h->thr[1] = t1;
                h->thr[2] = t2;
                rc = nd_build_buckets(h, st);
                if (rc != ND_OK) break;
                int32_t* res = nullptr;
                int32_t upd = 0;
                int64_t ev = 0;
                bool conv = false;
                cudaEventRecord(a, st);
                rc = nd_run(h, ND_SND, passes, nullptr, &res, &upd, &ev, &conv, st);
                cudaEventRecord(b, st);
                if (rc != ND_OK) break;
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (best_ms < 0 || ms < best_ms) { best_ms = ms; best = {t0, t1, t2}; }
            }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != ND_OK) return rc;
    for (int i = 0; i < 3; ++i) h->thr[i] = best[i];
    ND_TRY(nd_build_buckets(h, st));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[std::make_tuple(dev, h->r, h->s, size_class(h))] = best;
    }
    if (thr_out) for (int i = 0; i < 3; ++i) thr_out[i] = best[i];
    if (best_ms_out) *best_ms_out = best_ms;
    return ND_OK;
}

nd_status nd_last_passes(const nd_incidence* h, int64_t* changed, int64_t* evaluated, int64_t* incidences,
                         int32_t cap, int32_t* passes) {
    if (!h || !passes) { nd_set_error("NULL argument"); return ND_E_INVAL; }
    ND_CLAIM(const_cast<nd_incidence*>(h));
    const int32_t n = (int32_t)h->last_changed.size();
    *passes = n;
    for (int32_t i = 0; i < n && i < cap; ++i) {
        if (changed) changed[i] = h->last_changed[i];
        if (evaluated) evaluated[i] = h->last_evals[i];
        if (incidences) incidences[i] = h->last_incs[i];
    }
    return ND_OK;
}

nd_status nd_prof_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    if (on) {
        for (auto& e : g_prof) { e.launches = 0; e.ms = 0.0; }
    }
    g_prof_on = (on != 0);
    return ND_OK;
}

nd_status nd_prof_read(int i, const char** name, int64_t* launches, double* total_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    if (i < 0 || i >= (int)g_prof.size()) return ND_E_INVAL;
    if (name) *name = g_prof[i].name.c_str();
    if (launches) *launches = g_prof[i].launches;
    if (total_ms) *total_ms = g_prof[i].ms;
    return ND_OK;
}

}  // extern "C"
