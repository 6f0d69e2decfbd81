/*
 * Plain SND over all host cores, for the CPU baseline of the benchmark.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: only the tests and the CPU
 * baseline of the benchmark may load this file's library.  It shares no
 * code, header or table with the CUDA library.
 *
 * The arithmetic is that of orc_snd in oracle.c, unchanged:
 *   - tau_0 = d_s (Alg. 2 starts from the S-degrees, Def. 1);
 *   - one pass evaluates, for every r-clique R, rho of each s-clique S of R
 *     as the minimum tau_p over the other r-cliques of S (Def. 4), and sets
 *     tau(R) to the h-index of those values, found by sorting (Def. 3),
 *     reading only the previous pass's array tau_p (Alg. 2).
 * The only difference is that the loop over R of each pass, and the loops of
 * the incidence construction, are split over OpenMP threads.  Each R is
 * written by one thread and reads only tau_p, so the result of a pass does
 * not depend on the split.  (1,2) and (2,3) only.
 *
 * Incidence (Def. 1): for (1,2) the s-cliques of vertex u are its edges, and
 * the other r-clique of each is the neighbour.  For (2,3) the r-cliques are
 * the edges u < v in lexicographic order; the s-cliques of edge (u,v) are the
 * triangles {u,v,w}, w a common neighbour (sorted merge of the two rows), and
 * their other r-cliques are the edges (u,w) and (v,w).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OMT_OK 0
#define OMT_E_INVAL (-1)
#define OMT_E_NOMEM (-2)
#define OMT_E_THM1 (-3)
#define OMT_E_RS (-4)

typedef struct omt_ctx {
    int r, q;
    int64_t num_r;
    int64_t *inc_off; /* num_r + 1 */
    int32_t *inc;     /* inc_off[num_r] * q */
    int owns;         /* inc_off / inc allocated here (r = 2) */
    int32_t max_ds;
} omt_ctx;

int omt_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void set_threads(int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

void omt_free(omt_ctx *c) {
    if (!c) return;
    if (c->owns) { free(c->inc_off); free(c->inc); }
    free(c);
}

/* first slot of row u holding a neighbour larger than u (rows sorted) */
static int64_t first_upper(const int64_t *rp, const int32_t *col, int64_t u) {
    int64_t lo = rp[u], hi = rp[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] <= u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int64_t find_slot(const int64_t *rp, const int32_t *col, int64_t u, int32_t v) {
    int64_t lo = rp[u], hi = rp[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (lo < rp[u + 1] && col[lo] == v) ? lo : -1;
}

/* The incidence of the graph (simple, symmetric, sorted CSR: the caller
 * passes what the oracle has validated).  rp / col must outlive the context
 * for r = 1 (the CSR is the incidence). */
int omt_create(int64_t n, const int64_t *rp, const int32_t *col, int r, int threads, omt_ctx **out) {
    *out = NULL;
    if (r != 1 && r != 2) return OMT_E_RS;
    if (n < 0) return OMT_E_INVAL;
    set_threads(threads);
    omt_ctx *c = (omt_ctx *)calloc(1, sizeof(omt_ctx));
    if (!c) return OMT_E_NOMEM;
    c->r = r;
    c->q = r == 1 ? 1 : 2;
    if (r == 1) {
        c->num_r = n;
        c->inc_off = (int64_t *)rp;
        c->inc = (int32_t *)col;
        int32_t mx = 0;
        for (int64_t u = 0; u < n; ++u)
            if (rp[u + 1] - rp[u] > mx) mx = (int32_t)(rp[u + 1] - rp[u]);
        c->max_ds = mx;
        *out = c;
        return OMT_OK;
    }
    const int64_t nnz = rp[n];
    int64_t *ebase = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    int64_t *fup = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    int32_t *slot_eid = (int32_t *)malloc(sizeof(int32_t) * (nnz + 1));
    if (!ebase || !fup || !slot_eid) { free(ebase); free(fup); free(slot_eid); free(c); return OMT_E_NOMEM; }
    /* edges owned by each row (u < v), and their first ids */
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u) fup[u] = first_upper(rp, col, u);
    int64_t m = 0;
    for (int64_t u = 0; u < n; ++u) { ebase[u] = m; m += rp[u + 1] - fup[u]; }
    ebase[n] = m;
    c->num_r = m;
    if (m > INT32_MAX) { free(ebase); free(fup); free(slot_eid); free(c); return OMT_E_INVAL; }
    /* edge id of every CSR slot: (u, v) with u < v is ebase[u] + its rank
     * among the upper slots of row u; (u, v) with v < u is the same edge seen
     * from row v */
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
            int32_t v = col[p];
            if (v > u) {
                slot_eid[p] = (int32_t)(ebase[u] + (p - fup[u]));
            } else {
                int64_t q = find_slot(rp, col, v, (int32_t)u);
                if (q < 0) { bad = 1; slot_eid[p] = -1; continue; }
                slot_eid[p] = (int32_t)(ebase[v] + (q - fup[v]));
            }
        }
    }
    /* endpoints of every edge */
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (m + 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (m + 1));
    c->inc_off = (int64_t *)malloc(sizeof(int64_t) * (m + 1));
    c->owns = 1;
    if (bad || !eu || !ev || !c->inc_off) {
        free(ebase); free(fup); free(slot_eid); free(eu); free(ev); omt_free(c);
        return bad ? OMT_E_INVAL : OMT_E_NOMEM;
    }
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u)
        for (int64_t p = fup[u]; p < rp[u + 1]; ++p) {
            eu[ebase[u] + (p - fup[u])] = (int32_t)u;
            ev[ebase[u] + (p - fup[u])] = col[p];
        }
    /* triangles per edge: common neighbours of u and v (sorted merge) */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = rp[eu[e]], ie = rp[eu[e] + 1], j = rp[ev[e]], je = rp[ev[e] + 1], k = 0;
        while (i < ie && j < je) {
            if (col[i] < col[j]) i++;
            else if (col[j] < col[i]) j++;
            else { k++; i++; j++; }
        }
        c->inc_off[e + 1] = k;
    }
    c->inc_off[0] = 0;
    int32_t mx = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (c->inc_off[e + 1] > mx) mx = (int32_t)c->inc_off[e + 1];
        c->inc_off[e + 1] += c->inc_off[e];
    }
    c->max_ds = mx;
    c->inc = (int32_t *)malloc(sizeof(int32_t) * (2 * c->inc_off[m] + 1));
    if (!c->inc) { free(ebase); free(fup); free(slot_eid); free(eu); free(ev); omt_free(c); return OMT_E_NOMEM; }
    /* fill: the triangle {u,v,w} of edge (u,v) lists edges (u,w) and (v,w) */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = rp[eu[e]], ie = rp[eu[e] + 1], j = rp[ev[e]], je = rp[ev[e] + 1], k = c->inc_off[e];
        while (i < ie && j < je) {
            if (col[i] < col[j]) i++;
            else if (col[j] < col[i]) j++;
            else {
                c->inc[2 * k] = slot_eid[i];
                c->inc[2 * k + 1] = slot_eid[j];
                k++; i++; j++;
            }
        }
    }
    free(ebase); free(fup); free(slot_eid); free(eu); free(ev);
    *out = c;
    return OMT_OK;
}

int64_t omt_num_r(const omt_ctx *c) { return c->num_r; }
int64_t omt_num_incidences(const omt_ctx *c) { return c->inc_off[c->num_r]; }

static int cmp_desc(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x < y) - (x > y);
}

/* H by sorting (Def. 3): the largest h with at least h values >= h */
static int32_t hindex_sorted(int32_t *vals, int64_t len) {
    qsort(vals, (size_t)len, sizeof(int32_t), cmp_desc);
    int64_t h = 0;
    while (h < len && vals[h] >= h + 1) h++;
    return (int32_t)h;
}

/* At most `passes` SND passes (Alg. 2) on tau, from d_s when init_from_ds;
 * stops after a pass with no change.  *updating_out = passes that changed a
 * tau, *evals_out = r-cliques evaluated, *sweeps_out = passes run. */
int omt_snd(const omt_ctx *c, int32_t *tau, int init_from_ds, int32_t passes, int threads, int32_t *sweeps_out,
            int32_t *updating_out, int64_t *evals_out) {
    set_threads(threads);
    const int64_t N = c->num_r;
    if (init_from_ds) {
#pragma omp parallel for schedule(static)
        for (int64_t R = 0; R < N; ++R) tau[R] = (int32_t)(c->inc_off[R + 1] - c->inc_off[R]);
    }
    int32_t *tp = (int32_t *)malloc(sizeof(int32_t) * (N + 1));
    if (!tp) return OMT_E_NOMEM;
    int32_t sweeps = 0, updating = 0;
    int64_t evals = 0;
    int st = OMT_OK;
    while (sweeps < passes) {
        memcpy(tp, tau, sizeof(int32_t) * N);
        int changed = 0, raised = 0, nomem = 0;
#pragma omp parallel reduction(| : changed, raised, nomem)
        {
            int32_t *L = (int32_t *)malloc(sizeof(int32_t) * ((int64_t)c->max_ds + 1));
            if (!L) nomem = 1;
#pragma omp for schedule(dynamic, 256)
            for (int64_t R = 0; R < N; ++R) {
                if (!L) continue;
                const int64_t b = c->inc_off[R], e = c->inc_off[R + 1];
                for (int64_t j = b; j < e; ++j) {
                    const int32_t *S = c->inc + j * c->q;
                    int32_t rho = tp[S[0]];
                    for (int k = 1; k < c->q; ++k) if (tp[S[k]] < rho) rho = tp[S[k]];
                    L[j - b] = rho;
                }
                const int32_t h = hindex_sorted(L, e - b);
                if (h > tp[R]) raised = 1;
                if (h != tp[R]) changed = 1;
                tau[R] = h;
            }
            free(L);
        }
        if (nomem) { st = OMT_E_NOMEM; break; }
        if (raised) { st = OMT_E_THM1; break; }
        sweeps++;
        evals += N;
        if (!changed) break;
        updating++;
    }
    free(tp);
    if (sweeps_out) *sweeps_out = sweeps;
    if (updating_out) *updating_out = updating;
    if (evals_out) *evals_out = evals;
    return st;
}
