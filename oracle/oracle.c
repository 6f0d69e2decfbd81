/*
 * CPU oracle for local nucleus decomposition (Sariyuce, Seshadhri, Pinar,
 * "Local Algorithms for Hierarchical Dense Subgraph Discovery").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this file's library.  It shares no
 * code, header or table with the CUDA library and must never serve as a
 * fallback for it.
 *
 * Plain, slow, single-threaded C.  Every routine follows one passage:
 *   - input: a simple undirected graph as a symmetric CSR ... Section 2
 *   - r-cliques, s-cliques and the S-degree d_s ............ Section 2, Def. 1
 *   - h-index H(K) by sorting ............................... Section 2.2, Def. 3
 *   - kappa_s by peeling (Batagelj-Zaversnik bins) .......... Section 2, Alg. 1
 *   - update operator U and SND ............................. Section 3 Def. 4, Section 4.1 Alg. 2
 *   - AND, with and without notification .................... Section 4.2 Alg. 3, Section 4.3
 *   - degree levels ......................................... Section 3.1, Def. 5
 *   - Kendall-Tau of tau against kappa (tau-b) .............. Section 5.2, Fig. 7
 *
 * Readings of the paper used here:
 *   - rho(S,R) is the minimum over the r-cliques of S other than R (Def. 4
 *     and Fig. 4); the min over the whole neighbourhood N_s(R) written in the
 *     algorithm listings is read as the same thing.
 *   - H of the empty multiset is 0; an r-clique in no s-clique keeps tau = 0.
 *   - AND with notification: an updated r-clique notifies the neighbours
 *     whose tau is >= the new value; it does not re-activate itself (the
 *     reading that reproduces the 9 computations in 3 iterations traced for
 *     Fig. 6).
 *   - Iteration counts: `sweeps` counts every pass over the r-cliques,
 *     `updating` counts the passes that changed at least one tau (the two
 *     iterations the paper gives SND on Fig. 5 are updating passes).
 *   - Canonical r-clique ids: lexicographic order of the sorted vertex tuple.
 *   - Kendall-Tau: the paper compares the ranking of the r-cliques by tau
 *     with the ranking by kappa and does not name the variant; with the many
 *     ties of integer indices the tie-corrected tau-b is used.
 *
 * Parity is pinned by the tests in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_INVAL (-1)
#define ORC_E_NOMEM (-2)
#define ORC_E_THM1 (-3) /* an update raised a tau: Thm. 1 says this never happens */
#define ORC_E_RS (-4)

typedef struct orc_ctx {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    int r, s, q;
    int64_t num_r;
    /* edges u<v in lexicographic order (r >= 2) */
    int64_t m;
    int32_t *eu, *ev;
    int64_t *ebase; /* edge id of (u,v) = ebase[u] + position of v in row u */
    /* triangles u<v<w grouped by edge (u,v), w ascending (r == 3) */
    int64_t *tri_off; /* m+1 */
    int32_t *tri_w;
    int64_t ntri;
    /* oracle-owned incidence: for each R, q ids per s-clique containing R */
    int64_t *inc_off; /* num_r + 1, counts s-cliques */
    int32_t *inc;     /* inc_off[num_r] * q */
    int32_t maxdeg;
} orc_ctx;

/* ---- adjacency helpers (Section 2: simple undirected graph) ---- */

static int64_t row_find(const orc_ctx *c, int32_t u, int32_t v) {
    int64_t lo = c->rp[u], hi = c->rp[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (c->col[mid] < v) lo = mid + 1; else hi = mid;
    }
    if (lo < c->rp[u + 1] && c->col[lo] == v) return lo;
    return -1;
}

static int adjacent(const orc_ctx *c, int32_t u, int32_t v) { return row_find(c, u, v) >= 0; }

static int64_t edge_id(const orc_ctx *c, int32_t u, int32_t v) {
    if (u > v) { int32_t t = u; u = v; v = t; }
    int64_t p = row_find(c, u, v);
    if (p < 0) return -1;
    return c->ebase[u] + p;
}

static void sort3(int32_t *a, int32_t *b, int32_t *x) {
    int32_t t;
    if (*a > *b) { t = *a; *a = *b; *b = t; }
    if (*b > *x) { t = *b; *b = *x; *x = t; }
    if (*a > *b) { t = *a; *a = *b; *b = t; }
}

static int64_t tri_id(const orc_ctx *c, int32_t a, int32_t b, int32_t x) {
    sort3(&a, &b, &x);
    int64_t e = edge_id(c, a, b);
    if (e < 0) return -1;
    int64_t lo = c->tri_off[e], hi = c->tri_off[e + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (c->tri_w[mid] < x) lo = mid + 1; else hi = mid;
    }
    if (lo < c->tri_off[e + 1] && c->tri_w[lo] == x) return lo;
    return -1;
}

/* common neighbours of u and v (sorted merge), written to out; returns count */
static int64_t common2(const orc_ctx *c, int32_t u, int32_t v, int32_t *out) {
    int64_t i = c->rp[u], ie = c->rp[u + 1], j = c->rp[v], je = c->rp[v + 1], k = 0;
    while (i < ie && j < je) {
        int32_t a = c->col[i], b = c->col[j];
        if (a < b) i++;
        else if (b < a) j++;
        else { if (out) out[k] = a; k++; i++; j++; }
    }
    return k;
}

/* ---- s-cliques containing R, listed as the q other r-cliques of each (Def. 1) ---- */

/* Writes q ids per s-clique of R into buf (may be NULL to count).  tmp must
 * hold maxdeg ints.  Returns the number of s-cliques, or -1 on a lookup
 * failure (cannot happen on a valid graph). */
static int64_t s_cliques_of(const orc_ctx *c, int64_t R, int32_t *buf, int32_t *tmp) {
    if (c->r == 1) {
        int32_t u = (int32_t)R;
        int64_t k = 0;
        for (int64_t p = c->rp[u]; p < c->rp[u + 1]; ++p, ++k)
            if (buf) buf[k] = c->col[p];
        return k;
    }
    if (c->r == 2) {
        int32_t u = c->eu[R], v = c->ev[R];
        int64_t k = common2(c, u, v, tmp);
        if (buf)
            for (int64_t i = 0; i < k; ++i) {
                int64_t a = edge_id(c, u, tmp[i]), b = edge_id(c, v, tmp[i]);
                if (a < 0 || b < 0) return -1;
                buf[2 * i] = (int32_t)a;
                buf[2 * i + 1] = (int32_t)b;
            }
        return k;
    }
    /* r == 3: triangle (u,v,w) = (eu[e], ev[e], tri_w[R]) where e owns R */
    int64_t lo = 0, hi = c->m;
    while (hi - lo > 1) { /* largest e with tri_off[e] <= R */
        int64_t mid = lo + (hi - lo) / 2;
        if (c->tri_off[mid] <= R) lo = mid; else hi = mid;
    }
    while (lo + 1 <= c->m && c->tri_off[lo + 1] <= R) lo++;
    int32_t u = c->eu[lo], v = c->ev[lo], w = c->tri_w[R];
    int64_t k2 = common2(c, u, v, tmp), k = 0;
    for (int64_t i = 0; i < k2; ++i) {
        int32_t x = tmp[i];
        if (x == w || !adjacent(c, w, x)) continue;
        if (buf) {
            int64_t a = tri_id(c, u, v, x), b = tri_id(c, u, w, x), d = tri_id(c, v, w, x);
            if (a < 0 || b < 0 || d < 0) return -1;
            buf[3 * k] = (int32_t)a;
            buf[3 * k + 1] = (int32_t)b;
            buf[3 * k + 2] = (int32_t)d;
        }
        k++;
    }
    return k;
}

/* ---- construction ---- */

/* The graph of Section 2 is simple and undirected: rows strictly increasing
 * (no duplicate edge), no self-loop, every id in range, and the adjacency
 * symmetric.  Anything else is rejected, never repaired. */
static int validate(int64_t n, const int64_t *rp, const int32_t *col) {
    if (n < 0 || rp[0] != 0) return ORC_E_INVAL;
    /* offsets first: non-decreasing, so every row lies inside col[0, rp[n]) */
    for (int64_t u = 0; u < n; ++u)
        if (rp[u + 1] < rp[u]) return ORC_E_INVAL;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
            int32_t v = col[p];
            if (v < 0 || v >= n || v == u) return ORC_E_INVAL;
            if (p > rp[u] && col[p - 1] >= v) return ORC_E_INVAL;
        }
    }
    /* symmetry: build the transpose by a counting sort (rows visited in
     * increasing u, so its rows come out sorted); the graph is symmetric iff
     * the transpose equals the CSR itself */
    const int64_t nnz = rp[n];
    int64_t *tp = (int64_t *)calloc((size_t)n + 2, sizeof(int64_t));
    int32_t *tc = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nnz + 1));
    if (!tp || !tc) { free(tp); free(tc); return ORC_E_NOMEM; }
    for (int64_t p = 0; p < nnz; ++p) tp[col[p] + 1]++;
    for (int64_t v = 0; v < n; ++v) tp[v + 1] += tp[v];
    int st = ORC_OK;
    for (int64_t v = 0; v <= n && st == ORC_OK; ++v)
        if (tp[v] != rp[v]) st = ORC_E_INVAL;
    if (st == ORC_OK) {
        for (int64_t u = 0; u < n; ++u)
            for (int64_t p = rp[u]; p < rp[u + 1]; ++p) tc[tp[col[p]]++] = (int32_t)u;
        for (int64_t p = 0; p < nnz && st == ORC_OK; ++p)
            if (tc[p] != col[p]) st = ORC_E_INVAL;
    }
    free(tp); free(tc);
    return st;
}

void orc_free(orc_ctx *c) {
    if (!c) return;
    free(c->eu); free(c->ev); free(c->ebase); free(c->tri_off); free(c->tri_w);
    free(c->inc_off); free(c->inc);
    free(c);
}

/* The r-cliques of the graph and, with with_incidence, the s-cliques of each
 * (Def. 1): vertices for r = 1; edges u < v in lexicographic order for r = 2;
 * for r = 3 the triangles u < v < w, grouped by their edge (u, v) and listed
 * by w.  Each s-clique of R is stored as the ids of its q other r-cliques. */
int orc_create(int64_t n, const int64_t *rp, const int32_t *col, int r, int s, int with_incidence,
               orc_ctx **out) {
    *out = NULL;
    if (!((r == 1 && s == 2) || (r == 2 && s == 3) || (r == 3 && s == 4))) return ORC_E_RS;
    int st = validate(n, rp, col);
    if (st) return st;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!c) return ORC_E_NOMEM;
    c->n = n; c->rp = rp; c->col = col; c->r = r; c->s = s;
    c->q = (r == 1) ? 1 : (r == 2 ? 2 : 3); /* C(s,r) - 1 */
    c->maxdeg = 0;
    for (int64_t u = 0; u < n; ++u)
        if (rp[u + 1] - rp[u] > c->maxdeg) c->maxdeg = (int32_t)(rp[u + 1] - rp[u]);
    if (r == 1) {
        c->num_r = n;
    } else {
        c->m = rp[n] / 2;
        c->eu = (int32_t *)malloc(sizeof(int32_t) * (c->m + 1));
        c->ev = (int32_t *)malloc(sizeof(int32_t) * (c->m + 1));
        c->ebase = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
        if (!c->eu || !c->ev || !c->ebase) { orc_free(c); return ORC_E_NOMEM; }
        int64_t e = 0;
        for (int64_t u = 0; u < n; ++u) {
            int64_t first = -1;
            for (int64_t p = rp[u]; p < rp[u + 1]; ++p)
                if (col[p] > u) {
                    if (first < 0) first = p;
                    c->eu[e] = (int32_t)u; c->ev[e] = col[p]; e++;
                }
            c->ebase[u] = (first < 0) ? 0 : (e - (rp[u + 1] - first)) - first;
        }
        if (e != c->m) { orc_free(c); return ORC_E_INVAL; }
        c->num_r = c->m;
        if (r == 3) {
            int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (c->maxdeg + 1));
            c->tri_off = (int64_t *)malloc(sizeof(int64_t) * (c->m + 1));
            if (!tmp || !c->tri_off) { free(tmp); orc_free(c); return ORC_E_NOMEM; }
            int64_t t = 0;
            for (int64_t k = 0; k < c->m; ++k) {
                c->tri_off[k] = t;
                int64_t cnt = common2(c, c->eu[k], c->ev[k], tmp);
                for (int64_t i = 0; i < cnt; ++i) t += (tmp[i] > c->ev[k]);
            }
            c->tri_off[c->m] = t;
            c->ntri = t;
            c->tri_w = (int32_t *)malloc(sizeof(int32_t) * (t + 1));
            if (!c->tri_w) { free(tmp); orc_free(c); return ORC_E_NOMEM; }
            for (int64_t k = 0; k < c->m; ++k) {
                int64_t cnt = common2(c, c->eu[k], c->ev[k], tmp), o = c->tri_off[k];
                for (int64_t i = 0; i < cnt; ++i)
                    if (tmp[i] > c->ev[k]) c->tri_w[o++] = tmp[i];
            }
            free(tmp);
            c->num_r = t;
        }
    }
    if (with_incidence) {
        int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (c->maxdeg + 1));
        c->inc_off = (int64_t *)malloc(sizeof(int64_t) * (c->num_r + 1));
        if (!tmp || !c->inc_off) { free(tmp); orc_free(c); return ORC_E_NOMEM; }
        int64_t tot = 0;
        for (int64_t R = 0; R < c->num_r; ++R) {
            c->inc_off[R] = tot;
            int64_t k = s_cliques_of(c, R, NULL, tmp);
            if (k < 0) { free(tmp); orc_free(c); return ORC_E_INVAL; }
            tot += k;
        }
        c->inc_off[c->num_r] = tot;
        c->inc = (int32_t *)malloc(sizeof(int32_t) * (tot * c->q + 1));
        if (!c->inc) { free(tmp); orc_free(c); return ORC_E_NOMEM; }
        for (int64_t R = 0; R < c->num_r; ++R)
            if (s_cliques_of(c, R, c->inc + c->inc_off[R] * c->q, tmp) < 0) {
                free(tmp); orc_free(c); return ORC_E_INVAL;
            }
        free(tmp);
    }
    *out = c;
    return ORC_OK;
}

int64_t orc_num_r(const orc_ctx *c) { return c->num_r; }
int64_t orc_num_s_incidences(const orc_ctx *c) { return c->inc_off ? c->inc_off[c->num_r] : -1; }
int orc_q(const orc_ctx *c) { return c->q; }

/* r-clique vertex tuples in canonical order: the lexicographic order of the
 * sorted vertex tuples (the id convention both implementations share) */
void orc_r_tuples(const orc_ctx *c, int32_t *out) {
    if (c->r == 1) {
        for (int64_t u = 0; u < c->n; ++u) out[u] = (int32_t)u;
    } else if (c->r == 2) {
        for (int64_t e = 0; e < c->m; ++e) { out[2 * e] = c->eu[e]; out[2 * e + 1] = c->ev[e]; }
    } else {
        for (int64_t e = 0; e < c->m; ++e)
            for (int64_t t = c->tri_off[e]; t < c->tri_off[e + 1]; ++t) {
                out[3 * t] = c->eu[e]; out[3 * t + 1] = c->ev[e]; out[3 * t + 2] = c->tri_w[t];
            }
    }
}

/* d_s(R): number of s-cliques containing R (Def. 1), counted from adjacency */
int orc_s_degree(const orc_ctx *c, int32_t *ds) {
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (c->maxdeg + 1));
    if (!tmp) return ORC_E_NOMEM;
    for (int64_t R = 0; R < c->num_r; ++R) {
        int64_t k = s_cliques_of(c, R, NULL, tmp);
        if (k < 0) { free(tmp); return ORC_E_INVAL; }
        ds[R] = (int32_t)k;
    }
    free(tmp);
    return ORC_OK;
}

/* ---- h-index (Def. 3): largest h with at least h values >= h; by sorting ---- */

static int cmp_desc(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x < y) - (x > y);
}

int32_t orc_hindex(int32_t *vals, int64_t len) {
    qsort(vals, (size_t)len, sizeof(int32_t), cmp_desc);
    int64_t h = 0;
    while (h < len && vals[h] >= h + 1) h++;
    return (int32_t)h;
}

/* ---- peeling, Alg. 1 (with Batagelj-Zaversnik bin sort for the queue) ---- */

int orc_peel(const orc_ctx *c, int32_t *kappa) {
    int64_t N = c->num_r;
    int st = ORC_OK;
    int32_t *d = (int32_t *)malloc(sizeof(int32_t) * (N + 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (c->maxdeg + 1));
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * ((int64_t)c->maxdeg * c->q + 1));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (N + 1));
    int64_t *vert = (int64_t *)malloc(sizeof(int64_t) * (N + 1));
    char *done = (char *)calloc((size_t)N + 1, 1);
    int64_t *bin = NULL;
    if (!d || !tmp || !buf || !pos || !vert || !done) { st = ORC_E_NOMEM; goto out; }
    st = orc_s_degree(c, d);
    if (st) goto out;
    int32_t md = 0;
    for (int64_t R = 0; R < N; ++R) if (d[R] > md) md = d[R];
    bin = (int64_t *)calloc((size_t)md + 2, sizeof(int64_t));
    if (!bin) { st = ORC_E_NOMEM; goto out; }
    for (int64_t R = 0; R < N; ++R) bin[d[R]]++;
    int64_t start = 0;
    for (int32_t k = 0; k <= md; ++k) { int64_t num = bin[k]; bin[k] = start; start += num; }
    for (int64_t R = 0; R < N; ++R) { pos[R] = bin[d[R]]; vert[pos[R]] = R; bin[d[R]]++; }
    for (int32_t k = md; k >= 1; --k) bin[k] = bin[k - 1];
    bin[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t R = vert[i];
        kappa[R] = d[R]; /* popped with minimum remaining S-degree */
        int64_t ns = s_cliques_of(c, R, buf, tmp);
        if (ns < 0) { st = ORC_E_INVAL; goto out; }
        for (int64_t j = 0; j < ns; ++j) {
            const int32_t *S = buf + j * c->q;
            int skip = 0;
            for (int k = 0; k < c->q; ++k) if (done[S[k]]) skip = 1;
            if (skip) continue; /* an r-clique of this s-clique is already peeled */
            for (int k = 0; k < c->q; ++k) {
                int64_t Rp = S[k];
                if (d[Rp] > d[R]) {
                    int32_t du = d[Rp];
                    int64_t pu = pos[Rp], pw = bin[du], w = vert[pw];
                    if (Rp != w) { pos[Rp] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = Rp; }
                    bin[du]++;
                    d[Rp]--;
                }
            }
        }
        done[R] = 1;
    }
out:
    free(d); free(tmp); free(buf); free(pos); free(vert); free(done); free(bin);
    return st;
}

/* ---- update operator (Def. 4) evaluated for one R against the array src ---- */

static int32_t update_one(const orc_ctx *c, int64_t R, const int32_t *src, int32_t *L) {
    int64_t b = c->inc_off[R], e = c->inc_off[R + 1];
    for (int64_t j = b; j < e; ++j) {
        const int32_t *S = c->inc + j * c->q;
        int32_t rho = src[S[0]];
        for (int k = 1; k < c->q; ++k) if (src[S[k]] < rho) rho = src[S[k]];
        L[j - b] = rho;
    }
    return orc_hindex(L, e - b);
}

/* tau_0 = d_s (Alg. 2 and Alg. 3 start from the S-degrees); with
 * init_from_ds = 0 the caller's tau is the start (any kappa <= tau <= d_s) */
static int init_tau(const orc_ctx *c, int32_t *tau, int init_from_ds) {
    if (!c->inc_off) return ORC_E_INVAL;
    if (init_from_ds)
        for (int64_t R = 0; R < c->num_r; ++R) tau[R] = (int32_t)(c->inc_off[R + 1] - c->inc_off[R]);
    return ORC_OK;
}

static int32_t max_ds(const orc_ctx *c) {
    int64_t mx = 0;
    for (int64_t R = 0; R < c->num_r; ++R)
        if (c->inc_off[R + 1] - c->inc_off[R] > mx) mx = c->inc_off[R + 1] - c->inc_off[R];
    return (int32_t)mx;
}

/* SND, Alg. 2: tau_{t+1} = U tau_t from the backup array; stops after a pass
 * with no change or after max_sweeps passes. */
int orc_snd(const orc_ctx *c, int32_t *tau, int init_from_ds, int32_t max_sweeps,
            int32_t *sweeps_out, int32_t *updating_out, int64_t *evals_out) {
    int st = init_tau(c, tau, init_from_ds);
    if (st) return st;
    int64_t N = c->num_r;
    int32_t *tp = (int32_t *)malloc(sizeof(int32_t) * (N + 1));
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * (max_ds(c) + 1));
    if (!tp || !L) { free(tp); free(L); return ORC_E_NOMEM; }
    int32_t sweeps = 0, updating = 0;
    int64_t evals = 0;
    while (sweeps < max_sweeps) {
        int flag = 0;
        memcpy(tp, tau, sizeof(int32_t) * N);
        for (int64_t R = 0; R < N; ++R) {
            int32_t h = update_one(c, R, tp, L);
            evals++;
            if (h > tp[R]) { st = ORC_E_THM1; goto out; }
            if (h != tp[R]) flag = 1;
            tau[R] = h;
        }
        sweeps++;
        if (!flag) break;
        updating++;
    }
out:
    if (sweeps_out) *sweeps_out = sweeps;
    if (updating_out) *updating_out = updating;
    if (evals_out) *evals_out = evals;
    free(tp); free(L);
    return st;
}

/* AND, Alg. 3: in-place updates in the given order (NULL = id order); with
 * notify, only notified r-cliques are recomputed (Section 4.3).  PartialAnd
 * (end of Section 4.3) is the same loop restricted to a member set P
 * (members[R] != 0): only members start active, only members are ever
 * notified, and non-members keep their initial tau.  members = NULL means
 * every r-clique is a member. */
int orc_and_partial(const orc_ctx *c, int32_t *tau, int init_from_ds, const int64_t *order, int notify,
                    const char *members, int32_t max_sweeps, int32_t *sweeps_out, int32_t *updating_out,
                    int64_t *evals_out) {
    int st = init_tau(c, tau, init_from_ds);
    if (st) return st;
    int64_t N = c->num_r;
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * (max_ds(c) + 1));
    char *act = (char *)malloc((size_t)N + 1);
    if (!L || !act) { free(L); free(act); return ORC_E_NOMEM; }
    for (int64_t R = 0; R < N; ++R) act[R] = members ? (members[R] != 0) : 1;
    int32_t sweeps = 0, updating = 0;
    int64_t evals = 0;
    while (sweeps < max_sweeps) {
        int flag = 0;
        for (int64_t i = 0; i < N; ++i) {
            int64_t R = order ? order[i] : i;
            if (members && !members[R]) continue;
            if (notify) {
                if (!act[R]) continue;
                act[R] = 0;
            }
            int32_t h = update_one(c, R, tau, L);
            evals++;
            if (h > tau[R]) { st = ORC_E_THM1; goto out; }
            if (h != tau[R]) {
                flag = 1;
                if (notify) {
                    for (int64_t j = c->inc_off[R]; j < c->inc_off[R + 1]; ++j)
                        for (int k = 0; k < c->q; ++k) {
                            int32_t Rp = c->inc[j * c->q + k];
                            if (h <= tau[Rp] && (!members || members[Rp])) act[Rp] = 1;
                        }
                }
                tau[R] = h;
            }
        }
        sweeps++;
        if (!flag) break;
        updating++;
    }
out:
    if (sweeps_out) *sweeps_out = sweeps;
    if (updating_out) *updating_out = updating;
    if (evals_out) *evals_out = evals;
    free(L); free(act);
    return st;
}

int orc_and(const orc_ctx *c, int32_t *tau, int init_from_ds, const int64_t *order, int notify,
            int32_t max_sweeps, int32_t *sweeps_out, int32_t *updating_out, int64_t *evals_out) {
    return orc_and_partial(c, tau, init_from_ds, order, notify, NULL, max_sweeps, sweeps_out, updating_out,
                           evals_out);
}

/* SND restricted to a member set: members are updated synchronously from the
 * previous pass (Alg. 2), non-members keep their tau.  Used to pin PartialAnd:
 * both iterate a monotone operator down from the same start, so they reach
 * the same (greatest) fixed point. */
int orc_snd_partial(const orc_ctx *c, int32_t *tau, int init_from_ds, const char *members, int32_t max_sweeps,
                    int32_t *sweeps_out) {
    int st = init_tau(c, tau, init_from_ds);
    if (st) return st;
    int64_t N = c->num_r;
    int32_t *tp = (int32_t *)malloc(sizeof(int32_t) * (N + 1));
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * (max_ds(c) + 1));
    if (!tp || !L) { free(tp); free(L); return ORC_E_NOMEM; }
    int32_t sweeps = 0;
    while (sweeps < max_sweeps) {
        int flag = 0;
        memcpy(tp, tau, sizeof(int32_t) * N);
        for (int64_t R = 0; R < N; ++R) {
            if (!members[R]) continue;
            int32_t h = update_one(c, R, tp, L);
            if (h > tp[R]) { st = ORC_E_THM1; goto out; }
            if (h != tp[R]) flag = 1;
            tau[R] = h;
        }
        sweeps++;
        if (!flag) break;
    }
out:
    if (sweeps_out) *sweeps_out = sweeps;
    free(tp); free(L);
    return st;
}

/* ---- degree levels, Def. 5: remove every r-clique of the current minimum
 * S-degree together with its s-cliques, level by level.  Returns the number
 * of non-empty levels (or a negative status). ---- */

int32_t orc_degree_levels(const orc_ctx *c, int32_t *level_of) {
    int64_t N = c->num_r;
    int32_t *d = (int32_t *)malloc(sizeof(int32_t) * (N + 1));
    char *alive = (char *)malloc((size_t)N + 1);
    char *inL = (char *)calloc((size_t)N + 1, 1);
    int64_t *Ls = (int64_t *)malloc(sizeof(int64_t) * (N + 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (c->maxdeg + 1));
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * ((int64_t)c->maxdeg * c->q + 1));
    int32_t levels = 0;
    if (!d || !alive || !inL || !Ls || !tmp || !buf) { levels = ORC_E_NOMEM; goto out; }
    if (orc_s_degree(c, d)) { levels = ORC_E_INVAL; goto out; }
    memset(alive, 1, (size_t)N + 1);
    int64_t remaining = N;
    while (remaining > 0) {
        int32_t mn = INT32_MAX;
        for (int64_t R = 0; R < N; ++R) if (alive[R] && d[R] < mn) mn = d[R];
        int64_t nl = 0;
        for (int64_t R = 0; R < N; ++R)
            if (alive[R] && d[R] == mn) { Ls[nl++] = R; inL[R] = 1; if (level_of) level_of[R] = levels; }
        for (int64_t i = 0; i < nl; ++i) {
            int64_t R = Ls[i];
            int64_t ns = s_cliques_of(c, R, buf, tmp);
            for (int64_t j = 0; j < ns; ++j) {
                const int32_t *S = buf + j * c->q;
                int ok = 1, owner = 1;
                for (int k = 0; k < c->q; ++k) {
                    if (!alive[S[k]]) ok = 0;             /* s-clique already gone */
                    if (inL[S[k]] && S[k] < R) owner = 0; /* handled by a smaller member */
                }
                if (!ok || !owner) continue;
                for (int k = 0; k < c->q; ++k)
                    if (!inL[S[k]]) d[S[k]]--;
            }
        }
        for (int64_t i = 0; i < nl; ++i) { alive[Ls[i]] = 0; inL[Ls[i]] = 0; }
        remaining -= nl;
        levels++;
    }
out:
    free(d); free(alive); free(inL); free(Ls); free(tmp); free(buf);
    return levels;
}

/* Kendall's tau-b of two integer sequences (Section 5.2, Fig. 7: similarity
 * of the order of the r-cliques by tau_t with the order by kappa).  Every
 * unordered pair {i, j} is visited: S accumulates sign(x_i - x_j) *
 * sign(y_i - y_j), tx and ty count the pairs tied in x and in y, and
 * tau_b = S / sqrt((n0 - tx) (n0 - ty)) with n0 = n (n - 1) / 2.  Writes the
 * three counts; returns tau_b, or NaN when either sequence is constant.
 * O(n^2): for small n only. */
double orc_kendall_tau_b(const int32_t *x, const int32_t *y, int64_t n, int64_t *s_out, int64_t *tx_out,
                         int64_t *ty_out) {
    int64_t S = 0, tx = 0, ty = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            const int sx = (x[i] > x[j]) - (x[i] < x[j]);
            const int sy = (y[i] > y[j]) - (y[i] < y[j]);
            S += sx * sy;
            tx += (sx == 0);
            ty += (sy == 0);
        }
    }
    if (s_out) *s_out = S;
    if (tx_out) *tx_out = tx;
    if (ty_out) *ty_out = ty;
    const double n0 = (double)n * (double)(n - 1) / 2.0;
    const double den = (n0 - (double)tx) * (n0 - (double)ty);
    if (!(den > 0.0)) return 0.0 / 0.0;
    return (double)S / sqrt(den);
}
