/*
 * folty_oracle.c -- plain, slow CPU oracle for thresholded triadic queries
 *                   "exists u, exists v, forall_rho w" on temporal graphs
 *                   (FOLTY, arXiv 2507.17215).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file. The CUDA library never calls it and shares no
 * code, header or table with it.
 *
 * What it computes (all integer arithmetic, int64 where products appear):
 *
 *   1. Section 2 (Preliminaries): the static graph G_S drops directions, parallel
 *      edges and self-loops; N(u) is u's neighbourhood in G_S; E_{x,y} is the list
 *      of temporal edges from x to y sorted by timestamp, duplicates kept.
 *   2. Section 2 ("How to solve FOL queries"): a temporal edge e = (x, y, t) forms a
 *      delta-temporal triangle with w when there are temporal edges (x, w, t2) and
 *      (y, w, t3) with t <= t2 <= t3 <= t + delta. Direction variants: "out" is that
 *      motif; "in" takes (w, x, t2) and (w, y, t3); "either" accepts both
 *      directions for each of the two witness edges (the paper's remark that other
 *      temporal triangles are handled the same way, Sections 1.2 and 6).
 *   3. c_e = number of w in N(x) cap N(y) that form such a triangle with e; one
 *      vertex counts once however many (t2, t3) match (Section 2, in-count/out-count).
 *      Default evaluation is the greedy test proved exact in Theorem 3.1: take the
 *      first a in A with t(a) >= t, then the first b in B with t(b) >= t(a), and
 *      accept when t(b) <= t + delta. The "brute" mode tries every (a, b) in A x B.
 *      Both scan the lists linearly.
 *   4. Threshold (Algorithm 5, Algorithm 6 last loop, Definition 1.1): the universe
 *      size U(e) is |N(x)| (head), |N(y)| (tail) or |N(x) cap N(y)| (common, the
 *      Insights variant). forall_rho with rho = num/den holds when
 *      c_e * den >= num * U(e) and c_e >= 1; exists holds when c_e >= 1.
 *   5. Solutions (Definition 1.2 and the certificate discussion of Section 1.2): an
 *      ordered pair (x, y) is a solution when at least one temporal edge x -> y is a
 *      certificate; it is reported with max c_e over E_{x,y} and the number of
 *      certificates, sorted by (x, y). The certificates themselves are listed by
 *      input index.
 *   6. Triples (Definition 1.2, all three quantifiers existential): (x, y, w) for every
 *      directed pair with a temporal edge x -> y that forms a triangle with witness w,
 *      sorted by (x, y, w).
 *   7. Vertex queries (Section 4, exists-forall-forall and exists-forall-exists): with the
 *      pairs of step 5 as the set L, vertex u is a solution when the number of v with
 *      (u, v) in L is >= 1 and, for an outer rho1 = num1/den1, count * den1 >=
 *      num1 * |N(u)|. The inner query is the pair query itself (forall_rho2 for
 *      exists-forall-forall, the existential quantifier for exists-forall-exists).
 *
 * Self-loops are not edges of G_S; they get c_e = 0 and are never certificates.
 * Parallelism: each temporal edge's c_e is independent, so an OpenMP loop over
 * edges computes them; nothing else is parallel.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n;
    int64_t m;
    const int32_t *src, *dst;          /* caller's arrays, input order */
    const int64_t *t;
    /* temporal edges without self-loops, sorted by (src, dst, t, input index) */
    int64_t m_kept;
    int64_t *order;                    /* input index of each sorted edge */
    int32_t *s_src, *s_dst;
    int64_t *s_t;
    /* N(u) as sorted unique neighbour lists (CSR) */
    int64_t *nbr_ptr;                  /* n + 1 */
    int32_t *nbr;
} oracle_graph;

/* ------------------------------------------------------------------ sorting helpers */

static const oracle_graph *g_sort_ctx;  /* qsort has no context argument */

static int cmp_edge(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    const oracle_graph *g = g_sort_ctx;
    if (g->src[a] != g->src[b]) return g->src[a] < g->src[b] ? -1 : 1;
    if (g->dst[a] != g->dst[b]) return g->dst[a] < g->dst[b] ? -1 : 1;
    if (g->t[a] != g->t[b]) return g->t[a] < g->t[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

static int cmp_pair(const void *pa, const void *pb) {
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------ graph building */

void oracle_graph_free(void *p) {
    oracle_graph *g = (oracle_graph *)p;
    if (!g) return;
    free(g->order); free(g->s_src); free(g->s_dst); free(g->s_t);
    free(g->nbr_ptr); free(g->nbr);
    free(g);
}

/* Builds E_{x,y} (sorted edge array) and N(u). Returns NULL on bad input. */
void *oracle_graph_new(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                       const int64_t *t) {
    if (n < 0 || m < 0) return NULL;
    for (int64_t i = 0; i < m; i++)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || t[i] < 0) return NULL;
    oracle_graph *g = (oracle_graph *)calloc(1, sizeof(oracle_graph));
    g->n = n; g->m = m; g->src = src; g->dst = dst; g->t = t;

    int64_t kept = 0;
    for (int64_t i = 0; i < m; i++) kept += (src[i] != dst[i]);
    g->m_kept = kept;
    g->order = (int64_t *)malloc(sizeof(int64_t) * (kept ? kept : 1));
    kept = 0;
    for (int64_t i = 0; i < m; i++)
        if (src[i] != dst[i]) g->order[kept++] = i;
    g_sort_ctx = g;
    qsort(g->order, (size_t)kept, sizeof(int64_t), cmp_edge);
    g->s_src = (int32_t *)malloc(sizeof(int32_t) * (kept ? kept : 1));
    g->s_dst = (int32_t *)malloc(sizeof(int32_t) * (kept ? kept : 1));
    g->s_t = (int64_t *)malloc(sizeof(int64_t) * (kept ? kept : 1));
    for (int64_t k = 0; k < kept; k++) {
        g->s_src[k] = src[g->order[k]];
        g->s_dst[k] = dst[g->order[k]];
        g->s_t[k] = t[g->order[k]];
    }

    /* N(u): both orientations of every non-loop temporal edge, sorted, made unique */
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (2 * kept + 1));
    int64_t np_ = 0;
    for (int64_t k = 0; k < kept; k++) {
        pairs[2 * np_] = g->s_src[k]; pairs[2 * np_ + 1] = g->s_dst[k]; np_++;
        pairs[2 * np_] = g->s_dst[k]; pairs[2 * np_ + 1] = g->s_src[k]; np_++;
    }
    qsort(pairs, (size_t)np_, 2 * sizeof(int32_t), cmp_pair);
    g->nbr_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (np_ ? np_ : 1));
    int64_t nn = 0;
    for (int64_t k = 0; k < np_; k++) {
        if (k > 0 && pairs[2 * k] == pairs[2 * k - 2] && pairs[2 * k + 1] == pairs[2 * k - 1])
            continue;
        g->nbr[nn++] = pairs[2 * k + 1];
        g->nbr_ptr[pairs[2 * k] + 1]++;
    }
    for (int32_t u = 0; u < n; u++) g->nbr_ptr[u + 1] += g->nbr_ptr[u];
    free(pairs);
    return g;
}

int64_t oracle_kept_edges(void *p) { return ((oracle_graph *)p)->m_kept; }

int32_t oracle_degree(void *p, int32_t u) {
    oracle_graph *g = (oracle_graph *)p;
    return (int32_t)(g->nbr_ptr[u + 1] - g->nbr_ptr[u]);
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ list access */

/* E_{x,y}: timestamps of the temporal edges x -> y, ascending. Found by bisecting the
 * (src, dst)-sorted edge array for the first and the last position of (x, y). */
static const int64_t *edge_list(const oracle_graph *g, int32_t x, int32_t y, int64_t *len) {
    int64_t lo = 0, hi = g->m_kept;                 /* first position >= (x, y) */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->s_src[mid] < x || (g->s_src[mid] == x && g->s_dst[mid] < y)) lo = mid + 1;
        else hi = mid;
    }
    int64_t begin = lo;
    hi = g->m_kept;                                  /* first position > (x, y) */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->s_src[mid] < x || (g->s_src[mid] == x && g->s_dst[mid] <= y)) lo = mid + 1;
        else hi = mid;
    }
    *len = lo - begin;
    return g->s_t + begin;
}

typedef struct { int64_t *v; int64_t len, cap; } buf64;

static void buf_reserve(buf64 *b, int64_t want) {
    if (b->cap < want) {
        b->cap = want > 2 * b->cap ? want : 2 * b->cap;
        b->v = (int64_t *)realloc(b->v, sizeof(int64_t) * (size_t)b->cap);
    }
}

/* The witness list A (or B) of a direction variant, as one ascending list:
 * out: E_{p,w}; in: E_{w,p}; either: E_{p,w} merged with E_{w,p}. */
static void witness_list(const oracle_graph *g, int dir, int32_t p, int32_t w, buf64 *out) {
    int64_t l1 = 0, l2 = 0;
    const int64_t *a = NULL, *b = NULL;
    if (dir == 0 || dir == 2) a = edge_list(g, p, w, &l1);
    if (dir == 1 || dir == 2) b = edge_list(g, w, p, &l2);
    buf_reserve(out, l1 + l2 + 1);
    int64_t i = 0, j = 0, k = 0;
    while (i < l1 && j < l2) out->v[k++] = (a[i] <= b[j]) ? a[i++] : b[j++];
    while (i < l1) out->v[k++] = a[i++];
    while (j < l2) out->v[k++] = b[j++];
    out->len = k;
}

/* Theorem 3.1: first a >= t, then first b >= a; hit iff that b <= t + delta. */
static int witness_greedy(const buf64 *A, const buf64 *B, int64_t t, int64_t delta) {
    int64_t i = 0;
    while (i < A->len && A->v[i] < t) i++;
    if (i == A->len) return 0;
    int64_t t2 = A->v[i];
    int64_t j = 0;
    while (j < B->len && B->v[j] < t2) j++;
    if (j == B->len) return 0;
    return B->v[j] <= t + delta;
}

/* The definition itself: some (a, b) in A x B with t <= a <= b <= t + delta. */
static int witness_brute(const buf64 *A, const buf64 *B, int64_t t, int64_t delta) {
    for (int64_t i = 0; i < A->len; i++)
        for (int64_t j = 0; j < B->len; j++)
            if (t <= A->v[i] && A->v[i] <= B->v[j] && B->v[j] <= t + delta) return 1;
    return 0;
}

/* c_e for input edge e, plus |N(x) cap N(y)| in *common (may be NULL). */
static int32_t edge_count(const oracle_graph *g, int64_t e, int64_t delta, int dir, int brute,
                          int32_t *common, buf64 *A, buf64 *B) {
    int32_t x = g->src[e], y = g->dst[e];
    int64_t t = g->t[e];
    if (x == y) { if (common) *common = 0; return 0; }
    int64_t i = g->nbr_ptr[x], ie = g->nbr_ptr[x + 1];
    int64_t j = g->nbr_ptr[y], je = g->nbr_ptr[y + 1];
    int32_t c = 0, cn = 0;
    while (i < ie && j < je) {                 /* merge N(x) and N(y) */
        if (g->nbr[i] < g->nbr[j]) { i++; continue; }
        if (g->nbr[i] > g->nbr[j]) { j++; continue; }
        int32_t w = g->nbr[i];
        i++; j++;
        cn++;
        witness_list(g, dir, x, w, A);
        witness_list(g, dir, y, w, B);
        c += brute ? witness_brute(A, B, t, delta) : witness_greedy(A, B, t, delta);
    }
    if (common) *common = cn;
    return c;
}

/* Definition 1.2 with three existential quantifiers: the triples (x, y, w) for which
 * some temporal edge x -> y forms a delta-temporal triangle with witness w (Section 2,
 * the same witness test as c_e), sorted by (x, y, w). Writes the first cap triples and
 * returns how many there are, or -1 on a bad argument. */
int64_t oracle_triples(void *p, int64_t delta, int dir, int64_t cap, int32_t *tx, int32_t *ty, int32_t *tw) {
    oracle_graph *g = (oracle_graph *)p;
    if (!g || delta < 0 || dir < 0 || dir > 2 || cap < 0) return -1;
    buf64 A = {0}, B = {0};
    int64_t k = 0;
    for (int64_t b = 0; b < g->m_kept;) {
        int32_t x = g->s_src[b], y = g->s_dst[b];
        int64_t e = b;
        while (e < g->m_kept && g->s_src[e] == x && g->s_dst[e] == y) e++;
        int64_t i = g->nbr_ptr[x], ie = g->nbr_ptr[x + 1];
        int64_t j = g->nbr_ptr[y], je = g->nbr_ptr[y + 1];
        while (i < ie && j < je) {  /* w in N(x) cap N(y), ascending */
            if (g->nbr[i] < g->nbr[j]) { i++; continue; }
            if (g->nbr[i] > g->nbr[j]) { j++; continue; }
            int32_t w = g->nbr[i];
            i++; j++;
            witness_list(g, dir, x, w, &A);
            witness_list(g, dir, y, w, &B);
            int hit = 0;
            for (int64_t q = b; q < e && !hit; q++) hit = witness_greedy(&A, &B, g->s_t[q], delta);
            if (hit) {
                if (k < cap) { tx[k] = x; ty[k] = y; tw[k] = w; }
                k++;
            }
        }
        b = e;
    }
    free(A.v);
    free(B.v);
    return k;
}

/* c_e for the input edges idx[0..n_idx) (all m edges when idx is NULL), into out[],
 * and |N(x) cap N(y)| into common_out[] when it is not NULL. Returns 0, or -1 on a
 * bad argument. */
int oracle_counts(void *p, int64_t delta, int dir, int brute, int64_t n_idx,
                  const int64_t *idx, int32_t *out, int32_t *common_out) {
    oracle_graph *g = (oracle_graph *)p;
    if (!g || delta < 0 || dir < 0 || dir > 2) return -1;
    int64_t cnt = idx ? n_idx : g->m;
    int bad = 0;
#pragma omp parallel
    {
        buf64 A = {0, 0, 0}, B = {0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t k = 0; k < cnt; k++) {
            int64_t e = idx ? idx[k] : k;
            if (e < 0 || e >= g->m) { bad = 1; continue; }
            int32_t cn = 0;
            out[k] = edge_count(g, e, delta, dir, brute, &cn, &A, &B);
            if (common_out) common_out[k] = cn;
        }
        free(A.v); free(B.v);
    }
    return bad ? -1 : 0;
}

/* Universe size U(e) of Definition 1.1's thresholded quantifier. */
static int64_t universe_size(const oracle_graph *g, int universe, int32_t x, int32_t y,
                             int32_t common) {
    if (universe == 0) return g->nbr_ptr[x + 1] - g->nbr_ptr[x];
    if (universe == 1) return g->nbr_ptr[y + 1] - g->nbr_ptr[y];
    return common;
}

/* Is edge e (count c) a certificate? Definition 1.1 with rho = num/den (exact). */
static int certifies(int quant, int64_t c, int64_t U, int64_t num, int64_t den) {
    if (c < 1) return 0;
    if (quant == 0) return 1;
    return c * den >= num * U;
}

/* Full query. counts[m] (input order) and common[m] are outputs; the pair arrays
 * need room for m entries. Returns the number of pairs, or -1 on a bad argument. */
int64_t oracle_query(void *p, int64_t delta, int64_t rho_num, int64_t rho_den, int quant,
                     int dir, int universe, int brute, int32_t *counts, int32_t *common,
                     int32_t *pu, int32_t *pv, int32_t *pcount, int32_t *pncert,
                     int64_t *n_cert_edges) {
    oracle_graph *g = (oracle_graph *)p;
    if (!g || rho_den <= 0 || rho_num < 0 || rho_num > rho_den || quant < 0 || quant > 1 ||
        universe < 0 || universe > 2)
        return -1;
    if (oracle_counts(p, delta, dir, brute, 0, NULL, counts, common) != 0) return -1;
    int64_t np_ = 0, ncert_total = 0;
    int64_t k = 0;
    while (k < g->m_kept) {                   /* runs of equal (src, dst) = E_{x,y} */
        int32_t x = g->s_src[k], y = g->s_dst[k];
        int32_t best = 0, ncert = 0;
        while (k < g->m_kept && g->s_src[k] == x && g->s_dst[k] == y) {
            int64_t e = g->order[k];
            int32_t c = counts[e];
            if (c > best) best = c;
            ncert += certifies(quant, c, universe_size(g, universe, x, y, common[e]),
                               rho_num, rho_den);
            k++;
        }
        if (ncert > 0) {
            pu[np_] = x; pv[np_] = y; pcount[np_] = best; pncert[np_] = ncert;
            np_++;
            ncert_total += ncert;
        }
    }
    if (n_cert_edges) *n_cert_edges = ncert_total;
    return np_;
}

/* Section 4: vertices u with count(u) = #{v : (u, v) a solution pair} meeting the outer
 * threshold. pu[0..np) are the solution pairs' heads (any order). Writes the vertex ids
 * ascending with their counts; returns how many. */
int64_t oracle_vertices(void *p, int64_t np, const int32_t *pu, int64_t num1, int64_t den1, int32_t *vout,
                        int32_t *cout) {
    oracle_graph *g = (oracle_graph *)p;
    if (!g || den1 <= 0 || num1 < 0 || num1 > den1) return -1;
    int32_t *cnt = (int32_t *)calloc((size_t)g->n + 1, sizeof(int32_t));
    for (int64_t i = 0; i < np; i++) cnt[pu[i]]++;  /* each pair (u, v) appears once */
    int64_t k = 0;
    for (int32_t u = 0; u < g->n; u++) {
        int64_t deg = g->nbr_ptr[u + 1] - g->nbr_ptr[u];
        if (cnt[u] >= 1 && (int64_t)cnt[u] * den1 >= num1 * deg) {
            vout[k] = u;
            cout[k] = cnt[u];
            k++;
        }
    }
    free(cnt);
    return k;
}

/* Input indices (ascending) of the certificates, from per-edge counts in input order. */
int64_t oracle_certificates(void *p, const int32_t *counts, const int32_t *common, int64_t rho_num,
                            int64_t rho_den, int quant, int universe, int64_t *out) {
    oracle_graph *g = (oracle_graph *)p;
    int64_t k = 0;
    for (int64_t e = 0; e < g->m; e++) {
        if (g->src[e] == g->dst[e]) continue;
        if (certifies(quant, counts[e], universe_size(g, universe, g->src[e], g->dst[e], common[e]), rho_num,
                      rho_den))
            out[k++] = e;
    }
    return k;
}
