/*
 * folty_paper.c -- the paper's own counting procedure for the "out" motif, written as
 *                  an independent CPU cross-check (FOLTY, arXiv 2507.17215).
 *
 * TEST INFRASTRUCTURE, like folty_oracle.c: only the test suite loads it. It shares no
 * code with the oracle or with the CUDA library.
 *
 * Where the oracle tests every common neighbour of every temporal edge directly, this
 * file follows the paper's source-only route to the same per-edge counts c_e:
 *
 *   1. Section 2: G_S, the degeneracy order pi (Matula-Beck: repeatedly remove a vertex
 *      of smallest remaining degree, smallest id first) and the orientation
 *      u -> v iff pi(u) < pi(v). E_{x,y} = temporal edges x -> y sorted by time.
 *   2. Section 3.1 (out-neighbours): for every oriented (u, v) and w in N+(u) adjacent
 *      to v, Algorithm 1 (case 1) counts w for the edges of E_{u,v} with the first entry
 *      of L2 = E_{u,w} at or after t (a linear merge) and the first entry of
 *      L3 = E_{v,w} at or after that (a binary search); Algorithm 2 (case 2) counts w
 *      for the edges of E_{v,u} with the first entry of L2 = E_{v,w} at or after t and
 *      the last entry of L3 = E_{u,w} at or before t + delta. Theorem 3.1 and its
 *      case-2 twin make both tests exact. (The "exceeds" of the binary-search primitive
 *      is read as "at least", as the proof of Theorem 3.1 needs.)
 *   3. Section 3.2 (in-neighbours): a common neighbour a of x and y that precedes both in
 *      pi is the source of the triangle. For e in E_{x,y} it contributes when t(e) lies
 *      in one of the intervals [max(0, t(L23[e2]) - delta), t(e2)] over e2 in
 *      L2 = E_{x,a} with t(e2) <= t(L23[e2]) <= t(e2) + delta, L23[e2] being the first
 *      entry of L3 = E_{y,a} at or after t(e2) (the interval theorem of Section 3.2).
 *      Each source's interval list is inserted into the segment tree T_{x,y} of the
 *      static edge (Algorithm 4), and in-count[e] is the sum of the counters on the
 *      root-to-leaf path of t(e).
 *   4. Appendix A.1: the segment tree is built over the distinct timestamps of E_{x,y}
 *      (only those are ever queried; an interval is replaced by the range of timestamps
 *      it contains, skipped when it contains none). One source's list goes in with three
 *      passes: phase 1 colours grey each canonical node that has no grey node above it;
 *      phase 2 turns back to white each canonical node that has a grey node above it;
 *      phase 3 adds 1 to the counter of each canonical node that is still grey (and
 *      whitens it, recording the source in its vertex field), skipping a node below a
 *      grey node or below a counted node whose vertex field is the same source. So each
 *      source counts at most once on any root-to-leaf path, and exactly once where one of
 *      its intervals covers the leaf.
 *   5. c_e = out-count[e] + in-count[e].
 *
 * Readings of the garbled passages (the in-neighbour list assignments of Section 3.2 and
 * Algorithm 4; the appendix's phase-3 call and ">" thresholds): the lists above are the
 * ones the interval theorem needs, the third insertion pass is phase 3, and a counter
 * "> 0" blocks. The passes' "return" skips the canonical node at hand (the subtree
 * below the blocking node); the interval's other canonical nodes are still visited, so
 * that a blocker on one side of an interval does not hide its other side.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ segment tree */

typedef struct {
    int r;                 /* leaves: distinct timestamps ts[0..r) */
    const int64_t *ts;
    int32_t *counter;      /* 4r nodes */
    int32_t *vertex;
    uint8_t *grey;
} SegTree;

static int seg_init(SegTree *T, const int64_t *ts, int r) {
    T->r = r;
    T->ts = ts;
    size_t nodes = (size_t)(r > 0 ? 4 * r : 1);
    T->counter = (int32_t *)calloc(nodes, sizeof(int32_t));
    T->vertex = (int32_t *)malloc(nodes * sizeof(int32_t));
    T->grey = (uint8_t *)calloc(nodes, 1);
    if (!T->counter || !T->vertex || !T->grey) return -1;
    for (size_t i = 0; i < nodes; i++) T->vertex[i] = -1;
    return 0;
}

static void seg_free(SegTree *T) {
    free(T->counter);
    free(T->vertex);
    free(T->grey);
}

/* Phase 1: grey the canonical nodes of [ql, qr] that have no grey node above them. */
static void phase1(SegTree *T, int node, int l, int r, int ql, int qr) {
    if (qr < l || r < ql) return;
    if (T->grey[node]) return; /* a grey node on the way: skip */
    if (ql <= l && r <= qr) {
        T->grey[node] = 1;
        return;
    }
    int mid = (l + r) / 2;
    phase1(T, 2 * node, l, mid, ql, qr);
    phase1(T, 2 * node + 1, mid + 1, r, ql, qr);
}

/* Phase 2: whiten the grey canonical nodes that have a grey node above them. */
static void phase2(SegTree *T, int node, int l, int r, int ql, int qr, int grey_above) {
    if (qr < l || r < ql) return;
    if (ql <= l && r <= qr) {
        if (grey_above && T->grey[node]) T->grey[node] = 0;
        return;
    }
    int g = grey_above || T->grey[node];
    int mid = (l + r) / 2;
    phase2(T, 2 * node, l, mid, ql, qr, g);
    phase2(T, 2 * node + 1, mid + 1, r, ql, qr, g);
}

/* Phase 3: count the still-grey canonical nodes once for source z. */
static void phase3(SegTree *T, int node, int l, int r, int ql, int qr, int z) {
    if (qr < l || r < ql) return;
    if (ql <= l && r <= qr) {
        if (T->grey[node]) {
            T->grey[node] = 0;
            T->counter[node] += 1;
            T->vertex[node] = z;
        }
        return;
    }
    if (T->grey[node]) return;                                  /* grey above: skip */
    if (T->counter[node] > 0 && T->vertex[node] == z) return;   /* z counted above */
    int mid = (l + r) / 2;
    phase3(T, 2 * node, l, mid, ql, qr, z);
    phase3(T, 2 * node + 1, mid + 1, r, ql, qr, z);
}

/* Leaf range [i, j] of the timestamps inside [lo, hi]; returns 0 when there are none. */
static int snap(const SegTree *T, int64_t lo, int64_t hi, int *i, int *j) {
    int a = 0, b = T->r; /* first ts >= lo */
    while (a < b) {
        int m = (a + b) / 2;
        if (T->ts[m] < lo) a = m + 1;
        else b = m;
    }
    int c = 0, d = T->r; /* first ts > hi */
    while (c < d) {
        int m = (c + d) / 2;
        if (T->ts[m] <= hi) c = m + 1;
        else d = m;
    }
    *i = a;
    *j = c - 1;
    return a <= c - 1;
}

/* One source's interval list, with the three passes of the appendix. */
static void seg_insert_list(SegTree *T, const int64_t *lo, const int64_t *hi, int k, int z) {
    if (T->r == 0) return;
    for (int pass = 1; pass <= 3; pass++) {
        for (int q = 0; q < k; q++) {
            int i, j;
            if (!snap(T, lo[q], hi[q], &i, &j)) continue;
            if (pass == 1) phase1(T, 1, 0, T->r - 1, i, j);
            else if (pass == 2) phase2(T, 1, 0, T->r - 1, i, j, 0);
            else phase3(T, 1, 0, T->r - 1, i, j, z);
        }
    }
}

/* Sum of the counters on the root-to-leaf path of timestamp t (0 when t is no leaf). */
static int64_t seg_lookup(const SegTree *T, int64_t t) {
    int a = 0, b = T->r;
    while (a < b) {
        int m = (a + b) / 2;
        if (T->ts[m] < t) a = m + 1;
        else b = m;
    }
    if (a >= T->r || T->ts[a] != t) return 0;
    int64_t sum = 0;
    int node = 1, l = 0, r = T->r - 1;
    while (1) {
        sum += T->counter[node];
        if (l == r) break;
        int mid = (l + r) / 2;
        if (a <= mid) {
            node = 2 * node;
            r = mid;
        } else {
            node = 2 * node + 1;
            l = mid + 1;
        }
    }
    return sum;
}

/* Test hook: a tree over ts[0..r) (distinct, ascending), the lists of nlists sources
 * (source s owns intervals [off[s], off[s+1]) of lo/hi, inserted in order), then the
 * path sums at the query times. Returns 0, or -1 on allocation failure. */
int paper_segtree_counts(const int64_t *ts, int r, const int64_t *lo, const int64_t *hi, const int32_t *off,
                         int nlists, const int64_t *query, int nq, int64_t *out) {
    SegTree T;
    if (seg_init(&T, ts, r) != 0) {
        seg_free(&T);
        return -1;
    }
    for (int s = 0; s < nlists; s++) seg_insert_list(&T, lo + off[s], hi + off[s], off[s + 1] - off[s], s);
    for (int q = 0; q < nq; q++) out[q] = seg_lookup(&T, query[q]);
    seg_free(&T);
    return 0;
}

/* ------------------------------------------------------------------ graph */

typedef struct {
    int32_t n;
    int64_t mk;           /* kept (non-loop) temporal edges */
    int64_t *eidx;        /* input index of each sorted edge, sorted by (x, y, t, index) */
    int32_t *ex, *ey;
    int64_t *et;
    /* static graph */
    int32_t S;
    int32_t *sa, *sb;     /* static edge s = {sa[s] < sb[s]} */
    int64_t *rowptr;      /* CSR of G_S with neighbour ids and static edge ids, sorted by neighbour */
    int32_t *nbr, *nsid;
    int64_t *run_b, *run_e; /* run of E_{x,y}: static edge s, direction d: [run_b[2s+d], run_e[2s+d]) */
    int32_t *rank;        /* degeneracy order pi */
} PGraph;

static int cmp64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y);
}

static const int32_t *g_x, *g_y;
static const int64_t *g_t;

static int cmp_edge(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (g_x[a] != g_x[b]) return g_x[a] < g_x[b] ? -1 : 1;
    if (g_y[a] != g_y[b]) return g_y[a] < g_y[b] ? -1 : 1;
    if (g_t[a] != g_t[b]) return g_t[a] < g_t[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/* Static edge id of {x, y}, or -1. */
static int32_t static_id(const PGraph *G, int32_t x, int32_t y) {
    int64_t a = G->rowptr[x], b = G->rowptr[x + 1];
    while (a < b) {
        int64_t m = (a + b) / 2;
        if (G->nbr[m] < y) a = m + 1;
        else b = m;
    }
    return (a < G->rowptr[x + 1] && G->nbr[a] == y) ? G->nsid[a] : -1;
}

/* The sorted run E_{x,y} (x != y adjacent): [*b, *e) of the sorted edge arrays. */
static void run_of(const PGraph *G, int32_t x, int32_t y, int64_t *b, int64_t *e) {
    int32_t s = static_id(G, x, y);
    int d = (x == G->sa[s]) ? 0 : 1;
    *b = G->run_b[2 * s + d];
    *e = G->run_e[2 * s + d];
}

static int build(PGraph *G, int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t) {
    memset(G, 0, sizeof(*G));
    G->n = n;
    int64_t mk = 0;
    for (int64_t i = 0; i < m; i++) mk += (src[i] != dst[i]);
    G->mk = mk;
    G->eidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(mk > 0 ? mk : 1));
    if (!G->eidx) return -1;
    int64_t k = 0;
    for (int64_t i = 0; i < m; i++)
        if (src[i] != dst[i]) G->eidx[k++] = i;
    g_x = src;
    g_y = dst;
    g_t = t;
    qsort(G->eidx, (size_t)mk, sizeof(int64_t), cmp_edge);
    G->ex = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mk + 1));
    G->ey = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mk + 1));
    G->et = (int64_t *)malloc(sizeof(int64_t) * (size_t)(mk + 1));
    if (!G->ex || !G->ey || !G->et) return -1;
    for (int64_t i = 0; i < mk; i++) {
        G->ex[i] = src[G->eidx[i]];
        G->ey[i] = dst[G->eidx[i]];
        G->et[i] = t[G->eidx[i]];
    }
    /* static edges: distinct unordered pairs */
    int64_t *pk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(mk > 0 ? mk : 1));
    if (!pk) return -1;
    for (int64_t i = 0; i < mk; i++) {
        int64_t a = G->ex[i] < G->ey[i] ? G->ex[i] : G->ey[i], b = G->ex[i] ^ G->ey[i] ^ a;
        pk[i] = a * (int64_t)n + b;
    }
    qsort(pk, (size_t)mk, sizeof(int64_t), cmp64);
    int32_t S = 0;
    for (int64_t i = 0; i < mk; i++)
        if (i == 0 || pk[i] != pk[i - 1]) pk[S++] = pk[i];
    G->S = S;
    G->sa = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S + 1));
    G->sb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S + 1));
    G->rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    G->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * S + 1));
    G->nsid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * S + 1));
    G->run_b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * S + 1));
    G->run_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * S + 1));
    G->rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!G->sa || !G->sb || !G->rowptr || !G->nbr || !G->nsid || !G->run_b || !G->run_e || !G->rank) {
        free(pk);
        return -1;
    }
    for (int32_t s = 0; s < S; s++) {
        G->sa[s] = (int32_t)(pk[s] / n);
        G->sb[s] = (int32_t)(pk[s] % n);
        G->rowptr[G->sa[s] + 1]++;
        G->rowptr[G->sb[s] + 1]++;
    }
    free(pk);
    for (int32_t v = 0; v < n; v++) G->rowptr[v + 1] += G->rowptr[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!fill) return -1;
    memcpy(fill, G->rowptr, sizeof(int64_t) * (size_t)(n + 1));
    /* static edges are sorted by (a, b): rows come out sorted by neighbour when the b-side
     * entries (neighbours a < v) are placed before the a-side ones (neighbours b > v) */
    for (int32_t s = 0; s < S; s++) {
        int32_t v = G->sb[s];
        G->nbr[fill[v]] = G->sa[s];
        G->nsid[fill[v]++] = s;
    }
    for (int32_t s = 0; s < S; s++) {
        int32_t v = G->sa[s];
        G->nbr[fill[v]] = G->sb[s];
        G->nsid[fill[v]++] = s;
    }
    free(fill);
    for (int32_t s = 0; s < 2 * S; s++) G->run_b[s] = G->run_e[s] = 0;
    for (int64_t i = 0; i < mk; i++) {
        int32_t s = static_id(G, G->ex[i], G->ey[i]);
        int d = (G->ex[i] == G->sa[s]) ? 0 : 1;
        if (i == 0 || G->ex[i] != G->ex[i - 1] || G->ey[i] != G->ey[i - 1]) G->run_b[2 * s + d] = i;
        G->run_e[2 * s + d] = i + 1;
    }
    /* degeneracy order: smallest remaining degree first, smallest id among ties */
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    uint8_t *gone = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!deg || !gone) return -1;
    for (int32_t v = 0; v < n; v++) deg[v] = (int32_t)(G->rowptr[v + 1] - G->rowptr[v]);
    for (int32_t pos = 0; pos < n; pos++) {
        int32_t best = -1;
        for (int32_t v = 0; v < n; v++)
            if (!gone[v] && (best < 0 || deg[v] < deg[best])) best = v;
        gone[best] = 1;
        G->rank[best] = pos;
        for (int64_t j = G->rowptr[best]; j < G->rowptr[best + 1]; j++)
            if (!gone[G->nbr[j]]) deg[G->nbr[j]]--;
    }
    free(deg);
    free(gone);
    return 0;
}

static void release(PGraph *G) {
    free(G->eidx);
    free(G->ex);
    free(G->ey);
    free(G->et);
    free(G->sa);
    free(G->sb);
    free(G->rowptr);
    free(G->nbr);
    free(G->nsid);
    free(G->run_b);
    free(G->run_e);
    free(G->rank);
}

/* ------------------------------------------------------------------ Section 3 */

/* First index in [b, e) with et >= key (e when none): the linear and binary-search
 * primitives return the same index; the callers below use the one each algorithm names. */
static int64_t first_at_least_bs(const int64_t *et, int64_t b, int64_t e, int64_t key) {
    while (b < e) {
        int64_t m = (b + e) / 2;
        if (et[m] < key) b = m + 1;
        else e = m;
    }
    return b;
}

/* Algorithm 1 (case 1): e in L1 = E_{u,v}, L2 = E_{u,w}, L3 = E_{v,w}. */
static void out_case1(const PGraph *G, int32_t u, int32_t v, int32_t w, int64_t delta, int32_t *cnt) {
    int64_t b1, e1, b2, e2, b3, e3;
    run_of(G, u, v, &b1, &e1);
    run_of(G, u, w, &b2, &e2);
    run_of(G, v, w, &b3, &e3);
    if (b1 >= e1 || b2 >= e2 || b3 >= e3) return;
    int64_t p2 = b2; /* linear merge: first entry of L2 at or after t, for t ascending */
    for (int64_t i = b1; i < e1; i++) {
        while (p2 < e2 && G->et[p2] < G->et[i]) p2++;
        if (p2 >= e2) break;
        int64_t p3 = first_at_least_bs(G->et, b3, e3, G->et[p2]);
        if (p3 < e3 && G->et[p3] <= G->et[i] + delta) cnt[i]++;
    }
}

/* Algorithm 2 (case 2): e in L1 = E_{v,u}, L2 = E_{v,w}, L3 = E_{u,w}. */
static void out_case2(const PGraph *G, int32_t u, int32_t v, int32_t w, int64_t delta, int32_t *cnt) {
    int64_t b1, e1, b2, e2, b3, e3;
    run_of(G, v, u, &b1, &e1);
    run_of(G, v, w, &b2, &e2);
    run_of(G, u, w, &b3, &e3);
    if (b1 >= e1 || b2 >= e2 || b3 >= e3) return;
    int64_t p3 = b3; /* linear: last entry of L3 at or before t + delta, for t ascending */
    for (int64_t i = b1; i < e1; i++) {
        while (p3 < e3 && G->et[p3] <= G->et[i] + delta) p3++;
        int64_t last3 = p3 - 1; /* < b3 when none */
        int64_t p2 = first_at_least_bs(G->et, b2, e2, G->et[i]);
        if (p2 < e2 && last3 >= b3 && G->et[p2] <= G->et[last3]) cnt[i]++;
    }
}

/* The interval list I_{a,x,y}: L2 = E_{x,a}, L3 = E_{y,a}. Returns the count written. */
static int interval_list(const PGraph *G, int32_t a, int32_t x, int32_t y, int64_t delta, int64_t *lo,
                         int64_t *hi) {
    int64_t b2, e2, b3, e3;
    run_of(G, x, a, &b2, &e2);
    run_of(G, y, a, &b3, &e3);
    int k = 0;
    int64_t p3 = b3; /* linear merge: first entry of L3 at or after t(e2) */
    for (int64_t i = b2; i < e2; i++) {
        while (p3 < e3 && G->et[p3] < G->et[i]) p3++;
        if (p3 >= e3) break;
        if (G->et[p3] <= G->et[i] + delta) {
            lo[k] = G->et[p3] - delta > 0 ? G->et[p3] - delta : 0;
            hi[k] = G->et[i];
            k++;
        }
    }
    return k;
}

/* Per-edge counts c_e (input order; self-loops 0) of the out motif by the paper's
 * procedure. Returns 0, or -1 on bad arguments or allocation failure. */
int paper_counts(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t, int64_t delta,
                 int32_t *out) {
    if (n < 0 || m < 0 || delta < 0) return -1;
    for (int64_t i = 0; i < m; i++)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || t[i] < 0) return -1;
    PGraph G;
    if (build(&G, n, m, src, dst, t) != 0) {
        release(&G);
        return -1;
    }
    const int64_t mk = G.mk;
    int32_t *cnt = (int32_t *)calloc((size_t)(mk > 0 ? mk : 1), sizeof(int32_t));
    /* one segment tree per directed run, over its distinct timestamps */
    int64_t *tsbuf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(mk > 0 ? mk : 1));
    int64_t *tsoff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * G.S + 1));
    SegTree *trees = (SegTree *)calloc((size_t)(2 * G.S + 1), sizeof(SegTree));
    int64_t *lo = (int64_t *)malloc(sizeof(int64_t) * (size_t)(mk > 0 ? mk : 1));
    int64_t *hi = (int64_t *)malloc(sizeof(int64_t) * (size_t)(mk > 0 ? mk : 1));
    int ok = cnt && tsbuf && tsoff && trees && lo && hi;
    int64_t used = 0;
    for (int32_t q = 0; ok && q < 2 * G.S; q++) {
        tsoff[q] = used;
        int r = 0;
        for (int64_t i = G.run_b[q]; i < G.run_e[q]; i++)
            if (r == 0 || tsbuf[used + r - 1] != G.et[i]) tsbuf[used + r++] = G.et[i];
        if (seg_init(&trees[q], tsbuf + used, r) != 0) ok = 0;
        used += r;
    }
    /* Algorithm 3 (out-neighbours) and the interval insertions of Algorithm 4 */
    for (int32_t u = 0; ok && u < n; u++) {
        for (int64_t j = G.rowptr[u]; j < G.rowptr[u + 1]; j++) {
            const int32_t v = G.nbr[j];
            if (G.rank[v] < G.rank[u]) continue; /* (u, v) in G->_pi */
            for (int64_t k2 = G.rowptr[u]; k2 < G.rowptr[u + 1]; k2++) {
                const int32_t w = G.nbr[k2];
                if (w == v || G.rank[w] < G.rank[u] || static_id(&G, v, w) < 0) continue; /* w in N+(u) cap N(v) */
                out_case1(&G, u, v, w, delta, cnt);
                out_case2(&G, u, v, w, delta, cnt);
                /* u precedes v and w: it is the source for the edges between v and w;
                 * each such triangle once, from its smaller-ranked other vertex */
                if (G.rank[v] < G.rank[w]) {
                    int32_t s = static_id(&G, v, w);
                    int k;
                    k = interval_list(&G, u, v, w, delta, lo, hi);
                    seg_insert_list(&trees[2 * s + (v == G.sa[s] ? 0 : 1)], lo, hi, k, u);
                    k = interval_list(&G, u, w, v, delta, lo, hi);
                    seg_insert_list(&trees[2 * s + (w == G.sa[s] ? 0 : 1)], lo, hi, k, u);
                }
            }
        }
    }
    /* in-counts by lookup, then c_e in input order */
    if (ok) {
        for (int32_t q = 0; q < 2 * G.S; q++)
            for (int64_t i = G.run_b[q]; i < G.run_e[q]; i++) cnt[i] += (int32_t)seg_lookup(&trees[q], G.et[i]);
        for (int64_t i = 0; i < m; i++) out[i] = 0;
        for (int64_t i = 0; i < mk; i++) out[G.eidx[i]] = cnt[i];
    }
    if (trees)
        for (int32_t q = 0; q < 2 * G.S; q++) seg_free(&trees[q]);
    free(trees);
    free(tsbuf);
    free(tsoff);
    free(lo);
    free(hi);
    free(cnt);
    release(&G);
    return ok ? 0 : -1;
}
