/*
 * folty.h -- C ABI of the GB300 library for thresholded first-order-logic triadic
 * queries "exists u, exists v, forall_rho w" on temporal networks (FOLTY,
 * arXiv 2507.17215).
 *
 * Problem (paper Section 1.2, Definitions 1.1 and 1.2; Section 2):
 *   A temporal graph is a list of directed triples (u, v, t): u the head, v the
 *   destination, t the timestamp; parallel edges in both directions are allowed.
 *   G_S is the static graph without directions, parallel edges and self-loops, N(u)
 *   the neighbourhood of u in G_S, E_{x,y} the time-sorted list of edges x -> y.
 *   A temporal edge e = (x, y, t) forms a delta-temporal triangle with w when there are
 *   edges (x, w, t2) and (y, w, t3) with t <= t2 <= t3 <= t + delta ("out" motif;
 *   "in" uses (w, x, t2), (w, y, t3); "either" accepts both directions per edge).
 *   c_e counts the w in N(x) cap N(y) that do (each w at most once). e is a
 *   certificate of the query when c_e >= 1 and, for forall_rho, c_e * rho_den >=
 *   rho_num * U(e), U(e) being |N(x)|, |N(y)| or |N(x) cap N(y)| (Algorithm 5,
 *   Algorithm 6, Insights). An ordered pair (x, y) is a solution when at least one
 *   edge x -> y certifies it.
 *
 * Conventions shared by every call:
 *   - Every call returns a folty_status and never aborts; on failure a thread-local
 *     message is available from folty_last_error().
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream). Device work is
 *     ordered on it; calls that return host data synchronise it first.
 *   - Device memory is taken from the caller's folty_allocator when one is given
 *     (e.g. PyTorch's caching allocator), otherwise stream-ordered from a pool the
 *     library creates per device (cudaMemPoolCreate), which keeps up to a quarter of
 *     the device's memory cached between calls for reuse.
 *   - Limits: 0 <= n < 2^30, 0 <= m < 2^31, 0 <= t < 2^62, 0 <= delta < 2^62.
 */
#ifndef FOLTY_H
#define FOLTY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct folty_graph folty_graph; /* opaque; owns all of its device memory */

typedef enum {
    FOLTY_OK = 0,
    FOLTY_EINVAL = 1,   /* bad argument: ids outside [0,n), t or delta out of range, ... */
    FOLTY_ENOMEM = 2,   /* the allocator returned NULL (nothing leaks)                 */
    FOLTY_ECUDA = 3,    /* a CUDA call or kernel failed                                 */
    FOLTY_ESTATE = 4,   /* call made in the wrong state (query before preprocess)       */
    FOLTY_ETIMEOUT = 5  /* a bounded device-side wait ran out                           */
} folty_status;

/* Device allocator supplied by the caller. alloc returns a device pointer usable on
 * "stream" (or NULL when out of memory); free releases it in stream order. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
} folty_allocator;

enum { FOLTY_Q_EXISTS = 0, FOLTY_Q_FORALL_T = 1 };                    /* quantifier on w */
enum { FOLTY_DIR_OUT = 0, FOLTY_DIR_IN = 1, FOLTY_DIR_EITHER = 2 };   /* witness edges   */
enum { FOLTY_U_HEAD = 0, FOLTY_U_TAIL = 1, FOLTY_U_COMMON = 2 };      /* universe of w   */
enum { FOLTY_OUTER_NONE = 0, FOLTY_OUTER_FORALL_T = 1 };              /* quantifier on v */

/* One query (Definition 1.1). rho = rho_num / rho_den with 0 <= rho_num <= rho_den,
 * rho_den > 0; compared exactly in integers. want_edge_counts != 0 also returns c_e for
 * every input edge; want_certificates != 0 also lists every certificate;
 * want_triples != 0 also returns the solutions of the all-existential query
 * (Definition 1.2 with exists on u, v and w): every (x, y, w) such that some temporal
 * edge x -> y forms a delta-temporal triangle with witness w (direction variant dir;
 * rho, quant and universe do not apply to them).
 * outer = FOLTY_OUTER_FORALL_T adds the vertex queries of Section 4: with the solution
 * pairs as the set L, vertex u is a solution when #{v : (u, v) in L} >= 1 and
 * #{v : (u, v) in L} * outer_rho_den >= outer_rho_num * |N(u)| -- exists-forall-forall
 * when quant is FOLTY_Q_FORALL_T, exists-forall-exists when it is FOLTY_Q_EXISTS. */
typedef struct {
    int64_t delta;
    uint32_t rho_num, rho_den;
    uint8_t quant, dir, universe, want_edge_counts;
    uint8_t outer, want_certificates, want_triples, reserved;
    uint32_t outer_rho_num, outer_rho_den;
} folty_query_params;

/* Result of one query. The struct belongs to the caller; the arrays it points to are
 * host memory owned by the library and released by folty_free(result).
 *   u, v, count, ncert: n_pairs solutions sorted by (u, v) ascending; count = max c_e
 *                       over E_{u,v}; ncert = number of certificates on E_{u,v}.
 *   n_cert_edges:       total number of certificates.
 *   edge_count:         c_e for input edge i (self-loops get 0), length m, or NULL
 *                       when not requested.
 *   vertex, vertex_count: outer queries: the n_vertices solutions ascending, with the
 *                       number of solution pairs they head (NULL otherwise).
 *   certificate:        want_certificates: input indices of the n_cert_edges
 *                       certificates, ascending (NULL otherwise).
 *   triple_x, triple_y, triple_w: want_triples: the n_triples all-existential
 *                       solutions (x, y, w), sorted by (x, y, w) (NULL otherwise). */
typedef struct {
    uint64_t tag; /* written by the library; lets folty_free tell a result from a graph */
    int64_t n_pairs;
    int32_t *u, *v, *count, *ncert;
    int64_t n_cert_edges;
    int64_t m;
    int32_t *edge_count;
    int64_t n_vertices;
    int32_t *vertex, *vertex_count;
    int64_t *certificate;
    int64_t n_triples;
    int32_t *triple_x, *triple_y, *triple_w;
} folty_result;

/* Sizes and derived figures of a preprocessed graph. */
typedef struct {
    int32_t n;
    int64_t m;              /* input edges                                     */
    int64_t m_kept;         /* without self-loops                              */
    int64_t static_edges;   /* |E(G_S)|                                        */
    int32_t max_degree;     /* max |N(u)|                                      */
    int32_t degeneracy;     /* alpha = max core number (Definition 2.1)        */
    int32_t max_out_degree; /* max |N+(u)| in the oriented graph (<= alpha)    */
    int32_t peel_rounds;    /* rounds of the parallel peeling                  */
    int64_t triangles;      /* triangles of G_S                                */
    int64_t probes;         /* sum over triangles of the sizes of its 3 edges' */
                            /* temporal lists (= (edge, witness) pairs)        */
    int32_t sigma_max;      /* max multiplicity sigma(u,v) of a static edge    */
    int32_t time_sorted;    /* 1 if the input arrived sorted by t              */
    int64_t device_bytes;   /* device memory held by the graph                 */
} folty_graph_info;

/* Model traffic of one query's passes, in bytes (see the per-role formula in the design
 * notes): enumeration (done once at preprocess), window probes, threshold. */
typedef struct {
    int64_t enum_bytes;
    int64_t probe_bytes;
    int64_t threshold_bytes;
} folty_traffic_model;

/* Section 1.2 / Section 2 input. Copies the m edges (src[i] -> dst[i] at t[i]) into
 * device memory owned by the new graph and validates them. The three arrays may be
 * host or device pointers (detected per pointer); they stay owned by the caller and
 * are not referenced after the call returns. Memory of the current device and pinned
 * host memory, all three 16-byte aligned, are copied and checked by one kernel pass;
 * other input is copied first, then checked. alloc may be NULL. On success *out
 * receives a graph in the "loaded" state. Errors: FOLTY_EINVAL (n, m out of range, an
 * id outside [0, n), t outside [0, 2^62)), FOLTY_ENOMEM, FOLTY_ECUDA. */
folty_status folty_load_temporal_graph(int32_t n, int64_t m, const int32_t *src,
                                       const int32_t *dst, const int64_t *t,
                                       const folty_allocator *alloc, void *stream,
                                       folty_graph **out);

/* Section 2 preprocessing: drops self-loops, sorts edges into E_{x,y} lists, builds
 * G_S, its degeneracy order (Definition 2.1, by parallel peeling) and orientation,
 * and lists every triangle of G_S once. Moves the graph to the "preprocessed" state.
 * Errors: FOLTY_ESTATE (already preprocessed), FOLTY_ENOMEM, FOLTY_ECUDA,
 * FOLTY_ETIMEOUT (a device-side barrier of the peeling kernel gave up). */
folty_status folty_preprocess(folty_graph *g, void *stream);

/* One query (Algorithm 6 semantics): window probes for every (edge, witness) pair,
 * counts c_e, threshold, solution pairs. Fills *out (host arrays, library-owned).
 * Errors: FOLTY_ESTATE (not preprocessed), FOLTY_EINVAL (bad parameters),
 * FOLTY_ENOMEM, FOLTY_ECUDA. */
folty_status folty_query(folty_graph *g, const folty_query_params *q, folty_result *out,
                         void *stream);

/* nq queries answered together (outs[i] for qs[i]); results equal those of nq
 * folty_query calls. One probe pass per direction variant present serves every delta
 * of that variant: for a fixed (edge, witness) the searched t2, t3 do not depend on
 * delta (Theorem 3.1), so the gap t3 - t is computed once and binned by delta. */
folty_status folty_query_batch(folty_graph *g, const folty_query_params *qs, int32_t nq,
                               folty_result *outs, void *stream);

/* Frees a folty_graph* (all of its device memory) or the library-owned arrays of a
 * folty_result* (told apart by their tag). NULL and already-freed results are
 * ignored. Synchronises nothing; do not free a graph with work still in flight. */
void folty_free(void *obj);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char *folty_last_error(void);

/* Sizes of a preprocessed graph. Errors: FOLTY_EINVAL (NULL), FOLTY_ESTATE. */
folty_status folty_graph_get_info(const folty_graph *g, folty_graph_info *info);

/* Model traffic for one query with direction variant dir (computed on the device
 * from the triangle list; synchronises the stream). */
folty_status folty_graph_traffic_model(folty_graph *g, int32_t dir,
                                       folty_traffic_model *out, void *stream);

/* What one query's window-probe pass works on (delta, direction variant dir). Before
 * probing, a query keeps only the roles (temporal edges x -> y of one static edge, with
 * the third vertex of a triangle as witness) whose runs can meet the window at all; the
 * others cannot hit (Theorem 3.1's window test needs t <= t2 <= t3 <= t + delta). The
 * byte figures are the model the PROBE and SELECT stages of the profiler count. */
typedef struct {
    int64_t triangles, all_roles, all_probes;  /* 6 roles per triangle; every (edge, witness) */
    int64_t kept_triangles, kept_roles, kept_probes;
    int64_t select_bytes;  /* liveness pass: 30 B per triangle + 13 B per kept triangle */
    int64_t probe_bytes;   /* probe pass: 61 B per kept triangle + the per-role bytes    */
} folty_probe_stats;

/* Runs the selection of one query and counts what it keeps (synchronises the stream).
 * Errors: FOLTY_EINVAL (NULL, delta outside [0, 2^62), unknown dir), FOLTY_ESTATE. */
folty_status folty_graph_probe_stats(folty_graph *g, int64_t delta, int32_t dir, folty_probe_stats *out,
                                     void *stream);

/* The per-static-edge common-neighbour counts c_uv = |N(u) cap N(v)| of Section 3 (the
 * number of triangles of G_S on the edge): a[i] < b[i], c[i] for the static_edges
 * entries (host arrays of folty_graph_info.static_edges entries, caller-owned),
 * sorted by (a, b). Synchronises the stream. Errors: FOLTY_EINVAL, FOLTY_ESTATE. */
folty_status folty_graph_common_counts(folty_graph *g, int32_t *a, int32_t *b, int32_t *c,
                                       void *stream);

/* Core numbers of the static graph G_S (the k-core decomposition the degeneracy order of
 * Section 3 comes from): core[u] = the largest k such that u lies in a subgraph of
 * minimum degree k. core is a caller-owned host array of n entries. Synchronises the
 * stream. Errors: FOLTY_EINVAL (NULL), FOLTY_ESTATE (not preprocessed). */
folty_status folty_graph_core_numbers(folty_graph *g, int32_t *core, void *stream);

/* Number of kernels this library has launched in this process (all threads). */
uint64_t folty_kernel_launches(void);

/* Device time by stage, measured with CUDA events recorded on the launching stream
 * around every launch of the stage while profiling is on (collected after the calling
 * API function's final synchronisation), with the stage's model bytes (the bytes the
 * stage's algorithm must move, not what the hardware moved):
 *   PROBE     window probes of a query or batch pass over the kept roles (k_probe_live):
 *             per staged triangle 61 B, per kept role w sigma1 + w min(sigma2, sigma1
 *             ceil(log2(sigma2 + 1))) + the same for L3 + 8 sigma1 (w = bytes per stored
 *             timestamp), counted on the device;
 *   SORT      one radix pass: 8 B read for the histogram, 12 B read + 12 B written per key
 *             (8 B + 8 B for the temporal store's 32-bit sort ids with their values);
 *   PEEL      the degeneracy peeling: 12 B per adjacency entry + 16 B per vertex;
 *   THRESHOLD certificate test and per-pair reduction: 8 B per temporal edge (4 with 16-bit
 *             counters) + 20 B per directed pair;
 *   SELECT    the per-query selection of the triangles whose liveness byte admits the
 *             window (k_live_select): 1 B read per triangle; per kept triangle its record
 *             and its edges' run ends read and 13 B written, counted on the device;
 *   TRIANGLES triangle listing: 4 B per merged out-list entry + 8 B per static edge and
 *             16 B written per triangle (graphs past FOLTY_NOALLOC_MAX_EDGES edges: one
 *             pass into a layout bounded per oriented edge); graphs up to that size also
 *             count first (the same merge bytes again) and write 8 B more per triangle;
 *   ROLES     the run-ends table (12 B of run bounds + 4 timestamps read, one record
 *             written per static edge) and the liveness pass of one direction variant (16 B
 *             read and 1 B written per triangle, the run-ends table read once; after a
 *             one-pass listing, preprocessing's pass also moves each triangle into the
 *             dense layout: 16 B more written per triangle, and the per-edge counts and
 *             offsets read);
 *   BATCH     the batched threshold over the plain queries of a direction variant: the
 *             32-edge group bits, and (counted on the device) the bin row and 4 B of pair
 *             key of every edge in a group with a hit;
 *   STORE     the temporal store built beside the peeling: its span contains SORT spans.
 *             Time-ordered input with 32-bit offsets: 8 B per input edge for the sort ids
 *             and 16 B per edge and radix pass (the first pass reads 4 B more: the ids and
 *             the input times); other inputs: 24 B per input edge for the pair words and
 *             24 B per kept edge for the sorted arrays and run starts.
 * Totals are process-wide; profile one thread at a time. */
enum { FOLTY_STAGE_PROBE = 0, FOLTY_STAGE_SORT = 1, FOLTY_STAGE_PEEL = 2, FOLTY_STAGE_THRESHOLD = 3,
       FOLTY_STAGE_SELECT = 4, FOLTY_STAGE_TRIANGLES = 5, FOLTY_STAGE_ROLES = 6, FOLTY_STAGE_BATCH = 7,
       FOLTY_STAGE_STORE = 8, FOLTY_STAGE_COUNT = 9 };
typedef struct {
    int64_t launches; /* timed spans */
    double ms;        /* total device time */
    int64_t bytes;    /* total model bytes */
} folty_stage_profile;

/* Turns stage timing on (on != 0) or off and resets the totals. */
void folty_profile_enable(int32_t on);

/* Copies the totals of one stage. Errors: FOLTY_EINVAL (NULL, unknown stage). */
folty_status folty_profile_read(int32_t stage, folty_stage_profile *out);

/* ------------------------------------------------------------------ serving
 * A server keeps preprocessed graphs resident and answers queries as they arrive
 * (not in the paper: a serving layer over folty_query_batch). Each graph gets one
 * worker thread and one CUDA stream, so work on different graphs overlaps on the
 * device. A worker takes every query queued for its graph (up to max_batch) as one
 * batch -- queries that arrive while a batch runs form the next one (continuous
 * batching) -- shrinks the batch until its device footprint (per-delta bins and output
 * stages) fits the memory budget, waits until the budget has room, runs it and
 * completes the tickets. Results equal those of folty_query on the same graph. The
 * graphs stay owned by the caller and must outlive the server. */
typedef struct folty_server folty_server;

typedef struct {
    int64_t memory_budget_bytes; /* device bytes for in-flight batches; 0: half the free memory */
    int32_t max_batch;           /* queries per batch; 0: 256                                 */
} folty_server_config;

typedef struct {
    double queued_ms;   /* submit -> start of its batch       */
    double run_ms;      /* batch start -> results on the host */
    double latency_ms;  /* submit -> results on the host      */
    int64_t batch_id;
    int32_t batch_size;
    int32_t graph_index;
} folty_ticket_info;

typedef struct {
    int64_t batches, queries, queued;
    int64_t memory_budget_bytes, peak_memory_bytes;
    int64_t max_batches_in_flight;
} folty_server_stats;

/* Starts one worker per graph (all preprocessed). cfg may be NULL. Errors:
 * FOLTY_EINVAL, FOLTY_ESTATE (a graph not preprocessed), FOLTY_ECUDA. */
folty_status folty_server_create(folty_graph *const *graphs, int32_t n_graphs,
                                 const folty_server_config *cfg, folty_server **out);

/* Queues query q for graphs[graph_index]; *ticket identifies it. Thread-safe. Errors:
 * FOLTY_EINVAL (bad index or parameters), FOLTY_ESTATE (server shutting down). */
folty_status folty_server_submit(folty_server *sv, int32_t graph_index,
                                 const folty_query_params *q, int64_t *ticket);

/* Waits for a ticket (timeout_ms < 0: no limit) and moves its result into *out (free
 * it with folty_free); info (may be NULL) receives its timings. A ticket can be
 * collected once. Errors: FOLTY_EINVAL (unknown ticket), FOLTY_ETIMEOUT (not done in
 * time; the ticket stays collectable), or the status its batch failed with. */
folty_status folty_server_wait(folty_server *sv, int64_t ticket, int64_t timeout_ms,
                               folty_result *out, folty_ticket_info *info);

folty_status folty_server_get_stats(folty_server *sv, folty_server_stats *out);

/* Runs every queued query, stops the workers and frees uncollected results. */
void folty_server_destroy(folty_server *sv);

/* ------------------------------------------------------------------ autotuning
 * The library picks two kernel shapes per graph by timed trials on the device: the split
 * of the triangle passes between one thread and one whole warp per oriented edge (by
 * the total length of the edge's two out-lists), and the probe tile (the granularity in
 * which the flat probe space of the kept roles is partitioned over thread blocks) with
 * the probe kernel's blocks per SM. The split is timed during folty_preprocess, the
 * probe shape on the graph's first query; both are cached for the process under the
 * graph's statistics (sizes, triangles, probes), so later graphs of the same statistics
 * skip the trials. Every shape gives the same results. */
typedef struct {
    int32_t tri_heavy;           /* an oriented edge whose two out-lists hold more entries is
                                    intersected by a warp, otherwise by one thread          */
    int32_t probe_items;         /* probe tile = 256 * probe_items slots (4 or 8)          */
    int32_t probe_blocks_per_sm; /* 0: as many as fit                                      */
    int32_t tri_source;          /* 0 not yet chosen, 1 timed trials, 2 cache, 3 forced    */
    int32_t probe_source;
    float tri_ms[4];             /* trial times of the candidate splits (24, 48, 96, never) */
    float probe_ms[4];           /* of the candidate shapes (4, all), (8, all), (8, 2), (4, 4) */
} folty_tuning;

/* The shapes chosen for g. Errors: FOLTY_EINVAL (NULL), FOLTY_ESTATE (not preprocessed). */
folty_status folty_graph_tuning(const folty_graph *g, folty_tuning *out);

/* Uses the given shapes for every graph preprocessed or first queried afterwards instead
 * of tuning (all three 0: tune again). Errors: FOLTY_EINVAL (tri_heavy < 1, probe_items
 * not 4 or 8, probe_blocks_per_sm < 0). */
folty_status folty_tuning_force(int32_t tri_heavy, int32_t probe_items, int32_t probe_blocks_per_sm);

/* Forgets the cached shapes (the next graph of any statistics is tuned by trials). */
void folty_tuning_clear_cache(void);

/* Per-edge counts of one query without allocating anything (the paper has no
 * counterpart). For callers that cannot allocate device memory when they query: a
 * serving process that reserved its whole memory budget at start-up, latency-bound code
 * that must avoid the implicit device synchronisation of cudaMalloc/cudaFree, or a host
 * whose allocator must not be re-entered from inside a library call. Computes c_e of
 * every input edge for (delta, dir) -- the window-probe pass of folty_query -- into
 * edge_count: caller-owned device memory of m int32, input order, self-loops 0.
 *   - Allocates nothing: the counters the pass works in are one file-scope device array
 *     of FOLTY_NOALLOC_MAX_EDGES int32 (4 MiB) that every GPU loading the library holds
 *     until the process exits. A graph with more non-loop edges gives FOLTY_EINVAL.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call before any
 *     stream capture begins.
 *   - All calls share the array, which keeps the last call's contents; each call clears
 *     the part it uses before probing. Calls whose work overlaps on the GPU (other
 *     streams, other threads) race on it and give wrong counts: serialise them.
 *   - Call it with the graph's device current (the device that was current when the
 *     graph was loaded); edge_count must be memory of that device (cudaMalloc, a pool,
 *     PyTorch's allocator) holding at least m int32. The library checks the device and
 *     the kind of memory, not the length.
 *   - Stream-ordered on "stream"; does not synchronise it.
 * Errors: FOLTY_EINVAL (NULL, delta outside [0, 2^62), unknown dir, graph too large,
 * another device current, edge_count not memory of the graph's device), FOLTY_ESTATE
 * (not preprocessed), FOLTY_ECUDA. */
#define FOLTY_NOALLOC_MAX_EDGES (1 << 20)
folty_status folty_edge_counts_noalloc(folty_graph *g, int64_t delta, int32_t dir,
                                       int32_t *edge_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FOLTY_H */
