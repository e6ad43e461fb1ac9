// One query over a preprocessed graph (Algorithm 6 semantics, Algorithm 5 threshold):
//   A6  window probes: for every triangle {u, v, w} of G_S and every temporal edge
//       e = (x, y, t) on one of its three static edges, with witness z the third
//       vertex: t2 = first entry >= t of L2, t3 = first entry >= t2 of L3, hit iff both
//       exist and t3 <= t + delta (Theorem 3.1; Algorithms 1, 2 and 6). L2 = E_{x,z},
//       L3 = E_{y,z} for the paper's "out" motif, E_{z,x} and E_{z,y} for "in", and the
//       union of both directions for "either" (first entry of a union = min of the
//       first entries of its parts);
//   A7  c_e += hit. Every (e, witness) pair is probed once (each triangle is listed
//       once), so c_e counts distinct witnesses;
//   A8  certificate test per edge, max c_e and certificate count per directed pair,
//       compaction of the solution pairs and a sort by (u, v).
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>

#include "internal.cuh"
#include "scan.cuh"
#include "probe.cuh"

namespace folty {

// ================================================================== A6 + A7

// Block b handles probes [b * PB_TILE, (b + 1) * PB_TILE) of the flat probe space
// (triangle-major, then the triangle's three static edges, then their sorted temporal
// edges). The block stages the triangles overlapping its range in shared memory,
// threads take consecutive probes (coalesced T reads and counter updates).
template <typename TS, int DIR>
__global__ void __launch_bounds__(PB_THREADS) k_probe(const int4* __restrict__ tri,
                                                      const int64_t* __restrict__ tri_off,
                                                      const int64_t* __restrict__ tile_tri, int64_t P,
                                                      const int32_t* __restrict__ seg,
                                                      const TS* __restrict__ T, TS delta,
                                                      int32_t* __restrict__ cnt) {
    __shared__ TriStage st;
    const int64_t p0 = (int64_t)blockIdx.x * PB_TILE;
    const int32_t count = (int32_t)min((int64_t)PB_TILE, P - p0);
    stage_triangles(st, tri, tri_off, tile_tri, seg, DIR);
#pragma unroll 1
    for (int it = 0; it < PB_ITEMS; it++) {
        const int32_t local = it * PB_THREADS + (int32_t)threadIdx.x;
        if ((local & ~31) >= count) break;  // warp-uniform
        const bool active = local < count;
        Probe pr = locate_probe(st, local, active);
        if (!active) continue;
        const TS t = T[pr.pos];
        const TS t3 = probe_window<TS, DIR>(T, st.off[pr.j], pr.seg2, pr.seg3, t, delta);
        if (t3 != TsNone<TS>::value && (TS)(t3 - t) <= delta) atomicAdd(&cnt[pr.pos], 1);
    }
}

// ================================================================== A8

struct ThresholdArgs {
    const int32_t* cnt;
    const int32_t* sd;  // 2 * static id + direction of every sorted edge
    int64_t mk;
    const int32_t* ea;
    const int32_t* eb;
    const int32_t* deg;
    const int32_t* common;
    int quant, universe;
    int64_t num, den;
    int32_t* seg_max;    // [2S], zeroed
    int32_t* seg_ncert;  // [2S], zeroed
    unsigned long long* n_cert;
    const int32_t* perm;  // with cert_in: certificate flag of input edge perm[i]
    int32_t* cert_in;     // [m] or null
    const uint16_t* cnt16;  // 16-bit counts instead of cnt (batched queries), or null
    const int64_t* qp;      // may be null: a device block whose slots 2, 3 hold num, den
};

// Certificate test of Definition 1.1 with rho = num / den, exact in int64.
__device__ __forceinline__ bool certifies(int quant, int64_t c, int64_t U, int64_t num, int64_t den) {
    return c >= 1 && (quant == FOLTY_Q_EXISTS || c * den >= num * U);
}

constexpr int TH_THREADS = 256;
constexpr int TH_BATCH = 8;  // 32-edge chunks whose loads are in flight together, per warp

// Edge-major, so every warp gets the same amount of work: a warp takes TH_BATCH chunks
// of 32 consecutive sorted edges, loads their pair keys and counts together, and reduces
// each run of one directed pair within a chunk (runs are contiguous: the order is sorted
// by pair) with a ballot of run heads; a run with a non-zero max or certificates adds
// them to its pair with one atomic. The universe size is looked up only for edges with
// c >= 1 (no other edge can certify), and a chunk without such an edge is skipped. The
// universe, the quantifier and the certificate list are template parameters.
template <int UNI, int QUANT, bool CERT>
__global__ void __launch_bounds__(TH_THREADS) k_threshold(ThresholdArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t num = a.qp ? a.qp[2] : a.num, den = a.qp ? a.qp[3] : a.den;
    unsigned long long my_cert = 0;
    for (int64_t b0 = gw * 32 * TH_BATCH; b0 < a.mk; b0 += nw * 32 * TH_BATCH) {
        const int32_t* sd = a.sd + b0;
        const int32_t* cn = a.cnt + b0;
        const int32_t rem = (int32_t)min((int64_t)32 * TH_BATCH, a.mk - b0);
        int32_t kb[TH_BATCH], cb[TH_BATCH], ub[TH_BATCH];
#pragma unroll
        for (int k = 0; k < TH_BATCH; k++) {
            const int32_t i = k * 32 + lane;
            kb[k] = (i < rem) ? sd[i] : -1;
            cb[k] = (i < rem) ? (a.cnt16 ? (int32_t)a.cnt16[b0 + i] : cn[i]) : 0;
        }
        // universe sizes of the edges with c >= 1, the lookups of all chunks in flight at once
#pragma unroll
        for (int k = 0; k < TH_BATCH; k++) {
            ub[k] = 0;
            if (QUANT != FOLTY_Q_EXISTS && cb[k] >= 1) {
                const int32_t s = kb[k] >> 1;
                if (UNI == FOLTY_U_COMMON) ub[k] = a.common[s];
                else ub[k] = ((UNI == FOLTY_U_HEAD) != (bool)(kb[k] & 1)) ? a.ea[s] : a.eb[s];
            }
        }
        if (QUANT != FOLTY_Q_EXISTS && UNI != FOLTY_U_COMMON) {
#pragma unroll
            for (int k = 0; k < TH_BATCH; k++)
                if (cb[k] >= 1) ub[k] = a.deg[ub[k]];
        }
#pragma unroll
        for (int k = 0; k < TH_BATCH; k++) {
            if (k * 32 >= rem) break;  // warp-uniform
            const int32_t i = k * 32 + lane;
            const int32_t key = kb[k], c = cb[k];
            const bool sat = c >= 1 && (QUANT == FOLTY_Q_EXISTS || (int64_t)c * den >= num * (int64_t)ub[k]);
            if (CERT && i < rem) a.cert_in[a.perm[b0 + i]] = sat;
            if (!__any_sync(0xffffffffu, c > 0)) continue;  // nothing to reduce in this chunk
            // runs of one pair are contiguous lanes (past-the-end lanes hold key -1 and
            // come last, as a run of their own)
            const int prev = __shfl_up_sync(0xffffffffu, key, 1);
            const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || key != prev);
            const unsigned above = heads & ~((2u << lane) - 1u);
            const int start = 31 - __clz(heads & ((2u << lane) - 1u));
            const unsigned peers = (above ? (above & (0u - above)) - 1u : 0xffffffffu) & ~((1u << start) - 1u);
            const int run_max = __reduce_max_sync(peers, c);
            const int run_sat = __reduce_add_sync(peers, sat ? 1 : 0);
            if (key >= 0 && lane == start) {
                if (run_max > 0) atomicMax(&a.seg_max[key], run_max);
                if (run_sat > 0) atomicAdd(&a.seg_ncert[key], run_sat);
            }
            my_cert += sat ? 1ull : 0ull;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_cert += __shfl_xor_sync(0xffffffffu, my_cert, o);
    if (lane == 0 && my_cert) atomicAdd(a.n_cert, my_cert);
}

template <int UNI, int QUANT>
static void launch_threshold_q(const ThresholdArgs& a, bool cert, unsigned grid, cudaStream_t s) {
    if (cert) FOLTY_LAUNCH((k_threshold<UNI, QUANT, true>), grid, TH_THREADS, 0, s, a);
    else FOLTY_LAUNCH((k_threshold<UNI, QUANT, false>), grid, TH_THREADS, 0, s, a);
}

template <int UNI>
static void launch_threshold_u(const ThresholdArgs& a, bool cert, unsigned grid, cudaStream_t s) {
    if (a.quant == FOLTY_Q_EXISTS) launch_threshold_q<UNI, FOLTY_Q_EXISTS>(a, cert, grid, s);
    else launch_threshold_q<UNI, FOLTY_Q_FORALL_T>(a, cert, grid, s);
}

static void launch_threshold(const ThresholdArgs& a, unsigned grid, cudaStream_t s) {
    const bool cert = a.cert_in != nullptr;
    if (a.universe == FOLTY_U_HEAD) launch_threshold_u<FOLTY_U_HEAD>(a, cert, grid, s);
    else if (a.universe == FOLTY_U_TAIL) launch_threshold_u<FOLTY_U_TAIL>(a, cert, grid, s);
    else launch_threshold_u<FOLTY_U_COMMON>(a, cert, grid, s);
}

// Solution pairs come in two lists that are already sorted by (x, y): pairs x < y in
// static-edge order (sorted by (a, b)), and pairs x > y in by_b order (sorted by (b, a)).

// Flags, positions and compaction of the solution pairs in one pass: entry i < S is the
// directed pair ea -> eb of static edge i, entry S + j the pair eb -> ea of static edge
// by_b[j] (so both halves come out sorted by (x, y)); an entry is kept when the pair has a
// certificate. flag[i] (read by the vertex queries), the kept pairs at their prefix
// positions, and pos[S] = kept pairs x < y, pos[2S] = kept pairs in all. Tiles of
// PS_TILE entries in block start order, one decoupled look-back by warp 0.
constexpr int PS_ITEMS = 8;
constexpr int PS_TILE = SCAN_THREADS * PS_ITEMS;

__global__ void __launch_bounds__(SCAN_THREADS) k_pair_select(const int32_t* __restrict__ seg_ncert,
                                                              const int32_t* __restrict__ seg_max,
                                                              const int32_t* __restrict__ ea,
                                                              const int32_t* __restrict__ eb,
                                                              const int32_t* __restrict__ by_b, int64_t S,
                                                              unsigned long long* lb, unsigned int* counter, int* err,
                                                              int32_t* __restrict__ flag, int32_t* __restrict__ pos,
                                                              uint64_t* __restrict__ key, int32_t* __restrict__ cnt_c,
                                                              int32_t* __restrict__ nc_c) {
    __shared__ uint8_t sflag[PS_TILE];
    __shared__ int32_t wc[SCAN_THREADS / 32];
    __shared__ int32_t totc;
    __shared__ unsigned long long s_exc;
    __shared__ int64_t s_tile;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile, n2 = 2 * S;
    const int64_t base = tile * PS_TILE;
#pragma unroll
    for (int i = 0; i < PS_ITEMS; i++) {
        const int idx = i * SCAN_THREADS + threadIdx.x;
        const int64_t e = base + idx;
        int f = 0;
        if (e < n2) {
            f = (e < S) ? (seg_ncert[2 * e] > 0) : (seg_ncert[2 * (int64_t)by_b[e - S] + 1] > 0);
            flag[e] = f;
        }
        sflag[idx] = (uint8_t)f;
    }
    __syncthreads();
    int32_t c = 0;
#pragma unroll
    for (int i = 0; i < PS_ITEMS; i++) c += sflag[threadIdx.x * PS_ITEMS + i];
    const int32_t off = block_exclusive_sum<int32_t>(c, wc, &totc);
    if (threadIdx.x < 32) {
        volatile unsigned long long* v = lb;
        const unsigned long long tc = (unsigned long long)totc;
        if (tile == 0) {
            if (threadIdx.x == 0) {
                v[0] = SC_PREFIX | tc;
                s_exc = 0;
            }
        } else {
            if (threadIdx.x == 0) v[tile] = SC_AGG | tc;
            const unsigned long long ex = warp_lookback(v, tile, tc, err);
            if (threadIdx.x == 0) s_exc = ex;
        }
    }
    __syncthreads();
    int32_t p = (int32_t)s_exc + off;
#pragma unroll
    for (int i = 0; i < PS_ITEMS; i++) {
        const int item = threadIdx.x * PS_ITEMS + i;
        const int64_t e = base + item;
        if (e == S) pos[S] = p;
        if (!sflag[item]) continue;
        int64_t sdir;
        uint64_t x, y;
        if (e < S) {
            sdir = 2 * e;
            x = (uint64_t)ea[e];
            y = (uint64_t)eb[e];
        } else {
            const int32_t st = by_b[e - S];
            sdir = 2 * (int64_t)st + 1;
            x = (uint64_t)eb[st];
            y = (uint64_t)ea[st];
        }
        key[p] = (x << 32) | y;
        cnt_c[p] = seg_max[sdir];
        nc_c[p] = seg_ncert[sdir];
        p++;
    }
    if (base + PS_TILE >= n2 && threadIdx.x == 0) pos[n2] = (int32_t)s_exc + totc;
}


__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t n, uint64_t key) {
    int64_t lo = 0;
    while (n > 0) {
        int64_t half = n >> 1;
        if (a[lo + half] < key) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}

// Merge by rank: an entry's place in the output is its index in its own list plus the
// number of entries of the other list with a smaller key (keys of the lists differ).
__global__ void k_pair_merge(const uint64_t* __restrict__ key, const int32_t* __restrict__ cnt_c,
                             const int32_t* __restrict__ nc_c, int64_t nA, int64_t np, int32_t* __restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[p];
        const int64_t f = (p < nA) ? p + lower_bound_u64(key + nA, np - nA, k) : (p - nA) + lower_bound_u64(key, nA, k);
        out[f] = (int32_t)(k >> 32);
        out[np + f] = (int32_t)(k & 0xffffffffull);
        out[2 * np + f] = cnt_c[p];
        out[3 * np + f] = nc_c[p];
    }
}

// The same merge written straight into pinned host memory, for a pair count known only
// on the device (nA = pos[S], np = pos[2S]): skipped when np exceeds cap.
__global__ void k_pair_merge_stage(const uint64_t* __restrict__ key, const int32_t* __restrict__ cnt_c,
                                   const int32_t* __restrict__ nc_c, const int32_t* __restrict__ pos, int64_t S,
                                   int64_t cap, int32_t* __restrict__ out) {
    const int64_t nA = pos[S], np = pos[2 * S];
    if (np > cap) return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[p];
        const int64_t f = (p < nA) ? p + lower_bound_u64(key + nA, np - nA, k) : (p - nA) + lower_bound_u64(key, nA, k);
        out[f] = (int32_t)(k >> 32);
        out[np + f] = (int32_t)(k & 0xffffffffull);
        out[2 * np + f] = cnt_c[p];
        out[3 * np + f] = nc_c[p];
    }
}

template <typename C>
__global__ void k_edge_counts_input_order(const C* __restrict__ cnt, const int32_t* __restrict__ perm,
                                          int64_t mk, int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x)
        out[perm[i]] = cnt[i];
}

// Input indices of the flagged edges, ascending (pos = exclusive scan of flag).
__global__ void k_compact_indices(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t m,
                                  int64_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        if (flag[e]) out[pos[e]] = e;
}

// Section 4: number of solution pairs headed by each vertex (flag = pair flags of the
// two sorted lists, see k_pair_select).
__global__ void k_vertex_count(const int32_t* __restrict__ flag, int64_t S, const int32_t* __restrict__ ea,
                               const int32_t* __restrict__ eb, const int32_t* __restrict__ by_b,
                               int32_t* __restrict__ vcnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * S;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int32_t x = (i < S) ? ea[i] : eb[by_b[i - S]];
        atomicAdd(&vcnt[x], 1);
    }
}

// Outer threshold of Section 4: count >= 1 and count * den1 >= num1 * |N(u)|.
__global__ void k_vertex_flags(const int32_t* __restrict__ vcnt, const int32_t* __restrict__ deg, int64_t n,
                               int64_t num1, int64_t den1, int32_t* __restrict__ vflag) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = vcnt[u];
        vflag[u] = c >= 1 && c * den1 >= num1 * (int64_t)deg[u];
    }
}

__global__ void k_vertex_compact(const int32_t* __restrict__ vflag, const int32_t* __restrict__ vpos,
                                 const int32_t* __restrict__ vcnt, int64_t n, int64_t nv, int32_t* __restrict__ out) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (!vflag[u]) continue;
        out[vpos[u]] = (int32_t)u;
        out[nv + vpos[u]] = vcnt[u];
    }
}

// ================================================================== drivers

void validate_query(const folty_query_params& q) {
    if (q.delta < 0 || q.delta >= (1ll << 62)) fail(FOLTY_EINVAL, "delta outside [0, 2^62)");
    if (q.rho_den == 0 || q.rho_num > q.rho_den) fail(FOLTY_EINVAL, "rho must satisfy 0 <= rho_num <= rho_den, rho_den > 0");
    if (q.quant > FOLTY_Q_FORALL_T) fail(FOLTY_EINVAL, "unknown quantifier");
    if (q.dir > FOLTY_DIR_EITHER) fail(FOLTY_EINVAL, "unknown direction variant");
    if (q.universe > FOLTY_U_COMMON) fail(FOLTY_EINVAL, "unknown universe");
    if (q.outer > FOLTY_OUTER_FORALL_T) fail(FOLTY_EINVAL, "unknown outer quantifier");
    if (q.outer && (q.outer_rho_den == 0 || q.outer_rho_num > q.outer_rho_den))
        fail(FOLTY_EINVAL, "outer rho must satisfy 0 <= outer_rho_num <= outer_rho_den, outer_rho_den > 0");
}

template <typename TS, int DIR>
static void launch_probe_t(folty_graph* g, TS delta, int32_t* cnt, cudaStream_t s) {
    FOLTY_LAUNCH((k_probe<TS, DIR>), (unsigned)g->n_tiles, PB_THREADS, 0, s, g->tri, g->tri_off, g->tile_tri,
                 g->info.probes, g->seg, (const TS*)g->T, delta, cnt);
}

void launch_probe(folty_graph* g, int64_t delta, int dir, int32_t* cnt, cudaStream_t s) {
    if (g->info.probes <= 0) return;
    if (!g->tri_off || !g->tile_tri) fail(FOLTY_EINVAL, "the all-roles probe map was not built for this graph");
    if (g->n_tiles > 0x7fffffffll) fail(FOLTY_EINVAL, "probe space too large");
    if (g->ts32) {
        // every gap is below 2^32 - 1, so larger windows behave as 2^32 - 2
        const uint32_t d = delta >= 0xfffffffell ? 0xfffffffeu : (uint32_t)delta;
        if (dir == FOLTY_DIR_OUT) launch_probe_t<uint32_t, FOLTY_DIR_OUT>(g, d, cnt, s);
        else if (dir == FOLTY_DIR_IN) launch_probe_t<uint32_t, FOLTY_DIR_IN>(g, d, cnt, s);
        else launch_probe_t<uint32_t, FOLTY_DIR_EITHER>(g, d, cnt, s);
    } else {
        if (dir == FOLTY_DIR_OUT) launch_probe_t<int64_t, FOLTY_DIR_OUT>(g, delta, cnt, s);
        else if (dir == FOLTY_DIR_IN) launch_probe_t<int64_t, FOLTY_DIR_IN>(g, delta, cnt, s);
        else launch_probe_t<int64_t, FOLTY_DIR_EITHER>(g, delta, cnt, s);
    }
}

// Per-query device buffers of the threshold and output passes.
struct PairStage {
    int32_t* seg_max;    // [2S] max c_e per directed pair
    int32_t* seg_ncert;  // [2S] certificates per directed pair
    int32_t* flag;       // [2S + 1]
    int32_t* pos;        // [2S + 1]; pos[S] = pairs x < y, pos[2S] = all pairs
    uint64_t* key;       // [2S] compacted (x, y)
    int32_t* cnt_c;      // [2S]
    int32_t* nc_c;       // [2S]
    unsigned long long* n_cert;
    int32_t* cert_flag;  // [m + 1] certificate flags in input order (want_certificates)
    int32_t* cert_pos;   // [m + 1]
    int32_t* vcnt;       // [n + 1] solution pairs per head vertex (outer queries)
    int32_t* vflag;      // [n + 1]
    int32_t* vpos;       // [n + 1]
    unsigned long long* ctl;  // tile counter and look-back of k_pair_select
};

static PairStage pair_stage(Scratch& sc, const folty_graph* g, const folty_query_params& q) {
    const int64_t n2 = 2 * (int64_t)g->S;
    PairStage p;
    p.cert_flag = p.cert_pos = p.vcnt = p.vflag = p.vpos = nullptr;
    if (q.want_certificates) {
        p.cert_flag = sc.get<int32_t>(2 * (g->m + 1));
        p.cert_pos = p.cert_flag + g->m + 1;
    }
    if (q.outer) {
        p.vcnt = sc.get<int32_t>(3 * ((int64_t)g->n + 1));
        p.vflag = p.vcnt + g->n + 1;
        p.vpos = p.vflag + g->n + 1;
    }
    p.seg_max = sc.get<int32_t>(2 * n2 + 2);
    p.seg_ncert = p.seg_max + n2 + 1;
    p.flag = sc.get<int32_t>(2 * n2 + 2);
    p.pos = p.flag + n2 + 1;
    p.key = sc.get<uint64_t>(n2);
    p.cnt_c = sc.get<int32_t>(2 * n2 + 2);
    p.nc_c = p.cnt_c + n2 + 1;
    p.n_cert = sc.get<unsigned long long>(1);
    p.ctl = sc.get<unsigned long long>((n2 + PS_TILE - 1) / PS_TILE + 1);
    return p;
}

// Certificate test, per-pair reduction, flags, positions, compaction (no host sync).
static void pairs_device(folty_graph* g, const folty_query_params& q, const CountView& cnt, const PairStage& p,
                         Scratch* sc, cudaStream_t s, const int64_t* qp = nullptr) {
    const int T = 256;
    const int64_t mk = g->m_kept;
    const int64_t S = g->S, n2 = 2 * S;
    FOLTY_CUDA(cudaMemsetAsync(p.seg_max, 0, sizeof(int32_t) * (size_t)(2 * n2 + 2), s));
    FOLTY_CUDA(cudaMemsetAsync(p.n_cert, 0, sizeof(unsigned long long), s));
    if (p.cert_flag) FOLTY_CUDA(cudaMemsetAsync(p.cert_flag, 0, sizeof(int32_t) * (size_t)(g->m + 1), s));
    if (mk > 0) {
        if (p.cert_flag) ensure_perm(g, s);  // certificates are listed by input index
        ThresholdArgs a{cnt.c32, g->sd, mk, g->ea, g->eb, g->deg, g->common, (int)q.quant, (int)q.universe,
                        (int64_t)q.rho_num, (int64_t)q.rho_den, p.seg_max, p.seg_ncert, p.n_cert,
                        p.cert_flag ? g->perm : nullptr, p.cert_flag, cnt.c16, qp};
        StageSpan span(ST_THRESHOLD, s, 8 * mk);  // pair key + count per edge
        launch_threshold(a, grid_for((mk + TH_BATCH - 1) / TH_BATCH, TH_THREADS), s);
    }
    if (p.cert_flag) exclusive_scan(*sc, p.cert_flag, p.cert_pos, g->m);
    if (n2 > 0) {
        const int64_t tiles = (n2 + PS_TILE - 1) / PS_TILE;
        unsigned long long* ctl = p.ctl;  // tile counter, look-back
        FOLTY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(unsigned long long) * (size_t)(tiles + 1), s));
        FOLTY_LAUNCH(k_pair_select, (unsigned)tiles, SCAN_THREADS, 0, s, p.seg_ncert, p.seg_max, g->ea, g->eb, g->by_b,
                     S, ctl + 1, (unsigned int*)ctl, g->dev_err, p.flag, p.pos, p.key, p.cnt_c, p.nc_c);
    } else {
        FOLTY_CUDA(cudaMemsetAsync(p.pos, 0, sizeof(int32_t), s));
    }
    if (p.vcnt) {
        const int64_t n = g->n;
        FOLTY_CUDA(cudaMemsetAsync(p.vcnt, 0, sizeof(int32_t) * (size_t)(n + 1), s));
        if (n2 > 0) FOLTY_LAUNCH(k_vertex_count, grid_for(n2, T), T, 0, s, p.flag, S, g->ea, g->eb, g->by_b, p.vcnt);
        FOLTY_LAUNCH(k_vertex_flags, grid_for(n, T), T, 0, s, p.vcnt, g->deg, n, (int64_t)q.outer_rho_num,
                     (int64_t)q.outer_rho_den, p.vflag);
        exclusive_scan(*sc, p.vflag, p.vpos, n);
    }
}

void finish_queries(folty_graph* g, const folty_query_params* const* qs, const CountView* cnts, int nq,
                    folty_result* const* outs, cudaStream_t s) {
    const int T = 256;
    const int64_t S = g->S;
    const int64_t mk = g->m_kept;
    const int G = READBACK_MAX / 4;
    for (int g0 = 0; g0 < nq; g0 += G) {
        const int ng = std::min(G, nq - g0);
        Scratch sc(g->alloc, s, g->dev_err);
        std::vector<PairStage> st;
        // each query's pairs go straight to its share of the pinned pair stage when they
        // fit, and come back with the read-back below
        const int64_t cap = PAIR_STAGE / ng;
        g->stage_busy = 1;
        for (int i = 0; i < ng; i++) {
            st.push_back(pair_stage(sc, g, *qs[g0 + i]));
            pairs_device(g, *qs[g0 + i], cnts[g0 + i], st.back(), &sc, s);
            FOLTY_LAUNCH(k_pair_merge_stage, grid_for(cap, T, 1), T, 0, s, st.back().key, st.back().cnt_c,
                         st.back().nc_c, st.back().pos, S, cap, g->pair_stage + 4 * cap * i);
        }
        // one read-back for the group: pairs x < y, all pairs, certificates
        std::vector<const void*> ptrs;
        std::vector<int> sizes;
        for (int i = 0; i < ng; i++) {
            ptrs.push_back(st[i].pos + S);
            ptrs.push_back(st[i].pos + 2 * S);
            ptrs.push_back(st[i].n_cert);
            ptrs.push_back(st[i].vpos ? (const void*)(st[i].vpos + g->n) : (const void*)st[i].pos);
            sizes.insert(sizes.end(), {4, 4, 8, 4});
        }
        std::vector<int64_t> rb(4 * (size_t)ng);
        read_back(g, ptrs.data(), sizes.data(), 4 * ng, rb.data(), s);
        bool copies = false;  // device-to-host copies left to wait for
        for (int i = 0; i < ng; i++) {
            const folty_query_params& q = *qs[g0 + i];
            folty_result* out = outs[g0 + i];
            const int64_t nA = rb[4 * i], np = rb[4 * i + 1], nc = rb[4 * i + 2];
            const int64_t nv = q.outer ? rb[4 * i + 3] : 0;
            fill_result_host(out, np, g->m, q.want_edge_counts != 0, nv, q.outer != 0, nc, q.want_certificates != 0);
            out->n_cert_edges = nc;
            if (q.outer && nv > 0) {
                int32_t* vout = sc.get<int32_t>(2 * nv);
                FOLTY_LAUNCH(k_vertex_compact, grid_for(g->n, T), T, 0, s, st[i].vflag, st[i].vpos, st[i].vcnt,
                             (int64_t)g->n, nv, vout);
                FOLTY_CUDA(cudaMemcpyAsync(out->vertex, vout, sizeof(int32_t) * 2 * (size_t)nv, cudaMemcpyDeviceToHost, s));
                copies = true;
            }
            if (q.want_certificates && nc > 0) {
                int64_t* cout = sc.get<int64_t>(nc);
                FOLTY_LAUNCH(k_compact_indices, grid_for(g->m, T), T, 0, s, st[i].cert_flag, st[i].cert_pos, g->m, cout);
                FOLTY_CUDA(cudaMemcpyAsync(out->certificate, cout, sizeof(int64_t) * (size_t)nc, cudaMemcpyDeviceToHost, s));
                copies = true;
            }
            if (np > 0 && np <= cap) {
                const int32_t* staged = (const int32_t*)(g->host_stage + HOST_STAGE) + 4 * cap * i;
                std::memcpy(out->u, staged, sizeof(int32_t) * 4 * (size_t)np);
            } else if (np > 0) {
                int32_t* packed = sc.get<int32_t>(4 * np);
                FOLTY_LAUNCH(k_pair_merge, grid_for(np, T), T, 0, s, st[i].key, st[i].cnt_c, st[i].nc_c, nA, np,
                             packed);
                FOLTY_CUDA(cudaMemcpyAsync(out->u, packed, sizeof(int32_t) * 4 * (size_t)np, cudaMemcpyDeviceToHost, s));
                copies = true;
            }
            if (q.want_edge_counts && g->m > 0) {
                if (mk > 0) ensure_perm(g, s);
                int32_t* ec = sc.get<int32_t>(g->m);
                FOLTY_CUDA(cudaMemsetAsync(ec, 0, sizeof(int32_t) * (size_t)g->m, s));
                if (mk > 0 && cnts[g0 + i].c16)
                    FOLTY_LAUNCH(k_edge_counts_input_order<uint16_t>, grid_for(mk, T), T, 0, s, cnts[g0 + i].c16, g->perm,
                                 mk, ec);
                else if (mk > 0)
                    FOLTY_LAUNCH(k_edge_counts_input_order<int32_t>, grid_for(mk, T), T, 0, s, cnts[g0 + i].c32, g->perm,
                                 mk, ec);
                FOLTY_CUDA(cudaMemcpyAsync(out->edge_count, ec, sizeof(int32_t) * (size_t)g->m, cudaMemcpyDeviceToHost, s));
                copies = true;
            }
        }
        if (copies) FOLTY_CUDA(cudaStreamSynchronize(s));
    }
}

// ------------------------------------------------------------------ all-existential triples

// Flag i of the 6 * ntri roles as an int32 (input of the scan).
__global__ void k_triple_flags(const uint8_t* __restrict__ rflag, int64_t n6, int32_t* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n6; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = rflag[i];
}

// (x, y, w) of every role with a hit, in input vertex ids: role r = 2e + d of triangle t
// has certificate edge x -> y (static edge e, direction d) and witness z = 2 - e. The
// witness goes to key_w (the first sort key), x and y to xs and ys.
__global__ void k_triple_write(const int4* __restrict__ tri, const int32_t* __restrict__ ea,
                               const int32_t* __restrict__ eb, const uint8_t* __restrict__ rflag,
                               const int32_t* __restrict__ pos, int64_t ntri, uint64_t* __restrict__ key_w,
                               uint32_t* __restrict__ idx, int32_t* __restrict__ xs, int32_t* __restrict__ ys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 6 * ntri;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!rflag[i]) continue;
        const int64_t t = i / 6;
        const int r = (int)(i % 6);
        const int4 tr = tri[t];
        int32_t P[3];
        P[0] = (tr.w & 1) ? ea[tr.x] : eb[tr.x];  // u: bit 0 says u has the smaller id of {u, v}
        P[1] = ea[tr.x] + eb[tr.x] - P[0];
        P[2] = ea[tr.y] + eb[tr.y] - P[0];        // s_uw = {u, w}
        const int e = r >> 1, d = r & 1;
        const int p = (e == 2) ? 1 : 0, q = (e == 0) ? 1 : 2;
        const int x = ((d == 0) == id_less(tr.w, p, q)) ? p : q;
        const int k = pos[i];
        key_w[k] = (uint64_t)P[2 - e];
        idx[k] = (uint32_t)k;
        xs[k] = P[x];
        ys[k] = P[p + q - x];
    }
}

__global__ void k_triple_key_xy(const uint32_t* __restrict__ order, const int32_t* __restrict__ xs,
                                const int32_t* __restrict__ ys, int64_t n, int nb, uint64_t* __restrict__ key) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = order[i];
        key[i] = ((uint64_t)(uint32_t)xs[o] << nb) | (uint64_t)(uint32_t)ys[o];
    }
}

// out = [x... | y... | w...] in (x, y, w) order; order[i] indexes the written triples.
__global__ void k_triple_out(const uint32_t* __restrict__ order, const int32_t* __restrict__ xs,
                             const int32_t* __restrict__ ys, const uint64_t* __restrict__ ws, int64_t n,
                             int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = order[i];
        out[i] = xs[o];
        out[n + i] = ys[o];
        out[2 * n + i] = (int32_t)ws[o];
    }
}

// Triples of the roles flagged by the probe pass, sorted by (x, y, w) with two stable
// radix sorts (by w, then by (x, y)), into the result's host arrays. Synchronises.
static void triples_result(folty_graph* g, const uint8_t* rflag, folty_result* out, cudaStream_t s) {
    const int T = 256;
    const int64_t n6 = 6 * g->ntri;
    Scratch sc(g->alloc, s, g->dev_err);
    int32_t* flag = sc.get<int32_t>(n6 + 1);
    int32_t* pos = sc.get<int32_t>(n6 + 1);
    if (n6 > 0) FOLTY_LAUNCH(k_triple_flags, grid_for(n6, T), T, 0, s, rflag, n6, flag);
    exclusive_scan(sc, flag, pos, n6);
    const int64_t nt = read_i32(g, pos + n6, s);
    fill_result_triples(out, nt);
    if (nt == 0) return;
    uint64_t* kw = sc.get<uint64_t>(nt);
    uint64_t* kw_alt = sc.get<uint64_t>(nt);
    uint32_t* ix = sc.get<uint32_t>(nt);
    uint32_t* ix_alt = sc.get<uint32_t>(nt);
    int32_t* xs = sc.get<int32_t>(nt);
    int32_t* ys = sc.get<int32_t>(nt);
    FOLTY_LAUNCH(k_triple_write, grid_for(n6, T), T, 0, s, g->tri, g->ea, g->eb, rflag, pos, g->ntri, kw, ix, xs, ys);
    const int nb = bit_length((uint64_t)(g->n > 1 ? g->n - 1 : 1));
    // the witness value of written triple j stays in kw_src[j] (kept before sorting)
    uint64_t* kw_src = sc.get<uint64_t>(nt);
    FOLTY_CUDA(cudaMemcpyAsync(kw_src, kw, sizeof(uint64_t) * (size_t)nt, cudaMemcpyDeviceToDevice, s));
    const bool a1 = radix_sort_pairs(sc, kw, kw_alt, ix, ix_alt, nt, nb);
    read_back(g, nullptr, nullptr, 0, nullptr, s);  // the permutation indexes arrays next
    uint32_t* order1 = a1 ? ix_alt : ix;
    uint32_t* spare = a1 ? ix : ix_alt;
    uint64_t* kxy = a1 ? kw : kw_alt;  // free key buffers after the first sort
    uint64_t* kxy_alt = a1 ? kw_alt : kw;
    FOLTY_LAUNCH(k_triple_key_xy, grid_for(nt, T), T, 0, s, order1, xs, ys, nt, nb, kxy);
    const bool a2 = radix_sort_pairs(sc, kxy, kxy_alt, order1, spare, nt, 2 * nb);
    const uint32_t* order = a2 ? spare : order1;
    read_back(g, nullptr, nullptr, 0, nullptr, s);  // the sorts' look-backs completed
    int32_t* packed = sc.get<int32_t>(3 * nt);
    FOLTY_LAUNCH(k_triple_out, grid_for(nt, T), T, 0, s, order, xs, ys, kw_src, nt, packed);
    FOLTY_CUDA(cudaMemcpyAsync(out->triple_x, packed, sizeof(int32_t) * 3 * (size_t)nt, cudaMemcpyDeviceToHost, s));
    FOLTY_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ query plans

// A plain query (no per-edge counts, certificates, vertex or triple outputs) replays a
// CUDA graph captured once per graph and query shape (direction variant, quantifier,
// universe). Its window and rho reach the kernels through a device parameter block that
// the graph's first node copies from the graph's pinned stage, so no launch argument
// changes between queries: a query costs one graph launch and one synchronisation
// instead of about fifteen launches, memsets and allocations. The buffers the graphs
// work in are allocated once and owned by the graph.
constexpr int QP_SLOT = 448;  // pinned stage slots [QP_SLOT, QP_SLOT + 4): delta, delta32, num, den
static_assert(QP_SLOT > ERR_SLOT && QP_SLOT + 4 <= HOST_STAGE, "the parameter block has its own stage slots");

struct QueryPlans {
    CountView cnt;
    int32_t* cnt32 = nullptr;
    uint16_t* cnt16 = nullptr;
    ProbeBuffers pb{};
    PairStage ps{};
    int64_t* qp = nullptr;  // device parameter block [4]
    cudaStream_t cs = nullptr;  // capture stream
    cudaGraphExec_t exec[3][2][3] = {};
    int kernels[3][2][3] = {};  // kernel nodes of each captured sequence
};

void destroy_plans(folty_graph* g) {
    QueryPlans* qp = g->plans;
    if (!qp) return;
    for (auto& a : qp->exec)
        for (auto& b : a)
            for (auto& e : b)
                if (e) cudaGraphExecDestroy(e);
    if (qp->cs) cudaStreamDestroy(qp->cs);
    delete qp;
    g->plans = nullptr;
}

static QueryPlans* plans_of(folty_graph* g, cudaStream_t s) {
    if (g->plans) return g->plans;
    QueryPlans* p = new QueryPlans();
    g->plans = p;  // the buffers below are graph-owned; destroy_plans releases the rest
    const int64_t mk = g->m_kept, n2 = 2 * (int64_t)g->S;
    if (g->info.max_degree < 65535) p->cnt16 = graph_alloc<uint16_t>(g, mk + 2, s);
    else p->cnt32 = graph_alloc<int32_t>(g, mk, s);
    p->cnt = CountView{p->cnt32, p->cnt16};
    p->pb = probe_buffers(g, s);
    PairStage& ps = p->ps;
    std::memset(&ps, 0, sizeof(ps));
    ps.seg_max = graph_alloc<int32_t>(g, 2 * n2 + 2, s);
    ps.seg_ncert = ps.seg_max + n2 + 1;
    ps.flag = graph_alloc<int32_t>(g, 2 * n2 + 2, s);
    ps.pos = ps.flag + n2 + 1;
    ps.key = graph_alloc<uint64_t>(g, n2, s);
    ps.cnt_c = graph_alloc<int32_t>(g, 2 * n2 + 2, s);
    ps.nc_c = ps.cnt_c + n2 + 1;
    ps.n_cert = graph_alloc<unsigned long long>(g, 1, s);
    ps.ctl = graph_alloc<unsigned long long>(g, (n2 + PS_TILE - 1) / PS_TILE + 1, s);
    p->qp = graph_alloc<int64_t>(g, 4, s);
    FOLTY_CUDA(cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking));
    return p;
}

// The launch sequence of one plain query of shape (dir, quant, universe) on stream cs.
static void enqueue_plain_query(folty_graph* g, QueryPlans* p, int dir, int quant, int universe, cudaStream_t cs) {
    const int64_t mk = g->m_kept, S = g->S;
    FOLTY_CUDA(cudaMemcpyAsync(p->qp, g->host_stage + QP_SLOT, 4 * sizeof(int64_t), cudaMemcpyHostToDevice, cs));
    if (mk > 0 && p->cnt16) FOLTY_CUDA(cudaMemsetAsync(p->cnt16, 0, sizeof(uint16_t) * (size_t)(mk + 2), cs));
    if (mk > 0 && p->cnt32) FOLTY_CUDA(cudaMemsetAsync(p->cnt32, 0, sizeof(int32_t) * (size_t)mk, cs));
    enqueue_probe_pass(g, p->qp, dir, p->pb, p->cnt32, p->cnt16, cs);
    folty_query_params q{};
    q.dir = (uint8_t)dir;
    q.quant = (uint8_t)quant;
    q.universe = (uint8_t)universe;
    q.rho_den = 1;
    pairs_device(g, q, p->cnt, p->ps, nullptr, cs, p->qp);
    FOLTY_LAUNCH(k_pair_merge_stage, grid_for(PAIR_STAGE, 256, 1), 256, 0, cs, p->ps.key, p->ps.cnt_c, p->ps.nc_c,
                 p->ps.pos, S, PAIR_STAGE, g->pair_stage);
    const void* ptrs[3] = {p->ps.pos + S, p->ps.pos + 2 * S, p->ps.n_cert};
    const int sizes[3] = {4, 4, 8};
    enqueue_read_back(g, ptrs, sizes, 3, cs);
}

static cudaGraphExec_t plan_exec(folty_graph* g, QueryPlans* p, int dir, int quant, int universe) {
    cudaGraphExec_t& e = p->exec[dir][quant][universe];
    if (e) return e;
    FOLTY_CUDA(cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
        enqueue_plain_query(g, p, dir, quant, universe, p->cs);
    } catch (...) {
        cudaStreamEndCapture(p->cs, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        throw;
    }
    FOLTY_CUDA(cudaStreamEndCapture(p->cs, &graph));
    // the kernels a replay launches (the library's launch counter counts them)
    size_t nn = 0;
    int kernels = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
            for (size_t i = 0; i < nn; i++) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) kernels++;
            }
    }
    cudaGetLastError();
    p->kernels[dir][quant][universe] = kernels;
    const cudaError_t ie = cudaGraphInstantiate(&e, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        e = nullptr;
        fail(FOLTY_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
    return e;
}

static bool plans_enabled() {
    const char* env = std::getenv("FOLTY_QUERY_GRAPHS");
    return !(env && std::strcmp(env, "0") == 0);
}

static bool run_query_plan(folty_graph* g, const folty_query_params& q, folty_result* out, cudaStream_t s) {
    if (q.want_edge_counts || q.want_certificates || q.outer || q.want_triples) return false;
    if (profiling_on() || !plans_enabled()) return false;  // stage events are recorded by the launch path
    tune_probe(g, q.delta, q.dir, s);  // the captured sequence takes the tuned probe shape
    ensure_liveness(g, q.dir, s);      // the replay on s reads the variant's liveness row
    QueryPlans* p = plans_of(g, s);
    const cudaGraphExec_t e = plan_exec(g, p, q.dir, q.quant, q.universe);
    int64_t* hp = g->host_stage + QP_SLOT;
    hp[0] = q.delta;
    hp[1] = q.delta >= 0xfffffffell ? 0xfffffffell - 1 : q.delta;  // gaps of the 32-bit store stay below 2^32 - 1
    hp[2] = q.rho_num;
    hp[3] = q.rho_den;
    g->stage_busy = 1;
    FOLTY_CUDA(cudaGraphLaunch(e, s));
    g_launches.fetch_add((uint64_t)p->kernels[q.dir][q.quant][q.universe], std::memory_order_relaxed);
    FOLTY_CUDA(cudaStreamSynchronize(s));
    int64_t rb[3];
    collect_read_back(g, 3, rb, s);
    const int64_t nA = rb[0], np = rb[1], nc = rb[2];
    fill_result_host(out, np, g->m, false, 0, false, nc, false);
    out->n_cert_edges = nc;
    if (np > 0 && np <= PAIR_STAGE) {
        std::memcpy(out->u, (const int32_t*)(g->host_stage + HOST_STAGE), sizeof(int32_t) * 4 * (size_t)np);
    } else if (np > 0) {
        try {
            Scratch sc(g->alloc, s, g->dev_err);
            int32_t* packed = sc.get<int32_t>(4 * np);
            FOLTY_LAUNCH(k_pair_merge, grid_for(np, 256), 256, 0, s, p->ps.key, p->ps.cnt_c, p->ps.nc_c, nA, np, packed);
            FOLTY_CUDA(cudaMemcpyAsync(out->u, packed, sizeof(int32_t) * 4 * (size_t)np, cudaMemcpyDeviceToHost, s));
            FOLTY_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            release_result(out);
            throw;
        }
    }
    return true;
}

void run_query(folty_graph* g, const folty_query_params& q, folty_result* out, cudaStream_t s) {
    if (run_query_plan(g, q, out, s)) return;
    Scratch sc(g->alloc, s, g->dev_err);
    const int64_t mk = g->m_kept;
    // c_e counts distinct witnesses, so it is at most the largest degree of G_S: below
    // 2^16 - 1 the counters are 16 bits, two to a word (no carry reaches a neighbour)
    const bool c16 = g->info.max_degree < 65535;
    int32_t* cnt = c16 ? nullptr : sc.get<int32_t>(mk);
    uint16_t* cnt16 = c16 ? sc.get<uint16_t>(mk + 2) : nullptr;  // + 2: the last word is whole
    if (mk > 0 && c16) FOLTY_CUDA(cudaMemsetAsync(cnt16, 0, sizeof(uint16_t) * (size_t)(mk + 2), s));
    if (mk > 0 && !c16) FOLTY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)mk, s));
    uint8_t* rflag = nullptr;
    if (q.want_triples) {
        rflag = sc.get<uint8_t>(6 * g->ntri + 1);
        FOLTY_CUDA(cudaMemsetAsync(rflag, 0, (size_t)(6 * g->ntri + 1), s));
    }
    launch_probe_live(g, q.delta, q.dir, 0, cnt, nullptr, 0, 0, nullptr, s, rflag, cnt16);
    const folty_query_params* qp = &q;
    const CountView cv{cnt, cnt16};
    finish_queries(g, &qp, &cv, 1, &out, s);  // synchronises the stream
    if (q.want_triples) {
        try {
            triples_result(g, rflag, out, s);
        } catch (...) {
            release_result(out);
            throw;
        }
    }
}

// ================================================================== traffic model

// Per role (x, y; witness z): sigma1 = |E_{x,y}|, sigma2, sigma3 = the sizes of L2, L3
// for the direction variant, w = bytes per stored timestamp. Bytes = w sigma1 (read L1)
// + w min(sigma2, sigma1 * ceil(log2(sigma2 + 1))) + the same for L3 + 8 sigma1
// (counter read-modify-write).
__global__ void k_traffic(const int4* __restrict__ tri, int64_t ntri, const int32_t* __restrict__ seg, int dir,
                          int64_t w, unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ntri;
         i += (int64_t)gridDim.x * blockDim.x) {
        int4 tr = tri[i];
        int32_t off[9];
        const int32_t se[3] = {tr.x, tr.y, tr.z};
#pragma unroll
        for (int e = 0; e < 3; e++) {
            off[3 * e] = seg[2 * se[e]];
            off[3 * e + 1] = seg[2 * se[e] + 1];
            off[3 * e + 2] = seg[2 * se[e] + 2];
        }
#pragma unroll
        for (int e = 0; e < 3; e++) {
#pragma unroll
            for (int d = 0; d < 2; d++) {
                int64_t s1 = off[3 * e + d + 1] - off[3 * e + d];
                if (s1 == 0) continue;
                int c2, c3;
                role_segments(tr.w, e, d, dir, c2, c3);
                const int o2 = 3 * (c2 >> 1) + (c2 & 1), o3 = 3 * (c3 >> 1) + (c3 & 1);
                int64_t s2 = dir == FOLTY_DIR_EITHER ? off[o2 + 2] - off[o2] : off[o2 + 1] - off[o2];
                int64_t s3 = dir == FOLTY_DIR_EITHER ? off[o3 + 2] - off[o3] : off[o3 + 1] - off[o3];
                int64_t l2 = 64 - __clzll((unsigned long long)s2);
                int64_t l3 = 64 - __clzll((unsigned long long)s3);
                acc += w * s1 + w * min(s2, s1 * l2) + w * min(s3, s1 * l3) + 8 * s1;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

void traffic_model(folty_graph* g, int dir, folty_traffic_model* out, cudaStream_t s) {
    Scratch sc(g->alloc, s, g->dev_err);
    unsigned long long* acc = sc.get<unsigned long long>(1);
    FOLTY_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s));
    if (g->ntri > 0)
        FOLTY_LAUNCH(k_traffic, grid_for(g->ntri, 256), 256, 0, s, g->tri, g->ntri, g->seg, dir,
                     (int64_t)(g->ts32 ? 4 : 8), acc);
    out->probe_bytes = read_i64(g, (const int64_t*)acc, s);
    out->enum_bytes = g->enum_bytes;
    out->threshold_bytes = 4 * g->m_kept + 12 * 2 * (int64_t)g->S;
}

}  // namespace folty
