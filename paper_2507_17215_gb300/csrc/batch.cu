// Batched queries sharing the window probes.
//
// For a fixed (temporal edge e, witness w, direction variant) the searched t2 and t3
// of Theorem 3.1 do not depend on delta, so hit(delta) <=> g(e, w) = t3 - t <= delta.
// One probe pass per direction variant therefore serves every delta of that variant
// (live.cu, binning mode, roles kept for the largest delta of the pass): the pass bins
// g by the sorted distinct deltas D (bin j = first D_j >= g), and a prefix over the bins
// gives c_e(D_j) = #{w : g(e, w) <= D_j} for all j at once. Quantifier, rho and universe
// only enter the threshold (Definition 1.1; Algorithm 5), so one pass over the bins
// answers every query of the variant: k_batch_threshold walks each edge's bins in order,
// keeps the prefix in a register, tests each query's certificate condition at its bin and
// reduces each directed pair's run of edges within the warp; the solution pairs of all
// queries are appended as (query, rank of the pair in (u, v) order) keys and sorted once.
// Queries that also want per-edge counts, certificates or vertex solutions take the
// single-query threshold path on the prefix-summed bins instead. When the bins of all
// deltas do not fit in the memory budget, the deltas are cut into chunks, one probe pass
// per chunk (bin 0 of a chunk also holds every smaller gap).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>

#include "internal.cuh"
#include "probe.cuh"

namespace folty {

constexpr int BATCH_MAX_BINS = 1024;
static_assert(BATCH_MAX_BINS * sizeof(int64_t) <= 4 * PAIR_STAGE * sizeof(int32_t), "bin bounds fit the pair stage");

// Bins are edge-major: the kstride bins of sorted edge e are contiguous (k used, the rest
// zero), so that a thread reads an edge's bins with 16-byte loads.
//
// out[e] = c_e(D_j) = sum_{i <= j} bins[e][i]: the counts of one window (a query that
// wants per-edge outputs goes through the single-query threshold path on them).
template <typename C>
__global__ void k_bins_column(const C* __restrict__ bins, int kstride, int j, int64_t mk, C* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mk;
         e += (int64_t)gridDim.x * blockDim.x) {
        const C* row = bins + e * kstride;
        uint32_t run = 0;
        for (int i = 0; i <= j; i++) run += row[i];
        out[e] = (C)run;
    }
}

// ------------------------------------------------------------------ pair ranks

__device__ __forceinline__ int64_t lower_bound_pair(const int32_t* __restrict__ ka, const int32_t* __restrict__ kb,
                                                    const int32_t* __restrict__ idx, int64_t n, int32_t x, int32_t y) {
    int64_t lo = 0;
    while (n > 0) {
        const int64_t half = n >> 1;
        const int32_t i = idx ? idx[lo + half] : (int32_t)(lo + half);
        if (ka[i] < x || (ka[i] == x && kb[i] < y)) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}

// prank[2s + d] = position of the directed pair (x, y) of static edge s, direction d, in
// the (x, y) order of all directed pairs: pairs x < y are the static edges in (a, b)
// order, pairs x > y the static edges in (b, a) order (by_b); a pair's position is its
// index in its own list plus the number of pairs of the other list before it.
__global__ void k_pair_ranks(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                             const int32_t* __restrict__ by_b, int64_t S, int32_t* __restrict__ prank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * S; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < S) {  // (a, b) of static edge i; pairs (b', a') with b' < a, or b' == a and a' < b, precede it
            prank[2 * i] = (int32_t)(i + lower_bound_pair(eb, ea, by_b, S, ea[i], eb[i]));
        } else {  // (b, a) of static edge by_b[j]
            const int64_t j = i - S;
            const int32_t s = by_b[j];
            prank[2 * (int64_t)s + 1] = (int32_t)(j + lower_bound_pair(ea, eb, nullptr, S, eb[s], ea[s]));
        }
    }
}

static const int32_t* pair_ranks(folty_graph* g, cudaStream_t s) {
    if (!g->prank) {
        g->prank = graph_alloc<int32_t>(g, 2 * (int64_t)g->S, s);
        if (g->S > 0)
            FOLTY_LAUNCH(k_pair_ranks, grid_for(2 * (int64_t)g->S, 256), 256, 0, s, g->ea, g->eb, g->by_b,
                         (int64_t)g->S, g->prank);
    }
    return g->prank;
}

// ------------------------------------------------------------------ fused threshold

constexpr int BT_THREADS = 256;
constexpr int BT_WARPS = BT_THREADS / 32;
constexpr int BT_MAXQ = 256;  // queries of one fused pass
constexpr int BT_CHUNKS = 4;  // 16-byte chunks of an edge's bins loaded together per lane
// bins of one fused pass (their prefix sums sit in shared memory, per warp and lane)
constexpr int BT_KMAX = 128;

// A class of a pass's queries that differ only in their window: the same quantifier,
// universe and rho. Its queries are qs[qb, qe), sorted by bin; jmax = the last one's bin.
struct BatchClass {
    int32_t quant, universe;
    int64_t num, den;
    int32_t qb, qe, jmax, pad;
};

// One query of a fused pass.
struct BatchQuery {
    int32_t j;     // bin of its delta
    int32_t slot;  // index among the pass's queries (high bits of its output keys)
};

struct BatchArgs {
    const void* bins;  // C[mk][kstride], k bins used per row
    int k, kstride;
    int64_t mk;
    const int32_t* sd;   // 2 * static edge + direction of every sorted edge
    const int32_t* seg;  // run bounds: run r = [seg[r], seg[r + 1])
    const int32_t* ea;
    const int32_t* eb;
    const int32_t* deg;
    const int32_t* common;
    const int32_t* prank;
    const BatchClass* cls;
    int ncls;
    const BatchQuery* qs;  // by class, then bin
    int nq;
    int rb;  // bits of a pair rank
    int64_t per_warp;
    int64_t cap;
    unsigned long long* n_out;
    uint64_t* out_key;  // (slot << rb) | pair rank
    int32_t* out_run;   // the pair's run id 2s + d
    int32_t* out_cnt;   // max c_e over the pair's edges
    int32_t* out_nc;    // certificates among them
    const uint32_t* touched;    // bit g: some edge of [32 g, 32 g + 32) has a nonzero bin
    unsigned long long* prof;   // may be null: model bytes of the rows read
};

// x rounded up to the next start of a run (runs of one directed pair are contiguous).
__device__ __forceinline__ int64_t run_aligned(const int32_t* __restrict__ sd, const int32_t* __restrict__ seg,
                                               int64_t x, int64_t mk) {
    if (x <= 0) return 0;
    if (x >= mk) return mk;
    const int32_t r = sd[x];
    return (sd[x - 1] != r) ? x : (int64_t)seg[r + 1];
}

// Universe sizes of the pair of run r: |N(x)|, |N(y)|, |N(x) cap N(y)|.
__device__ __forceinline__ void universes(const BatchArgs& a, int32_t r, int64_t& uh, int64_t& ut, int64_t& uc) {
    const int32_t s = r >> 1;
    const int32_t x = (r & 1) ? a.eb[s] : a.ea[s], y = (r & 1) ? a.ea[s] : a.eb[s];
    uh = a.deg[x];
    ut = a.deg[y];
    uc = a.common[s];
}

// The smallest count that certifies for class c (Definition 1.1: c >= 1, and for
// forall_rho c * den >= num * U, i.e. c >= ceil(num * U / den) in integers).
__device__ __forceinline__ int64_t needed(const BatchClass& c, int64_t uh, int64_t ut, int64_t uc) {
    if (c.quant == FOLTY_Q_EXISTS) return 1;
    const int64_t U = c.universe == FOLTY_U_HEAD ? uh : c.universe == FOLTY_U_TAIL ? ut : uc;
    const int64_t v = (c.num * U + c.den - 1) / c.den;
    return v > 1 ? v : 1;
}

// Whether a sorted edge of [b, e) (e - b <= 32, so at most two groups) has a nonzero bin.
__device__ __forceinline__ bool touched_any(const uint32_t* __restrict__ t, int64_t b, int64_t e) {
    const int64_t g0 = b >> 5, g1 = (e - 1) >> 5;
    bool any = (__ldg(t + (g0 >> 5)) >> (g0 & 31)) & 1u;
    if (g1 != g0) any = any || ((__ldg(t + (g1 >> 5)) >> (g1 & 31)) & 1u);
    return any;
}

// Appends the pairs of the lanes with emit set (one atomic per warp).
__device__ __forceinline__ void emit_pairs(const BatchArgs& a, bool emit, int slot, int32_t r, int32_t cnt, int32_t nc) {
    const unsigned em = __ballot_sync(0xffffffffu, emit);
    if (!em) return;
    const int lane = threadIdx.x & 31;
    const int first = __ffs(em) - 1;
    unsigned long long base = 0;
    if (lane == first) base = atomicAdd(a.n_out, (unsigned long long)__popc(em));
    base = __shfl_sync(0xffffffffu, base, first);
    if (emit) {
        const unsigned long long i = base + __popc(em & ((1u << lane) - 1u));
        if (i < (unsigned long long)a.cap) {
            a.out_key[i] = ((uint64_t)slot << a.rb) | (uint64_t)(uint32_t)a.prank[r];
            a.out_run[i] = r;
            a.out_cnt[i] = cnt;
            a.out_nc[i] = nc;
        }
    }
}

// Prefix sums c_e(D_j) of the bins of one lane's edge (its row of kstride bins) into
// pref[j * 32 + lane] (zeros for an idle lane), BT_CHUNKS 16-byte loads in flight
// together; returns c_e(D_{k-1}).
template <typename C>
__device__ __forceinline__ uint32_t bin_prefix(const C* __restrict__ bins, int kstride, int k, int64_t e, bool on,
                                               C* pref) {
    constexpr int PER = 16 / sizeof(C);  // bins per 16-byte chunk of a row
    const int lane = threadIdx.x & 31;
    const uint4* row = reinterpret_cast<const uint4*>(bins + e * (int64_t)kstride);
    const int nch = (k + PER - 1) / PER;
    uint32_t run = 0;
    for (int c0 = 0; c0 < nch; c0 += BT_CHUNKS) {
        uint4 w[BT_CHUNKS];
#pragma unroll
        for (int u = 0; u < BT_CHUNKS; u++) w[u] = (on && c0 + u < nch) ? __ldg(row + c0 + u) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < BT_CHUNKS; u++) {
            const uint32_t ws[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
            for (int i = 0; i < PER; i++) {
                const int j = (c0 + u) * PER + i;
                run += sizeof(C) == 2 ? (ws[i >> 1] >> (16 * (i & 1))) & 0xffffu : ws[i & 3];
                if (j < k) pref[j * 32 + lane] = (C)run;
            }
        }
    }
    return run;
}

// c_e(D_{k-1}), the sum of one lane's row (its padding is zero), from registers only:
// most windows have no witness at any bin and skip the prefix sums in shared memory.
template <typename C>
__device__ __forceinline__ uint32_t row_sum(const C* __restrict__ bins, int kstride, int64_t e, bool on) {
    constexpr int PER = 16 / sizeof(C);
    const uint4* row = reinterpret_cast<const uint4*>(bins + e * (int64_t)kstride);
    const int nch = kstride / PER;
    uint32_t sum = 0;
    for (int c0 = 0; c0 < nch; c0 += BT_CHUNKS) {
        uint4 w[BT_CHUNKS];
#pragma unroll
        for (int u = 0; u < BT_CHUNKS; u++) w[u] = (on && c0 + u < nch) ? __ldcs(row + c0 + u) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < BT_CHUNKS; u++) {
            if (sizeof(C) == 2)
                sum += (w[u].x & 0xffffu) + (w[u].x >> 16) + (w[u].y & 0xffffu) + (w[u].y >> 16) + (w[u].z & 0xffffu) +
                       (w[u].z >> 16) + (w[u].w & 0xffffu) + (w[u].w >> 16);
            else
                sum += w[u].x + w[u].y + w[u].z + w[u].w;
        }
    }
    return sum;
}

// First bin j with pref[j * 32 + lane] >= need (k if none; the prefix is non-decreasing).
template <typename C>
__device__ __forceinline__ int first_bin(const C* pref, int k, int64_t need) {
    const int lane = threadIdx.x & 31;
    int lo = 0, len = k;
    while (len > 0) {
        const int half = len >> 1;
        if ((int64_t)pref[(lo + half) * 32 + lane] < need) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// Every warp takes a contiguous range of sorted edges whose ends are moved to run
// starts, so that no directed pair's run is split between warps. It walks the range in
// windows of at most 32 edges made of whole runs (lane = edge), or, for a run longer
// than 32 edges, in 32-edge pieces of that run with per-query totals in shared memory.
// Windows and pieces whose 32-edge groups received no hit are passed over without
// reading their rows: their counts are all zero. Such a skip may end inside a run; the
// run's remaining edges then form the next window (a window that starts inside a run
// treats its first edge as the run's head), and the skipped edges contribute nothing to
// the pair's maximum or certificates.
// For a window it keeps the prefix sums of its edges' bins in shared memory; per class
// of queries each lane finds, by a binary search, the first bin at which its edge
// certifies, and only the class's queries at or past the warp's smallest such bin are
// evaluated (c_e(D_j) grows with j, so an edge certifies exactly for those bins). A
// window whose edges have no witness at any window of the pass costs its bin reads only.
template <typename C>
__global__ void __launch_bounds__(BT_THREADS) k_batch_threshold(const BatchArgs a) {
    extern __shared__ __align__(16) unsigned char bt_smem[];
    BatchClass* scls = reinterpret_cast<BatchClass*>(bt_smem);
    BatchQuery* sq = reinterpret_cast<BatchQuery*>(scls + a.ncls);
    int32_t* lmax = reinterpret_cast<int32_t*>(sq + a.nq);  // [BT_WARPS][nq]
    int32_t* lnc = lmax + BT_WARPS * a.nq;                  // [BT_WARPS][nq]
    C* prefs = reinterpret_cast<C*>(lnc + BT_WARPS * a.nq);  // [BT_WARPS][k][32]
    for (int i = threadIdx.x; i < a.ncls; i += blockDim.x) scls[i] = a.cls[i];
    for (int i = threadIdx.x; i < a.nq; i += blockDim.x) sq[i] = a.qs[i];
    __syncthreads();
    const C* bins = static_cast<const C*>(a.bins);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    C* pref = prefs + (int64_t)wib * a.k * 32;
    int32_t* wmax = lmax + wib * a.nq;
    int32_t* wnc = lnc + wib * a.nq;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t p = run_aligned(a.sd, a.seg, warp * a.per_warp, a.mk);
    const int64_t hi = run_aligned(a.sd, a.seg, (warp + 1) * a.per_warp, a.mk);
    const int64_t row_bytes = (int64_t)a.kstride * (int64_t)sizeof(C);
    unsigned long long rows_read = 0;
    while (p < hi) {
        const int64_t we = min(p + 32, hi);
        if (!touched_any(a.touched, p, we)) {
            p = we;
            continue;
        }
        int64_t L = we - p;
        if (we < hi) {
            const int32_t rl = a.sd[we - 1];
            if (a.sd[we] == rl) L = (int64_t)a.seg[rl] - p;  // drop the run that continues past the window
        }
        if (L > 0) {
            // ---- whole runs in lanes [0, L)
            const bool on = lane < L;
            const int64_t e = p + lane;
            const int32_t key = on ? a.sd[e] : -1;
            const uint32_t cmax = row_sum<C>(bins, a.kstride, e, on);
            rows_read += (unsigned long long)L;
            p += L;
            if (!__any_sync(0xffffffffu, cmax > 0)) continue;
            // only lanes with a witness need their prefix sums (the others read zero)
            if (cmax > 0) bin_prefix<C>(bins, a.kstride, a.k, e, true, pref);
            __syncwarp();
            const int32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
            const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || key != prev);
            const unsigned above = heads & ~((2u << lane) - 1u);
            const int start = 31 - __clz(heads & ((2u << lane) - 1u));
            const unsigned peers = (above ? (above & (0u - above)) - 1u : 0xffffffffu) & ~((1u << start) - 1u);
            const bool leader = on && lane == start;
            int64_t uh = 0, ut = 0, uc = 0;
            if (cmax > 0) universes(a, key, uh, ut, uc);
            for (int ci = 0; ci < a.ncls; ci++) {
                const BatchClass c = scls[ci];
                const int64_t need = needed(c, uh, ut, uc);
                const int jmin = (cmax > 0 && (int64_t)cmax >= need) ? first_bin<C>(pref, a.k, need) : a.k;
                const int jlo = __reduce_min_sync(0xffffffffu, jmin);
                if (jlo > c.jmax) continue;  // no edge of the window certifies for this class
                for (int qi = c.qb; qi < c.qe; qi++) {
                    const BatchQuery q = sq[qi];
                    if (q.j < jlo) continue;
                    const bool sat = q.j >= jmin;
                    const int cq = cmax > 0 ? (int)pref[q.j * 32 + lane] : 0;
                    const int rmax = __reduce_max_sync(peers, cq);
                    const int rsat = __reduce_add_sync(peers, sat ? 1 : 0);
                    emit_pairs(a, leader && rsat > 0, q.slot, key, rmax, rsat);
                }
            }
            __syncwarp();
        } else {
            // ---- one run longer than 32 edges, in pieces
            const int32_t key = a.sd[p];
            const int64_t re = a.seg[key + 1];
            for (int i = lane; i < a.nq; i += 32) {
                wmax[i] = 0;
                wnc[i] = 0;
            }
            __syncwarp();
            int64_t uh, ut, uc;
            universes(a, key, uh, ut, uc);
            for (int64_t b = p; b < re; b += 32) {
                if (!touched_any(a.touched, b, min(b + 32, re))) continue;
                const int64_t e = b + lane;
                const bool on = e < re;
                const uint32_t cmax = row_sum<C>(bins, a.kstride, e, on);
                rows_read += (unsigned long long)min((int64_t)32, re - b);
                if (!__any_sync(0xffffffffu, cmax > 0)) continue;
                if (cmax > 0) bin_prefix<C>(bins, a.kstride, a.k, e, true, pref);
                __syncwarp();
                for (int ci = 0; ci < a.ncls; ci++) {
                    const BatchClass c = scls[ci];
                    const int64_t need = needed(c, uh, ut, uc);
                    const int jmin = (cmax > 0 && (int64_t)cmax >= need) ? first_bin<C>(pref, a.k, need) : a.k;
                    const int jlo = __reduce_min_sync(0xffffffffu, jmin);
                    if (jlo > c.jmax) continue;
                    for (int qi = c.qb; qi < c.qe; qi++) {
                        const BatchQuery q = sq[qi];
                        if (q.j < jlo) continue;
                        const int rmax = __reduce_max_sync(0xffffffffu, cmax > 0 ? (int)pref[q.j * 32 + lane] : 0);
                        const int rsat = __reduce_add_sync(0xffffffffu, q.j >= jmin ? 1 : 0);
                        if (lane == 0) {
                            wmax[qi] = max(wmax[qi], rmax);
                            wnc[qi] += rsat;
                        }
                    }
                }
                __syncwarp();
            }
            __syncwarp();
            for (int i0 = 0; i0 < a.nq; i0 += 32) {
                const int i = i0 + lane;
                const bool emit = i < a.nq && wnc[i] > 0;
                emit_pairs(a, emit, emit ? sq[i].slot : 0, key, emit ? wmax[i] : 0, emit ? wnc[i] : 0);
            }
            __syncwarp();
            p = re;
        }
    }
    // model bytes: the rows read and their run keys, once per warp
    if (a.prof && lane == 0 && rows_read)
        atomicAdd(a.prof, rows_read * (unsigned long long)(row_bytes + 4));
}

// Zeroes the rows of every 32-edge group marked in touched (the only rows a binned probe
// pass wrote), so that the bins are clear again for the next pass: one warp per group.
template <typename C>
__global__ void k_bins_clear(const uint32_t* __restrict__ touched, C* __restrict__ bins, int kstride, int64_t mk) {
    const int lane = threadIdx.x & 31;
    const int64_t ng = (mk + 31) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < ng; gi += nw) {
        if (!((__ldg(touched + (gi >> 5)) >> (gi & 31)) & 1u)) continue;
        const int64_t r0 = gi << 5, r1 = min(r0 + 32, mk);
        // rows of kstride * sizeof(C) bytes, a multiple of 16
        uint4* q = reinterpret_cast<uint4*>(bins + r0 * (int64_t)kstride);
        const int64_t n16 = (r1 - r0) * (int64_t)kstride * (int64_t)sizeof(C) / 16;
        for (int64_t i = lane; i < n16; i += 32) q[i] = make_uint4(0, 0, 0, 0);
    }
}

// Sorted solutions -> out = [u... | v... | count... | ncert...]; qstart[slot] = first
// index of the slot's solutions (left at -1 for a slot without any).
__global__ void k_batch_gather(const uint64_t* __restrict__ key, const uint32_t* __restrict__ order,
                               const int32_t* __restrict__ run, const int32_t* __restrict__ cnt,
                               const int32_t* __restrict__ nc, const int32_t* __restrict__ ea,
                               const int32_t* __restrict__ eb, int64_t n, int rb, int32_t* __restrict__ out,
                               int32_t* __restrict__ qstart) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = order[i];
        const int32_t r = run[o], s = r >> 1;
        out[i] = (r & 1) ? eb[s] : ea[s];
        out[n + i] = (r & 1) ? ea[s] : eb[s];
        out[2 * n + i] = cnt[o];
        out[3 * n + i] = nc[o];
        const int q = (int)(key[i] >> rb);
        if (i == 0 || (int)(key[i - 1] >> rb) != q) qstart[q] = (int32_t)i;
    }
}

__global__ void k_iota_u32(uint32_t* __restrict__ a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (uint32_t)i;
}

// ------------------------------------------------------------------ host side

static int64_t batch_bin_budget_bytes() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return (int64_t)1 << 30;
    }
    int64_t b = (int64_t)(free_b / 4);
    const int64_t cap = (int64_t)16 << 30;
    return b < cap ? b : cap;
}

static bool plain_query(const folty_query_params& q) {
    return !q.want_edge_counts && !q.want_certificates && !q.outer && !q.want_triples;
}

// Solution buffer entries of a fused pass: key, alternate key, run, count, certificates,
// two sort values (36 B each).
constexpr int64_t BT_ENTRY_BYTES = 36;
constexpr int64_t BT_DEFAULT_CAP = int64_t(1) << 22;

// Bins of one probe pass: the largest number of distinct deltas of one direction variant.
int64_t batch_footprint(const folty_graph* g, const folty_query_params* qs, int nq, int64_t* bins_part) {
    int64_t kmax = 0;
    for (int dir = 0; dir <= FOLTY_DIR_EITHER; dir++) {
        std::vector<int64_t> D;
        for (int i = 0; i < nq; i++)
            if (qs[i].dir == dir) D.push_back(qs[i].delta);
        std::sort(D.begin(), D.end());
        D.erase(std::unique(D.begin(), D.end()), D.end());
        kmax = std::max<int64_t>(kmax, (int64_t)D.size());
    }
    kmax = std::min<int64_t>(kmax, BATCH_MAX_BINS);
    const int64_t bins = ((kmax + 7) & ~int64_t(7)) * g->m_kept * 4;  // rows padded to 16 bytes
    // the fused pass: its solution buffer and the pair ranks
    int64_t fused = 0;
    bool any_plain = false;
    for (int i = 0; i < nq; i++) any_plain = any_plain || plain_query(qs[i]);
    if (any_plain) fused = BT_DEFAULT_CAP * BT_ENTRY_BYTES + 4 * 2 * (int64_t)g->S;
    // output stage per query of a read-back group of the single-query path (see
    // finish_queries): 6 int32 arrays of 2S + 1, compacted keys, packed output, edge counts
    // when asked
    const int64_t n2 = 2 * (int64_t)g->S;
    int64_t per_q = 6 * 4 * (n2 + 1) + 8 * n2 + 16 * n2 + 64;
    bool edges = false, certs = false, outer = false, other = false;
    for (int i = 0; i < nq; i++) {
        edges = edges || qs[i].want_edge_counts;
        certs = certs || qs[i].want_certificates;
        outer = outer || qs[i].outer;
        other = other || (!plain_query(qs[i]) && !qs[i].want_triples);
    }
    if (edges) per_q += 4 * g->m;
    if (other) per_q += 4 * g->m_kept;  // the query's counts gathered from the bin rows
    if (certs) per_q += 16 * (g->m + 1);
    if (outer) per_q += 14 * ((int64_t)g->n + 1);
    const int64_t group = other ? std::min<int64_t>(nq, READBACK_MAX / 4) : 0;
    // a triple query runs alone: role flags and scan (9 B per role), and up to one triple
    // per role through the two sorts (44 B each), on top of its own counters
    bool triples = false;
    for (int i = 0; i < nq; i++) triples = triples || qs[i].want_triples;
    const int64_t tri_part = triples ? 53 * 6 * g->ntri + 4 * g->m_kept + per_q : 0;
    if (bins_part) *bins_part = bins;
    return std::max(bins + fused + group * per_q, tri_part);
}

// The fused threshold of the plain queries `fq` (at most BT_MAXQ, with their bins j) over
// the bins of one probe pass (edge-major rows of kstride); fills their results.
template <typename C>
static void fused_threshold(folty_graph* g, const C* bins, const uint32_t* touched, int k, int kstride,
                            const std::vector<const folty_query_params*>& fq, const std::vector<int>& fj,
                            const std::vector<folty_result*>& fo, cudaStream_t s) {
    const int nq = (int)fq.size();
    const int64_t mk = g->m_kept;
    const int64_t S = g->S;
    Scratch sc(g->alloc, s, g->dev_err);
    const int32_t* prank = pair_ranks(g, s);
    // classes of queries that differ only in their window (quantifier, universe and rho
    // in lowest terms; rho is irrelevant to the existential quantifier), each sorted by bin
    struct Key {
        int quant, universe;
        int64_t num, den;
        bool operator<(const Key& o) const {
            return std::tie(quant, universe, num, den) < std::tie(o.quant, o.universe, o.num, o.den);
        }
    };
    std::map<Key, std::vector<int>> groups;
    for (int i = 0; i < nq; i++) {
        const folty_query_params& q = *fq[(size_t)i];
        Key key{(int)q.quant, (int)q.universe, (int64_t)q.rho_num, (int64_t)q.rho_den};
        if (q.quant == FOLTY_Q_EXISTS) key = Key{FOLTY_Q_EXISTS, 0, 0, 1};
        else {
            const int64_t gcd = std::gcd(key.num, key.den);
            key.num /= gcd;
            key.den /= gcd;
        }
        groups[key].push_back(i);
    }
    std::vector<BatchClass> hc;
    std::vector<BatchQuery> hq;
    for (auto& kv : groups) {
        std::vector<int>& v = kv.second;
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return fj[(size_t)x] < fj[(size_t)y]; });
        BatchClass c{kv.first.quant, kv.first.universe, kv.first.num, kv.first.den, (int32_t)hq.size(), 0, 0, 0};
        for (int i : v) hq.push_back(BatchQuery{fj[(size_t)i], i});
        c.qe = (int32_t)hq.size();
        c.jmax = hq.back().j;
        hc.push_back(c);
    }
    const int ncls = (int)hc.size();
    BatchClass* dc = sc.get<BatchClass>(ncls);
    BatchQuery* dq = sc.get<BatchQuery>(nq);
    FOLTY_CUDA(cudaMemcpyAsync(dc, hc.data(), sizeof(BatchClass) * (size_t)ncls, cudaMemcpyHostToDevice, s));
    FOLTY_CUDA(cudaMemcpyAsync(dq, hq.data(), sizeof(BatchQuery) * (size_t)nq, cudaMemcpyHostToDevice, s));
    // shared memory: classes, queries, per-warp long-run totals, per-warp prefix sums
    const size_t smem = sizeof(BatchClass) * (size_t)ncls + sizeof(BatchQuery) * (size_t)nq +
                        2 * sizeof(int32_t) * BT_WARPS * (size_t)nq + sizeof(C) * BT_WARPS * 32 * (size_t)k;
    // the attribute is the kernel's, shared by every thread: always the same bound (the
    // largest pass: BT_KMAX 16-bit or BT_KMAX / 2 32-bit bins), so that concurrent batches
    // (a server's workers) never lower it under one another's launch
    constexpr size_t smem_max = sizeof(BatchClass) * BT_MAXQ + sizeof(BatchQuery) * BT_MAXQ +
                                2 * sizeof(int32_t) * BT_WARPS * BT_MAXQ + 2 * BT_WARPS * 32 * BT_KMAX;
    if (smem > smem_max) fail(FOLTY_EINVAL, "batched threshold: too many bins or queries for one pass");
    FOLTY_CUDA(cudaFuncSetAttribute(k_batch_threshold<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    int per_sm = 0;
    FOLTY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_threshold<C>, BT_THREADS, smem));
    const int64_t blocks = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int64_t nwarps = blocks * BT_WARPS;
    BatchArgs a{};
    a.bins = bins;
    a.touched = touched;
    a.k = k;
    a.kstride = kstride;
    a.mk = mk;
    a.sd = g->sd;
    a.seg = g->seg;
    a.ea = g->ea;
    a.eb = g->eb;
    a.deg = g->deg;
    a.common = g->common;
    a.prank = prank;
    a.cls = dc;
    a.ncls = ncls;
    a.qs = dq;
    a.nq = nq;
    a.rb = bit_length((uint64_t)(2 * S > 1 ? 2 * S - 1 : 1));
    a.per_warp = (mk + nwarps - 1) / nwarps;
    a.n_out = sc.get<unsigned long long>(1);
    // each (query, directed pair) is emitted at most once; FOLTY_BATCH_SOLUTION_CAP sets a
    // smaller first buffer (the tests use it to run the second pass)
    int64_t cap = BT_DEFAULT_CAP;
    if (const char* env = std::getenv("FOLTY_BATCH_SOLUTION_CAP")) cap = std::max<int64_t>(1, std::atoll(env));
    cap = std::min<int64_t>(cap, std::max<int64_t>(1, (int64_t)nq * 2 * S));
    int64_t n_out = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        Scratch so(g->alloc, s, g->dev_err);
        a.cap = cap;
        a.out_key = so.get<uint64_t>(cap);
        a.out_run = so.get<int32_t>(cap);
        a.out_cnt = so.get<int32_t>(cap);
        a.out_nc = so.get<int32_t>(cap);
        FOLTY_CUDA(cudaMemsetAsync(a.n_out, 0, sizeof(unsigned long long), s));
        a.prof = nullptr;
        if (profiling_on()) {
            a.prof = g->prof_bytes + (g->prof_next++ % PROF_SLOTS);
            FOLTY_CUDA(cudaMemsetAsync(a.prof, 0, sizeof(unsigned long long), s));
        }
        {
            // model bytes: the group bits, plus (counted on the device) the rows of the
            // groups with a hit and their run keys
            StageSpan span(ST_BATCH, s, 4 * ((mk + 1023) / 1024), a.prof);
            if (mk > 0) FOLTY_LAUNCH(k_batch_threshold<C>, (unsigned)blocks, BT_THREADS, smem, s, a);
        }
        n_out = read_i64(g, (const int64_t*)a.n_out, s);
        if (n_out > cap) {  // the buffer was too small: run again with room for all
            cap = n_out;
            continue;
        }
        // sort by (query slot, pair rank); gather into per-query (u, v, count, ncert)
        const int64_t n = n_out;
        std::vector<int32_t> qstart((size_t)nq + 1, -1);
        std::vector<int32_t> host;
        const int32_t* packed_h = nullptr;
        if (n > 0) {
            uint64_t* kalt = so.get<uint64_t>(n);
            uint32_t* v0 = so.get<uint32_t>(n);
            uint32_t* v1 = so.get<uint32_t>(n);
            int32_t* packed = so.get<int32_t>(4 * n + nq + 1);
            int32_t* qs_dev = packed + 4 * n;
            FOLTY_LAUNCH(k_iota_u32, grid_for(n, 256), 256, 0, s, v0, n);
            const int bits = a.rb + bit_length((uint64_t)(nq > 1 ? nq - 1 : 1));
            const bool alt = radix_sort_pairs(so, a.out_key, kalt, v0, v1, n, bits);
            read_back(g, nullptr, nullptr, 0, nullptr, s);  // the sort's look-backs completed
            const uint64_t* ks = alt ? kalt : a.out_key;
            const uint32_t* ord = alt ? v1 : v0;
            FOLTY_CUDA(cudaMemsetAsync(qs_dev, 0xff, sizeof(int32_t) * (size_t)(nq + 1), s));
            FOLTY_LAUNCH(k_batch_gather, grid_for(n, 256), 256, 0, s, ks, ord, a.out_run, a.out_cnt, a.out_nc, g->ea,
                         g->eb, n, a.rb, packed, qs_dev);
            const size_t bytes = sizeof(int32_t) * (size_t)(4 * n + nq);
            if (bytes <= sizeof(int32_t) * 4 * (size_t)PAIR_STAGE) {
                g->stage_busy = 1;
                FOLTY_CUDA(cudaMemcpyAsync(g->pair_stage, packed, bytes, cudaMemcpyDeviceToHost, s));
                FOLTY_CUDA(cudaStreamSynchronize(s));
                g->stage_busy = 0;
                packed_h = (const int32_t*)(g->host_stage + HOST_STAGE);
            } else {
                host.resize(4 * (size_t)n + (size_t)nq);
                FOLTY_CUDA(cudaMemcpyAsync(host.data(), packed, bytes, cudaMemcpyDeviceToHost, s));
                FOLTY_CUDA(cudaStreamSynchronize(s));
                packed_h = host.data();
            }
            std::memcpy(qstart.data(), packed_h + 4 * n, sizeof(int32_t) * (size_t)nq);
        }
        qstart[(size_t)nq] = (int32_t)n;
        // the end of a slot's solutions is the next slot's start (slots without any are -1)
        for (int i = nq - 1; i >= 0; i--) {
            if (qstart[(size_t)i] < 0) qstart[(size_t)i] = qstart[(size_t)i + 1];
        }
        for (int i = 0; i < nq; i++) {
            const int64_t b = qstart[(size_t)i], e = qstart[(size_t)i + 1], np = e - b;
            folty_result* out = fo[(size_t)i];
            fill_result_host(out, np, g->m, false, 0, false, 0, false);
            int64_t ncert = 0;
            if (np > 0) {
                std::memcpy(out->u, packed_h + b, sizeof(int32_t) * (size_t)np);
                std::memcpy(out->v, packed_h + n + b, sizeof(int32_t) * (size_t)np);
                std::memcpy(out->count, packed_h + 2 * n + b, sizeof(int32_t) * (size_t)np);
                std::memcpy(out->ncert, packed_h + 3 * n + b, sizeof(int32_t) * (size_t)np);
                for (int64_t x = 0; x < np; x++) ncert += out->ncert[x];
            }
            out->n_cert_edges = ncert;
        }
        return;
    }
    fail(FOLTY_ECUDA, "batched threshold: the solution count grew between two passes over the same bins");
}

void run_query_batch(folty_graph* g, const folty_query_params* qs, int nq, folty_result* outs,
                     cudaStream_t s, int64_t bin_budget) {
    const int64_t mk = g->m_kept;
    const int64_t P = g->info.probes;
    // a batch of one (a server's batch under light load) is a single query: its captured
    // launch sequence is the shortest path
    if (nq == 1) {
        run_query(g, qs[0], &outs[0], s);
        return;
    }
    // a query that also wants the all-existential triples needs its own probe pass (the
    // role flags are per window, not per bin)
    for (int i = 0; i < nq; i++)
        if (qs[i].want_triples) run_query(g, qs[i], &outs[i], s);
    // group the queries by direction variant; distinct sorted deltas per group
    // 16-bit bins while no count can reach 2^16 (a count is at most the number of common
    // neighbours of an edge's ends, at most the largest degree): half the memory traffic
    // of the bins and of the threshold's reads
    const bool b16 = g->info.max_degree < 65535;
    const int64_t per_bin = mk * (int64_t)(b16 ? sizeof(uint16_t) : sizeof(int32_t));
    const int64_t budget = bin_budget > 0 ? bin_budget : batch_bin_budget_bytes();
    struct Pass {
        int dir;
        std::vector<int> members;
        std::vector<int64_t> D;
        int64_t chunk;
    };
    std::vector<Pass> passes;
    int kstride_max = 0;
    for (int dir = 0; dir <= FOLTY_DIR_EITHER; dir++) {
        Pass ps{dir, {}, {}, 0};
        for (int i = 0; i < nq; i++)
            if (qs[i].dir == dir && !qs[i].want_triples) ps.members.push_back(i);
        if (ps.members.empty()) continue;
        for (int i : ps.members) ps.D.push_back(qs[i].delta);
        std::sort(ps.D.begin(), ps.D.end());
        ps.D.erase(std::unique(ps.D.begin(), ps.D.end()), ps.D.end());
        int64_t chunk = per_bin > 0 ? budget / per_bin : (int64_t)ps.D.size();
        chunk = std::max<int64_t>(1, std::min<int64_t>({chunk, (int64_t)BATCH_MAX_BINS, (int64_t)ps.D.size()}));
        // the fused pass keeps every window's prefix sums in shared memory: at most BT_KMAX
        // 16-bit (BT_KMAX / 2 32-bit) bins per probe pass when plain queries are present
        bool plain = false;
        for (int i : ps.members) plain = plain || plain_query(qs[i]);
        if (plain) chunk = std::min<int64_t>(chunk, b16 ? BT_KMAX : BT_KMAX / 2);
        ps.chunk = chunk;
        const int kk = (int)chunk;
        kstride_max = std::max(kstride_max, b16 ? (kk + 7) & ~7 : (kk + 3) & ~3);
        passes.push_back(std::move(ps));
    }
    if (passes.empty()) return;
    // one bin buffer for every pass, cleared once: each pass marks the 32-edge groups it
    // writes, its consumers read only those, and k_bins_clear zeroes them again
    Scratch sb(g->alloc, s, g->dev_err);
    int32_t* bins = b16 ? nullptr : sb.get<int32_t>(mk * kstride_max);
    uint16_t* bins16 = b16 ? sb.get<uint16_t>(mk * kstride_max) : nullptr;
    const int64_t twords = (mk + 1023) / 1024 + 1;
    uint32_t* touched = sb.get<uint32_t>(twords);
    if (mk > 0) {
        if (b16) FOLTY_CUDA(cudaMemsetAsync(bins16, 0, sizeof(uint16_t) * (size_t)(mk * kstride_max), s));
        else FOLTY_CUDA(cudaMemsetAsync(bins, 0, sizeof(int32_t) * (size_t)(mk * kstride_max), s));
    }
    for (const Pass& ps : passes) {
        const int dir = ps.dir;
        const std::vector<int>& members = ps.members;
        const std::vector<int64_t>& D = ps.D;
        const int64_t chunk = ps.chunk;
        for (size_t c0 = 0; c0 < D.size(); c0 += (size_t)chunk) {
            const int k = (int)std::min<int64_t>(chunk, (int64_t)D.size() - (int64_t)c0);
            // edge-major rows of whole 16-byte chunks
            const int kstride = b16 ? (k + 7) & ~7 : (k + 3) & ~3;
            Scratch sc(g->alloc, s, g->dev_err);
            int64_t* dd = sc.get<int64_t>(k);
            std::vector<int64_t> hd(D.begin() + (long)c0, D.begin() + (long)c0 + k);
            // the bin bounds in the store's timestamp type (32-bit offsets: gaps stay
            // below 2^32 - 1, so larger windows behave as 2^32 - 2), staged in the graph's
            // pinned pair stage, which nothing uses before this chunk's threshold pass
            // (the last chunk's read-back has completed)
            void* hb = g->host_stage + HOST_STAGE;
            if (g->ts32) {
                uint32_t* h32 = static_cast<uint32_t*>(hb);
                for (int i = 0; i < k; i++) h32[i] = hd[i] >= 0xfffffffell ? 0xfffffffeu : (uint32_t)hd[i];
            } else {
                std::memcpy(hb, hd.data(), sizeof(int64_t) * (size_t)k);
            }
            g->stage_busy = 1;
            FOLTY_CUDA(cudaMemcpyAsync(dd, hb, (g->ts32 ? sizeof(uint32_t) : sizeof(int64_t)) * (size_t)k,
                                       cudaMemcpyHostToDevice, s));
            if (mk > 0) {
                FOLTY_CUDA(cudaMemsetAsync(touched, 0, sizeof(uint32_t) * (size_t)twords, s));
                if (P > 0)
                    launch_probe_live(g, hd[k - 1], dir, 1, nullptr, bins, k, kstride, dd, s, nullptr, bins16,
                                      touched);
            }
            // the chunk's queries: plain ones through the fused pass over the bins, the
            // others through the single-query path over their window's counts
            std::vector<const folty_query_params*> pq, fq;
            std::vector<int> pj;
            std::vector<CountView> fc;
            std::vector<folty_result*> po, fo;
            for (int i : members) {
                auto it = std::lower_bound(hd.begin(), hd.end(), qs[i].delta);
                if (it == hd.end() || *it != qs[i].delta) continue;  // another chunk
                const int j = (int)(it - hd.begin());
                if (plain_query(qs[i])) {
                    pq.push_back(&qs[i]);
                    pj.push_back(j);
                    po.push_back(&outs[i]);
                    continue;
                }
                fq.push_back(&qs[i]);
                // the query's counts c_e(D_j), gathered from the rows
                if (b16) {
                    uint16_t* col = sc.get<uint16_t>(mk + 2);
                    if (mk > 0)
                        FOLTY_LAUNCH(k_bins_column<uint16_t>, grid_for(mk, 256), 256, 0, s, bins16, kstride, j, mk, col);
                    fc.push_back(CountView{nullptr, col});
                } else {
                    int32_t* col = sc.get<int32_t>(mk);
                    if (mk > 0)
                        FOLTY_LAUNCH(k_bins_column<int32_t>, grid_for(mk, 256), 256, 0, s, bins, kstride, j, mk, col);
                    fc.push_back(CountView{col, nullptr});
                }
                fo.push_back(&outs[i]);
            }
            for (size_t q0 = 0; q0 < pq.size(); q0 += BT_MAXQ) {
                const size_t q1 = std::min(pq.size(), q0 + (size_t)BT_MAXQ);
                std::vector<const folty_query_params*> gq(pq.begin() + (long)q0, pq.begin() + (long)q1);
                std::vector<int> gj(pj.begin() + (long)q0, pj.begin() + (long)q1);
                std::vector<folty_result*> go(po.begin() + (long)q0, po.begin() + (long)q1);
                if (b16) fused_threshold<uint16_t>(g, bins16, touched, k, kstride, gq, gj, go, s);
                else fused_threshold<int32_t>(g, bins, touched, k, kstride, gq, gj, go, s);
            }
            if (!fq.empty()) finish_queries(g, fq.data(), fc.data(), (int)fq.size(), fo.data(), s);
            // every reader of this pass's bins is enqueued: clear the rows it wrote
            if (mk > 0) {
                const int64_t ng = (mk + 31) / 32;
                const unsigned blocks = (unsigned)std::min<int64_t>((ng + 7) / 8, (int64_t)num_sms() * 16);
                if (b16) FOLTY_LAUNCH(k_bins_clear<uint16_t>, blocks, 256, 0, s, touched, bins16, kstride, mk);
                else FOLTY_LAUNCH(k_bins_clear<int32_t>, blocks, 256, 0, s, touched, bins, kstride, mk);
            }
        }
    }
}

}  // namespace folty
