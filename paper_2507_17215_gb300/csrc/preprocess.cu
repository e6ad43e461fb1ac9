// Preprocessing of a loaded temporal graph (paper Section 2, Preliminaries, and the
// first steps of Algorithm 6):
//   A1  drop self-loops; sort temporal edges by (static pair, direction, t) so that
//       every E_{x,y} is a contiguous ascending run of the timestamp store T;
//   A2  static graph G_S as CSR, neighbours ascending, with static-edge ids;
//   A3  core numbers and a degeneracy order by parallel peeling (Definition 2.1 and
//       the Matula-Beck removal of Section 2, done a frontier at a time);
//   A4  orientation G->pi: u -> v iff (round(u), u) < (round(v), v); out-degree <= alpha;
//   A5  every triangle of G_S exactly once: (u, v) in G->, w in N+(u) cap N+(v)
//       (Algorithm 3's enumeration skeleton), with its per-triangle probe count.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <optional>

#include "internal.cuh"
#include "pairs.cuh"

#include <cooperative_groups.h>
namespace cg = cooperative_groups;
#include "probe.cuh"

namespace folty {

// ================================================================== A1

// Sort key of a temporal edge: 2 p(a, b) + dir with a = min, b = max id, dir = (src > dst)
// and p(a, b) = a (2n - a - 1) / 2 + (b - a - 1) the rank of the pair among all pairs
// a < b in (a, b) order, so keys order edges by (a, b, dir) within n (n - 1) values (one
// bit narrower than packing a and b side by side: 40 bits for a million vertices).
// Self-loops get the all-ones key of the used width and sort last.
__global__ void k_build_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                             int64_t m, int32_t n, uint64_t loop_key, uint64_t* __restrict__ key,
                             uint32_t* __restrict__ val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = src[i], y = dst[i];
        uint64_t k;
        if (x == y) {
            k = loop_key;
        } else {
            const uint64_t a = (uint64_t)min(x, y), b = (uint64_t)max(x, y);
            const uint64_t p = a * (2 * (uint64_t)n - a - 1) / 2 + (b - a - 1);
            k = 2 * p + (uint64_t)(x > y);
        }
        key[i] = k;
        val[i] = (uint32_t)i;
    }
}

__global__ void k_time_keys(const int64_t* __restrict__ t, int64_t m, int64_t tmin,
                            uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = (uint64_t)(t[i] - tmin);
        val[i] = (uint32_t)i;
    }
}

__global__ void k_gather_keys(const uint64_t* __restrict__ key_in, const uint32_t* __restrict__ order,
                              int64_t m, uint64_t* __restrict__ key_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        key_out[i] = key_in[order[i]];
}

// perm, T (gathered from t: 32-bit offsets from tmin, or the raw int64 timestamps), and
// the "new static pair" flag of every kept sorted position.
template <typename TS>
__global__ void k_store(const uint64_t* __restrict__ key, const uint32_t* __restrict__ order,
                        const TS* __restrict__ t, int64_t mk, int32_t* __restrict__ perm,
                        TS* __restrict__ T, int32_t* __restrict__ newpair) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = __ldcs(order + i);
        __stcs(perm + i, (int32_t)o);
        T[i] = t[o];
        const uint64_t k = __ldcs(key + i);
        __stcs(newpair + i, (int32_t)((i == 0) || ((k >> 1) != (key[i - 1] >> 1))));
    }
}

// 32-bit offsets t - tbase of the input timestamps. 4 bytes an edge keep the gather of
// k_store inside L2 for inputs of up to ~25M edges (the int64 input is twice that).
__global__ void k_offsets32(const int64_t* __restrict__ t, int64_t m, int64_t tbase, uint32_t* __restrict__ t32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        t32[i] = (uint32_t)(__ldcs(t + i) - tbase);
}

// Static edge ids and segment starts. pscan = exclusive scan of newpair.
__global__ void k_segments(const uint64_t* __restrict__ key, const int32_t* __restrict__ newpair,
                           const int32_t* __restrict__ pscan, int64_t mk, int32_t* __restrict__ sd,
                           int32_t* __restrict__ seg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = key[i];
        int32_t s = pscan[i] + newpair[i] - 1;
        int dir = (int)(k & 1);
        sd[i] = 2 * s + dir;
        if (newpair[i]) {
            seg[2 * s] = (int32_t)i;
            seg[2 * s + 1] = -1;
        }
    }
}

// Pairs a < b with first element below x: x (2n - x - 1) / 2.
__device__ __forceinline__ uint64_t pairs_before(int64_t x, int32_t n) {
    return (uint64_t)x * (uint64_t)(2 * (int64_t)n - x - 1) / 2;
}

// The pair (a, b) of rank p (inverse of the key of k_build_keys): a is the largest x with
// pairs_before(x) <= p, first estimated from the smaller root of x^2 - (2n - 1) x + 2p = 0
// (the discriminant (2n - 1)^2 - 8p is exact in 64 bits for n < 2^31; its square root is
// taken in single precision, a few units off at most for ids below 2^24), then corrected
// by exact integer comparisons.
__device__ __forceinline__ void pair_of_rank(uint64_t p, int32_t n, int32_t& a, int32_t& b) {
    const uint64_t c = 2 * (uint64_t)n - 1;
    const uint64_t disc = c * c - 8 * p;
    int64_t x = (int64_t)(((float)c - sqrtf((float)disc)) * 0.5f);
    x = x < 0 ? 0 : (x > n - 2 ? n - 2 : x);
    while (x > 0 && pairs_before(x, n) > p) x--;
    while (x + 1 <= n - 2 && pairs_before(x + 1, n) <= p) x++;
    a = (int32_t)x;
    b = (int32_t)(p - pairs_before(x, n) + (uint64_t)x + 1);
}

// Endpoints of static edge s from the key of its first temporal edge (one thread per
// static edge, so that no warp idles through the decoding).
__global__ void k_pair_ends(const uint64_t* __restrict__ key, const int32_t* __restrict__ seg, int32_t S,
                            int32_t n, int32_t* __restrict__ ea, int32_t* __restrict__ eb) {
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        int32_t x, y;
        pair_of_rank(key[seg[2 * s]] >> 1, n, x, y);
        ea[s] = x;
        eb[s] = y;
    }
}

// ---------------------------------------------------------------- dense pair ids
//
// When the distinct pairs are few enough, the edges are sorted by (pair id, direction)
// with pair ids numbered 0..S-1 in (a, b) order, instead of by the full pair key: the id
// and the direction bit need about log2(2S) bits, which leaves room for the edge's
// time rank in the same 64-bit word. The sort is then keys only and takes 3 digit
// passes on the medium graph instead of 5 passes with values. The distinct pairs come
// from an open-addressed table (linear probing from a multiplicative hash of the pair
// rank); they are sorted on their own (S entries), and each edge looks its id up by the
// table slot it kept from the insert.

constexpr int PAIR_COMPACT_ITEMS = 16;            // table slots per thread and step of the compaction

// Every non-loop edge's pair goes into the table (value rank + 1, 0 = empty), and edge i
// keeps its slot and direction in slotw[i] (PAIR_LOOP for a self-loop). A probe sequence
// that runs out sets *over.
__global__ void k_pair_insert(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m, int32_t n,
                              uint64_t* __restrict__ table, int lg, uint32_t* __restrict__ slotw,
                              int* __restrict__ over) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        __stcs(slotw + i, pair_slot_word(table, lg, src[i], dst[i], n, over));
}

// The occupied slots as (rank, slot) lists, in no particular order: each block takes
// PAIR_COMPACT_ITEMS * blockDim.x slots per step and reserves their entries with one
// global atomic. *cnt ends at the number of distinct pairs; entries past cap are not
// written (the caller then abandons the table).
__global__ void k_pair_table_compact(const uint64_t* __restrict__ table, int64_t tb, uint64_t* __restrict__ urank,
                               uint32_t* __restrict__ uslot, int* __restrict__ cnt, int cap) {
    __shared__ int wsum[32], base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t step = (int64_t)PAIR_COMPACT_ITEMS * blockDim.x;
    for (int64_t s0 = blockIdx.x * step; s0 < tb; s0 += gridDim.x * step) {
        uint64_t v[PAIR_COMPACT_ITEMS];
        int c = 0;
#pragma unroll
        for (int q = 0; q < PAIR_COMPACT_ITEMS; q++) {
            const int64_t sl = s0 + (int64_t)q * blockDim.x + threadIdx.x;
            v[q] = sl < tb ? table[sl] : 0;
            c += v[q] != 0;
        }
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < nw; w++) {
                const int x = wsum[w];
                wsum[w] = t;
                t += x;
            }
            base = t ? atomicAdd(cnt, t) : 0;
        }
        __syncthreads();
        int at = base + wsum[warp] + inc - c;
#pragma unroll
        for (int q = 0; q < PAIR_COMPACT_ITEMS; q++) {
            if (v[q] != 0) {
                if (at < cap) {
                    urank[at] = v[q] - 1;
                    uslot[at] = (uint32_t)(s0 + (int64_t)q * blockDim.x + threadIdx.x);
                }
                at++;
            }
        }
        __syncthreads();  // wsum and base are rewritten by the next step
    }
}

// Pair id j (position in rank order) of every table slot in use, and the pair's ends.
// The ranks come from a sort whose look-back could in principle run out (the graph's
// error word, checked by the host before the ids are used, then says so): slots and ends
// are kept inside their arrays whatever the input.
__global__ void k_pair_ids(const uint64_t* __restrict__ urank, const uint32_t* __restrict__ uslot, int32_t S,
                           int32_t n, int64_t tb, int32_t* __restrict__ sid, int32_t* __restrict__ ea,
                           int32_t* __restrict__ eb) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < S; j += gridDim.x * blockDim.x) {
        const uint32_t sl = uslot[j];
        if (sl < tb) sid[sl] = j;
        int32_t x, y;
        pair_of_rank(urank[j], n, x, y);
        ea[j] = min(x, n - 1);
        eb[j] = min(y, n - 1);
    }
}

// Sort word of the edge at time rank j (input index o = order[j], or j when the input is
// in time order): (2 pair id + direction) << ib | j; self-loops get 2S and sort last.
// With tv (32-bit stores), also the edge's 32-bit time offset t[o] - tmin, the value the
// sort carries along, so that the sorted timestamps need no gather; and sigma[p] counts
// the temporal edges of pair p, which the triangle passes need before the sort is done.
__global__ void k_pair_pack(const uint32_t* __restrict__ slotw, const uint32_t* __restrict__ order, int64_t m,
                            const int32_t* __restrict__ sid, int32_t S, int ib, uint64_t* __restrict__ packed,
                            const int64_t* __restrict__ t, int64_t tmin, uint32_t* __restrict__ tv,
                            int32_t* __restrict__ sigma) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = order ? (int64_t)order[j] : j;
        const uint32_t w = order ? slotw[o] : __ldcs(slotw + j);
        uint64_t c = 2 * (uint64_t)S;
        if (w != PAIR_LOOP) {
            const int32_t p = sid[w & ~PAIR_DIR];
            c = 2 * (uint64_t)p + (w >> 31);
            if ((unsigned)p < (unsigned)S) atomicAdd(&sigma[p], 1);
        }
        packed[j] = (c << ib) | (uint64_t)j;
        if (tv) tv[j] = (uint32_t)((order ? t[o] : __ldcs(t + j)) - tmin);
    }
}

// The first step of the store of a time-ordered input with 32-bit time offsets: each
// edge's sort id c = 2 pair id + direction (2S for a self-loop) into cw, and the number
// of edges of every id into cnt[0..2S] (zeroed; of consecutive edges of one id a thread
// sees, only the first adds, by their number; the self-loops are summed per warp first).
// Eight edges per thread (their id lookups in flight together), 16-byte loads and stores.
constexpr int STORE_IDS_EDGES = 8;  // consecutive edges per thread of k_store_ids
__global__ void __launch_bounds__(256) k_store_ids(const uint32_t* __restrict__ slotw, int64_t m,
                                                   const int32_t* __restrict__ sid, int32_t S,
                                                   uint32_t* __restrict__ cw, int32_t* __restrict__ cnt) {
    constexpr int E = STORE_IDS_EDGES;
    const int64_t nq = (m + E - 1) / E;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j0 = q * E;
        const bool full = j0 + E <= m;
        uint32_t w[E];
        if (full) {
#pragma unroll
            for (int h = 0; h < E / 4; h++) {
                const uint4 ww = __ldcs(reinterpret_cast<const uint4*>(slotw + j0) + h);
                w[4 * h] = ww.x;
                w[4 * h + 1] = ww.y;
                w[4 * h + 2] = ww.z;
                w[4 * h + 3] = ww.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) w[e] = j0 + e < m ? slotw[j0 + e] : PAIR_LOOP;
        }
        // all the id lookups in flight before any is used
        int32_t p[E];
#pragma unroll
        for (int e = 0; e < E; e++) p[e] = w[e] != PAIR_LOOP ? sid[w[e] & ~PAIR_DIR] : -1;
        uint32_t c[E];
#pragma unroll
        for (int e = 0; e < E; e++)
            c[e] = (unsigned)p[e] < (unsigned)S ? 2 * (uint32_t)p[e] + (w[e] >> 31) : 2 * (uint32_t)S;
        int loops = 0;
#pragma unroll
        for (int e = 0; e < E; e++) {
            if (c[e] >= 2 * (uint32_t)S) {
                loops += j0 + e < m;
                continue;
            }
            if (e > 0 && c[e - 1] == c[e]) continue;
            int run = 1;
#pragma unroll
            for (int f = e + 1; f < E; f++)
                if (f == e + run && c[f] == c[e]) run++;
            atomicAdd(&cnt[c[e]], run);
        }
        const unsigned am = __activemask();
        loops = __reduce_add_sync(am, loops);
        if (loops && (threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(&cnt[2 * (int64_t)S], loops);
        if (full) {
#pragma unroll
            for (int h = 0; h < E / 4; h++)
                __stcs(reinterpret_cast<uint4*>(cw + j0) + h, make_uint4(c[4 * h], c[4 * h + 1], c[4 * h + 2], c[4 * h + 3]));
        } else {
            for (int e = 0; e < E && j0 + e < m; e++) cw[j0 + e] = c[e];
        }
    }
}

// hist[p][b] (zeroed) = number of edges whose sort id has 8-bit digit p equal to b, for
// the sort's passes digits: from the per-id counts cnt[0..2S], one weighted addition per
// id rather than one per edge.
__global__ void __launch_bounds__(256) k_store_hist(const int32_t* __restrict__ cnt, int32_t S, int passes,
                                                    uint32_t* __restrict__ hist) {
    constexpr int B = 1 << STORE_DIGIT_BITS;
    __shared__ uint32_t h[STORE_MAX_PASSES][B];
    for (int i = threadIdx.x; i < STORE_MAX_PASSES * B; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t nc = 2 * (int64_t)S + 1;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)cnt[c];
        if (v == 0) continue;
        for (int p = 0; p < passes; p++) atomicAdd(&h[p][((uint32_t)c >> (STORE_DIGIT_BITS * p)) & (B - 1)], v);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * B; i += blockDim.x) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// sigma[p] = number of temporal edges of static edge p, from the runs' starts.
__global__ void k_store_sigma(const int32_t* __restrict__ seg, int32_t S, int32_t* __restrict__ sigma) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < S; p += (int64_t)gridDim.x * blockDim.x)
        sigma[p] = seg[2 * p + 2] - seg[2 * p];
}

// The run starts of sorted position i with word pk (its predecessor's word prev, ~0 for
// i = 0): seg[2s] = i where static edge s begins, seg[2s + 1] = i where its b -> a run
// begins (seg is all -1 before; k_segments_fix fills the b -> a starts of edges without
// one). c < 2S unless the pair ids' sort failed, which the host learns right after.
__device__ __forceinline__ void pair_run_starts(uint64_t pk, uint64_t prev, int ib, int32_t S, int64_t i,
                                                int32_t* __restrict__ seg) {
    const int32_t c = (int32_t)(pk >> ib);
    if ((unsigned)c >= (unsigned)(2 * S)) return;
    if ((prev >> (ib + 1)) != (uint64_t)(c >> 1)) seg[c & ~1] = (int32_t)i;
    if ((c & 1) && (prev >> ib) != (uint64_t)c) seg[c] = (int32_t)i;
}

// perm, T, sd and the run starts from the sorted words: position i holds time rank
// j = word mod 2^ib (input index order[j], or j) of pair id and direction word >> ib.
// SORTED: t holds the timestamps in sorted order already (the sort's values); otherwise
// they are gathered from the input order.
template <typename TS, bool SORTED>
__global__ void k_pair_store(const uint64_t* __restrict__ packed, const uint32_t* __restrict__ order, int64_t mk,
                             int32_t S, int ib, const TS* __restrict__ t, int32_t* __restrict__ perm,
                             TS* __restrict__ T, int32_t* __restrict__ sd, int32_t* __restrict__ seg) {
    const uint64_t jm = (1ull << ib) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t pk = __ldcs(packed + i);
        const int64_t j = (int64_t)(pk & jm);
        const uint32_t o = order ? order[j] : (uint32_t)j;
        __stcs(perm + i, (int32_t)o);
        T[i] = SORTED ? __ldcs(t + i) : t[o];
        __stcs(sd + i, (int32_t)(pk >> ib));
        pair_run_starts(pk, i > 0 ? packed[i - 1] : ~0ull, ib, S, i, seg);
    }
}

// The same for a 32-bit store whose timestamps came sorted with the words, four
// positions per thread with 16-byte loads and stores (the last quad may be partial).
__global__ void k_pair_store4(const uint64_t* __restrict__ packed, const uint32_t* __restrict__ order, int64_t mk,
                              int32_t S, int ib, const uint32_t* __restrict__ ts, int32_t* __restrict__ perm,
                              uint32_t* __restrict__ T, int32_t* __restrict__ sd, int32_t* __restrict__ seg) {
    const uint64_t jm = (1ull << ib) - 1;
    const int64_t nq = (mk + 3) >> 2;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = q << 2;
        const bool full = i0 + 4 <= mk;
        uint64_t pk[4];
        uint32_t tv[4];
        if (full) {
            const ulonglong2 a = __ldcs(reinterpret_cast<const ulonglong2*>(packed + i0));
            const ulonglong2 b = __ldcs(reinterpret_cast<const ulonglong2*>(packed + i0 + 2));
            const uint4 tt = __ldcs(reinterpret_cast<const uint4*>(ts + i0));
            pk[0] = a.x;
            pk[1] = a.y;
            pk[2] = b.x;
            pk[3] = b.y;
            tv[0] = tt.x;
            tv[1] = tt.y;
            tv[2] = tt.z;
            tv[3] = tt.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                pk[e] = i0 + e < mk ? packed[i0 + e] : 0;
                tv[e] = i0 + e < mk ? ts[i0 + e] : 0;
            }
        }
        int32_t o[4], c[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int64_t j = (int64_t)(pk[e] & jm);
            o[e] = order ? (int32_t)order[j] : (int32_t)j;
            c[e] = (int32_t)(pk[e] >> ib);
        }
        uint64_t prev = i0 > 0 ? packed[i0 - 1] : ~0ull;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (i0 + e < mk) pair_run_starts(pk[e], prev, ib, S, i0 + e, seg);
            prev = pk[e];
        }
        if (full) {
            __stcs(reinterpret_cast<int4*>(perm + i0), make_int4(o[0], o[1], o[2], o[3]));
            __stcs(reinterpret_cast<uint4*>(T + i0), make_uint4(tv[0], tv[1], tv[2], tv[3]));
            __stcs(reinterpret_cast<int4*>(sd + i0), make_int4(c[0], c[1], c[2], c[3]));
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (i0 + e < mk) {
                    perm[i0 + e] = o[e];
                    T[i0 + e] = tv[e];
                    sd[i0 + e] = c[e];
                }
            }
        }
    }
}

// seg[2s+1] = first b->a position of s (the full-key path, whose k_segments marks every
// b->a start -1 first).
__global__ void k_segments_split(const int32_t* __restrict__ sd, int64_t mk, int32_t S,
                                 int32_t* __restrict__ seg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = sd[i];
        if ((c & 1) && (unsigned)c < (unsigned)(2 * S) && (i == 0 || sd[i - 1] != c)) seg[c] = (int32_t)i;  // c = 2s+1
    }
}

// seg[2s+1] = the end of s when it has no b->a run.
__global__ void k_segments_fix(int32_t S, int64_t mk, int32_t* __restrict__ seg) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (seg[2 * s + 1] < 0) seg[2 * s + 1] = (s + 1 < S) ? seg[2 * s + 2] : (int32_t)mk;
        if (s == 0) seg[2 * S] = (int32_t)mk;
    }
}

// ================================================================== A2

// Runs of equal values in a sorted id array: first[x] = start index, last[x] = end
// index (exclusive) of the run of x. Ids absent from the array keep first = last = 0.
__global__ void k_runs(const int32_t* __restrict__ ids, const uint32_t* __restrict__ order, int32_t S,
                       int32_t* __restrict__ first, int32_t* __restrict__ last) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = order ? ids[order[j]] : ids[j];
        if (j == 0 || (order ? ids[order[j - 1]] : ids[j - 1]) != x) first[x] = (int32_t)j;
        if (j == S - 1 || (order ? ids[order[j + 1]] : ids[j + 1]) != x) last[x] = (int32_t)j + 1;
    }
}

// deg_hi = #static edges (u, b > u), deg_lo = #static edges (a < u, u), deg = sum.
__global__ void k_degrees(const int32_t* __restrict__ hi_first, const int32_t* __restrict__ hi_last,
                          const int32_t* __restrict__ lo_first, const int32_t* __restrict__ lo_last, int64_t n,
                          int32_t* __restrict__ deg_lo, int32_t* __restrict__ deg) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int32_t dl = lo_last[u] - lo_first[u];
        deg_lo[u] = dl;
        deg[u] = dl + (hi_last[u] - hi_first[u]);
    }
}

__global__ void k_edge_keys_b(const int32_t* __restrict__ eb, int32_t S, uint64_t* __restrict__ key,
                              uint32_t* __restrict__ val) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        key[s] = (uint64_t)eb[s];
        val[s] = (uint32_t)s;
    }
}

// Row u = [neighbours a < u (edges with b = u, ascending a)] [neighbours b > u].
__global__ void k_fill_adj(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb, int32_t S,
                           const int32_t* __restrict__ rowptr, const int32_t* __restrict__ deg_lo,
                           const int32_t* __restrict__ hi_start, const int32_t* __restrict__ lo_start,
                           const uint32_t* __restrict__ by_b, int32_t* __restrict__ adj,
                           int32_t* __restrict__ adj_eid, int32_t* __restrict__ adj_src) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S;
         j += (int64_t)gridDim.x * blockDim.x) {
        // upper part: static edges are sorted by (a, b)
        int32_t s = (int32_t)j;
        int32_t a = ea[s];
        int64_t p = (int64_t)rowptr[a] + deg_lo[a] + (s - hi_start[a]);
        adj[p] = eb[s];
        adj_eid[p] = s;
        adj_src[p] = a;
        // lower part: by_b lists static edges by (b, a)
        int32_t s2 = (int32_t)by_b[j];
        int32_t b = eb[s2];
        int64_t q = (int64_t)rowptr[b] + ((int32_t)j - lo_start[b]);
        adj[q] = ea[s2];
        adj_eid[q] = s2;
        adj_src[q] = b;
    }
}

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t n, int* __restrict__ out) {
    int best = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        best = max(best, a[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// osig[j] = temporal edges (both directions) of the static edge at out-list position j,
// and their maximum: the probe slots a triangle adds per edge, read by the triangle
// passes next to the out-list entries themselves. From the per-pair counts sigma when
// given, else from the run bounds.
__global__ void k_out_sigma(const int32_t* __restrict__ sigma, const int32_t* __restrict__ seg,
                            const int32_t* __restrict__ out_eid, int32_t S, int32_t* __restrict__ osig,
                            int* __restrict__ out) {
    int best = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = out_eid[j];
        const int32_t c = sigma ? sigma[e] : seg[2 * e + 2] - seg[2 * e];
        osig[j] = c;
        best = max(best, c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// ================================================================== A3

enum {
    C_BAR = 0,
    C_GEN = 1,
    C_ERR = 2,
    C_ACNT = 3,   // 2 slots
    C_MIN = 5,    // 2 slots
    C_FCNT = 7,   // 3 slots: light frontier sizes
    C_HCNT = 10,  // 3 slots: heavy frontier sizes
    C_ROUNDS = 13,
    C_ALPHA = 14,
    C_TAIL = 15,    // 1 when the grid kernel stopped early for the single-block tail
    C_TAIL_K = 16,  // state handed to the tail: level, round, alive buffer, alive count
    C_TAIL_R = 17,
    C_TAIL_AC = 18,
    C_TAIL_N = 19,
    C_RM = 20,  // 2 slots by level parity: vertices removed after the level's compaction
    C_SOLO = 22,    // 1 when the cluster tail stopped early for the single-CTA phase
    C_SOLO_K = 23,  // level and round handed to the single-CTA phase
    C_SOLO_R = 24,
    C_SLOTS = 28
};

struct PeelArgs {
    const int32_t* rowptr;
    const int32_t* adj;
    int32_t n;
    int32_t* deg;   // working copy of the degrees
    int32_t* rnd;   // removal round, -1 while alive
    int32_t* core;  // core number
    int32_t* alive[2];
    int32_t* fr[2];  // light frontier (degree <= PEEL_HEAVY): one warp per vertex
    int64_t* hr[2];  // heavy frontier as (vertex, piece) entries: piece << 32 | vertex
    int32_t hcap;    // capacity of hr[0], hr[1]: n + 2S / PEEL_PIECE + 1
    int* ctl;
    long long timeout_ns;
    int32_t tail_n;  // stop when at most this many vertices may still be alive
};

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident). The wait is
// bounded: after timeout_ns the block records an error and every block returns.
__device__ bool grid_barrier(int* ctl, long long timeout_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* vgen = (volatile int*)&ctl[C_GEN];
        volatile int* verr = (volatile int*)&ctl[C_ERR];
        int gen = *vgen;
        __threadfence();
        int arrived = atomicAdd(&ctl[C_BAR], 1);
        if (arrived == (int)gridDim.x - 1) {
            atomicExch(&ctl[C_BAR], 0);
            __threadfence();
            atomicAdd(&ctl[C_GEN], 1);
        } else {
            long long t0 = global_ns();
            while (*vgen == gen) {
                if (*verr) break;
                if (global_ns() - t0 > timeout_ns) {
                    atomicExch(&ctl[C_ERR], 1);
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)&ctl[C_ERR] == 0;
}

// Appends v for every lane with pred set; the whole warp must call it. A list never
// holds more than cap entries (each vertex joins at most one frontier and one alive
// list); an append beyond cap is dropped and recorded in *err instead of written.
__device__ __forceinline__ void warp_append(bool pred, int32_t v, int32_t* out, int* counter, int cap,
                                            int* err) {
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (!mask) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) {
        int idx = base + __popc(mask & ((1u << lane) - 1u));
        if (idx < cap) out[idx] = v;
        else atomicExch(err, 2);
    }
}

// Adds the number of lanes with pred set to *counter (one atomic per warp). The whole
// warp must call it.
__device__ __forceinline__ void warp_count(bool pred, int* counter) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (m && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(counter, __popc(m));
}

constexpr int PEEL_THREADS = 1024;
constexpr int PEEL_SHORT = 32;      // rows up to this length are walked by one thread,
constexpr int PEEL_CHUNK = 8;       // PEEL_CHUNK entries at a time
constexpr int PEEL_HEAVY = 128;     // vertices above this degree go to the heavy frontier
constexpr int PEEL_PIECE = PEEL_THREADS;  // adjacency entries per heavy piece
constexpr int PEEL_BUF = 4096;            // entries of each block-local append buffer

// Block-local staging of list appends: warps append into shared memory (one shared-memory
// atomic per warp) and peel_flush moves a phase's entries to the global list with one
// global atomic per block, instead of one contended global atomic per warp. Entries
// beyond PEEL_BUF go to the global list directly.
struct PeelBuf {
    int32_t* fr;  // light-frontier entries
    int32_t* al;  // alive-list entries
    int* n;       // n[0], n[1]: entries staged in fr, al; n[2]: removals counted; n[3], n[4]: bases
};

// Appends v for every lane with pred set to the block's buffer sbuf (count *scnt), or past
// its capacity to the global list (out, counter, cap). The whole warp must call it.
__device__ __forceinline__ void buf_append(bool pred, int32_t v, int32_t* sbuf, int* scnt, int32_t* out,
                                           int* counter, int cap, int* err) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(scnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    const int idx = base + __popc(m & ((1u << lane) - 1u));
    if (pred && idx < PEEL_BUF) sbuf[idx] = v;
    warp_append(pred && idx >= PEEL_BUF, v, out, counter, cap, err);
}

// Moves the block's staged entries to the global lists and its removal count to rm_cnt
// (null when the phase counts none); every thread of the block calls it after its last
// append of the phase. A list never holds more than cap entries: an entry beyond is
// dropped and recorded in *err.
__device__ __forceinline__ void peel_flush(PeelBuf pb, int32_t* fr_out, int* fr_cnt, int32_t* al_out, int* al_cnt,
                                           int* rm_cnt, int cap, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nf = min(pb.n[0], PEEL_BUF), na = min(pb.n[1], PEEL_BUF);
        pb.n[3] = nf ? atomicAdd(fr_cnt, nf) : 0;
        pb.n[4] = na ? atomicAdd(al_cnt, na) : 0;
        if (pb.n[2]) atomicAdd(rm_cnt, pb.n[2]);
    }
    __syncthreads();
    const int nf = min(pb.n[0], PEEL_BUF), na = min(pb.n[1], PEEL_BUF);
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const int idx = pb.n[3] + i;
        if (idx < cap) fr_out[idx] = pb.fr[i];
        else atomicExch(err, 2);
    }
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        const int idx = pb.n[4] + i;
        if (idx < cap) al_out[idx] = pb.al[i];
        else atomicExch(err, 2);
    }
    __syncthreads();
    if (threadIdx.x == 0) pb.n[0] = pb.n[1] = pb.n[2] = 0;
}

// Files vertex v (removed at round rr) in the frontier of round rr: light vertices as
// themselves (staged in the block's buffer), heavy ones as their PEEL_PIECE-entry pieces
// of adjacency. The whole warp must call it; b, e = v's row bounds.
__device__ __forceinline__ void frontier_append(const PeelArgs& a, const PeelBuf& pb, bool in, int32_t v, int32_t b,
                                                int32_t e, int rr) {
    const bool heavy = in && (e - b > PEEL_HEAVY);
    buf_append(in && !heavy, v, pb.fr, &pb.n[0], (rr & 1) ? a.fr[1] : a.fr[0], &a.ctl[C_FCNT + rr % 3], a.n,
               &a.ctl[C_ERR]);
    if (heavy) {
        const int np = (e - b + PEEL_PIECE - 1) / PEEL_PIECE;
        const int base = atomicAdd(&a.ctl[C_HCNT + rr % 3], np);
        if (base + np <= a.hcap) {
            int64_t* hr = (rr & 1) ? a.hr[1] : a.hr[0];
            for (int q = 0; q < np; q++) hr[base + q] = ((int64_t)q << 32) | (uint32_t)v;
        } else {
            atomicExch(&a.ctl[C_ERR], 2);
        }
    }
}

// Neighbour j of a vertex leaving in round r: its degree drops, and a vertex whose degree
// crosses k + 1 -> k joins round r + 1. A vertex that already left never crosses again
// (its degree was <= k when it left and only falls), so no liveness test is needed.
// The whole warp must call it.
__device__ __forceinline__ void peel_neighbour(const PeelArgs& a, const PeelBuf& pb, bool valid, int32_t j, int k,
                                               int r) {
    bool cross = false;
    int32_t v = 0, b = 0, e = 0;
    if (valid) {
        v = a.adj[j];
        int old = atomicSub(&a.deg[v], 1);
        if (old == k + 1) {
            cross = true;
            a.rnd[v] = r + 1;
            a.core[v] = k;
            b = a.rowptr[v];
            e = a.rowptr[v + 1];
        }
    }
    warp_count(cross, &pb.n[2]);
    frontier_append(a, pb, cross, v, b, e, r + 1);
}

// Vertex v (valid when cross) crossed k + 1 -> k in round r: it leaves in round r + 1.
// The whole warp must call it.
__device__ __forceinline__ void peel_crossing(const PeelArgs& a, const PeelBuf& pb, bool cross, int32_t v, int k,
                                              int r) {
    warp_count(cross, &pb.n[2]);
    int32_t rb = 0, re = 0;
    if (cross) {
        a.rnd[v] = r + 1;
        a.core[v] = k;
        rb = a.rowptr[v];
        re = a.rowptr[v + 1];
    }
    frontier_append(a, pb, cross, v, rb, re, r + 1);
}

// Parallel Matula-Beck peeling. Level k = smallest remaining degree; within a level,
// round after round, every remaining vertex of current degree <= k is removed at once
// and its neighbours' degrees drop. A vertex enters the next round exactly when its
// degree crosses k + 1 -> k. Each vertex gets core = k and the round it left in.
//
// One block per SM; every phase ends with one grid barrier. A level starts with one
// phase that compacts the alive list and, at the same time, takes the vertices of
// degree <= k + 1 as the next frontier (levels are usually consecutive); only when that
// frontier is empty does a second phase jump to the minimum degree. A round hands light
// frontier vertices to single warps; heavy ones (hubs) are filed as PEEL_PIECE-entry
// pieces of their adjacency, one block per piece, so no warp walks a hub alone.
//
// Counter discipline: a phase only appends to counters that no block reads before the
// phase's closing barrier, and only reads counters completed before its opening
// barrier. Frontier counters rotate over three slots by round number; every new
// frontier (level start, jump, next round) is filed under round r + 1, so the slot a
// slow block may still be reading (round r) is never written in the same phase.
__global__ void __launch_bounds__(PEEL_THREADS, 1) k_peel(PeelArgs a) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = gtid >> 5, nwarps = gsize >> 5;
    int* ctl = a.ctl;
    __shared__ int s_wmin[PEEL_THREADS / 32];
    __shared__ int32_t s_fr[PEEL_BUF], s_al[PEEL_BUF];
    __shared__ int s_n[5];
    const PeelBuf pb{s_fr, s_al, s_n};
    if (threadIdx.x < 5) s_n[threadIdx.x] = 0;
    __syncthreads();
    int k = -1, r = 0, lvl = 0, ac = 0, rounds = 0;
    int nalive = a.n;
    while (true) {
        // few vertices left: hand the rest to the cluster tail (all blocks agree: nalive
        // and the removals since the last compaction were read after the same barrier)
        const int removed = lvl > 0 ? *(volatile int*)&ctl[C_RM + ((lvl - 1) & 1)] : 0;
        if (nalive - removed <= a.tail_n) {
            if (gtid == 0) {
                ctl[C_TAIL] = 1;
                ctl[C_TAIL_K] = k;
                ctl[C_TAIL_R] = r;
                ctl[C_TAIL_AC] = ac;
                ctl[C_TAIL_N] = nalive;
                ctl[C_ROUNDS] = rounds;
            }
            return;
        }
        // ---- level start: compaction + frontier at k + 1, filed as round r + 1
        const int kk = k + 1;
        if (gtid == 0) {
            ctl[C_MIN + ((lvl + 1) & 1)] = INT_MAX;
            ctl[C_ACNT + ((lvl + 1) & 1)] = 0;
            ctl[C_RM + (lvl & 1)] = 0;
            ctl[C_FCNT + (r + 2) % 3] = 0;
            ctl[C_HCNT + (r + 2) % 3] = 0;
        }
        int lmin = INT_MAX;
        {
            const int32_t* acur = ac ? a.alive[1] : a.alive[0];
            int32_t* anxt = ac ? a.alive[0] : a.alive[1];
            for (int64_t base = gwarp * 32; base < nalive; base += nwarps * 32) {
                int64_t i = base + lane;
                bool keep = false, in = false;
                int32_t v = 0;
                int32_t rb = 0, re = 0;
                if (i < nalive) {
                    v = __ldcg(&acur[i]);
                    const int rv = __ldcg(&a.rnd[v]);
                    const int d = __ldcg(&a.deg[v]);
                    rb = a.rowptr[v];
                    re = a.rowptr[v + 1];
                    if (rv < 0) {
                        if (d <= kk) {
                            in = true;
                            a.rnd[v] = r + 1;
                            a.core[v] = kk;
                        } else {
                            keep = true;
                            lmin = min(lmin, d);
                        }
                    }
                }
                frontier_append(a, pb, in, v, rb, re, r + 1);
                buf_append(keep, v, pb.al, &pb.n[1], anxt, &ctl[C_ACNT + (lvl & 1)], a.n, &ctl[C_ERR]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
        if (lane == 0) s_wmin[threadIdx.x >> 5] = lmin;
        __syncthreads();
        if (threadIdx.x == 0) {
            int bm = INT_MAX;
            for (int w = 0; w < PEEL_THREADS / 32; w++) bm = min(bm, s_wmin[w]);
            if (bm != INT_MAX) atomicMin(&ctl[C_MIN + (lvl & 1)], bm);
        }
        peel_flush(pb, ((r + 1) & 1) ? a.fr[1] : a.fr[0], &ctl[C_FCNT + (r + 1) % 3], ac ? a.alive[0] : a.alive[1],
                   &ctl[C_ACNT + (lvl & 1)], nullptr, a.n, &ctl[C_ERR]);
        if (!grid_barrier(ctl, a.timeout_ns)) return;
        r += 1;
        ac ^= 1;
        nalive = *(volatile int*)&ctl[C_ACNT + (lvl & 1)];
        const int fs = *(volatile int*)&ctl[C_FCNT + r % 3] + *(volatile int*)&ctl[C_HCNT + r % 3];
        if (fs == 0) {
            if (nalive == 0) break;
            // no vertex of degree k + 1: jump to the smallest remaining degree, round r + 1
            const int kj = *(volatile int*)&ctl[C_MIN + (lvl & 1)];
            const int32_t* al = ac ? a.alive[1] : a.alive[0];
            for (int64_t base = gwarp * 32; base < nalive; base += nwarps * 32) {
                int64_t i = base + lane;
                bool in = false;
                int32_t v = 0;
                int32_t rb = 0, re = 0;
                if (i < nalive) {
                    v = __ldcg(&al[i]);
                    const int d = __ldcg(&a.deg[v]);
                    rb = a.rowptr[v];
                    re = a.rowptr[v + 1];
                    if (d <= kj) {
                        in = true;
                        a.rnd[v] = r + 1;
                        a.core[v] = kj;
                    }
                }
                warp_count(in, &pb.n[2]);
                frontier_append(a, pb, in, v, rb, re, r + 1);
            }
            k = kj;
            peel_flush(pb, ((r + 1) & 1) ? a.fr[1] : a.fr[0], &ctl[C_FCNT + (r + 1) % 3], nullptr, nullptr,
                       &ctl[C_RM + (lvl & 1)], a.n, &ctl[C_ERR]);
            if (!grid_barrier(ctl, a.timeout_ns)) return;
            r += 1;
        } else {
            k = kk;
        }
        // ---- rounds at level k (the first one has a non-empty frontier)
        while (true) {
            const int fsz = *(volatile int*)&ctl[C_FCNT + r % 3];
            const int hsz = *(volatile int*)&ctl[C_HCNT + r % 3];
            if (fsz + hsz == 0) break;
            if (gtid == 0) {
                ctl[C_FCNT + (r + 2) % 3] = 0;
                ctl[C_HCNT + (r + 2) % 3] = 0;
            }
            // light vertices: a row of at most PEEL_SHORT entries is walked by one thread,
            // PEEL_CHUNK entries at a time, a longer one (up to PEEL_HEAVY) by the whole warp
            // in turn; every load of a chunk is issued, then every decrement, before a result
            // is used
            const int32_t* F = (r & 1) ? a.fr[1] : a.fr[0];
            for (int64_t i0 = gwarp * 32; i0 < fsz; i0 += nwarps * 32) {
                const int64_t i = i0 + lane;
                const bool have = i < fsz;
                const int32_t u = have ? __ldcg(&F[i]) : 0;
                const int32_t b = have ? a.rowptr[u] : 0, e = have ? a.rowptr[u + 1] : 0;
                const bool shortrow = have && e - b <= PEEL_SHORT;
                const int chunks = __reduce_max_sync(0xffffffffu, shortrow ? (e - b + PEEL_CHUNK - 1) / PEEL_CHUNK : 0);
                for (int c = 0; c < chunks; c++) {  // warp-uniform trip count
                    const int32_t j0 = b + c * PEEL_CHUNK;
                    int32_t v[PEEL_CHUNK];
                    int old[PEEL_CHUNK];
#pragma unroll
                    for (int t = 0; t < PEEL_CHUNK; t++) v[t] = (shortrow && j0 + t < e) ? a.adj[j0 + t] : -1;
#pragma unroll
                    for (int t = 0; t < PEEL_CHUNK; t++) old[t] = (v[t] >= 0) ? atomicSub(&a.deg[v[t]], 1) : 0;
#pragma unroll
                    for (int t = 0; t < PEEL_CHUNK; t++)
                        peel_crossing(a, pb, v[t] >= 0 && old[t] == k + 1, v[t], k, r);
                }
                unsigned mm = __ballot_sync(0xffffffffu, have && !shortrow);
                while (mm) {
                    const int src = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const int32_t bb = __shfl_sync(0xffffffffu, b, src), ee = __shfl_sync(0xffffffffu, e, src);
                    constexpr int Q = PEEL_HEAVY / 32;
                    int32_t v[Q];
                    int old[Q];
#pragma unroll
                    for (int q = 0; q < Q; q++) {
                        const int32_t j = bb + q * 32 + lane;
                        v[q] = (j < ee) ? a.adj[j] : -1;
                    }
#pragma unroll
                    for (int q = 0; q < Q; q++) old[q] = (v[q] >= 0) ? atomicSub(&a.deg[v[q]], 1) : 0;
#pragma unroll
                    for (int q = 0; q < Q; q++) peel_crossing(a, pb, v[q] >= 0 && old[q] == k + 1, v[q], k, r);
                }
            }
            // heavy vertices: one block per piece of PEEL_PIECE adjacency entries
            const int64_t* H = (r & 1) ? a.hr[1] : a.hr[0];
            for (int pc = blockIdx.x; pc < hsz; pc += gridDim.x) {
                const int64_t hp = __ldcg(&H[pc]);
                const int32_t u = (int32_t)(hp & 0xffffffffll);
                const int32_t q = (int32_t)(hp >> 32);
                const int32_t j = a.rowptr[u] + q * PEEL_PIECE + (int32_t)threadIdx.x;
                peel_neighbour(a, pb, j < a.rowptr[u + 1], j, k, r);
            }
            peel_flush(pb, ((r + 1) & 1) ? a.fr[1] : a.fr[0], &ctl[C_FCNT + (r + 1) % 3], nullptr, nullptr,
                       &ctl[C_RM + (lvl & 1)], a.n, &ctl[C_ERR]);
            if (!grid_barrier(ctl, a.timeout_ns)) return;
            r++;
            rounds++;
        }
        lvl++;
    }
    if (gtid == 0) {
        ctl[C_ROUNDS] = rounds;
        ctl[C_ALPHA] = k;
    }
}

// ================================================================== A3 tail

// The last levels run on one thread-block cluster, on the subgraph induced by the vertices
// still alive, renumbered 0..NL-1 ("local" ids): degrees, row bounds and frontiers live
// in the CTAs' shared memory (each CTA owns the local ids congruent to its rank) and a
// round ends with one cluster barrier instead of a grid barrier.
constexpr int TAIL_THREADS = 1024;
constexpr int SOLO_DEG_CAP = 1 << 18;  // degree sum (remaining decrements) the single CTA takes over
constexpr int TAIL_OWN = 10240;  // local vertices owned per CTA: a C-CTA tail takes up to 10240 C

// Local ids for the vertices of the grid kernel's alive list that are still alive (at
// most cap; more would be an internal error, recorded in *err instead of written).
// Nothing to do when the grid kernel finished the peeling itself (ctl[C_TAIL] == 0).
__global__ void k_tail_select(const int32_t* __restrict__ alive0, const int32_t* __restrict__ alive1,
                              const int* __restrict__ ctl, const int32_t* __restrict__ rnd, int cap,
                              int32_t* __restrict__ L, int32_t* __restrict__ gmap, int* __restrict__ nl,
                              int* __restrict__ err) {
    if (ctl[C_TAIL] != 1) return;
    const int nalive = ctl[C_TAIL_N];
    const int32_t* __restrict__ alive = ctl[C_TAIL_AC] ? alive1 : alive0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalive;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = alive[i];
        if (rnd[v] < 0) {
            int li = atomicAdd(nl, 1);
            if (li < cap) {
                L[li] = v;
                gmap[v] = li;
            } else {
                atomicExch(err, 2);
            }
        }
    }
}

// Local degree (alive neighbours = current degree) and full row length per local id.
__global__ void k_tail_degrees(const int32_t* __restrict__ L, const int* __restrict__ nl,
                               const int32_t* __restrict__ deg, const int32_t* __restrict__ rowptr, int tn,
                               int32_t* __restrict__ ld, int32_t* __restrict__ d0) {
    const int n = *nl;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tn; i += gridDim.x * blockDim.x) {
        if (i < n) {
            int32_t v = L[i];
            ld[i] = deg[v];
            d0[i] = rowptr[v + 1] - rowptr[v];
        } else {
            ld[i] = 0;
            d0[i] = 0;
        }
    }
}

// Entry e of the concatenated full rows of the local vertices (eoff = prefix of d0):
// alive neighbours go to the owner's local row (order within a row is irrelevant).
constexpr int FILL_RUN = 8;  // consecutive entries per thread in the subgraph fills

__global__ void k_tail_fill(const int32_t* __restrict__ L, const int32_t* __restrict__ eoff, int tn,
                            const int32_t* __restrict__ rowptr, const int32_t* __restrict__ adj,
                            const int32_t* __restrict__ rnd, const int32_t* __restrict__ gmap,
                            const int32_t* __restrict__ lrow, const int32_t* __restrict__ ld,
                            int32_t* __restrict__ fillc, uint32_t* __restrict__ ladj, int* __restrict__ err) {
    const int64_t total = eoff[tn];
    // a thread takes FILL_RUN consecutive entries: one search for the first one's owner,
    // then the owner moves forward (rows average a few entries), and the alive entries of
    // each owner's part of the run take their places with one atomic (a hub's counter
    // would serialise one atomic per entry)
    const int64_t step = (int64_t)gridDim.x * blockDim.x * FILL_RUN;
    for (int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * FILL_RUN; e0 < total; e0 += step) {
        int lo = 0, hi = tn - 1;  // last owner with eoff[owner] <= e0
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (eoff[mid] <= e0) lo = mid;
            else hi = mid - 1;
        }
        const int64_t e1 = min(e0 + FILL_RUN, total);
        int64_t e = e0;
        while (e < e1) {
            while (lo + 1 < tn && eoff[lo + 1] <= e) lo++;
            const int64_t end = (lo + 1 < tn) ? min(e1, (int64_t)eoff[lo + 1]) : e1;  // this owner's part
            uint32_t keep[FILL_RUN];
            int nk = 0;
            const int32_t rb = rowptr[L[lo]];
            for (; e < end; e++) {
                const int32_t v = adj[rb + (int32_t)(e - eoff[lo])];
                if (rnd[v] < 0) keep[nk++] = (uint32_t)gmap[v];
            }
            if (nk) {
                const int p = atomicAdd(&fillc[lo], nk);
                if (p + nk <= ld[lo]) {
                    for (int q = 0; q < nk; q++) ladj[lrow[lo] + p + q] = keep[q];
                } else {
                    atomicExch(err, 3);  // more alive neighbours than the degree says
                }
            }
        }
    }
}

struct TailArgs {
    const int* nl;
    const int32_t* L;
    const int32_t* ld;
    const int32_t* lrow;
    const uint32_t* ladj;
    int32_t* rnd;
    int32_t* core;
    int* ctl;
    // hand-off to the single-CTA phase once at most solo_cap vertices are left: their
    // local ids (slist), current degrees (sdeg), and map2[local id] = position in slist
    int solo_cap;
    int* ns;
    int32_t* slist;
    int32_t* sdeg;
    int32_t* map2;
    // decrements of a heavy round, by owner and slot (owner * TAIL_OWN + slot), zero
    // between rounds
    int32_t* dec;
};

constexpr int TAIL_AGG_MIN = 128;  // frontier size from which a round's decrements go through L2
constexpr int TAIL_SHORT = 32;   // rows up to this length: one thread, TAIL_CHUNK loads at a time
constexpr int TAIL_CHUNK = 8;
constexpr int TAIL_LIGHT = 256;  // rows up to this length: one warp, all loads in flight at once
constexpr int TAIL_HCAP = 512;   // heavy vertices per CTA and round (more wait for the next pass)

// Shared memory of one tail CTA of a C-CTA cluster. Local vertex v is owned by CTA v % C
// at slot q = v / C; the owner keeps its degree, row bounds and global id, and the
// frontier lists hold owned slots: a thread that drives a vertex's degree across k + 1 -> k
// files it directly in the owner's next frontier through distributed shared memory.
template <int C>
struct TailShared {
    static constexpr int OWN = TAIL_OWN;
    int32_t odeg[OWN];
    int32_t orb[OWN], ore[OWN];  // row [orb, ore) of ladj
    int32_t oL[OWN];             // global id
    uint16_t FL[2][OWN];         // frontier by round parity (owned slots)
    uint16_t FH[TAIL_HCAP];      // heavy rows of the current round
    int cntL[3], cntH[2], smin[2];
    int acnt[2];                 // owned vertices alive at the level start, by level parity
    int adeg[2];                 // their degree sum (twice the edges left), by level parity
    int made[2];                 // crossings this CTA filed (anywhere) in a round, by round parity
    int slots[2][C][4];          // every CTA's values of one cluster barrier, by barrier parity
};

// Neighbours vv[0..N) (negative: none) lose one degree each in round r at level k: all N
// decrements are issued before any result is used, then every k + 1 -> k crossing files
// its vertex in the owner's frontier of round r + 1.
template <int C, int N>
__device__ __forceinline__ void tail_decrement(TailShared<C>& sh, cg::cluster_group& cl, const int (&vv)[N], int k,
                                               int r, int32_t* __restrict__ dec) {
    if (dec) {
        // a heavy round: many frontier rows share their targets, and one shared-memory
        // atomic of the target's owner per decrement would queue at that SM; the
        // decrements add up in L2 instead, and each owner applies its own after the
        // round's barrier
#pragma unroll
        for (int t = 0; t < N; t++)
            if (vv[t] >= 0) atomicAdd(&dec[(vv[t] % C) * TAIL_OWN + vv[t] / C], 1);
        return;
    }
    int old[N];
#pragma unroll
    for (int t = 0; t < N; t++)
        old[t] = (vv[t] >= 0) ? atomicSub(&cl.map_shared_rank(sh.odeg, vv[t] % C)[vv[t] / C], 1) : 0;
#pragma unroll
    for (int t = 0; t < N; t++) {
        if (vv[t] >= 0 && old[t] == k + 1) {
            TailShared<C>* p = cl.map_shared_rank(&sh, vv[t] % C);
            const int at = atomicAdd(&p->cntL[(r + 1) % 3], 1);
            p->FL[(r + 1) & 1][at] = (uint16_t)(vv[t] / C);
            atomicAdd(&sh.made[r & 1], 1);
        }
    }
}

// Publishes this CTA's values v of the next cluster barrier (number s) in every CTA's
// slot s & 1 (threads 0..C-1 each write one CTA's copy); after the barrier, tail_totals
// combines the C copies from this CTA's own shared memory, without a remote read after
// the barrier. A slot is rewritten two barriers later, after every CTA has read it. The
// values must be final (the caller's __syncthreads) before the call.
template <int C>
__device__ __forceinline__ void tail_publish(TailShared<C>& sh, cg::cluster_group& cl, int s, int4 v) {
    if (threadIdx.x < C) {
        TailShared<C>* q = cl.map_shared_rank(&sh, (int)threadIdx.x);
        int* d = q->slots[s & 1][cl.block_rank()];
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    }
}

// After the barrier: the sums of the C copies' x, z, w and the minimum of their y (each
// warp reduces them for itself).
template <int C>
__device__ __forceinline__ int4 tail_totals(const TailShared<C>& sh, int s) {
    const int lane = threadIdx.x & 31;
    int x = 0, y = INT_MAX, z = 0, w = 0;
    if (lane < C) {
        const int* d = sh.slots[s & 1][lane];
        x = d[0];
        y = d[1];
        z = d[2];
        w = d[3];
    }
    return make_int4(__reduce_add_sync(0xffffffffu, x), __reduce_min_sync(0xffffffffu, y),
                     __reduce_add_sync(0xffffffffu, z), __reduce_add_sync(0xffffffffu, w));
}

// The same peeling as k_peel (levels, rounds, k + 1 -> k crossings), on the local
// subgraph, continuing the level k and round r where the grid kernel stopped.
//
// A vertex is alive at a level start exactly when its degree exceeds the finished level
// k (a removed vertex had degree <= k when it left, and degrees only fall). Frontier
// counters rotate over three rounds (round r reads slot r % 3 of every CTA, crossings
// append to (r + 1) % 3, and each CTA clears its own (r + 2) % 3, which no CTA touches in
// round r); the level minima alternate by level parity. Every decision that ends a loop
// is taken by all CTAs from the same values read between the same two cluster barriers,
// so the CTAs always meet at the same barrier. In a round, the owner of each frontier
// vertex writes its round and core number and walks its row: its own thread for a short
// row, its warp for a medium one, the whole CTA for a heavy one, every load of a walk in
// flight before its first decrement.
template <int C>
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_peel_tail(TailArgs a) {
    using Sh = TailShared<C>;
    constexpr int OWN = Sh::OWN;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    Sh& sh = *reinterpret_cast<Sh*>(smem);
    if (a.ctl[C_TAIL] != 1) return;  // the grid kernel finished (every CTA reads the same value)
    const int rank = (int)cl.block_rank();
    const int nl = *a.nl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int q = tid; q < OWN; q += TAIL_THREADS) {
        const int v = q * C + rank;
        const bool in = v < nl;
        sh.odeg[q] = in ? a.ld[v] : 0;
        sh.orb[q] = in ? a.lrow[v] : 0;
        sh.ore[q] = in ? a.lrow[v + 1] : 0;
        sh.oL[q] = in ? a.L[v] : 0;
    }
    if (tid < 3) sh.cntL[tid] = 0;
    if (tid < 2) {
        sh.cntH[tid] = 0;
        sh.smin[tid] = INT_MAX;
        sh.acnt[tid] = 0;
        sh.adeg[tid] = 0;
        sh.made[tid] = 0;
    }
    int k = a.ctl[C_TAIL_K], r = a.ctl[C_TAIL_R], rounds = a.ctl[C_ROUNDS], lvl = 0, gs = 0;
    bool handed = false;
    cl.sync();
    while (true) {
        // ---- level start: owned vertices of degree k + 1 join round r + 1
        if (tid == 0) {
            sh.cntL[(r + 2) % 3] = 0;
            sh.cntH[(r + 1) & 1] = 0;
            sh.made[0] = sh.made[1] = 0;  // no crossings are filed before the next round
            sh.smin[(lvl + 1) & 1] = INT_MAX;
            sh.acnt[(lvl + 1) & 1] = 0;
            sh.adeg[(lvl + 1) & 1] = 0;
        }
        int kk = k + 1;
        int lmin = INT_MAX;
        for (int q0 = 0; q0 < OWN; q0 += TAIL_THREADS) {
            const int q = q0 + tid;
            bool rem = false, alive = false;
            if (q < OWN && q * C + rank < nl) {
                const int d = sh.odeg[q];
                if (d > k) {
                    alive = true;
                    if (d <= kk) rem = true;
                    else lmin = min(lmin, d);
                }
            }
            warp_count(alive, &sh.acnt[lvl & 1]);
            const int dsum = __reduce_add_sync(0xffffffffu, alive ? sh.odeg[q] : 0);
            if (lane == 0 && dsum) atomicAdd(&sh.adeg[lvl & 1], dsum);
            const unsigned m = __ballot_sync(0xffffffffu, rem);
            if (m) {
                const int leader = __ffs(m) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(&sh.cntL[(r + 1) % 3], __popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (rem) sh.FL[(r + 1) & 1][base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)q;
            }
        }
        lmin = __reduce_min_sync(0xffffffffu, lmin);
        if (lane == 0 && lmin != INT_MAX) atomicMin(&sh.smin[lvl & 1], lmin);
        __syncthreads();  // the level start's own filings, minimum and sums are final
        tail_publish(sh, cl, gs,
                     make_int4(sh.cntL[(r + 1) % 3], sh.smin[lvl & 1], sh.acnt[lvl & 1], sh.adeg[lvl & 1]));
        cl.sync();
        const int4 g = tail_totals(sh, gs++);
        // the single CTA takes over once few vertices and few edges are left (dense
        // remainders, such as planted communities, keep the cluster's sixteen SMs)
        if (g.z > 0 && g.z <= a.solo_cap && g.w <= SOLO_DEG_CAP) {
            // few vertices left: export them (local id, current degree) to the single-CTA
            // phase, which starts this level again; the frontier filed above is dropped
            for (int q0 = 0; q0 < OWN; q0 += TAIL_THREADS) {
                const int q = q0 + tid;
                const int v = q * C + rank;
                const bool alive = q < OWN && v < nl && sh.odeg[q] > k;
                const unsigned m = __ballot_sync(0xffffffffu, alive);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int base = 0;
                    if (lane == leader) base = atomicAdd(a.ns, __popc(m));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (alive) {
                        const int i = base + __popc(m & ((1u << lane) - 1u));
                        if (i < a.solo_cap) {
                            a.slist[i] = v;
                            a.sdeg[i] = sh.odeg[q];
                            a.map2[v] = i;
                        } else {
                            atomicExch(&a.ctl[C_ERR], 2);
                        }
                    }
                }
            }
            if (rank == 0 && tid == 0) {
                a.ctl[C_SOLO] = 1;
                a.ctl[C_SOLO_K] = k;
                a.ctl[C_SOLO_R] = r;
                a.ctl[C_ROUNDS] = rounds;
            }
            handed = true;
            break;
        }
        int total = g.x;
        if (total == 0) {
            if (g.y == INT_MAX) break;  // nothing left anywhere
            kk = g.y;                   // jump to the smallest remaining degree
            cl.sync();  // every CTA has read the empty totals before appends resume
            for (int q0 = 0; q0 < OWN; q0 += TAIL_THREADS) {
                const int q = q0 + tid;
                bool rem = false;
                if (q < OWN && q * C + rank < nl) {
                    const int d = sh.odeg[q];
                    rem = d > k && d <= kk;
                }
                const unsigned m = __ballot_sync(0xffffffffu, rem);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int base = 0;
                    if (lane == leader) base = atomicAdd(&sh.cntL[(r + 1) % 3], __popc(m));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (rem) sh.FL[(r + 1) & 1][base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)q;
                }
            }
            cl.sync();
            total = 1;  // some vertex has the minimum degree: the jump frontier is not empty
        }
        k = kk;
        r += 1;
        // ---- rounds at level k
        while (total > 0) {
            const int nL = sh.cntL[r % 3];
            int32_t* const rdec = total >= TAIL_AGG_MIN ? a.dec : nullptr;  // the same in every CTA
            if (tid == 0) {
                sh.cntL[(r + 2) % 3] = 0;
                sh.cntH[(r + 1) & 1] = 0;  // read in round r + 1, after this round's barriers
                sh.made[(r + 1) & 1] = 0;
            }
            // one pass, up to 32 frontier vertices per warp, dealt round-robin over the warps
            // (a small frontier spreads one vertex per warp): round and core number; a short
            // row is walked by its own lane, a medium one by the whole warp in turn, and a
            // heavy one is left to the whole CTA below
            const uint16_t* fl = sh.FL[r & 1];
            constexpr int NW = TAIL_THREADS / 32;
            for (int i0 = warp; i0 - warp < nL; i0 += TAIL_THREADS) {
                const int i = i0 + lane * NW;
                const bool have = i < nL;
                const int q = have ? fl[i] : 0;
                const int b = have ? sh.orb[q] : 0, e = have ? sh.ore[q] : 0;
                if (have) {
                    a.rnd[sh.oL[q]] = r;
                    a.core[sh.oL[q]] = k;
                }
                // a short row is walked by its own lane (TAIL_CHUNK loads at a time) when the
                // frontier gives every warp several rows, or when it takes one step anyway;
                // in a small frontier the whole warp walks it in one step
                const bool lanewalk = nL > 4 * NW || e - b <= TAIL_CHUNK;
                const bool shortrow = have && e - b <= TAIL_SHORT && lanewalk;
                bool medium = have && !shortrow;
                if (have && e - b > TAIL_LIGHT) {
                    const int h = atomicAdd(&sh.cntH[r & 1], 1);
                    if (h < TAIL_HCAP) {
                        sh.FH[h] = (uint16_t)q;
                        medium = false;
                    }
                }
                if (shortrow) {
                    for (int j0 = b; j0 < e; j0 += TAIL_CHUNK) {
                        int vv[TAIL_CHUNK];
#pragma unroll
                        for (int t = 0; t < TAIL_CHUNK; t++) vv[t] = (j0 + t < e) ? (int)a.ladj[j0 + t] : -1;
                        tail_decrement<C>(sh, cl, vv, k, r, rdec);
                    }
                }
                unsigned mm = __ballot_sync(0xffffffffu, medium);
                while (mm) {
                    const int src = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const int bb = __shfl_sync(0xffffffffu, b, src), ee = __shfl_sync(0xffffffffu, e, src);
                    for (int j0 = bb; j0 < ee; j0 += TAIL_LIGHT) {
                        int vv[TAIL_LIGHT / 32];
#pragma unroll
                        for (int t = 0; t < TAIL_LIGHT / 32; t++) {
                            const int j = j0 + t * 32 + lane;
                            vv[t] = (j < ee) ? (int)a.ladj[j] : -1;
                        }
                        tail_decrement<C>(sh, cl, vv, k, r, rdec);
                    }
                }
            }
            __syncthreads();  // this round's heavy list is complete
            // the whole CTA per heavy row
            const int nH = min(sh.cntH[r & 1], TAIL_HCAP);
            for (int h = 0; h < nH; h++) {
                const int q = sh.FH[h];
                const int b = sh.orb[q], e = sh.ore[q];
                for (int j0 = b; j0 < e; j0 += 4 * TAIL_THREADS) {
                    int vv[4];
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const int j = j0 + t * TAIL_THREADS + tid;
                        vv[t] = (j < e) ? (int)a.ladj[j] : -1;
                    }
                    tail_decrement<C>(sh, cl, vv, k, r, rdec);
                }
            }
            if (rdec) {
                // every CTA's decrements are in L2: each owner applies its own, and files the
                // vertices that crossed k + 1 -> k (the sum may cross in one step)
                cl.sync();
                for (int q0 = 0; q0 < OWN; q0 += TAIL_THREADS) {
                    const int q = q0 + tid;
                    bool cross = false;
                    if (q < OWN && q * C + rank < nl) {
                        int32_t* dp = rdec + rank * TAIL_OWN + q;
                        const int d = __ldcg(dp);
                        if (d) {
                            *dp = 0;
                            const int old = sh.odeg[q];
                            sh.odeg[q] = old - d;
                            cross = old > k && old - d <= k;
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, cross);
                    if (m) {
                        const int leader = __ffs(m) - 1;
                        int base = 0;
                        if (lane == leader) {
                            base = atomicAdd(&sh.cntL[(r + 1) % 3], __popc(m));
                            atomicAdd(&sh.made[r & 1], __popc(m));
                        }
                        base = __shfl_sync(0xffffffffu, base, leader);
                        if (cross) sh.FL[(r + 1) & 1][base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)q;
                    }
                }
            }
            __syncthreads();  // this CTA's crossings of the round are counted
            tail_publish(sh, cl, gs, make_int4(sh.made[r & 1], INT_MAX, 0, 0));
            cl.sync();
            r++;
            rounds++;
            total = tail_totals(sh, gs++).x;
        }
        lvl++;
    }
    if (rank == 0 && tid == 0 && !handed) {
        a.ctl[C_ROUNDS] = rounds;
        a.ctl[C_ALPHA] = k;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Launch configuration of the tail on one cluster of C CTAs.
template <int C>
static cudaLaunchConfig_t tail_config(cudaLaunchAttribute* attr, cudaStream_t s) {
    const size_t smem = sizeof(TailShared<C>);
    FOLTY_CUDA(cudaFuncSetAttribute(k_peel_tail<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (C > 8) FOLTY_CUDA(cudaFuncSetAttribute(k_peel_tail<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// CTAs of the tail's cluster: 16 when the device places such a cluster, else 8.
static int tail_cluster_size(cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config<16>(attr, s);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_peel_tail<16>, &cfg) == cudaSuccess && clusters >= 1) return 16;
    cudaGetLastError();
    cfg = tail_config<8>(attr, s);
    if (cudaOccupancyMaxActiveClusters(&clusters, k_peel_tail<8>, &cfg) == cudaSuccess && clusters >= 1) return 8;
    cudaGetLastError();
    fail(FOLTY_ECUDA, "peeling: the device cannot place the tail's thread-block cluster");
}

template <int C>
static void launch_tail(const TailArgs& ta, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config<C>(attr, s);
    FOLTY_CUDA(cudaLaunchKernelEx(&cfg, k_peel_tail<C>, ta));
    after_launch("k_peel_tail");
}

// ================================================================== A3 last levels

// Once at most SOLO_CAP vertices are left, a single CTA finishes the peeling: degrees, row
// starts and frontiers of the remaining subgraph fit in its shared memory, so a round ends
// with __syncthreads instead of a cluster barrier. Vertices are renumbered 0..ns-1 again
// ("solo" ids, 16-bit) in the order the cluster exported them.
constexpr int SOLO_THREADS = 1024;
constexpr int SOLO_CAP = 12288;  // vertices of the single-CTA phase
constexpr int SOLO_PASS = 2048;  // frontier vertices laid out per pass (2 per thread)
constexpr int SOLO_CHUNK = 8;    // adjacency entries per thread in flight together (large frontiers)
constexpr int SOLO_CHUNK_S = 2;
constexpr int SOLO_COARSE = 1024;  // coarse owner table of a large frontier's flat entries  // the same for small frontiers (W <= 2048 in one step; less code)

// Cluster row length and global id of each exported vertex (0 past the exported count).
__global__ void k_solo_rows(const int* __restrict__ ctl, const int* __restrict__ ns_p,
                            const int32_t* __restrict__ slist, const int32_t* __restrict__ lrow,
                            const int32_t* __restrict__ L, int32_t* __restrict__ dl, int32_t* __restrict__ sgid) {
    if (ctl[C_SOLO] != 1) return;
    const int ns = *ns_p;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < SOLO_CAP; i += gridDim.x * blockDim.x) {
        if (i < ns) {
            const int32_t v = slist[i];
            dl[i] = lrow[v + 1] - lrow[v];
            sgid[i] = L[v];
        } else {
            dl[i] = 0;
        }
    }
}

// Entry e of the concatenated cluster rows of the exported vertices (eo = prefix of dl):
// an alive neighbour (map2 >= 0) goes to its owner's row of the remaining subgraph, in
// solo ids (order within a row is irrelevant). Every row must come out with exactly the
// degree the cluster exported (its alive neighbours): fc counts them, and the
// single-CTA kernel checks the count; an entry beyond it is recorded in *err (4).
// L2 residency of the single-CTA phase's rows: written and read with an "evict last"
// policy, so that the streaming kernels of the temporal store, which run beside the
// peeling, evict their own lines first; set back to normal when the phase ends.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ int ld_keep_u16(const uint16_t* p, uint64_t pol) {
    unsigned short v;
    asm("ld.global.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return (int)v;
}

__device__ __forceinline__ void st_keep_u16(uint16_t* p, uint16_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u16 [%0], %1, %2;" ::"l"(p), "h"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void l2_release_line(const void* p) {
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(p) : "memory");
}

__global__ void k_solo_fill(const int* __restrict__ ctl, const int32_t* __restrict__ eo,
                            const int32_t* __restrict__ slist, const int32_t* __restrict__ sdeg,
                            const int32_t* __restrict__ srow, const int32_t* __restrict__ lrow,
                            const uint32_t* __restrict__ ladj, const int32_t* __restrict__ map2,
                            int32_t* __restrict__ fc, uint16_t* __restrict__ sadj, int* __restrict__ err) {
    if (ctl[C_SOLO] != 1 || ctl[C_ERR] != 0) return;
    const uint64_t keep = l2_keep_policy();
    const int64_t total = eo[SOLO_CAP];
    const int64_t step = (int64_t)gridDim.x * blockDim.x * FILL_RUN;
    for (int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * FILL_RUN; e0 < total; e0 += step) {
        int lo = 0, hi = SOLO_CAP - 1;  // last owner with eo[owner] <= e0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (eo[mid] <= e0) lo = mid;
            else hi = mid - 1;
        }
        const int64_t e1 = min(e0 + FILL_RUN, total);
        for (int64_t e = e0; e < e1; e++) {
            while (lo + 1 < SOLO_CAP && eo[lo + 1] <= e) lo++;
            const int32_t m = map2[ladj[lrow[slist[lo]] + (int32_t)(e - eo[lo])]];
            if (m >= 0) {
                const int p = atomicAdd(&fc[lo], 1);
                if (p < sdeg[lo]) st_keep_u16(&sadj[srow[lo] + p], (uint16_t)m, keep);
                else atomicExch(err, 4);
            }
        }
    }
}

struct SoloArgs {
    const int* ns;
    const int32_t* sdeg;
    const int32_t* fc;    // entries k_solo_fill wrote per row (must equal sdeg)
    const int32_t* srow;  // exclusive prefix of sdeg: row i = sadj[srow[i], srow[i + 1])
    const uint16_t* sadj;
    const int32_t* sgid;  // global vertex id
    int32_t* rnd;
    int32_t* core;
    int* ctl;
};

// Once at most BM_CAP vertices are left, their induced subgraph moves into shared memory
// as a bit matrix (row v, bit u: edge v-u), so that a round reads no global memory.
constexpr int BM_CAP = 960;
constexpr int BM_W = BM_CAP / 32;  // words per row

struct SoloShared {
    int cnt[3];                // frontier sizes, rotating over three rounds
    int smin[2];               // smallest degree above the level, by level parity
    int acnt[2];               // vertices alive at the level start, by level parity
    int wsum[SOLO_THREADS / 32];
    int sx[32], sb[32];        // small frontier: exclusive prefix of row lengths, row start - prefix
    int sW;                    // small frontier: total row length
    uint16_t coarse[SOLO_COARSE];  // large frontier: row holding flat entry b << cs
    int32_t rs[SOLO_CAP + 1];
    uint16_t FL[2][SOLO_CAP];  // frontier by round parity; FL[0] / FL[1] hold the bit-matrix phase's
                               // id map / its small arrays
    int32_t P[SOLO_PASS + 1];  // prefix of the row lengths of one pass of a large frontier
    int32_t D[SOLO_PASS];      // row start - P: adjacency index of flat entry x is D[o] + x
    union {
        int32_t deg[SOLO_CAP];
        uint32_t bm[BM_CAP * BM_W];  // bit-matrix phase (replaces deg)
    } u;
};
static_assert(sizeof(SoloShared) <= 232448, "single-CTA phase exceeds the shared memory of a CTA");
static_assert(4 * BM_CAP * 2 + 2 * BM_CAP * 3 <= 2 * SOLO_CAP, "bit-matrix phase arrays fit one frontier list");

constexpr int SOLO_SLOTS = SOLO_CAP / SOLO_THREADS;  // vertices each thread checks at level starts
static_assert(SOLO_CAP % SOLO_THREADS == 0 && SOLO_SLOTS <= 32, "level-start slots fit one mask word");

// Appends solo id v to the frontier list for every lane with pred set (one shared-memory
// atomic per warp). A list never holds more than SOLO_CAP entries (a vertex joins one
// frontier); an append beyond that is dropped and the count, above SOLO_CAP, reports it.
// The whole warp must call it.
__device__ __forceinline__ void solo_append(bool pred, int v, uint16_t* fl, int* cnt) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    const int at = base + __popc(m & ((1u << lane) - 1u));
    if (pred && at < SOLO_CAP) fl[at] = (uint16_t)v;
}

// The same append for one thread alone (no warp-wide step), into a list of cap entries.
__device__ __forceinline__ void solo_push(int v, uint16_t* fl, int* cnt, int cap = SOLO_CAP) {
    const int at = atomicAdd(cnt, 1);
    if (at < cap) fl[at] = (uint16_t)v;
}

// Row entries at or past ns cannot come from rows that k_solo_fill checked; such an
// entry is dropped and flags an internal error. Checked after all N loads were issued,
// so that the loads overlap.
template <int N>
__device__ __forceinline__ void solo_check_rows(int (&vv)[N], int ns, int* ctl) {
#pragma unroll
    for (int c = 0; c < N; c++) {
        if (vv[c] >= ns) {
            atomicExch(&ctl[C_ERR], 5);
            vv[c] = -1;
        }
    }
}

// Neighbours vv[0..N) (negative: none) lose one degree each at level k; a k + 1 -> k
// crossing files the vertex in the next frontier. Only the first nch items can hold
// neighbours; nch must be the same across the warp, which must call it whole.
template <int N>
__device__ __forceinline__ void solo_decrement(SoloShared& sh, const int (&vv)[N], int nch, int k, uint16_t* fn,
                                               int* cn, const uint16_t* sadj) {
    int old[N];
#pragma unroll
    for (int c = 0; c < N; c++) old[c] = vv[c] >= 0 ? atomicSub(&sh.u.deg[vv[c]], 1) : 0;
#pragma unroll
    for (int c = 0; c < N; c++) {
        if (c < nch) {
            const bool joins = vv[c] >= 0 && old[c] == k + 1;
            solo_append(joins, vv[c], fn, cn);
            // the next round reads this vertex's row: start its first line on the way to L1
            if (joins) asm volatile("prefetch.global.L1 [%0];" ::"l"(sadj + sh.rs[vv[c]]));
        }
    }
}

// The last levels on the bit matrix. At entry every thread's mask lists its alive slots
// (degree > k) at the start of level k + 1, n3 <= BM_CAP of them in all; the level starts
// again here. New ids 0..n3-1 follow the slots in thread order; FL[0] maps slot -> new
// id while the matrix is built, FL[1] holds the new ids' degrees, global ids, frontier
// lists and slots. A round hands each frontier vertex to one warp, whose lanes each take
// one 32-bit word of its row and decrement the degree of every neighbour in it.
__device__ __forceinline__ void bm_phase(SoloShared& sh, const SoloArgs& a, int ns, int n3, unsigned mine, int& k,
                                         int& r, int& rounds, int& lvl, int& steps, bool& bad) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t keep = l2_keep_policy();
    constexpr uint16_t NONE = 0xffff;
    uint16_t* map = sh.FL[0];
    int32_t* deg3 = reinterpret_cast<int32_t*>(sh.FL[1]);
    int32_t* gid3 = deg3 + BM_CAP;
    uint16_t* fl3 = reinterpret_cast<uint16_t*>(gid3 + BM_CAP);  // two lists of BM_CAP
    uint16_t* n2o = fl3 + 2 * BM_CAP;
    // ---- new ids: block-wide exclusive prefix of the alive slot counts
    for (int i = tid; i < SOLO_CAP; i += SOLO_THREADS) map[i] = NONE;
    const int mc = __popc(mine);
    int inc = mc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();  // the level start's reads of wsum and the frontier counts are done
    if (lane == 31) sh.wsum[warp] = inc;
    if (tid == 0) {
        sh.cnt[(r + 1) % 3] = 0;  // the frontier filed by the level start is dropped
        sh.smin[lvl & 1] = INT_MAX;
    }
    __syncthreads();
    if (warp == 0) {
        const int w = sh.wsum[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        sh.wsum[lane] = wi - w;
    }
    __syncthreads();
    int id = sh.wsum[warp] + inc - mc;
    for (unsigned m = mine; m; m &= m - 1) {
        const int i = tid + (__ffs(m) - 1) * SOLO_THREADS;
        if (id < BM_CAP) {
            map[i] = (uint16_t)id;
            n2o[id] = (uint16_t)i;
            deg3[id] = sh.u.deg[i];
            gid3[id] = a.sgid[i];
        }
        id++;
    }
    __syncthreads();
    // ---- the matrix (it overlays the degrees just copied)
    for (int w = tid; w < BM_CAP * BM_W; w += SOLO_THREADS) sh.u.bm[w] = 0;
    __syncthreads();
    for (int v = warp; v < n3; v += SOLO_THREADS / 32) {
        const int o = n2o[v];
        const int b = sh.rs[o], e = sh.rs[o + 1];
        for (int j0 = b; j0 < e; j0 += 8 * 32) {
            int nb[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const int j = j0 + t * 32 + lane;
                nb[t] = j < e ? ld_keep_u16(&a.sadj[j], keep) : -1;
            }
#pragma unroll
            for (int t = 0; t < 8; t++) {
                if (nb[t] < 0 || nb[t] >= ns) continue;
                const int u = map[nb[t]];
                if (u != NONE) atomicOr(&sh.u.bm[v * BM_W + (u >> 5)], 1u << (u & 31));
            }
        }
    }
    // ---- levels and rounds on the matrix
    while (true) {
        __syncthreads();
        uint16_t* fs = fl3 + ((r + 1) & 1) * BM_CAP;
        int* cs = &sh.cnt[(r + 1) % 3];
        int kk = k + 1, lmin = INT_MAX;
        if (tid < n3) {
            const int d = deg3[tid];
            if (d > k) {
                if (d <= kk) solo_push(tid, fs, cs, BM_CAP);
                else lmin = d;
            }
        }
        lmin = __reduce_min_sync(0xffffffffu, lmin);
        if (lane == 0 && lmin != INT_MAX) atomicMin(&sh.smin[lvl & 1], lmin);
        __syncthreads();
        const int c0 = *cs, m0 = sh.smin[lvl & 1];
        if (tid == 0) sh.smin[(lvl + 1) & 1] = INT_MAX;
        if (++steps > 2 * ns + 2 || c0 > BM_CAP) {
            bad = true;
            return;
        }
        if (c0 == 0) {
            if (m0 == INT_MAX) return;  // nothing left
            kk = m0;
            __syncthreads();  // every thread has read c0 before the jump appends
            if (tid < n3) {
                const int d = deg3[tid];
                if (d > k && d <= kk) solo_push(tid, fs, cs, BM_CAP);
            }
        }
        k = kk;
        r += 1;
        lvl++;
        while (true) {
            __syncthreads();  // the round's frontier is complete
            const int nL = sh.cnt[r % 3];
            if (tid == 0) sh.cnt[(r + 2) % 3] = 0;
            if (nL == 0) break;
            if (++steps > 2 * ns + 2 || nL > BM_CAP) {
                bad = true;
                return;
            }
            const uint16_t* fl = fl3 + (r & 1) * BM_CAP;
            uint16_t* fn = fl3 + ((r + 1) & 1) * BM_CAP;
            int* cn = &sh.cnt[(r + 1) % 3];
            // 32 S threads per frontier vertex (S = 4, 2, 1 as the frontier grows): thread t
            // takes bits [(t / 32) 32 / S, (t / 32 + 1) 32 / S) of word t % 32 of the row, so
            // that a small frontier spreads its decrements over more lanes
            const int S = nL <= 8 ? 4 : nL <= 16 ? 2 : 1;
            const int per = 32 * S, bits = 32 / S;
            const int sub = tid % per, wd = sub & 31;
            const unsigned slice = S == 1 ? 0xffffffffu : (((1u << bits) - 1u) << ((sub >> 5) * bits));
            for (int i = tid / per; i < nL; i += SOLO_THREADS / per) {
                const int v = fl[i];
                if (wd < BM_W) {
                    unsigned w = sh.u.bm[v * BM_W + wd] & slice;
                    while (w) {
                        const int u = wd * 32 + __ffs(w) - 1;
                        w &= w - 1;
                        if (atomicSub(&deg3[u], 1) == k + 1) solo_push(u, fn, cn, BM_CAP);
                    }
                }
                if (sub == 0) {
                    a.rnd[gid3[v]] = r;
                    a.core[gid3[v]] = k;
                }
            }
            r++;
            rounds++;
        }
    }
}

// The same peeling once more (levels, rounds, k + 1 -> k crossings), continuing the level
// k and round r where the cluster stopped. A round lays the frontier's rows out flat (a
// prefix of their lengths) and deals the entries to all threads alike. A frontier of at
// most 32 vertices (most rounds) is laid out by every warp in its own registers, so such
// a round costs one barrier, one adjacency load and one shared-memory decrement per
// entry; a larger one goes through shared memory in passes of SOLO_PASS vertices. At a
// level start each thread checks the vertices it owns (tid + j SOLO_THREADS) that were
// still alive at the previous one.
__global__ void __launch_bounds__(SOLO_THREADS, 1) k_peel_solo(SoloArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    SoloShared& sh = *reinterpret_cast<SoloShared*>(smem);
    if (a.ctl[C_SOLO] != 1 || a.ctl[C_ERR] != 0) return;
    const int ns = *a.ns;
    if (ns > SOLO_CAP) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t keep = l2_keep_policy();
    int miscount = 0;
    for (int i = tid; i <= ns; i += SOLO_THREADS) {
        if (i < ns) {
            sh.u.deg[i] = a.sdeg[i];
            miscount |= a.fc[i] != a.sdeg[i];
        }
        sh.rs[i] = a.srow[i];
    }
    unsigned mine = 0;  // owned slots alive at the last level start
    for (int j = 0; j < SOLO_SLOTS; j++)
        if (tid + j * SOLO_THREADS < ns) mine |= 1u << j;
    if (tid < 3) sh.cnt[tid] = 0;
    if (tid < 2) {
        sh.smin[tid] = INT_MAX;
        sh.acnt[tid] = 0;
    }
    int k = a.ctl[C_SOLO_K], r = a.ctl[C_SOLO_R], rounds = a.ctl[C_ROUNDS], lvl = 0;
    int n3 = 0;  // vertices handed to the bit-matrix phase
    // every level and every round removes at least one vertex: more than 2 ns + 2 steps
    // (or a frontier above SOLO_CAP) can only come from an internal error
    int steps = 0;
    bool bad = false;
    if (__syncthreads_or(miscount)) {
        if (tid == 0) atomicExch(&a.ctl[C_ERR], 4);
        return;
    }
    while (true) {
        // ---- level start: vertices of degree k + 1 (or the smallest degree) join round
        // r + 1 (r is the empty round that ended the last level, or the hand-off round)
        uint16_t* fs = sh.FL[(r + 1) & 1];
        int* cs = &sh.cnt[(r + 1) % 3];
        int kk = k + 1, lmin = INT_MAX, na = 0;
        for (unsigned m = mine; m; m &= m - 1) {
            const int j = __ffs(m) - 1, i = tid + j * SOLO_THREADS;
            const int d = sh.u.deg[i];
            if (d <= k) {
                mine &= ~(1u << j);  // left at an earlier level
                continue;
            }
            na++;
            if (d <= kk) solo_push(i, fs, cs);
            else lmin = min(lmin, d);
        }
        lmin = __reduce_min_sync(0xffffffffu, lmin);
        na = __reduce_add_sync(0xffffffffu, na);
        if (lane == 0) {
            if (lmin != INT_MAX) atomicMin(&sh.smin[lvl & 1], lmin);
            if (na) atomicAdd(&sh.acnt[lvl & 1], na);
        }
        __syncthreads();
        const int c0 = *cs, m0 = sh.smin[lvl & 1], alive = sh.acnt[lvl & 1];
        if (tid == 0) {  // both last read at the previous level start
            sh.smin[(lvl + 1) & 1] = INT_MAX;
            sh.acnt[(lvl + 1) & 1] = 0;
        }
        if (++steps > 2 * ns + 2 || c0 > SOLO_CAP) {
            bad = true;
            break;
        }
        if (c0 == 0 && m0 == INT_MAX) break;  // nothing left
        if (alive <= BM_CAP) {  // the rest fits the bit matrix (this level starts again there)
            n3 = alive;
            break;
        }
        if (c0 == 0) {
            kk = m0;                   // jump to the smallest remaining degree
            __syncthreads();           // every thread has read c0 before the jump appends
            for (unsigned m = mine; m; m &= m - 1) {
                const int i = tid + (__ffs(m) - 1) * SOLO_THREADS;
                if (sh.u.deg[i] <= kk) solo_push(i, fs, cs);  // every kept slot has degree > k + 1
            }
        }
        k = kk;
        r += 1;
        lvl++;
        // ---- rounds at level k
        while (true) {
            __syncthreads();  // the round's frontier is complete
            const int nL = sh.cnt[r % 3];
            if (tid == 0) sh.cnt[(r + 2) % 3] = 0;  // read in round r - 1, appended to in round r + 1
            if (nL == 0) break;
            if (++steps > 2 * ns + 2 || nL > SOLO_CAP) {
                bad = true;
                break;
            }
            const uint16_t* fl = sh.FL[r & 1];
            uint16_t* fn = sh.FL[(r + 1) & 1];
            int* cn = &sh.cnt[(r + 1) % 3];
            if (nL <= 32) {
                // warp 0 lays the (at most 32) rows out: lane o holds frontier vertex o
                int gid = -1;
                if (warp == 0) {
                    const bool have = lane < nL;
                    const int q = have ? fl[lane] : 0;
                    const int rb = have ? sh.rs[q] : 0;
                    const int len = have ? sh.rs[q + 1] - rb : 0;
                    if (have) gid = a.sgid[q];
                    int inc = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    sh.sx[lane] = inc - len;
                    sh.sb[lane] = rb - (inc - len);
                    if (lane == 31) sh.sW = inc;
                }
                __syncthreads();
                const int W = sh.sW;
                for (int x0 = 0; x0 < W; x0 += SOLO_THREADS * SOLO_CHUNK_S) {
                    if (x0 + warp * 32 >= W) break;  // nothing left for this warp (warp-uniform)
                    const int nch = min(SOLO_CHUNK_S, (W - x0 + SOLO_THREADS - 1) / SOLO_THREADS);  // block-uniform
                    int vv[SOLO_CHUNK_S];
#pragma unroll
                    for (int c = 0; c < SOLO_CHUNK_S; c++) {
                        const int x = x0 + c * SOLO_THREADS + tid;
                        vv[c] = -1;
                        if (c < nch && x < W) {
                            int lo = 0;  // last row o < nL with sx[o] <= x
#pragma unroll
                            for (int st = 16; st > 0; st >>= 1)
                                if (lo + st < nL && sh.sx[lo + st] <= x) lo += st;
                            vv[c] = ld_keep_u16(&a.sadj[sh.sb[lo] + x], keep);
                        }
                    }
                    solo_check_rows(vv, ns, a.ctl);
                    solo_decrement(sh, vv, nch, k, fn, cn, a.sadj);
                }
                if (gid >= 0) {
                    a.rnd[gid] = r;
                    a.core[gid] = k;
                }
            } else {
                for (int p0 = 0; p0 < nL; p0 += SOLO_PASS) {
                    const int np = min(SOLO_PASS, nL - p0);
                    // two frontier vertices per thread: row lengths, global ids
                    int len[2], rb[2], gid[2];
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const int i = 2 * tid + u;
                        len[u] = 0;
                        rb[u] = 0;
                        gid[u] = -1;
                        if (i < np) {
                            const int q = fl[p0 + i];
                            rb[u] = sh.rs[q];
                            len[u] = sh.rs[q + 1] - rb[u];
                            gid[u] = a.sgid[q];
                        }
                    }
                    // block-wide exclusive prefix of the thread sums
                    const int mysum = len[0] + len[1];
                    int inc = mysum;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    if (lane == 31) sh.wsum[warp] = inc;
                    __syncthreads();
                    if (warp == 0) {
                        int w = sh.wsum[lane], wi = w;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int y = __shfl_up_sync(0xffffffffu, wi, o);
                            if (lane >= o) wi += y;
                        }
                        sh.wsum[lane] = wi - w;  // exclusive warp offsets
                        if (lane == 31) sh.P[np] = wi;
                    }
                    __syncthreads();
                    const int ex = sh.wsum[warp] + inc - mysum;
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const int i = 2 * tid + u;
                        if (i < np) {
                            const int off = ex + (u ? len[0] : 0);
                            sh.P[i] = off;
                            sh.D[i] = rb[u] - off;
                        }
                    }
                    __syncthreads();
                    const int W = sh.P[np];
                    // coarse owners: entry b << cs lies in row coarse[b] (cs keeps W >> cs below
                    // SOLO_COARSE), so that an entry's row is searched between two of them
                    const int cs = max(4, 32 - __clz(max(W, 1) >> 10));
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const int i = 2 * tid + u;
                        if (i < np) {
                            const int b0 = (sh.P[i] + (1 << cs) - 1) >> cs, b1 = (sh.P[i + 1] + (1 << cs) - 1) >> cs;
                            for (int b = b0; b < b1 && b < SOLO_COARSE; b++) sh.coarse[b] = (uint16_t)i;
                        }
                    }
                    __syncthreads();
                    for (int x0 = 0; x0 < W; x0 += SOLO_THREADS * SOLO_CHUNK) {
                        if (x0 + warp * 32 >= W) break;  // nothing left for this warp (warp-uniform)
                        const int nch = min(SOLO_CHUNK, (W - x0 + SOLO_THREADS - 1) / SOLO_THREADS);
                        int vv[SOLO_CHUNK];
#pragma unroll
                        for (int c = 0; c < SOLO_CHUNK; c++) {
                            const int x = x0 + c * SOLO_THREADS + tid;
                            vv[c] = -1;
                            if (c < nch && x < W) {
                                const int b = x >> cs;  // last row with P[row] <= x, from coarse[b]
                                int lo = sh.coarse[b], hi = ((b + 1) << cs) < W ? sh.coarse[b + 1] : np - 1;
                                while (lo < hi) {
                                    const int mid = (lo + hi + 1) >> 1;
                                    if (sh.P[mid] <= x) lo = mid;
                                    else hi = mid - 1;
                                }
                                vv[c] = ld_keep_u16(&a.sadj[sh.D[lo] + x], keep);
                            }
                        }
                        solo_check_rows(vv, ns, a.ctl);
                        solo_decrement(sh, vv, nch, k, fn, cn, a.sadj);
                    }
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        if (gid[u] >= 0) {
                            a.rnd[gid[u]] = r;
                            a.core[gid[u]] = k;
                        }
                    }
                    __syncthreads();  // P and D are rewritten by the next pass
                }
            }
            r++;
            rounds++;
        }
        if (bad) break;
    }
    if (n3 > 0 && !bad) bm_phase(sh, a, ns, n3, mine, k, r, rounds, lvl, steps, bad);
    // the rows' lines go back to normal eviction priority
    for (int x = tid * 64; x < sh.rs[ns]; x += SOLO_THREADS * 64) l2_release_line(a.sadj + x);
    if (tid == 0) {
        if (bad) atomicExch(&a.ctl[C_ERR], 2);
        a.ctl[C_ROUNDS] = rounds;
        a.ctl[C_ALPHA] = k;
    }
}

static void launch_solo(const SoloArgs& sa, cudaStream_t s) {
    const int smem = (int)sizeof(SoloShared);
    FOLTY_CUDA(cudaFuncSetAttribute(k_peel_solo, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FOLTY_LAUNCH(k_peel_solo, 1, SOLO_THREADS, smem, s, sa);
}

__global__ void k_iota(int32_t* __restrict__ a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// ================================================================== A4

__device__ __forceinline__ bool rank_less(int32_t u, int32_t v, const int32_t* __restrict__ rnd) {
    int32_t ru = rnd[u], rv = rnd[v];
    return ru < rv || (ru == rv && u < v);
}

// Entry j of the adjacency (owner u, neighbour v) is kept as u -> v when v comes later
// in the degeneracy order.
__global__ void k_orient_flags(const int32_t* __restrict__ adj_src, const int32_t* __restrict__ adj,
                               const int32_t* __restrict__ rnd, int64_t n2, int32_t* __restrict__ flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n2;
         j += (int64_t)gridDim.x * blockDim.x)
        flag[j] = rank_less(adj_src[j], adj[j], rnd);
}

// Kept entries at their scanned positions: rows stay in ascending neighbour order.
__global__ void k_orient_fill(const int32_t* __restrict__ adj_src, const int32_t* __restrict__ adj,
                              const int32_t* __restrict__ adj_eid, const int32_t* __restrict__ flag,
                              const int32_t* __restrict__ opos, int64_t n2, int32_t* __restrict__ out_nbr,
                              int32_t* __restrict__ out_eid, int32_t* __restrict__ out_src) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n2;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[j]) continue;
        int32_t p = opos[j];
        out_nbr[p] = adj[j];
        out_eid[p] = adj_eid[j];
        out_src[p] = adj_src[j];
    }
}

// outptr[u] = opos[rowptr[u]]; also the maximum out-degree.
__global__ void k_outptr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ opos, int64_t n,
                         int32_t* __restrict__ outptr, int* __restrict__ max_out) {
    int best = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = opos[rowptr[u]];
        outptr[u] = o;
        if (u < n) best = max(best, opos[rowptr[u + 1]] - o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_out, best);
}

// ================================================================== A5

// Thread per oriented edge (u, v): merge N+(u) and N+(v) (both ascending by id).
// Triangles of oriented edge u -> v: the common out-neighbours w of u and v (both lists
// sorted). A light edge is merged by one thread; a heavy edge (|out(u)| + |out(v)| >
// heavy_min, the degeneracy core) is intersected by the whole warp: out(u) goes into an
// open-addressed hash table in the warp's shared memory, with each entry's edge id and
// temporal edge count (built once for the consecutive edges of u the warp meets), and the
// lanes look up their share of out(v), the loads of the next share issued before the
// lookups. Both passes find the same set, so the counts match the writes.
constexpr int TRI_THREADS = 256;
constexpr int TRI_HEAVY = 48;
constexpr int TRI_HCAP = 256;    // out(u) entries a warp's table holds (longer lists: one lane merges)
constexpr int TRI_HSLOTS = 512;  // table slots (load at most one half)
// the largest bounded layout of a one-pass listing (the scratch copy and the graph's
// array each hold that many bytes); a larger bound takes the counting pass
constexpr int64_t TRI_BOUND_MAX_BYTES = int64_t(16) << 30;

// FOLTY_TRI_LAYOUT=counted: every graph takes the counting pass before the listing.
inline bool tri_layout_counted() {
    const char* env = std::getenv("FOLTY_TRI_LAYOUT");
    return env && std::strcmp(env, "counted") == 0;
}

// One warp's hash table of out(u): neighbour id per slot (-1: empty) and its position in
// out(u); by position, the static edge id and temporal edge count of (u, w).
struct TriHashW {
    int32_t key[TRI_HSLOTS];
    int16_t pos[TRI_HSLOTS];
    int32_t sig[TRI_HCAP];
    int32_t eid[TRI_HCAP];
};

__device__ __forceinline__ uint32_t tri_hash(int32_t w) { return ((uint32_t)w * 0x9E3779B1u) >> 23; }

// Builds the warp's table of out(u) = [i1, e1) (e1 - i1 <= TRI_HCAP). The whole warp
// must call it. With at most TRI_HCAP keys in TRI_HSLOTS slots every probe sequence ends.
template <bool EID>
__device__ __forceinline__ void warp_hash_out(const int32_t* __restrict__ nbr, const int32_t* __restrict__ osig,
                                              const int32_t* __restrict__ eid, int32_t i1, int32_t e1,
                                              TriHashW& H) {
    const int lane = threadIdx.x & 31;
    __syncwarp();  // the previous table's lookups are done
    for (int t = lane; t < TRI_HSLOTS; t += 32) H.key[t] = -1;
    __syncwarp();
    for (int t = lane; t < e1 - i1; t += 32) {
        const int32_t w = nbr[i1 + t];
        H.sig[t] = osig[i1 + t];
        if (EID) H.eid[t] = eid[i1 + t];
        uint32_t h = tri_hash(w);
        for (int p = 0; p < TRI_HSLOTS; p++) {
            if (atomicCAS(&H.key[h], -1, w) == -1) {
                H.pos[h] = (int16_t)t;
                break;
            }
            h = (h + 1) & (TRI_HSLOTS - 1);
        }
    }
    __syncwarp();
}

// Looks up out(v) = [i2, e2) of the out-lists (nbr, osig and, when EID, eid by position)
// in the warp's table of out(u). Calls hit(found, w, sig_u, eid_u, sig_v, eid_v) once per
// lane and step (w = -1 for an idle lane): the counts and (EID) ids of the static edges
// (u, w) and (v, w) of a common neighbour w. The whole warp must call it.
template <bool EID, typename F>
__device__ __forceinline__ void warp_probe_out(const int32_t* __restrict__ nbr, const int32_t* __restrict__ osig,
                                               const int32_t* __restrict__ eid, int32_t i2, int32_t e2,
                                               const TriHashW& H, F&& hit) {
    const int lane = threadIdx.x & 31;
    int32_t w = -1, sv = 0, ev = 0;
    if (i2 + lane < e2) {
        w = nbr[i2 + lane];
        sv = osig[i2 + lane];
        if (EID) ev = eid[i2 + lane];
    }
    for (int32_t ib0 = i2; ib0 < e2; ib0 += 32) {
        const int32_t ib = ib0 + lane;
        // the next share's loads, in flight during this share's lookups
        int32_t wn = -1, sn = 0, en = 0;
        if (ib + 32 < e2) {
            wn = nbr[ib + 32];
            sn = osig[ib + 32];
            if (EID) en = eid[ib + 32];
        }
        int pu = -1;
        if (ib < e2) {
            uint32_t h = tri_hash(w);
            for (int p = 0; p < TRI_HSLOTS; p++) {
                const int32_t k = H.key[h];
                if (k == w) {
                    pu = H.pos[h];
                    break;
                }
                if (k < 0) break;
                h = (h + 1) & (TRI_HSLOTS - 1);
            }
        }
        hit(pu >= 0, w, pu >= 0 ? H.sig[pu] : 0, (EID && pu >= 0) ? H.eid[pu] : 0, sv, ev);
        w = wn;
        sv = sn;
        ev = en;
    }
}

// Also the probe slots of each oriented edge's triangles (sum over them of the three
// edges' temporal edge counts) into pcnt (may be null), and of all triangles into
// *probes, so that the triangles' probe offsets are known before they are written.
// Like the writing pass, an edge whose two out-lists hold more than heavy_min entries is
// intersected by the whole warp (the thread-versus-warp split the autotuner picks).
__global__ void __launch_bounds__(TRI_THREADS) k_tri_count(const int32_t* __restrict__ outptr,
                                                           const int32_t* __restrict__ out_nbr,
                                                           const int32_t* __restrict__ out_src,
                                                           const int32_t* __restrict__ osig, int32_t S,
                                                           int32_t* __restrict__ cnt, int64_t* __restrict__ pcnt,
                                                           unsigned long long* __restrict__ merged,
                                                           unsigned long long* __restrict__ probes, int heavy_min) {
    __shared__ TriHashW table[TRI_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0, pacc = 0;
    int32_t hashed = -1;  // the vertex whose out-list is in this warp's table
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); j0 < S; j0 += stride) {
        const int64_t j = j0 + lane;
        int32_t u = 0, i1 = 0, e1 = 0, i2 = 0, e2 = 0, sig_uv = 0;
        if (j < S) {
            u = out_src[j];
            const int32_t v = out_nbr[j];
            sig_uv = osig[j];
            i1 = outptr[u];
            e1 = outptr[u + 1];
            i2 = outptr[v];
            e2 = outptr[v + 1];
            acc += (unsigned long long)((e1 - i1) + (e2 - i2));
        }
        const bool heavy = j < S && (e1 - i1) + (e2 - i2) > heavy_min && e1 - i1 <= TRI_HCAP;
        if (j < S && !heavy) {
            int32_t c = 0;
            unsigned long long ps = 0;
            int32_t a1 = i1, a2 = i2;
            while (a1 < e1 && a2 < e2) {
                const int32_t x = out_nbr[a1], y = out_nbr[a2];
                if (x == y) {
                    c++;
                    ps += (unsigned long long)(osig[a1] + osig[a2]);
                }
                a1 += (x <= y);
                a2 += (y <= x);
            }
            if (c) ps += (unsigned long long)c * (unsigned long long)sig_uv;
            pacc += ps;
            cnt[j] = c;
            if (pcnt) pcnt[j] = (int64_t)ps;
        }
        unsigned hm = __ballot_sync(0xffffffffu, heavy);
        while (hm) {
            const int src = __ffs(hm) - 1;
            hm &= hm - 1;
            const int32_t b1 = __shfl_sync(0xffffffffu, i1, src), f1 = __shfl_sync(0xffffffffu, e1, src);
            const int32_t b2 = __shfl_sync(0xffffffffu, i2, src), f2 = __shfl_sync(0xffffffffu, e2, src);
            const int32_t hs = __shfl_sync(0xffffffffu, sig_uv, src), hu = __shfl_sync(0xffffffffu, u, src);
            if (hu != hashed) {
                warp_hash_out<false>(out_nbr, osig, nullptr, b1, f1, table[warp]);
                hashed = hu;
            }
            int32_t c = 0;
            unsigned long long hp = 0;
            warp_probe_out<false>(out_nbr, osig, nullptr, b2, f2, table[warp],
                                  [&](bool found, int32_t, int32_t su, int32_t, int32_t sv, int32_t) {
                                      if (found) {
                                          c++;
                                          hp += (unsigned long long)(su + sv);
                                      }
                                  });
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c += __shfl_xor_sync(0xffffffffu, c, o);
                hp += __shfl_xor_sync(0xffffffffu, hp, o);
            }
            if (lane == 0) {
                hp += (unsigned long long)c * (unsigned long long)hs;
                cnt[j0 + src] = c;
                if (pcnt) pcnt[j0 + src] = (int64_t)hp;
                pacc += hp;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        pacc += __shfl_xor_sync(0xffffffffu, pacc, o);
    }
    if (lane == 0 && acc) atomicAdd(merged, acc);
    if (lane == 0 && pacc) atomicAdd(probes, pacc);
}

// tile_tri[b] = triangle holding probe min(b * tile, P - 1), for b in [0, tiles].
__global__ void k_tile_starts(const int64_t* __restrict__ tri_off, int64_t ntri, int64_t P, int64_t tiles,
                              int tile, int64_t* __restrict__ tile_tri) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= tiles;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = min(b * (int64_t)tile, P - 1);
        int64_t lo = 0, hi = ntri - 1;  // largest t with tri_off[t] <= p
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (tri_off[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        tile_tri[b] = lo;
    }
}

// Writes every triangle, with OFF its probe offset (the running sum of the probe slots of
// the triangles before it, from the counting pass's prefix per oriented edge), and counts
// the triangles on every static edge. The triangles of oriented edge j start at toff[j].
// BOUND (no counting pass before it): toff[j] is the prefix of the per-edge bounds
// min(|N+(u)|, |N+(v)|), the pass writes each edge's triangle count to cnt[j], and adds
// the list lengths merged to merged[0] and the triangles' probe slots to merged[1].
template <bool OFF, bool BOUND = false>
__global__ void __launch_bounds__(TRI_THREADS) k_tri_write(const int32_t* __restrict__ outptr,
                                                           const int32_t* __restrict__ out_nbr,
                                                           const int32_t* __restrict__ out_eid,
                                                           const int32_t* __restrict__ out_src,
                                                           const int32_t* __restrict__ osig, int32_t S,
                                                           const int64_t* __restrict__ toff,
                                                           const int64_t* __restrict__ poff, int4* __restrict__ tri,
                                                           int64_t* __restrict__ tri_off, int32_t* __restrict__ common,
                                                           int heavy_min, int32_t* __restrict__ cnt = nullptr,
                                                           unsigned long long* __restrict__ merged = nullptr) {
    static_assert(!(OFF && BOUND), "probe offsets need the counting pass");
    __shared__ TriHashW table[TRI_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0, pacc = 0;  // BOUND: list lengths merged, probe slots
    int32_t hashed = -1;  // the vertex whose out-list is in this warp's table
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); j0 < S; j0 += stride) {
        const int64_t j = j0 + lane;
        int32_t u = 0, v = 0, s_uv = 0, sig_uv = 0, i1 = 0, e1 = 0, i2 = 0, e2 = 0;
        if (j < S) {
            u = out_src[j];
            v = out_nbr[j];
            s_uv = out_eid[j];
            sig_uv = osig[j];
            i1 = outptr[u];
            e1 = outptr[u + 1];
            i2 = outptr[v];
            e2 = outptr[v + 1];
            if (BOUND) acc += (unsigned long long)((e1 - i1) + (e2 - i2));
        }
        const bool heavy = j < S && (e1 - i1) + (e2 - i2) > heavy_min && e1 - i1 <= TRI_HCAP;
        if (j < S && !heavy) {
            int64_t p = toff[j], q = OFF ? poff[j] : 0;
            int32_t n_here = 0;
            unsigned long long ps = 0;
            int32_t a1 = i1, a2 = i2;
            while (a1 < e1 && a2 < e2) {
                const int32_t x = out_nbr[a1], y = out_nbr[a2];
                if (x == y) {
                    const int32_t w = x, s_uw = out_eid[a1], s_vw = out_eid[a2];
                    const int flags = (u < v ? 1 : 0) | (u < w ? 2 : 0) | (v < w ? 4 : 0);
                    tri[p] = make_int4(s_uv, s_uw, s_vw, flags);
                    if (OFF) {
                        tri_off[p] = q;
                        q += (int64_t)sig_uv + osig[a1] + osig[a2];
                    }
                    if (BOUND) ps += (unsigned long long)(sig_uv + osig[a1] + osig[a2]);
                    atomicAdd(&common[s_uw], 1);
                    atomicAdd(&common[s_vw], 1);
                    p++;
                    n_here++;
                }
                a1 += (x <= y);
                a2 += (y <= x);
            }
            if (n_here) atomicAdd(&common[s_uv], n_here);
            if (BOUND) {
                cnt[j] = n_here;
                pacc += ps;
            }
        }
        unsigned hm = __ballot_sync(0xffffffffu, heavy);
        while (hm) {
            const int src = __ffs(hm) - 1;
            hm &= hm - 1;
            const int32_t b1 = __shfl_sync(0xffffffffu, i1, src), f1 = __shfl_sync(0xffffffffu, e1, src);
            const int32_t b2 = __shfl_sync(0xffffffffu, i2, src), f2 = __shfl_sync(0xffffffffu, e2, src);
            const int32_t hu = __shfl_sync(0xffffffffu, u, src), hv = __shfl_sync(0xffffffffu, v, src);
            const int32_t hs = __shfl_sync(0xffffffffu, s_uv, src), hsig = __shfl_sync(0xffffffffu, sig_uv, src);
            int64_t p = (lane == 0) ? toff[j0 + src] : 0, q = (OFF && lane == 0) ? poff[j0 + src] : 0;
            p = __shfl_sync(0xffffffffu, p, 0);
            q = __shfl_sync(0xffffffffu, q, 0);
            int n_here = 0;
            if (hu != hashed) {
                warp_hash_out<true>(out_nbr, osig, out_eid, b1, f1, table[warp]);
                hashed = hu;
            }
            warp_probe_out<true>(
                out_nbr, osig, out_eid, b2, f2, table[warp],
                [&](bool found, int32_t w, int32_t su, int32_t s_uw, int32_t sv, int32_t s_vw) {
                    const unsigned m = __ballot_sync(0xffffffffu, found);
                    // the hits' probe offsets: a warp prefix of their costs, in lane order
                    const int64_t c = found ? (int64_t)hsig + su + sv : 0;
                    int64_t inc = c;
                    if (OFF) {
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                            if (lane >= o) inc += y;
                        }
                    }
                    if (found) {
                        const int64_t at = p + __popc(m & ((1u << lane) - 1u));
                        const int flags = (hu < hv ? 1 : 0) | (hu < w ? 2 : 0) | (hv < w ? 4 : 0);
                        tri[at] = make_int4(hs, s_uw, s_vw, flags);
                        if (OFF) tri_off[at] = q + inc - c;
                        atomicAdd(&common[s_uw], 1);
                        atomicAdd(&common[s_vw], 1);
                    }
                    if (BOUND) pacc += (unsigned long long)c;
                    p += __popc(m);
                    if (OFF) q += __shfl_sync(0xffffffffu, inc, 31);
                    n_here += __popc(m);
                });
            if (lane == 0 && n_here) atomicAdd(&common[hs], n_here);
            if (BOUND && lane == 0) cnt[j0 + src] = n_here;
        }
    }
    if (BOUND) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            pacc += __shfl_xor_sync(0xffffffffu, pacc, o);
        }
        if (lane == 0 && acc) atomicAdd(merged, acc);
        if (lane == 0 && pacc) atomicAdd(merged + 1, pacc);
    }
}

// bnd[j] = min(|N+(u)|, |N+(v)|) for oriented edge j = (u, v): at most that many common
// out-neighbours, so an upper bound of the triangles the listing finds on j.
__global__ void k_tri_bound(const int32_t* __restrict__ outptr, const int32_t* __restrict__ out_src,
                            const int32_t* __restrict__ out_nbr, int32_t S, int64_t* __restrict__ bnd) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = out_src[j], v = out_nbr[j];
        bnd[j] = min(outptr[u + 1] - outptr[u], outptr[v + 1] - outptr[v]);
    }
}

// ================================================================== driver

// A non-blocking stream of this thread (of the device's highest or default priority)
// for work that runs beside the caller's stream: fork() makes it wait for everything
// enqueued on the caller's stream so far, join() makes the caller's stream wait for
// everything enqueued on it. A fork that was not joined (an error in between) is
// drained on destruction.
class SideStream {
  public:
    SideStream(cudaStream_t s, bool high) : s_(s), high_(high) {}
    ~SideStream() {
        if (forked_) cudaStreamSynchronize(aux_);
        if (ev_[0]) cudaEventDestroy(ev_[0]);
        if (ev_[1]) cudaEventDestroy(ev_[1]);
    }
    SideStream(const SideStream&) = delete;
    SideStream& operator=(const SideStream&) = delete;

    cudaStream_t fork() {
        // per device and priority, kept for the thread's life
        thread_local std::vector<cudaStream_t> streams[2];
        int dev = 0;
        FOLTY_CUDA(cudaGetDevice(&dev));
        auto& v = streams[high_ ? 1 : 0];
        if ((int)v.size() <= dev) v.resize(dev + 1, nullptr);
        if (!v[dev]) {
            int least = 0, greatest = 0;
            FOLTY_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            FOLTY_CUDA(cudaStreamCreateWithPriority(&v[dev], cudaStreamNonBlocking, high_ ? greatest : least));
        }
        aux_ = v[dev];
        for (auto& e : ev_)
            if (!e) FOLTY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        FOLTY_CUDA(cudaEventRecord(ev_[0], s_));
        FOLTY_CUDA(cudaStreamWaitEvent(aux_, ev_[0], 0));
        forked_ = true;
        return aux_;
    }
    void join() {
        FOLTY_CUDA(cudaEventRecord(ev_[1], aux_));
        FOLTY_CUDA(cudaStreamWaitEvent(s_, ev_[1], 0));
        forked_ = false;
    }

  private:
    cudaStream_t s_;
    bool high_;
    cudaStream_t aux_ = nullptr;
    cudaEvent_t ev_[2] = {nullptr, nullptr};
    bool forked_ = false;
};

// The sorted values index other arrays: a sort whose look-back ran out must stop here
// (read_back checks the graph's error word).
static void sort_check(folty_graph* g, cudaStream_t s) { read_back(g, nullptr, nullptr, 0, nullptr, s); }

// The second half of A1 with dense pair ids: the temporal edges sorted by (pair id,
// direction, time rank) into the store (perm, T, sd, seg). It needs nothing of the
// static graph's later steps, and they nothing of it before the triangle pass, so it
// runs on a second stream beside the peeling.
struct StoreJob {
    const uint32_t* slotw;  // [m] pair table slot and direction of each input edge
    const uint32_t* order;  // time order of an unsorted input, or null
    const int32_t* sid;     // [table] dense pair id of each table slot
    int ib;                 // bits of a time rank
};

// sigma (S entries, zeroed here) receives each static edge's temporal edge count, and
// packed_ev is recorded once it is complete.
static void temporal_store(folty_graph* g, const StoreJob& job, Scratch& sc, int32_t* sigma, cudaEvent_t packed_ev) {
    const int T = 256;
    const int64_t m = g->m, mk = g->m_kept;
    const int32_t S = g->S;
    const int ib = job.ib;
    cudaStream_t s = sc.stream();
    const int cbits = bit_length((uint64_t)(2 * S));
    if (!job.order && g->ts32) {
        // time-ordered input with 32-bit offsets: the sort ids and their counts (4 B slot
        // word read and 4 B id written per edge), then the stable sort of the ids, whose
        // first pass reads the ids and times (12 B per edge, 8 B written) and whose last
        // writes T and sd (8 B read and written per edge, as the passes between). perm,
        // the same order of the input indices, is sorted on first use from the ids the
        // graph keeps, except for graphs the allocation-free entry point takes (it needs
        // perm and may not allocate): they get it here.
        const int passes = cbits > STORE_DIGIT_BITS ? (cbits + STORE_DIGIT_BITS - 1) / STORE_DIGIT_BITS : 1;
        StageSpan span(ST_STORE, s, 8 * m + 16 * m * passes + 4 * m);
        const bool eager = mk <= FOLTY_NOALLOC_MAX_EDGES;
        uint32_t* cw = eager ? sc.get<uint32_t>(m) : graph_alloc<uint32_t>(g, m, s);
        int32_t* cnt = sc.get<int32_t>(2 * (int64_t)S + 1);
        uint32_t* hist = eager ? sc.get<uint32_t>(STORE_MAX_PASSES << STORE_DIGIT_BITS)
                               : graph_alloc<uint32_t>(g, STORE_MAX_PASSES << STORE_DIGIT_BITS, s);
        FOLTY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (2 * (size_t)S + 1), s));
        FOLTY_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (STORE_MAX_PASSES << STORE_DIGIT_BITS), s));
        // one block per 2048 edges: short blocks, so that the peel's kernels on the
        // high-priority streams get SMs as soon as any block ends
        FOLTY_LAUNCH(k_store_ids, (unsigned)(((m + STORE_IDS_EDGES - 1) / STORE_IDS_EDGES + T - 1) / T), T, 0, s,
                     job.slotw, m, job.sid, S, cw, cnt);
        // the runs: seg[c] = first sorted position of id c, seg[2S] = mk
        exclusive_scan(sc, cnt, g->seg, 2 * (int64_t)S);
        FOLTY_LAUNCH(k_store_sigma, grid_for(S, T), T, 0, s, g->seg, S, sigma);
        FOLTY_CUDA(cudaEventRecord(packed_ev, s));
        FOLTY_LAUNCH(k_store_hist, grid_for(2 * (int64_t)S + 1, T, 2), T, 0, s, cnt, S, passes, hist);
        const StoreSortArgs sa{cw, g->in_t, g->tmin, m, cbits, hist, (uint32_t*)g->T, g->sd, nullptr, mk};
        store_sort(sc, sa);
        if (eager) {
            g->perm = graph_alloc<int32_t>(g, mk, s);
            StoreSortArgs pa = sa;
            pa.perm = g->perm;
            perm_sort(sc, pa);
        } else {
            g->cw = cw;
            g->store_hist = hist;
            g->store_cbits = cbits;
        }
        return;
    }
    g->perm = graph_alloc<int32_t>(g, mk, s);
    // the whole store, beside the peeling: its pair words and time offsets (4 B slot and
    // 8 B time read, 12 B written per input edge) and the sorted arrays (the word and the
    // time read, perm, T and sd written: 24 B per kept edge); the sort passes inside are
    // also SORT spans
    StageSpan span(ST_STORE, s, 24 * m + 24 * mk);
    // edges by (pair id, direction, time rank), sorted on the id and direction bits; a
    // 32-bit store carries each edge's time offset through the sort as its value
    uint64_t* packed = sc.get<uint64_t>(m);
    uint64_t* packed_alt = sc.get<uint64_t>(m);
    uint32_t* tv = g->ts32 ? sc.get<uint32_t>(m) : nullptr;
    uint32_t* tv_alt = g->ts32 ? sc.get<uint32_t>(m) : nullptr;
    FOLTY_CUDA(cudaMemsetAsync(sigma, 0, sizeof(int32_t) * (size_t)S, s));
    FOLTY_LAUNCH(k_pair_pack, (unsigned)((m + T - 1) / T), T, 0, s, job.slotw, job.order, m, job.sid, S, ib, packed,
                 g->in_t, g->tmin, tv, sigma);
    FOLTY_CUDA(cudaEventRecord(packed_ev, s));
    const bool palt = g->ts32 ? radix_sort_pairs(sc, packed, packed_alt, tv, tv_alt, m, ib, cbits)
                              : radix_sort_keys(sc, packed, packed_alt, m, ib, cbits);
    const uint64_t* sp = palt ? packed_alt : packed;
    FOLTY_CUDA(cudaMemsetAsync(g->seg, 0xff, sizeof(int32_t) * (2 * (size_t)S + 1), s));
    if (g->ts32)
        FOLTY_LAUNCH(k_pair_store4, (unsigned)(((mk + 3) / 4 + T - 1) / T), T, 0, s, sp, job.order, mk, S, ib,
                     palt ? tv_alt : tv, g->perm, (uint32_t*)g->T, g->sd, g->seg);
    else
        FOLTY_LAUNCH((k_pair_store<int64_t, false>), grid_for(mk, T), T, 0, s, sp, job.order, mk, S, ib, g->in_t,
                     g->perm, (int64_t*)g->T, g->sd, g->seg);
    FOLTY_LAUNCH(k_segments_fix, grid_for(S, T), T, 0, s, S, mk, g->seg);
}

// A1 with dense pair ids (see k_pair_insert) up to the static edge list (ea, eb) and
// the job of the temporal store: false, with nothing of the graph written, when the
// table cannot serve (too many distinct pairs, a probe sequence ran out, or ids and
// time ranks do not fit one word); FOLTY_PAIR_SORT=keys forces that answer. The
// distinct-pair sort is checked by the next read-back (before any of its consumers but
// the guarded k_pair_ids index with it).
static bool pair_ids_sort(folty_graph* g, Scratch& sc, const uint32_t* order, cudaStream_t s, StoreJob* job) {
    const int T = 256;
    const int64_t m = g->m, mk = g->m_kept;
    const int32_t n = g->n;
    if (pair_table_forced_off()) return false;
    if (mk == 0 || n < 2) return false;
    const int ib = bit_length((uint64_t)(m - 1));
    const int lg_max = pair_table_lg_max(m);
    int lg = pair_table_lg_first(m);
    int64_t tb = 0, S64 = 0;
    int cap = 0;
    uint64_t* table = nullptr;
    uint64_t* urank = nullptr;
    uint32_t* uslot = nullptr;
    // the first try's table, slot words and flags ([0] a probe ran out, [1] distinct
    // pairs) may already be filled by the load
    const bool pre = g->pre_table != nullptr && g->pre_lg == lg;
    int* flags = pre ? g->pre_flags : sc.get<int>(2);
    uint32_t* slotw = pre ? g->pre_slotw : sc.get<uint32_t>(m);
    bool first = true;
    while (true) {
        tb = 1ll << lg;
        cap = (int)(tb / 2);  // load factor at most 1/2
        if (first && pre) {
            table = g->pre_table;
        } else {
            table = sc.get<uint64_t>(tb);
            FOLTY_CUDA(cudaMemsetAsync(table, 0, sizeof(uint64_t) * (size_t)tb, s));
            FOLTY_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
            FOLTY_LAUNCH(k_pair_insert, grid_for(m, T), T, 0, s, g->in_src, g->in_dst, m, n, table, lg, slotw, flags);
        }
        first = false;
        urank = sc.get<uint64_t>(cap);
        uslot = sc.get<uint32_t>(cap);
        FOLTY_LAUNCH(k_pair_table_compact, grid_for(tb, (int64_t)T * PAIR_COMPACT_ITEMS), T, 0, s, table, tb, urank, uslot,
                     flags + 1, cap);
        const void* ptrs[2] = {flags, flags + 1};
        int sizes[2] = {4, 4};
        int64_t fv[2];
        read_back(g, ptrs, sizes, 2, fv, s);
        S64 = fv[1];
        if (fv[0] == 0 && S64 <= cap) break;
        if (lg == lg_max) return false;
        lg = lg_max;
    }
    if (bit_length((uint64_t)(2 * S64)) + ib > 64) return false;
    const int32_t S = (int32_t)S64;
    // the distinct pairs in (a, b) order: ids, ends
    uint64_t* urank_alt = sc.get<uint64_t>(S);
    uint32_t* uslot_alt = sc.get<uint32_t>(S);
    const int rank_bits = bit_length((uint64_t)n * (uint64_t)(n - 1) / 2);
    const bool ualt = radix_sort_pairs(sc, urank, urank_alt, uslot, uslot_alt, S, rank_bits);
    const uint64_t* ur = ualt ? urank_alt : urank;
    const uint32_t* us = ualt ? uslot_alt : uslot;
    g->S = S;
    g->ea = graph_alloc<int32_t>(g, S, s);
    g->eb = graph_alloc<int32_t>(g, S, s);
    g->seg = graph_alloc<int32_t>(g, 2 * (int64_t)S + 1, s);
    int32_t* sid = sc.get<int32_t>(tb);
    FOLTY_LAUNCH(k_pair_ids, grid_for(S, T), T, 0, s, ur, us, S, n, tb, sid, g->ea, g->eb);
    *job = StoreJob{slotw, order, sid, ib};
    return true;
}

// A1 with the full pair key (2 p(a, b) + direction, see k_build_keys) and the input
// index (or time rank) as the value.
static void pair_key_sort(folty_graph* g, Scratch& sc, const uint32_t* order, cudaStream_t s) {
    const int T = 256;
    const int64_t m = g->m, mk = g->m_kept;
    const int32_t n = g->n;
    const int key_bits = n > 1 ? bit_length((uint64_t)n * (uint64_t)(n - 1)) : 1;  // keys < n (n - 1)
    const uint64_t loop_key = (key_bits >= 64) ? ~0ull : ((1ull << key_bits) - 1);
    g->perm = graph_alloc<int32_t>(g, mk, s);
    uint64_t* key = sc.get<uint64_t>(m);
    uint64_t* key_alt = sc.get<uint64_t>(m);
    uint32_t* val = sc.get<uint32_t>(m);
    uint32_t* val_alt = sc.get<uint32_t>(m);
    FOLTY_LAUNCH(k_build_keys, grid_for(m, T), T, 0, s, g->in_src, g->in_dst, m, n, loop_key, key, val);
    uint64_t* skey = key;
    uint32_t* sval = val;
    if (order) {
        // keys in time order, values the input indices: the stable sort keeps time order
        FOLTY_LAUNCH(k_gather_keys, grid_for(m, T), T, 0, s, key, order, m, key_alt);
        FOLTY_CUDA(cudaMemcpyAsync(val, order, sizeof(uint32_t) * (size_t)m, cudaMemcpyDeviceToDevice, s));
        const bool alt = radix_sort_pairs(sc, key_alt, key, val, val_alt, m, key_bits);
        skey = alt ? key : key_alt;
        sval = alt ? val_alt : val;
    } else {
        const bool alt = radix_sort_pairs(sc, key, key_alt, val, val_alt, m, key_bits);
        skey = alt ? key_alt : key;
        sval = alt ? val_alt : val;
    }
    sort_check(g, s);
    int32_t* newpair = sc.get<int32_t>(mk + 1);
    int32_t* pscan = sc.get<int32_t>(mk + 1);
    // 32-bit offsets of the input timestamps, written right before the gather so that
    // they are still in L2 there
    uint32_t* t32 = (g->ts32 && mk > 0) ? sc.get<uint32_t>(m) : nullptr;
    if (mk > 0) {
        if (t32) FOLTY_LAUNCH(k_offsets32, grid_for(m, T), T, 0, s, g->in_t, m, g->tmin, t32);
        if (g->ts32)
            FOLTY_LAUNCH(k_store<uint32_t>, grid_for(mk, T), T, 0, s, skey, sval, t32, mk, g->perm, (uint32_t*)g->T,
                         newpair);
        else
            FOLTY_LAUNCH(k_store<int64_t>, grid_for(mk, T), T, 0, s, skey, sval, g->in_t, mk, g->perm, (int64_t*)g->T,
                         newpair);
    }
    exclusive_scan(sc, newpair, pscan, mk);
    const int32_t S = read_i32(g, pscan + mk, s);
    g->S = S;
    g->ea = graph_alloc<int32_t>(g, S, s);
    g->eb = graph_alloc<int32_t>(g, S, s);
    g->seg = graph_alloc<int32_t>(g, 2 * (int64_t)S + 1, s);
    if (mk > 0) {
        FOLTY_LAUNCH(k_segments, grid_for(mk, T), T, 0, s, skey, newpair, pscan, mk, g->sd, g->seg);
        FOLTY_LAUNCH(k_pair_ends, grid_for(S, T), T, 0, s, skey, g->seg, S, n, g->ea, g->eb);
        FOLTY_LAUNCH(k_segments_split, grid_for(mk, T), T, 0, s, g->sd, mk, S, g->seg);
        FOLTY_LAUNCH(k_segments_fix, grid_for(S, T), T, 0, s, S, mk, g->seg);
    } else {
        FOLTY_CUDA(cudaMemsetAsync(g->seg, 0, sizeof(int32_t), s));
    }
}

// The counting pass of the triangle listing (tcnt per oriented edge; merged list entries
// and probe slots into merged[0], merged[1], zeroed here) under the graph's split between
// one thread and one warp per oriented edge: forced, cached under the graph's statistics,
// or picked by timing the pass under each candidate split. All candidates count the same
// triangles, so the last trial's outputs stand. trials_only: the trials (when the split
// is neither forced nor cached) and nothing else, for a listing without counting pass.
static void tune_triangles(folty_graph* g, const int32_t* outptr, const int32_t* out_nbr, const int32_t* out_src,
                           const int32_t* osig, int32_t* tcnt, int64_t* pcnt, unsigned long long* merged,
                           cudaStream_t s, bool trials_only) {
    const int32_t S = g->S;
    const unsigned grid = grid_for(S, TRI_THREADS);
    const std::vector<int64_t> key{g->n, g->m_kept, S};
    bool trials = !(tune_forced(&g->tune, false) || tune_lookup(key, &g->tune, false)) && !profiling_on();
    if (!trials && trials_only) return;
    if (!trials) {
        FOLTY_CUDA(cudaMemsetAsync(merged, 0, 2 * sizeof(unsigned long long), s));
        FOLTY_LAUNCH(k_tri_count, grid, TRI_THREADS, 0, s, outptr, out_nbr, out_src, osig, S, tcnt, pcnt, merged,
                     merged + 1, g->tune.tri_heavy);
        return;
    }
    cudaEvent_t ev[TUNE_TRIALS + 1];
    for (auto& e : ev) FOLTY_CUDA(cudaEventCreate(&e));
    int best = 1;
    try {
        for (int c = 0; c < TUNE_TRIALS; c++) {
            FOLTY_CUDA(cudaMemsetAsync(merged, 0, 2 * sizeof(unsigned long long), s));
            FOLTY_CUDA(cudaEventRecord(ev[0], s));
            FOLTY_LAUNCH(k_tri_count, grid, TRI_THREADS, 0, s, outptr, out_nbr, out_src, osig, S, tcnt, pcnt, merged,
                         merged + 1, TRI_HEAVY_CAND[c]);
            FOLTY_CUDA(cudaEventRecord(ev[c + 1], s));
            FOLTY_CUDA(cudaEventSynchronize(ev[c + 1]));
            FOLTY_CUDA(cudaEventElapsedTime(&g->tune.tri_ms[c], ev[0], ev[c + 1]));
            if (g->tune.tri_ms[c] < g->tune.tri_ms[best]) best = c;
        }
    } catch (...) {
        for (auto& e : ev) cudaEventDestroy(e);
        throw;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    g->tune.tri_heavy = TRI_HEAVY_CAND[best];
    g->tune.tri_source = 1;
    tune_store(key, g->tune, false);
}

void ensure_perm(folty_graph* g, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g->perm_mu);
    if (g->perm) {
        if (g->perm_ev) FOLTY_CUDA(cudaStreamWaitEvent(s, g->perm_ev, 0));
        return;
    }
    if (!g->cw) fail(FOLTY_EINVAL, "graph has no store to order");
    int32_t* perm = graph_alloc<int32_t>(g, g->m_kept, s);
    Scratch sc(g->alloc, s, g->dev_err);
    perm_sort(sc, StoreSortArgs{g->cw, nullptr, 0, g->m, g->store_cbits, g->store_hist, nullptr, nullptr, perm,
                                g->m_kept});
    FOLTY_CUDA(cudaEventCreateWithFlags(&g->perm_ev, cudaEventDisableTiming));
    FOLTY_CUDA(cudaEventRecord(g->perm_ev, s));
    g->perm = perm;
}

static void preprocess_on(folty_graph* g, cudaStream_t s) {
    const int T = 256;
    const int64_t m = g->m;
    const int32_t n = g->n;
    Scratch sc(g->alloc, s, g->dev_err);

    // ---------------- A1: canonical order
    const int nb = bit_length((uint64_t)(n > 1 ? n - 1 : 1));
    const int64_t mk = g->m_kept;
    // 32-bit offsets from tmin when the time range leaves room for the "none" marker
    g->ts32 = (g->tmax - g->tmin) < (int64_t)0xffffffffll;
    if (g->ts32) g->T = graph_alloc<uint32_t>(g, mk, s);
    else g->T = graph_alloc<int64_t>(g, mk, s);
    g->sd = graph_alloc<int32_t>(g, mk, s);
    // time order of an input that is not sorted by time (stable): order[j] = input index
    uint32_t* order = nullptr;
    if (!g->info.time_sorted && m > 1) {
        uint64_t* tk = sc.get<uint64_t>(m);
        uint64_t* tk_alt = sc.get<uint64_t>(m);
        uint32_t* iv = sc.get<uint32_t>(m);
        uint32_t* iv_alt = sc.get<uint32_t>(m);
        FOLTY_LAUNCH(k_time_keys, grid_for(m, T), T, 0, s, g->in_t, m, g->tmin, tk, iv);
        const bool alt = radix_sort_pairs(sc, tk, tk_alt, iv, iv_alt, m, bit_length((uint64_t)(g->tmax - g->tmin)));
        sort_check(g, s);
        order = alt ? iv_alt : iv;
    }
    StoreJob job{};
    const bool ids = pair_ids_sort(g, sc, order, s, &job);
    if (!ids) pair_key_sort(g, sc, order, s);
    const int32_t S = g->S;
    // the temporal store of the dense-id path: on a side stream of default priority from
    // the end of the grid peel on (beside the rest of the peel and the triangle passes,
    // which run on streams of the highest priority and take SMs first), joined after the
    // triangle passes (which need only its per-pair counts). On an error in between, the
    // side streams are drained before the call's buffers go.
    SideStream side(s, false);
    SideStream hi(s, true);
    struct EventHolder {
        cudaEvent_t e = nullptr;
        ~EventHolder() {
            if (e) cudaEventDestroy(e);
        }
    } packed_ev;
    int32_t* sigma = nullptr;
    cudaStream_t store_s = nullptr;
    if (ids) {
        FOLTY_CUDA(cudaEventCreateWithFlags(&packed_ev.e, cudaEventDisableTiming));
        sigma = sc.get<int32_t>(S > 0 ? S : 1);
    }

    // ---------------- A2: static CSR
    // static edges are sorted by (a, b); a stable sort by b lists them by (b, a)
    uint32_t* by_b = nullptr;
    if (S > 0) {
        uint64_t* bk = sc.get<uint64_t>(S);
        uint64_t* bk_alt = sc.get<uint64_t>(S);
        uint32_t* bv = sc.get<uint32_t>(S);
        uint32_t* bv_alt = sc.get<uint32_t>(S);
        FOLTY_LAUNCH(k_edge_keys_b, grid_for(S, T), T, 0, s, g->eb, S, bk, bv);
        bool alt = radix_sort_pairs(sc, bk, bk_alt, bv, bv_alt, S, nb);
        by_b = alt ? bv_alt : bv;
        sort_check(g, s);
    }
    g->by_b = graph_alloc<int32_t>(g, S, s);
    if (S > 0) FOLTY_CUDA(cudaMemcpyAsync(g->by_b, by_b, sizeof(int32_t) * (size_t)S, cudaMemcpyDeviceToDevice, s));
    int32_t* runs = sc.get<int32_t>(4 * ((int64_t)n + 1));  // hi_first, hi_last, lo_first, lo_last
    int32_t* hi_first = runs;
    int32_t* hi_last = runs + (n + 1);
    int32_t* lo_first = runs + 2 * ((int64_t)n + 1);
    int32_t* lo_last = runs + 3 * ((int64_t)n + 1);
    FOLTY_CUDA(cudaMemsetAsync(runs, 0, sizeof(int32_t) * 4 * ((size_t)n + 1), s));
    if (S > 0) {
        FOLTY_LAUNCH(k_runs, grid_for(S, T), T, 0, s, g->ea, (const uint32_t*)nullptr, S, hi_first, hi_last);
        FOLTY_LAUNCH(k_runs, grid_for(S, T), T, 0, s, g->eb, by_b, S, lo_first, lo_last);
    }
    int32_t* deg_lo = sc.get<int32_t>((int64_t)n + 1);
    g->deg = graph_alloc<int32_t>(g, (int64_t)n + 1, s);
    FOLTY_LAUNCH(k_degrees, grid_for(n, T), T, 0, s, hi_first, hi_last, lo_first, lo_last, (int64_t)n, deg_lo,
                 g->deg);
    int32_t* rowptr = sc.get<int32_t>((int64_t)n + 1);
    exclusive_scan(sc, g->deg, rowptr, n);
    const int64_t n2 = 2 * (int64_t)S;
    int32_t* adj = sc.get<int32_t>(n2);
    int32_t* adj_eid = sc.get<int32_t>(n2);
    int32_t* adj_src = sc.get<int32_t>(n2);
    if (S > 0)
        FOLTY_LAUNCH(k_fill_adj, grid_for(S, T), T, 0, s, g->ea, g->eb, S, rowptr, deg_lo, hi_first, lo_first,
                     by_b, adj, adj_eid, adj_src);

    // ---------------- A3: peeling
    int* peel_ctl = nullptr;
    g->core = graph_alloc<int32_t>(g, n, s);
    int32_t* core = g->core;
    int32_t* rnd = sc.get<int32_t>(n);
    {
        PeelArgs pa;
        pa.rowptr = rowptr;
        pa.adj = adj;
        pa.n = n;
        pa.deg = sc.get<int32_t>(n);
        FOLTY_CUDA(cudaMemcpyAsync(pa.deg, g->deg, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        FOLTY_CUDA(cudaMemsetAsync(rnd, 0xff, sizeof(int32_t) * (size_t)n, s));
        pa.rnd = rnd;
        pa.core = core;
        pa.alive[0] = sc.get<int32_t>(n);
        pa.alive[1] = sc.get<int32_t>(n);
        pa.fr[0] = sc.get<int32_t>(n);
        pa.fr[1] = sc.get<int32_t>(n);
        pa.hcap = (int32_t)((int64_t)n + (2 * (int64_t)S) / PEEL_PIECE + 1);
        pa.hr[0] = sc.get<int64_t>(pa.hcap);
        pa.hr[1] = sc.get<int64_t>(pa.hcap);
        pa.ctl = sc.get<int>(C_SLOTS);
        pa.timeout_ns = 10ll * 1000 * 1000 * 1000;
        const int tail_c = tail_cluster_size(s);
        pa.tail_n = TAIL_OWN * tail_c;
        int init[C_SLOTS] = {0};
        init[C_MIN] = INT_MAX;
        init[C_MIN + 1] = INT_MAX;
        int* init_dev = (int*)(g->host_stage + READBACK_MAX + 16);  // pinned staging
        std::memcpy(init_dev, init, sizeof(init));
        g->stage_busy = 1;
        FOLTY_CUDA(cudaMemcpyAsync(pa.ctl, init_dev, sizeof(init), cudaMemcpyHostToDevice, s));
        FOLTY_LAUNCH(k_iota, grid_for(n, T), T, 0, s, pa.alive[0], (int64_t)n);
        int per_sm = 0;
        FOLTY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel, PEEL_THREADS, 0));
        if (per_sm < 1) fail(FOLTY_ECUDA, "peeling kernel cannot be resident");
        if (per_sm > 1) per_sm = 1;
        dim3 grid(num_sms() * per_sm), block(PEEL_THREADS);
        void* args[] = {&pa};
        StageSpan span(ST_PEEL, s, 12 * 2 * (int64_t)S + 16 * (int64_t)n);
        if (n > 0) {
            FOLTY_CUDA(cudaLaunchCooperativeKernel((const void*)k_peel, grid, block, args, 0, s));
            after_launch("k_peel");
        }
        // the store and, at the end of its stream, the run-ends table (ready when it is
        // joined), after the grid peel: the cooperative peel waits for SMs that the store's
        // blocks hold (it took 0.8 ms instead of 0.3 beside the store's first pass), and
        // the store still ends before the triangle listing
        if (ids) {
            store_s = side.fork();
            Scratch sc2(g->alloc, store_s, g->dev_err);
            temporal_store(g, job, sc2, sigma, packed_ev.e);
            build_run_ends(g, store_s);
        }
        if (n > 0) {
            // the cluster and single-CTA phases: latency-bound chains of small rounds, on
            // a high-priority side stream so that their blocks go first on SMs that the
            // temporal store's kernels free
            const cudaStream_t ts = hi.fork();
            Scratch sct(g->alloc, ts, g->dev_err);
            // cluster tail on the induced subgraph of the vertices the grid kernel left;
            // always enqueued (its kernels do nothing when the grid kernel finished), so
            // no host round trip separates the two
            const int tn = pa.tail_n;
            int32_t* L = sct.get<int32_t>(tn);
            int32_t* gmap = sct.get<int32_t>(n);
            int32_t* ld = sct.get<int32_t>(tn + 1);
            int32_t* d0 = sct.get<int32_t>(tn + 1);
            int32_t* lrow = sct.get<int32_t>(tn + 1);
            int32_t* eoff = sct.get<int32_t>(tn + 1);
            // zeroed together: the local vertex count, then the fill counters
            int32_t* zblk = sct.get<int32_t>(tn + 1);
            int* nl = zblk;
            int32_t* fillc = zblk + 1;
            uint32_t* ladj = sct.get<uint32_t>(2 * (int64_t)S);
            FOLTY_CUDA(cudaMemsetAsync(zblk, 0, sizeof(int32_t) * (size_t)(tn + 1), ts));
            FOLTY_LAUNCH(k_tail_select, grid_for(n, T), T, 0, ts, pa.alive[0], pa.alive[1], pa.ctl, rnd, tn, L, gmap,
                         nl, pa.ctl + C_ERR);
            FOLTY_LAUNCH(k_tail_degrees, grid_for(tn, T), T, 0, ts, L, nl, pa.deg, rowptr, tn, ld, d0);
            exclusive_scan(sct, ld, lrow, tn);
            exclusive_scan(sct, d0, eoff, tn);
            FOLTY_LAUNCH(k_tail_fill, grid_for(2 * (int64_t)S, T), T, 0, ts, L, eoff, tn, rowptr, adj, rnd, gmap,
                         lrow, ld, fillc, ladj, pa.ctl + C_ERR);
            // single-CTA phase for the last SOLO_CAP vertices (does nothing unless the
            // cluster hands off)
            // zeroed together: the exported count, the degrees, the fill counters
            int32_t* sblk = sct.get<int32_t>(1 + (SOLO_CAP + 1) + SOLO_CAP);
            int* ns = sblk;
            int32_t* sdeg = sblk + 1;
            int32_t* fc = sdeg + (SOLO_CAP + 1);
            int32_t* slist = sct.get<int32_t>(SOLO_CAP);
            int32_t* srow = sct.get<int32_t>(SOLO_CAP + 1);
            int32_t* dl = sct.get<int32_t>(SOLO_CAP + 1);
            int32_t* eo = sct.get<int32_t>(SOLO_CAP + 1);
            int32_t* sgid = sct.get<int32_t>(SOLO_CAP);
            int32_t* map2 = sct.get<int32_t>(tn);
            uint16_t* sadj = sct.get<uint16_t>(2 * (int64_t)S);
            FOLTY_CUDA(cudaMemsetAsync(sblk, 0, sizeof(int32_t) * (size_t)(1 + (SOLO_CAP + 1) + SOLO_CAP), ts));
            FOLTY_CUDA(cudaMemsetAsync(map2, 0xff, sizeof(int32_t) * (size_t)tn, ts));
            int32_t* tdec = sct.get<int32_t>((int64_t)TAIL_OWN * tail_c);
            FOLTY_CUDA(cudaMemsetAsync(tdec, 0, sizeof(int32_t) * (size_t)TAIL_OWN * (size_t)tail_c, ts));
            TailArgs ta{nl, L, ld, lrow, ladj, rnd, core, pa.ctl, SOLO_CAP, ns, slist, sdeg, map2, tdec};
            if (tail_c == 16) launch_tail<16>(ta, ts);
            else launch_tail<8>(ta, ts);
            FOLTY_LAUNCH(k_solo_rows, grid_for(SOLO_CAP, T), T, 0, ts, pa.ctl, ns, slist, lrow, L, dl, sgid);
            exclusive_scan(sct, sdeg, srow, SOLO_CAP);
            exclusive_scan(sct, dl, eo, SOLO_CAP);
            FOLTY_LAUNCH(k_solo_fill, grid_for(2 * (int64_t)S, T), T, 0, ts, pa.ctl, eo, slist, sdeg, srow, lrow, ladj,
                         map2, fc, sadj, pa.ctl + C_ERR);
            launch_solo(SoloArgs{ns, sdeg, fc, srow, sadj, sgid, rnd, core, pa.ctl}, ts);
            hi.join();
        }
        peel_ctl = pa.ctl;  // rounds, alpha and the error word are read with the triangle totals
    }

    // ---------------- A4: orientation
    int* stat = sc.get<int>(4);  // max degree, max out-degree, max sigma, (pad)
    FOLTY_CUDA(cudaMemsetAsync(stat, 0, sizeof(int) * 4, s));
    int32_t* oflag = sc.get<int32_t>(n2 + 1);
    int32_t* opos = sc.get<int32_t>(n2 + 1);
    if (n2 > 0) FOLTY_LAUNCH(k_orient_flags, grid_for(n2, T), T, 0, s, adj_src, adj, rnd, n2, oflag);
    exclusive_scan(sc, oflag, opos, n2);
    int32_t* outptr = sc.get<int32_t>((int64_t)n + 1);
    FOLTY_LAUNCH(k_outptr, grid_for((int64_t)n + 1, T), T, 0, s, rowptr, opos, (int64_t)n, outptr, stat + 1);
    int32_t* out_nbr = sc.get<int32_t>(S);
    int32_t* out_eid = sc.get<int32_t>(S);
    int32_t* out_src = sc.get<int32_t>(S);
    if (n2 > 0)
        FOLTY_LAUNCH(k_orient_fill, grid_for(n2, T), T, 0, s, adj_src, adj, adj_eid, oflag, opos, n2, out_nbr,
                     out_eid, out_src);

    // ---------------- A5: triangles
    // the triangle listing needs the static graph and every static edge's temporal edge
    // count, not the store itself: it runs beside the store's sort (joined before the
    // run-ends table)
    if (ids) FOLTY_CUDA(cudaStreamWaitEvent(s, packed_ev.e, 0));
    g->common = graph_alloc<int32_t>(g, S, s);
    FOLTY_CUDA(cudaMemsetAsync(g->common, 0, sizeof(int32_t) * ((size_t)S > 0 ? (size_t)S : 1), s));
    int32_t* tcnt = sc.get<int32_t>((int64_t)S + 1);
    int64_t* toff = sc.get<int64_t>((int64_t)S + 1);
    unsigned long long* merged = sc.get<unsigned long long>(2);  // list lengths merged, probe slots
    FOLTY_CUDA(cudaMemsetAsync(merged, 0, 2 * sizeof(unsigned long long), s));
    int32_t* osig = sc.get<int32_t>(S);
    if (S > 0) FOLTY_LAUNCH(k_out_sigma, grid_for(S, T), T, 0, s, sigma, g->seg, out_eid, S, osig, stat + 2);
    FOLTY_LAUNCH(k_max_i32, grid_for(n, T), T, 0, s, g->deg, (int64_t)n, stat + 0);
    // the all-roles probe map (each triangle's first slot in the flat space of every
    // role's probes, and the tile starts) serves only the allocation-free per-edge counts,
    // which take graphs of at most FOLTY_NOALLOC_MAX_EDGES edges; the queries lay out the
    // kept roles of their own selection
    const bool probe_map = g->m_kept <= FOLTY_NOALLOC_MAX_EDGES;
    int64_t* pcnt = probe_map ? sc.get<int64_t>((int64_t)S + 1) : nullptr;  // slots per oriented edge, then prefix
    // Larger graphs list their triangles in one pass into a bounded layout (the triangles
    // of oriented edge (u, v) from the prefix of the bounds min(|N+(u)|, |N+(v)|) on)
    // that the liveness pass makes dense while it computes the out motif's bytes: no
    // counting pass before the listing, and no wait for its total. The probe map needs
    // the counting pass's slots per edge, and a bound past TRI_BOUND_MAX_BYTES takes the
    // counting pass too.
    bool bounded = !probe_map && S > 0 && !tri_layout_counted();
    int64_t* boff = nullptr;
    std::optional<StageSpan> tri_span;
    int4* tri_b = nullptr;  // the bounded layout, moved into g->tri by the liveness pass
    TriLayout layout{};
    if (bounded) {
        boff = sc.get<int64_t>((int64_t)S + 1);
        FOLTY_LAUNCH(k_tri_bound, grid_for(S, T), T, 0, s, outptr, out_src, out_nbr, S, boff);
        exclusive_scan(sc, boff, boff, S);
    }
    // the counting pass merges the two out-lists of every oriented edge: 4 B per merged
    // entry (known after its read-back) + 8 B per static edge
    std::optional<StageSpan> count_span;
    auto count_pass = [&]() {
        count_span.emplace(ST_TRIANGLES, s, 8 * (int64_t)S);
        FOLTY_CUDA(cudaMemsetAsync(merged, 0, 2 * sizeof(unsigned long long), s));
        if (S > 0) tune_triangles(g, outptr, out_nbr, out_src, osig, tcnt, pcnt, merged, s, false);
        exclusive_scan(sc, tcnt, toff, S);
        if (probe_map) exclusive_scan(sc, pcnt, pcnt, S);
        count_span->end();
    };
    auto counted = [&](int64_t total, int64_t list_len, int64_t probes) {
        g->ntri = total;
        g->info.probes = probes;
        g->enum_bytes = 4 * list_len + 8 * (int64_t)S;
        count_span->add_bytes(4 * list_len);
    };
    if (!bounded) count_pass();
    int64_t bound = 0;
    {
        const void* ptrs[9] = {bounded ? (const void*)(boff + S) : (const void*)(toff + S), stat + 0, stat + 1,
                               stat + 2, merged, merged + 1, peel_ctl + C_ERR, peel_ctl + C_ROUNDS, peel_ctl + C_ALPHA};
        int sizes[9] = {8, 4, 4, 4, 8, 8, 4, 4, 4};
        int64_t outv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        read_back(g, ptrs, sizes, peel_ctl ? 9 : 6, outv, s);  // no peeling state for n = 0
        if (outv[6] == 1) fail(FOLTY_ETIMEOUT, "peeling: a grid barrier wait ran out");
        if (outv[6] != 0)
            fail(FOLTY_ECUDA, "peeling: internal error " + std::to_string(outv[6]) +
                                  " (2: a vertex list overflowed, 3/4: a subgraph row count differs, 5: a row entry "
                                  "is out of range)");
        g->info.peel_rounds = (int32_t)outv[7];
        g->info.degeneracy = (int32_t)outv[8];
        g->info.max_degree = (int32_t)outv[1];
        g->info.max_out_degree = (int32_t)outv[2];
        g->info.sigma_max = (int32_t)outv[3];
        if (bounded) bound = outv[0];
        else counted(outv[0], outv[4], outv[5]);
    }
    if (bounded && bound > TRI_BOUND_MAX_BYTES / (int64_t)sizeof(int4)) {
        bounded = false;
        count_pass();
        const void* ptrs[3] = {toff + S, merged, merged + 1};
        int sizes[3] = {8, 8, 8};
        int64_t outv[3] = {0, 0, 0};
        read_back(g, ptrs, sizes, 3, outv, s);
        counted(outv[0], outv[1], outv[2]);
    }
    if (bounded) {
        // the autotuner's trials (the first graph of its size only) time the counting pass
        tune_triangles(g, outptr, out_nbr, out_src, osig, tcnt, pcnt, merged, s, true);
        tri_b = sc.get<int4>(bound);
        // the graph's array holds bound entries, the first ntri of them the triangles
        // (moved there by the liveness pass): an array of ntri would wait for the
        // listing's total, a host round trip
        g->tri = graph_alloc<int4>(g, bound, s);
        g->tri_off = nullptr;
        FOLTY_CUDA(cudaMemsetAsync(merged, 0, 2 * sizeof(unsigned long long), s));
        // the listing (8 B per static edge + 4 B per merged entry + 16 B per triangle):
        // the totals come with the read-back after the store's join
        tri_span.emplace(ST_TRIANGLES, s, 8 * (int64_t)S);
        // one warp per 32 oriented edges, in short blocks: the dense communities' edges
        // take far longer than the rest
        FOLTY_LAUNCH((k_tri_write<false, true>), (unsigned)((S + TRI_THREADS - 1) / TRI_THREADS), TRI_THREADS, 0, s,
                     outptr, out_nbr,
                     out_eid, out_src, osig, S, boff, nullptr, tri_b, nullptr, g->common, g->tune.tri_heavy, tcnt,
                     merged);
        exclusive_scan(sc, tcnt, toff, S);
        tri_span->end();
        layout = TriLayout{tcnt, toff, boff, tri_b};
    } else {
        const int64_t ntri = g->ntri;
        g->tri = graph_alloc<int4>(g, ntri, s);
        g->tri_off = probe_map ? graph_alloc<int64_t>(g, ntri + 1, s) : nullptr;
        if (S > 0) {
            // the listing pass merges the same lists and writes 16 + 8 B per triangle
            StageSpan span(ST_TRIANGLES, s, g->enum_bytes + (probe_map ? 24 : 16) * ntri);
            if (probe_map)
                FOLTY_LAUNCH(k_tri_write<true>, grid_for(S, TRI_THREADS), TRI_THREADS, 0, s, outptr, out_nbr, out_eid,
                             out_src, osig, S, toff, pcnt, g->tri, g->tri_off, g->common, g->tune.tri_heavy);
            else
                FOLTY_LAUNCH(k_tri_write<false>, grid_for(S, TRI_THREADS), TRI_THREADS, 0, s, outptr, out_nbr,
                             out_eid, out_src, osig, S, toff, pcnt, g->tri, g->tri_off, g->common, g->tune.tri_heavy);
        }
        // the probe offsets of the triangles come from the writing pass; the last entry is the total
        if (probe_map)
            FOLTY_CUDA(cudaMemcpyAsync(g->tri_off + ntri, pcnt + S, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    }
    if (ids) side.join();
    if (bounded) {
        // the listing's totals; the same read-back checks the store's sort, which completed
        // before its arrays index anything
        const void* ptrs[3] = {toff + S, merged, merged + 1};
        int sizes[3] = {8, 8, 8};
        int64_t outv[3] = {0, 0, 0};
        read_back(g, ptrs, sizes, 3, outv, s);
        g->ntri = outv[0];
        g->info.probes = outv[2];
        g->enum_bytes = 4 * outv[1] + 8 * (int64_t)S;
        tri_span->add_bytes(g->enum_bytes - 8 * (int64_t)S + 16 * g->ntri);
    } else if (ids) {
        sort_check(g, s);  // the store's sort completed before its arrays index anything
    }
    // the raw input is no longer needed
    graph_release(g, g->in_src, s);
    graph_release(g, g->in_dst, s);
    graph_release(g, g->in_t, s);
    g->in_src = g->in_dst = nullptr;
    g->in_t = nullptr;
    // and neither is the pair table the load filled
    graph_release(g, g->pre_table, s);
    graph_release(g, g->pre_slotw, s);
    graph_release(g, g->pre_flags, s);
    g->pre_table = nullptr;
    g->pre_slotw = nullptr;
    g->pre_flags = nullptr;
    // the run-ends table (built beside the triangle passes with the store) and every
    // triangle's liveness bytes
    if (!ids) build_run_ends(g, s);
    prepare_liveness(g, s);
    triangle_liveness(g, s, bounded ? &layout : nullptr);
    g->info.triangles = g->ntri;
    // tile -> first triangle map of the all-roles probe kernel (query independent)
    g->n_tiles = probe_map ? (g->info.probes + PB_TILE - 1) / PB_TILE : 0;
    g->tile_tri = probe_map ? graph_alloc<int64_t>(g, g->n_tiles + 1, s) : nullptr;
    if (probe_map && g->info.probes > 0)
        FOLTY_LAUNCH(k_tile_starts, grid_for(g->n_tiles + 1, T), T, 0, s, g->tri_off, g->ntri, g->info.probes,
                     g->n_tiles, PB_TILE, g->tile_tri);
    g->prof_bytes = graph_alloc<unsigned long long>(g, PROF_SLOTS, s);
    g->info.static_edges = S;
    g->state = 1;
    FOLTY_CUDA(cudaStreamSynchronize(s));
}

// Preprocessing runs on a stream of the device's highest priority, forked from the
// caller's stream and joined back at the end. The temporal store runs beside the peel
// and the triangle passes on a stream of default priority (its kernels take one block
// per chunk of work, so their blocks retire quickly), and the chain that decides the
// preprocessing's length takes SMs first whenever blocks retire: measured with events on
// the paper-scale graph, the peel's set-up kernels and the orientation otherwise waited
// behind the store's kernels for ≈ 1 ms each.
void preprocess_graph(folty_graph* g, cudaStream_t s) {
    SideStream pri(s, true);
    preprocess_on(g, pri.fork());
    pri.join();
}

}  // namespace folty
