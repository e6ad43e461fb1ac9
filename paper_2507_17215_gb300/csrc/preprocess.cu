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
#include <climits>

#include "internal.cuh"
#include "probe.cuh"

namespace folty {

// ================================================================== A1

// Sort key of a temporal edge: (a, b, dir) with a = min, b = max id, dir = (src > dst).
// Self-loops get the all-ones key of the used width and sort last.
__global__ void k_build_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                             int64_t m, int nb, uint64_t loop_key, uint64_t* __restrict__ key,
                             uint32_t* __restrict__ val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = src[i], y = dst[i];
        uint64_t k;
        if (x == y) {
            k = loop_key;
        } else {
            uint64_t a = (uint64_t)min(x, y), b = (uint64_t)max(x, y);
            k = (a << (nb + 1)) | (b << 1) | (uint64_t)(x > y);
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

// perm, T, and the "new static pair" flag of every kept sorted position.
__global__ void k_store(const uint64_t* __restrict__ key, const uint32_t* __restrict__ order,
                        const int64_t* __restrict__ t, int64_t mk, int32_t* __restrict__ perm,
                        int64_t* __restrict__ T, int32_t* __restrict__ newpair) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t o = order[i];
        perm[i] = (int32_t)o;
        T[i] = t[o];
        newpair[i] = (i == 0) || ((key[i] >> 1) != (key[i - 1] >> 1));
    }
}

// Static edge ids, endpoints, segment starts. pscan = exclusive scan of newpair.
__global__ void k_segments(const uint64_t* __restrict__ key, const int32_t* __restrict__ newpair,
                           const int32_t* __restrict__ pscan, int64_t mk, int nb,
                           int32_t* __restrict__ sd, int32_t* __restrict__ ea,
                           int32_t* __restrict__ eb, int32_t* __restrict__ seg) {
    const uint64_t vmask = (nb >= 31) ? 0x7fffffffull : ((1ull << nb) - 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = key[i];
        int32_t s = pscan[i] + newpair[i] - 1;
        int dir = (int)(k & 1);
        sd[i] = 2 * s + dir;
        if (newpair[i]) {
            ea[s] = (int32_t)(k >> (nb + 1));
            eb[s] = (int32_t)((k >> 1) & vmask);
            seg[2 * s] = (int32_t)i;
            seg[2 * s + 1] = -1;
        }
    }
}

// seg[2s+1] = first b->a position of s, or the end of s when it has none.
__global__ void k_segments_split(const int32_t* __restrict__ sd, int64_t mk, int32_t S,
                                 int32_t* __restrict__ seg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = sd[i];
        if ((c & 1) && (i == 0 || sd[i - 1] != c)) seg[c] = (int32_t)i;  // c = 2s+1
    }
}

__global__ void k_segments_fix(int32_t S, int64_t mk, int32_t* __restrict__ seg) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (seg[2 * s + 1] < 0) seg[2 * s + 1] = (s + 1 < S) ? seg[2 * s + 2] : (int32_t)mk;
        if (s == 0) seg[2 * S] = (int32_t)mk;
    }
}

// ================================================================== A2

__global__ void k_count_degrees(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                                int32_t S, int32_t* __restrict__ deg_hi, int32_t* __restrict__ deg_lo) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&deg_hi[ea[s]], 1);  // s lists b > a in a's row
        atomicAdd(&deg_lo[eb[s]], 1);  // s lists a < b in b's row
    }
}

__global__ void k_add(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t n,
                      int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
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
                           int32_t* __restrict__ adj_eid) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S;
         j += (int64_t)gridDim.x * blockDim.x) {
        // upper part: static edges are sorted by (a, b)
        int32_t s = (int32_t)j;
        int32_t a = ea[s];
        int64_t p = (int64_t)rowptr[a] + deg_lo[a] + (s - hi_start[a]);
        adj[p] = eb[s];
        adj_eid[p] = s;
        // lower part: by_b lists static edges by (b, a)
        int32_t s2 = (int32_t)by_b[j];
        int32_t b = eb[s2];
        int64_t q = (int64_t)rowptr[b] + ((int32_t)j - lo_start[b]);
        adj[q] = ea[s2];
        adj_eid[q] = s2;
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

__global__ void k_max_sigma(const int32_t* __restrict__ seg, int32_t S, int* __restrict__ out) {
    int best = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x)
        best = max(best, seg[2 * s + 2] - seg[2 * s]);
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
    C_FCNT = 7,   // 3 slots
    C_ROUNDS = 10,
    C_ALPHA = 11,
    C_SLOTS = 16
};

struct PeelArgs {
    const int32_t* rowptr;
    const int32_t* adj;
    int32_t n;
    int32_t* deg;   // working copy of the degrees
    int32_t* rnd;   // removal round, -1 while alive
    int32_t* core;  // core number
    int32_t* alive[2];
    int32_t* fr[2];
    int* ctl;
    long long timeout_ns;
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
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)&ctl[C_ERR] == 0;
}

// Appends v for every lane with pred set; the whole warp must call it.
__device__ __forceinline__ void warp_append(bool pred, int32_t v, int32_t* out, int* counter) {
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (!mask) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) out[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

constexpr int PEEL_THREADS = 256;

// Parallel Matula-Beck peeling. Level k = smallest remaining degree; within a level,
// round after round, every remaining vertex of current degree <= k is removed at once
// and its neighbours' degrees drop. A vertex enters the next round exactly when its
// degree crosses k + 1 -> k. Each vertex gets core = k and the round it left in.
__global__ void __launch_bounds__(PEEL_THREADS) k_peel(PeelArgs a) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = gtid >> 5, nwarps = gsize >> 5;
    int* ctl = a.ctl;
    __shared__ int s_wmin[PEEL_THREADS / 32];
    int k = 0, r = 0, lvl = 0, ac = 0;
    int nalive = a.n;
    while (true) {
        // ---- P1: compact the alive list, find the minimum remaining degree
        if (gtid == 0) {
            ctl[C_MIN + ((lvl + 1) & 1)] = INT_MAX;
            ctl[C_ACNT + ((lvl + 1) & 1)] = 0;
        }
        int lmin = INT_MAX;
        const int32_t* acur = a.alive[ac];
        int32_t* anxt = a.alive[ac ^ 1];
        for (int64_t base = gwarp * 32; base < nalive; base += nwarps * 32) {
            int64_t i = base + lane;
            bool keep = false;
            int32_t v = 0;
            if (i < nalive) {
                v = __ldcg(&acur[i]);
                keep = __ldcg(&a.rnd[v]) < 0;
                if (keep) lmin = min(lmin, __ldcg(&a.deg[v]));
            }
            warp_append(keep, v, anxt, &ctl[C_ACNT + (lvl & 1)]);
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
        if (!grid_barrier(ctl, a.timeout_ns)) return;
        nalive = *(volatile int*)&ctl[C_ACNT + (lvl & 1)];
        if (nalive == 0) break;
        int mn = *(volatile int*)&ctl[C_MIN + (lvl & 1)];
        if (mn > k) k = mn;
        ac ^= 1;
        // ---- P2: the level's first frontier
        {
            const int32_t* al = a.alive[ac];
            int32_t* F = a.fr[r & 1];
            if (gtid == 0) ctl[C_FCNT + (r + 1) % 3] = 0;
            for (int64_t base = gwarp * 32; base < nalive; base += nwarps * 32) {
                int64_t i = base + lane;
                bool in = false;
                int32_t v = 0;
                if (i < nalive) {
                    v = __ldcg(&al[i]);
                    if (__ldcg(&a.deg[v]) <= k) {
                        in = true;
                        a.rnd[v] = r;
                        a.core[v] = k;
                    }
                }
                warp_append(in, v, F, &ctl[C_FCNT + r % 3]);
            }
        }
        if (!grid_barrier(ctl, a.timeout_ns)) return;
        // ---- P3: rounds at level k
        while (true) {
            int fs = *(volatile int*)&ctl[C_FCNT + r % 3];
            if (fs == 0) break;
            const int32_t* F = a.fr[r & 1];
            int32_t* Fn = a.fr[(r + 1) & 1];
            if (gtid == 0) ctl[C_FCNT + (r + 2) % 3] = 0;
            for (int64_t i = gwarp; i < fs; i += nwarps) {
                int32_t u = __ldcg(&F[i]);
                int32_t b = a.rowptr[u], e = a.rowptr[u + 1];
                for (int32_t j0 = b; j0 < e; j0 += 32) {
                    int32_t j = j0 + lane;
                    bool cross = false;
                    int32_t v = 0;
                    if (j < e) {
                        v = a.adj[j];
                        if (__ldcg(&a.rnd[v]) < 0) {
                            int old = atomicSub(&a.deg[v], 1);
                            if (old == k + 1) {
                                cross = true;
                                a.rnd[v] = r + 1;
                                a.core[v] = k;
                            }
                        }
                    }
                    warp_append(cross, v, Fn, &ctl[C_FCNT + (r + 1) % 3]);
                }
            }
            if (!grid_barrier(ctl, a.timeout_ns)) return;
            r++;
        }
        lvl++;
    }
    if (gtid == 0) {
        ctl[C_ROUNDS] = r;
        ctl[C_ALPHA] = k;
    }
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

// Warp per vertex: number of neighbours later in the degeneracy order.
__global__ void k_out_degree(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ adj,
                             const int32_t* __restrict__ rnd, int32_t n, int32_t* __restrict__ outdeg) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gw; u < n; u += nw) {
        int cnt = 0;
        for (int32_t j = rowptr[u] + lane; j < rowptr[u + 1]; j += 32) cnt += rank_less((int32_t)u, adj[j], rnd);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) outdeg[u] = cnt;
    }
}

// Warp per vertex: out-neighbours in ascending id order (the row order), with ids of
// the static edges and the tail vertex of each oriented edge.
__global__ void k_out_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ adj_eid, const int32_t* __restrict__ rnd,
                           int32_t n, const int32_t* __restrict__ outptr, int32_t* __restrict__ out_nbr,
                           int32_t* __restrict__ out_eid, int32_t* __restrict__ out_src) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gw; u < n; u += nw) {
        int32_t w = outptr[u];
        for (int32_t j0 = rowptr[u]; j0 < rowptr[u + 1]; j0 += 32) {
            int32_t j = j0 + lane;
            bool keep = false;
            int32_t v = 0;
            if (j < rowptr[u + 1]) {
                v = adj[j];
                keep = rank_less((int32_t)u, v, rnd);
            }
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                int32_t p = w + __popc(mask & ((1u << lane) - 1u));
                out_nbr[p] = v;
                out_eid[p] = adj_eid[j];
                out_src[p] = (int32_t)u;
            }
            w += __popc(mask);
        }
    }
}

// ================================================================== A5

// Thread per oriented edge (u, v): merge N+(u) and N+(v) (both ascending by id).
__global__ void k_tri_count(const int32_t* __restrict__ outptr, const int32_t* __restrict__ out_nbr,
                            const int32_t* __restrict__ out_src, int32_t S, int32_t* __restrict__ cnt,
                            unsigned long long* __restrict__ merged) {
    unsigned long long acc = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = out_src[j], v = out_nbr[j];
        int32_t i1 = outptr[u], e1 = outptr[u + 1], i2 = outptr[v], e2 = outptr[v + 1];
        acc += (unsigned long long)((e1 - i1) + (e2 - i2));
        int32_t c = 0;
        while (i1 < e1 && i2 < e2) {
            int32_t x = out_nbr[i1], y = out_nbr[i2];
            c += (x == y);
            i1 += (x <= y);
            i2 += (y <= x);
        }
        cnt[j] = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(merged, acc);
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

__global__ void k_tri_write(const int32_t* __restrict__ outptr, const int32_t* __restrict__ out_nbr,
                            const int32_t* __restrict__ out_eid, const int32_t* __restrict__ out_src,
                            int32_t S, const int64_t* __restrict__ toff, const int32_t* __restrict__ seg,
                            int4* __restrict__ tri, int64_t* __restrict__ cost,
                            int32_t* __restrict__ common) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = out_src[j], v = out_nbr[j], s_uv = out_eid[j];
        int32_t i1 = outptr[u], e1 = outptr[u + 1], i2 = outptr[v], e2 = outptr[v + 1];
        int64_t p = toff[j];
        int32_t n_here = 0;
        int32_t sig_uv = seg[2 * s_uv + 2] - seg[2 * s_uv];
        while (i1 < e1 && i2 < e2) {
            int32_t x = out_nbr[i1], y = out_nbr[i2];
            if (x == y) {
                int32_t w = x, s_uw = out_eid[i1], s_vw = out_eid[i2];
                int flags = (u < v ? 1 : 0) | (u < w ? 2 : 0) | (v < w ? 4 : 0);
                tri[p] = make_int4(s_uv, s_uw, s_vw, flags);
                cost[p] = (int64_t)sig_uv + (seg[2 * s_uw + 2] - seg[2 * s_uw]) +
                          (seg[2 * s_vw + 2] - seg[2 * s_vw]);
                atomicAdd(&common[s_uw], 1);
                atomicAdd(&common[s_vw], 1);
                p++;
                n_here++;
            }
            i1 += (x <= y);
            i2 += (y <= x);
        }
        if (n_here) atomicAdd(&common[s_uv], n_here);
    }
}

// ================================================================== driver

void preprocess_graph(folty_graph* g, cudaStream_t s) {
    const int T = 256;
    const int64_t m = g->m;
    const int32_t n = g->n;
    Scratch sc(g->alloc, s);

    // ---------------- A1: canonical order
    const int nb = bit_length((uint64_t)(n > 1 ? n - 1 : 1));
    const int key_bits = 2 * nb + 1;
    const uint64_t loop_key = (key_bits >= 64) ? ~0ull : ((1ull << key_bits) - 1);
    const int64_t mk = g->m_kept;
    uint64_t* key = sc.get<uint64_t>(m);
    uint64_t* key_alt = sc.get<uint64_t>(m);
    uint32_t* val = sc.get<uint32_t>(m);
    uint32_t* val_alt = sc.get<uint32_t>(m);
    FOLTY_LAUNCH(k_build_keys, grid_for(m, T), T, 0, s, g->in_src, g->in_dst, m, nb, loop_key, key, val);
    uint64_t* skey = key;
    uint32_t* sval = val;
    if (!g->info.time_sorted && m > 1) {
        // stable sort by t first, then (stably) by the pair key
        int64_t tmin = g->tmin, tmax = g->tmax;
        uint64_t* tk = sc.get<uint64_t>(m);
        uint64_t* tk_alt = sc.get<uint64_t>(m);
        FOLTY_LAUNCH(k_time_keys, grid_for(m, T), T, 0, s, g->in_t, m, tmin, tk, val);
        bool alt = radix_sort_pairs(sc, tk, tk_alt, val, val_alt, m, bit_length((uint64_t)(tmax - tmin)));
        uint32_t* order = alt ? val_alt : val;
        uint32_t* other = alt ? val : val_alt;
        FOLTY_LAUNCH(k_gather_keys, grid_for(m, T), T, 0, s, key, order, m, key_alt);
        // keys now in key_alt, values in order; sort (key_alt, order)
        bool alt2 = radix_sort_pairs(sc, key_alt, key, order, other, m, key_bits);
        skey = alt2 ? key : key_alt;
        sval = alt2 ? other : order;
    } else {
        bool alt = radix_sort_pairs(sc, key, key_alt, val, val_alt, m, key_bits);
        skey = alt ? key_alt : key;
        sval = alt ? val_alt : val;
    }
    g->perm = graph_alloc<int32_t>(g, mk, s);
    g->T = graph_alloc<int64_t>(g, mk, s);
    g->sd = graph_alloc<int32_t>(g, mk, s);
    int32_t* newpair = sc.get<int32_t>(mk + 1);
    int32_t* pscan = sc.get<int32_t>(mk + 1);
    if (mk > 0) FOLTY_LAUNCH(k_store, grid_for(mk, T), T, 0, s, skey, sval, g->in_t, mk, g->perm, g->T, newpair);
    exclusive_scan(sc, newpair, pscan, mk);
    const int32_t S = read_i32(g, pscan + mk, s);
    g->S = S;
    g->ea = graph_alloc<int32_t>(g, S, s);
    g->eb = graph_alloc<int32_t>(g, S, s);
    g->seg = graph_alloc<int32_t>(g, 2 * (int64_t)S + 1, s);
    if (mk > 0) {
        FOLTY_LAUNCH(k_segments, grid_for(mk, T), T, 0, s, skey, newpair, pscan, mk, nb, g->sd, g->ea, g->eb, g->seg);
        FOLTY_LAUNCH(k_segments_split, grid_for(mk, T), T, 0, s, g->sd, mk, S, g->seg);
        FOLTY_LAUNCH(k_segments_fix, grid_for(S, T), T, 0, s, S, mk, g->seg);
    } else {
        FOLTY_CUDA(cudaMemsetAsync(g->seg, 0, sizeof(int32_t), s));
    }
    // the raw input is no longer needed
    graph_release(g, g->in_src, s);
    graph_release(g, g->in_dst, s);
    graph_release(g, g->in_t, s);
    g->in_src = g->in_dst = nullptr;
    g->in_t = nullptr;

    // ---------------- A2: static CSR
    int32_t* deg_hi = sc.get<int32_t>((int64_t)n + 1);
    int32_t* deg_lo = sc.get<int32_t>((int64_t)n + 1);
    FOLTY_CUDA(cudaMemsetAsync(deg_hi, 0, sizeof(int32_t) * ((size_t)n + 1), s));
    FOLTY_CUDA(cudaMemsetAsync(deg_lo, 0, sizeof(int32_t) * ((size_t)n + 1), s));
    if (S > 0) FOLTY_LAUNCH(k_count_degrees, grid_for(S, T), T, 0, s, g->ea, g->eb, S, deg_hi, deg_lo);
    g->deg = graph_alloc<int32_t>(g, (int64_t)n + 1, s);
    FOLTY_LAUNCH(k_add, grid_for(n, T), T, 0, s, deg_hi, deg_lo, (int64_t)n, g->deg);
    int32_t* rowptr = sc.get<int32_t>((int64_t)n + 1);
    int32_t* hi_start = sc.get<int32_t>((int64_t)n + 1);
    int32_t* lo_start = sc.get<int32_t>((int64_t)n + 1);
    exclusive_scan(sc, g->deg, rowptr, n);
    exclusive_scan(sc, deg_hi, hi_start, n);
    exclusive_scan(sc, deg_lo, lo_start, n);
    int32_t* adj = sc.get<int32_t>(2 * (int64_t)S);
    int32_t* adj_eid = sc.get<int32_t>(2 * (int64_t)S);
    if (S > 0) {
        uint64_t* bk = sc.get<uint64_t>(S);
        uint64_t* bk_alt = sc.get<uint64_t>(S);
        uint32_t* bv = sc.get<uint32_t>(S);
        uint32_t* bv_alt = sc.get<uint32_t>(S);
        FOLTY_LAUNCH(k_edge_keys_b, grid_for(S, T), T, 0, s, g->eb, S, bk, bv);
        bool alt = radix_sort_pairs(sc, bk, bk_alt, bv, bv_alt, S, nb);
        FOLTY_LAUNCH(k_fill_adj, grid_for(S, T), T, 0, s, g->ea, g->eb, S, rowptr, deg_lo, hi_start, lo_start,
                     alt ? bv_alt : bv, adj, adj_eid);
    }

    // ---------------- A3: peeling
    int32_t* core = sc.get<int32_t>(n);
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
        pa.ctl = sc.get<int>(C_SLOTS);
        pa.timeout_ns = 10ll * 1000 * 1000 * 1000;
        int init[C_SLOTS] = {0};
        init[C_MIN] = INT_MAX;
        init[C_MIN + 1] = INT_MAX;
        int* init_dev = (int*)(g->host_stage + 48);  // pinned staging
        std::memcpy(init_dev, init, sizeof(init));
        FOLTY_CUDA(cudaMemcpyAsync(pa.ctl, init_dev, sizeof(init), cudaMemcpyHostToDevice, s));
        FOLTY_LAUNCH(k_iota, grid_for(n, T), T, 0, s, pa.alive[0], (int64_t)n);
        int per_sm = 0;
        FOLTY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel, PEEL_THREADS, 0));
        if (per_sm < 1) fail(FOLTY_ECUDA, "peeling kernel cannot be resident");
        if (per_sm > 4) per_sm = 4;
        dim3 grid(num_sms() * per_sm), block(PEEL_THREADS);
        void* args[] = {&pa};
        if (n > 0) {
            FOLTY_CUDA(cudaLaunchCooperativeKernel((const void*)k_peel, grid, block, args, 0, s));
            after_launch("k_peel");
        }
        const void* ptrs[3] = {pa.ctl + C_ERR, pa.ctl + C_ROUNDS, pa.ctl + C_ALPHA};
        int sizes[3] = {4, 4, 4};
        int64_t outv[3];
        read_back(g, ptrs, sizes, 3, outv, s);
        if (n > 0 && outv[0] != 0) fail(FOLTY_ETIMEOUT, "peeling: a grid barrier wait ran out");
        g->info.peel_rounds = (int32_t)(n > 0 ? outv[1] : 0);
        g->info.degeneracy = (int32_t)(n > 0 ? outv[2] : 0);
    }

    // ---------------- A4: orientation
    int32_t* outdeg = sc.get<int32_t>((int64_t)n + 1);
    int32_t* outptr = sc.get<int32_t>((int64_t)n + 1);
    FOLTY_LAUNCH(k_out_degree, grid_for((int64_t)n * 32, T), T, 0, s, rowptr, adj, rnd, n, outdeg);
    exclusive_scan(sc, outdeg, outptr, n);
    int32_t* out_nbr = sc.get<int32_t>(S);
    int32_t* out_eid = sc.get<int32_t>(S);
    int32_t* out_src = sc.get<int32_t>(S);
    FOLTY_LAUNCH(k_out_fill, grid_for((int64_t)n * 32, T), T, 0, s, rowptr, adj, adj_eid, rnd, n, outptr,
                 out_nbr, out_eid, out_src);

    // ---------------- A5: triangles
    g->common = graph_alloc<int32_t>(g, S, s);
    FOLTY_CUDA(cudaMemsetAsync(g->common, 0, sizeof(int32_t) * ((size_t)S > 0 ? (size_t)S : 1), s));
    int32_t* tcnt = sc.get<int32_t>((int64_t)S + 1);
    int64_t* toff = sc.get<int64_t>((int64_t)S + 1);
    int* stat = sc.get<int>(4);  // max degree, max out-degree, max sigma, (pad)
    unsigned long long* merged = sc.get<unsigned long long>(1);
    FOLTY_CUDA(cudaMemsetAsync(stat, 0, sizeof(int) * 4, s));
    FOLTY_CUDA(cudaMemsetAsync(merged, 0, sizeof(unsigned long long), s));
    if (S > 0) FOLTY_LAUNCH(k_tri_count, grid_for(S, T), T, 0, s, outptr, out_nbr, out_src, S, tcnt, merged);
    exclusive_scan(sc, tcnt, toff, S);
    FOLTY_LAUNCH(k_max_i32, grid_for(n, T), T, 0, s, g->deg, (int64_t)n, stat + 0);
    FOLTY_LAUNCH(k_max_i32, grid_for(n, T), T, 0, s, outdeg, (int64_t)n, stat + 1);
    if (S > 0) FOLTY_LAUNCH(k_max_sigma, grid_for(S, T), T, 0, s, g->seg, S, stat + 2);
    {
        const void* ptrs[5] = {toff + S, stat + 0, stat + 1, stat + 2, merged};
        int sizes[5] = {8, 4, 4, 4, 8};
        int64_t outv[5];
        read_back(g, ptrs, sizes, 5, outv, s);
        g->ntri = outv[0];
        g->info.max_degree = (int32_t)outv[1];
        g->info.max_out_degree = (int32_t)outv[2];
        g->info.sigma_max = (int32_t)outv[3];
        g->enum_bytes = 4 * outv[4] + 8 * (int64_t)S;
    }
    const int64_t ntri = g->ntri;
    g->tri = graph_alloc<int4>(g, ntri, s);
    g->tri_off = graph_alloc<int64_t>(g, ntri + 1, s);
    int64_t* cost = sc.get<int64_t>(ntri + 1);
    if (S > 0)
        FOLTY_LAUNCH(k_tri_write, grid_for(S, T), T, 0, s, outptr, out_nbr, out_eid, out_src, S, toff, g->seg,
                     g->tri, cost, g->common);
    exclusive_scan(sc, cost, g->tri_off, ntri);
    g->info.triangles = ntri;
    g->info.probes = read_i64(g, g->tri_off + ntri, s);
    // tile -> first triangle map of the probe kernels (query independent)
    g->n_tiles = (g->info.probes + PB_TILE - 1) / PB_TILE;
    g->tile_tri = graph_alloc<int64_t>(g, g->n_tiles + 1, s);
    if (g->info.probes > 0)
        FOLTY_LAUNCH(k_tile_starts, grid_for(g->n_tiles + 1, T), T, 0, s, g->tri_off, ntri, g->info.probes,
                     g->n_tiles, PB_TILE, g->tile_tri);
    g->info.static_edges = S;
    g->state = 1;
    FOLTY_CUDA(cudaStreamSynchronize(s));
}

}  // namespace folty
