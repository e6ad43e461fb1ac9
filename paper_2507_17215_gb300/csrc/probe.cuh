// Window-probe machinery shared by the single-query, batched and allocation-free
// kernels.
//
// Flat probe space: triangle-major (tri_off = prefix of per-triangle sizes), inside a
// triangle its three static edges {u,v}, {u,w}, {v,w} in that order, inside a static
// edge its temporal edges in sorted order (E_{a->b} then E_{b->a}, a < b by id).
// A probe is one (temporal edge, witness) pair.
//
// Timestamps are stored as TS: uint32_t offsets t - t_min when the graph's time range
// fits, int64_t otherwise. Window tests only use differences, so both give the same
// answers.
#pragma once

#include <climits>

#include "internal.cuh"

namespace folty {

constexpr int PB_THREADS = 256;
constexpr int PB_ITEMS = 8;
constexpr int PB_TILE = PB_THREADS * PB_ITEMS;
// every triangle holds >= 3 probes, so a tile overlaps at most 1 + ceil(TILE / 3)
// triangles (+1 for the one that may start exactly at the next tile)
constexpr int PB_MAXTRI = PB_TILE / 3 + 4;

template <typename TS>
struct TsNone;
template <>
struct TsNone<uint32_t> {
    static constexpr uint32_t value = 0xffffffffu;
};
template <>
struct TsNone<int64_t> {
    static constexpr int64_t value = LLONG_MAX;
};

// Segment k (0..5) of a staged triangle = direction k & 1 of its static edge k >> 1:
// [off[3 * (k >> 1) + (k & 1)], off[3 * (k >> 1) + (k & 1) + 1]). MAXTRI = the triangles a
// tile can overlap.
template <int MAXTRI>
struct TriStageT {
    int32_t base[MAXTRI + 1];  // first probe of the triangle, relative to the tile start
    int32_t off[MAXTRI][9];    // per static edge e: [start of a->b, start of b->a, end]
    uint64_t desc[MAXTRI];     // per (e, d): L2 segment code | L3 segment code << 3
    int32_t nt;
};
using TriStage = TriStageT<PB_MAXTRI>;

// id(vertex a) < id(vertex b) for triangle-local vertices a != b in {0 = u, 1 = v, 2 = w};
// flags bit0: id(u) < id(v), bit1: id(u) < id(w), bit2: id(v) < id(w).
__host__ __device__ __forceinline__ bool id_less(int flags, int a, int b) {
    int lo = a < b ? a : b;
    int hi = a + b - lo;
    bool l = (flags >> (lo + hi - 1)) & 1;
    return (a == lo) ? l : !l;
}

// Segment codes of the role whose L1 is direction d of static edge e. Edge e joins
// local vertices (0,1), (0,2), (1,2); its witness is vertex 2 - e; the static edge
// joining local vertices i and j is edge i + j - 1. "out": L2 = E_{x,z}, L3 = E_{y,z};
// "in": E_{z,x}, E_{z,y}; "either": both directions of those static edges (the code's
// direction bit is then unused).
__host__ __device__ __forceinline__ void role_segments(int flags, int e, int d, int dir, int& seg2, int& seg3) {
    const int p = (e == 2) ? 1 : 0, q = (e == 0) ? 1 : 2, z = 2 - e;
    const int x = ((d == 0) == id_less(flags, p, q)) ? p : q;  // direction 0 runs small id -> large id
    const int y = p + q - x;
    const int exz = x + z - 1, eyz = y + z - 1;
    int d2 = id_less(flags, x, z) ? 0 : 1;  // E_{x,z}
    int d3 = id_less(flags, y, z) ? 0 : 1;  // E_{y,z}
    if (dir == FOLTY_DIR_IN) {
        d2 ^= 1;
        d3 ^= 1;
    } else if (dir == FOLTY_DIR_EITHER) {
        d2 = d3 = 0;
    }
    seg2 = 2 * exz + d2;
    seg3 = 2 * eyz + d3;
}

__device__ __forceinline__ uint64_t role_descriptor(int flags, int dir) {
    uint64_t desc = 0;
#pragma unroll
    for (int e = 0; e < 3; e++) {
#pragma unroll
        for (int d = 0; d < 2; d++) {
            int s2, s3;
            role_segments(flags, e, d, dir, s2, s3);
            desc |= (uint64_t)(s2 | (s3 << 3)) << (6 * (2 * e + d));
        }
    }
    return desc;
}

// First index in [b, e) with T[i] >= key (e if none); branch-free halving.
template <typename TS>
__device__ __forceinline__ int32_t lower_bound_ts(const TS* __restrict__ T, int32_t b, int32_t e, TS key) {
    int32_t len = e - b;
    while (len > 1) {
        int32_t half = len >> 1;
        b = (T[b + half - 1] < key) ? b + half : b;
        len -= half;
    }
    return b + ((len == 1 && T[b] < key) ? 1 : 0);
}

template <typename TS>
__device__ __forceinline__ TS first_at_least(const TS* __restrict__ T, int32_t b, int32_t e, TS key) {
    int32_t i = lower_bound_ts(T, b, e, key);
    return i < e ? T[i] : TsNone<TS>::value;
}

// First entry >= key of one sorted run, or TsNone. The run's last entry is checked
// before searching (runs of different static edges rarely overlap in time).
template <typename TS>
__device__ __forceinline__ TS first_at_least_checked(const TS* __restrict__ T, int32_t b, int32_t e, TS key) {
    if (b == e || T[e - 1] < key) return TsNone<TS>::value;
    return T[lower_bound_ts(T, b, e, key)];
}

// x - t > delta for x >= t (no overflow)
template <typename TS>
__device__ __forceinline__ bool beyond(TS x, TS t, TS delta) {
    return (TS)(x - t) > delta;
}

// Theorem 3.1: t2 = first entry >= t of L2, t3 = first entry >= t2 of L3 (the first entry
// of a union of sorted runs is the smallest of their first entries). Returns t3, or
// TsNone when t2 or t3 does not exist or when t2 alone already lies beyond t + delta
// (then t3 >= t2 does too, so the caller's window test fails either way). Runs whose
// first entry lies beyond t + delta are skipped without a search.
template <typename TS, int DIR>
__device__ __forceinline__ TS probe_window(const TS* __restrict__ T, const int32_t* off, int seg2, int seg3,
                                           TS t, TS delta) {
    const TS NONE = TsNone<TS>::value;
    const int o2 = 3 * (seg2 >> 1) + (seg2 & 1), o3 = 3 * (seg3 >> 1) + (seg3 & 1);
    TS t2 = NONE;
    {
        const int32_t b = off[o2], e = off[o2 + 1];
        if (b < e && !(T[b] > t && beyond(T[b], t, delta))) t2 = first_at_least_checked(T, b, e, t);
    }
    if (DIR == FOLTY_DIR_EITHER) {
        const int32_t b = off[o2 + 1], e = off[o2 + 2];
        if (b < e && !(T[b] > t && beyond(T[b], t, delta))) {
            TS x = first_at_least_checked(T, b, e, t);
            t2 = x < t2 ? x : t2;
        }
    }
    if (t2 == NONE || beyond(t2, t, delta)) return NONE;
    TS t3 = first_at_least_checked(T, off[o3], off[o3 + 1], t2);
    if (DIR == FOLTY_DIR_EITHER) {
        TS x = first_at_least_checked(T, off[o3 + 1], off[o3 + 2], t2);
        t3 = x < t3 ? x : t3;
    }
    return t3;
}

// Stages the triangles overlapping this block's probe tile: tile_tri[b] is the triangle
// holding probe min(b * PB_TILE, P - 1).
__device__ __forceinline__ void stage_triangles(TriStage& st, const int4* __restrict__ tri,
                                                const int64_t* __restrict__ tri_off,
                                                const int64_t* __restrict__ tile_tri,
                                                const int32_t* __restrict__ seg, int dir) {
    const int64_t t0 = tile_tri[blockIdx.x];
    const int nt = (int)(tile_tri[blockIdx.x + 1] - t0 + 1);
    const int64_t p0 = (int64_t)blockIdx.x * PB_TILE;
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        int4 tr = tri[t0 + j];
        st.base[j] = (int32_t)(tri_off[t0 + j] - p0);
        st.desc[j] = role_descriptor(tr.w, dir);
        const int32_t se[3] = {tr.x, tr.y, tr.z};
#pragma unroll
        for (int e = 0; e < 3; e++) {
            st.off[j][3 * e] = seg[2 * se[e]];
            st.off[j][3 * e + 1] = seg[2 * se[e] + 1];
            st.off[j][3 * e + 2] = seg[2 * se[e] + 2];
        }
    }
    if (threadIdx.x == 0) {
        st.nt = nt;
        st.base[nt] = INT_MAX;
    }
    __syncthreads();
}

struct Probe {
    int32_t pos;         // sorted position of the temporal edge (L1 entry)
    int32_t seg2, seg3;  // segment codes of L2 and L3
    int32_t j;           // staged triangle
};

// Locates probe `local` (tile-relative) for every lane of the warp. All lanes call it
// (warp-uniform); `active` marks lanes with a probe. One lane bisects for the warp's
// first probe, then each lane walks forward (a warp's 32 consecutive probes span few
// triangles).
__device__ __forceinline__ Probe locate_probe(const TriStage& st, int32_t local, bool active) {
    const int lane = threadIdx.x & 31;
    int32_t first = __shfl_sync(0xffffffffu, local, 0);
    int j0 = 0;
    if (lane == 0) {
        int lo = 0, hi = st.nt - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (st.base[mid] <= first) lo = mid;
            else hi = mid - 1;
        }
        j0 = lo;
    }
    int j = __shfl_sync(0xffffffffu, j0, 0);
    Probe pr;
    pr.pos = 0;
    pr.seg2 = pr.seg3 = 0;
    if (active) {
        while (st.base[j + 1] <= local) j++;
        const int32_t* off = st.off[j];
        int32_t o = local - st.base[j];
        int e = 0;
        int32_t s0 = off[2] - off[0];
        if (o >= s0) {
            o -= s0;
            e = 1;
            int32_t s1 = off[5] - off[3];
            if (o >= s1) {
                o -= s1;
                e = 2;
            }
        }
        pr.pos = off[3 * e] + o;
        const int d = pr.pos >= off[3 * e + 1];
        const int code = (int)((st.desc[j] >> (6 * (2 * e + d))) & 63);
        pr.seg2 = code & 7;
        pr.seg3 = code >> 3;
    }
    pr.j = j;
    return pr;
}

}  // namespace folty
