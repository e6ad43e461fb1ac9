// Window-probe machinery shared by the single-query and the batched kernels.
//
// Flat probe space: triangle-major (tri_off = prefix of per-triangle sizes), inside a
// triangle its three static edges {u,v}, {u,w}, {v,w} in that order, inside a static
// edge its temporal edges in sorted order (E_{a->b} then E_{b->a}, a < b by id).
// A probe is one (temporal edge, witness) pair.
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
constexpr int64_t PROBE_NONE = LLONG_MAX;

struct TriStage {
    int64_t base[PB_MAXTRI + 1];
    int32_t off[PB_MAXTRI][9];  // per static edge e: [start of a->b, start of b->a, end]
    int32_t flags[PB_MAXTRI];   // bit0: id(u) < id(v), bit1: id(u) < id(w), bit2: id(v) < id(w)
    int32_t nt;
};

struct Lists {
    int32_t b2, e2, b2b, e2b;  // L2 (second range only for "either")
    int32_t b3, e3, b3b, e3b;  // L3
};

// id(vertex a) < id(vertex b) for triangle-local vertices a != b in {0 = u, 1 = v, 2 = w}.
__device__ __forceinline__ bool id_less(int flags, int a, int b) {
    int lo = a < b ? a : b;
    int hi = a + b - lo;
    bool l = (flags >> (lo + hi - 1)) & 1;
    return (a == lo) ? l : !l;
}

// Lists of the role whose L1 is direction d of static edge e of the triangle.
// Edge e joins local vertices (0,1), (0,2), (1,2); its witness is vertex 2 - e; the
// static edge joining local vertices i and j is edge i + j - 1.
__device__ __forceinline__ Lists role_lists(const int32_t* off, int flags, int e, int d, int dir) {
    const int p = (e == 2) ? 1 : 0, q = (e == 0) ? 1 : 2, z = 2 - e;
    // direction 0 of a static edge runs from its smaller id to its larger id
    const int x = ((d == 0) == id_less(flags, p, q)) ? p : q;
    const int y = p + q - x;
    const int exz = x + z - 1, eyz = y + z - 1;
    Lists L;
    if (dir == FOLTY_DIR_EITHER) {
        L.b2 = off[3 * exz];
        L.e2 = off[3 * exz + 1];
        L.b2b = off[3 * exz + 1];
        L.e2b = off[3 * exz + 2];
        L.b3 = off[3 * eyz];
        L.e3 = off[3 * eyz + 1];
        L.b3b = off[3 * eyz + 1];
        L.e3b = off[3 * eyz + 2];
    } else {
        int d2 = id_less(flags, x, z) ? 0 : 1;  // E_{x,z}
        int d3 = id_less(flags, y, z) ? 0 : 1;  // E_{y,z}
        if (dir == FOLTY_DIR_IN) {              // E_{z,x}, E_{z,y}
            d2 ^= 1;
            d3 ^= 1;
        }
        L.b2 = off[3 * exz + d2];
        L.e2 = off[3 * exz + d2 + 1];
        L.b3 = off[3 * eyz + d3];
        L.e3 = off[3 * eyz + d3 + 1];
        L.b2b = L.e2b = L.b3b = L.e3b = 0;
    }
    return L;
}

__device__ __forceinline__ int64_t first_at_least(const int64_t* __restrict__ T, int32_t b, int32_t e,
                                                  int64_t key) {
    int32_t i = lower_bound_i64(T, b, e, key);
    return i < e ? T[i] : PROBE_NONE;
}

// Theorem 3.1: t2 = first entry >= t of L2, t3 = first entry >= t2 of L3. Returns t3
// (PROBE_NONE when either does not exist).
__device__ __forceinline__ int64_t probe_window(const int64_t* __restrict__ T, int64_t t, const Lists& L) {
    int64_t t2 = first_at_least(T, L.b2, L.e2, t);
    if (L.e2b > L.b2b) t2 = min(t2, first_at_least(T, L.b2b, L.e2b, t));
    if (t2 == PROBE_NONE) return PROBE_NONE;
    int64_t t3 = first_at_least(T, L.b3, L.e3, t2);
    if (L.e3b > L.b3b) t3 = min(t3, first_at_least(T, L.b3b, L.e3b, t2));
    return t3;
}

// Stages the triangles overlapping probes [p0, p1) of this block. tile_tri[b] is the
// triangle holding probe min(b * PB_TILE, P - 1).
__device__ __forceinline__ void stage_triangles(TriStage& st, const int4* __restrict__ tri,
                                                const int64_t* __restrict__ tri_off,
                                                const int64_t* __restrict__ tile_tri,
                                                const int32_t* __restrict__ seg) {
    const int64_t t0 = tile_tri[blockIdx.x];
    const int nt = (int)(tile_tri[blockIdx.x + 1] - t0 + 1);
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        int4 tr = tri[t0 + j];
        st.base[j] = tri_off[t0 + j];
        st.flags[j] = tr.w;
        const int32_t se[3] = {tr.x, tr.y, tr.z};
#pragma unroll
        for (int e = 0; e < 3; e++) {
            st.off[j][3 * e] = seg[2 * se[e]];
            st.off[j][3 * e + 1] = seg[2 * se[e] + 1];
            st.off[j][3 * e + 2] = seg[2 * se[e] + 2];
        }
    }
    if (threadIdx.x == 0) st.nt = nt;
    __syncthreads();
}

struct Probe {
    int32_t j;    // staged triangle
    int32_t e;    // static edge of the triangle (0..2)
    int32_t d;    // direction of the temporal edge on it
    int32_t pos;  // sorted position of the temporal edge
};

__device__ __forceinline__ Probe locate_probe(const TriStage& st, int64_t p) {
    int lo = 0, hi = st.nt - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (st.base[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    const int32_t* off = st.off[lo];
    int32_t o = (int32_t)(p - st.base[lo]);
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
    Probe pr;
    pr.j = lo;
    pr.e = e;
    pr.pos = off[3 * e] + o;
    pr.d = pr.pos >= off[3 * e + 1];
    return pr;
}

}  // namespace folty
