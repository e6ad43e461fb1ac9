// The window buckets of a triangle's roles, shared by the triangle listing (which writes
// each triangle's liveness bytes as it finds it) and the per-query selection (which
// recomputes the roles of the triangles it keeps).
//
// A role (temporal edges x -> y of one static edge, witness z; lists L1 = E_{x,y}, L2,
// L3 of its direction variant) can only produce a window match t <= t2 <= t3 <= t + delta
// if its runs overlap in time: L2 must end at or after L1 starts, L3 must end at or
// after max(L1.first, L2.first), and L2 and L3 must start by L1.last + delta. The first
// two conditions do not depend on delta; the last two hold exactly when
// delta >= dmin = max(0, L2.first - L1.last, L3.first - L1.last). A role's bucket is the
// bit length b of dmin (0 for dmin = 0, DMIN_NEVER for "never"), so 2^(b-1) <= dmin: a
// query keeps a role when delta >= 2^(b-1), which holds whenever delta >= dmin.
#pragma once

#include "internal.cuh"
#include "probe.cuh"

namespace folty {

constexpr uint8_t DMIN_NEVER = 255;

// Time span of the union of runs a and b (b < 0: run a alone) from the first and last
// timestamps of the six runs of a triangle, in the store's timestamp type V. Called with
// indices the compiler knows, so the arrays stay in registers.
template <typename V>
__device__ __forceinline__ bool span_of(const V* f, const V* l, const bool* ne, int a, int b, V& first, V& last) {
    bool any = false;
    if (ne[a]) {
        first = f[a];
        last = l[a];
        any = true;
    }
    if (b >= 0 && ne[b]) {
        first = any ? min(first, f[b]) : f[b];
        last = any ? max(last, l[b]) : l[b];
        any = true;
    }
    return any;
}

__device__ __forceinline__ int bit_len(uint32_t x) { return 32 - __clz(x); }
__device__ __forceinline__ int bit_len(int64_t x) { return 64 - __clzll((unsigned long long)x); }

// Bucket of role r (= 2k + d: direction d of frame edge k) for direction variant DIR, of
// a triangle whose local vertices 0, 1, 2 are in id order (flags = 7, so that every run
// index below is a constant), from the first and last timestamps of its six runs. The
// arithmetic stays in the store's type (32-bit offsets for most graphs): dmin =
// max(0, L2.first - L1.last, L3.first - L1.last) never needs a sign.
template <int DIR, typename V>
__device__ __forceinline__ uint8_t frame_bucket(const V* f, const V* l, const bool* ne, int r) {
    if (!ne[r]) return DMIN_NEVER;
    int s2, s3;
    role_segments(7, r >> 1, r & 1, DIR, s2, s3);
    const bool both = DIR == FOLTY_DIR_EITHER;  // s2, s3 are the d = 0 runs then
    V f2 = 0, l2 = 0, f3 = 0, l3 = 0;
    const bool a2 = span_of<V>(f, l, ne, s2, both ? s2 + 1 : -1, f2, l2);
    const bool a3 = span_of<V>(f, l, ne, s3, both ? s3 + 1 : -1, f3, l3);
    const V f1 = f[r], l1 = l[r];
    if (!(a2 && a3 && l2 >= f1 && l3 >= (f2 > f1 ? f2 : f1))) return DMIN_NEVER;
    const V d2 = f2 > l1 ? (V)(f2 - l1) : (V)0, d3 = f3 > l1 ? (V)(f3 - l1) : (V)0;
    return (uint8_t)bit_len(d2 > d3 ? d2 : d3);  // 0 for dmin = 0
}

// First and last timestamp and size of both runs of one static edge (direction 0 =
// small id -> large id, then direction 1); first = last = 0 for an empty run.
template <typename TS>
struct __align__(16) RunEnds {
    TS f0, l0, f1, l1;
    int32_t n0, n1, pad0, pad1;
};

// The six runs of triangle tr in its id-order frame: the triangle is relabelled so that
// its local vertices are in id order (a rank per vertex from the three id-order bits);
// its three static edges are then read from the run-ends table in that frame, one
// aligned record each, so that every thread runs the same code whatever the triangle's
// id order. oe[k] = the stored edge (0: s_uv, 1: s_uw, 2: s_vw) that is frame edge k.
template <typename TS>
struct FrameRuns {
    TS f[6], l[6];
    int32_t n[6];
    bool ne[6];
    int oe[3];
};

template <typename TS>
__device__ __forceinline__ void frame_runs(const int4 tr, const RunEnds<TS>* __restrict__ ends, FrameRuns<TS>& fr) {
    const int b0 = tr.w & 1, b1 = (tr.w >> 1) & 1, b2 = (tr.w >> 2) & 1;
    // rank of each local vertex among the three ids
    const int rk0 = (b0 ^ 1) + (b1 ^ 1), rk1 = b0 + (b2 ^ 1), rk2 = b1 + b2;
    // stored edge e joins local vertices (0,1), (0,2), (1,2); in the sorted frame it
    // joins ranks (rk_p, rk_q), i.e. frame edge rk_p + rk_q - 1
    const int k0 = rk0 + rk1 - 1, k1 = rk0 + rk2 - 1;
    int32_t se[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        fr.oe[k] = (k == k0) ? 0 : (k == k1) ? 1 : 2;
        se[k] = (k == k0) ? tr.x : (k == k1) ? tr.y : tr.z;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const RunEnds<TS> re = ends[se[k]];
        fr.n[2 * k] = re.n0;
        fr.n[2 * k + 1] = re.n1;
        fr.ne[2 * k] = re.n0 > 0;
        fr.ne[2 * k + 1] = re.n1 > 0;
        fr.f[2 * k] = re.f0;
        fr.l[2 * k] = re.l0;
        fr.f[2 * k + 1] = re.f1;
        fr.l[2 * k + 1] = re.l1;
    }
}

// The liveness bytes of triangle tr: per direction variant, the smallest bucket of its six
// roles (DMIN_NEVER when none can hit at any window), written to tlive[dir * tstride + t].
template <typename TS>
__device__ __forceinline__ void write_liveness(const int4 tr, const RunEnds<TS>* __restrict__ ends, int64_t t,
                                               int64_t tstride, uint8_t* __restrict__ tlive) {
    FrameRuns<TS> fr;
    frame_runs<TS>(tr, ends, fr);
    uint8_t m0 = DMIN_NEVER, m1 = DMIN_NEVER, m2 = DMIN_NEVER;
#pragma unroll
    for (int r = 0; r < 6; r++) {
        m0 = min(m0, frame_bucket<FOLTY_DIR_OUT, TS>(fr.f, fr.l, fr.ne, r));
        m1 = min(m1, frame_bucket<FOLTY_DIR_IN, TS>(fr.f, fr.l, fr.ne, r));
        m2 = min(m2, frame_bucket<FOLTY_DIR_EITHER, TS>(fr.f, fr.l, fr.ne, r));
    }
    tlive[t] = m0;
    tlive[tstride + t] = m1;
    tlive[2 * tstride + t] = m2;
}

}  // namespace folty
