// The window buckets of a triangle's roles, shared by the liveness pass after the
// triangle listing (which writes each triangle's liveness bytes) and the per-query
// selection (which recomputes the roles of the triangles it keeps).
#pragma once

#include "internal.cuh"
#include "probe.cuh"

namespace folty {

constexpr uint8_t DMIN_NEVER = 255;

// An empty run is stored as first = the largest value of the timestamp type and last =
// 0 (unsigned 32-bit offsets, which stay below 2^32 - 1) or -1 (64-bit timestamps, which
// are >= 0). The window conditions below then fail for an empty run without a flag, and
// the union of two runs is (min of the firsts, max of the lasts) whether they are empty
// or not.
template <typename V>
struct RunEmpty;
template <>
struct RunEmpty<uint32_t> {
    static constexpr uint32_t first = 0xffffffffu, last = 0u;
};
template <>
struct RunEmpty<int64_t> {
    static constexpr int64_t first = INT64_MAX, last = -1;
};

__device__ __forceinline__ int bit_len(uint32_t x) { return 32 - __clz(x); }
__device__ __forceinline__ int bit_len(int64_t x) { return 64 - __clzll((unsigned long long)x); }

// First and last timestamp (empty runs encoded as above) and size of both runs of one
// static edge (direction 0 = small id -> large id, then direction 1).
template <typename TS>
struct __align__(16) RunEnds {
    TS f0, l0, f1, l1;
    int32_t n0, n1, pad0, pad1;
};

// The six runs of triangle tr in its id-order frame: the triangle is relabelled so that
// its local vertices are in id order (a rank per vertex from the three id-order bits);
// its three static edges are then read from the run-ends table in that frame, one
// aligned record each, so that every thread runs the same code whatever the triangle's
// id order. Run r = 2k + d is direction d of frame edge k; fu, lu span both directions of
// frame edge k. oe[k] = the stored edge (0: s_uv, 1: s_uw, 2: s_vw) that is frame edge k.
template <typename TS>
struct FrameRuns {
    TS f[6], l[6], fu[3], lu[3];
    int32_t n[6];
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
        fr.f[2 * k] = re.f0;
        fr.l[2 * k] = re.l0;
        fr.f[2 * k + 1] = re.f1;
        fr.l[2 * k + 1] = re.l1;
        fr.fu[k] = min(re.f0, re.f1);
        fr.lu[k] = max(re.l0, re.l1);
    }
}

// The "never" dmin: the largest value of V (real gaps stay below it).
template <typename V>
__device__ __forceinline__ V dmin_never() {
    return RunEmpty<V>::first;
}

// A role (temporal edges x -> y of one static edge, witness z; lists L1 = E_{x,y}, L2,
// L3 of its direction variant) can only produce a window match t <= t2 <= t3 <= t + delta
// if its runs overlap in time: L2 must end at or after L1 starts, L3 must end at or
// after max(L1.first, L2.first), and L2 and L3 must start by L1.last + delta. With every
// run non-empty (L3's emptiness is the only one the first two conditions miss: f3 <= l3
// tests it), the last two hold exactly when delta >= dmin = max(0, L2.first - L1.last,
// L3.first - L1.last). dmin of role r (= 2k + d) for direction variant DIR, of a
// triangle in its id-order frame (flags = 7, so that every run index below is a
// constant); dmin_never() when the role can never hit. The arithmetic stays in the
// store's type: dmin never needs a sign.
template <int DIR, typename V>
__device__ __forceinline__ V frame_dmin(const FrameRuns<V>& fr, int r) {
    int s2, s3;
    role_segments(7, r >> 1, r & 1, DIR, s2, s3);
    const bool both = DIR == FOLTY_DIR_EITHER;  // both directions of the static edges of s2, s3
    const V f1 = fr.f[r], l1 = fr.l[r];
    const V f2 = both ? fr.fu[s2 >> 1] : fr.f[s2], l2 = both ? fr.lu[s2 >> 1] : fr.l[s2];
    const V f3 = both ? fr.fu[s3 >> 1] : fr.f[s3], l3 = both ? fr.lu[s3 >> 1] : fr.l[s3];
    const bool ok = (l2 >= f1) & (l3 >= max(f1, f2)) & (f3 <= l3);
    const V top = max(max(f2, f3), l1);
    return ok ? (V)(top - l1) : dmin_never<V>();
}

// The bucket of a dmin: its bit length (0 for dmin = 0), DMIN_NEVER for "never". A
// query keeps a role of bucket b when delta >= 2^(b-1), which holds whenever
// delta >= dmin (2^(b-1) <= dmin).
template <typename V>
__device__ __forceinline__ uint8_t dmin_bucket(V d) {
    return d == dmin_never<V>() ? DMIN_NEVER : (uint8_t)bit_len(d);
}

// Bucket of role r for direction variant DIR (see frame_dmin).
template <int DIR, typename V>
__device__ __forceinline__ uint8_t frame_bucket(const FrameRuns<V>& fr, int r) {
    return dmin_bucket<V>(frame_dmin<DIR, V>(fr, r));
}

// The liveness byte of triangle tr for direction variant DIR: the smallest bucket of its
// six roles (DMIN_NEVER when none can hit at any window). The bit length is monotone, so
// the smallest bucket is the bucket of the smallest dmin.
template <typename TS, int DIR>
__device__ __forceinline__ uint8_t liveness_byte(const int4 tr, const RunEnds<TS>* __restrict__ ends) {
    FrameRuns<TS> fr;
    frame_runs<TS>(tr, ends, fr);
    TS m = frame_dmin<DIR, TS>(fr, 0);
#pragma unroll
    for (int r = 1; r < 6; r++) m = min(m, frame_dmin<DIR, TS>(fr, r));
    return dmin_bucket<TS>(m);
}

}  // namespace folty
