// Window probes restricted to roles that can hit.
//
// A role (temporal edges x -> y of one static edge, witness z; lists L1 = E_{x,y}, L2,
// L3 of its direction variant) can only produce a window match t <= t2 <= t3 <= t + delta
// if its runs overlap in time: L2 must end at or after L1 starts, L3 must end at or
// after max(L1.first, L2.first), and L2 and L3 must start by L1.last + delta. The first
// two conditions do not depend on delta; the last two hold exactly when
// delta >= dmin = max(0, L2.first - L1.last, L3.first - L1.last).
//
// A role's bucket is a conservative form of dmin for one direction variant: its bit
// length b (0 for dmin = 0, 255 for "never"), so 2^(b-1) <= dmin. A query keeps a role
// when delta >= 2^(b-1), which holds whenever delta >= dmin: no role that can hit is
// dropped (a few that cannot are kept). Preprocessing stores the first and last
// timestamp and the size of every run (the run-ends table) and, per triangle and
// direction variant, the smallest bucket of its six roles (one byte). A query reads that
// byte for every triangle; only the triangles it keeps (typically a few in ten thousand)
// get their six roles' buckets and sizes from the run-ends table. It then lays the kept
// roles out in a flat probe space (3 idle slots per triangle keep the tile staging bound)
// and probes only those, with the exact window test of Theorem 3.1.
#include <type_traits>

#include "internal.cuh"
#include "liveness.cuh"
#include "probe.cuh"
#include "scan.cuh"

namespace folty {

constexpr int LIVE_IDLE = 3;  // idle slots per kept triangle (keeps >= 3 slots per triangle)

template <typename TS>
__global__ void k_run_ends(const int32_t* __restrict__ seg, int64_t S, const TS* __restrict__ T,
                           RunEnds<TS>* __restrict__ ends) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < S; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o0 = seg[2 * e], o1 = seg[2 * e + 1], o2 = seg[2 * e + 2];
        RunEnds<TS> r;
        r.n0 = o1 - o0;
        r.n1 = o2 - o1;
        r.f0 = r.n0 > 0 ? T[o0] : RunEmpty<TS>::first;
        r.l0 = r.n0 > 0 ? T[o1 - 1] : RunEmpty<TS>::last;
        r.f1 = r.n1 > 0 ? T[o1] : RunEmpty<TS>::first;
        r.l1 = r.n1 > 0 ? T[o2 - 1] : RunEmpty<TS>::last;
        r.pad0 = r.pad1 = 0;
        ends[e] = r;
    }
}

// The liveness byte of every listed triangle for direction variant DIR (liveness_byte),
// one thread per triangle: consecutive triangles share their first edge, so its record
// mostly comes from L1.
template <typename TS, int DIR>
__global__ void k_tri_live(const int4* __restrict__ tri, int64_t ntri, const RunEnds<TS>* __restrict__ ends,
                           uint8_t* __restrict__ row) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntri; t += (int64_t)gridDim.x * blockDim.x)
        row[t] = liveness_byte<TS, DIR>(__ldcs(tri + t), ends);
}

// The same while the triangles move from the bounded layout of a one-pass listing into
// the dense one: the cnt[j] triangles of oriented edge j from tri_b[boff[j] ...] to
// tri[toff[j] ...] (toff: prefix of cnt). A warp takes 32 consecutive edges, whose
// triangles are contiguous in tri; its lanes stride over them, two triangles a lane per
// step (both loads in flight before either is used), and find each one's edge by a
// binary search of the lanes' running counts. One warp per 32 edges and short blocks:
// the dense communities' edges hold far more triangles than the rest.
template <typename TS, int DIR>
__global__ void k_tri_live_copy(const int32_t* __restrict__ cnt, const int64_t* __restrict__ toff,
                                const int64_t* __restrict__ boff, int32_t S, const int4* __restrict__ tri_b,
                                int4* __restrict__ tri, const RunEnds<TS>* __restrict__ ends,
                                uint8_t* __restrict__ row) {
    const int lane = threadIdx.x & 31;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) & ~31ll;
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); j0 < S; j0 += wstride) {
        const int64_t j = j0 + lane;
        const int32_t c = j < S ? cnt[j] : 0;
        const int64_t src0 = j < S ? boff[j] : 0;
        int32_t inc = c;  // inclusive running count over the warp's edges
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
        if (total == 0) continue;
        const int64_t dst0 = toff[j0];
        for (int32_t t0 = 0; t0 < total; t0 += 64) {
            int4 tr[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int32_t t = t0 + 32 * h + lane;
                int e = 0;  // the first lane whose running count exceeds t
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int32_t v = __shfl_sync(0xffffffffu, inc, e + step - 1);
                    if (v <= t) e += step;
                }
                const int32_t before = __shfl_sync(0xffffffffu, inc - c, e);
                const int64_t from = __shfl_sync(0xffffffffu, src0, e);
                tr[h] = t < total ? __ldcs(tri_b + from + (t - before)) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int32_t t = t0 + 32 * h + lane;
                if (t < total) {
                    tri[dst0 + t] = tr[h];
                    row[dst0 + t] = liveness_byte<TS, DIR>(tr[h], ends);
                }
            }
        }
    }
}

__device__ __forceinline__ bool bucket_live(uint8_t b, int64_t delta) {
    return b != DMIN_NEVER && (b == 0 || delta >= ((int64_t)1 << (b - 1)));
}

// Role mask (stored role order: bit 2e + d = direction d of stored edge e) and kept
// probes of triangle tr at window delta for direction variant DIR.
template <typename TS, int DIR>
__device__ __forceinline__ int kept_roles_of(const int4 tr, const RunEnds<TS>* __restrict__ ends, int64_t delta,
                                             int64_t& probes) {
    FrameRuns<TS> fr;
    frame_runs<TS>(tr, ends, fr);
    int m = 0;
    int64_t c = 0;
#pragma unroll
    for (int r = 0; r < 6; r++) {
        if (bucket_live(frame_bucket<DIR, TS>(fr, r), delta)) {  // never for an empty run
            m |= 1 << (2 * fr.oe[r >> 1] + (r & 1));
            c += fr.n[r];
        }
    }
    probes = c;
    return m;
}

// Kept roles of every triangle for one query: kept triangle j = L[j] with its role mask
// lmask[j] and its first probe slot loff[j] (prefix of the kept triangles' costs = kept
// probes + LIVE_IDLE idle slots); totals[0] = kept triangles, totals[1] = slots,
// loff[totals[0]] = totals[1]; and the probe tiles' map: ltile[b] = kept triangle holding
// slot min(b * ptile, slots - 1) for b <= the number of probe tiles (each kept triangle
// writes the tile starts inside its slots).
//
// Three passes without a look-back: every warp takes LS_WARP consecutive triangles (a
// lane LS_ITEMS of them, read as 16-byte chunks of their liveness bytes: the smallest
// bucket of each triangle's roles for this direction variant); k_live_sums writes the
// warp's number of kept triangles and their cost, k_live_offsets turns those into
// exclusive prefixes (one block), and k_live_write writes the kept triangles at them.
// Only the triangles whose byte admits delta read their record and run ends: they are
// few, but cluster, so a warp deals its candidates round-robin over its lanes (candidate
// k of the warp, in triangle order, goes to lane k mod 32), and the write pass orders
// their costs by a warp scan per round of 32.
constexpr int LS_ITEMS = 64;
constexpr int LS_WARP = 32 * LS_ITEMS;  // 2048 triangles per warp
constexpr int LS_THREADS = 256;
constexpr int LS_BLOCK = (LS_THREADS / 32) * LS_WARP;

// Bit i of the result: triangle t0 + i (i < LS_ITEMS) is kept at delta (rows are padded
// with DMIN_NEVER to whole 16-byte chunks). A byte b admits delta exactly when
// b <= B = bit length of delta (b = 0 always, b >= 1 when delta >= 2^(b-1); DMIN_NEVER
// never, as B <= 63): four bytes at a time, (0x80 + B) - (b & 0x7f) keeps bit 7 set
// exactly for b <= B (bytes never borrow from one another, and 255 & 0x7f = 127 > B), and
// one multiplication gathers the four bit-7s.
__device__ __forceinline__ uint64_t live_mask(const uint8_t* __restrict__ tlive, int64_t t0, int64_t ntri,
                                              int64_t delta) {
    const uint32_t B = delta > 0 ? (uint32_t)(64 - __clzll((unsigned long long)delta)) : 0u;
    const uint32_t bias = 0x80808080u | (B * 0x01010101u);
    uint64_t lm = 0;
#pragma unroll
    for (int h = 0; h < LS_ITEMS / 16; h++) {
        uint4 w = make_uint4(~0u, ~0u, ~0u, ~0u);
        if (t0 + 16 * h < ntri) w = __ldcs(reinterpret_cast<const uint4*>(tlive + t0 + 16 * h));
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t hit = (bias - (ws[q] & 0x7f7f7f7fu)) & 0x80808080u;
            const uint32_t nib = ((hit >> 7) * 0x10204080u) >> 28;  // bit j = byte j admits delta
            lm |= (uint64_t)nib << (16 * h + 4 * q);
        }
    }
    return lm;
}

// The warp's candidates: this lane's mask lm, the number of candidates of the lanes
// before it (pre) and of the warp (returned).
__device__ __forceinline__ int warp_candidates(uint64_t lm, int& pre) {
    const int lane = threadIdx.x & 31;
    const int own = __popcll(lm);
    int inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    pre = inc - own;
    return __shfl_sync(0xffffffffu, inc, 31);
}

// Position within the warp's range of candidate k (< the warp's total): the lane l with
// pre[l] <= k < pre[l + 1], and the (k - pre[l])-th set bit of its mask. The whole warp
// must call it.
__device__ __forceinline__ int candidate_at(int k, uint64_t lm, int pre) {
    int l = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int pc = __shfl_sync(0xffffffffu, pre, l + step);
        if (pc <= k) l += step;
    }
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)lm, l);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(lm >> 32), l);
    const int n = k - __shfl_sync(0xffffffffu, pre, l);  // 0-based rank among l's candidates
    const int plo = __popc(lo);
    const int bit = n < plo ? __fns(lo, 0, n + 1) : 32 + __fns(hi, 0, n - plo + 1);
    return l * LS_ITEMS + bit;
}

// Per warp: its kept triangles and their total cost.
template <typename TS, int DIR>
__global__ void __launch_bounds__(LS_THREADS) k_live_sums(const uint8_t* __restrict__ tlive,
                                                          const int4* __restrict__ tri,
                                                          const RunEnds<TS>* __restrict__ ends, int64_t ntri,
                                                          int64_t delta, const int64_t* __restrict__ qp,
                                                          int32_t* __restrict__ wcnt, int64_t* __restrict__ wcost) {
    if (qp) delta = qp[0];  // the window from a device parameter block (replayed query plans)
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * LS_THREADS + threadIdx.x) >> 5;
    const int64_t tw = w * LS_WARP;
    const uint64_t lm = live_mask(tlive, tw + (int64_t)lane * LS_ITEMS, ntri, delta);
    int pre;
    const int total = warp_candidates(lm, pre);
    int64_t cost = 0;
    for (int k0 = 0; k0 < total; k0 += 32) {
        const int k = k0 + lane;
        const int at = candidate_at(min(k, total - 1), lm, pre);
        if (k < total) {
            int64_t pr;
            kept_roles_of<TS, DIR>(tri[tw + at], ends, delta, pr);
            cost += pr + LIVE_IDLE;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, o);
    if (lane == 0) {
        wcnt[w] = total;
        wcost[w] = cost;
    }
}

// One block: the warps' counts and costs become exclusive prefixes in place; the totals,
// the end of loff and of the tile map, and the kept triangles' model bytes.
template <typename TS>
__global__ void __launch_bounds__(1024) k_live_offsets(int32_t* __restrict__ wcnt, int64_t* __restrict__ wcost,
                                                       int64_t nw, int64_t* __restrict__ totals,
                                                       int64_t* __restrict__ loff, int64_t* __restrict__ ltile,
                                                       int64_t max_tiles, int64_t ptile,
                                                       unsigned long long* __restrict__ prof) {
    __shared__ int64_t sc[32], sp[32];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t per = (nw + 1023) / 1024;
    const int64_t b = (int64_t)threadIdx.x * per, e = min(b + per, nw);
    int64_t c = 0, p = 0;
    for (int64_t i = b; i < e; i++) {
        c += wcnt[i];
        p += wcost[i];
    }
    int64_t ic = c, ip = p;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t yc = __shfl_up_sync(0xffffffffu, ic, o), yp = __shfl_up_sync(0xffffffffu, ip, o);
        if (lane >= o) {
            ic += yc;
            ip += yp;
        }
    }
    if (lane == 31) {
        sc[wi] = ic;
        sp[wi] = ip;
    }
    __syncthreads();
    if (wi == 0) {
        int64_t xc = sc[lane], xp = sp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t yc = __shfl_up_sync(0xffffffffu, xc, o), yp = __shfl_up_sync(0xffffffffu, xp, o);
            if (lane >= o) {
                xc += yc;
                xp += yp;
            }
        }
        sc[lane] = xc;  // inclusive over warps
        sp[lane] = xp;
    }
    __syncthreads();
    int64_t oc = ic - c + (wi ? sc[wi - 1] : 0), op = ip - p + (wi ? sp[wi - 1] : 0);
    for (int64_t i = b; i < e; i++) {
        const int32_t x = wcnt[i];
        const int64_t y = wcost[i];
        wcnt[i] = (int32_t)oc;
        wcost[i] = op;
        oc += x;
        op += y;
    }
    if (threadIdx.x == 0) {
        const int64_t nl = sc[31], P = sp[31];
        totals[0] = nl;
        totals[1] = P;
        loff[nl] = P;
        const int64_t tiles = (P + ptile - 1) / ptile;
        if (P > 0 && tiles <= max_tiles) ltile[tiles] = nl - 1;
        if (prof) atomicAdd(prof, (unsigned long long)((16 + 3 * sizeof(RunEnds<TS>) + 13) * nl));
    }
}

// Per warp: its kept triangles at their prefixes, with their masks, first slots and tile
// starts.
template <typename TS, int DIR>
__global__ void __launch_bounds__(LS_THREADS) k_live_write(const uint8_t* __restrict__ tlive,
                                                           const int4* __restrict__ tri,
                                                           const RunEnds<TS>* __restrict__ ends, int64_t ntri,
                                                           int64_t delta, const int64_t* __restrict__ qp,
                                                           const int32_t* __restrict__ woffc,
                                                           const int64_t* __restrict__ woffp, int32_t* __restrict__ L,
                                                           int64_t* __restrict__ loff, uint8_t* __restrict__ lmask,
                                                           int64_t* __restrict__ ltile, int64_t max_tiles,
                                                           int64_t ptile) {
    if (qp) delta = qp[0];
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * LS_THREADS + threadIdx.x) >> 5;
    const int64_t tw = w * LS_WARP;
    const uint64_t lm = live_mask(tlive, tw + (int64_t)lane * LS_ITEMS, ntri, delta);
    int pre;
    const int total = warp_candidates(lm, pre);
    if (total == 0) return;  // warp-uniform
    const int64_t bc = woffc[w];
    int64_t run = woffp[w];
    for (int k0 = 0; k0 < total; k0 += 32) {
        const int k = k0 + lane;
        const int at = candidate_at(min(k, total - 1), lm, pre);
        int m = 0;
        int64_t v = 0;
        if (k < total) {
            int64_t pr;
            m = kept_roles_of<TS, DIR>(tri[tw + at], ends, delta, pr);
            v = pr + LIVE_IDLE;
        }
        int64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (k < total) {
            const int64_t jc = bc + k, jp = run + inc - v;
            L[jc] = (int32_t)(tw + at);
            loff[jc] = jp;
            lmask[jc] = (uint8_t)m;
            for (int64_t b = (jp + ptile - 1) / ptile; b * ptile < jp + v && b <= max_tiles; b++) ltile[b] = jc;
        }
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
}

// Model bytes of a staged triangle's kept roles (its first slot lies in this tile):
// staging 61 B, and per role w sigma1 + w min(sigma2, sigma1 ceil(log2(sigma2 + 1))) + the
// same for L3 + 8 sigma1, w = bytes per timestamp.
template <typename TS, int DIR>
__device__ __forceinline__ unsigned long long kept_role_bytes(const int32_t* off, int m, uint64_t desc) {
    const int64_t w = sizeof(TS);
    unsigned long long b = 61;
    for (int r = 0; r < 6; r++) {
        if (!((m >> r) & 1)) continue;
        const int64_t s1 = off[3 * (r >> 1) + (r & 1) + 1] - off[3 * (r >> 1) + (r & 1)];
        const int code = (int)((desc >> (6 * r)) & 63);
        const int c2 = code & 7, c3 = code >> 3;
        const int o2 = 3 * (c2 >> 1) + (c2 & 1), o3 = 3 * (c3 >> 1) + (c3 & 1);
        const int64_t s2 = DIR == FOLTY_DIR_EITHER ? off[o2 + 2] - off[o2] : off[o2 + 1] - off[o2];
        const int64_t s3 = DIR == FOLTY_DIR_EITHER ? off[o3 + 2] - off[o3] : off[o3 + 1] - off[o3];
        const int64_t l2 = 64 - __clzll((unsigned long long)s2), l3 = 64 - __clzll((unsigned long long)s3);
        b += (unsigned long long)(w * s1 + w * min(s2, s1 * l2) + w * min(s3, s1 * l3) + 8 * s1);
    }
    return b;
}

struct LiveArgs {
    const int4* tri;
    const int32_t* seg;
    const int32_t* L;
    const int64_t* loff;
    const uint8_t* lmask;
    const int64_t* ltile;
    const int64_t* P;  // device: total slots
    int32_t* cnt;      // MODE 0
    int32_t* bins;     // MODE 1, or
    uint32_t* bins16;  // MODE 1: 16-bit counts, two to a word
    int64_t mk;
    int k;             // MODE 1: number of bins
    int kstride;       // MODE 1: bins per edge row (k rounded up to whole 16-byte rows)
    unsigned long long* prof;  // model bytes of the kept roles (may be null)
    uint8_t* rflag;    // MODE 0, may be null: 6 * triangle + role flags of roles with a hit
    const int64_t* qp; // may be null: a device block whose slot 0 (64-bit store) or 1 (32-bit
                       // store) holds the window, read instead of the delta argument
    uint32_t* touched; // MODE 1, may be null: bit g set when a sorted edge of group g (edges
                       // [32 g, 32 g + 32)) received a binned hit
};

// MODE 0: cnt[pos] += hit at window delta. MODE 1: bin the gap t3 - t (<= delta, the
// largest bin bound) against the sorted bounds deltas[0..k). A block takes probe tiles of
// PB_THREADS * ITEMS slots (the tile size the autotuner picks).
template <typename TS, int DIR, int MODE, int ITEMS>
__global__ void __launch_bounds__(PB_THREADS) k_probe_live(LiveArgs a, const TS* __restrict__ T, TS delta,
                                                           const TS* __restrict__ deltas) {
    constexpr int TILE = PB_THREADS * ITEMS;
    constexpr int MAXTRI = TILE / 3 + 4;  // every kept triangle holds >= 3 slots
    __shared__ TriStageT<MAXTRI> st;
    __shared__ uint8_t smask[MAXTRI];
    __shared__ TS sD[1024];
    if (a.qp) delta = (TS)a.qp[sizeof(TS) == 4 ? 1 : 0];
    if (MODE == 1)
        for (int i = threadIdx.x; i < a.k; i += blockDim.x) sD[i] = deltas[i];
    const int64_t P = *a.P;
    const int64_t tiles = (P + TILE - 1) / TILE;
    for (int64_t b = blockIdx.x; b < tiles; b += gridDim.x) {
        __syncthreads();  // the previous tile's stage is no longer read
        const int64_t t0 = a.ltile[b];
        const int nt = (int)(a.ltile[b + 1] - t0 + 1);
        const int64_t p0 = b * (int64_t)TILE;
        unsigned long long pbytes = 0;
        for (int j = threadIdx.x; j < nt; j += blockDim.x) {
            const int4 tr = a.tri[a.L[t0 + j]];
            st.base[j] = (int32_t)(a.loff[t0 + j] - p0);
            st.desc[j] = role_descriptor(tr.w, DIR);
            smask[j] = a.lmask[t0 + j];
            const int32_t se[3] = {tr.x, tr.y, tr.z};
#pragma unroll
            for (int e = 0; e < 3; e++) {
                st.off[j][3 * e] = a.seg[2 * se[e]];
                st.off[j][3 * e + 1] = a.seg[2 * se[e] + 1];
                st.off[j][3 * e + 2] = a.seg[2 * se[e] + 2];
            }
            if (a.prof && st.base[j] >= 0) pbytes += kept_role_bytes<TS, DIR>(st.off[j], smask[j], st.desc[j]);
        }
        if (a.prof) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pbytes += __shfl_xor_sync(0xffffffffu, pbytes, o);
            if ((threadIdx.x & 31) == 0 && pbytes) atomicAdd(a.prof, pbytes);
        }
        if (threadIdx.x == 0) {
            st.nt = nt;
            st.base[nt] = INT_MAX;
        }
        __syncthreads();
        const int32_t count = (int32_t)min((int64_t)TILE, P - p0);
#pragma unroll 1
        for (int it = 0; it < ITEMS; it++) {
            const int32_t local = it * PB_THREADS + (int32_t)threadIdx.x;
            if ((local & ~31) >= count) break;  // warp-uniform
            bool active = local < count;
            // triangle of the slot: one lane bisects for the warp, lanes walk forward
            const int lane = threadIdx.x & 31;
            const int32_t first = __shfl_sync(0xffffffffu, local, 0);
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
            if (!active) continue;
            while (st.base[j + 1] <= local) j++;
            int32_t o = local - st.base[j] - LIVE_IDLE;
            if (o < 0) continue;  // idle slot
            const int32_t* off = st.off[j];
            const int m = smask[j];
            int r = 0;
            for (; r < 6; r++) {
                if (!((m >> r) & 1)) continue;
                const int32_t s1 = off[3 * (r >> 1) + (r & 1) + 1] - off[3 * (r >> 1) + (r & 1)];
                if (o < s1) break;
                o -= s1;
            }
            if (r == 6) continue;  // cannot happen: o < the kept roles' total
            const int32_t pos = off[3 * (r >> 1) + (r & 1)] + o;
            const int code = (int)((st.desc[j] >> (6 * r)) & 63);
            const TS t = T[pos];
            const TS t3 = probe_window<TS, DIR>(T, off, code & 7, code >> 3, t, delta);
            if (t3 == TsNone<TS>::value) continue;
            const TS gap = (TS)(t3 - t);
            if (gap > delta) continue;
            if (MODE == 0) {
                if (a.bins16) atomicAdd(&a.bins16[pos >> 1], 1u << (16 * (pos & 1)));
                else atomicAdd(&a.cnt[pos], 1);
                if (a.rflag) a.rflag[6 * (int64_t)a.L[t0 + j] + r] = 1;
            } else {
                const int jb = lower_bound_ts<TS>(sD, 0, a.k, gap);
                const int64_t x = (int64_t)pos * a.kstride + jb;  // edge-major: an edge's bins are contiguous
                if (a.bins16) atomicAdd(&a.bins16[x >> 1], 1u << (16 * (int)(x & 1)));
                else atomicAdd(&a.bins[x], 1);
                if (a.touched) {
                    // a plain read first: most hits find their group's bit already set
                    const uint32_t bit = 1u << ((pos >> 5) & 31);
                    if (!(a.touched[pos >> 10] & bit)) atomicOr(&a.touched[pos >> 10], bit);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host side

template <typename TS>
static void run_ends_t(folty_graph* g, cudaStream_t s) {
    const int64_t S = g->S;
    RunEnds<TS>* ends = static_cast<RunEnds<TS>*>(g->run_ends);
    // per static edge: 12 B of run bounds and 4 timestamps read, its record written
    StageSpan span(ST_ROLES, s, S * (12 + 4 * (int64_t)sizeof(TS) + (int64_t)sizeof(RunEnds<TS>)));
    if (S > 0) FOLTY_LAUNCH(k_run_ends<TS>, grid_for(S, 256), 256, 0, s, g->seg, S, (const TS*)g->T, ends);
}

void build_run_ends(folty_graph* g, cudaStream_t s) {
    g->run_ends = g->ts32 ? (void*)graph_alloc<RunEnds<uint32_t>>(g, g->S, s)
                          : (void*)graph_alloc<RunEnds<int64_t>>(g, g->S, s);
    if (g->ts32) run_ends_t<uint32_t>(g, s);
    else run_ends_t<int64_t>(g, s);
}

void prepare_liveness(folty_graph* g, cudaStream_t s) {
    const int64_t ntri = g->ntri;
    // three rows of liveness bytes, each padded with DMIN_NEVER to whole 16-byte chunks
    // (triangle_liveness writes the first ntri bytes of each)
    g->tlive_stride = (ntri + 15) & ~int64_t(15);
    g->tlive = graph_alloc<uint8_t>(g, 3 * g->tlive_stride, s);
    for (int d = 0; d < 3; d++)
        if (g->tlive_stride > ntri)
            FOLTY_CUDA(cudaMemsetAsync(g->tlive + d * g->tlive_stride + ntri, DMIN_NEVER,
                                       (size_t)(g->tlive_stride - ntri), s));
}

template <typename TS>
static void liveness_row_t(folty_graph* g, int dir, cudaStream_t s) {
    const int64_t ntri = g->ntri;
    // per triangle: its record read and one byte written; the run-ends table (shared by
    // the triangles of an edge, and small) read once
    StageSpan span(ST_ROLES, s, ntri * (16 + 1) + g->S * (int64_t)sizeof(RunEnds<TS>));
    if (ntri == 0) return;
    const RunEnds<TS>* ends = (const RunEnds<TS>*)g->run_ends;
    uint8_t* row = g->tlive + (int64_t)dir * g->tlive_stride;
    const unsigned grid = grid_for(ntri, 256);
    if (dir == FOLTY_DIR_OUT) FOLTY_LAUNCH((k_tri_live<TS, FOLTY_DIR_OUT>), grid, 256, 0, s, g->tri, ntri, ends, row);
    else if (dir == FOLTY_DIR_IN) FOLTY_LAUNCH((k_tri_live<TS, FOLTY_DIR_IN>), grid, 256, 0, s, g->tri, ntri, ends, row);
    else FOLTY_LAUNCH((k_tri_live<TS, FOLTY_DIR_EITHER>), grid, 256, 0, s, g->tri, ntri, ends, row);
}

// Each direction variant's liveness row is computed by the first call that needs it
// (preprocessing computes the paper's "out" motif's): a graph queried with one variant
// only pays for that one.
void ensure_liveness(folty_graph* g, int dir, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g->live_mu);
    if (!g->live_ready[dir]) {
        if (g->ts32) liveness_row_t<uint32_t>(g, dir, s);
        else liveness_row_t<int64_t>(g, dir, s);
        if (!g->live_ev[dir]) FOLTY_CUDA(cudaEventCreateWithFlags(&g->live_ev[dir], cudaEventDisableTiming));
        FOLTY_CUDA(cudaEventRecord(g->live_ev[dir], s));
        g->live_ready[dir] = 1;
    } else {
        FOLTY_CUDA(cudaStreamWaitEvent(s, g->live_ev[dir], 0));
    }
}

template <typename TS>
static void liveness_copy_t(folty_graph* g, const TriLayout& from, cudaStream_t s) {
    const int64_t ntri = g->ntri;
    // per triangle: its record read in the bounded layout and written in the dense one,
    // and one byte written; the per-edge counts, offsets and run ends read once
    StageSpan span(ST_ROLES, s, ntri * (16 + 16 + 1) + g->S * (int64_t)(4 + 8 + 8 + sizeof(RunEnds<TS>)));
    if (ntri == 0) return;
    FOLTY_LAUNCH((k_tri_live_copy<TS, FOLTY_DIR_OUT>), (unsigned)((g->S + 255) / 256), 256, 0, s, from.cnt, from.toff,
                 from.boff, g->S, from.tri_b, g->tri, (const RunEnds<TS>*)g->run_ends,
                 g->tlive + (int64_t)FOLTY_DIR_OUT * g->tlive_stride);
}

void triangle_liveness(folty_graph* g, cudaStream_t s, const TriLayout* from) {
    if (!from) {
        ensure_liveness(g, FOLTY_DIR_OUT, s);
        return;
    }
    std::lock_guard<std::mutex> lock(g->live_mu);
    if (g->ts32) liveness_copy_t<uint32_t>(g, *from, s);
    else liveness_copy_t<int64_t>(g, *from, s);
    if (!g->live_ev[FOLTY_DIR_OUT]) FOLTY_CUDA(cudaEventCreateWithFlags(&g->live_ev[FOLTY_DIR_OUT], cudaEventDisableTiming));
    FOLTY_CUDA(cudaEventRecord(g->live_ev[FOLTY_DIR_OUT], s));
    g->live_ready[FOLTY_DIR_OUT] = 1;
}

// The probe kernel of the graph's tuned shape: tile of PB_THREADS * items slots,
// blocks per SM as many as fit or the tuned count.
template <typename TS, int MODE, int ITEMS>
static void launch_live_shape(const folty_graph* g, int dir, const LiveArgs& la, int blocks, TS delta,
                              const TS* deltas, cudaStream_t s) {
    int per_sm = 0;
    FOLTY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_live<TS, 0, MODE, ITEMS>, PB_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    if (blocks > 0 && blocks < per_sm) per_sm = blocks;
    const unsigned grid = (unsigned)(num_sms() * per_sm);
    const TS* T = (const TS*)g->T;
    if (dir == FOLTY_DIR_OUT)
        FOLTY_LAUNCH((k_probe_live<TS, FOLTY_DIR_OUT, MODE, ITEMS>), grid, PB_THREADS, 0, s, la, T, delta, deltas);
    else if (dir == FOLTY_DIR_IN)
        FOLTY_LAUNCH((k_probe_live<TS, FOLTY_DIR_IN, MODE, ITEMS>), grid, PB_THREADS, 0, s, la, T, delta, deltas);
    else
        FOLTY_LAUNCH((k_probe_live<TS, FOLTY_DIR_EITHER, MODE, ITEMS>), grid, PB_THREADS, 0, s, la, T, delta, deltas);
}

template <typename TS, int MODE>
static void launch_live_t(const folty_graph* g, int dir, const LiveArgs& la, TS delta, const TS* deltas,
                          cudaStream_t s) {
    if (g->tune.probe_items == 4) launch_live_shape<TS, MODE, 4>(g, dir, la, g->tune.probe_blocks, delta, deltas, s);
    else launch_live_shape<TS, MODE, 8>(g, dir, la, g->tune.probe_blocks, delta, deltas, s);
}

template <typename TS>
static void launch_select_t(const folty_graph* g, int dir, const uint8_t* tl, int64_t delta, const ProbeBuffers& ls,
                            unsigned long long* prof, const int64_t* qp, cudaStream_t s) {
    const RunEnds<TS>* ends = static_cast<const RunEnds<TS>*>(g->run_ends);
    const int64_t ntri = g->ntri;
    const int64_t tile = (int64_t)PB_THREADS * g->tune.probe_items;
    const unsigned blocks = (unsigned)((ntri + LS_BLOCK - 1) / LS_BLOCK);
#define FOLTY_SUMS_ARGS tl, g->tri, ends, ntri, delta, qp, ls.wcnt, ls.wcost
#define FOLTY_WRITE_ARGS \
    tl, g->tri, ends, ntri, delta, qp, ls.wcnt, ls.wcost, ls.L, ls.loff, ls.lmask, ls.ltile, ls.max_tiles, tile
    if (dir == FOLTY_DIR_OUT)
        FOLTY_LAUNCH((k_live_sums<TS, FOLTY_DIR_OUT>), blocks, LS_THREADS, 0, s, FOLTY_SUMS_ARGS);
    else if (dir == FOLTY_DIR_IN)
        FOLTY_LAUNCH((k_live_sums<TS, FOLTY_DIR_IN>), blocks, LS_THREADS, 0, s, FOLTY_SUMS_ARGS);
    else
        FOLTY_LAUNCH((k_live_sums<TS, FOLTY_DIR_EITHER>), blocks, LS_THREADS, 0, s, FOLTY_SUMS_ARGS);
    FOLTY_LAUNCH(k_live_offsets<TS>, 1, 1024, 0, s, ls.wcnt, ls.wcost, ls.nw, ls.totals, ls.loff, ls.ltile,
                 ls.max_tiles, tile, prof);
    if (dir == FOLTY_DIR_OUT)
        FOLTY_LAUNCH((k_live_write<TS, FOLTY_DIR_OUT>), blocks, LS_THREADS, 0, s, FOLTY_WRITE_ARGS);
    else if (dir == FOLTY_DIR_IN)
        FOLTY_LAUNCH((k_live_write<TS, FOLTY_DIR_IN>), blocks, LS_THREADS, 0, s, FOLTY_WRITE_ARGS);
    else
        FOLTY_LAUNCH((k_live_write<TS, FOLTY_DIR_EITHER>), blocks, LS_THREADS, 0, s, FOLTY_WRITE_ARGS);
#undef FOLTY_SUMS_ARGS
#undef FOLTY_WRITE_ARGS
}

// Buffers of one selection: from a call's scratch, or owned by the graph. The tile map
// has room for the smallest probe tile the tuner may pick.
constexpr int PB_TILE_MIN = PB_THREADS * 4;

template <typename A>
static ProbeBuffers make_probe_buffers(const folty_graph* g, A&& get) {
    const int64_t ntri = g->ntri;
    ProbeBuffers ls;
    ls.L = get((int32_t*)nullptr, ntri + 1);
    ls.loff = get((int64_t*)nullptr, ntri + 1);
    ls.lmask = get((uint8_t*)nullptr, ntri + 1);
    ls.totals = get((int64_t*)nullptr, 2);
    ls.max_tiles = (g->info.probes + LIVE_IDLE * ntri + PB_TILE_MIN - 1) / PB_TILE_MIN;
    ls.ltile = get((int64_t*)nullptr, ls.max_tiles + 2);
    ls.nw = (ntri + LS_BLOCK - 1) / LS_BLOCK * (LS_THREADS / 32);  // the selection's warps
    ls.wcnt = get((int32_t*)nullptr, ls.nw + 1);
    ls.wcost = get((int64_t*)nullptr, ls.nw + 1);
    return ls;
}

ProbeBuffers probe_buffers(folty_graph* g, cudaStream_t s) {
    return make_probe_buffers(g, [&](auto* tag, int64_t n) {
        return graph_alloc<std::remove_pointer_t<decltype(tag)>>(g, n, s);
    });
}

// Selects the roles kept for delta (or the window in qp) into ls. prof_sel (may be null)
// receives the selection's model bytes beyond its one byte per triangle.
static void enqueue_select(folty_graph* g, int64_t delta, int dir, const ProbeBuffers& ls, int* err,
                           unsigned long long* prof_sel, const int64_t* qp, cudaStream_t s) {
    (void)err;  // no waits: the selection cannot run out of time
    StageSpan span(ST_SELECT, s, g->ntri, prof_sel);
    const uint8_t* tl = g->tlive + (int64_t)dir * g->tlive_stride;
    if (g->ts32) launch_select_t<uint32_t>(g, dir, tl, delta, ls, prof_sel, qp, s);
    else launch_select_t<int64_t>(g, dir, tl, delta, ls, prof_sel, qp, s);
}

static ProbeBuffers select_live(folty_graph* g, int64_t delta, int dir, Scratch& sc, cudaStream_t s,
                                unsigned long long* prof_sel) {
    const ProbeBuffers ls = make_probe_buffers(g, [&](auto* tag, int64_t n) {
        return sc.get<std::remove_pointer_t<decltype(tag)>>(n);
    });
    ensure_liveness(g, dir, s);
    enqueue_select(g, delta, dir, ls, sc.err(), prof_sel, nullptr, s);
    return ls;
}

// Kept roles for delta (the largest window of the pass), then the probe kernel.
// mode 0: counts into cnt; mode 1: bins (deltas = k sorted bounds in the store's type).
void launch_probe_live(folty_graph* g, int64_t delta, int dir, int mode, int32_t* cnt, int32_t* bins, int k,
                       int kstride, const void* deltas, cudaStream_t s, uint8_t* rflag, uint16_t* bins16,
                       uint32_t* touched) {
    const int64_t ntri = g->ntri;
    if (ntri == 0 || g->info.probes == 0) return;
    tune_probe(g, delta, dir, s);
    Scratch sc(g->alloc, s, g->dev_err);
    // model bytes counted on the device: the selection reads one liveness byte per
    // triangle, and per kept one its record and run ends, and writes 13 B; the probes'
    // bytes per staged triangle and kept role are summed by the probe kernel
    unsigned long long* prof_sel = nullptr;
    unsigned long long* prof = nullptr;
    if (profiling_on()) {
        prof_sel = g->prof_bytes + (g->prof_next++ % PROF_SLOTS);
        prof = g->prof_bytes + (g->prof_next++ % PROF_SLOTS);
        FOLTY_CUDA(cudaMemsetAsync(prof_sel, 0, sizeof(unsigned long long), s));
        FOLTY_CUDA(cudaMemsetAsync(prof, 0, sizeof(unsigned long long), s));
    }
    const ProbeBuffers ls = select_live(g, delta, dir, sc, s, prof_sel);
    StageSpan span(ST_PROBE, s, 0, prof);
    LiveArgs la{g->tri, g->seg, ls.L, ls.loff, ls.lmask, ls.ltile, ls.totals + 1, cnt, bins, (uint32_t*)bins16,
                g->m_kept, k, kstride, prof, rflag, nullptr, touched};
    if (g->ts32) {
        const uint32_t d32 = delta >= 0xfffffffell ? 0xfffffffeu : (uint32_t)delta;
        if (mode == 0) launch_live_t<uint32_t, 0>(g, dir, la, d32, nullptr, s);
        else launch_live_t<uint32_t, 1>(g, dir, la, d32, (const uint32_t*)deltas, s);
    } else {
        if (mode == 0) launch_live_t<int64_t, 0>(g, dir, la, delta, nullptr, s);
        else launch_live_t<int64_t, 1>(g, dir, la, delta, (const int64_t*)deltas, s);
    }
}

void enqueue_probe_pass(folty_graph* g, const int64_t* qp, int dir, const ProbeBuffers& pb, int32_t* cnt,
                        uint16_t* cnt16, cudaStream_t s) {
    if (g->ntri == 0 || g->info.probes == 0) return;
    enqueue_select(g, 0, dir, pb, g->dev_err, nullptr, qp, s);
    LiveArgs la{g->tri, g->seg, pb.L, pb.loff, pb.lmask, pb.ltile, pb.totals + 1, cnt, nullptr, (uint32_t*)cnt16,
                g->m_kept, 0, 0, nullptr, nullptr, qp};
    if (g->ts32) launch_live_t<uint32_t, 0>(g, dir, la, 0u, nullptr, s);
    else launch_live_t<int64_t, 0>(g, dir, la, 0, nullptr, s);
}

// ------------------------------------------------------------------ autotuning

// The probe shape of g: forced, cached under the graph's statistics, or picked by timing
// each candidate (tile, blocks per SM) on the probe pass of the first query's (delta,
// dir) after one selection; the candidates give identical counts (every probe is made
// once whatever the tile), so only their times differ.
void tune_probe(folty_graph* g, int64_t delta, int dir, cudaStream_t s) {
    if (g->tune.probe_source != 0) return;
    if (tune_forced(&g->tune, true)) return;
    const std::vector<int64_t> key{g->n, g->m_kept, g->S, g->ntri, g->info.probes, g->ts32};
    if (tune_lookup(key, &g->tune, true)) return;
    if (g->ntri == 0 || g->info.probes == 0 || profiling_on()) return;  // nothing to time (or events in use)
    Scratch sc(g->alloc, s, g->dev_err);
    const int64_t mk = g->m_kept;
    const bool c16 = g->info.max_degree < 65535;
    int32_t* cnt = c16 ? nullptr : sc.get<int32_t>(mk);
    uint16_t* cnt16 = c16 ? sc.get<uint16_t>(mk + 2) : nullptr;
    cudaEvent_t ev[TUNE_TRIALS + 1];
    for (auto& e : ev) FOLTY_CUDA(cudaEventCreate(&e));
    float best = 0.f;
    int bi = 1;
    try {
        TuneParams t = g->tune;
        for (int c = 0; c < TUNE_TRIALS; c++) {
            g->tune.probe_items = PROBE_CAND[c][0];
            g->tune.probe_blocks = PROBE_CAND[c][1];
            // the selection's tile map depends on the tile, so each trial selects again
            // (outside its timed span)
            const ProbeBuffers ls = select_live(g, delta, dir, sc, s, nullptr);
            if (cnt16) FOLTY_CUDA(cudaMemsetAsync(cnt16, 0, sizeof(uint16_t) * (size_t)(mk + 2), s));
            else FOLTY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)mk, s));
            LiveArgs la{g->tri, g->seg, ls.L, ls.loff, ls.lmask, ls.ltile, ls.totals + 1, cnt, nullptr,
                        (uint32_t*)cnt16, mk, 0, 0, nullptr, nullptr, nullptr};
            FOLTY_CUDA(cudaEventRecord(ev[0], s));
            if (g->ts32) {
                const uint32_t d32 = delta >= 0xfffffffell ? 0xfffffffeu : (uint32_t)delta;
                launch_live_t<uint32_t, 0>(g, dir, la, d32, nullptr, s);
            } else {
                launch_live_t<int64_t, 0>(g, dir, la, delta, nullptr, s);
            }
            FOLTY_CUDA(cudaEventRecord(ev[c + 1], s));
            FOLTY_CUDA(cudaEventSynchronize(ev[c + 1]));
            float ms = 0.f;
            FOLTY_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[c + 1]));
            t.probe_ms[c] = ms;
            if (c == 0 || ms < best) {
                best = ms;
                bi = c;
            }
        }
        t.probe_items = PROBE_CAND[bi][0];
        t.probe_blocks = PROBE_CAND[bi][1];
        t.probe_source = 1;
        g->tune.probe_items = t.probe_items;
        g->tune.probe_blocks = t.probe_blocks;
        g->tune.probe_source = 1;
        std::memcpy(g->tune.probe_ms, t.probe_ms, sizeof(t.probe_ms));
        tune_store(key, g->tune, true);
    } catch (...) {
        for (auto& e : ev) cudaEventDestroy(e);
        g->tune.probe_items = 8;
        g->tune.probe_blocks = 0;
        throw;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    read_back(g, nullptr, nullptr, 0, nullptr, s);  // a trial's look-back wait that ran out surfaces here
}

// ------------------------------------------------------------------ selection statistics

// Kept roles, their probes and the probe pass's model bytes over the kept triangles of a
// selection: out[0] += roles, out[1] += probes (sigma1 of the kept roles), out[2] +=
// model bytes (the same per-triangle and per-role figures the probe kernel counts).
template <typename TS, int DIR>
__global__ void k_live_stats(const int4* __restrict__ tri, const int32_t* __restrict__ seg,
                             const int32_t* __restrict__ L, const uint8_t* __restrict__ lmask,
                             const int64_t* __restrict__ totals, unsigned long long* __restrict__ out) {
    const int64_t nl = totals[0];
    unsigned long long roles = 0, probes = 0, bytes = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nl; j += (int64_t)gridDim.x * blockDim.x) {
        const int4 tr = tri[L[j]];
        const int m = lmask[j];
        const int32_t se[3] = {tr.x, tr.y, tr.z};
        int32_t off[9];
#pragma unroll
        for (int e = 0; e < 3; e++) {
            off[3 * e] = seg[2 * se[e]];
            off[3 * e + 1] = seg[2 * se[e] + 1];
            off[3 * e + 2] = seg[2 * se[e] + 2];
        }
        roles += (unsigned long long)__popc(m);
        for (int r = 0; r < 6; r++)
            if ((m >> r) & 1) probes += (unsigned long long)(off[3 * (r >> 1) + (r & 1) + 1] - off[3 * (r >> 1) + (r & 1)]);
        bytes += kept_role_bytes<TS, DIR>(off, m, role_descriptor(tr.w, DIR));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        roles += __shfl_xor_sync(0xffffffffu, roles, o);
        probes += __shfl_xor_sync(0xffffffffu, probes, o);
        bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    }
    if ((threadIdx.x & 31) == 0 && roles) {
        atomicAdd(&out[0], roles);
        atomicAdd(&out[1], probes);
        atomicAdd(&out[2], bytes);
    }
}

template <typename TS>
static void live_stats_t(const folty_graph* g, int dir, const ProbeBuffers& ls, unsigned long long* acc,
                         cudaStream_t s) {
    const unsigned grid = grid_for(g->ntri, 256);
    if (dir == FOLTY_DIR_OUT)
        FOLTY_LAUNCH((k_live_stats<TS, FOLTY_DIR_OUT>), grid, 256, 0, s, g->tri, g->seg, ls.L, ls.lmask, ls.totals, acc);
    else if (dir == FOLTY_DIR_IN)
        FOLTY_LAUNCH((k_live_stats<TS, FOLTY_DIR_IN>), grid, 256, 0, s, g->tri, g->seg, ls.L, ls.lmask, ls.totals, acc);
    else
        FOLTY_LAUNCH((k_live_stats<TS, FOLTY_DIR_EITHER>), grid, 256, 0, s, g->tri, g->seg, ls.L, ls.lmask, ls.totals,
                     acc);
}

void probe_stats(folty_graph* g, int64_t delta, int dir, folty_probe_stats* out, cudaStream_t s) {
    std::memset(out, 0, sizeof(*out));
    out->triangles = g->ntri;
    out->all_roles = 6 * g->ntri;
    out->all_probes = g->info.probes;  // every (temporal edge, witness) pair
    out->select_bytes = g->ntri;
    if (g->ntri == 0 || g->info.probes == 0) return;
    Scratch sc(g->alloc, s, g->dev_err);
    const ProbeBuffers ls = select_live(g, delta, dir, sc, s, nullptr);
    unsigned long long* acc = sc.get<unsigned long long>(3);
    FOLTY_CUDA(cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), s));
    if (g->ts32) live_stats_t<uint32_t>(g, dir, ls, acc, s);
    else live_stats_t<int64_t>(g, dir, ls, acc, s);
    const void* ptrs[4] = {ls.totals, acc, acc + 1, acc + 2};
    int sizes[4] = {8, 8, 8, 8};
    int64_t v[4];
    read_back(g, ptrs, sizes, 4, v, s);
    out->kept_triangles = v[0];
    out->kept_roles = v[1];
    out->kept_probes = v[2];
    out->probe_bytes = v[3];
    out->select_bytes += (int64_t)(16 + 3 * (g->ts32 ? sizeof(RunEnds<uint32_t>) : sizeof(RunEnds<int64_t>)) + 13) * v[0];
}

}  // namespace folty
