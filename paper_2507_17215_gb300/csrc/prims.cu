// Device-wide primitives: exclusive prefix sum and a stable LSD radix sort.
//
// Both are bandwidth-bound streaming passes: tiles of 2048 (scan) or 4096 (sort)
// elements per 256-thread block, coalesced loads, block offsets from a recursive scan
// of per-tile totals. The sort takes 11-bit digits (a 41-bit key in 4 passes).
#include "internal.cuh"

namespace folty {

int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

// ================================================================== scan

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* warp_tot, T* block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == SCAN_THREADS / 32 - 1) *block_total = wi;
    }
    __syncthreads();
    return warp_tot[warp] + inc - v;
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const TIn* __restrict__ in, int64_t n,
                                                              TOut* __restrict__ bsum) {
    __shared__ TOut warp_tot[SCAN_THREADS / 32];
    __shared__ TOut total;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    TOut acc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < n) acc += (TOut)in[idx];
    }
    block_exclusive_sum<TOut>(acc, warp_tot, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Scans one tile; adds the tile's offset (boff[block], or 0 when boff is null). The
// last tile also writes out[n] = grand total.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const TIn* in, TOut* out, int64_t n,
                                                            const TOut* __restrict__ boff) {
    __shared__ TOut tile[SCAN_TILE];
    __shared__ TOut warp_tot[SCAN_THREADS / 32];
    __shared__ TOut total;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int idx = i * SCAN_THREADS + threadIdx.x;
        int64_t g = base + idx;
        tile[idx] = (g < n) ? (TOut)in[g] : TOut(0);
    }
    __syncthreads();
    TOut loc[SCAN_ITEMS];
    TOut sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        loc[i] = sum;
        sum += tile[threadIdx.x * SCAN_ITEMS + i];
    }
    TOut off = block_exclusive_sum<TOut>(sum, warp_tot, &total);
    TOut bo = boff ? boff[blockIdx.x] : TOut(0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) tile[threadIdx.x * SCAN_ITEMS + i] = loc[i] + off + bo;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int idx = i * SCAN_THREADS + threadIdx.x;
        int64_t g = base + idx;
        if (g < n) out[g] = tile[idx];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = bo + total;
}

template <typename TIn, typename TOut>
static void scan_impl(Scratch& sc, const TIn* in, TOut* out, int64_t n) {
    cudaStream_t s = sc.stream();
    if (n <= 0) {
        FOLTY_CUDA(cudaMemsetAsync(out, 0, sizeof(TOut), s));
        return;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        FOLTY_LAUNCH((k_scan_down<TIn, TOut>), 1, SCAN_THREADS, 0, s, in, out, n, (const TOut*)nullptr);
        return;
    }
    TOut* bsum = sc.get<TOut>(nb + 1);
    FOLTY_LAUNCH((k_scan_reduce<TIn, TOut>), (unsigned)nb, SCAN_THREADS, 0, s, in, n, bsum);
    scan_impl<TOut, TOut>(sc, bsum, bsum, nb);
    FOLTY_LAUNCH((k_scan_down<TIn, TOut>), (unsigned)nb, SCAN_THREADS, 0, s, in, out, n, (const TOut*)bsum);
}

void exclusive_scan(Scratch& sc, const int32_t* in, int32_t* out, int64_t n) { scan_impl(sc, in, out, n); }
void exclusive_scan(Scratch& sc, const int32_t* in, int64_t* out, int64_t n) { scan_impl(sc, in, out, n); }
void exclusive_scan(Scratch& sc, const int64_t* in, int64_t* out, int64_t n) { scan_impl(sc, in, out, n); }
void exclusive_scan(Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n) { scan_impl(sc, in, out, n); }

// ================================================================== radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys per block
constexpr int RS_BITS = 11;
constexpr int RS_BINS = 1 << RS_BITS;

// Per-tile digit histogram, stored digit-major: hist[d * nblocks + block].
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                        int shift, uint32_t* __restrict__ hist,
                                                        int nblocks) {
    __shared__ uint32_t h[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * RS_THREADS + threadIdx.x;
        if (idx < n) {
            unsigned d = (unsigned)(keys[idx] >> shift) & (RS_BINS - 1);
            // aggregate equal digits within the warp before touching shared memory
            unsigned peers = __match_any_sync(__activemask(), d);
            if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&h[d], __popc(peers));
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) hist[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// Stable scatter. Warp w owns keys [base + w*32*ITEMS, ...) in order; within a warp the
// keys are ranked step by step with __match_any_sync, then warps are ordered per digit.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ keys,
                                                           const uint32_t* __restrict__ vals,
                                                           uint64_t* __restrict__ okeys,
                                                           uint32_t* __restrict__ ovals, int64_t n,
                                                           int shift,
                                                           const uint32_t* __restrict__ offs,
                                                           int nblocks) {
    // per-warp digit counts and offsets; at most RS_TILE = 4096 keys per block, so 16 bits
    __shared__ uint16_t wh[RS_WARPS][RS_BINS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wh[0][0])[i] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * 32 * RS_ITEMS;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = wbase + (int64_t)i * 32 + lane;
        bool valid = idx < n;
        k[i] = valid ? keys[idx] : 0ull;
        v[i] = valid ? vals[idx] : 0u;
        unsigned d = valid ? ((unsigned)(k[i] >> shift) & (RS_BINS - 1)) : (unsigned)RS_BINS;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned before = 0;
        if (valid) before = wh[warp][d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[warp][d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        rank[i] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wh[w][d];
            wh[w][d] = (uint16_t)run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = wbase + (int64_t)i * 32 + lane;
        if (idx < n) {
            unsigned d = (unsigned)(k[i] >> shift) & (RS_BINS - 1);
            uint32_t pos = offs[(int64_t)d * nblocks + blockIdx.x] + wh[warp][d] + rank[i];
            okeys[pos] = k[i];
            ovals[pos] = v[i];
        }
    }
}

bool radix_sort_pairs(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                      uint32_t* vals_alt, int64_t n, int bits) {
    if (n <= 1 || bits <= 0) return false;
    if (n >= (int64_t)0xffffffffll) fail(FOLTY_EINVAL, "radix sort: too many keys");
    cudaStream_t s = sc.stream();
    int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    int64_t hn = (int64_t)nblocks * RS_BINS;
    uint32_t* hist = sc.get<uint32_t>(hn + 1);
    bool alt = false;
    for (int shift = 0; shift < bits; shift += RS_BITS) {
        uint64_t* ki = alt ? keys_alt : keys;
        uint64_t* ko = alt ? keys : keys_alt;
        uint32_t* vi = alt ? vals_alt : vals;
        uint32_t* vo = alt ? vals : vals_alt;
        FOLTY_LAUNCH(k_rs_hist, nblocks, RS_THREADS, 0, s, ki, n, shift, hist, nblocks);
        exclusive_scan(sc, hist, hist, hn);
        FOLTY_LAUNCH(k_rs_scatter, nblocks, RS_THREADS, 0, s, ki, vi, ko, vo, n, shift, hist, nblocks);
        alt = !alt;
    }
    return alt;
}

}  // namespace folty
