// Device-wide primitives: exclusive prefix sum and a stable LSD radix sort.
//
// Both are bandwidth-bound streaming passes: tiles of 2048 (scan) or 4096 (sort)
// elements per 256-thread block, coalesced loads, block offsets from a recursive scan
// of per-tile totals (scan); one kernel per 8-bit digit with a decoupled look-back (sort).
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
//
// Stable LSD radix sort, one kernel per 8-bit digit ("onesweep"): the histograms of all
// digits come from one read of the keys up front; each pass takes tiles of 4096 keys in
// the order blocks start (a dynamic tile counter), ranks them by digit within the tile
// (warp multisplit with __match_any_sync), publishes the tile's digit counts, and adds
// the counts of all earlier tiles by looking back over their published values (decoupled
// look-back: a tile's entry holds either its own count or its inclusive prefix). Keys are
// then staged in shared memory in digit order, so that the global writes of each digit's
// run are contiguous.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys per tile
constexpr int RS_BITS = 8;
constexpr int RS_BINS = 1 << RS_BITS;
constexpr int RS_MAX_PASSES = 8;
constexpr unsigned long long LB_AGG = 1ull << 62;     // entry holds the tile's own count
constexpr unsigned long long LB_PREFIX = 1ull << 63;  // entry holds the inclusive prefix
constexpr unsigned long long LB_VALUE = LB_AGG - 1;

// hist[p][b] = number of keys whose digit p is b, for all passes at once.
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist_all(const uint64_t* __restrict__ keys, int64_t n, int passes,
                                                            uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[2][RS_MAX_PASSES][RS_BINS];  // two copies: even and odd warps
    for (int i = threadIdx.x; i < 2 * RS_MAX_PASSES * RS_BINS; i += RS_THREADS) (&h[0][0][0])[i] = 0;
    __syncthreads();
    const int copy = (threadIdx.x >> 5) & 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; p++) atomicAdd(&h[copy][p][(unsigned)(k >> (RS_BITS * p)) & (RS_BINS - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_BINS; i += RS_THREADS) {
        const uint32_t c = (&h[0][0][0])[i] + (&h[1][0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// base[p][b] = exclusive prefix of hist[p][.] (one block of RS_BINS threads).
__global__ void k_rs_bases(const uint32_t* __restrict__ hist, int passes, uint32_t* __restrict__ base) {
    __shared__ uint32_t wt[RS_BINS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int p = 0; p < passes; p++) {
        const uint32_t v = hist[p * RS_BINS + threadIdx.x];
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wt[w] = inc;
        __syncthreads();
        uint32_t off = 0;
        for (int j = 0; j < w; j++) off += wt[j];
        base[p * RS_BINS + threadIdx.x] = off + inc - v;
        __syncthreads();
    }
}

struct OnesweepArgs {
    const uint64_t* keys;
    const uint32_t* vals;
    uint64_t* okeys;
    uint32_t* ovals;
    int64_t n;
    int shift;
    const uint32_t* base;  // [RS_BINS] digit bases of this pass
    unsigned long long* lb;  // [tiles][RS_BINS] look-back entries, zeroed
    unsigned int* tile_counter;  // zeroed
    int* err;
    long long timeout_ns;
};

__device__ __forceinline__ long long rs_now() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_onesweep(OnesweepArgs a) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t* skey = (uint64_t*)rs_smem;                  // RS_TILE
    uint32_t* sval = (uint32_t*)(skey + RS_TILE);         // RS_TILE
    __shared__ uint16_t wh[RS_WARPS][RS_BINS];            // per-warp counts, then offsets
    __shared__ uint32_t bstart[RS_BINS];                  // tile-local start of each digit
    __shared__ unsigned long long gofs[RS_BINS];          // global start of each digit's run
    __shared__ uint32_t wt[RS_THREADS / 32];
    __shared__ int s_tile, s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wh[0][0])[i] = 0;
    if (threadIdx.x == 0) {
        s_tile = (int)atomicAdd(a.tile_counter, 1u);
        s_fail = 0;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t t0 = tile * RS_TILE;
    const int tn = (int)min((int64_t)RS_TILE, a.n - t0);
    // ---- rank within the tile: warp w owns keys [w * 32 * ITEMS, ...) in order
    const int wbase = warp * 32 * RS_ITEMS;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint16_t rank[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        const int idx = wbase + i * 32 + lane;
        const bool valid = idx < tn;
        k[i] = valid ? a.keys[t0 + idx] : 0ull;
        v[i] = valid ? a.vals[t0 + idx] : 0u;
        const unsigned d = valid ? ((unsigned)(k[i] >> a.shift) & (RS_BINS - 1)) : (unsigned)RS_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned before = 0;
        if (valid) before = wh[warp][d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[warp][d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        rank[i] = (uint16_t)(before + __popc(peers & lt_mask));
    }
    __syncthreads();
    // ---- per digit (thread d): warp offsets, tile count, publish, look back
    const int d = threadIdx.x;  // RS_THREADS == RS_BINS
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) {
        const uint32_t c = wh[w][d];
        wh[w][d] = (uint16_t)cnt;
        cnt += c;
    }
    volatile unsigned long long* lb = a.lb;
    lb[tile * RS_BINS + d] = (tile == 0 ? LB_PREFIX : LB_AGG) | cnt;
    {   // tile-local exclusive scan of the digit counts
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wt[warp] = inc;
        __syncthreads();
        uint32_t off = 0;
        for (int j = 0; j < warp; j++) off += wt[j];
        bstart[d] = off + inc - cnt;
    }
    unsigned long long excl = 0;
    if (tile > 0) {
        int64_t p = tile - 1;
        const long long t_start = rs_now();
        while (p >= 0) {
            const unsigned long long e = lb[p * RS_BINS + d];
            if (e == 0) {  // predecessor has not published yet
                if (rs_now() - t_start > a.timeout_ns) {
                    s_fail = 1;
                    atomicExch(a.err, 1);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            excl += e & LB_VALUE;
            if (e & LB_PREFIX) break;
            p--;
        }
        lb[tile * RS_BINS + d] = LB_PREFIX | (excl + cnt);
    }
    gofs[d] = (unsigned long long)a.base[d] + excl;
    __syncthreads();
    if (s_fail) return;  // block-uniform: positions are unknown
    // ---- stage in digit order, then write each digit's run contiguously
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        const int idx = wbase + i * 32 + lane;
        if (idx < tn) {
            const unsigned dd = (unsigned)(k[i] >> a.shift) & (RS_BINS - 1);
            const int lpos = (int)bstart[dd] + wh[warp][dd] + rank[i];
            skey[lpos] = k[i];
            sval[lpos] = v[i];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < tn; idx += RS_THREADS) {
        const uint64_t kk = skey[idx];
        const unsigned dd = (unsigned)(kk >> a.shift) & (RS_BINS - 1);
        const unsigned long long pos = gofs[dd] + (unsigned long long)(idx - (int)bstart[dd]);
        a.okeys[pos] = kk;
        a.ovals[pos] = sval[idx];
    }
}

constexpr size_t RS_DYN_SMEM = RS_TILE * (sizeof(uint64_t) + sizeof(uint32_t));

bool radix_sort_pairs(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                      uint32_t* vals_alt, int64_t n, int bits, int* err) {
    if (n <= 1 || bits <= 0) return false;
    if (n >= (int64_t)0xffffffffll) fail(FOLTY_EINVAL, "radix sort: too many keys");
    cudaStream_t s = sc.stream();
    const int passes = (bits + RS_BITS - 1) / RS_BITS;
    const int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    uint32_t* hist = sc.get<uint32_t>(2 * RS_MAX_PASSES * RS_BINS);
    uint32_t* base = hist + RS_MAX_PASSES * RS_BINS;
    unsigned long long* lb = sc.get<unsigned long long>(tiles * RS_BINS);
    unsigned int* counter = sc.get<unsigned int>(1);
    FOLTY_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * RS_MAX_PASSES * RS_BINS, s));
    {
        StageSpan span(ST_SORT, s, 8 * n);  // all digit histograms: one read of the keys
        FOLTY_LAUNCH(k_rs_hist_all, grid_for(n, RS_THREADS, 4), RS_THREADS, 0, s, keys, n, passes, hist);
        FOLTY_LAUNCH(k_rs_bases, 1, RS_BINS, 0, s, hist, passes, base);
    }
    FOLTY_CUDA(cudaFuncSetAttribute(k_rs_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_DYN_SMEM));
    bool alt = false;
    for (int p = 0; p < passes; p++) {
        StageSpan span(ST_SORT, s, 24 * n);  // 12 B read + 12 B written per key
        FOLTY_CUDA(cudaMemsetAsync(lb, 0, sizeof(unsigned long long) * (size_t)(tiles * RS_BINS), s));
        FOLTY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
        OnesweepArgs oa{alt ? keys_alt : keys, alt ? vals_alt : vals, alt ? keys : keys_alt, alt ? vals : vals_alt,
                        n, RS_BITS * p, base + p * RS_BINS, lb, counter, err, 10ll * 1000 * 1000 * 1000};
        FOLTY_LAUNCH(k_rs_onesweep, (unsigned)tiles, RS_THREADS, RS_DYN_SMEM, s, oa);
        alt = !alt;
    }
    return alt;
}

}  // namespace folty
