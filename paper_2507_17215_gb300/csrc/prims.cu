// Device-wide primitives: exclusive prefix sum and a stable LSD radix sort.
//
// Both are bandwidth-bound streaming passes over tiles of 4096 elements (2048 for 8-byte
// scans) per 256-thread block, with coalesced loads and stores; a tile's offset comes
// from a decoupled look-back over the totals that earlier tiles publish, so each pass is
// a single kernel. Every look-back wait is bounded in time and reports through the
// scratch error word.
#include "internal.cuh"
#include "scan.cuh"

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
//
// Single pass: tiles are taken in the order blocks start (a dynamic tile counter); each
// tile publishes its total, then warp 0 looks back over up to 32 earlier tiles at a
// time until it meets one whose entry already holds an inclusive prefix (decoupled
// look-back). Entries pack a 2-bit status with a 62-bit value, so totals must stay
// below 2^62 (all scanned values are non-negative counts).

// One tile of TILE = SCAN_THREADS * ITEMS elements: coalesced loads into shared memory
// (padded so that each thread's run of ITEMS is conflict-free), a sequential sum per
// thread, a block scan, the look-back, and coalesced stores. The last tile also writes
// out[n] = the grand total. in may equal out.
template <typename TIn, typename TOut, int ITEMS>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const TIn* in, TOut* out, int64_t n,
                                                       unsigned long long* lb, unsigned int* counter, int* err) {
    constexpr int TILE = SCAN_THREADS * ITEMS;
    constexpr int PADW = 128 / sizeof(TOut);  // one pad element per 128 bytes
    __shared__ TOut buf[TILE + TILE / PADW];
    __shared__ TOut warp_tot[SCAN_THREADS / 32];
    __shared__ TOut total;
    __shared__ unsigned long long s_excl;
    __shared__ int64_t s_tile;
    auto pad = [](int i) { return i + i / PADW; };
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * TILE;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const int idx = i * SCAN_THREADS + threadIdx.x;
        const int64_t g = base + idx;
        buf[pad(idx)] = (g < n) ? (TOut)in[g] : TOut(0);
    }
    __syncthreads();
    TOut loc[ITEMS];
    TOut sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        loc[i] = buf[pad(threadIdx.x * ITEMS + i)];
        sum += loc[i];
    }
    const TOut off = block_exclusive_sum<TOut>(sum, warp_tot, &total);
    if (threadIdx.x < 32) {
        volatile unsigned long long* vlb = lb;
        const unsigned long long tot = (unsigned long long)total;
        if (tile == 0) {
            if (threadIdx.x == 0) {
                vlb[0] = SC_PREFIX | tot;
                s_excl = 0;
            }
        } else {
            if (threadIdx.x == 0) vlb[tile] = SC_AGG | tot;
            const unsigned long long ex = warp_lookback(vlb, tile, tot, err);
            if (threadIdx.x == 0) s_excl = ex;
        }
    }
    __syncthreads();
    TOut run = (TOut)s_excl + off;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        buf[pad(threadIdx.x * ITEMS + i)] = run;
        run += loc[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const int idx = i * SCAN_THREADS + threadIdx.x;
        const int64_t g = base + idx;
        if (g < n) out[g] = buf[pad(idx)];
    }
    if (base + TILE >= n && threadIdx.x == 0) out[n] = (TOut)s_excl + total;
}

template <typename TIn, typename TOut>
static void scan_impl(Scratch& sc, const TIn* in, TOut* out, int64_t n) {
    cudaStream_t s = sc.stream();
    if (n <= 0) {
        FOLTY_CUDA(cudaMemsetAsync(out, 0, sizeof(TOut), s));
        return;
    }
    constexpr int ITEMS = sizeof(TOut) == 4 ? 16 : 8;
    constexpr int TILE = SCAN_THREADS * ITEMS;
    const int64_t tiles = (n + TILE - 1) / TILE;
    // one zeroed block: the tile counter, then one look-back entry per tile
    unsigned long long* ctl = sc.get<unsigned long long>(tiles + 1);
    FOLTY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(unsigned long long) * (size_t)(tiles + 1), s));
    FOLTY_LAUNCH((k_scan<TIn, TOut, ITEMS>), (unsigned)tiles, SCAN_THREADS, 0, s, in, out, n, ctl + 1,
                 (unsigned int*)ctl, sc.err());
}

void exclusive_scan(Scratch& sc, const int32_t* in, int32_t* out, int64_t n) { scan_impl(sc, in, out, n); }
void exclusive_scan(Scratch& sc, const int32_t* in, int64_t* out, int64_t n) { scan_impl(sc, in, out, n); }
void exclusive_scan(Scratch& sc, const int64_t* in, int64_t* out, int64_t n) { scan_impl(sc, in, out, n); }
void exclusive_scan(Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n) { scan_impl(sc, in, out, n); }

// ================================================================== radix sort
//
// Stable LSD radix sort, one kernel per 8-bit digit ("onesweep"): the histograms of all
// digits come from one read of the keys up front; each pass takes tiles of 4096 keys in
// the order blocks start (a dynamic tile counter), ranks them by digit within the tile,
// publishes the tile's digit counts, and adds the counts of all earlier tiles by looking
// back over their published values (decoupled look-back: a tile's entry holds either its
// own count or its inclusive prefix). The tile is then listed in digit order through
// shared memory, so that the global writes of each digit's run are contiguous.

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys per tile
constexpr int RS_BITS = 8;
constexpr int RS_BINS = 1 << RS_BITS;
constexpr int RS_MAX_PASSES = 8;
constexpr unsigned long long LB_AGG = 1ull << 62;     // entry holds the tile's own count
constexpr unsigned long long LB_PREFIX = 1ull << 63;  // entry holds the inclusive prefix
constexpr unsigned long long LB_VALUE = LB_AGG - 1;

// hist[p][b] = number of keys whose digit p (bits lo + 8p ...) is b, for all passes at once.
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist_all(const uint64_t* __restrict__ keys, int64_t n, int lo,
                                                            int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[2][RS_MAX_PASSES][RS_BINS];  // two copies: even and odd warps
    for (int i = threadIdx.x; i < 2 * RS_MAX_PASSES * RS_BINS; i += RS_THREADS) (&h[0][0][0])[i] = 0;
    __syncthreads();
    const int copy = (threadIdx.x >> 5) & 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; p++)
            atomicAdd(&h[copy][p][(unsigned)(k >> (lo + RS_BITS * p)) & (RS_BINS - 1)], 1u);
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
    const uint32_t* vals;  // null for a keys-only sort
    uint64_t* okeys;
    uint32_t* ovals;
    int64_t n;
    int shift;
    const uint32_t* base;  // [RS_BINS] digit bases of this pass
    unsigned long long* lb;  // [tiles][RS_BINS] look-back entries, zeroed
    unsigned int* tile_counter;  // zeroed
    int* err;
    long long timeout_ns;
    // 32-bit keys (the store's sorts): keys32 and okeys32 in place of keys and okeys
    const uint32_t* keys32;
    uint32_t* okeys32;
    // the store's first pass (ST_FIRST): key j = cw[j], value t[j] - tmin (ST_IOTA: j),
    // read from the edge list itself (keys and vals unused)
    const uint32_t* cw;
    const int64_t* t;
    int64_t tmin;
    // its last pass (ST_LAST): sorted position i < limit gets T[i] = value and sd[i] =
    // key (ST_IOTA: perm[i] = value); okeys and ovals are unused, and the positions past
    // limit (the self-loops' ids) are dropped
    int32_t* perm;
    uint32_t* T;
    int32_t* sd;
    int64_t limit;
};

constexpr int ST_FIRST = 1;
constexpr int ST_LAST = 2;
constexpr int ST_IOTA = 4;

// Lanes whose 8-bit digit equals this lane's, from one ballot per bit (far cheaper than
// __match_any_sync on this GPU).
__device__ __forceinline__ unsigned digit_peers(unsigned d) {
    unsigned m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < RS_BITS; b++) {
        const bool bit = (d >> b) & 1u;
        const unsigned on = __ballot_sync(0xffffffffu, bit);
        m &= bit ? on : ~on;
    }
    return m;
}

// One pass of one 8-bit digit over a tile of NT * RS_ITEMS keys:
//  1. every load of the tile is issued before any is used; keys and values are staged
//     in shared memory in load order;
//  2. ranks within the tile: warp w owns keys [w * 32 * ITEMS, ...) in order, ranked by
//     digit with per-bit ballots and per-warp 16-bit counters (stable);
//  3. thread d < RS_BINS (one per digit) turns the per-warp counts into offsets,
//     publishes the tile's count of digit d and looks back over earlier tiles for its
//     global offset;
//  4. a 16-bit permutation in shared memory lists the tile in digit order, and the
//     writes of each digit's run are contiguous. Positions are 32-bit (n < 2^32).
// V: values travel with the keys (a keys-only sort moves 8 bytes a key instead of 12).
// NT: threads per block. The keys-only sort runs 512-thread blocks: tiles of 8192 keys
// halve the tiles in flight, and with them the depth of every look-back, and double the
// length of each digit's written run.
// K: the key type; 32-bit keys (the store's sorts, key-value only) move 8 bytes a key.
// MODE (ST_FIRST, ST_LAST, ST_IOTA flags, 32-bit keys only): the store's passes that
// build their keys from the edge list and write the store's arrays instead of keys and
// values.
template <bool V, int NT, int MODE = 0, typename K = uint64_t>
__global__ void __launch_bounds__(NT, V ? (sizeof(K) == 4 ? 4 : 3) : (NT == 512 ? 2 : 4))
    k_rs_onesweep(OnesweepArgs a) {
    static_assert(sizeof(K) == 8 || V, "32-bit keys carry values");
    static_assert(MODE == 0 || sizeof(K) == 4, "the store's passes sort 32-bit ids");
    constexpr int WARPS = NT / 32;
    constexpr int TILE = NT * RS_ITEMS;
    static_assert(NT % RS_BINS == 0 && NT >= RS_BINS, "one thread per digit at least");
    extern __shared__ __align__(16) unsigned char rs_smem[];
    K* skey = (K*)rs_smem;                                  // TILE, load order
    uint32_t* sval = (uint32_t*)(skey + TILE);              // TILE, load order (V only)
    uint16_t* sperm = (uint16_t*)(V ? (void*)(sval + TILE) : (void*)sval);  // TILE, digit order -> load order
    __shared__ uint16_t wh[WARPS][RS_BINS];                 // per-warp counts, then offsets
    __shared__ uint32_t bstart[RS_BINS];                    // tile-local start of each digit
    __shared__ uint32_t adj[RS_BINS];                       // final position of digit-order slot j: adj + j
    __shared__ uint32_t wt[RS_BINS / 32];
    __shared__ int s_tile, s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < WARPS * RS_BINS; i += NT) (&wh[0][0])[i] = 0;
    if (threadIdx.x == 0) {
        s_tile = (int)atomicAdd(a.tile_counter, 1u);
        s_fail = 0;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t t0 = tile * TILE;
    const int tn = (int)min((int64_t)TILE, a.n - t0);
    const K* kin = (sizeof(K) == 8 ? (const K*)a.keys : (const K*)a.keys32) + t0;
    K* kout = sizeof(K) == 8 ? (K*)a.okeys : (K*)a.okeys32;
    const uint32_t* vin = a.vals + t0;
    const int wbase = warp * 32 * RS_ITEMS;
    // ---- 1. loads, staging, digits
    uint32_t info[RS_ITEMS];  // digit | rank within (warp, digit) << 8
    {
        K kr[RS_ITEMS];
        uint32_t vr[RS_ITEMS];
#pragma unroll
        for (int i = 0; i < RS_ITEMS; i++) {
            const int idx = wbase + i * 32 + lane;
            if (MODE & ST_FIRST) {
                kr[i] = (idx < tn) ? (K)__ldcs(a.cw + t0 + idx) : (K)0;
                if (MODE & ST_IOTA) vr[i] = (uint32_t)(t0 + idx);
                else vr[i] = (idx < tn) ? (uint32_t)(__ldcs(a.t + t0 + idx) - a.tmin) : 0u;
            } else {
                kr[i] = (idx < tn) ? kin[idx] : (K)0;
                if (V) vr[i] = (idx < tn) ? vin[idx] : 0u;
            }
        }
#pragma unroll
        for (int i = 0; i < RS_ITEMS; i++) {
            const int idx = wbase + i * 32 + lane;
            if (idx < tn) {
                skey[idx] = kr[i];
                if (V) sval[idx] = vr[i];
            }
            info[i] = (unsigned)(kr[i] >> a.shift) & (RS_BINS - 1);
        }
    }
    // ---- 2. ranks: every item's peer mask first (independent ballot chains the scheduler
    // can interleave), then the per-warp counters item by item
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned pm[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) pm[i] = digit_peers(info[i]);
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        const int idx = wbase + i * 32 + lane;
        const bool valid = idx < tn;
        const unsigned dd = info[i];
        const unsigned peers = pm[i] & __ballot_sync(0xffffffffu, valid);
        unsigned before = 0;
        if (valid) before = wh[warp][dd];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[warp][dd] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        info[i] = dd | ((before + __popc(peers & lt_mask)) << 8);
    }
    __syncthreads();
    // ---- 3. per digit (thread d < RS_BINS): warp offsets, tile count, publish, look back
    const int d = threadIdx.x;
    const bool dig = d < RS_BINS;  // whole warps: RS_BINS is a multiple of 32
    uint32_t cnt = 0;
    if (dig) {
#pragma unroll
        for (int w = 0; w < WARPS; w++) {
            const uint32_t c = wh[w][d];
            wh[w][d] = (uint16_t)cnt;
            cnt += c;
        }
    }
    volatile unsigned long long* lb = a.lb;
    if (dig) lb[tile * RS_BINS + d] = (tile == 0 ? LB_PREFIX : LB_AGG) | cnt;
    uint32_t bs = 0;
    {   // tile-local exclusive scan of the digit counts (warps of digit threads)
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (dig && lane == 31) wt[warp] = inc;
        __syncthreads();
        if (dig) {
            uint32_t off = 0;
            for (int j = 0; j < warp; j++) off += wt[j];
            bs = off + inc - cnt;
            bstart[d] = bs;
        }
    }
    unsigned long long excl = 0;
    if (dig && tile > 0) {
        // four entries in flight per step; an entry not yet published is polled again
        int64_t p = tile - 1;
        long long t_start = 0;
        bool done = false;
        while (!done) {
            unsigned long long e[4];
#pragma unroll
            for (int j = 0; j < 4; j++) e[j] = (p - j >= 0) ? (unsigned long long)lb[(p - j) * RS_BINS + d] : LB_PREFIX;
            bool stall = false;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (!done && !stall) {
                    if (e[j] == 0) {
                        stall = true;
                    } else {
                        excl += e[j] & LB_VALUE;
                        p--;
                        if (e[j] & LB_PREFIX) done = true;
                    }
                }
            }
            if (stall && !done) {
                const long long t = globaltimer_ns();
                if (t_start == 0) {
                    t_start = t;
                } else if (t - t_start > a.timeout_ns) {
                    s_fail = 1;
                    atomicExch(a.err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        lb[tile * RS_BINS + d] = LB_PREFIX | (excl + cnt);
    }
    if (dig) adj[d] = (uint32_t)((unsigned long long)a.base[d] + excl) - bs;  // mod 2^32
    __syncthreads();
    if (s_fail) return;  // block-uniform: positions are unknown
    // ---- 4. digit-order permutation, then contiguous runs
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        const int idx = wbase + i * 32 + lane;
        if (idx < tn) {
            const unsigned dd = info[i] & (RS_BINS - 1);
            sperm[bstart[dd] + wh[warp][dd] + (info[i] >> 8)] = (uint16_t)idx;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < tn; j += NT) {
        const int src = sperm[j];
        const K kk = skey[src];
        const uint32_t pos = adj[(unsigned)(kk >> a.shift) & (RS_BINS - 1)] + (uint32_t)j;
        if (MODE & ST_LAST) {
            if ((int64_t)pos < a.limit) {
                if (MODE & ST_IOTA) {
                    __stcs(a.perm + pos, (int32_t)sval[src]);
                } else {
                    __stcs(a.T + pos, sval[src]);
                    __stcs(a.sd + pos, (int32_t)kk);
                }
            }
        } else {
            kout[pos] = kk;
            if (V) a.ovals[pos] = sval[src];
        }
    }
}

constexpr int RS_NT_K = 512;  // threads of a keys-only block
constexpr size_t RS_DYN_SMEM = RS_TILE * (sizeof(uint64_t) + sizeof(uint32_t) + sizeof(uint16_t));
constexpr size_t RS_DYN_SMEM_K = (size_t)RS_NT_K * RS_ITEMS * (sizeof(uint64_t) + sizeof(uint16_t));

// Sorts by the digits of bits [lo, lo + bits); vals may be null (keys only).
static bool radix_sort_impl(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                            int64_t n, int lo, int bits) {
    if (n <= 1 || bits <= 0) return false;
    if (n >= (int64_t)0xffffffffll) fail(FOLTY_EINVAL, "radix sort: too many keys");
    cudaStream_t s = sc.stream();
    const bool kv = vals != nullptr;
    const int passes = (bits + RS_BITS - 1) / RS_BITS;
    const int64_t tile = kv ? RS_TILE : (int64_t)RS_NT_K * RS_ITEMS;
    const int64_t tiles = (n + tile - 1) / tile;
    uint32_t* hist = sc.get<uint32_t>(2 * RS_MAX_PASSES * RS_BINS);
    uint32_t* base = hist + RS_MAX_PASSES * RS_BINS;
    // one zeroed block per pass: the tile counter, then the look-back entries
    unsigned long long* lbc = sc.get<unsigned long long>(tiles * RS_BINS + 1);
    unsigned int* counter = (unsigned int*)lbc;
    unsigned long long* lb = lbc + 1;
    FOLTY_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * RS_MAX_PASSES * RS_BINS, s));
    {
        StageSpan span(ST_SORT, s, 8 * n);  // all digit histograms: one read of the keys
        FOLTY_LAUNCH(k_rs_hist_all, grid_for(n, RS_THREADS, 4), RS_THREADS, 0, s, keys, n, lo, passes, hist);
        FOLTY_LAUNCH(k_rs_bases, 1, RS_BINS, 0, s, hist, passes, base);
    }
    if (kv) {
        FOLTY_CUDA(cudaFuncSetAttribute(k_rs_onesweep<true, RS_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)RS_DYN_SMEM));
    } else {
        FOLTY_CUDA(cudaFuncSetAttribute(k_rs_onesweep<false, RS_NT_K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)RS_DYN_SMEM_K));
        // two blocks of 90 KB each need the largest shared-memory carveout
        FOLTY_CUDA(cudaFuncSetAttribute(k_rs_onesweep<false, RS_NT_K>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    }
    bool alt = false;
    for (int p = 0; p < passes; p++) {
        StageSpan span(ST_SORT, s, (kv ? 24 : 16) * n);  // keys (and values) read and written once
        FOLTY_CUDA(cudaMemsetAsync(lbc, 0, sizeof(unsigned long long) * (size_t)(tiles * RS_BINS + 1), s));
        OnesweepArgs oa{alt ? keys_alt : keys, kv ? (alt ? vals_alt : vals) : nullptr, alt ? keys : keys_alt,
                        kv ? (alt ? vals : vals_alt) : nullptr, n, lo + RS_BITS * p, base + p * RS_BINS, lb, counter,
                        sc.err(), LOOKBACK_TIMEOUT_NS};
        if (kv) FOLTY_LAUNCH((k_rs_onesweep<true, RS_THREADS>), (unsigned)tiles, RS_THREADS, RS_DYN_SMEM, s, oa);
        else FOLTY_LAUNCH((k_rs_onesweep<false, RS_NT_K>), (unsigned)tiles, RS_NT_K, RS_DYN_SMEM_K, s, oa);
        alt = !alt;
    }
    return alt;
}

bool radix_sort_pairs(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                      uint32_t* vals_alt, int64_t n, int bits) {
    return radix_sort_impl(sc, keys, keys_alt, vals, vals_alt, n, 0, bits);
}

bool radix_sort_pairs(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                      int64_t n, int lo, int bits) {
    return radix_sort_impl(sc, keys, keys_alt, vals, vals_alt, n, lo, bits);
}

bool radix_sort_keys(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, int64_t n, int lo, int bits) {
    return radix_sort_impl(sc, keys, keys_alt, nullptr, nullptr, n, lo, bits);
}

static_assert(STORE_DIGIT_BITS == RS_BITS, "the caller's digit histograms match the passes");

template <int MODE>
static void store_pass(const OnesweepArgs& oa, int64_t tiles, cudaStream_t s) {
    constexpr size_t smem = RS_TILE * (sizeof(uint32_t) + sizeof(uint32_t) + sizeof(uint16_t));
    FOLTY_CUDA(cudaFuncSetAttribute(k_rs_onesweep<true, RS_THREADS, MODE, uint32_t>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FOLTY_LAUNCH((k_rs_onesweep<true, RS_THREADS, MODE, uint32_t>), (unsigned)tiles, RS_THREADS, smem, s, oa);
}

// The key-value sort of 32-bit sort ids (radix_sort_pairs' passes on 32-bit keys) whose
// first pass reads the ids and values from the edge list and whose last writes the
// store's arrays: no packed words, and no pass that unpacks the sorted ones.
template <bool IOTA>
static void store_sort_impl(Scratch& sc, const StoreSortArgs& a) {
    const int64_t n = a.n;
    if (n <= 0) return;
    if (n >= (int64_t)0xffffffffll) fail(FOLTY_EINVAL, "store sort: too many edges");
    const int passes = a.cbits > RS_BITS ? (a.cbits + RS_BITS - 1) / RS_BITS : 1;
    if (passes > STORE_MAX_PASSES) fail(FOLTY_EINVAL, "store sort: sort ids past 32 bits");
    cudaStream_t s = sc.stream();
    const int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    uint32_t* base = sc.get<uint32_t>(STORE_MAX_PASSES * RS_BINS);
    unsigned long long* lbc = sc.get<unsigned long long>(tiles * RS_BINS + 1);
    FOLTY_LAUNCH(k_rs_bases, 1, RS_BINS, 0, s, a.hist, passes, base);
    // the ids and values between passes, ping-ponged
    uint32_t* kb[2] = {nullptr, nullptr};
    uint32_t* vb[2] = {nullptr, nullptr};
    for (int i = 0; i < 2 && i < passes - 1; i++) {
        kb[i] = sc.get<uint32_t>(n);
        vb[i] = sc.get<uint32_t>(n);
    }
    constexpr int F = ST_FIRST | (IOTA ? ST_IOTA : 0), L = ST_LAST | (IOTA ? ST_IOTA : 0);
    for (int p = 0; p < passes; p++) {
        // 8 B read and written per edge (the first pass reads a 4 B id and an 8 B time, or
        // the id alone; the last writes two 4 B entries, or one)
        StageSpan span(ST_SORT, s, 16 * n);
        FOLTY_CUDA(cudaMemsetAsync(lbc, 0, sizeof(unsigned long long) * (size_t)(tiles * RS_BINS + 1), s));
        OnesweepArgs oa{};
        oa.keys32 = p > 0 ? kb[(p - 1) & 1] : nullptr;
        oa.vals = p > 0 ? vb[(p - 1) & 1] : nullptr;
        oa.okeys32 = kb[p & 1];
        oa.ovals = vb[p & 1];
        oa.n = n;
        oa.shift = RS_BITS * p;
        oa.base = base + p * RS_BINS;
        oa.lb = lbc + 1;
        oa.tile_counter = (unsigned int*)lbc;
        oa.err = sc.err();
        oa.timeout_ns = LOOKBACK_TIMEOUT_NS;
        oa.cw = a.cw;
        oa.t = a.t;
        oa.tmin = a.tmin;
        oa.perm = a.perm;
        oa.T = a.T;
        oa.sd = a.sd;
        oa.limit = a.limit;
        const bool first = p == 0, last = p == passes - 1;
        if (first && last) store_pass<F | L>(oa, tiles, s);
        else if (first) store_pass<F>(oa, tiles, s);
        else if (last) store_pass<L>(oa, tiles, s);
        else store_pass<0>(oa, tiles, s);
    }
}

void store_sort(Scratch& sc, const StoreSortArgs& a) { store_sort_impl<false>(sc, a); }
void perm_sort(Scratch& sc, const StoreSortArgs& a) { store_sort_impl<true>(sc, a); }

}  // namespace folty
