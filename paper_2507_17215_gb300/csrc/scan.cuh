// Device helpers of the single-pass scans (decoupled look-back), shared by the generic
// scan in prims.cu and the fused passes that scan while they select.
#pragma once
#include "internal.cuh"

namespace folty {

constexpr int SCAN_THREADS = 256;
constexpr unsigned long long SC_AGG = 1ull << 62;
constexpr unsigned long long SC_PREFIX = 1ull << 63;
constexpr unsigned long long SC_VALUE = SC_AGG - 1;
constexpr long long LOOKBACK_TIMEOUT_NS = 10ll * 1000 * 1000 * 1000;

__device__ __forceinline__ long long globaltimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

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

// Decoupled look-back by one warp: the sum of all tiles before `tile`. Publishes the
// tile's inclusive prefix. A wait that runs out sets *err and returns the partial sum
// (which never exceeds the true prefix: every value is non-negative).
__device__ __forceinline__ unsigned long long warp_lookback(volatile unsigned long long* lb, int64_t tile, unsigned long long total,
                                            int* err) {
    const int lane = threadIdx.x & 31;
    unsigned long long excl = 0;
    int64_t p = tile - 1;
    long long t_start = 0;
    while (p >= 0) {
        const int64_t q = p - lane;
        const unsigned long long e = (q >= 0) ? lb[q] : (SC_PREFIX | 0ull);
        const unsigned prefix = __ballot_sync(0xffffffffu, (e & SC_PREFIX) != 0);
        const unsigned waiting = __ballot_sync(0xffffffffu, e == 0);
        const int first = prefix ? __ffs(prefix) - 1 : 31;  // the lanes that matter: 0..first
        const unsigned need = (first == 31) ? 0xffffffffu : ((2u << first) - 1u);
        if (waiting & need) {
            const long long t = globaltimer_ns();
            if (t_start == 0) t_start = t;
            else if (t - t_start > LOOKBACK_TIMEOUT_NS) {
                if (lane == 0) atomicExch(err, 1);
                break;  // partial sum
            }
            __nanosleep(64);
            continue;
        }
        unsigned long long v = (lane <= first) ? (e & SC_VALUE) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (prefix) break;
        p -= 32;
    }
    if (lane == 0) lb[tile] = SC_PREFIX | (excl + total);
    return excl;
}


}  // namespace folty
