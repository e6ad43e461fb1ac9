// The dense pair-id table shared by the load (which fills it while it copies device or
// pinned input) and the preprocessing (which fills it otherwise, and numbers its pairs).
// An open-addressed table of 2^lg slots (linear probing from a multiplicative hash of the
// pair rank); slot value = rank + 1, 0 = empty.
#pragma once
#include <cstdlib>
#include <cstring>

#include "internal.cuh"

namespace folty {

constexpr int PAIR_MAX_PROBE = 4096;                       // longer probe sequences abandon the table
constexpr uint64_t PAIR_HASH_MUL = 0x9E3779B97F4A7C15ull;  // 2^64 / golden ratio (Fibonacci hashing)
constexpr uint32_t PAIR_LOOP = 0x7fffffffu;  // slot word of a self-loop
constexpr uint32_t PAIR_DIR = 0x80000000u;   // direction bit of a slot word (tables hold < 2^31 slots)

__device__ __forceinline__ uint64_t pair_rank_of(int32_t x, int32_t y, int32_t n) {
    const uint64_t a = (uint64_t)min(x, y), b = (uint64_t)max(x, y);
    return a * (2 * (uint64_t)n - a - 1) / 2 + (b - a - 1);
}

// Slot holding table value key (rank + 1), placing it in the first empty slot of its probe
// sequence when absent; -1 after PAIR_MAX_PROBE steps.
__device__ __forceinline__ int64_t pair_slot(uint64_t* table, int lg, uint64_t key) {
    const uint64_t mask = (1ull << lg) - 1;
    uint64_t h = (key * PAIR_HASH_MUL) >> (64 - lg);
    for (int pr = 0; pr < PAIR_MAX_PROBE; pr++) {
        const uint64_t cur = __ldcg(&table[h]);
        if (cur == key) return (int64_t)h;
        if (cur == 0) {
            const unsigned long long old =
                atomicCAS((unsigned long long*)&table[h], 0ull, (unsigned long long)key);
            if (old == 0 || old == key) return (int64_t)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Slot word of edge x -> y: its pair's slot and direction, PAIR_LOOP for a self-loop; a
// probe sequence that runs out sets *over.
__device__ __forceinline__ uint32_t pair_slot_word(uint64_t* table, int lg, int32_t x, int32_t y, int32_t n,
                                                   int* over) {
    if (x == y) return PAIR_LOOP;
    const int64_t sl = pair_slot(table, lg, pair_rank_of(x, y, n) + 1);
    if (sl < 0) {
        atomicExch(over, 1);
        return PAIR_LOOP;
    }
    return (uint32_t)sl | (x > y ? PAIR_DIR : 0u);
}

// log2 of the table's largest size for m edges (at least 2m slots, up to 2^23) and of
// its first try: at least m / 12 slots (room for m / 24 distinct pairs at a load factor
// of 1/2, i.e. a mean multiplicity of 24 or more, as in the workloads' Zipf
// multiplicities), at most 2^22 slots (32 MB, which stays in L2).
inline int pair_table_lg_max(int64_t m) {
    int b = 0;
    for (uint64_t v = (uint64_t)(2 * m - 1); v; v >>= 1) b++;
    return b < 10 ? 10 : (b > 23 ? 23 : b);
}
inline int pair_table_lg_first(int64_t m) {
    int b = 0;
    for (uint64_t v = (uint64_t)((m + 11) / 12); v; v >>= 1) b++;
    b = b < 10 ? 10 : (b > 22 ? 22 : b);
    return pair_table_lg_max(m) < b ? pair_table_lg_max(m) : b;
}

// The dense-id path is off when FOLTY_PAIR_SORT=keys (the full-key sort then runs).
inline bool pair_table_forced_off() {
    const char* env = std::getenv("FOLTY_PAIR_SORT");
    return env && std::strcmp(env, "keys") == 0;
}

}  // namespace folty
