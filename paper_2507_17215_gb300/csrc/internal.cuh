// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "folty.h"

namespace folty {

// ------------------------------------------------------------------ errors

struct Error {
    folty_status status;
    std::string msg;
};

[[noreturn]] inline void fail(folty_status st, const std::string& msg) { throw Error{st, msg}; }

inline void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        fail(FOLTY_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}
#define FOLTY_CUDA(expr) ::folty::cuda_check((expr), #expr)

void set_last_error(const std::string& msg);

// ------------------------------------------------------------------ launches

extern std::atomic<uint64_t> g_launches;

inline void after_launch(const char* name) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(FOLTY_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
}

#define FOLTY_LAUNCH(kernel, grid, block, smem, stream, ...)                   \
    do {                                                                       \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);            \
        ::folty::after_launch(#kernel);                                        \
    } while (0)

// Number of SMs of the current device (cached per device).
int num_sms();

// Grid for a grid-stride loop over n items: enough blocks to cover n, capped at a
// whole number of waves over all SMs.
inline unsigned grid_for(int64_t n, int block, int waves = 8) {
    int64_t need = (n + block - 1) / block;
    int64_t cap = (int64_t)num_sms() * waves;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

// ------------------------------------------------------------------ memory

struct Allocator {
    folty_allocator a{};
    bool user = false;

    void* get(size_t bytes, cudaStream_t s) const;
    void put(void* p, cudaStream_t s) const;
};

// Temporary device buffers of one call, released (stream-ordered) when it goes out of
// scope, also on error.
class Scratch {
  public:
    // err: the device error word of the graph the call works on (see read_back)
    Scratch(const Allocator& a, cudaStream_t s, int* err) : a_(a), s_(s), err_(err) {}
    ~Scratch() {
        for (void* p : ptrs_) a_.put(p, s_);
    }
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;

    // Buffers of at least CHUNK / 4 bytes are allocated on their own; smaller ones are
    // carved, 256-byte aligned, from shared chunks of CHUNK bytes, so that the many
    // counters, block aggregates and per-vertex arrays of one call cost a few allocator
    // calls rather than one each (a caller's allocator may be a costly callback).
    static constexpr size_t CHUNK = size_t(8) << 20;
    template <typename T>
    T* get(int64_t count) {
        size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes >= CHUNK / 4) return static_cast<T*>(take(bytes));
        if (bytes > left_) {
            cur_ = static_cast<char*>(take(CHUNK));
            left_ = CHUNK;
        }
        T* p = reinterpret_cast<T*>(cur_);
        cur_ += bytes;
        left_ -= bytes;
        return p;
    }
    cudaStream_t stream() const { return s_; }
    const Allocator& allocator() const { return a_; }
    int* err() const { return err_; }

  private:
    void* take(size_t bytes) {
        void* p = a_.get(bytes, s_);
        if (!p) fail(FOLTY_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        ptrs_.push_back(p);
        return p;
    }
    const Allocator& a_;
    cudaStream_t s_;
    int* err_;
    std::vector<void*> ptrs_;
    char* cur_ = nullptr;
    size_t left_ = 0;
};

// ------------------------------------------------------------------ the graph

constexpr int PROF_SLOTS = 64;       // probe-stage byte counters per graph
constexpr int HOST_STAGE = 512;      // pinned int64 slots per graph
constexpr int64_t PAIR_STAGE = 1 << 16;  // solution pairs staged in pinned memory per read-back
constexpr int READBACK_MAX = 384;    // slots [0, READBACK_MAX) serve read_back
constexpr int ERR_SLOT = READBACK_MAX + 8;  // the device error word's copy (load uses +0..+4, peeling +16..+27)
constexpr uint64_t GRAPH_TAG = 0x464f4c5459475248ull;   // "FOLTYGRH"
constexpr uint64_t RESULT_TAG = 0x464f4c5459525354ull;  // "FOLTYRST"
constexpr uint64_t FREED_TAG = 0x464f4c5459465245ull;   // "FOLTYFRE"

struct QueryPlans;  // query.cu

// Kernel shapes the autotuner (tune.cu) picks for a graph: the split of the triangle
// passes between one thread and one warp per oriented edge (by the length of the two
// out-lists), and the probe tile (the granularity the flat probe space is partitioned in)
// and grid of the probe kernel.
constexpr int TUNE_TRIALS = 4;
struct TuneParams {
    int32_t tri_heavy = 48;   // edges whose two out-lists hold more entries go to a whole warp
    int32_t probe_items = 8;  // probe tile = PB_THREADS * probe_items slots (4 or 8)
    int32_t probe_blocks = 0; // probe blocks per SM (0 = as many as fit)
    int32_t tri_source = 0;   // 0 default, 1 timed trials, 2 cache, 3 forced
    int32_t probe_source = 0;
    float tri_ms[TUNE_TRIALS] = {0, 0, 0, 0};    // trial times of the candidates
    float probe_ms[TUNE_TRIALS] = {0, 0, 0, 0};
};
constexpr int32_t TRI_HEAVY_CAND[TUNE_TRIALS] = {24, 48, 96, 1 << 30};
constexpr int32_t PROBE_CAND[TUNE_TRIALS][2] = {{4, 0}, {8, 0}, {8, 2}, {4, 4}};  // (items, blocks per SM)

}  // namespace folty

struct folty_graph {
    uint64_t tag;
    folty::Allocator alloc;
    int device;
    int state;  // 0 loaded, 1 preprocessed
    int32_t n;
    int64_t m;
    // ---- loaded input (device copies; released by preprocess)
    int32_t* in_src;
    int32_t* in_dst;
    int64_t* in_t;
    // the first try of the pair table, filled by a load of device or pinned input
    // (pairs.cuh; released by preprocess): table of 2^pre_lg slots, slot words, flags
    uint64_t* pre_table;
    uint32_t* pre_slotw;
    int* pre_flags;
    int pre_lg;
    // ---- preprocessed store (device)
    int64_t m_kept;
    int32_t* perm;    // [m_kept] input index of each sorted temporal edge (null while cw
                      // is kept for it: ensure_perm)
    uint32_t* cw;     // [m] sort id of each input edge (2 * static edge id + direction,
                      // 2S for a self-loop), kept when perm is made on first use
    uint32_t* store_hist;  // digit histograms of the sort ids (with cw)
    int store_cbits;       // significant bits of a sort id (with cw)
    std::mutex perm_mu;
    cudaEvent_t perm_ev;   // recorded after perm's sort on the stream of its first use
    void* T;          // [m_kept] timestamps sorted by (static edge, direction, t): uint32
                      // offsets t - tmin when ts32, else int64
    int ts32;
    int32_t* sd;      // [m_kept] 2 * static edge id + direction bit
    int32_t S;        // static edges
    int32_t* seg;     // [2S + 1]: E_{a->b} = [seg[2s], seg[2s+1]), E_{b->a} = [seg[2s+1], seg[2s+2])
    int32_t* ea;      // [S] smaller endpoint a
    int32_t* eb;      // [S] larger endpoint b
    int32_t* deg;     // [n] |N(u)|
    int32_t* core;    // [n] core numbers of G_S
    int32_t* common;  // [S] |N(a) cap N(b)| = triangles on the static edge
    int32_t* by_b;    // [S] static edge ids ordered by (b, a)
    int32_t* prank;   // [2S] rank of directed pair 2s + d in (u, v) order (batched queries; made on first use)
    int64_t ntri;
    int4* tri;        // [ntri] {s_uv, s_uw, s_vw, id-order bits}, u < v < w in degeneracy rank
    int64_t* tri_off; // [ntri + 1] prefix of per-triangle probe counts (null past FOLTY_NOALLOC_MAX_EDGES edges)
    int64_t* tile_tri;  // [probe tiles + 1] triangle holding each tile's first probe (null with tri_off)
    unsigned long long* prof_bytes;  // [PROF_SLOTS] device counters of probe-stage model bytes
    int prof_next;                   // next slot
    void* run_ends;     // [S] first and last timestamp and size of both runs of every static edge
    uint8_t* tlive;     // [3][tlive_stride] per direction variant, the smallest window bucket of a triangle's roles
    int64_t tlive_stride;
    // a direction variant's row of tlive is written by the first call that needs it
    // (ensure_liveness): the row is ready once live_ev[dir] (recorded on that call's
    // stream) has completed
    std::mutex live_mu;
    int live_ready[3];
    cudaEvent_t live_ev[3];
    int64_t n_tiles;
    int64_t enum_bytes; // model bytes of the triangle enumeration
    int64_t tmin, tmax; // timestamp range of the input
    // ---- statistics
    folty_graph_info info;
    // ---- pinned host staging for small device->host reads
    int64_t* host_stage;  // HOST_STAGE entries, then 4 * PAIR_STAGE int32 (pair_stage)
    int64_t* stage_dev;   // device address of host_stage
    int32_t* pair_stage;  // kernel-written pair output (device address of the same memory)
    int stage_busy;       // an asynchronous copy into or out of host_stage may be pending
    int* dev_err;         // device error word: a bounded wait in a kernel ran out
    std::vector<std::pair<void*, size_t>>* owned;  // device buffers owned by the graph
    folty::QueryPlans* plans;  // captured launch sequences of plain queries (query.cu), made on first use
    folty::TuneParams tune;    // kernel shapes (tune.cu)
};

namespace folty {

// Allocates a device buffer owned by the graph (freed by folty_free).
template <typename T>
T* graph_alloc(folty_graph* g, int64_t count, cudaStream_t s) {
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    void* p = g->alloc.get(bytes, s);
    if (!p) fail(FOLTY_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    g->owned->push_back({p, bytes});
    g->info.device_bytes += (int64_t)bytes;
    return static_cast<T*>(p);
}
void graph_release(folty_graph* g, void* p, cudaStream_t s);

// Reads `count` int64 values from device memory through the graph's pinned staging
// buffer (synchronises the stream). Also reads the graph's device error word: when a
// bounded wait in an earlier kernel ran out, the word is cleared and the call fails with
// FOLTY_ETIMEOUT before any value is used. count may be 0 (a plain check).
void read_back(folty_graph* g, const void* const* dev_ptrs, const int* sizes, int count,
               int64_t* out, cudaStream_t s);
// The two halves of read_back: the gathering launch (no synchronisation; capturable in
// a CUDA graph), and, after the caller synchronised the stream, the error check and the
// values.
void enqueue_read_back(folty_graph* g, const void* const* dev_ptrs, const int* sizes, int count, cudaStream_t s);
void collect_read_back(folty_graph* g, int count, int64_t* out, cudaStream_t s);
int64_t read_i64(folty_graph* g, const int64_t* p, cudaStream_t s);
int32_t read_i32(folty_graph* g, const int32_t* p, cudaStream_t s);

// ------------------------------------------------------------------ primitives (prims.cu)

// Exclusive prefix sum of in[0..n) into out[0..n], out[n] = total. in may equal out
// (then out needs n + 1 slots).
void exclusive_scan(Scratch& sc, const int32_t* in, int32_t* out, int64_t n);
void exclusive_scan(Scratch& sc, const int32_t* in, int64_t* out, int64_t n);
void exclusive_scan(Scratch& sc, const int64_t* in, int64_t* out, int64_t n);
void exclusive_scan(Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n);

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits). Buffers ping-pong
// between (keys, vals) and (keys_alt, vals_alt); returns true when the result ended
// up in the *_alt buffers. A look-back wait that runs out sets the scratch error word and
// leaves the output unusable: the caller checks the word before the values index anything.
bool radix_sort_pairs(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                      uint32_t* vals_alt, int64_t n, int bits);
// The same ordered by key bits [lo, lo + bits) (lower bits ride along).
bool radix_sort_pairs(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                      int64_t n, int lo, int bits);
// The same for keys alone, ordered by key bits [lo, lo + bits) (lower bits ride along).
bool radix_sort_keys(Scratch& sc, uint64_t* keys, uint64_t* keys_alt, int64_t n, int lo, int bits);

// The temporal store's sort of a time-ordered edge list: the n edges by sort id cw[j]
// (< 2^cbits; equal ids keep input order), each carrying its time offset t[j] - tmin;
// sorted position i < limit receives T[i] = t[j] - tmin and sd[i] = cw[j] (the positions
// past limit hold the largest ids and are dropped). hist[p][b]: the number of ids whose
// 8-bit digit p (bits 8p ...) is b, for the ceil(cbits / 8) passes, counted by the
// caller. Like radix_sort_pairs, a look-back wait that runs out sets the scratch error
// word. perm_sort: the same order, perm[i] = j (t, T and sd unused).
constexpr int STORE_DIGIT_BITS = 8;
constexpr int STORE_MAX_PASSES = 4;
struct StoreSortArgs {
    const uint32_t* cw;
    const int64_t* t;
    int64_t tmin;
    int64_t n;
    int cbits;
    const uint32_t* hist;  // [STORE_MAX_PASSES][1 << STORE_DIGIT_BITS]
    uint32_t* T;
    int32_t* sd;
    int32_t* perm;
    int64_t limit;
};
void store_sort(Scratch& sc, const StoreSortArgs& a);
void perm_sort(Scratch& sc, const StoreSortArgs& a);

int bit_length(uint64_t x);

// ------------------------------------------------------------------ pipeline stages

void preprocess_graph(folty_graph* g, cudaStream_t s);          // preprocess.cu
void run_query(folty_graph* g, const folty_query_params& q, folty_result* out,
               cudaStream_t s);                                  // query.cu
void destroy_plans(folty_graph* g);                              // query.cu
// bin_budget: device bytes the per-delta bins may take (<= 0: a quarter of the free
// memory, at most 16 GiB); deltas beyond it are handled in further probe passes.
void run_query_batch(folty_graph* g, const folty_query_params* qs, int nq,
                     folty_result* outs, cudaStream_t s, int64_t bin_budget = 0);  // batch.cu
// Device bytes a batch of these queries takes beyond the graph (bins + output stages).
int64_t batch_footprint(const folty_graph* g, const folty_query_params* qs, int nq, int64_t* bins_part);
void traffic_model(folty_graph* g, int dir, folty_traffic_model* out, cudaStream_t s);

void validate_query(const folty_query_params& q);
// Device-time profiling by stage (folty_profile_enable/read). While profiling is on,
// a ProfileScope at an API entry collects the StageSpans opened during the call: each
// span records CUDA events on the launching stream around a stage's launches, with the
// stage's model bytes (host-known, plus an optional device-side counter). The scope's
// commit(), called after the call's final stream synchronisation, adds the elapsed
// times to process-wide totals.
enum { ST_PROBE = 0, ST_SORT = 1, ST_PEEL = 2, ST_THRESHOLD = 3, ST_SELECT = 4, ST_TRIANGLES = 5, ST_ROLES = 6,
       ST_BATCH = 7, ST_STORE = 8, ST_COUNT = 9 };
static_assert(ST_COUNT == FOLTY_STAGE_COUNT, "stage numbering follows folty.h");

class StageSpan {
  public:
    StageSpan(int stage, cudaStream_t s, int64_t bytes, const unsigned long long* dev_bytes = nullptr);
    ~StageSpan();
    StageSpan(const StageSpan&) = delete;
    StageSpan& operator=(const StageSpan&) = delete;
    // Adds model bytes that became known after the span opened (e.g. from a read-back).
    void add_bytes(int64_t bytes);
    // Closes the span now (the destructor then records nothing).
    void end();

  private:
    int idx_ = -1;
    bool ended_ = false;
    cudaStream_t s_;
};

class ProfileScope {
  public:
    ProfileScope();
    ~ProfileScope();
    void commit();  // after the call's final synchronisation

  private:
    bool active_ = false;
};
bool profiling_on();

// Window-probe pass of one query into counters cnt[m_kept] (sorted order, zeroed).
void launch_probe(folty_graph* g, int64_t delta, int dir, int32_t* cnt, cudaStream_t s);
// Window probes of the roles that can hit (live.cu): mode 0 counts hits at delta into
// cnt or, with bins16 (cnt null), into 16-bit counters two to a word; mode 1 bins gaps
// <= delta against the k sorted bounds `deltas` (in the timestamp store's type) into
// edge-major rows of kstride bins (bin j of sorted edge e at e * kstride + j), as int32 or,
// with bins16 (bins null), as 16-bit counts (counts must stay below 2^16).
// rflag (mode 0, may be null): byte 6 * triangle + role set to 1 when the role has a hit.
// touched (mode 1, may be null): bit g of word g / 32 set when one of sorted edges
// [32 g, 32 g + 32) received a binned hit (the caller clears the words first).
void launch_probe_live(folty_graph* g, int64_t delta, int dir, int mode, int32_t* cnt, int32_t* bins, int k,
                       int kstride, const void* deltas, cudaStream_t s, uint8_t* rflag = nullptr,
                       uint16_t* bins16 = nullptr, uint32_t* touched = nullptr);
// Autotuner (tune.cu). Parameters are cached process-wide by graph statistics (a key of
// int64 values); forced parameters (folty_tuning_force) take precedence over both.
bool tune_lookup(const std::vector<int64_t>& key, TuneParams* p, bool probe);
void tune_store(const std::vector<int64_t>& key, const TuneParams& p, bool probe);
bool tune_forced(TuneParams* p, bool probe);
// Picks the probe tile and grid for g by timed trials of the probe pass of (delta, dir),
// unless forced or cached (live.cu); the triangle split is picked in preprocess.cu.
void tune_probe(folty_graph* g, int64_t delta, int dir, cudaStream_t s);

// The run-ends table (live.cu; needs the sorted store), the rows of per-triangle
// liveness bytes with their padding; triangle_liveness then fills the out motif's row
// from the listed triangles. With from, the triangles still lie in the bounded layout
// of a one-pass listing, and the same pass moves them into g->tri.
struct TriLayout {
    const int32_t* cnt;   // [S] triangles of each oriented edge
    const int64_t* toff;  // [S + 1] prefix of cnt
    const int64_t* boff;  // [S + 1] prefix of the per-edge bounds: edge j's triangles at tri_b[boff[j] ...]
    const int4* tri_b;
};
void build_run_ends(folty_graph* g, cudaStream_t s);
void prepare_liveness(folty_graph* g, cudaStream_t s);
void triangle_liveness(folty_graph* g, cudaStream_t s, const TriLayout* from = nullptr);
// Makes the liveness row of direction variant dir ready for work enqueued on s after the
// call: computes it on s the first time (thread-safe), else makes s wait for the
// computation. Not while s is capturing.
void ensure_liveness(folty_graph* g, int dir, cudaStream_t s);
// Makes g->perm (sorted position -> input index) if the graph kept the sort ids instead,
// on stream s, once; later calls make s wait for it.
void ensure_perm(folty_graph* g, cudaStream_t s);
// Device buffers of one query's probe stage (kept triangles, probe tiles, look-back
// control).
struct ProbeBuffers {
    int32_t* L;
    int64_t* loff;
    uint8_t* lmask;
    int64_t* totals;  // kept triangles, slots
    int64_t* ltile;
    int64_t max_tiles;
    int32_t* wcnt;    // per selection warp: kept triangles, then their exclusive prefix
    int64_t* wcost;   // per selection warp: their slots, then the exclusive prefix
    int64_t nw;
};
// The same buffers owned by the graph (held by its query plans).
ProbeBuffers probe_buffers(folty_graph* g, cudaStream_t s);
// Selection and probes of one query into counters (cnt or cnt16, zeroed), the window
// taken from the device parameter block qp (slot 0: 64-bit, slot 1: the 32-bit store's
// clamped value): no host value in any launch, so a captured sequence replays for any
// window.
void enqueue_probe_pass(folty_graph* g, const int64_t* qp, int dir, const ProbeBuffers& pb, int32_t* cnt,
                        uint16_t* cnt16, cudaStream_t s);
// Kept roles, probes and model bytes of one query's selection (live.cu; synchronises).
void probe_stats(folty_graph* g, int64_t delta, int dir, folty_probe_stats* out, cudaStream_t s);
// The same pass with the counters in a file-scope device array (noalloc.cu).
void edge_counts_noalloc(folty_graph* g, int64_t delta, int dir, int32_t* edge_count, cudaStream_t s);
// Per-edge counts of one query: int32 (c32) or 16-bit (c16), the other null.
struct CountView {
    const int32_t* c32;
    const uint16_t* c16;
};
// Threshold, pair output and result copy-out of nq queries at once (per-edge counts
// cnts[i], sorted order): one stream synchronisation for the whole group, a second
// one only when lists that did not fit the pinned pair stage (or edge counts,
// certificates, vertex lists) are copied out after it.
void finish_queries(folty_graph* g, const folty_query_params* const* qs, const CountView* cnts, int nq,
                    folty_result* const* outs, cudaStream_t s);

void fill_result_host(folty_result* out, int64_t n_pairs, int64_t m, bool want_edges, int64_t n_vertices,
                      bool want_vertices, int64_t n_certs, bool want_certs);
// Host arrays for n all-existential triples in a filled result.
void fill_result_triples(folty_result* out, int64_t n);
// Frees a result's host arrays and marks it freed.
void release_result(folty_result* r);

// ------------------------------------------------------------------ device helpers

// First index in [lo, hi) with a[i] >= key (hi if none).
__device__ __forceinline__ int lower_bound_i64(const int64_t* __restrict__ a, int lo, int hi,
                                               int64_t key) {
    int len = hi - lo;
    while (len > 0) {
        int half = len >> 1;
        if (a[lo + half] < key) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

}  // namespace folty
