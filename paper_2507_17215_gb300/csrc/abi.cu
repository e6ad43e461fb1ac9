// The C ABI of folty.h: argument checks, object lifetime, error reporting, and the
// load step (copy + validation of the input edge list).
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <unordered_map>

#include "internal.cuh"
#include "pairs.cuh"

namespace folty {

std::atomic<uint64_t> g_launches{0};

static thread_local std::string t_last_error;

static std::atomic<int> g_profile_on{0};
static std::mutex g_profile_mu;
static folty_stage_profile g_stages[ST_COUNT];

struct StageRecord {
    int stage;
    cudaEvent_t a, b;
    int64_t bytes;
    const unsigned long long* dev_bytes;
};
static thread_local std::vector<StageRecord>* t_records = nullptr;

bool profiling_on() { return g_profile_on.load() != 0; }

StageSpan::StageSpan(int stage, cudaStream_t s, int64_t bytes, const unsigned long long* dev_bytes) : s_(s) {
    if (!t_records) return;
    StageRecord r{stage, nullptr, nullptr, bytes, dev_bytes};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(r.a, s);
    t_records->push_back(r);
    idx_ = (int)t_records->size() - 1;
}

void StageSpan::add_bytes(int64_t bytes) {
    if (idx_ >= 0 && t_records && idx_ < (int)t_records->size()) (*t_records)[idx_].bytes += bytes;
}

void StageSpan::end() {
    if (!ended_ && idx_ >= 0 && t_records && idx_ < (int)t_records->size()) cudaEventRecord((*t_records)[idx_].b, s_);
    ended_ = true;
}

StageSpan::~StageSpan() { end(); }

ProfileScope::ProfileScope() {
    if (profiling_on() && !t_records) {
        t_records = new std::vector<StageRecord>();
        active_ = true;
    }
}

void ProfileScope::commit() {
    if (!active_) return;
    std::lock_guard<std::mutex> lock(g_profile_mu);
    for (auto& r : *t_records) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int64_t bytes = r.bytes;
        if (r.dev_bytes) {
            unsigned long long v = 0;
            if (cudaMemcpy(&v, r.dev_bytes, sizeof(v), cudaMemcpyDeviceToHost) == cudaSuccess) bytes += (int64_t)v;
            else cudaGetLastError();
        }
        g_stages[r.stage].launches += 1;
        g_stages[r.stage].ms += ms;
        g_stages[r.stage].bytes += bytes;
    }
}

ProfileScope::~ProfileScope() {
    if (!active_) return;
    for (auto& r : *t_records) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete t_records;
    t_records = nullptr;
}

void set_last_error(const std::string& msg) { t_last_error = msg; }

int num_sms() {
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    FOLTY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) FOLTY_CUDA(cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev));
    return cache[dev];
}

// The library's own stream-ordered pool of the current device: created on first use and
// kept for the process. Unlike the device's default pool (release threshold 0, which
// hands freed memory back to the driver at every synchronisation, so that the next
// preprocessing maps it again), it keeps up to a quarter of the device's memory cached
// across calls.
static cudaMemPool_t library_pool() {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) total_b = 0;
        uint64_t keep = total_b / 4;
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
        pools[dev] = p;
    }
    return pools[dev];
}

// Freed blocks of the library pool, kept for the next request of the same rounded size:
// an allocation from the pool that is not the size of a block just freed costs the host
// about a microsecond per megabyte (measured: 0.3 ms for 280 MB, 1 to 1.4 ms for 1.8 GB,
// with the pool's reserved memory unchanged), and the stream waits for the host meanwhile.
// A cached block is handed out only once the event recorded at its free has completed
// (all work before the free is done, on every stream ordered before it), so that reuse
// adds no wait between streams; otherwise the request goes to the pool. At most a
// quarter of the device's memory stays cached; the oldest blocks go back to the pool,
// and all of a device's cached blocks do when the pool cannot serve a request.
namespace {
struct CachedBlock {
    void* p;
    size_t bytes;
    int dev;
    cudaEvent_t ev;
};
std::mutex g_cache_mu;
std::vector<CachedBlock> g_cache;                    // freed blocks, oldest first
std::unordered_map<void*, std::pair<size_t, int>> g_live;  // pool block -> rounded size, device
std::vector<cudaEvent_t> g_spare_events;
size_t g_cache_bytes = 0;
size_t g_cache_cap = 0;

size_t round_block(size_t bytes) {
    const size_t q = bytes >= (size_t(1) << 20) ? (size_t(2) << 20) : 512;
    return (bytes + q - 1) / q * q;
}
}  // namespace

void* Allocator::get(size_t bytes, cudaStream_t s) const {
    if (bytes == 0) bytes = 16;
    if (user) return a.alloc(bytes, (void*)s, a.ctx);
    bytes = round_block(bytes);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        for (size_t i = g_cache.size(); i-- > 0;) {
            CachedBlock& c = g_cache[i];
            if (c.dev != dev || c.bytes != bytes) continue;
            const cudaError_t q = cudaEventQuery(c.ev);
            if (q != cudaSuccess) {
                if (q != cudaErrorNotReady) cudaGetLastError();
                continue;
            }
            void* p = c.p;
            g_spare_events.push_back(c.ev);
            g_cache_bytes -= c.bytes;
            g_cache.erase(g_cache.begin() + (long)i);
            g_live[p] = {bytes, dev};
            return p;
        }
    }
    cudaMemPool_t pool = library_pool();
    void* p = nullptr;
    if (!pool) return nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        // the pool is out of memory: the cached blocks of this device go back to it first
        // (ordered after their frees on s, where the retry allocates), then one more try
        {
            std::lock_guard<std::mutex> lock(g_cache_mu);
            for (size_t i = 0; i < g_cache.size();) {
                CachedBlock c = g_cache[i];
                if (c.dev != dev) {
                    i++;
                    continue;
                }
                g_cache.erase(g_cache.begin() + (long)i);
                g_cache_bytes -= c.bytes;
                if (cudaStreamWaitEvent(s, c.ev, 0) != cudaSuccess) cudaGetLastError();
                cudaFreeAsync(c.p, s);
                g_spare_events.push_back(c.ev);
            }
        }
        if (cudaMallocFromPoolAsync(&p, bytes, pool, s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    }
    std::lock_guard<std::mutex> lock(g_cache_mu);
    g_live[p] = {bytes, dev};
    if (g_cache_cap == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) cudaGetLastError();
        g_cache_cap = total_b / 4 > 0 ? total_b / 4 : (size_t(1) << 30);
    }
    return p;
}

void Allocator::put(void* p, cudaStream_t s) const {
    if (!p) return;
    if (user) {
        a.free(p, (void*)s, a.ctx);
        return;
    }
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto it = g_live.find(p);
    cudaEvent_t ev = nullptr;
    if (!g_spare_events.empty()) {
        ev = g_spare_events.back();
        g_spare_events.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ev = nullptr;
    }
    if (it == g_live.end() || !ev || cudaEventRecord(ev, s) != cudaSuccess) {
        cudaGetLastError();
        if (ev) g_spare_events.push_back(ev);
        if (it != g_live.end()) g_live.erase(it);
        cudaFreeAsync(p, s);
        return;
    }
    g_cache.push_back(CachedBlock{p, it->second.first, it->second.second, ev});
    g_cache_bytes += it->second.first;
    g_live.erase(it);
    // over the cap: the oldest blocks of this device back to the pool, ordered after their
    // frees (s is a stream of the current device)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
    for (size_t i = 0; g_cache_bytes > g_cache_cap && i + 1 < g_cache.size();) {
        CachedBlock c = g_cache[i];
        if (c.dev != dev) {
            i++;
            continue;
        }
        g_cache.erase(g_cache.begin() + (long)i);
        g_cache_bytes -= c.bytes;
        if (cudaStreamWaitEvent(s, c.ev, 0) != cudaSuccess) cudaGetLastError();
        cudaFreeAsync(c.p, s);
        g_spare_events.push_back(c.ev);
    }
}

void graph_release(folty_graph* g, void* p, cudaStream_t s) {
    if (!p) return;
    auto& v = *g->owned;
    for (size_t i = 0; i < v.size(); i++) {
        if (v[i].first == p) {
            g->info.device_bytes -= (int64_t)v[i].second;
            v.erase(v.begin() + (long)i);
            g->alloc.put(p, s);
            return;
        }
    }
}

// The values of one read-back, gathered by one thread block into the pinned stage (one
// launch instead of a copy per value).
struct ReadbackArgs {
    const void* p[READBACK_MAX];
    uint8_t wide[READBACK_MAX];  // 1: an int64 value, 0: an int32 one (sign-extended)
    int count;
    const int* dev_err;  // may be null
    int64_t* out;        // device address of the stage's slots [0, count)
    int32_t* herr;       // device address of the error slot
};

__global__ void k_read_back(const __grid_constant__ ReadbackArgs a) {
    for (int i = threadIdx.x; i < a.count; i += blockDim.x)
        a.out[i] = a.wide[i] ? *static_cast<const int64_t*>(a.p[i]) : (int64_t)*static_cast<const int32_t*>(a.p[i]);
    if (threadIdx.x == 0) *a.herr = a.dev_err ? *a.dev_err : 0;
}

void enqueue_read_back(folty_graph* g, const void* const* dev_ptrs, const int* sizes, int count, cudaStream_t s) {
    if (count > READBACK_MAX) fail(FOLTY_EINVAL, "read_back: too many values");
    ReadbackArgs a;
    for (int i = 0; i < count; i++) {
        if (sizes[i] != 4 && sizes[i] != 8) fail(FOLTY_EINVAL, "read_back: values are 4 or 8 bytes");
        a.p[i] = dev_ptrs[i];
        a.wide[i] = sizes[i] == 8;
    }
    a.count = count;
    a.dev_err = g->dev_err;
    a.out = g->stage_dev;
    a.herr = (int32_t*)(g->stage_dev + ERR_SLOT);
    g->stage_busy = 1;
    FOLTY_LAUNCH(k_read_back, 1, 128, 0, s, a);
}

void collect_read_back(folty_graph* g, int count, int64_t* out, cudaStream_t s) {
    g->stage_busy = 0;
    if (*(volatile int32_t*)(g->host_stage + ERR_SLOT)) {
        FOLTY_CUDA(cudaMemsetAsync(g->dev_err, 0, sizeof(int32_t), s));
        fail(FOLTY_ETIMEOUT, "a bounded wait in a device look-back ran out; the results of this call are void");
    }
    for (int i = 0; i < count; i++) out[i] = ((volatile int64_t*)g->host_stage)[i];
}

void read_back(folty_graph* g, const void* const* dev_ptrs, const int* sizes, int count, int64_t* out,
               cudaStream_t s) {
    enqueue_read_back(g, dev_ptrs, sizes, count, s);
    FOLTY_CUDA(cudaStreamSynchronize(s));
    collect_read_back(g, count, out, s);
}

int64_t read_i64(folty_graph* g, const int64_t* p, cudaStream_t s) {
    const void* ptrs[1] = {p};
    int sizes[1] = {8};
    int64_t v;
    read_back(g, ptrs, sizes, 1, &v, s);
    return v;
}

int32_t read_i32(folty_graph* g, const int32_t* p, cudaStream_t s) {
    const void* ptrs[1] = {p};
    int sizes[1] = {4};
    int64_t v;
    read_back(g, ptrs, sizes, 1, &v, s);
    return (int32_t)v;
}

void fill_result_host(folty_result* out, int64_t n_pairs, int64_t m, bool want_edges, int64_t n_vertices,
                      bool want_vertices, int64_t n_certs, bool want_certs) {
    std::memset(out, 0, sizeof(*out));
    out->tag = RESULT_TAG;
    out->n_pairs = n_pairs;
    out->m = want_edges ? m : 0;
    if (n_pairs > 0) {
        int32_t* block = (int32_t*)std::malloc(sizeof(int32_t) * 4 * (size_t)n_pairs);
        if (!block) fail(FOLTY_ENOMEM, "host allocation of the result failed");
        out->u = block;
        out->v = block + n_pairs;
        out->count = block + 2 * n_pairs;
        out->ncert = block + 3 * n_pairs;
    }
    bool ok = true;
    if (want_edges) {
        out->edge_count = (int32_t*)std::calloc((size_t)(m > 0 ? m : 1), sizeof(int32_t));
        ok = ok && out->edge_count;
    }
    if (want_vertices) {
        out->n_vertices = n_vertices;
        out->vertex = (int32_t*)std::malloc(sizeof(int32_t) * 2 * (size_t)(n_vertices > 0 ? n_vertices : 1));
        out->vertex_count = out->vertex ? out->vertex + n_vertices : nullptr;
        ok = ok && out->vertex;
    }
    if (want_certs) {
        out->certificate = (int64_t*)std::malloc(sizeof(int64_t) * (size_t)(n_certs > 0 ? n_certs : 1));
        ok = ok && out->certificate;
    }
    if (!ok) {
        std::free(out->u);
        std::free(out->edge_count);
        std::free(out->vertex);
        std::free(out->certificate);
        std::memset(out, 0, sizeof(*out));
        fail(FOLTY_ENOMEM, "host allocation of the result failed");
    }
}

void fill_result_triples(folty_result* out, int64_t n) {
    out->n_triples = n;
    int32_t* block = (int32_t*)std::malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    if (!block) fail(FOLTY_ENOMEM, "host allocation of the result failed");
    out->triple_x = block;
    out->triple_y = block + n;
    out->triple_w = block + 2 * n;
}

void release_result(folty_result* r) {
    std::free(r->u);
    std::free(r->edge_count);
    std::free(r->vertex);
    std::free(r->certificate);
    std::free(r->triple_x);
    r->u = r->v = r->count = r->ncert = r->edge_count = nullptr;
    r->vertex = r->vertex_count = nullptr;
    r->certificate = nullptr;
    r->triple_x = r->triple_y = r->triple_w = nullptr;
    r->n_pairs = 0;
    r->n_triples = 0;
    r->tag = FREED_TAG;
}

// Pinned staging blocks (HOST_STAGE int64 read-back slots, then room for PAIR_STAGE
// solution pairs), recycled across graphs: a cudaMallocHost
// and its cudaFreeHost (which synchronises the device) cost more than a medium
// graph's whole query. A block goes back to the list only when no copy into or out of
// it can still be pending; otherwise it is freed.
static std::mutex g_stage_mu;
static std::vector<int64_t*> g_stage_free;
constexpr size_t STAGE_KEEP = 64;

static int64_t* stage_take() {
    {
        std::lock_guard<std::mutex> lock(g_stage_mu);
        if (!g_stage_free.empty()) {
            int64_t* p = g_stage_free.back();
            g_stage_free.pop_back();
            return p;
        }
    }
    int64_t* p = nullptr;
    FOLTY_CUDA(cudaMallocHost((void**)&p, HOST_STAGE * sizeof(int64_t) + 4 * PAIR_STAGE * sizeof(int32_t)));
    return p;
}

static void stage_give(int64_t* p, bool busy) {
    if (!busy) {
        std::lock_guard<std::mutex> lock(g_stage_mu);
        if (g_stage_free.size() < STAGE_KEEP) {
            g_stage_free.push_back(p);
            return;
        }
    }
    cudaFreeHost(p);
}

static void free_graph(folty_graph* g) {
    destroy_plans(g);
    for (auto& e : g->live_ev)
        if (e) cudaEventDestroy(e);
    if (g->perm_ev) cudaEventDestroy(g->perm_ev);
    if (g->owned) {
        for (auto& o : *g->owned) g->alloc.put(o.first, 0);
        delete g->owned;
        g->owned = nullptr;
    }
    if (g->host_stage) stage_give(g->host_stage, g->stage_busy != 0);
    g->tag = FREED_TAG;
    delete g;
}

// ------------------------------------------------------------------ load

// Checks ids and timestamps, finds the t range, counts self-loops and detects
// time-sorted input. stat: [0] first bad index + 1 (min), [1] tmin, [2] tmax,
// [3] unsorted flag, [4] self-loops.
struct EdgeStat {
    unsigned long long bad = ~0ull, tmin = ~0ull, tmax = 0, unsorted = 0, loops = 0;

    __device__ __forceinline__ void edge(int64_t i, int32_t x, int32_t y, int64_t ti, int64_t tprev, int32_t n) {
        bool ok = x >= 0 && x < n && y >= 0 && y < n && ti >= 0 && ti < (1ll << 62);
        if (!ok && (unsigned long long)i < bad) bad = (unsigned long long)i;
        if (ok) {
            tmin = min(tmin, (unsigned long long)ti);
            tmax = max(tmax, (unsigned long long)ti);
        }
        if (tprev > ti) unsorted = 1;
        loops += (x == y);
    }

    __device__ __forceinline__ void flush(unsigned long long* __restrict__ stat) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bad = min(bad, __shfl_xor_sync(0xffffffffu, bad, o));
            tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
            tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
            unsorted |= __shfl_xor_sync(0xffffffffu, unsorted, o);
            loops += __shfl_xor_sync(0xffffffffu, loops, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (bad != ~0ull) atomicMin(&stat[0], bad);
            atomicMin(&stat[1], tmin);
            atomicMax(&stat[2], tmax);
            if (unsorted) atomicOr(&stat[3], 1ull);
            if (loops) atomicAdd(&stat[4], loops);
        }
    }
};

__global__ void k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           const int64_t* __restrict__ t, int64_t m, int32_t n,
                           unsigned long long* __restrict__ stat) {
    EdgeStat st;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        st.edge(i, src[i], dst[i], t[i], i > 0 ? t[i - 1] : 0, n);
    st.flush(stat);
}

// The pair table's first try, filled while the load reads the edges (INSERT): the
// slot word of every edge (PAIR_LOOP for a self-loop or an invalid edge, which fails the
// load anyway).
struct LoadPairs {
    uint64_t* table;
    int lg;
    uint32_t* slotw;
    int* over;
};

template <bool INSERT>
__device__ __forceinline__ uint32_t load_slot_word(const LoadPairs& lp, int32_t x, int32_t y, int32_t n) {
    if (!INSERT || x < 0 || x >= n || y < 0 || y >= n) return PAIR_LOOP;
    return pair_slot_word(lp.table, lp.lg, x, y, n, lp.over);
}

// The same checks fused with the copy of the input into the graph's own arrays: one
// read and one write of every input byte. The input is device memory or pinned host
// memory (read over the host link, as fast as a copy engine's pull); with INSERT the
// edges' pairs also go into the pair table (work that the host link's pace leaves room
// for). Four edges per thread and iteration (16-byte accesses; all pointers 16-byte
// aligned), the previous edge's timestamp from the neighbouring lane, the m mod 4 last
// edges one by one.
template <bool INSERT>
__global__ void k_load_copy(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            const int64_t* __restrict__ t, int64_t m, int32_t n, int32_t* __restrict__ osrc,
                            int32_t* __restrict__ odst, int64_t* __restrict__ ot,
                            unsigned long long* __restrict__ stat, LoadPairs lp) {
    EdgeStat st;
    const int lane = threadIdx.x & 31;
    const int64_t m4 = m >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t j0 = tid - lane; j0 < m4; j0 += stride) {  // warp-uniform trip count
        const int64_t j = j0 + lane;
        const bool act = j < m4;
        int4 x{}, y{};
        longlong2 t01{}, t23{};
        if (act) {
            x = __ldcs(reinterpret_cast<const int4*>(src) + j);
            y = __ldcs(reinterpret_cast<const int4*>(dst) + j);
            t01 = __ldcs(reinterpret_cast<const longlong2*>(t) + 2 * j);
            t23 = __ldcs(reinterpret_cast<const longlong2*>(t) + 2 * j + 1);
        }
        int64_t tp = __shfl_up_sync(0xffffffffu, (long long)t23.y, 1);
        if (lane == 0) tp = j > 0 ? t[4 * j - 1] : 0;
        if (act) {
            reinterpret_cast<int4*>(osrc)[j] = x;
            reinterpret_cast<int4*>(odst)[j] = y;
            reinterpret_cast<longlong2*>(ot)[2 * j] = t01;
            reinterpret_cast<longlong2*>(ot)[2 * j + 1] = t23;
            const int64_t i = 4 * j;
            st.edge(i, x.x, y.x, t01.x, tp, n);
            st.edge(i + 1, x.y, y.y, t01.y, t01.x, n);
            st.edge(i + 2, x.z, y.z, t23.x, t01.y, n);
            st.edge(i + 3, x.w, y.w, t23.y, t23.x, n);
            if (INSERT) {
                // the four edges' first probes issued together (most find their pair, or
                // an empty slot, there); the rest of a probe sequence one edge at a time
                const int32_t xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
                uint32_t ws[4];
                uint64_t key[4], h[4], cur[4];
                bool ok[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    ok[e] = xs[e] >= 0 && xs[e] < n && ys[e] >= 0 && ys[e] < n && xs[e] != ys[e];
                    key[e] = ok[e] ? pair_rank_of(xs[e], ys[e], n) + 1 : 0;
                    h[e] = (key[e] * PAIR_HASH_MUL) >> (64 - lp.lg);
                    cur[e] = ok[e] ? __ldcg(&lp.table[h[e]]) : 0;
                }
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    if (!ok[e]) ws[e] = PAIR_LOOP;
                    else if (cur[e] == key[e]) ws[e] = (uint32_t)h[e] | (xs[e] > ys[e] ? PAIR_DIR : 0u);
                    else ws[e] = load_slot_word<INSERT>(lp, xs[e], ys[e], n);
                }
                reinterpret_cast<uint4*>(lp.slotw)[j] = make_uint4(ws[0], ws[1], ws[2], ws[3]);
            }
        }
    }
    for (int64_t i = 4 * m4 + tid; i < m; i += stride) {
        const int32_t x = src[i], y = dst[i];
        const int64_t ti = t[i];
        osrc[i] = x;
        odst[i] = y;
        ot[i] = ti;
        st.edge(i, x, y, ti, i > 0 ? t[i - 1] : 0, n);
        if (INSERT) lp.slotw[i] = load_slot_word<INSERT>(lp, x, y, n);
    }
    st.flush(stat);
}

// The address under which kernels of the current device read p: p itself for memory
// of this device, the mapped address for pinned host memory; NULL otherwise (pageable
// host memory, another device's memory).
static const void* kernel_address(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice && a.device == dev) return p;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

static void load_graph(folty_graph* g, const int32_t* src, const int32_t* dst, const int64_t* t,
                       cudaStream_t s) {
    const int64_t m = g->m;
    g->in_src = graph_alloc<int32_t>(g, m, s);
    g->in_dst = graph_alloc<int32_t>(g, m, s);
    g->in_t = graph_alloc<int64_t>(g, m, s);
    g->dev_err = graph_alloc<int>(g, 1, s);
    FOLTY_CUDA(cudaMemsetAsync(g->dev_err, 0, sizeof(int), s));
    auto a16 = [](const void* p) { return p && ((uintptr_t)p & 15) == 0; };
    const void* ksrc = m > 0 ? kernel_address(src) : nullptr;
    const void* kdst = m > 0 ? kernel_address(dst) : nullptr;
    const void* kt = m > 0 ? kernel_address(t) : nullptr;
    const bool fused = a16(ksrc) && a16(kdst) && a16(kt) && a16(g->in_src) && a16(g->in_dst) && a16(g->in_t);
    if (m > 0 && !fused) {
        FOLTY_CUDA(cudaMemcpyAsync(g->in_src, src, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault, s));
        FOLTY_CUDA(cudaMemcpyAsync(g->in_dst, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault, s));
        FOLTY_CUDA(cudaMemcpyAsync(g->in_t, t, sizeof(int64_t) * (size_t)m, cudaMemcpyDefault, s));
    }
    Scratch sc(g->alloc, s, g->dev_err);
    unsigned long long* stat = sc.get<unsigned long long>(5);
    unsigned long long init[5] = {~0ull, ~0ull, 0ull, 0ull, 0ull};
    std::memcpy(g->host_stage + READBACK_MAX, init, sizeof(init));
    g->stage_busy = 1;
    FOLTY_CUDA(cudaMemcpyAsync(stat, g->host_stage + READBACK_MAX, sizeof(init), cudaMemcpyHostToDevice, s));
    // the pair table's first try rides along with a fused load (the preprocessing uses
    // it when its first try has the same size)
    bool insert = fused && g->n >= 2 && !pair_table_forced_off();
    LoadPairs lp{nullptr, 0, nullptr, nullptr};
    if (insert) {
        lp.lg = pair_table_lg_first(m);
        g->pre_lg = lp.lg;
        g->pre_table = graph_alloc<uint64_t>(g, 1ll << lp.lg, s);
        g->pre_slotw = graph_alloc<uint32_t>(g, m, s);
        g->pre_flags = graph_alloc<int>(g, 2, s);
        if (!a16(g->pre_slotw)) {  // a caller's allocator may not align it for 16-byte stores
            graph_release(g, g->pre_table, s);
            graph_release(g, g->pre_slotw, s);
            graph_release(g, g->pre_flags, s);
            g->pre_table = nullptr;
            g->pre_slotw = nullptr;
            g->pre_flags = nullptr;
            insert = false;
        } else {
            FOLTY_CUDA(cudaMemsetAsync(g->pre_table, 0, sizeof(uint64_t) * ((size_t)1 << lp.lg), s));
            FOLTY_CUDA(cudaMemsetAsync(g->pre_flags, 0, 2 * sizeof(int), s));
            lp = LoadPairs{g->pre_table, lp.lg, g->pre_slotw, g->pre_flags};
        }
    }
    if (fused && insert)
        FOLTY_LAUNCH(k_load_copy<true>, grid_for(m / 4 + 1, 256, 8), 256, 0, s, (const int32_t*)ksrc,
                     (const int32_t*)kdst, (const int64_t*)kt, m, g->n, g->in_src, g->in_dst, g->in_t, stat, lp);
    else if (fused)
        FOLTY_LAUNCH(k_load_copy<false>, grid_for(m / 4 + 1, 256, 4), 256, 0, s, (const int32_t*)ksrc,
                     (const int32_t*)kdst, (const int64_t*)kt, m, g->n, g->in_src, g->in_dst, g->in_t, stat, lp);
    else if (m > 0)
        FOLTY_LAUNCH(k_validate, grid_for(m, 256), 256, 0, s, g->in_src, g->in_dst, g->in_t, m, g->n, stat);
    const void* ptrs[5] = {stat, stat + 1, stat + 2, stat + 3, stat + 4};
    int sizes[5] = {8, 8, 8, 8, 8};
    int64_t v[5];
    read_back(g, ptrs, sizes, 5, v, s);
    if ((unsigned long long)v[0] != ~0ull)
        fail(FOLTY_EINVAL, "edge " + std::to_string(v[0]) + ": vertex id outside [0, n) or timestamp outside [0, 2^62)");
    g->tmin = (m > 0) ? v[1] : 0;
    g->tmax = (m > 0) ? v[2] : 0;
    g->info.time_sorted = v[3] ? 0 : 1;
    g->m_kept = m - v[4];
    g->info.n = g->n;
    g->info.m = m;
    g->info.m_kept = g->m_kept;
}

template <typename F>
static folty_status guarded(F&& f) {
    try {
        f();
        t_last_error.clear();
        return FOLTY_OK;
    } catch (const Error& e) {
        t_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        t_last_error = "host allocation failed";
        return FOLTY_ENOMEM;
    } catch (...) {
        t_last_error = "unexpected internal error";
        return FOLTY_ECUDA;
    }
}

static folty_graph* checked_graph(const folty_graph* g) {
    if (!g || g->tag != GRAPH_TAG) fail(FOLTY_EINVAL, "not a folty graph");
    return const_cast<folty_graph*>(g);
}

}  // namespace folty

using namespace folty;

extern "C" {

folty_status folty_load_temporal_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                       const int64_t* t, const folty_allocator* alloc, void* stream,
                                       folty_graph** out) {
    folty_graph* g = nullptr;
    folty_status st = guarded([&] {
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        *out = nullptr;
        if (n < 0 || n >= (1 << 30)) fail(FOLTY_EINVAL, "n outside [0, 2^30)");
        if (m < 0 || m >= 0x7fffffffll) fail(FOLTY_EINVAL, "m outside [0, 2^31 - 1)");
        if (m > 0 && (!src || !dst || !t)) fail(FOLTY_EINVAL, "edge arrays are NULL");
        if (alloc && (!alloc->alloc || !alloc->free)) fail(FOLTY_EINVAL, "allocator without alloc/free");
        cudaStream_t s = (cudaStream_t)stream;
        g = new folty_graph();
        std::memset((void*)g, 0, sizeof(*g));
        g->tag = GRAPH_TAG;
        g->owned = new std::vector<std::pair<void*, size_t>>();
        if (alloc) {
            g->alloc.a = *alloc;
            g->alloc.user = true;
        }
        FOLTY_CUDA(cudaGetDevice(&g->device));
        g->host_stage = stage_take();
        void* dp = nullptr;
        FOLTY_CUDA(cudaHostGetDevicePointer(&dp, g->host_stage, 0));
        g->stage_dev = (int64_t*)dp;
        g->pair_stage = (int32_t*)(g->stage_dev + HOST_STAGE);
        g->n = n;
        g->m = m;
        load_graph(g, src, dst, t, s);
        *out = g;
    });
    if (st != FOLTY_OK && g) free_graph(g);
    return st;
}

folty_status folty_preprocess(folty_graph* g, void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (g->state != 0) fail(FOLTY_ESTATE, "graph already preprocessed");
        ProfileScope prof;
        preprocess_graph(g, (cudaStream_t)stream);  // ends with a stream synchronisation
        prof.commit();
    });
}

folty_status folty_query(folty_graph* g, const folty_query_params* q, folty_result* out, void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (!q || !out) fail(FOLTY_EINVAL, "query or result is NULL");
        if (g->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        validate_query(*q);
        ProfileScope prof;
        run_query(g, *q, out, (cudaStream_t)stream);  // ends with a stream synchronisation
        prof.commit();
    });
}

folty_status folty_query_batch(folty_graph* g, const folty_query_params* qs, int32_t nq, folty_result* outs,
                               void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (nq < 0 || (nq > 0 && (!qs || !outs))) fail(FOLTY_EINVAL, "bad query array");
        if (g->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        for (int i = 0; i < nq; i++) validate_query(qs[i]);
        for (int i = 0; i < nq; i++) std::memset(&outs[i], 0, sizeof(folty_result));
        try {
            ProfileScope prof;
            run_query_batch(g, qs, nq, outs, (cudaStream_t)stream);  // ends synchronised
            prof.commit();
        } catch (...) {
            for (int i = 0; i < nq; i++)
                if (outs[i].tag == RESULT_TAG) release_result(&outs[i]);
            throw;
        }
    });
}

void folty_free(void* obj) {
    if (!obj) return;
    uint64_t tag;
    std::memcpy(&tag, obj, sizeof(tag));
    if (tag == GRAPH_TAG) free_graph((folty_graph*)obj);
    else if (tag == RESULT_TAG) release_result((folty_result*)obj);
}

const char* folty_last_error(void) { return t_last_error.c_str(); }

folty_status folty_graph_get_info(const folty_graph* g, folty_graph_info* info) {
    return guarded([&] {
        folty_graph* gg = checked_graph(g);
        if (!info) fail(FOLTY_EINVAL, "info is NULL");
        if (gg->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        *info = gg->info;
    });
}

folty_status folty_graph_traffic_model(folty_graph* g, int32_t dir, folty_traffic_model* out, void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        if (dir < 0 || dir > 2) fail(FOLTY_EINVAL, "unknown direction variant");
        if (g->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        traffic_model(g, dir, out, (cudaStream_t)stream);
    });
}

folty_status folty_graph_tuning(const folty_graph* g, folty_tuning* out) {
    return guarded([&] {
        folty_graph* gg = checked_graph(g);
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        if (gg->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        const TuneParams& t = gg->tune;
        out->tri_heavy = t.tri_heavy;
        out->probe_items = t.probe_items;
        out->probe_blocks_per_sm = t.probe_blocks;
        out->tri_source = t.tri_source;
        out->probe_source = t.probe_source;
        for (int i = 0; i < 4; i++) {
            out->tri_ms[i] = t.tri_ms[i];
            out->probe_ms[i] = t.probe_ms[i];
        }
    });
}

folty_status folty_graph_probe_stats(folty_graph* g, int64_t delta, int32_t dir, folty_probe_stats* out,
                                     void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        if (delta < 0 || delta >= (1ll << 62)) fail(FOLTY_EINVAL, "delta outside [0, 2^62)");
        if (dir < 0 || dir > FOLTY_DIR_EITHER) fail(FOLTY_EINVAL, "unknown direction variant");
        if (g->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        probe_stats(g, delta, dir, out, (cudaStream_t)stream);
    });
}

folty_status folty_graph_common_counts(folty_graph* g, int32_t* a, int32_t* b, int32_t* c, void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (g->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        if (g->S > 0 && (!a || !b || !c)) fail(FOLTY_EINVAL, "output arrays are NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t bytes = sizeof(int32_t) * (size_t)g->S;
        if (g->S > 0) {
            FOLTY_CUDA(cudaMemcpyAsync(a, g->ea, bytes, cudaMemcpyDeviceToHost, s));
            FOLTY_CUDA(cudaMemcpyAsync(b, g->eb, bytes, cudaMemcpyDeviceToHost, s));
            FOLTY_CUDA(cudaMemcpyAsync(c, g->common, bytes, cudaMemcpyDeviceToHost, s));
        }
        FOLTY_CUDA(cudaStreamSynchronize(s));
    });
}

folty_status folty_graph_core_numbers(folty_graph* g, int32_t* core, void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (g->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        if (g->n > 0 && !core) fail(FOLTY_EINVAL, "core is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        if (g->n > 0)
            FOLTY_CUDA(cudaMemcpyAsync(core, g->core, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
        FOLTY_CUDA(cudaStreamSynchronize(s));
    });
}

uint64_t folty_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

folty_status folty_edge_counts_noalloc(folty_graph* g, int64_t delta, int32_t dir, int32_t* edge_count,
                                       void* stream) {
    return guarded([&] {
        checked_graph(g);
        if (!edge_count && g->m > 0) fail(FOLTY_EINVAL, "edge_count is NULL");
        if (delta < 0 || delta >= (1ll << 62)) fail(FOLTY_EINVAL, "delta outside [0, 2^62)");
        if (dir < 0 || dir > FOLTY_DIR_EITHER) fail(FOLTY_EINVAL, "unknown direction variant");
        if (g->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        // the kernels run on the current device and read the graph's arrays: that must be
        // the graph's device, and edge_count must be memory of it (the kernels write m
        // int32 through it; host memory or another device's memory is refused here)
        int dev = -1;
        FOLTY_CUDA(cudaGetDevice(&dev));
        if (dev != g->device)
            fail(FOLTY_EINVAL, "the current device (" + std::to_string(dev) + ") is not the graph's device (" +
                                   std::to_string(g->device) + ")");
        if (g->m > 0) {
            cudaPointerAttributes pa{};
            if (cudaPointerGetAttributes(&pa, edge_count) != cudaSuccess) {
                cudaGetLastError();
                fail(FOLTY_EINVAL, "edge_count is not device memory");
            }
            if (pa.type != cudaMemoryTypeDevice || pa.device != dev)
                fail(FOLTY_EINVAL, "edge_count must be device memory of the graph's device");
        }
        edge_counts_noalloc(g, delta, dir, edge_count, (cudaStream_t)stream);
    });
}

void folty_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lock(g_profile_mu);
    for (auto& st : g_stages) st = folty_stage_profile{0, 0.0, 0};
    g_profile_on.store(on ? 1 : 0);
}

folty_status folty_profile_read(int32_t stage, folty_stage_profile* out) {
    return guarded([&] {
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        if (stage < 0 || stage >= ST_COUNT) fail(FOLTY_EINVAL, "unknown stage");
        std::lock_guard<std::mutex> lock(g_profile_mu);
        *out = g_stages[stage];
    });
}

}  // extern "C"
