// Per-edge counts of one query without any device allocation.
//
// Some callers cannot allocate device memory at query time: a serving process that
// reserved its whole memory budget at start-up, latency-bound code that must not hit
// the implicit device synchronisation of cudaMalloc/cudaFree, or a host whose
// allocator must not be re-entered from inside a library call. For them the
// window-probe pass of folty_query has this variant: the per-edge counters it works in
// (sorted edge order) live in a file-scope device array instead of memory from an
// allocator, and the counts go to a device buffer the caller provides. The paper has
// no counterpart.
#include <mutex>

#include "internal.cuh"
#include "probe.cuh"

namespace folty {

// Counts from sorted order back to input order.
__global__ void k_noalloc_scatter(const int32_t* __restrict__ cnt, const int32_t* __restrict__ perm, int64_t mk,
                                  int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mk;
         i += (int64_t)gridDim.x * blockDim.x)
        out[perm[i]] = cnt[i];
}

// Counters of the last call, shared by every call in the process (one copy per device
// that loads the library, held until the process exits).
static __device__ __align__(256) int32_t g_noalloc_counts[FOLTY_NOALLOC_MAX_EDGES];

// Device address of g_noalloc_counts, looked up once per device with that device
// current. In host code the array's name is only a host-side stand-in.
static int32_t* noalloc_counts_on_current_device() {
    static std::mutex mu;
    static std::vector<int32_t*> addr;
    int dev = 0;
    FOLTY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if ((int)addr.size() <= dev) addr.resize((size_t)dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_counts);
        if (e != cudaSuccess) fail(FOLTY_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        addr[dev] = static_cast<int32_t*>(p);
    }
    return addr[dev];
}

void edge_counts_noalloc(folty_graph* g, int64_t delta, int dir, int32_t* edge_count, cudaStream_t s) {
    const int64_t mk = g->m_kept;
    if (mk > FOLTY_NOALLOC_MAX_EDGES)
        fail(FOLTY_EINVAL, "graph has " + std::to_string(mk) + " non-loop edges; the allocation-free path holds at most " +
                               std::to_string((long long)FOLTY_NOALLOC_MAX_EDGES));
    if (mk > 0 && !g->perm) fail(FOLTY_EINVAL, "graph has no input order of its store");  // made by preprocessing
    int32_t* cnt = noalloc_counts_on_current_device();
    if (g->m > 0) FOLTY_CUDA(cudaMemsetAsync(edge_count, 0, sizeof(int32_t) * (size_t)g->m, s));
    if (mk == 0) return;
    FOLTY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)mk, s));  // previous call's counts
    launch_probe(g, delta, dir, cnt, s);
    FOLTY_LAUNCH(k_noalloc_scatter, grid_for(mk, 256), 256, 0, s, cnt, g->perm, mk, edge_count);
}

}  // namespace folty
