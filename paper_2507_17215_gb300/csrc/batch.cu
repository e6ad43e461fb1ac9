// Batched queries sharing the window probes.
//
// For a fixed (temporal edge e, witness w, direction variant) the searched t2 and t3
// of Theorem 3.1 do not depend on delta, so hit(delta) <=> g(e, w) = t3 - t <= delta.
// One probe pass per direction variant therefore serves every delta of that variant
// (live.cu, binning mode, roles kept for the largest delta of the pass): the pass bins
// g by the sorted distinct deltas D (bin j = first D_j >= g), a prefix
// over the bins gives c_e(D_j) = #{w : g(e, w) <= D_j} for all j at once, and each
// query's threshold pass (the single-query code) reads its column. Quantifier, rho and
// universe only enter that last pass. When the bins of all deltas do not fit in the
// memory budget, the deltas are cut into chunks, one probe pass per chunk (bin 0 of a
// chunk also holds every smaller gap).
#include <algorithm>
#include <cstring>
#include <map>

#include "internal.cuh"
#include "probe.cuh"

namespace folty {

constexpr int BATCH_MAX_BINS = 1024;
static_assert(BATCH_MAX_BINS * sizeof(int64_t) <= 4 * PAIR_STAGE * sizeof(int32_t), "bin bounds fit the pair stage");

// bins[j][e] <- sum_{i <= j} bins[i][e]
template <typename C>
__global__ void k_bins_prefix(C* __restrict__ bins, int k, int64_t mk) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mk;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t run = 0;
        for (int j = 0; j < k; j++) {
            int64_t o = (int64_t)j * mk + e;
            run += bins[o];
            bins[o] = (C)run;
        }
    }
}

static int64_t batch_bin_budget_bytes() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return (int64_t)1 << 30;
    }
    int64_t b = (int64_t)(free_b / 4);
    const int64_t cap = (int64_t)16 << 30;
    return b < cap ? b : cap;
}

// Bins of one probe pass: the largest number of distinct deltas of one direction variant.
int64_t batch_footprint(const folty_graph* g, const folty_query_params* qs, int nq, int64_t* bins_part) {
    int64_t kmax = 0;
    for (int dir = 0; dir <= FOLTY_DIR_EITHER; dir++) {
        std::vector<int64_t> D;
        for (int i = 0; i < nq; i++)
            if (qs[i].dir == dir) D.push_back(qs[i].delta);
        std::sort(D.begin(), D.end());
        D.erase(std::unique(D.begin(), D.end()), D.end());
        kmax = std::max<int64_t>(kmax, (int64_t)D.size());
    }
    kmax = std::min<int64_t>(kmax, BATCH_MAX_BINS);
    const int64_t bins = kmax * g->m_kept * 4;
    // output stage per query of a read-back group (see finish_queries): 6 int32 arrays
    // of 2S + 1, compacted keys, packed output, edge counts when asked
    const int64_t n2 = 2 * (int64_t)g->S;
    int64_t per_q = 6 * 4 * (n2 + 1) + 8 * n2 + 16 * n2 + 64;
    bool edges = false, certs = false, outer = false;
    for (int i = 0; i < nq; i++) {
        edges = edges || qs[i].want_edge_counts;
        certs = certs || qs[i].want_certificates;
        outer = outer || qs[i].outer;
    }
    if (edges) per_q += 4 * g->m;
    if (certs) per_q += 16 * (g->m + 1);
    if (outer) per_q += 14 * ((int64_t)g->n + 1);
    const int64_t group = std::min<int64_t>(nq, READBACK_MAX / 4);
    // a triple query runs alone: role flags and scan (9 B per role), and up to one triple
    // per role through the two sorts (44 B each), on top of its own counters
    bool triples = false;
    for (int i = 0; i < nq; i++) triples = triples || qs[i].want_triples;
    const int64_t tri_part = triples ? 53 * 6 * g->ntri + 4 * g->m_kept + per_q : 0;
    if (bins_part) *bins_part = bins;
    return std::max(bins + group * per_q, tri_part);
}

void run_query_batch(folty_graph* g, const folty_query_params* qs, int nq, folty_result* outs,
                     cudaStream_t s, int64_t bin_budget) {
    const int64_t mk = g->m_kept;
    const int64_t P = g->info.probes;
    // a query that also wants the all-existential triples needs its own probe pass (the
    // role flags are per window, not per bin)
    for (int i = 0; i < nq; i++)
        if (qs[i].want_triples) run_query(g, qs[i], &outs[i], s);
    // group the queries by direction variant; distinct sorted deltas per group
    for (int dir = 0; dir <= FOLTY_DIR_EITHER; dir++) {
        std::vector<int> members;
        for (int i = 0; i < nq; i++)
            if (qs[i].dir == dir && !qs[i].want_triples) members.push_back(i);
        if (members.empty()) continue;
        std::vector<int64_t> D;
        for (int i : members) D.push_back(qs[i].delta);
        std::sort(D.begin(), D.end());
        D.erase(std::unique(D.begin(), D.end()), D.end());
        // 16-bit bins while no count can reach 2^16 (a count is at most the number of
        // common neighbours of an edge's ends, at most the largest degree): half the
        // memory traffic of the bins, their prefix and the threshold's column reads
        const bool b16 = g->info.max_degree < 65535;
        const int64_t per_bin = mk * (int64_t)(b16 ? sizeof(uint16_t) : sizeof(int32_t));
        const int64_t budget = bin_budget > 0 ? bin_budget : batch_bin_budget_bytes();
        int64_t chunk = per_bin > 0 ? budget / per_bin : (int64_t)D.size();
        chunk = std::max<int64_t>(1, std::min<int64_t>({chunk, (int64_t)BATCH_MAX_BINS, (int64_t)D.size()}));
        for (size_t c0 = 0; c0 < D.size(); c0 += (size_t)chunk) {
            const int k = (int)std::min<int64_t>(chunk, (int64_t)D.size() - (int64_t)c0);
            Scratch sc(g->alloc, s, g->dev_err);
            int32_t* bins = b16 ? nullptr : sc.get<int32_t>(mk * k);
            uint16_t* bins16 = b16 ? sc.get<uint16_t>(mk * k + 2) : nullptr;  // + 2: the last word is whole
            int64_t* dd = sc.get<int64_t>(k);
            std::vector<int64_t> hd(D.begin() + (long)c0, D.begin() + (long)c0 + k);
            // the bin bounds in the store's timestamp type (32-bit offsets: gaps stay
            // below 2^32 - 1, so larger windows behave as 2^32 - 2)
            // staged in the graph's pinned pair stage, which nothing uses before this
            // chunk's threshold pass (the last chunk's read-back has completed)
            void* hb = g->host_stage + HOST_STAGE;
            if (g->ts32) {
                uint32_t* h32 = static_cast<uint32_t*>(hb);
                for (int i = 0; i < k; i++) h32[i] = hd[i] >= 0xfffffffell ? 0xfffffffeu : (uint32_t)hd[i];
            } else {
                std::memcpy(hb, hd.data(), sizeof(int64_t) * (size_t)k);
            }
            g->stage_busy = 1;
            FOLTY_CUDA(cudaMemcpyAsync(dd, hb, (g->ts32 ? sizeof(uint32_t) : sizeof(int64_t)) * (size_t)k,
                                       cudaMemcpyHostToDevice, s));
            if (mk > 0) {
                if (b16) FOLTY_CUDA(cudaMemsetAsync(bins16, 0, sizeof(uint16_t) * (size_t)(mk * k + 2), s));
                else FOLTY_CUDA(cudaMemsetAsync(bins, 0, sizeof(int32_t) * (size_t)(mk * k), s));
                if (P > 0) launch_probe_live(g, hd[k - 1], dir, 1, nullptr, bins, k, dd, s, nullptr, bins16);
                if (k > 1 && b16) FOLTY_LAUNCH(k_bins_prefix<uint16_t>, grid_for(mk, 256), 256, 0, s, bins16, k, mk);
                if (k > 1 && !b16) FOLTY_LAUNCH(k_bins_prefix<int32_t>, grid_for(mk, 256), 256, 0, s, bins, k, mk);
            }
            std::vector<const folty_query_params*> fq;
            std::vector<CountView> fc;
            std::vector<folty_result*> fo;
            for (int i : members) {
                auto it = std::lower_bound(hd.begin(), hd.end(), qs[i].delta);
                if (it == hd.end() || *it != qs[i].delta) continue;  // another chunk
                const int j = (int)(it - hd.begin());
                fq.push_back(&qs[i]);
                if (b16) fc.push_back(CountView{nullptr, bins16 + (int64_t)j * mk});
                else fc.push_back(CountView{bins + (int64_t)j * mk, nullptr});
                fo.push_back(&outs[i]);
            }
            finish_queries(g, fq.data(), fc.data(), (int)fq.size(), fo.data(), s);
        }
    }
}

}  // namespace folty
