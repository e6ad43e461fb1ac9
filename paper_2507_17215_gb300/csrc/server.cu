// Query server over resident preprocessed graphs: continuous batching per graph,
// admission by device memory, one worker thread and one CUDA stream per graph so that
// work on different graphs overlaps on the device.
//
// A worker waits for queued queries of its graph, takes everything queued (up to
// max_batch) as one batch, shrinks the batch until its device footprint fits the
// server's memory budget, waits until the budget has room (queries arriving meanwhile
// join the next batch), runs the batch (folty_query_batch semantics: one probe pass
// per direction variant) on its stream and completes the tickets.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "internal.cuh"

namespace folty {

constexpr uint64_t SERVER_TAG = 0x464f4c5459535256ull;  // "FOLTYSRV"

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
    int64_t id = 0;
    int32_t gi = 0;
    folty_query_params q{};
    folty_result res{};
    folty_status st = FOLTY_OK;
    std::string err;
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t batch_id = 0;
    int32_t batch_size = 0;
    bool done = false;
};

struct Worker {
    folty_graph* g = nullptr;
    cudaStream_t stream = nullptr;
    std::deque<std::shared_ptr<Ticket>> queue;
    std::thread th;
};

}  // namespace folty

struct folty_server {
    uint64_t tag;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_mem;
    std::vector<folty::Worker*> workers;
    std::unordered_map<int64_t, std::shared_ptr<folty::Ticket>> tickets;
    int64_t next_id = 1, next_batch = 1;
    bool stop = false;
    int64_t budget = 0, used = 0, peak_used = 0;
    int32_t max_batch = 256;
    int64_t batches = 0, queries = 0, max_in_flight = 0, in_flight = 0;
};

namespace folty {

static void worker_loop(folty_server* sv, Worker* w) {
    cudaSetDevice(w->g->device);
    while (true) {
        std::vector<std::shared_ptr<Ticket>> batch;
        int64_t est = 0, bins = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stop || !w->queue.empty(); });
            if (w->queue.empty()) return;  // stop requested and nothing left to do
            while (!w->queue.empty() && (int32_t)batch.size() < sv->max_batch) {
                batch.push_back(w->queue.front());
                w->queue.pop_front();
            }
            // admission: shrink the batch until it fits the budget on its own
            std::vector<folty_query_params> qs;
            for (auto& t : batch) qs.push_back(t->q);
            est = batch_footprint(w->g, qs.data(), (int)qs.size(), &bins);
            while (est > sv->budget && batch.size() > 1) {
                w->queue.push_front(batch.back());
                batch.pop_back();
                qs.pop_back();
                est = batch_footprint(w->g, qs.data(), (int)qs.size(), &bins);
            }
            // wait for room (a batch larger than the whole budget runs alone)
            sv->cv_mem.wait(lk, [&] { return sv->used + est <= sv->budget || sv->used == 0; });
            sv->used += est;
            sv->peak_used = std::max(sv->peak_used, sv->used);
            sv->in_flight += 1;
            sv->max_in_flight = std::max(sv->max_in_flight, sv->in_flight);
            const int64_t bid = sv->next_batch++;
            const double t0 = now_ms();
            for (auto& t : batch) {
                t->t_start = t0;
                t->batch_id = bid;
                t->batch_size = (int32_t)batch.size();
            }
        }
        std::vector<folty_query_params> qs;
        for (auto& t : batch) qs.push_back(t->q);
        std::vector<folty_result> outs(batch.size());
        folty_status st = FOLTY_OK;
        std::string err;
        try {
            // bins may use the batch's admitted share (at least one bin column)
            const int64_t bin_budget = std::max<int64_t>(bins, w->g->m_kept * 4);
            run_query_batch(w->g, qs.data(), (int)qs.size(), outs.data(), w->stream, bin_budget);
        } catch (const Error& e) {
            st = e.status;
            err = e.msg;
        } catch (...) {
            st = FOLTY_ECUDA;
            err = "unexpected internal error";
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->used -= est;
            sv->in_flight -= 1;
            sv->batches += 1;
            sv->queries += (int64_t)batch.size();
            const double t1 = now_ms();
            for (size_t i = 0; i < batch.size(); i++) {
                auto& t = batch[i];
                if (st == FOLTY_OK) t->res = outs[i];
                else if (outs[i].tag == RESULT_TAG) folty_free(&outs[i]);
                t->st = st;
                t->err = err;
                t->t_done = t1;
                t->done = true;
            }
        }
        sv->cv_mem.notify_all();
        sv->cv_done.notify_all();
    }
}

template <typename F>
static folty_status guarded_server(F&& f) {
    try {
        f();
        set_last_error("");
        return FOLTY_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    } catch (...) {
        set_last_error("unexpected internal error");
        return FOLTY_ECUDA;
    }
}

static folty_server* checked_server(folty_server* sv) {
    if (!sv || sv->tag != SERVER_TAG) fail(FOLTY_EINVAL, "not a folty server");
    return sv;
}

static void shutdown_server(folty_server* sv) {
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (Worker* w : sv->workers)
        if (w->th.joinable()) w->th.join();
    for (Worker* w : sv->workers) {
        if (w->stream) cudaStreamDestroy(w->stream);
        delete w;
    }
    sv->workers.clear();
    for (auto& kv : sv->tickets)
        if (kv.second->res.tag == RESULT_TAG) folty_free(&kv.second->res);
    sv->tickets.clear();
}

}  // namespace folty

using namespace folty;

extern "C" {

folty_status folty_server_create(folty_graph* const* graphs, int32_t n_graphs, const folty_server_config* cfg,
                                 folty_server** out) {
    folty_server* sv = nullptr;
    folty_status st = guarded_server([&] {
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        *out = nullptr;
        if (n_graphs <= 0 || !graphs) fail(FOLTY_EINVAL, "no graphs");
        for (int i = 0; i < n_graphs; i++) {
            if (!graphs[i] || graphs[i]->tag != GRAPH_TAG) fail(FOLTY_EINVAL, "not a folty graph");
            if (graphs[i]->state != 1) fail(FOLTY_ESTATE, "graph not preprocessed");
        }
        sv = new folty_server();
        sv->tag = SERVER_TAG;
        sv->max_batch = (cfg && cfg->max_batch > 0) ? cfg->max_batch : 256;
        if (cfg && cfg->memory_budget_bytes > 0) {
            sv->budget = cfg->memory_budget_bytes;
        } else {
            size_t free_b = 0, total_b = 0;
            FOLTY_CUDA(cudaMemGetInfo(&free_b, &total_b));
            sv->budget = (int64_t)(free_b / 2);
        }
        for (int i = 0; i < n_graphs; i++) {
            Worker* w = new Worker();
            w->g = graphs[i];
            sv->workers.push_back(w);
            int cur = 0;
            FOLTY_CUDA(cudaGetDevice(&cur));
            FOLTY_CUDA(cudaSetDevice(w->g->device));
            FOLTY_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
            FOLTY_CUDA(cudaSetDevice(cur));
        }
        for (Worker* w : sv->workers) w->th = std::thread(worker_loop, sv, w);
        *out = sv;
    });
    if (st != FOLTY_OK && sv) {
        shutdown_server(sv);
        delete sv;
    }
    return st;
}

folty_status folty_server_submit(folty_server* sv, int32_t graph_index, const folty_query_params* q,
                                 int64_t* ticket) {
    return guarded_server([&] {
        checked_server(sv);
        if (!q || !ticket) fail(FOLTY_EINVAL, "query or ticket is NULL");
        if (graph_index < 0 || graph_index >= (int32_t)sv->workers.size()) fail(FOLTY_EINVAL, "graph index out of range");
        validate_query(*q);
        auto t = std::make_shared<Ticket>();
        t->gi = graph_index;
        t->q = *q;
        t->t_submit = now_ms();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (sv->stop) fail(FOLTY_ESTATE, "server is shutting down");
            t->id = sv->next_id++;
            sv->tickets[t->id] = t;
            sv->workers[graph_index]->queue.push_back(t);
        }
        sv->cv_work.notify_all();
        *ticket = t->id;
    });
}

folty_status folty_server_wait(folty_server* sv, int64_t ticket, int64_t timeout_ms, folty_result* out,
                               folty_ticket_info* info) {
    folty_status result_status = FOLTY_OK;
    std::string result_err;
    folty_status st = guarded_server([&] {
        checked_server(sv);
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        std::memset(out, 0, sizeof(*out));
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->tickets.find(ticket);
        if (it == sv->tickets.end()) fail(FOLTY_EINVAL, "unknown ticket");
        std::shared_ptr<Ticket> t = it->second;
        auto ready = [&] { return t->done; };
        if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
        else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            fail(FOLTY_ETIMEOUT, "ticket not completed within the timeout");
        sv->tickets.erase(ticket);
        if (info) {
            info->queued_ms = t->t_start - t->t_submit;
            info->run_ms = t->t_done - t->t_start;
            info->latency_ms = t->t_done - t->t_submit;
            info->batch_id = t->batch_id;
            info->batch_size = t->batch_size;
            info->graph_index = t->gi;
        }
        result_status = t->st;
        result_err = t->err;
        if (t->st == FOLTY_OK) {
            *out = t->res;
            t->res.tag = 0;  // ownership moved to the caller
        }
    });
    if (st != FOLTY_OK) return st;
    if (result_status != FOLTY_OK) set_last_error(result_err);
    return result_status;
}

folty_status folty_server_get_stats(folty_server* sv, folty_server_stats* out) {
    return guarded_server([&] {
        checked_server(sv);
        if (!out) fail(FOLTY_EINVAL, "out is NULL");
        std::lock_guard<std::mutex> lk(sv->mu);
        out->batches = sv->batches;
        out->queries = sv->queries;
        out->memory_budget_bytes = sv->budget;
        out->peak_memory_bytes = sv->peak_used;
        out->max_batches_in_flight = sv->max_in_flight;
        int64_t pending = 0;
        for (auto* w : sv->workers) pending += (int64_t)w->queue.size();
        out->queued = pending;
    });
}

void folty_server_destroy(folty_server* sv) {
    if (!sv || sv->tag != SERVER_TAG) return;
    shutdown_server(sv);
    sv->tag = FREED_TAG;
    delete sv;
}

}  // extern "C"
