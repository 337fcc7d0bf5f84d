// Query server: a host thread that admits submitted queries into the slots of the next
// batched edge-map launch while device memory allows, runs them, and hands results back
// through tickets.  Submit and poll are thread-safe and never block on the device.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

kairos_status kairos_run_queries(kairos_graph *g, const kairos_query *qs, int32_t nq, uint32_t *out,
                                 kairos_query_stats *stats, int lanes);
kairos_status kairos_row_checksums(kairos_graph *g, const uint32_t *x, int rows, uint64_t *cs, uint32_t *reached);

using clk = std::chrono::steady_clock;

namespace {
struct Ticket {
    kairos_query q;
    uint32_t *out;
    clk::time_point submitted;
    bool done = false;
    kairos_result_info info{};
};
}  // namespace

struct kairos_server {
    kairos_graph *g = nullptr;
    int slots = 64;
    int capacity = 4096;
    int64_t reserve = 1LL << 30;
    uint32_t *rows = nullptr;  // [slots][n] device staging of results
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
};

namespace {

// Slots admitted for the next batch: bounded by the configured maximum and by what the
// device can hold beyond the reserve (labels, scan bounds and staging: 12 bytes per vertex
// per slot).
int admissible_slots(kairos_server *S) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const int64_t per_slot = S->g->n * 12;
    int64_t spare = (int64_t)free_b - S->reserve;
    int64_t fit = spare > 0 ? spare / std::max<int64_t>(per_slot, 1) : 0;
    return (int)std::max<int64_t>(1, std::min<int64_t>(S->slots, fit + S->g->work.lanes));
}

void worker(kairos_server *S) {
    kairos_graph *g = S->g;
    std::vector<uint64_t> batch;
    std::vector<kairos_query> qs;
    std::vector<kairos_query_stats> st;
    std::vector<uint64_t> cs;
    std::vector<uint32_t> reached;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
            if (S->pending.empty() && S->stop) return;
            const int take = admissible_slots(S);
            batch.clear();
            qs.clear();
            while (!S->pending.empty() && (int)batch.size() < take) {
                uint64_t id = S->pending.front();
                S->pending.pop_front();
                batch.push_back(id);
                qs.push_back(S->tickets[id].q);
            }
        }
        const int k = (int)batch.size();
        st.assign(k, kairos_query_stats{});
        cs.assign(k, 0);
        reached.assign(k, 0);
        kairos_status status;
        {
            std::lock_guard<std::mutex> glk(g->mu);
            status = kairos_run_queries(g, qs.data(), k, S->rows, st.data(), g->tuning.lanes);
            if (status == KAIROS_OK) status = kairos_row_checksums(g, S->rows, k, cs.data(), reached.data());
        }
        // deliver each row to its ticket's buffer (host or device)
        std::vector<kairos_status> per(k, status);
        if (status == KAIROS_OK) {
            for (int i = 0; i < k; ++i) {
                uint32_t *dst;
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    dst = S->tickets[batch[i]].out;
                }
                cudaError_t e = cudaMemcpyAsync(dst, S->rows + (int64_t)i * g->n, (size_t)g->n * 4, cudaMemcpyDefault,
                                                g->stream);
                if (e != cudaSuccess) per[i] = kairos::cuda_fail(e, "serve: deliver result");
            }
            cudaError_t e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess)
                for (int i = 0; i < k; ++i) per[i] = kairos::cuda_fail(e, "serve: deliver result");
        }
        const auto now = clk::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (int i = 0; i < k; ++i) {
                Ticket &T = S->tickets[batch[i]];
                T.info.status = per[i];
                T.info.reached = reached[i];
                T.info.relaxed_edges = st[i].relaxed_edges;
                T.info.checksum = cs[i];
                T.info.latency_ms = std::chrono::duration<double, std::milli>(now - T.submitted).count();
                T.done = true;
            }
        }
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

kairos_status kairos_serve_create(kairos_graph *g, const kairos_serve_opts *opts, kairos_server **out) {
    if (!g || !out) return kairos::fail(KAIROS_ERR_INVALID_ARG, "serve create: NULL argument");
    kairos_server *S = new (std::nothrow) kairos_server();
    if (!S) return kairos::fail(KAIROS_ERR_OOM, "serve create: host allocation failed");
    S->g = g;
    if (opts) {
        if (opts->max_slots < 0 || opts->queue_capacity < 0 || opts->reserve_bytes < 0) {
            delete S;
            return kairos::fail(KAIROS_ERR_INVALID_ARG, "serve create: negative option");
        }
        if (opts->max_slots) S->slots = opts->max_slots;
        if (opts->queue_capacity) S->capacity = opts->queue_capacity;
        if (opts->reserve_bytes) S->reserve = opts->reserve_bytes;
    }
    S->rows = (uint32_t *)g->A.get((size_t)S->slots * g->n * 4);
    if (!S->rows) {
        delete S;
        return kairos::fail(KAIROS_ERR_OOM, "serve create: device allocation failed");
    }
    try {
        S->th = std::thread(worker, S);
    } catch (...) {
        g->A.put(S->rows);
        delete S;
        return kairos::fail(KAIROS_ERR_OOM, "serve create: thread start failed");
    }
    *out = S;
    return KAIROS_OK;
}

kairos_status kairos_serve_submit(kairos_server *S, const kairos_query *q, uint32_t *out, uint64_t *ticket) {
    if (!S || !q || !out || !ticket) return kairos::fail(KAIROS_ERR_INVALID_ARG, "serve submit: NULL argument");
    const kairos_graph *g = S->g;
    if (q->vertex < 0 || q->vertex >= g->n || q->kind > 1 || q->strict > 1 || q->ta > q->tw ||
        q->tw > kairos::TMAX || (q->kind == KAIROS_LD && !g->has_rev))
        return kairos::fail(KAIROS_ERR_INVALID_ARG, "serve submit: invalid query");
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->pending.size() >= S->capacity) return kairos::fail(KAIROS_ERR_BUSY, "serve submit: queue full");
    const uint64_t id = S->next_ticket++;
    Ticket T;
    T.q = *q;
    T.out = out;
    T.submitted = clk::now();
    S->tickets.emplace(id, T);
    S->pending.push_back(id);
    *ticket = id;
    S->cv_work.notify_one();
    return KAIROS_OK;
}

kairos_status kairos_serve_poll(kairos_server *S, uint64_t ticket, int64_t timeout_us, kairos_result_info *info) {
    if (!S || !info) return kairos::fail(KAIROS_ERR_INVALID_ARG, "serve poll: NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return kairos::fail(KAIROS_ERR_INVALID_ARG, "serve poll: unknown ticket");
    auto ready = [&] { return S->tickets[ticket].done; };
    if (!ready()) {
        if (timeout_us < 0) S->cv_done.wait(lk, ready);
        else if (timeout_us > 0) S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    it = S->tickets.find(ticket);
    if (!it->second.done) return kairos::fail(KAIROS_ERR_NOT_READY, "serve poll: not finished");
    *info = it->second.info;
    S->tickets.erase(it);
    return KAIROS_OK;
}

void kairos_serve_destroy(kairos_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    S->g->A.put(S->rows);
    delete S;
}

}  // extern "C"
