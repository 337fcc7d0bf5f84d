// One query stream over several continuous-batching servers, each on its own graph replica
// (normally one per GPU).  Queries are independent, so the replicas share nothing and no
// collective is involved: a submission goes to one replica and its ticket is polled there.
//
// Routing: an output buffer in device memory names its device, so the query goes to the
// least-loaded replica on that device (the result is written in place there); a host buffer
// goes to the least-loaded replica of all.  Load = submitted minus completed queries; ties go
// to the replica after the last one chosen.  A full replica (BUSY) passes the query to the
// next-least-loaded eligible one; the router is BUSY only when all of them are.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

struct kairos_router {
    struct Replica {
        kairos_server *s;
        int device;
        int64_t load = 0;
        uint64_t submitted = 0, completed = 0;
    };
    std::vector<Replica> rep;
    std::mutex mu;
    std::unordered_map<uint64_t, std::pair<int, uint64_t>> tickets;  // router ticket -> (replica, server ticket)
    uint64_t next_ticket = 1;
    int last = -1;
};

using namespace kairos;

namespace {

int buffer_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (at.type == cudaMemoryTypeDevice) ? at.device : -1;
}

}  // namespace

extern "C" {

kairos_status kairos_router_create(kairos_server *const *servers, int32_t n, kairos_router **out) {
    if (!servers || n < 1 || !out) return fail(KAIROS_ERR_INVALID_ARG, "router create: bad argument");
    kairos_router *R = new (std::nothrow) kairos_router();
    if (!R) return fail(KAIROS_ERR_OOM, "router create: host allocation failed");
    for (int i = 0; i < n; ++i) {
        if (!servers[i]) {
            delete R;
            return fail(KAIROS_ERR_INVALID_ARG, "router create: NULL server");
        }
        kairos_router::Replica r;
        r.s = servers[i];
        r.device = kairos_server_device(servers[i]);
        R->rep.push_back(r);
    }
    *out = R;
    return KAIROS_OK;
}

kairos_status kairos_router_submit(kairos_router *R, const kairos_query *q, uint32_t *out, uint64_t *ticket) {
    if (!R || !q || !out || !ticket) return fail(KAIROS_ERR_INVALID_ARG, "router submit: NULL argument");
    const int dev = buffer_device(out);
    std::lock_guard<std::mutex> lk(R->mu);
    const int nr = (int)R->rep.size();
    // eligible replicas, least loaded first, ties in turn after the last choice
    std::vector<int> order;
    for (int k = 1; k <= nr; ++k) {
        const int i = (R->last + k) % nr;
        if (dev < 0 || R->rep[i].device == dev) order.push_back(i);
    }
    if (order.empty()) return fail(KAIROS_ERR_INVALID_ARG, "router submit: no replica on the output buffer's device");
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return R->rep[a].load < R->rep[b].load; });
    kairos_status st = KAIROS_ERR_BUSY;
    for (int i : order) {
        uint64_t t = 0;
        st = kairos_serve_submit(R->rep[i].s, q, out, &t);
        if (st == KAIROS_ERR_BUSY) continue;
        if (st != KAIROS_OK) return st;
        const uint64_t id = R->next_ticket++;
        R->tickets[id] = {i, t};
        R->rep[i].load += 1;
        R->rep[i].submitted += 1;
        R->last = i;
        *ticket = id;
        return KAIROS_OK;
    }
    return fail(KAIROS_ERR_BUSY, "router submit: every eligible replica's queue is full");
}

kairos_status kairos_router_poll(kairos_router *R, uint64_t ticket, int64_t timeout_us, kairos_result_info *info) {
    if (!R || !info) return fail(KAIROS_ERR_INVALID_ARG, "router poll: NULL argument");
    std::pair<int, uint64_t> where;
    {
        std::lock_guard<std::mutex> lk(R->mu);
        auto it = R->tickets.find(ticket);
        if (it == R->tickets.end()) return fail(KAIROS_ERR_INVALID_ARG, "router poll: unknown ticket");
        where = it->second;
    }
    // wait outside the lock: other threads keep submitting and polling
    kairos_status st = kairos_serve_poll(R->rep[where.first].s, where.second, timeout_us, info);
    if (st == KAIROS_OK) {
        std::lock_guard<std::mutex> lk(R->mu);
        if (R->tickets.erase(ticket)) {
            R->rep[where.first].load -= 1;
            R->rep[where.first].completed += 1;
        }
    }
    return st;
}

int32_t kairos_router_replica_counts(const kairos_router *R, uint64_t *submitted, uint64_t *completed, int32_t n) {
    if (!R) return 0;
    kairos_router *M = const_cast<kairos_router *>(R);
    std::lock_guard<std::mutex> lk(M->mu);
    const int k = std::min<int>(n, (int)R->rep.size());
    for (int i = 0; i < k; ++i) {
        if (submitted) submitted[i] = R->rep[i].submitted;
        if (completed) completed[i] = R->rep[i].completed;
    }
    return (int32_t)R->rep.size();
}

void kairos_router_destroy(kairos_router *R) { delete R; }

}  // extern "C"
