// Continuous-batching query server.
//
// One host thread drives two resumable batched edge-maps ("sessions"): earliest arrival
// on the forward graph and latest departure on the mirrored reverse graph, each with W
// query lanes whose state ([n][W] labels and scan bounds, frontier queue and bitmap,
// counters) stays on the device between launches.  The thread alternates launches of a
// few rounds between the sessions.  After each launch it
//   - retires every lane whose query finished: a lane that lowered no label in the last
//     round has nothing left to expand (work only ever comes from a lowered label), as has
//     every lane once the frontier is empty; its column is read out on the device into the
//     ticket's buffer, with the reached count and checksum;
//   - admits waiting queries into free lanes while device memory stays above the reserve:
//     the lane's column is reset and its source joins the frontier of the next round.
// So a query that arrives while others run is admitted at the next launch boundary and
// shares the edge loads of the running batch.  Lanes never interact (each has its own
// labels and bounds), so every answer equals that of the same query alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "trace.h"

using clk = std::chrono::steady_clock;
using namespace kairos;

namespace {

struct Ticket {
    kairos_query q;
    uint32_t *out;
    bool out_on_device;
    clk::time_point submitted;
    bool done = false;
    kairos_result_info info{};
};

struct Session {
    int kind = 0;
    const Csr *csr = nullptr;
    int W = 0;
    uint32_t *arr = nullptr, *prev = nullptr, *bm = nullptr, *bigb = nullptr, *owner = nullptr, *stage = nullptr;
    int32_t *queue = nullptr;
    BigEntry *big = nullptr;
    uint32_t cap_big = 0, cap_chunks = 0;
    EdgeMapCtr *ctr = nullptr, *ctr_host = nullptr;
    unsigned long long *stats = nullptr, *stats_host = nullptr;  // [W][2] reached, checksum
    uint32_t r = 0;          // next round to run
    bool fresh = true;       // next launch initialises the whole state
    uint32_t running = 0;    // lanes holding a query
    uint32_t pending_seed = 0;  // lanes admitted since the last launch
    uint64_t ticket[MAX_LANES] = {};
    uint64_t relaxed_base[MAX_LANES] = {};
    uint32_t admitted_round[MAX_LANES] = {};
    LaneParams lp{};
    cudaStream_t s = nullptr;  // the session's stream (the graph's for EA, the server's own for LD)
    bool launched = false;     // a slice is in flight
    uint32_t last_seeded = 0;  // lanes seeded by the slice in flight (diagnostics)
    std::chrono::steady_clock::time_point t_launch;
};

}  // namespace

struct kairos_server {
    kairos_graph *g = nullptr;
    int device = 0;  // the graph's device: the worker thread runs there
    int slots = 16;
    int capacity = 4096;
    int64_t reserve = 256LL << 20;
    int slice = 2;
    FILE *log = nullptr;  // KAIROS_SERVE_LOG: one line per session step (diagnostics)
    Session sess[2];
    cudaStream_t side = nullptr;  // the latest-departure session's stream
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
};

namespace {

void free_session(const Allocator &A, Session &S) {
    A.put(S.arr);
    A.put(S.prev);
    A.put(S.bm);
    A.put(S.queue);
    A.put(S.big);
    A.put(S.bigb);
    A.put(S.owner);
    A.put(S.stage);
    A.put(S.ctr);
    A.put(S.stats);
    if (S.ctr_host) cudaFreeHost(S.ctr_host);
    if (S.stats_host) cudaFreeHost(S.stats_host);
    const int kind = S.kind;
    const Csr *csr = S.csr;
    cudaStream_t st = S.s;
    S = Session();
    S.kind = kind;
    S.csr = csr;
    S.s = st;
}

kairos_status alloc_session(kairos_graph *g, Session &S, int W) {
    const Allocator &A = g->A;
    const int64_t n = g->n, nwords = (n + 31) / 32;
    uint64_t vbig = 0, nch = 0;
    kairos_status st = split_capacity(A, g->stream, n, S.csr->off, g->tuning.warp_max_edges, g->tuning.chunk_edges,
                                      &vbig, &nch);
    if (st != KAIROS_OK) return st;
    S.W = W;
    S.cap_big = (uint32_t)(vbig + 1);
    S.cap_chunks = (uint32_t)(nch + 1);
    S.arr = (uint32_t *)A.get((size_t)n * W * 4);
    S.prev = (uint32_t *)A.get((size_t)n * W * 4);
    S.stage = (uint32_t *)A.get((size_t)n * W * 4);
    S.bm = (uint32_t *)A.get((size_t)nwords * 2 * 4);
    S.queue = (int32_t *)A.get((size_t)n * 2 * 4);
    S.big = (BigEntry *)A.get((size_t)S.cap_big * sizeof(BigEntry));
    S.bigb = (uint32_t *)A.get((size_t)S.cap_big * W * 2 * 4);
    S.owner = (uint32_t *)A.get((size_t)S.cap_chunks * 4);
    S.ctr = (EdgeMapCtr *)A.get(sizeof(EdgeMapCtr));
    S.stats = (unsigned long long *)A.get((size_t)MAX_LANES * 16);
    if (!S.arr || !S.prev || !S.stage || !S.bm || !S.queue || !S.big || !S.bigb || !S.owner || !S.ctr || !S.stats) {
        free_session(A, S);
        return fail(KAIROS_ERR_OOM, "serve: device allocation failed");
    }
    cudaError_t e = cudaMallocHost(&S.ctr_host, sizeof(EdgeMapCtr));
    if (e == cudaSuccess) e = cudaMallocHost(&S.stats_host, (size_t)MAX_LANES * 16);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.owner, 0xFF, (size_t)S.cap_chunks * 4, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        free_session(A, S);
        return cuda_fail(e, "serve: session setup");
    }
    S.fresh = true;
    return KAIROS_OK;
}

EdgeMapArgs session_args(kairos_graph *g, Session &S) {
    const int64_t n = g->n, nwords = (n + 31) / 32;
    EdgeMapArgs a;
    std::memset(&a, 0, sizeof(a));
    a.off = S.csr->off;
    a.dst = S.csr->dst;
    a.t = S.csr->t;
    a.lam = S.csr->lam;
    a.fidx = S.csr->fidx;
    a.fence = S.csr->fence;
    a.n = n;
    a.arr = S.arr;
    a.prev = S.prev;
    a.bm[0] = S.bm;
    a.bm[1] = S.bm + nwords;
    a.queue[0] = S.queue;
    a.queue[1] = S.queue + n;
    a.big = S.big;
    a.bigb = S.bigb;
    a.chunk_owner = S.owner;
    a.cap_big = S.cap_big;
    a.cap_chunks = S.cap_chunks;
    a.ctr = S.ctr;
    a.out = nullptr;
    a.out_stride = n;
    a.lanes = S.lp;
    a.lanes.nlanes = S.W;
    a.max_rounds = 0xFFFFFFFFu;
    a.spin_limit = DEFAULT_SPIN_LIMIT;
    a.warp_max_edges = g->tuning.warp_max_edges;
    a.chunk_edges = g->tuning.chunk_edges;
    a.dense_div = g->tuning.dense_div;
    a.count_relaxed = 1;
    // resumable slices keep the queue frontier, so the bitmap-frontier mode (1) is replaced
    // by the all-segment mode (0); otherwise the graph's tuned mode applies
    // resumable slices run the frontier kernel: modes 1 and 3 relax with mode 0 there
    a.relax_mode = (g->tuning.relax_mode == 1 || g->tuning.relax_mode == 3) ? 0 : g->tuning.relax_mode;
    a.running_mask = S.running;
    return a;
}

bool memory_allows(kairos_server *V) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown: do not block admission
    }
    return (int64_t)free_b >= V->reserve;
}

// Lane q of S takes ticket id (S and the ticket table are guarded by V->mu).
void admit(kairos_server *V, Session &S, int q, uint64_t id) {
    const Ticket &T = V->tickets[id];
    S.ticket[q] = id;
    S.running |= 1u << q;
    S.pending_seed |= 1u << q;
    LaneParams &lp = S.lp;
    lp.src[q] = T.q.vertex;
    lp.row[q] = 0;
    lp.strict_mask = (lp.strict_mask & ~(1u << q)) | ((uint32_t)T.q.strict << q);
    if (S.kind == KAIROS_EA) {
        lp.ta[q] = T.q.ta;
        lp.tw[q] = T.q.tw;
        lp.mirror_mask &= ~(1u << q);
    } else {
        lp.ta[q] = TMAX - T.q.tw;
        lp.tw[q] = TMAX - T.q.ta;
        lp.mirror_mask |= 1u << q;
    }
}

// Enqueue one slice of S on its stream (seeds, the resumed launch, the counter read-back);
// `share` sessions launch together, each with 1/share of the resident blocks when the graph's
// tuning keeps two launches in flight.
kairos_status launch_session(kairos_server *V, Session &S, int share) {
    TraceRange tr(S.kind == KAIROS_EA ? "serve slice (earliest arrival)" : "serve slice (latest departure)");
    kairos_graph *g = V->g;
    cudaStream_t s = S.s;
    EdgeMapArgs a = session_args(g, S);
    const uint32_t seeds = S.pending_seed;
    if (S.fresh) {
        KAIROS_CUDA(cudaMemsetAsync(S.ctr, 0, sizeof(EdgeMapCtr), s), "serve: counters");
        S.r = 0;
        for (int q = 0; q < MAX_LANES; ++q) S.relaxed_base[q] = 0;
        a.resume = 0;  // the kernel initialises every lane and seeds the running ones
    } else {
        a.resume = 1;  // retired lanes were reset to unreached when they were read out
        for (int q = 0; q < S.W; ++q)
            if ((seeds >> q) & 1u)
                KAIROS_CUDA(seed_lane(a, S.W, q, S.lp.src[q], S.lp.ta[q], S.r, s), "serve: seed lane");
    }
    for (int q = 0; q < S.W; ++q)
        if ((seeds >> q) & 1u) S.admitted_round[q] = S.r;
    a.round_begin = S.r;
    a.round_end = S.r + (uint32_t)V->slice;
    int bps = 0;
    int grid = edgemap_max_grid(S.W, g->lam_bits, a.relax_mode, &bps);
    if (grid <= 0) return fail(KAIROS_ERR_CUDA, "serve: no resident launch shape");
    if (g->tuning.blocks_per_sm > 0 && g->tuning.blocks_per_sm < bps) grid = g->tuning.blocks_per_sm * g->sm_count;
    else if (share == 2) grid = std::max(1, bps / 2) * g->sm_count;  // both slices resident at once
    S.t_launch = clk::now();
    KAIROS_CUDA(edgemap_launch(a, S.W, g->lam_bits, grid, s), "serve: edge-map launch");
    KAIROS_CUDA(cudaMemcpyAsync(S.ctr_host, S.ctr, sizeof(EdgeMapCtr), cudaMemcpyDeviceToHost, s), "serve: counters");
    S.launched = true;
    S.last_seeded = seeds;
    S.fresh = false;
    S.pending_seed = 0;
    return KAIROS_OK;
}

// Wait for S's slice, then retire its finished lanes (labels out, lanes reset).  Appends the
// tickets finished to `done`.
kairos_status finish_session(kairos_server *V, Session &S, std::vector<std::pair<uint64_t, kairos_result_info>> &done) {
    kairos_graph *g = V->g;
    cudaStream_t s = S.s;
    S.launched = false;
    const uint32_t seeds = S.last_seeded;
    KAIROS_CUDA(cudaStreamSynchronize(s), "serve: edge-map");
    const double launch_ms = std::chrono::duration<double, std::milli>(clk::now() - S.t_launch).count();
    const EdgeMapCtr &c = *S.ctr_host;
    if (c.err) {
        S.fresh = true;  // the state is unusable: fail the lanes and start over
        for (int q = 0; q < S.W; ++q)
            if ((S.running >> q) & 1u) {
                kairos_result_info info{};
                info.status = (c.err == KERR_CAPACITY) ? KAIROS_ERR_INTERNAL : KAIROS_ERR_TIMEOUT;
                done.emplace_back(S.ticket[q], info);
            }
        S.running = 0;
        return KAIROS_OK;
    }
    S.r = c.rounds;
    const bool empty = c.qcount[S.r % 3].v == 0;
    uint32_t finished = empty ? S.running : (S.running & ~c.last_active);
    uint32_t timed_out = 0;
    for (int q = 0; q < S.W; ++q)
        if (((S.running & ~finished) >> q) & 1u && (uint64_t)(S.r - S.admitted_round[q]) > (uint64_t)g->n + 1)
            timed_out |= 1u << q;
    finished |= timed_out;
    if (V->log)
        fprintf(V->log, "kind=%d r=%u running=%u seeded=%u finished=%u launch_ms=%.3f\n", S.kind, S.r,
                (unsigned)__builtin_popcount(S.running), (unsigned)__builtin_popcount(seeds),
                (unsigned)__builtin_popcount(finished), launch_ms);
    if (!finished) return KAIROS_OK;
    KAIROS_CUDA(cudaMemsetAsync(S.stats, 0, (size_t)MAX_LANES * 16, s), "serve: readout stats");
    // one pass reads out every finished lane and resets it for its next query
    RetireArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.mask = finished;
    ra.mirror_mask = S.lp.mirror_mask;
    std::vector<std::pair<int, uint32_t *>> to_host;
    for (int q = 0; q < S.W; ++q) {
        if (!((finished >> q) & 1u) || ((timed_out >> q) & 1u)) continue;
        uint32_t *dst;
        bool on_dev;
        {
            std::lock_guard<std::mutex> lk(V->mu);
            const Ticket &T = V->tickets[S.ticket[q]];
            dst = T.out;
            on_dev = T.out_on_device;
        }
        ra.out[q] = on_dev ? dst : S.stage + (int64_t)q * g->n;
        ra.write_mask |= 1u << q;
        if (!on_dev) to_host.emplace_back(q, dst);
    }
    KAIROS_CUDA(retire_lanes(S.arr, S.prev, g->n, S.W, ra, S.stats, s), "serve: retire lanes");
    for (auto &h : to_host)
        KAIROS_CUDA(cudaMemcpyAsync(h.second, S.stage + (int64_t)h.first * g->n, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s),
                    "serve: deliver result");
    KAIROS_CUDA(cudaMemcpyAsync(S.stats_host, S.stats, (size_t)MAX_LANES * 16, cudaMemcpyDeviceToHost, s), "serve: stats");
    KAIROS_CUDA(cudaStreamSynchronize(s), "serve: readout");
    for (int q = 0; q < S.W; ++q) {
        if (!((finished >> q) & 1u)) continue;
        kairos_result_info info{};
        if ((timed_out >> q) & 1u) {
            info.status = KAIROS_ERR_TIMEOUT;
        } else {
            info.status = KAIROS_OK;
            info.reached = (uint32_t)S.stats_host[2 * q];
            info.checksum = S.stats_host[2 * q + 1];
            info.relaxed_edges = c.relaxed[q] - S.relaxed_base[q];
        }
        done.emplace_back(S.ticket[q], info);
        S.relaxed_base[q] = c.relaxed[q];
    }
    S.running &= ~finished;
    return KAIROS_OK;
}

void worker(kairos_server *V) {
    cudaSetDevice(V->device);  // a new thread starts on device 0
    std::vector<std::pair<uint64_t, kairos_result_info>> done;
    int turn = 0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(V->mu);
            V->cv_work.wait(lk, [&] {
                return V->stop || !V->pending.empty() || V->sess[0].running || V->sess[1].running;
            });
            if (V->stop && V->pending.empty() && !V->sess[0].running && !V->sess[1].running) return;
            // admission into free lanes, oldest first, while memory allows
            if (!V->pending.empty() && memory_allows(V)) {
                for (auto it = V->pending.begin(); it != V->pending.end();) {
                    Session &S = V->sess[V->tickets[*it].q.kind];
                    const uint32_t all = S.W >= 32 ? 0xFFFFFFFFu : ((1u << S.W) - 1u);
                    const uint32_t free_lanes = all & ~S.running;
                    if (!free_lanes || !S.W) {
                        ++it;
                        continue;
                    }
                    admit(V, S, __builtin_ctz(free_lanes), *it);
                    it = V->pending.erase(it);
                }
            }
        }
        // one slice per session with work, alternating which goes first; when the graph's tuning
        // keeps two launches in flight, both sessions' slices run at once on their own streams
        done.clear();
        kairos_status st = KAIROS_OK;
        {
            std::lock_guard<std::mutex> glk(V->g->mu);
            const bool together = V->g->tuning.concurrent >= 2 && V->sess[0].running && V->sess[1].running;
            for (int k = 0; k < 2 && st == KAIROS_OK; ++k) {
                Session &S = V->sess[(turn + k) & 1];
                if (!S.running) continue;
                st = launch_session(V, S, together ? 2 : 1);
                if (st == KAIROS_OK && !together) st = finish_session(V, S, done);
            }
            for (int k = 0; k < 2; ++k) {  // the slices still in flight (also after a failure)
                Session &S = V->sess[(turn + k) & 1];
                if (!S.launched) continue;
                const kairos_status st2 = finish_session(V, S, done);
                if (st == KAIROS_OK) st = st2;
            }
        }
        turn ^= 1;
        if (st != KAIROS_OK) {  // a CUDA failure: fail everything in flight and reset
            for (Session &S : V->sess) {
                for (int q = 0; q < S.W; ++q)
                    if ((S.running >> q) & 1u) {
                        kairos_result_info info{};
                        info.status = st;
                        done.emplace_back(S.ticket[q], info);
                    }
                S.running = 0;
                S.pending_seed = 0;
                S.fresh = true;
            }
        }
        if (!done.empty()) {
            const auto now = clk::now();
            {
                std::lock_guard<std::mutex> lk(V->mu);
                for (auto &d : done) {
                    Ticket &T = V->tickets[d.first];
                    T.info = d.second;
                    T.info.latency_ms = std::chrono::duration<double, std::milli>(now - T.submitted).count();
                    T.done = true;
                }
            }
            V->cv_done.notify_all();
        }
    }
}

}  // namespace

int kairos::kairos_server_device(const kairos_server *V) { return V ? V->device : -1; }

namespace {

bool device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

kairos_status kairos_serve_create(kairos_graph *g, const kairos_serve_opts *opts, kairos_server **out) {
    if (!g || !out) return fail(KAIROS_ERR_INVALID_ARG, "serve create: NULL argument");
    kairos_server *V = new (std::nothrow) kairos_server();
    if (!V) return fail(KAIROS_ERR_OOM, "serve create: host allocation failed");
    V->g = g;
    V->device = g->device;
    if (opts) {
        if (opts->max_slots < 0 || opts->queue_capacity < 0 || opts->reserve_bytes < 0 || opts->rounds_per_slice < 0) {
            delete V;
            return fail(KAIROS_ERR_INVALID_ARG, "serve create: negative option");
        }
        if (opts->max_slots) {
            const int L = opts->max_slots;
            if (!(L == 2 || L == 4 || L == 8 || L == 16 || L == 32)) {
                delete V;
                return fail(KAIROS_ERR_INVALID_ARG, "serve create: max_slots must be 2, 4, 8, 16 or 32");
            }
            V->slots = L;
        }
        if (opts->queue_capacity) V->capacity = opts->queue_capacity;
        if (opts->reserve_bytes) V->reserve = opts->reserve_bytes;
        if (opts->rounds_per_slice) V->slice = opts->rounds_per_slice;
    }
    V->sess[0].kind = KAIROS_EA;
    V->sess[0].csr = &g->fwd;
    V->sess[1].kind = KAIROS_LD;
    V->sess[1].csr = &g->rev;
    if (cudaStreamCreateWithFlags(&V->side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete V;
        return fail(KAIROS_ERR_CUDA, "serve create: stream creation failed");
    }
    V->sess[0].s = g->stream;
    V->sess[1].s = V->side;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        for (int k = 0; k < 2; ++k) {
            if (k == 1 && !g->has_rev) continue;
            // lanes per session: the largest width up to max_slots that fits beside the reserve
            kairos_status st = KAIROS_ERR_OOM;
            for (int W = V->slots; W >= 2 && st == KAIROS_ERR_OOM; W /= 2) {
                size_t free_b = 0, total_b = 0;
                if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
                    (int64_t)free_b - V->reserve < (int64_t)g->n * W * 16 + (int64_t)g->m)
                    continue;
                cudaGetLastError();
                st = alloc_session(g, V->sess[k], W);
            }
            if (st != KAIROS_OK) {
                free_session(g->A, V->sess[0]);
                free_session(g->A, V->sess[1]);
                cudaStreamDestroy(V->side);
                delete V;
                return st == KAIROS_ERR_OOM ? fail(st, "serve create: not enough device memory for two lanes") : st;
            }
        }
    }
    if (const char *path = getenv("KAIROS_SERVE_LOG")) V->log = fopen(path, "a");
    try {
        V->th = std::thread(worker, V);
    } catch (...) {
        free_session(g->A, V->sess[0]);
        free_session(g->A, V->sess[1]);
        cudaStreamDestroy(V->side);
        delete V;
        return fail(KAIROS_ERR_OOM, "serve create: thread start failed");
    }
    *out = V;
    return KAIROS_OK;
}

kairos_status kairos_serve_submit(kairos_server *V, const kairos_query *q, uint32_t *out, uint64_t *ticket) {
    if (!V || !q || !out || !ticket) return fail(KAIROS_ERR_INVALID_ARG, "serve submit: NULL argument");
    const kairos_graph *g = V->g;
    if (q->vertex < 0 || q->vertex >= g->n || q->kind > 1 || q->strict > 1 || q->ta > q->tw || q->tw > TMAX ||
        (q->kind == KAIROS_LD && !g->has_rev))
        return fail(KAIROS_ERR_INVALID_ARG, "serve submit: invalid query");
    const bool on_dev = device_ptr(out);
    std::lock_guard<std::mutex> lk(V->mu);
    if ((int)V->pending.size() >= V->capacity) return fail(KAIROS_ERR_BUSY, "serve submit: queue full");
    const uint64_t id = V->next_ticket++;
    Ticket T;
    T.q = *q;
    T.out = out;
    T.out_on_device = on_dev;
    T.submitted = clk::now();
    V->tickets.emplace(id, T);
    V->pending.push_back(id);
    *ticket = id;
    V->cv_work.notify_one();
    return KAIROS_OK;
}

kairos_status kairos_serve_poll(kairos_server *V, uint64_t ticket, int64_t timeout_us, kairos_result_info *info) {
    if (!V || !info) return fail(KAIROS_ERR_INVALID_ARG, "serve poll: NULL argument");
    std::unique_lock<std::mutex> lk(V->mu);
    auto it = V->tickets.find(ticket);
    if (it == V->tickets.end()) return fail(KAIROS_ERR_INVALID_ARG, "serve poll: unknown ticket");
    auto ready = [&] { return V->tickets[ticket].done; };
    if (!ready()) {
        if (timeout_us < 0) V->cv_done.wait(lk, ready);
        else if (timeout_us > 0) V->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    it = V->tickets.find(ticket);
    if (!it->second.done) return fail(KAIROS_ERR_NOT_READY, "serve poll: not finished");
    *info = it->second.info;
    V->tickets.erase(it);
    return KAIROS_OK;
}

void kairos_serve_destroy(kairos_server *V) {
    if (!V) return;
    {
        std::lock_guard<std::mutex> lk(V->mu);
        V->stop = true;
    }
    V->cv_work.notify_all();
    if (V->th.joinable()) V->th.join();
    {
        std::lock_guard<std::mutex> lk(V->g->mu);
        cudaStreamSynchronize(V->g->stream);
        cudaStreamSynchronize(V->side);
        free_session(V->g->A, V->sess[0]);
        free_session(V->g->A, V->sess[1]);
        cudaStreamDestroy(V->side);
    }
    if (V->log) fclose(V->log);
    delete V;
}

}  // extern "C"
