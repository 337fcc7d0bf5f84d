// C ABI of the library: graph lifecycle, the query workspace, single and batched queries,
// launch-shape tuning.  Host code only orchestrates; every step of a query runs in the
// kernels of edgemap.cu and build.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "trace.h"

using namespace kairos;

namespace kairos {

namespace {
thread_local std::string g_err;
}

kairos_status fail(kairos_status st, const std::string &m) {
    g_err = m;
    return st;
}

kairos_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? KAIROS_ERR_OOM : KAIROS_ERR_CUDA;
}

void apply_test_hooks(EdgeMapArgs &a) {
    if (const char *v = getenv("KAIROS_SPIN_LIMIT")) a.spin_limit = strtoull(v, nullptr, 10);
    if (const char *v = getenv("KAIROS_ROUND_CAP")) a.max_rounds = (uint32_t)strtoul(v, nullptr, 10);
}

void *Allocator::get(size_t bytes) const {
    if (bytes == 0) bytes = 1;
    if (alloc) return alloc(bytes, ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Allocator::put(void *p) const {
    if (!p) return;
    if (release) release(p, ctx);
    else cudaFree(p);
}

}  // namespace kairos

namespace {

// Where the kernels may write an output buffer directly: device memory as it is, and
// page-locked host memory through its device mapping (the writes cross the CPU-GPU link
// inside the launch, no staging copy).  Pageable host memory gives nullptr: it is staged
// on the device and copied.  *pinned tells page-locked host memory apart (its device mapping
// may be the same address, as on systems whose GPU shares the host's page tables).
uint32_t *direct_out(uint32_t *p, bool *pinned) {
    *pinned = false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        *pinned = true;
        return (uint32_t *)at.devicePointer;
    }
    return nullptr;
}

void release_work_arrays(kairos_graph *g) {
    auto &w = g->work;
    const auto &A = g->A;
    A.put(w.arr);
    A.put(w.prev);
    A.put(w.bm);
    A.put(w.queue);
    A.put(w.big);
    A.put(w.bigb);
    A.put(w.chunk_owner);
    A.put(w.stage);
    w.arr = w.prev = w.bm = w.bigb = w.chunk_owner = w.stage = nullptr;
    w.queue = nullptr;
    w.big = nullptr;
    A.put(w.arr2);
    A.put(w.prev2);
    A.put(w.bm2);
    A.put(w.queue2);
    A.put(w.big2);
    A.put(w.bigb2);
    A.put(w.chunk_owner2);
    w.arr2 = w.prev2 = w.bm2 = w.bigb2 = w.chunk_owner2 = nullptr;
    w.queue2 = nullptr;
    w.big2 = nullptr;
    w.lanes = 0;
    w.cap_big = w.cap_chunks = 0;
    w.bytes = 0;
}

kairos_status ensure_work(kairos_graph *g, int lanes, bool need_stage, bool need_second) {
    auto &w = g->work;
    const int wm = g->tuning.warp_max_edges, ch = g->tuning.chunk_edges;
    if (w.arr && w.lanes == lanes && w.warp_max == wm && w.chunk == ch && (!need_second || w.arr2)) {
        if (need_stage && !w.stage) {
            w.stage = (uint32_t *)g->A.get((size_t)g->n * lanes * 4);
            if (!w.stage) return fail(KAIROS_ERR_OOM, "query workspace: device allocation failed");
            w.bytes += (size_t)g->n * lanes * 4;
        }
        return KAIROS_OK;
    }
    release_work_arrays(g);
    const int64_t n = g->n;
    const int64_t nwords = (n + 31) / 32;
    uint64_t v1 = 0, c1 = 0, v2 = 0, c2 = 0;
    kairos_status st = split_capacity(g->A, g->stream, n, g->fwd.off, wm, ch, &v1, &c1);
    if (st != KAIROS_OK) return st;
    if (g->has_rev) {
        st = split_capacity(g->A, g->stream, n, g->rev.off, wm, ch, &v2, &c2);
        if (st != KAIROS_OK) return st;
    }
    const uint64_t cap_big = std::max(v1, v2) + 1, cap_chunks = std::max(c1, c2) + 1;
    if (cap_chunks > 0xFFFFFFF0ull || cap_big > 0xFFFFFFF0ull)
        return fail(KAIROS_ERR_INVALID_ARG, "query workspace: too many split ranges for this chunk size");
    const auto &A = g->A;
    w.arr = (uint32_t *)A.get((size_t)n * lanes * 4);
    w.prev = (uint32_t *)A.get((size_t)n * lanes * 4);
    w.bm = (uint32_t *)A.get((size_t)nwords * 2 * 4);
    w.queue = (int32_t *)A.get((size_t)n * 2 * 4);
    w.big = (BigEntry *)A.get((size_t)cap_big * sizeof(BigEntry));
    w.bigb = (uint32_t *)A.get((size_t)cap_big * lanes * 2 * 4);
    w.chunk_owner = (uint32_t *)A.get((size_t)cap_chunks * 4);
    if (need_stage) w.stage = (uint32_t *)A.get((size_t)n * lanes * 4);
    if (need_second) {
        w.arr2 = (uint32_t *)A.get((size_t)n * lanes * 4);
        w.prev2 = (uint32_t *)A.get((size_t)n * lanes * 4);
        w.bm2 = (uint32_t *)A.get((size_t)nwords * 2 * 4);
        w.queue2 = (int32_t *)A.get((size_t)n * 2 * 4);
        w.big2 = (BigEntry *)A.get((size_t)cap_big * sizeof(BigEntry));
        w.bigb2 = (uint32_t *)A.get((size_t)cap_big * lanes * 2 * 4);
        w.chunk_owner2 = (uint32_t *)A.get((size_t)cap_chunks * 4);
    }
    if (!w.arr || !w.prev || !w.bm || !w.queue || !w.big || !w.bigb || !w.chunk_owner || (need_stage && !w.stage) ||
        (need_second && (!w.arr2 || !w.prev2 || !w.bm2 || !w.queue2 || !w.big2 || !w.bigb2 || !w.chunk_owner2))) {
        release_work_arrays(g);
        return fail(KAIROS_ERR_OOM, "query workspace: device allocation failed");
    }
    KAIROS_CUDA(cudaMemsetAsync(w.chunk_owner, 0xFF, (size_t)cap_chunks * 4, g->stream), "workspace init");
    if (need_second)
        KAIROS_CUDA(cudaMemsetAsync(w.chunk_owner2, 0xFF, (size_t)cap_chunks * 4, g->stream), "workspace init");
    w.lanes = lanes;
    w.warp_max = wm;
    w.chunk = ch;
    w.cap_big = (uint32_t)cap_big;
    w.cap_chunks = (uint32_t)cap_chunks;
    const size_t set_bytes = (size_t)n * lanes * 8 + (size_t)nwords * 8 + (size_t)n * 8 +
                             cap_big * (sizeof(BigEntry) + lanes * 8) + cap_chunks * 4;
    w.bytes = set_bytes * (need_second ? 2 : 1) + (need_stage ? (size_t)n * lanes * 4 : 0);
    return KAIROS_OK;
}

kairos_status check_query(const kairos_graph *g, const kairos_query &q) {
    if (q.vertex < 0 || (int64_t)q.vertex >= g->n) return fail(KAIROS_ERR_INVALID_ARG, "query vertex out of range");
    if (q.kind > 1) return fail(KAIROS_ERR_INVALID_ARG, "query kind must be KAIROS_EA or KAIROS_LD");
    if (q.strict > 1) return fail(KAIROS_ERR_INVALID_ARG, "query strict must be 0 or 1");
    if (q.ta > q.tw || q.tw > TMAX) return fail(KAIROS_ERR_INVALID_ARG, "query window needs ta <= tw <= KAIROS_TIME_MAX");
    if (q.kind == KAIROS_LD && !g->has_rev)
        return fail(KAIROS_ERR_INVALID_ARG, "latest departure needs the reverse graph (built with skip_reverse)");
    return KAIROS_OK;
}

// Lane q of a launch takes query Q; latest departure runs as earliest arrival on the
// mirrored reverse graph over [TMAX - tw, TMAX - ta].
void lane_set(LaneParams &lp, int q, const kairos_query &Q, int64_t row) {
    lp.src[q] = Q.vertex;
    if (Q.kind == KAIROS_EA) {
        lp.ta[q] = Q.ta;
        lp.tw[q] = Q.tw;
    } else {
        lp.ta[q] = TMAX - Q.tw;
        lp.tw[q] = TMAX - Q.ta;
        lp.mirror_mask |= 1u << q;
    }
    if (Q.strict) lp.strict_mask |= 1u << q;
    lp.row[q] = row;
}

EdgeMapArgs make_args(kairos_graph *g, const Csr &c, const LaneParams &lp, uint32_t *out, int64_t stride,
                      uint32_t *arr_alias, int count_relaxed, EdgeMapCtr *ctr, int slot = 0) {
    auto &w = g->work;
    const bool s2 = slot == 1;  // the second workspace (concurrent launches)
    const int64_t n = g->n, nwords = (n + 31) / 32;
    EdgeMapArgs a;
    std::memset(&a, 0, sizeof(a));
    a.off = c.off;
    a.dst = c.dst;
    a.t = c.t;
    a.lam = c.lam;
    a.fidx = c.fidx;
    a.fence = c.fence;
    a.n = n;
    a.arr = arr_alias ? arr_alias : (s2 ? w.arr2 : w.arr);
    a.prev = s2 ? w.prev2 : w.prev;
    a.bm[0] = s2 ? w.bm2 : w.bm;
    a.bm[1] = a.bm[0] + nwords;
    a.queue[0] = s2 ? w.queue2 : w.queue;
    a.queue[1] = a.queue[0] + n;
    a.big = s2 ? w.big2 : w.big;
    a.bigb = s2 ? w.bigb2 : w.bigb;
    a.chunk_owner = s2 ? w.chunk_owner2 : w.chunk_owner;
    a.cap_big = w.cap_big;
    a.cap_chunks = w.cap_chunks;
    a.ctr = ctr;
    a.out = out;
    a.out_stride = stride;
    a.out_is_arr = (arr_alias != nullptr && out == arr_alias) ? 1 : 0;
    a.lanes = lp;
    a.max_rounds = (uint32_t)std::min<int64_t>(n + 1, 0xFFFFFFF0LL);
    a.spin_limit = DEFAULT_SPIN_LIMIT;
    apply_test_hooks(a);
    a.warp_max_edges = g->tuning.warp_max_edges;
    a.chunk_edges = g->tuning.chunk_edges;
    a.dense_div = g->tuning.dense_div;
    a.hidx = c.hidx;
    a.hhdr = c.hhdr;
    a.hcum = c.hcum;
    a.hrow = c.hrow;
    a.select_permille = c.hidx ? g->tuning.select_permille : 0;
    a.count_relaxed = count_relaxed;
    a.relax_mode = g->tuning.relax_mode;
    a.resume = 0;
    a.round_begin = 0;
    a.round_end = 0xFFFFFFFFu;
    a.running_mask = 0xFFFFFFFFu;
    static const int phase_clock = getenv("KAIROS_PHASE_CLOCK") ? atoi(getenv("KAIROS_PHASE_CLOCK")) : 0;
    a.phase_clock = phase_clock;
    return a;
}

kairos_status ctr_error(int err) {
    if (err == KERR_BARRIER_TIMEOUT) return fail(KAIROS_ERR_TIMEOUT, "edge-map: a grid barrier wait ran past its limit");
    if (err == KERR_WAIT_TIMEOUT) return fail(KAIROS_ERR_TIMEOUT, "edge-map: a wait for a published chunk ran past its limit");
    if (err == KERR_ROUNDS) return fail(KAIROS_ERR_TIMEOUT, "edge-map: round cap (n + 1) reached");
    return fail(KAIROS_ERR_INTERNAL, "edge-map: split-range capacity exceeded");
}

// One launch of a call: its arguments and the queries of its lanes.
struct Planned {
    EdgeMapArgs a;
    std::vector<int> qid;
    const uint32_t *host_src;  // device rows to copy to host outputs (nullptr: none)
};

kairos_status ensure_ctr_slots(kairos_graph *g, size_t count) {
    auto &w = g->work;
    if (w.ctr_slots >= count) return KAIROS_OK;
    g->A.put(w.ctrs);
    if (w.ctrs_host) cudaFreeHost(w.ctrs_host);
    w.ctrs = nullptr;
    w.ctrs_host = nullptr;
    w.ctr_slots = 0;
    const size_t want = std::max<size_t>(count, 8);
    w.ctrs = (EdgeMapCtr *)g->A.get(want * sizeof(EdgeMapCtr));
    if (!w.ctrs) return fail(KAIROS_ERR_OOM, "query counters: device allocation failed");
    KAIROS_CUDA(cudaMallocHost(&w.ctrs_host, want * sizeof(EdgeMapCtr)), "query counters: pinned allocation");
    w.ctr_slots = want;
    return KAIROS_OK;
}

void drop_graph(kairos_graph *g) {
    auto &w = g->work;
    if (w.graph_exec) cudaGraphExecDestroy(w.graph_exec);
    w.graph_exec = nullptr;
    w.graph_key.clear();
    cudaGetLastError();
}

// ---- stream mode (relax_mode 3) -------------------------------------------------------------

void release_stream_work(kairos_graph *g) {
    for (auto &sw : g->sw) {
        g->A.put(sw.arr);
        g->A.put(sw.minrow);
        g->A.put(sw.rsum);
        g->A.put(sw.fbm);
        g->A.put(sw.fq);
        g->A.put(sw.stage);
        sw = kairos_graph::StreamWork();
    }
}

int64_t default_block_edges(const kairos_graph *g) {
    if (g->tuning.block_edges > 0) return g->tuning.block_edges;
    return std::max<int64_t>(g->m / 512, 4096);
}

// The time-ordered records of the directions the call needs, cut for the current block size.
kairos_status ensure_time_stream(kairos_graph *g, bool fwd, bool rev) {
    const int64_t eb = default_block_edges(g);
    for (int d = 0; d < 2; ++d) {
        if (d == 0 ? !fwd : !rev) continue;
        TimeStream &ts = d == 0 ? g->ts_fwd : g->ts_rev;
        const Csr &c = d == 0 ? g->fwd : g->rev;
        if (!ts.rec) {
            ts.rec = (StreamRec *)g->A.get((size_t)std::max<int64_t>(g->m, 1) * sizeof(StreamRec));
            if (!ts.rec) return fail(KAIROS_ERR_OOM, "time stream: device allocation failed");
            kairos_status st = build_time_stream(g->A, g->stream, g->n, g->m, c, g->lam_bits, ts.rec);
            if (st != KAIROS_OK) {
                free_time_stream(g->A, &ts);
                return st;
            }
        }
        if (!ts.bnd || ts.block_edges != eb) {
            kairos_status st = cut_time_blocks(g->A, g->stream, g->m, eb, &ts);
            if (st != KAIROS_OK) return st;
        }
        kairos_status st = build_vertex_spans(g->A, g->stream, g->n, c, &ts);
        if (st != KAIROS_OK) return st;
    }
    return KAIROS_OK;
}

kairos_status ensure_stream_work(kairos_graph *g, int W, int slots) {
    const int64_t n = g->n, nwords = (n + 31) / 32;
    for (int i = 0; i < slots; ++i) {
        auto &sw = g->sw[i];
        if (sw.arr && sw.lanes == W) continue;
        g->A.put(sw.arr);
        g->A.put(sw.minrow);
        g->A.put(sw.rsum);
        g->A.put(sw.fbm);
        g->A.put(sw.fq);
        g->A.put(sw.stage);
        sw = kairos_graph::StreamWork();
        sw.arr = (uint32_t *)g->A.get((size_t)n * W * 4);
        sw.minrow = (uint32_t *)g->A.get((size_t)n * 4);
        sw.rsum = (unsigned long long *)g->A.get((size_t)n * 16);
        sw.fbm = (uint32_t *)g->A.get((size_t)nwords * 4);
        sw.fq = (int32_t *)g->A.get((size_t)n * 2 * 4);
        if (!sw.arr || !sw.minrow || !sw.rsum || !sw.fbm || !sw.fq) {
            release_stream_work(g);
            return fail(KAIROS_ERR_OOM, "stream workspace: device allocation failed");
        }
        sw.lanes = W;
        sw.bytes = (size_t)n * W * 4 + (size_t)n * 28 + (size_t)nwords * 4;
    }
    return KAIROS_OK;
}

// Device staging rows for host outputs of the first `slots` launch slots.
kairos_status ensure_stream_stage(kairos_graph *g, int slots) {
    for (int i = 0; i < slots; ++i) {
        auto &sw = g->sw[i];
        if (sw.stage) continue;
        sw.stage = (uint32_t *)g->A.get((size_t)g->n * sw.lanes * 4);
        if (!sw.stage) return fail(KAIROS_ERR_OOM, "stream staging: device allocation failed");
        sw.bytes += (size_t)g->n * sw.lanes * 4;
    }
    return KAIROS_OK;
}

kairos_status ensure_sctr_slots(kairos_graph *g, size_t count) {
    if (g->sctr_slots >= count) return KAIROS_OK;
    g->A.put(g->sctrs);
    if (g->sctrs_host) cudaFreeHost(g->sctrs_host);
    g->sctrs = nullptr;
    g->sctrs_host = nullptr;
    g->sctr_slots = 0;
    const size_t want = std::max<size_t>(count, 8);
    g->sctrs = (StreamCtr *)g->A.get(want * sizeof(StreamCtr));
    if (!g->sctrs) return fail(KAIROS_ERR_OOM, "stream counters: device allocation failed");
    KAIROS_CUDA(cudaMallocHost(&g->sctrs_host, want * sizeof(StreamCtr)), "stream counters: pinned allocation");
    g->sctr_slots = want;
    return KAIROS_OK;
}

kairos_status stream_error(const StreamCtr &c) {
    const std::string at = " (time block " + std::to_string(c.err_block) + ", fix-up round " +
                           (c.err_round == 0xFFFFFFFFu ? std::string("-") : std::to_string(c.err_round)) + ")";
    if (c.err == KERR_FIX_ROUNDS) return fail(KAIROS_ERR_TIMEOUT, "stream edge-map: fix-up round cap reached");
    if (c.err == KERR_BARRIER_TIMEOUT)
        return fail(KAIROS_ERR_TIMEOUT, "stream edge-map: a grid barrier wait ran past its limit" + at);
    return fail(KAIROS_ERR_INTERNAL, "stream edge-map: device error");
}

struct StreamPlanned {
    StreamArgs a;
    std::vector<int> qid;
    bool host_out;
};

// Queries through the time-ordered edge-map, `lanes` (32 or 64) per launch; the same contract
// as kairos_run_queries.
kairos_status run_stream_queries(kairos_graph *g, const kairos_query *qs, int32_t nq, uint32_t *out,
                                 kairos_query_stats *stats, int lanes) {
    const int64_t n = g->n;
    uint32_t *const host_out = out;  // the caller's pointer (staged copies go there)
    bool dev = true, pinned = false;  // outputs the kernels can write (device or page-locked memory)
    if (out) {
        uint32_t *d = direct_out(out, &pinned);
        dev = d != nullptr;
        if (d) out = d;
    }
    bool need_f = false, need_r = false;
    int64_t n_launch = 0;
    for (int kind = 0; kind < 2; ++kind) {
        int64_t c = 0;
        for (int i = 0; i < nq; ++i) c += qs[i].kind == kind;
        n_launch += (c + lanes - 1) / lanes;
        if (c) (kind == 0 ? need_f : need_r) = true;
    }
    const int C = dev ? (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)std::max(g->tuning.concurrent, 1), n_launch, 4}))
                      : 1;
    // Host outputs are staged: each launch writes its rows to device memory and the copy engine
    // moves them to the host on the launch's stream, overlapping the launches still running.
    // Only a page-locked output of a call with one launch in flight is written by the kernel
    // directly (kernel writes across the CPU-GPU link stalled the grid barriers of a launch
    // running beside them).
    const bool staged = out && (!dev || (pinned && C >= 2));
    kairos_status st = ensure_time_stream(g, need_f, need_r);
    if (st != KAIROS_OK) return st;
    st = ensure_stream_work(g, lanes, C);
    if (st != KAIROS_OK) return st;
    if (staged) {
        st = ensure_stream_stage(g, C);
        if (st != KAIROS_OK) return st;
    }
    auto &w = g->work;
    if (C >= 2 && !g->sfork)
        KAIROS_CUDA(cudaEventCreateWithFlags(&g->sfork, cudaEventDisableTiming), "concurrent launches: event");
    for (int k = 0; k + 1 < C; ++k)
        if (!g->sside[k]) {
            KAIROS_CUDA(cudaStreamCreateWithFlags(&g->sside[k], cudaStreamNonBlocking), "concurrent launches: stream");
            KAIROS_CUDA(cudaEventCreateWithFlags(&g->sjoin[k], cudaEventDisableTiming), "concurrent launches: event");
        }
    g->last_kernel_ms = 0;
    cudaStream_t s = g->stream;
    std::vector<StreamPlanned> plan;
    std::vector<int> idx;
    uint32_t round_cap = (uint32_t)std::min<int64_t>(n + 1, 0xFFFFFFF0LL);
    if (const char *v = getenv("KAIROS_ROUND_CAP")) round_cap = (uint32_t)strtoul(v, nullptr, 10);
    unsigned long long spin = DEFAULT_SPIN_LIMIT;
    if (const char *v = getenv("KAIROS_SPIN_LIMIT")) spin = strtoull(v, nullptr, 10);
    for (int kind = 0; kind < 2; ++kind) {
        idx.clear();
        for (int i = 0; i < nq; ++i)
            if (qs[i].kind == kind) idx.push_back(i);
        const Csr &csr = kind == KAIROS_EA ? g->fwd : g->rev;
        const TimeStream &ts = kind == KAIROS_EA ? g->ts_fwd : g->ts_rev;
        for (size_t c = 0; c < idx.size(); c += lanes) {
            const int k = (int)std::min<size_t>(lanes, idx.size() - c);
            const int slot = (int)(plan.size() % C);
            StreamPlanned P;
            StreamArgs &a = P.a;
            std::memset(&a, 0, sizeof(a));
            uint32_t lo_t = INF, hi_t = 0;
            for (int j = 0; j < k; ++j) {
                const kairos_query &Q = qs[idx[c + j]];
                a.lanes.src[j] = Q.vertex;
                if (Q.kind == KAIROS_EA) {
                    a.lanes.ta[j] = Q.ta;
                    a.lanes.tw[j] = Q.tw;
                } else {
                    a.lanes.ta[j] = TMAX - Q.tw;
                    a.lanes.tw[j] = TMAX - Q.ta;
                    a.lanes.mirror_mask |= 1ull << j;
                }
                if (Q.strict) a.lanes.strict_mask |= 1ull << j;
                a.lanes.row[j] = (out && !staged) ? idx[c + j] : j;
                lo_t = std::min(lo_t, a.lanes.ta[j]);
                hi_t = std::max(hi_t, a.lanes.tw[j]);
            }
            a.lanes.nlanes = k;
            // blocks that can hold a usable departure of some lane: [block of lo_t, block after hi_t)
            const uint32_t *bt = ts.bt_host;
            const int nb = ts.nblk;
            int kb = (int)(std::upper_bound(bt, bt + nb, lo_t) - bt) - 1;
            if (kb < 0) kb = 0;
            int ke = (int)(std::upper_bound(bt, bt + nb, hi_t) - bt);
            if (ke < kb) ke = kb;
            a.rec = ts.rec;
            a.bnd = ts.bnd;
            a.bt = ts.bt;
            a.span = ts.span;
            a.k_begin = kb;
            a.k_end = ke;
            a.off = csr.off;
            a.dst = csr.dst;
            a.t = csr.t;
            a.lam = csr.lam;
            a.n = n;
            const auto &sw = g->sw[slot];
            a.arr = sw.arr;
            a.minrow = sw.minrow;
            a.rsum = sw.rsum;
            a.fbm = sw.fbm;
            a.fq[0] = sw.fq;
            a.fq[1] = sw.fq + n;
            a.out = out ? (staged ? sw.stage : out) : nullptr;
            a.out_stride = n;
            a.max_fix_rounds = round_cap;
            a.spin_limit = spin;
            a.count_relaxed = stats != nullptr;
            static const int phase_clock = getenv("KAIROS_PHASE_CLOCK") ? atoi(getenv("KAIROS_PHASE_CLOCK")) : 0;
            a.phase_clock = phase_clock;
            P.qid.assign(idx.begin() + c, idx.begin() + c + k);
            P.host_out = staged;
            plan.push_back(std::move(P));
        }
    }
    if (plan.empty()) return KAIROS_OK;
    st = ensure_sctr_slots(g, plan.size());
    if (st != KAIROS_OK) return st;
    for (size_t i = 0; i < plan.size(); ++i) plan[i].a.ctr = g->sctrs + i;
    int bps = 0;
    int grid = stream_max_grid(lanes, g->lam_bits, g->sm_count, &bps);
    if (grid <= 0) return fail(KAIROS_ERR_CUDA, "stream edge-map: no resident launch shape (occupancy query failed)");
    // grid of each launch slot: with launches in flight the resident blocks per SM are shared out in
    // proportion to each slot's time blocks (its sweep rounds), at least one each, so that the slot with
    // the longer sweep is not left alone on a fraction of the GPU; all launches in flight stay resident
    std::vector<int> slot_grid(C, grid);
    if (g->tuning.blocks_per_sm > 0 && g->tuning.blocks_per_sm < bps) {
        grid = g->tuning.blocks_per_sm * g->sm_count;
        for (int k = 0; k < C; ++k) slot_grid[k] = grid;
    } else if (C >= 2) {
        grid = std::max(1, bps / C) * g->sm_count;
        std::vector<double> cost(C, 0.0);
        double total = 0;
        for (size_t i = 0; i < plan.size(); ++i) {
            const double c = 1.0 + (plan[i].a.k_end - plan[i].a.k_begin);
            cost[i % C] += c;
            total += c;
        }
        if (bps >= C) {
            std::vector<int> b(C, 1);
            int left = bps - C;
            while (left > 0) {  // each remaining block to the slot with the most cost per block
                int best = 0;
                for (int k = 1; k < C; ++k)
                    if (cost[k] / b[k] > cost[best] / b[best]) best = k;
                ++b[best];
                --left;
            }
            for (int k = 0; k < C; ++k) slot_grid[k] = b[k] * g->sm_count;
        } else {
            for (int k = 0; k < C; ++k) slot_grid[k] = grid;
        }
    }

    auto enqueue = [&]() -> kairos_status {
        if (C >= 2) {  // fork: the side streams start after everything before this call
            KAIROS_CUDA(cudaEventRecord(g->sfork, s), "concurrent launches: fork");
            for (int k = 0; k + 1 < C; ++k)
                KAIROS_CUDA(cudaStreamWaitEvent(g->sside[k], g->sfork, 0), "concurrent launches: fork");
        }
        for (size_t i = 0; i < plan.size(); ++i) {
            const int slot = (int)(i % C);
            cudaStream_t si = slot ? g->sside[slot - 1] : s;
            KAIROS_CUDA(cudaMemsetAsync(plan[i].a.ctr, 0, sizeof(StreamCtr), si), "stream edge-map counters");
            KAIROS_CUDA(stream_launch(plan[i].a, lanes, g->lam_bits, slot_grid[slot], si), "stream edge-map launch");
            if (plan[i].host_out) {  // the copy engine, on the launch's stream
                const std::vector<int> &q = plan[i].qid;
                const uint32_t *src = g->sw[slot].stage;
                for (size_t j = 0; j < q.size(); ++j)
                    KAIROS_CUDA(cudaMemcpyAsync(host_out + (int64_t)q[j] * n, src + (int64_t)j * n, (size_t)n * 4,
                                                cudaMemcpyDeviceToHost, si),
                                "copy labels to host");
            }
        }
        for (int k = 0; k + 1 < C; ++k) {  // join: the call's stream waits for the side streams
            KAIROS_CUDA(cudaEventRecord(g->sjoin[k], g->sside[k]), "concurrent launches: join");
            KAIROS_CUDA(cudaStreamWaitEvent(s, g->sjoin[k], 0), "concurrent launches: join");
        }
        return KAIROS_OK;
    };

    KAIROS_CUDA(cudaEventRecord(w.ev0, s), "event record");
    // device and page-locked outputs: the whole sequence (launches in flight on their streams, and
    // for staged page-locked outputs the copies after each launch) is captured into a CUDA graph and
    // replayed while the same call repeats; pageable outputs are copied by the host path
    const bool capturable = dev && s != nullptr && !getenv("KAIROS_NO_GRAPH");
    bool launched = false;
    if (capturable) {
        std::string key("stream", 6);
        key.append((const char *)slot_grid.data(), slot_grid.size() * sizeof(int));
        key.append((const char *)&host_out, sizeof(host_out));
        for (const StreamPlanned &P : plan) {
            key.append((const char *)&P.a, sizeof(StreamArgs));
            key.append((const char *)P.qid.data(), P.qid.size() * sizeof(int));
        }
        if (w.graph_exec && w.graph_key == key) {
            KAIROS_CUDA(cudaGraphLaunch(w.graph_exec, s), "graph launch");
            launched = true;
            ++g->graph_launches;
        } else {
            drop_graph(g);
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const kairos_status est = enqueue();
                const cudaError_t ce = cudaStreamEndCapture(s, &graph);
                if (est == KAIROS_OK && ce == cudaSuccess && graph &&
                    cudaGraphInstantiate(&w.graph_exec, graph, 0) == cudaSuccess) {
                    w.graph_key = key;
                    KAIROS_CUDA(cudaGraphLaunch(w.graph_exec, s), "graph launch");
                    launched = true;
                    ++g->graph_launches;
                }
                if (graph) cudaGraphDestroy(graph);
            }
            cudaGetLastError();
        }
    }
    if (!launched) {
        st = enqueue();
        if (st != KAIROS_OK) return st;
    }
    KAIROS_CUDA(cudaEventRecord(w.ev1, s), "event record");
    KAIROS_CUDA(cudaMemcpyAsync(g->sctrs_host, g->sctrs, plan.size() * sizeof(StreamCtr), cudaMemcpyDeviceToHost, s),
                "stream edge-map counters");
    KAIROS_CUDA(cudaStreamSynchronize(s), "stream edge-map");
    float ms = 0;
    KAIROS_CUDA(cudaEventElapsedTime(&ms, w.ev0, w.ev1), "event time");
    g->last_kernel_ms = ms;
    g->last_launches = (int)plan.size();
    g->last_sctr = g->sctrs_host[plan.size() - 1];
    for (size_t i = 0; i < plan.size(); ++i) {
        const StreamCtr &res = g->sctrs_host[i];
        if (res.err) return stream_error(res);
        if (stats) {
            for (size_t j = 0; j < plan[i].qid.size(); ++j) {
                kairos_query_stats &S = stats[plan[i].qid[j]];
                S.relaxed_edges = res.relaxed[j];
                S.scanned_edges = res.scanned;
                S.rounds = res.blocks + res.fix_rounds;
                S.reached = res.reached[j];
            }
        }
    }
    return KAIROS_OK;
}

}  // namespace

// Shared by the public query calls, the autotuner and the server.  out == nullptr runs the
// queries without writing labels anywhere (timing only).  All launches of the call are
// enqueued back to back (one counter slot each) and read back once; when the outputs are
// device memory and the graph has its own stream, the whole sequence is captured into a
// CUDA graph, which is replayed while the same call repeats.
kairos_status kairos::kairos_run_queries(kairos_graph *g, const kairos_query *qs, int32_t nq, uint32_t *out,
                                 kairos_query_stats *stats, int lanes) {
    if (g->tuning.relax_mode == 3 && lanes >= 32) return run_stream_queries(g, qs, nq, out, stats, lanes);
    lanes = std::min(lanes, MAX_LANES);
    const int64_t n = g->n;
    uint32_t *const host_out = out;  // the caller's pointer (staged copies go there)
    // page-locked host outputs are written directly, like device ones, but never serve as
    // the one-lane label array (its atomics would cross the CPU-GPU link)
    bool pinned = false, dev = true;
    if (out) {
        uint32_t *d = direct_out(out, &pinned);
        dev = d != nullptr;
        if (d) out = d;
    }
    // launches kept in flight together: two (second workspace and stream) when asked for, the
    // outputs are device memory and the call has at least two launches (kernel writes to
    // page-locked host memory stalled the grid barriers of a launch running beside them)
    int64_t n_launch = 0;
    for (int kind = 0; kind < 2; ++kind) {
        int64_t c = 0;
        for (int i = 0; i < nq; ++i) c += qs[i].kind == kind;
        n_launch += (c + lanes - 1) / lanes;
    }
    const int C = (dev && !pinned && g->tuning.concurrent >= 2 && n_launch >= 2) ? 2 : 1;
    kairos_status st = ensure_work(g, lanes, out && !dev && lanes > 1, C == 2);
    if (st != KAIROS_OK) return st;
    auto &w = g->work;
    if (C == 2 && !w.side) {
        KAIROS_CUDA(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking), "concurrent launches: stream");
        KAIROS_CUDA(cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming), "concurrent launches: event");
        KAIROS_CUDA(cudaEventCreateWithFlags(&w.join, cudaEventDisableTiming), "concurrent launches: event");
    }
    g->last_kernel_ms = 0;
    cudaStream_t s = g->stream;

    // plan the launches: queries grouped by kind, `lanes` per launch
    std::vector<Planned> plan;
    std::vector<int> idx;
    for (int kind = 0; kind < 2; ++kind) {
        idx.clear();
        for (int i = 0; i < nq; ++i)
            if (qs[i].kind == kind) idx.push_back(i);
        const Csr &csr = kind == KAIROS_EA ? g->fwd : g->rev;
        for (size_t c = 0; c < idx.size(); c += lanes) {
            const int k = (int)std::min<size_t>(lanes, idx.size() - c);
            LaneParams lp;
            std::memset(&lp, 0, sizeof(lp));
            lp.nlanes = k;
            uint32_t *o = nullptr, *alias = nullptr;
            for (int j = 0; j < k; ++j) lane_set(lp, j, qs[idx[c + j]], j);
            const uint32_t *host_src = nullptr;
            const int slot = (int)(plan.size() % C);
            if (lanes == 1) {
                alias = (out && dev && !pinned) ? out + (int64_t)idx[c] * n : (slot ? w.arr2 : w.arr);
                o = out ? (pinned ? out + (int64_t)idx[c] * n : alias) : nullptr;
                if (out && !dev) host_src = w.arr;
            } else if (out) {
                if (dev) {
                    o = out;
                    for (int j = 0; j < k; ++j) lp.row[j] = idx[c + j];
                } else {
                    o = w.stage;
                    host_src = w.stage;
                }
            }
            Planned P;
            P.a = make_args(g, csr, lp, o, n, alias, stats != nullptr, nullptr, slot);
            P.qid.assign(idx.begin() + c, idx.begin() + c + k);
            P.host_src = host_src;
            plan.push_back(std::move(P));
        }
    }
    if (plan.empty()) return KAIROS_OK;
    st = ensure_ctr_slots(g, plan.size());
    if (st != KAIROS_OK) return st;
    for (size_t i = 0; i < plan.size(); ++i) plan[i].a.ctr = w.ctrs + i;
    int bps = 0;
    int grid = edgemap_max_grid(lanes, g->lam_bits, g->tuning.relax_mode, &bps);
    if (grid <= 0) return fail(KAIROS_ERR_CUDA, "edge-map: no resident launch shape (occupancy query failed)");
    if (g->tuning.blocks_per_sm > 0 && g->tuning.blocks_per_sm < bps) grid = g->tuning.blocks_per_sm * g->sm_count;
    else if (C == 2) grid = std::max(1, bps / 2) * g->sm_count;  // both launches resident at once

    auto enqueue = [&](bool direct) -> kairos_status {
        if (C == 2) {  // fork: the side stream starts after everything before this call
            KAIROS_CUDA(cudaEventRecord(w.fork, s), "concurrent launches: fork");
            KAIROS_CUDA(cudaStreamWaitEvent(w.side, w.fork, 0), "concurrent launches: fork");
        }
        for (size_t i = 0; i < plan.size(); ++i) {
            cudaStream_t si = (C == 2 && (i % 2)) ? w.side : s;
            KAIROS_CUDA(cudaMemsetAsync(plan[i].a.ctr, 0, sizeof(EdgeMapCtr), si), "edge-map counters");
            KAIROS_CUDA(edgemap_launch(plan[i].a, lanes, g->lam_bits, grid, si), "edge-map launch");
            if (direct && plan[i].host_src) {
                const std::vector<int> &q = plan[i].qid;
                for (size_t j = 0; j < q.size(); ++j)
                    KAIROS_CUDA(cudaMemcpyAsync(host_out + (int64_t)q[j] * n, plan[i].host_src + (int64_t)j * n,
                                                (size_t)n * 4, cudaMemcpyDeviceToHost, s),
                                "copy labels to host");
            }
        }
        if (C == 2) {  // join: the call's stream waits for the side stream's launches
            KAIROS_CUDA(cudaEventRecord(w.join, w.side), "concurrent launches: join");
            KAIROS_CUDA(cudaStreamWaitEvent(s, w.join, 0), "concurrent launches: join");
        }
        return KAIROS_OK;
    };

    KAIROS_CUDA(cudaEventRecord(w.ev0, s), "event record");
    const bool capturable = dev && s != nullptr && !getenv("KAIROS_NO_GRAPH");
    bool launched = false;
    if (capturable) {
        // key: everything the captured launches depend on
        std::string key((const char *)&grid, sizeof(grid));
        for (const Planned &P : plan) key.append((const char *)&P.a, sizeof(EdgeMapArgs));
        if (w.graph_exec && w.graph_key == key) {
            KAIROS_CUDA(cudaGraphLaunch(w.graph_exec, s), "graph launch");
            launched = true;
            ++g->graph_launches;
        } else {
            drop_graph(g);
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const kairos_status est = enqueue(false);
                const cudaError_t ce = cudaStreamEndCapture(s, &graph);
                if (est == KAIROS_OK && ce == cudaSuccess && graph &&
                    cudaGraphInstantiate(&w.graph_exec, graph, 0) == cudaSuccess) {
                    w.graph_key = key;
                    KAIROS_CUDA(cudaGraphLaunch(w.graph_exec, s), "graph launch");
                    launched = true;
                    ++g->graph_launches;
                }
                if (graph) cudaGraphDestroy(graph);
            }
            cudaGetLastError();  // a failed capture falls back to direct launches
        }
    }
    if (!launched) {
        st = enqueue(true);
        if (st != KAIROS_OK) return st;
    }
    KAIROS_CUDA(cudaEventRecord(w.ev1, s), "event record");
    KAIROS_CUDA(cudaMemcpyAsync(w.ctrs_host, w.ctrs, plan.size() * sizeof(EdgeMapCtr), cudaMemcpyDeviceToHost, s),
                "edge-map counters");
    KAIROS_CUDA(cudaStreamSynchronize(s), "edge-map");
    float ms = 0;
    KAIROS_CUDA(cudaEventElapsedTime(&ms, w.ev0, w.ev1), "event time");
    g->last_kernel_ms = ms;
    g->last_launches = (int)plan.size();
    std::memcpy(w.ctr_host, &w.ctrs_host[plan.size() - 1], sizeof(EdgeMapCtr));  // last launch, for diagnostics
    for (size_t i = 0; i < plan.size(); ++i) {
        const EdgeMapCtr &res = w.ctrs_host[i];
        if (res.err) return ctr_error(res.err);
        if (stats) {
            for (size_t j = 0; j < plan[i].qid.size(); ++j) {
                kairos_query_stats &S = stats[plan[i].qid[j]];
                S.relaxed_edges = res.relaxed[j];
                S.scanned_edges = res.scanned;
                S.rounds = res.rounds;
                S.reached = res.reached[j];
            }
        }
    }
    return KAIROS_OK;
}

extern "C" {

kairos_status kairos_graph_build(const kairos_edge_list *el, const kairos_graph_opts *opts, kairos_graph **out) {
    TraceRange tr("kairos_graph_build");
    if (!el || !out) return fail(KAIROS_ERR_INVALID_ARG, "graph build: NULL argument");
    const int64_t n = el->n_vertices, m = el->n_edges;
    if (n < 1 || n >= (1LL << 31)) return fail(KAIROS_ERR_INVALID_ARG, "graph build: need 1 <= n_vertices < 2^31");
    if (m < 0 || m >= (1LL << 32)) return fail(KAIROS_ERR_INVALID_ARG, "graph build: need 0 <= n_edges < 2^32");
    if (el->lambda_bits != 16 && el->lambda_bits != 32)
        return fail(KAIROS_ERR_INVALID_ARG, "graph build: lambda_bits must be 16 or 32");
    if (m > 0 && (!el->src || !el->dst || !el->t_dep || !el->lambda))
        return fail(KAIROS_ERR_INVALID_ARG, "graph build: NULL edge array");
    kairos_graph *g = new (std::nothrow) kairos_graph();
    if (!g) return fail(KAIROS_ERR_OOM, "graph build: host allocation failed");
    g->n = n;
    g->m = m;
    g->lam_bits = el->lambda_bits;
    if (opts) {
        g->stream = (cudaStream_t)opts->stream;
        g->A.alloc = opts->alloc;
        g->A.release = opts->free;
        g->A.ctx = opts->alloc_ctx;
        if ((opts->alloc == nullptr) != (opts->free == nullptr)) {
            delete g;
            return fail(KAIROS_ERR_INVALID_ARG, "graph build: alloc and free must be given together");
        }
    }
    const bool want_rev = !(opts && opts->skip_reverse);
    g->tuning.lanes = 1;
    g->tuning.blocks_per_sm = 0;
    g->tuning.warp_max_edges = 128;
    g->tuning.chunk_edges = 512;
    g->tuning.dense_div = 16;
    g->tuning.concurrent = 1;
    auto bail = [&](kairos_status st) {
        kairos_graph_free(g);
        return st;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    g->device = dev;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaEventCreate(&g->work.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&g->work.ev1);
    if (e == cudaSuccess) e = cudaMallocHost(&g->work.ctr_host, sizeof(EdgeMapCtr));
    if (e != cudaSuccess) return bail(cuda_fail(e, "graph build: setup"));

    const size_t lam_sz = el->lambda_bits == 16 ? 2 : 4;
    const int32_t *src = el->src, *dst = el->dst;
    const uint32_t *t = el->t_dep;
    const void *lam = el->lambda;
    void *copies[4] = {nullptr, nullptr, nullptr, nullptr};
    auto drop_copies = [&]() {
        for (void *p : copies) g->A.put(p);
    };
    cudaStream_t s = g->stream;
    if (!el->on_device && m > 0) {
        const size_t sz[4] = {(size_t)m * 4, (size_t)m * 4, (size_t)m * 4, (size_t)m * lam_sz};
        const void *hs[4] = {el->src, el->dst, el->t_dep, el->lambda};
        for (int i = 0; i < 4; ++i) {
            copies[i] = g->A.get(sz[i]);
            if (!copies[i]) {
                drop_copies();
                return bail(fail(KAIROS_ERR_OOM, "graph build: device allocation failed"));
            }
            e = cudaMemcpyAsync(copies[i], hs[i], sz[i], cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                drop_copies();
                return bail(cuda_fail(e, "graph build: copy edges to device"));
            }
        }
        src = (const int32_t *)copies[0];
        dst = (const int32_t *)copies[1];
        t = (const uint32_t *)copies[2];
        lam = copies[3];
    }
    auto t0 = std::chrono::steady_clock::now();
    int flags = 0;
    kairos_status st = validate_edges(s, n, m, src, dst, t, lam, el->lambda_bits, &flags, g->A);
    if (st == KAIROS_OK && (flags & 1)) st = fail(KAIROS_ERR_INVALID_ARG, "graph build: vertex id out of range");
    if (st == KAIROS_OK && (flags & 2)) st = fail(KAIROS_ERR_OVERFLOW, "graph build: t + lambda exceeds KAIROS_TIME_MAX");
    if (st == KAIROS_OK) st = build_csr(g->A, s, n, m, src, dst, t, lam, el->lambda_bits, 0, &g->fwd);
    if (st == KAIROS_OK && want_rev) {
        st = build_csr(g->A, s, n, m, src, dst, t, lam, el->lambda_bits, 1, &g->rev);
        if (st == KAIROS_OK) g->has_rev = 1;
    }
    drop_copies();
    if (st != KAIROS_OK) return bail(st);
    g->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = g;
    return KAIROS_OK;
}

kairos_status kairos_index_build(kairos_graph *g, uint32_t threshold) {
    TraceRange tr("kairos_index_build");
    if (!g) return fail(KAIROS_ERR_INVALID_ARG, "index build: NULL graph");
    std::lock_guard<std::mutex> lk(g->mu);
    if (threshold == 0) threshold = 1;
    auto t0 = std::chrono::steady_clock::now();
    kairos_status st = build_index(g->A, g->stream, g->n, threshold, &g->fwd);
    if (st == KAIROS_OK && g->has_rev) st = build_index(g->A, g->stream, g->n, threshold, &g->rev);
    if (st != KAIROS_OK) {
        free_index(g->A, &g->fwd);
        free_index(g->A, &g->rev);
        g->theta = KAIROS_NO_INDEX;
        return st;
    }
    g->theta = threshold;
    g->index_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return KAIROS_OK;
}

void kairos_graph_free(kairos_graph *g) {
    if (!g) return;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        cudaStreamSynchronize(g->stream);
        cudaGetLastError();
        release_work_arrays(g);
        release_stream_work(g);
        for (int k = 0; k < 3; ++k) {
            if (g->sside[k]) cudaStreamDestroy(g->sside[k]);
            if (g->sjoin[k]) cudaEventDestroy(g->sjoin[k]);
        }
        if (g->sfork) cudaEventDestroy(g->sfork);
        free_time_stream(g->A, &g->ts_fwd);
        free_time_stream(g->A, &g->ts_rev);
        g->A.put(g->sctrs);
        if (g->sctrs_host) cudaFreeHost(g->sctrs_host);
        release_fastest_scratch(g);
        release_duration_scratch(g);
        free_csr(g->A, &g->fwd);
        free_csr(g->A, &g->rev);
        if (g->work.ctr_host) cudaFreeHost(g->work.ctr_host);
        g->A.put(g->work.ctrs);
        if (g->work.ctrs_host) cudaFreeHost(g->work.ctrs_host);
        if (g->work.graph_exec) cudaGraphExecDestroy(g->work.graph_exec);
        if (g->work.side) cudaStreamDestroy(g->work.side);
        if (g->work.fork) cudaEventDestroy(g->work.fork);
        if (g->work.join) cudaEventDestroy(g->work.join);
        if (g->work.ev0) cudaEventDestroy(g->work.ev0);
        if (g->work.ev1) cudaEventDestroy(g->work.ev1);
        cudaGetLastError();
    }
    delete g;
}

kairos_status kairos_graph_get_info(const kairos_graph *g, kairos_graph_info *info) {
    if (!g || !info) return fail(KAIROS_ERR_INVALID_ARG, "graph info: NULL argument");
    info->n_vertices = g->n;
    info->n_edges = g->m;
    info->lambda_bits = g->lam_bits;
    info->index_threshold = g->theta;
    info->indexed_vertices = g->fwd.indexed;
    const int64_t per_dir = (g->n + 1) * 8 + g->m * (8 + (g->lam_bits == 16 ? 2 : 4));
    info->device_bytes = per_dir * (g->has_rev ? 2 : 1) + (g->fwd.n_fence + g->rev.n_fence) * 4 +
                         (g->fwd.fidx ? g->n * 4 : 0) + (g->rev.fidx ? g->n * 4 : 0) + (int64_t)g->work.bytes +
                         (g->ts_fwd.rec ? g->m * 16 : 0) + (g->ts_rev.rec ? g->m * 16 : 0) +
                         (g->ts_fwd.span ? g->n * 8 : 0) + (g->ts_rev.span ? g->n * 8 : 0) + (int64_t)g->sw[0].bytes +
                         (int64_t)g->sw[1].bytes;
    info->build_ms = g->build_ms;
    info->index_ms = g->index_ms;
    info->graph_launches = g->graph_launches;
    return KAIROS_OK;
}

kairos_status kairos_batch_query(kairos_graph *g, const kairos_query *qs, int32_t n, uint32_t *out,
                                 kairos_query_stats *stats) {
    if (!g || (n > 0 && (!qs || !out)) || n < 0) return fail(KAIROS_ERR_INVALID_ARG, "batch query: bad argument");
    for (int i = 0; i < n; ++i) {
        kairos_status st = check_query(g, qs[i]);
        if (st != KAIROS_OK) return st;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    TraceRange tr("kairos_batch_query");
    return kairos_run_queries(g, qs, n, out, stats, g->tuning.lanes);
}

static kairos_status single(kairos_graph *g, int kind, int32_t v, uint32_t ta, uint32_t tw, uint32_t *out) {
    if (!g || !out) return fail(KAIROS_ERR_INVALID_ARG, "query: NULL argument");
    kairos_query q;
    std::memset(&q, 0, sizeof(q));
    q.vertex = v;
    q.ta = ta;
    q.tw = tw;
    q.kind = (uint8_t)kind;
    kairos_status st = check_query(g, q);
    if (st != KAIROS_OK) return st;
    std::lock_guard<std::mutex> lk(g->mu);
    TraceRange tr(kind == KAIROS_EA ? "kairos_earliest_arrival" : "kairos_latest_departure");
    return kairos_run_queries(g, &q, 1, out, nullptr, 1);
}

kairos_status kairos_earliest_arrival(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, uint32_t *out) {
    return single(g, KAIROS_EA, src, ta, tw, out);
}

kairos_status kairos_latest_departure(kairos_graph *g, int32_t dst, uint32_t ta, uint32_t tw, uint32_t *out) {
    return single(g, KAIROS_LD, dst, ta, tw, out);
}

kairos_status kairos_get_tuning(const kairos_graph *g, kairos_tuning *t) {
    if (!g || !t) return fail(KAIROS_ERR_INVALID_ARG, "get tuning: NULL argument");
    *t = g->tuning;
    return KAIROS_OK;
}

kairos_status kairos_set_tuning(kairos_graph *g, const kairos_tuning *t) {
    if (!g || !t) return fail(KAIROS_ERR_INVALID_ARG, "set tuning: NULL argument");
    const int L = t->lanes;
    if (!(L == 1 || L == 2 || L == 4 || L == 8 || L == 16 || L == 32 || L == 64))
        return fail(KAIROS_ERR_INVALID_ARG, "tuning: lanes must be 1, 2, 4, 8, 16, 32 or 64");
    if (L == 64 && t->relax_mode != 3) return fail(KAIROS_ERR_INVALID_ARG, "tuning: 64 lanes need relax_mode 3");
    if (t->relax_mode == 3 && L < 32) return fail(KAIROS_ERR_INVALID_ARG, "tuning: relax_mode 3 needs 32 or 64 lanes");
    if (t->block_edges < 0) return fail(KAIROS_ERR_INVALID_ARG, "tuning: block_edges >= 0");
    if (t->select_permille < 0 || t->select_permille > 1000)
        return fail(KAIROS_ERR_INVALID_ARG, "tuning: select_permille in [0, 1000]");
    if (t->blocks_per_sm < 0 || t->blocks_per_sm > 32) return fail(KAIROS_ERR_INVALID_ARG, "tuning: blocks_per_sm in [0, 32]");
    if (t->warp_max_edges < 32 || t->warp_max_edges > (1 << 16))
        return fail(KAIROS_ERR_INVALID_ARG, "tuning: warp_max_edges in [32, 65536]");
    if (t->chunk_edges < 32 || t->chunk_edges % 32 || t->chunk_edges > (1 << 24))
        return fail(KAIROS_ERR_INVALID_ARG, "tuning: chunk_edges a multiple of 32 in [32, 2^24]");
    if (t->dense_div < 0) return fail(KAIROS_ERR_INVALID_ARG, "tuning: dense_div >= 0");
    if (t->relax_mode < 0 || t->relax_mode > 3) return fail(KAIROS_ERR_INVALID_ARG, "tuning: relax_mode is 0, 1, 2 or 3");
    if (t->concurrent < 0 || t->concurrent > 4 || t->concurrent == 3 || (t->concurrent == 4 && t->relax_mode != 3))
        return fail(KAIROS_ERR_INVALID_ARG, "tuning: concurrent is 0, 1, 2, or 4 with relax_mode 3");
    std::lock_guard<std::mutex> lk(g->mu);
    g->tuning = *t;
    return KAIROS_OK;
}

kairos_status kairos_autotune(kairos_graph *g, const kairos_query *sample, int32_t n, kairos_tuning *best) {
    return kairos_autotune_from(g, sample, n, 1, best);
}

kairos_status kairos_autotune_from(kairos_graph *g, const kairos_query *sample, int32_t n, int32_t min_lanes,
                                   kairos_tuning *best) {
    if (!g || !sample || n <= 0 || min_lanes < 1) return fail(KAIROS_ERR_INVALID_ARG, "autotune: bad argument");
    for (int i = 0; i < n; ++i) {
        kairos_status st = check_query(g, sample[i]);
        if (st != KAIROS_OK) return st;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    const kairos_tuning base = g->tuning;
    kairos_tuning win = base;
    double win_ms = -1;
    const int lanes_set[] = {1, 2, 4, 8, 16, 32};
    const int wmax_set[] = {32, 128, 512};
    // {dense_div, relax_mode}: queue or bitmap frontier; all-segment, candidate-pass or
    // unconditional relaxation
    const int shape_set[][2] = {{0, 0}, {16, 0}, {0, 2}, {16, 2}, {0, 1}};
    for (int L : lanes_set) {
        if (L < min_lanes) continue;
        for (int wm : wmax_set) {
            for (const auto &sh : shape_set) {
                if (L == 1 && sh[1] == 2) continue;  // one lane: the two checked modes coincide
                kairos_tuning c = base;
                c.lanes = L;
                c.warp_max_edges = wm;
                c.dense_div = sh[0];
                c.relax_mode = sh[1];
                g->tuning = c;
                kairos_status st = kairos_run_queries(g, sample, n, nullptr, nullptr, L);
                if (st == KAIROS_ERR_OOM) continue;  // this lane width does not fit: skip it
                if (st != KAIROS_OK) {
                    g->tuning = base;
                    return st;
                }
                const double ms = g->last_kernel_ms;
                if (win_ms < 0 || ms < win_ms) {
                    win_ms = ms;
                    win = c;
                }
            }
        }
    }
    // the time-ordered mode at 32 and 64 lanes, one or two launches in flight, three block sizes
    for (int L : {32, 64}) {
        for (int cc : {1, 2, 4}) {
            for (int div : {512, 2048, 8192}) {
                kairos_tuning c = base;
                c.lanes = L;
                c.relax_mode = 3;
                c.concurrent = cc;
                c.blocks_per_sm = 0;
                c.block_edges = (int32_t)std::min<int64_t>(std::max<int64_t>(g->m / div, 4096), 1 << 30);
                g->tuning = c;
                kairos_status st = kairos_run_queries(g, sample, n, nullptr, nullptr, L);
                if (st == KAIROS_ERR_OOM) continue;
                if (st != KAIROS_OK) {
                    g->tuning = base;
                    return st;
                }
                if (win_ms < 0 || g->last_kernel_ms < win_ms) {
                    win_ms = g->last_kernel_ms;
                    win = c;
                }
            }
        }
    }
    if (win_ms < 0) {
        g->tuning = base;
        return fail(KAIROS_ERR_OOM, "autotune: no launch shape fits in device memory");
    }
    if (win.relax_mode == 3) {  // the frontier-mode refinements below do not apply
        g->tuning = win;
        if (best) *best = win;
        return KAIROS_OK;
    }
    // coordinate descent on the winner: chunk size, then resident blocks per SM
    auto try_shape = [&](const kairos_tuning &c) -> kairos_status {
        g->tuning = c;
        kairos_status st = kairos_run_queries(g, sample, n, nullptr, nullptr, c.lanes);
        if (st == KAIROS_ERR_OOM) return KAIROS_OK;
        if (st != KAIROS_OK) return st;
        if (g->last_kernel_ms < win_ms) {
            win_ms = g->last_kernel_ms;
            win = c;
        }
        return KAIROS_OK;
    };
    for (int ch : {256, 1024, 2048}) {
        kairos_tuning c = win;
        c.chunk_edges = ch;
        kairos_status st = try_shape(c);
        if (st != KAIROS_OK) {
            g->tuning = base;
            return st;
        }
    }
    int bps = 0;
    edgemap_max_grid(win.lanes, g->lam_bits, win.relax_mode, &bps);
    for (int b = 1; b < bps; ++b) {
        kairos_tuning c = win;
        c.blocks_per_sm = b;
        kairos_status st = try_shape(c);
        if (st != KAIROS_OK) {
            g->tuning = base;
            return st;
        }
    }
    if (win.concurrent < 2) {  // two launches in flight, half the resident blocks each
        kairos_tuning c = win;
        c.concurrent = 2;
        c.blocks_per_sm = 0;
        kairos_status st = try_shape(c);
        if (st != KAIROS_OK) {
            g->tuning = base;
            return st;
        }
    }
    g->tuning = win;
    if (best) *best = win;
    return KAIROS_OK;
}

kairos_status kairos_autotune_index(kairos_graph *g, const kairos_query *sample, int32_t n, const uint32_t *thetas,
                                    int32_t n_thetas, uint32_t *best, double *ms_out) {
    if (!g || !sample || n <= 0 || !thetas || n_thetas <= 0) return fail(KAIROS_ERR_INVALID_ARG, "autotune index: bad argument");
    for (int i = 0; i < n; ++i) {
        kairos_status st = check_query(g, sample[i]);
        if (st != KAIROS_OK) return st;
    }
    uint32_t win = KAIROS_NO_INDEX;
    double win_ms = -1;
    for (int k = 0; k < n_thetas; ++k) {
        kairos_status st = kairos_index_build(g, thetas[k]);
        if (st != KAIROS_OK) return st;
        std::lock_guard<std::mutex> lk(g->mu);
        st = kairos_run_queries(g, sample, n, nullptr, nullptr, g->tuning.lanes);
        if (st != KAIROS_OK) return st;
        const double ms = g->last_kernel_ms;
        if (ms_out) ms_out[k] = ms;
        if (win_ms < 0 || ms < win_ms) {
            win_ms = ms;
            win = thetas[k];
        }
    }
    kairos_status st = kairos_index_build(g, win);
    if (st != KAIROS_OK) return st;
    if (best) *best = win;
    return KAIROS_OK;
}

const char *kairos_last_error(void) { return g_err.c_str(); }

const char *kairos_status_string(kairos_status s) {
    switch (s) {
        case KAIROS_OK: return "KAIROS_OK";
        case KAIROS_ERR_INVALID_ARG: return "KAIROS_ERR_INVALID_ARG";
        case KAIROS_ERR_OOM: return "KAIROS_ERR_OOM";
        case KAIROS_ERR_CUDA: return "KAIROS_ERR_CUDA";
        case KAIROS_ERR_OVERFLOW: return "KAIROS_ERR_OVERFLOW";
        case KAIROS_ERR_NOT_READY: return "KAIROS_ERR_NOT_READY";
        case KAIROS_ERR_BUSY: return "KAIROS_ERR_BUSY";
        case KAIROS_ERR_TIMEOUT: return "KAIROS_ERR_TIMEOUT";
        case KAIROS_ERR_INTERNAL: return "KAIROS_ERR_INTERNAL";
    }
    return "unknown kairos_status";
}

double kairos_last_kernel_ms(const kairos_graph *g) { return g ? g->last_kernel_ms : 0.0; }

int32_t kairos_last_round_profile(const kairos_graph *g, int32_t max_rounds, uint32_t *frontier, uint32_t *chunks,
                                  double *ms) {
    if (!g || max_rounds < 0 || !g->work.ctr_host) return 0;
    const EdgeMapCtr &c = *g->work.ctr_host;
    const int r = (int)std::min<unsigned>(c.rounds, (unsigned)std::min(max_rounds, PROFILE_ROUNDS));
    for (int i = 0; i < r; ++i) {
        if (frontier) frontier[i] = c.round_frontier[i];
        if (chunks) chunks[i] = c.round_chunks[i];
        if (ms) ms[i] = (double)(c.round_ns[i + 1] - c.round_ns[i]) * 1e-6;
    }
    return r;
}

int32_t kairos_last_stream_profile(const kairos_graph *g, uint64_t *out23) {
    if (!g || !out23) return 0;
    const StreamCtr &c = g->last_sctr;
    const uint64_t v[23] = {c.blocks, c.fix_rounds, c.fix_vertices, c.fix_edges, c.cand, c.scanned,
                            c.phase_cycles[0], c.phase_cycles[1], c.phase_cycles[2], c.phase_cycles[3],
                            c.cand_lanes[0], c.cand_lanes[1], c.cand_lanes[2], c.cand_lanes[3], c.cand_pairs,
                            c.cand_improving, c.lanes_lowered, c.wall_ns[0], c.wall_ns[1], c.wall_ns[2],
                            c.segments[0], c.segments[1], c.segments[2]};
    for (int i = 0; i < 23; ++i) out23[i] = v[i];
    return 23;
}

int32_t kairos_last_phase_cycles(const kairos_graph *g, uint64_t *cycles8) {
    if (!g || !cycles8 || !g->work.ctr_host) return 0;
    for (int i = 0; i < 8; ++i) cycles8[i] = g->work.ctr_host->phase_cycles[i];
    return 8;
}

}  // extern "C"
