// Shortest durations (least total travel time; the "shortest path" among the minimal temporal
// paths of Sec. 2.3) and temporal BFS (least number of edges; Table 4's T. BFS read over
// time-respecting paths) as one label-correcting computation over edge labels.
//
// For a usable edge e = (u, v, t, lam) let D(e) be the least total duration of a
// time-respecting path from the source that ends with e, and let
//     f_u(tau) = min { D(e') : e' enters u and arrives by tau (before tau under
//                      StrictlySucceeds) },   f_src = 0 for every departure in the window.
// Then D(e) = lam + f_u(t) and the answer at v != src is the minimum D over v's in-edges.
// Every round relaxes the out-edges of the vertices whose f changed, and then recomputes
// f for the heads whose in-edge labels dropped.  f_u is a suffix minimum over u's in-edges
// in the reversed graph's order (latest arrival first); the slot from which the in-edges
// arrive in time for an out-edge depends only on the graph, so it is found once per graph
// (a binary search over the reversed list's mirrored times) and kept.  Labels only fall,
// and after k rounds every path of k edges is accounted for; simple paths suffice, so at
// most n rounds.
// Work per round follows the changes: when an in-edge label of u drops, f_u changes only from
// that edge's arrival on, so u's next relaxation starts at the first out-edge departing then
// (its list is in departure order); and u's suffix minima are recomputed only from the
// highest slot whose label dropped down to the start of its list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "trace.h"

namespace kairos {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int64_t SD_LONG = 2048;  // in-list stretches longer than this get a whole block

// from_cur[v]: earliest arrival whose label dropped, for v's coming relaxation; from_next[v]:
// the same, collected during a relaxation round; hislot[v]: 1 + the highest slot of v's in-list
// whose label dropped (0: none).
__global__ void sd_init_kernel(int64_t m, int64_t n, uint32_t *d, uint32_t *sm, uint8_t *changed, uint8_t *active,
                               uint32_t *from_cur, uint32_t *from_next, uint32_t *hislot, int32_t src) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        d[i] = INF;
        sm[i] = INF;
    }
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        changed[v] = 0;
        active[v] = (v == src);
        from_cur[v] = (v == src) ? 0u : INF;  // the source starts paths at every departure
        from_next[v] = INF;
        hislot[v] = 0;
    }
}

constexpr uint32_t SD_NONE = 0xFFFFFFFFu;
constexpr int SD_CHUNK = 256;  // out-edges per relaxation work item

struct SdChunk {
    uint64_t begin;  // first forward edge
    int32_t u;       // its tail
    uint32_t len;    // edges (<= SD_CHUNK)
};

// pred[i] = the first slot of u's in-list (latest arrival first) whose edge arrives by t_i
// (before t_i under StrictlySucceeds), SD_NONE if none: a property of the graph, computed once
// per predicate.  f_u(t_i) is then the suffix minimum at that slot.
__global__ void sd_pred_kernel(int64_t n, int64_t m, const uint64_t *__restrict__ off, const uint32_t *__restrict__ t,
                               const uint64_t *__restrict__ roff, const uint32_t *__restrict__ rt, int strict,
                               uint32_t *pred) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;  // the tail: last u with off[u] <= i
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= (uint64_t)i) lo = mid; else hi = mid;
        }
        const uint64_t r0 = roff[lo], r1 = roff[lo + 1];
        const uint32_t key = TMAX - t[i];  // in-edges arriving by t: mirrored time >= key (> when strict)
        uint64_t a = r0, b = r1;
        while (a < b) {
            const uint64_t mid = (a + b) >> 1;
            const bool below = strict ? (rt[mid] <= key) : (rt[mid] < key);
            if (below) a = mid + 1; else b = mid;
        }
        pred[i] = a < r1 ? (uint32_t)a : SD_NONE;
    }
}

// Every active vertex u registers the out-edges its changed f_u can improve: those departing
// at or after the earliest dropped arrival (after it under StrictlySucceeds; the source: all),
// as SD_CHUNK-edge work items (one counter atomic per warp).
__global__ void sd_register_kernel(int64_t n, const uint64_t *__restrict__ off, const uint32_t *__restrict__ t,
                                   uint8_t *active, const uint32_t *__restrict__ from_cur, int32_t src, int strict,
                                   SdChunk *chunks, unsigned *chunk_count) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t u = base + threadIdx.x;
        uint64_t e0 = 0, e1 = 0;
        if (u < n && active[u]) {
            active[u] = 0;
            e0 = off[u];
            e1 = off[u + 1];
            if (u != src) {
                const uint32_t from = from_cur[u];
                uint64_t hi = e1;
                while (e0 < hi) {
                    const uint64_t mid = (e0 + hi) >> 1;
                    const bool before = strict ? (t[mid] <= from) : (t[mid] < from);
                    if (before) e0 = mid + 1; else hi = mid;
                }
            }
        }
        const uint32_t nch = e1 > e0 ? (uint32_t)((e1 - e0 + SD_CHUNK - 1) / SD_CHUNK) : 0u;
        uint32_t incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        unsigned c0 = 0;
        if (lane == 31 && total) c0 = atomicAdd(chunk_count, total);
        c0 = __shfl_sync(FULL, c0, 31) + incl - nch;
        for (uint32_t c = 0; c < nch; ++c) {
            SdChunk ch;
            ch.begin = e0 + (uint64_t)c * SD_CHUNK;
            ch.u = (int32_t)u;
            ch.len = (uint32_t)min((uint64_t)SD_CHUNK, e1 - ch.begin);
            chunks[c0 + c] = ch;
        }
    }
}

// Relax the registered out-edges: D(e) = min(D(e), lam + f_u(t)), f_u(t) = sm[pred[e]] (0 for
// the source).  A warp takes one chunk at a time.  ctr[0]: set when some label dropped;
// ctr[1]: edges examined.
template <typename LamT>
__global__ void sd_relax_kernel(const SdChunk *__restrict__ chunks, const unsigned *__restrict__ chunk_count,
                                const int32_t *__restrict__ dst, const uint32_t *__restrict__ t,
                                const LamT *__restrict__ lam, const uint32_t *__restrict__ pred,
                                const uint32_t *__restrict__ slot, uint32_t *d, const uint32_t *__restrict__ sm,
                                uint8_t *changed, uint32_t *from_next, uint32_t *hislot, int32_t src, uint32_t ta,
                                uint32_t tw, int unit, unsigned long long *ctr) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned count = *chunk_count;
    unsigned long long examined = 0;
    bool dropped = false;
    for (int64_t c = warp; c < (int64_t)count; c += nwarps) {
        const SdChunk ch = chunks[c];
        for (uint32_t k = lane; k < ch.len; k += 32) {
            const uint64_t i = ch.begin + k;
            const uint32_t ti = t[i];
            const uint32_t li = (uint32_t)lam[i];
            if (ti < ta || (uint64_t)ti + li > tw) continue;
            ++examined;
            uint32_t b = 0;
            if (ch.u != src) {
                const uint32_t p = pred[i];
                b = p != SD_NONE ? sm[p] : INF;
            }
            if (b == INF) continue;
            // a path's total duration (at most tw - ta) or its number of edges (at most n - 1)
            const uint32_t cand = b + (unit ? 1u : li);
            const uint32_t j = slot[i];
            if (cand < d[j]) {  // the label may be stale (never below the current one)
                const int32_t v = dst[i];
                atomicMin(&d[j], cand);
                atomicMin(&from_next[v], ti + li);
                atomicMax(&hislot[v], j + 1u);
                changed[v] = 1;
                dropped = true;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) examined += __shfl_xor_sync(FULL, examined, o);
    const bool any = __any_sync(FULL, dropped);
    if (lane == 0) {
        if (examined) atomicAdd(&ctr[1], examined);
        if (any) atomicExch(&ctr[0], 1ull);
    }
}

// Recompute the suffix minima of the in-edge labels of every changed vertex (latest arrival
// first, so the suffix from a slot covers the in-edges arriving no later); it becomes active.
__global__ void sd_suffix_kernel(int64_t n, const uint64_t *__restrict__ roff, const uint32_t *d, uint32_t *sm,
                                 uint8_t *changed, uint8_t *active, uint32_t *from_cur, uint32_t *from_next,
                                 uint32_t *hislot, uint32_t *long_v, uint32_t *long_top, unsigned *long_count) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const int64_t v0 = base + lane;
        const bool on = v0 < n && changed[v0];
        unsigned todo = __ballot_sync(FULL, on);
        uint32_t top = 0;
        if (on) {
            changed[v0] = 0;
            active[v0] = 1;
            from_cur[v0] = from_next[v0];
            from_next[v0] = INF;
            top = hislot[v0];
            hislot[v0] = 0;
        }
        while (todo) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t v = base + k;
            const int64_t b = (int64_t)roff[v];
            // slots above the highest dropped one keep their labels and suffix minima
            const int64_t e = (int64_t)__shfl_sync(FULL, top, k);
            if (e - b > SD_LONG) {  // a long stretch: recomputed by sd_suffix_long_kernel
                if (lane == 0) {
                    const unsigned q = atomicAdd(long_count, 1u);
                    long_v[q] = (uint32_t)v;
                    long_top[q] = (uint32_t)(e - b);
                }
                continue;
            }
            uint32_t carry = (e < (int64_t)roff[v + 1]) ? sm[e] : INF;
            for (int64_t cb = e; cb > b; cb -= 32) {
                const int64_t j = cb - 32 + lane;
                uint32_t x = j >= b ? d[j] : INF;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_down_sync(FULL, x, o);
                    if (lane + o < 32) x = min(x, y);
                }
                x = min(x, carry);
                if (j >= b) sm[j] = x;
                carry = __shfl_sync(FULL, x, 0);
            }
        }
    }
}

// Suffix minima of the long stretches listed by sd_suffix_kernel, one block per stretch, 256
// slots per step: warp suffix scans, then the warps' minima combined through shared memory.
__global__ void __launch_bounds__(256) sd_suffix_long_kernel(const uint64_t *__restrict__ roff, const uint32_t *d,
                                                             uint32_t *sm, const uint32_t *long_v,
                                                             const uint32_t *long_top, const unsigned *long_count) {
    __shared__ uint32_t wmin[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned count = *long_count;
    for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
        const int64_t v = long_v[q];
        const int64_t b = (int64_t)roff[v], e = b + (int64_t)long_top[q];
        uint32_t carry = (e < (int64_t)roff[v + 1]) ? sm[e] : INF;
        for (int64_t cb = e; cb > b; cb -= 256) {
            const int64_t j = cb - 256 + threadIdx.x;
            uint32_t x = j >= b ? d[j] : INF;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_down_sync(FULL, x, o);
                if (lane + o < 32) x = min(x, y);
            }
            if (lane == 0) wmin[wid] = x;  // the minimum of this warp's 32 slots
            __syncthreads();
            uint32_t later = carry;  // slots after this warp's: later warps of the step, then carry
            for (int w2 = wid + 1; w2 < 8; ++w2) later = min(later, wmin[w2]);
            x = min(x, later);
            if (j >= b) sm[j] = x;
            uint32_t all = carry;
            for (int w2 = 0; w2 < 8; ++w2) all = min(all, wmin[w2]);
            carry = all;
            __syncthreads();  // wmin is rewritten by the next step
        }
    }
}

__global__ void sd_result_kernel(int64_t n, const uint64_t *__restrict__ roff, const uint32_t *__restrict__ sm,
                                 int32_t src, uint32_t *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = (v == src) ? 0u : (roff[v] < roff[v + 1] ? sm[roff[v]] : INF);
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

kairos_status ensure_duration_state(kairos_graph *g) {
    auto &w = g->work;
    if (w.sd_slot) return KAIROS_OK;
    const int64_t n = g->n, m = std::max<int64_t>(g->m, 1);
    const auto &A = g->A;
    w.sd_slot = (uint32_t *)A.get((size_t)m * 4);
    w.sd_d = (uint32_t *)A.get((size_t)m * 4);
    w.sd_sm = (uint32_t *)A.get((size_t)m * 4);
    w.sd_changed = (uint8_t *)A.get((size_t)n);
    w.sd_active = (uint8_t *)A.get((size_t)n);
    w.sd_from = (uint32_t *)A.get((size_t)n * 5 * 4 + 16);  // from_cur, from_next, hislot, long list, counters
    // work items: every active vertex's registered range in SD_CHUNK pieces
    w.sd_chunks = A.get(((size_t)m / SD_CHUNK + (size_t)n + 1) * sizeof(SdChunk));
    w.sd_ctr = (unsigned long long *)A.get(2 * sizeof(unsigned long long));
    cudaError_t e = cudaMallocHost(&w.sd_ctr_host, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        w.sd_ctr_host = nullptr;
    }
    if (!w.sd_slot || !w.sd_d || !w.sd_sm || !w.sd_changed || !w.sd_active || !w.sd_from || !w.sd_chunks ||
        !w.sd_ctr || !w.sd_ctr_host) {
        release_duration_scratch(g);
        return fail(KAIROS_ERR_OOM, "shortest duration: device allocation failed");
    }
    kairos_status st = build_reverse_slots(A, g->stream, n, g->m, g->fwd, g->lam_bits, w.sd_slot);
    if (st != KAIROS_OK) release_duration_scratch(g);
    return st;
}

// The in-time slot of every edge under one predicate (computed on first use).
kairos_status ensure_pred(kairos_graph *g, int strict) {
    auto &w = g->work;
    if (w.sd_pred[strict]) return KAIROS_OK;
    const int64_t n = g->n, m = g->m;
    w.sd_pred[strict] = (uint32_t *)g->A.get((size_t)std::max<int64_t>(m, 1) * 4);
    if (!w.sd_pred[strict]) return fail(KAIROS_ERR_OOM, "shortest duration: device allocation failed");
    if (m > 0) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)g->sm_count * 16));
        sd_pred_kernel<<<grid, 256, 0, g->stream>>>(n, m, g->fwd.off, g->fwd.t, g->rev.off, g->rev.t, strict,
                                                    w.sd_pred[strict]);
        KAIROS_CUDA(cudaGetLastError(), "shortest duration: in-time slots");
    }
    return KAIROS_OK;
}

}  // namespace

void release_duration_scratch(kairos_graph *g) {
    auto &w = g->work;
    const auto &A = g->A;
    A.put(w.sd_slot);
    A.put(w.sd_d);
    A.put(w.sd_sm);
    A.put(w.sd_changed);
    A.put(w.sd_active);
    A.put(w.sd_from);
    A.put(w.sd_pred[0]);
    A.put(w.sd_pred[1]);
    A.put(w.sd_chunks);
    A.put(w.sd_ctr);
    if (w.sd_ctr_host) cudaFreeHost(w.sd_ctr_host);
    w.sd_slot = w.sd_d = w.sd_sm = nullptr;
    w.sd_changed = w.sd_active = nullptr;
    w.sd_from = nullptr;
    w.sd_pred[0] = w.sd_pred[1] = nullptr;
    w.sd_chunks = nullptr;
    w.sd_ctr = w.sd_ctr_host = nullptr;
}

}  // namespace kairos

using namespace kairos;

// Least total cost from src: the durations (unit = 0, shortest durations) or one per edge
// (unit = 1, temporal BFS).
static kairos_status least_cost(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, int32_t strict, int unit,
                                uint32_t *out, kairos_duration_stats *stats) {
    if (!g || !out) return fail(KAIROS_ERR_INVALID_ARG, "shortest duration: NULL argument");
    if (src < 0 || (int64_t)src >= g->n) return fail(KAIROS_ERR_INVALID_ARG, "shortest duration: source out of range");
    if (ta > tw || tw > TMAX) return fail(KAIROS_ERR_INVALID_ARG, "shortest duration: need ta <= tw <= KAIROS_TIME_MAX");
    if (strict != 0 && strict != 1) return fail(KAIROS_ERR_INVALID_ARG, "shortest duration: strict is 0 or 1");
    if (!g->has_rev)
        return fail(KAIROS_ERR_INVALID_ARG, "shortest duration: the graph was built without its reverse (skip_reverse)");
    std::lock_guard<std::mutex> lk(g->mu);
    TraceRange tr(unit ? "kairos_temporal_bfs" : "kairos_shortest_duration");
    kairos_status st = ensure_duration_state(g);
    if (st == KAIROS_OK) st = ensure_pred(g, strict);
    if (st != KAIROS_OK) return st;
    auto &w = g->work;
    cudaStream_t s = g->stream;
    const int64_t n = g->n, m = g->m;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(n, m) + 255) / 256, (int64_t)g->sm_count * 16));
    const int vgrid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g->sm_count * 16));
    KAIROS_CUDA(cudaEventRecord(w.ev0, s), "event record");
    uint32_t *from_cur = w.sd_from, *from_next = w.sd_from + n, *hislot = w.sd_from + 2 * n;
    uint32_t *long_v = w.sd_from + 3 * n, *long_top = w.sd_from + 4 * n;
    unsigned *long_count = (unsigned *)(w.sd_from + 5 * n);
    unsigned *chunk_count = long_count + 1;
    SdChunk *chunks = (SdChunk *)w.sd_chunks;
    const uint32_t *pred = w.sd_pred[strict];
    const int rgrid = g->sm_count * 8;  // relaxation: 8 warps per block, a chunk per warp at a time
    sd_init_kernel<<<grid, 256, 0, s>>>(m, n, w.sd_d, w.sd_sm, w.sd_changed, w.sd_active, from_cur, from_next,
                                        hislot, src);
    KAIROS_CUDA(cudaGetLastError(), "shortest duration: init");
    KAIROS_CUDA(cudaMemsetAsync(w.sd_ctr, 0, 2 * sizeof(unsigned long long), s), "shortest duration: counters");
    uint64_t rounds = 0;
    const uint64_t cap = (uint64_t)n + 1;
    for (;;) {
        if (rounds >= cap) return fail(KAIROS_ERR_TIMEOUT, "shortest duration: round cap (n + 1) reached");
        ++rounds;
        KAIROS_CUDA(cudaMemsetAsync(w.sd_ctr, 0, sizeof(unsigned long long), s), "shortest duration: flag");
        KAIROS_CUDA(cudaMemsetAsync(chunk_count, 0, sizeof(unsigned), s), "shortest duration: work items");
        sd_register_kernel<<<vgrid, 256, 0, s>>>(n, g->fwd.off, g->fwd.t, w.sd_active, from_cur, src, strict, chunks,
                                                 chunk_count);
        KAIROS_CUDA(cudaGetLastError(), "shortest duration: register");
        if (g->lam_bits == 16)
            sd_relax_kernel<uint16_t><<<rgrid, 256, 0, s>>>(chunks, chunk_count, g->fwd.dst, g->fwd.t,
                                                            (const uint16_t *)g->fwd.lam, pred, w.sd_slot, w.sd_d,
                                                            w.sd_sm, w.sd_changed, from_next, hislot, src, ta, tw,
                                                            unit, w.sd_ctr);
        else
            sd_relax_kernel<uint32_t><<<rgrid, 256, 0, s>>>(chunks, chunk_count, g->fwd.dst, g->fwd.t,
                                                            (const uint32_t *)g->fwd.lam, pred, w.sd_slot, w.sd_d,
                                                            w.sd_sm, w.sd_changed, from_next, hislot, src, ta, tw,
                                                            unit, w.sd_ctr);
        KAIROS_CUDA(cudaGetLastError(), "shortest duration: relax");
        KAIROS_CUDA(cudaMemcpyAsync(w.sd_ctr_host, w.sd_ctr, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s),
                    "shortest duration: flag");
        KAIROS_CUDA(cudaStreamSynchronize(s), "shortest duration: round");
        if (w.sd_ctr_host[0] == 0) break;  // no label dropped: the suffix minima are final
        KAIROS_CUDA(cudaMemsetAsync(long_count, 0, sizeof(unsigned), s), "shortest duration: long list");
        sd_suffix_kernel<<<vgrid, 256, 0, s>>>(n, g->rev.off, w.sd_d, w.sd_sm, w.sd_changed, w.sd_active, from_cur,
                                               from_next, hislot, long_v, long_top, long_count);
        KAIROS_CUDA(cudaGetLastError(), "shortest duration: suffix minima");
        sd_suffix_long_kernel<<<g->sm_count * 4, 256, 0, s>>>(g->rev.off, w.sd_d, w.sd_sm, long_v, long_top,
                                                                long_count);
        KAIROS_CUDA(cudaGetLastError(), "shortest duration: suffix minima");
    }
    uint32_t *res = out;
    const bool dev = on_device(out);
    if (!dev) {
        res = (uint32_t *)g->A.get((size_t)n * 4);
        if (!res) return fail(KAIROS_ERR_OOM, "shortest duration: device allocation failed");
    }
    sd_result_kernel<<<vgrid, 256, 0, s>>>(n, g->rev.off, w.sd_sm, src, res);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(w.ev1, s);
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(out, res, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (!dev) g->A.put(res);
    if (e != cudaSuccess) return cuda_fail(e, "shortest duration: result");
    float ms = 0;
    if (cudaEventElapsedTime(&ms, w.ev0, w.ev1) == cudaSuccess) g->last_kernel_ms = ms;
    cudaGetLastError();
    if (stats) {
        stats->rounds = rounds;
        stats->examined_edges = w.sd_ctr_host[1];
    }
    return KAIROS_OK;
}

extern "C" kairos_status kairos_shortest_duration(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw,
                                                  int32_t strict, uint32_t *out, kairos_duration_stats *stats) {
    return least_cost(g, src, ta, tw, strict, 0, out, stats);
}

extern "C" kairos_status kairos_temporal_bfs(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, int32_t strict,
                                             uint32_t *out, kairos_duration_stats *stats) {
    return least_cost(g, src, ta, tw, strict, 1, out, stats);
}
