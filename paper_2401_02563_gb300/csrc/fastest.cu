// Fastest paths (minimum duration; Sec. 2.3 lists them among the minimal temporal paths) on
// the batched edge-map.
//
// A fastest path from s to v leaves s by one of s's out-edges, at some departure time d.
// Earliest arrival from s inside [d, tw] is the end of a path that leaves s at or after d, so
// EA_d[v] - d is at least the duration of that path; and for the d at which a fastest path
// leaves, EA_d[v] is at most that path's end.  Hence
//     fastest[v] = min over the distinct departure times d of s's usable out-edges of
//                  (EA_d[v] - d),
// which the library computes with one earliest-arrival lane per d (packed tuning.lanes per
// persistent launch, each edge load shared by the lanes) and a device reduction over the
// lanes' label rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "trace.h"

namespace kairos {
namespace {

constexpr size_t FAST_ROW_BUDGET = size_t(1) << 30;  // bytes of label rows per pass
constexpr int64_t FAST_MAX_ROWS = 1024;               // start-time lanes per pass

__global__ void fastest_init_kernel(uint32_t *best, int64_t n, int32_t src) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        best[v] = (v == src) ? 0u : INF;
}

// best[v] = min(best[v], min over rows q of rows[q][v] - d[q]) over reached labels.  Each row
// is read once, coalesced; the k start times sit in shared memory.
__global__ void fastest_reduce_kernel(const uint32_t *__restrict__ rows, int k, int64_t n,
                                      const uint32_t *__restrict__ d, uint32_t *__restrict__ best) {
    __shared__ uint32_t sd[FAST_MAX_ROWS];
    for (int q = threadIdx.x; q < k; q += blockDim.x) sd[q] = d[q];
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t m = best[v];
        for (int q = 0; q < k; ++q) {
            const uint32_t x = __ldcs(&rows[(int64_t)q * n + v]);
            if (x != INF && x - sd[q] < m) m = x - sd[q];  // x >= d: EA_d labels start at d
        }
        best[v] = m;
    }
}

int grid_for(int64_t n, int sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Distinct departure times d of src's usable out-edges (d >= ta, d + lambda <= tw), ascending
// (the list is stored in departure order).
kairos_status start_times(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, std::vector<uint32_t> &D) {
    cudaStream_t s = g->stream;
    uint64_t o[2] = {0, 0};
    KAIROS_CUDA(cudaMemcpyAsync(o, g->fwd.off + src, sizeof(o), cudaMemcpyDeviceToHost, s), "fastest path: offsets");
    KAIROS_CUDA(cudaStreamSynchronize(s), "fastest path: offsets");
    const uint64_t deg = o[1] - o[0];
    D.clear();
    if (deg == 0) return KAIROS_OK;
    std::vector<uint32_t> t(deg), lam(deg);
    KAIROS_CUDA(cudaMemcpyAsync(t.data(), g->fwd.t + o[0], deg * 4, cudaMemcpyDeviceToHost, s), "fastest path: times");
    if (g->lam_bits == 16) {
        std::vector<uint16_t> l16(deg);
        KAIROS_CUDA(cudaMemcpyAsync(l16.data(), (const uint16_t *)g->fwd.lam + o[0], deg * 2, cudaMemcpyDeviceToHost, s),
                    "fastest path: durations");
        KAIROS_CUDA(cudaStreamSynchronize(s), "fastest path: durations");
        for (uint64_t i = 0; i < deg; ++i) lam[i] = l16[i];
    } else {
        KAIROS_CUDA(cudaMemcpyAsync(lam.data(), (const uint32_t *)g->fwd.lam + o[0], deg * 4, cudaMemcpyDeviceToHost, s),
                    "fastest path: durations");
        KAIROS_CUDA(cudaStreamSynchronize(s), "fastest path: durations");
    }
    for (uint64_t i = 0; i < deg; ++i)
        if (t[i] >= ta && (uint64_t)t[i] + lam[i] <= tw && (D.empty() || D.back() != t[i])) D.push_back(t[i]);
    return KAIROS_OK;
}

kairos_status ensure_fastest_scratch(kairos_graph *g, int64_t rows, bool need_best) {
    auto &w = g->work;
    const int64_t n = g->n;
    if (w.fast_rows_cap < rows) {
        g->A.put(w.fast_rows);
        g->A.put(w.fast_d);
        w.fast_rows = (uint32_t *)g->A.get((size_t)rows * n * 4);
        w.fast_d = (uint32_t *)g->A.get((size_t)rows * 4);
        w.fast_rows_cap = (w.fast_rows && w.fast_d) ? rows : 0;
        if (!w.fast_rows_cap) {
            g->A.put(w.fast_rows);
            g->A.put(w.fast_d);
            w.fast_rows = w.fast_d = nullptr;
            return fail(KAIROS_ERR_OOM, "fastest path: device allocation of label rows failed");
        }
    }
    if (need_best && !w.fast_best) {
        w.fast_best = (uint32_t *)g->A.get((size_t)n * 4);
        if (!w.fast_best) return fail(KAIROS_ERR_OOM, "fastest path: device allocation failed");
    }
    return KAIROS_OK;
}

}  // namespace

void release_fastest_scratch(kairos_graph *g) {
    auto &w = g->work;
    g->A.put(w.fast_rows);
    g->A.put(w.fast_best);
    g->A.put(w.fast_d);
    w.fast_rows = w.fast_best = w.fast_d = nullptr;
    w.fast_rows_cap = 0;
}

}  // namespace kairos

using namespace kairos;

extern "C" kairos_status kairos_fastest_path(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, int32_t strict,
                                             uint32_t *out, kairos_fastest_stats *stats) {
    if (!g || !out) return fail(KAIROS_ERR_INVALID_ARG, "fastest path: NULL argument");
    if (src < 0 || (int64_t)src >= g->n) return fail(KAIROS_ERR_INVALID_ARG, "fastest path: source out of range");
    if (ta > tw || tw > TMAX) return fail(KAIROS_ERR_INVALID_ARG, "fastest path: need ta <= tw <= KAIROS_TIME_MAX");
    if (strict != 0 && strict != 1) return fail(KAIROS_ERR_INVALID_ARG, "fastest path: strict is 0 or 1");
    std::lock_guard<std::mutex> lk(g->mu);
    TraceRange tr("kairos_fastest_path");
    cudaStream_t s = g->stream;
    const int64_t n = g->n;
    kairos_fastest_stats fs;
    std::memset(&fs, 0, sizeof(fs));

    std::vector<uint32_t> D;
    kairos_status st = start_times(g, src, ta, tw, D);
    if (st != KAIROS_OK) return st;
    fs.start_times = D.size();

    const int W = g->tuning.lanes;
    int64_t rows = (int64_t)(FAST_ROW_BUDGET / ((size_t)n * 4)) / W * W;
    rows = std::max<int64_t>(W, std::min<int64_t>(rows, FAST_MAX_ROWS / W * W));
    rows = std::min<int64_t>(rows, ((int64_t)D.size() + W - 1) / W * W);
    const bool dev = on_device(out);
    st = ensure_fastest_scratch(g, std::max<int64_t>(rows, 1), !dev);
    if (st != KAIROS_OK) return st;
    auto &w = g->work;
    uint32_t *best = dev ? out : w.fast_best;
    const int grid = grid_for(n, g->sm_count);
    fastest_init_kernel<<<grid, 256, 0, s>>>(best, n, src);
    KAIROS_CUDA(cudaGetLastError(), "fastest path: init");

    std::vector<kairos_query> qs;
    std::vector<kairos_query_stats> qst;
    for (size_t c = 0; c < D.size(); c += (size_t)rows) {
        const int k = (int)std::min<size_t>((size_t)rows, D.size() - c);
        qs.assign(k, kairos_query{});
        for (int j = 0; j < k; ++j) {
            qs[j].vertex = src;
            qs[j].ta = D[c + j];
            qs[j].tw = tw;
            qs[j].kind = KAIROS_EA;
            qs[j].strict = (uint8_t)strict;
        }
        qst.assign(k, kairos_query_stats{});
        st = kairos_run_queries(g, qs.data(), k, w.fast_rows, stats ? qst.data() : nullptr, W);
        if (st != KAIROS_OK) return st;
        fs.launches += (uint64_t)((k + W - 1) / W);
        for (int j = 0; j < k; ++j) fs.relaxed_edges += qst[j].relaxed_edges;
        KAIROS_CUDA(cudaMemcpyAsync(w.fast_d, D.data() + c, (size_t)k * 4, cudaMemcpyHostToDevice, s),
                    "fastest path: start times");
        fastest_reduce_kernel<<<grid, 256, 0, s>>>(w.fast_rows, k, n, w.fast_d, best);
        KAIROS_CUDA(cudaGetLastError(), "fastest path: reduce");
    }
    if (!dev) KAIROS_CUDA(cudaMemcpyAsync(out, best, (size_t)n * 4, cudaMemcpyDeviceToHost, s), "fastest path: copy out");
    KAIROS_CUDA(cudaStreamSynchronize(s), "fastest path");
    if (stats) *stats = fs;
    return KAIROS_OK;
}
