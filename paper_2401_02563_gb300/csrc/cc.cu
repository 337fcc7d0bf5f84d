// Temporal connected components within a window [ta, tw] (the connectivity application of
// Sec. 2.3 / Table 4, adapted to a start and end time as Sec. 6 describes): the connected
// components of the undirected graph of the edges usable in the window (t >= ta and
// t + lam <= tw); out[v] = the smallest vertex id of v's component.
//
// One pass of concurrent union-find over the usable edges (a warp per vertex, its window
// prefix found by binary search in the time-sorted list): each edge links the larger of its
// endpoints' roots under the smaller one with a compare-and-swap that succeeds only while the
// larger is still a root, retrying with the new roots otherwise; finds halve paths as they go.
// Parents only ever move to smaller ids, so the trees stay acyclic and every component's root
// is its smallest vertex.  A final pass gives every vertex its root.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "trace.h"

using namespace kairos;

namespace {

constexpr unsigned CC_RETRY_LIMIT = 1u << 22;  // link attempts per edge before giving up (error)

__device__ __forceinline__ int32_t cc_find(int32_t *parent, int32_t x) {
    for (;;) {
        const int32_t p = __ldcg(&parent[x]);
        if (p == x) return x;
        const int32_t gp = __ldcg(&parent[p]);
        if (gp != p) __stcg(&parent[x], gp);  // halving: gp is an ancestor of x
        x = gp;
    }
}

__global__ void cc_init(int64_t n, int32_t *parent) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = (int32_t)v;
}

template <typename LamT>
__global__ void cc_link(int64_t n, const uint64_t *off, const int32_t *dst, const uint32_t *t, const LamT *lam,
                        uint32_t ta, uint32_t tw, int32_t *parent, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < n; u += nw) {
        const uint64_t o0 = off[u];
        const uint32_t deg = (uint32_t)(off[u + 1] - o0);
        uint32_t b = 0;
        if (lane == 0) {  // first departure at or after ta
            uint32_t lo = 0, hi = deg;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (t[o0 + mid] < ta) lo = mid + 1; else hi = mid;
            }
            b = lo;
        }
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        for (uint32_t i = b + lane; i < deg; i += 32) {
            const uint32_t ti = t[o0 + i];
            if (ti > tw) break;  // departures only grow along the list
            if ((uint64_t)ti + (uint32_t)lam[o0 + i] > tw) continue;
            int32_t x = (int32_t)u, y = dst[o0 + i];
            for (unsigned k = 0;; ++k) {
                const int32_t rx = cc_find(parent, x), ry = cc_find(parent, y);
                if (rx == ry) break;
                const int32_t hi = max(rx, ry), lo = min(rx, ry);
                if (atomicCAS(&parent[hi], hi, lo) == hi) break;
                if (k >= CC_RETRY_LIMIT) {
                    atomicExch(err, 1);
                    break;
                }
                x = rx;
                y = ry;
            }
        }
    }
}

__global__ void cc_finish(int64_t n, int32_t *parent, uint32_t *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = (uint32_t)cc_find(parent, (int32_t)v);
}

uint32_t *writable_out(uint32_t *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
    if (at.type == cudaMemoryTypeHost && at.devicePointer) return (uint32_t *)at.devicePointer;
    return nullptr;
}

}  // namespace

extern "C" kairos_status kairos_temporal_cc(kairos_graph *g, uint32_t ta, uint32_t tw, uint32_t *out) {
    if (!g || !out) return fail(KAIROS_ERR_INVALID_ARG, "temporal CC: NULL argument");
    if (ta > tw || tw > TMAX) return fail(KAIROS_ERR_INVALID_ARG, "temporal CC: need ta <= tw <= KAIROS_TIME_MAX");
    std::lock_guard<std::mutex> lk(g->mu);
    TraceRange tr("kairos_temporal_cc");
    const int64_t n = g->n;
    cudaStream_t s = g->stream;
    int32_t *parent = (int32_t *)g->A.get((size_t)n * 4);
    int *err = (int *)g->A.get(sizeof(int));
    uint32_t *dout = writable_out(out);
    uint32_t *stage = dout ? nullptr : (uint32_t *)g->A.get((size_t)n * 4);
    auto drop = [&]() {
        g->A.put(parent);
        g->A.put(err);
        g->A.put(stage);
    };
    if (!parent || !err || (!dout && !stage)) {
        drop();
        return fail(KAIROS_ERR_OOM, "temporal CC: device allocation failed");
    }
    const unsigned grid = (unsigned)std::max(1, g->sm_count * 8);
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        cc_init<<<grid, 256, 0, s>>>(n, parent);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (g->lam_bits == 16)
            cc_link<uint16_t><<<grid, 256, 0, s>>>(n, g->fwd.off, g->fwd.dst, g->fwd.t, (const uint16_t *)g->fwd.lam, ta, tw,
                                                   parent, err);
        else
            cc_link<uint32_t><<<grid, 256, 0, s>>>(n, g->fwd.off, g->fwd.dst, g->fwd.t, (const uint32_t *)g->fwd.lam, ta, tw,
                                                   parent, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        cc_finish<<<grid, 256, 0, s>>>(n, parent, dout ? dout : stage);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !dout) e = cudaMemcpyAsync(out, stage, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    drop();
    if (e != cudaSuccess) return cuda_fail(e, "temporal CC");
    if (herr) return fail(KAIROS_ERR_INTERNAL, "temporal CC: a link loop exceeded its retry limit");
    return KAIROS_OK;
}
