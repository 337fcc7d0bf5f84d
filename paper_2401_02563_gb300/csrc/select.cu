// Selective access (Sec. 5): per-vertex (start, duration) density histograms built on the
// device (kairos_selectivity_build), the cardinality estimate of a temporal predicate with the
// exact count beside it (kairos_selectivity_estimate, used for the estimator-accuracy measure of
// Sec. 6.5), and the stored histogram of one vertex (kairos_selectivity_histogram).  The
// edge-map's per-vertex access choice (Eq. 3) uses the same estimate (hist.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "hist.cuh"

using namespace kairos;

namespace {

// First index i in [0, deg) with tl[i] >= key, by one lane.
__device__ __forceinline__ uint32_t lb_one(const uint32_t *__restrict__ tl, uint32_t deg, uint64_t key) {
    uint32_t lo = 0, hi = deg;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(&tl[mid]) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One warp per vertex: the estimate (UINT64_MAX without a histogram) and the exact count of
// edges departing in [a, b] and arriving by tw.
template <typename LamT>
__global__ void estimate_kernel(int32_t nv, const int32_t *verts, const uint64_t *off, const uint32_t *t, const LamT *lam,
                                const uint32_t *hidx, const HistHdr *hhdr, const uint32_t *hcum, uint64_t a, uint64_t b,
                                uint64_t tw, unsigned long long *est, unsigned long long *exact) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w0; k < nv; k += nw) {
        const int32_t u = verts[k];
        const uint64_t o0 = off[u];
        const uint32_t deg = (uint32_t)(off[u + 1] - o0);
        if (lane == 0) {
            const uint32_t hx = hidx ? hidx[u] : NO_HIST;
            est[k] = hx == NO_HIST ? ~0ull : hist_estimate(hhdr[hx], hcum + (size_t)hx * HIST_B * HIST_B, a, b, tw);
        }
        uint32_t lo = 0, hi = 0;
        if (lane == 0 && a <= b) {
            lo = lb_one(t + o0, deg, a);
            hi = lb_one(t + o0, deg, b + 1);
        }
        lo = __shfl_sync(0xFFFFFFFFu, lo, 0);
        hi = __shfl_sync(0xFFFFFFFFu, hi, 0);
        unsigned long long c = 0;
        for (uint32_t i = lo + lane; i < hi; i += 32) c += ((uint64_t)t[o0 + i] + (uint32_t)lam[o0 + i] <= tw) ? 1 : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0 && exact) exact[k] = c;
    }
}

// Bucket counts of histogram h (differences of its row-wise prefix sums).
__global__ void hist_counts_kernel(const uint32_t *hcum, uint32_t h, uint32_t *counts) {
    for (int i = threadIdx.x; i < HIST_B * HIST_B; i += blockDim.x) {
        const uint32_t *row = hcum + (size_t)h * HIST_B * HIST_B + (i / HIST_B) * HIST_B;
        const int j = i % HIST_B;
        counts[i] = row[j] - (j ? row[j - 1] : 0u);
    }
}

const Csr *direction(const kairos_graph *g, int32_t kind) {
    if (kind == KAIROS_EA) return &g->fwd;
    if (kind == KAIROS_LD && g->has_rev) return &g->rev;
    return nullptr;
}

}  // namespace

extern "C" {

kairos_status kairos_selectivity_build(kairos_graph *g, uint32_t min_degree) {
    if (!g) return fail(KAIROS_ERR_INVALID_ARG, "selectivity build: NULL graph");
    std::lock_guard<std::mutex> lk(g->mu);
    kairos_status st = build_histograms(g->A, g->stream, g->n, min_degree, g->lam_bits, &g->fwd);
    if (st == KAIROS_OK && g->has_rev) st = build_histograms(g->A, g->stream, g->n, min_degree, g->lam_bits, &g->rev);
    if (st != KAIROS_OK) {
        free_histograms(g->A, &g->fwd);
        free_histograms(g->A, &g->rev);
    }
    return st;
}

kairos_status kairos_selectivity_estimate(kairos_graph *g, int32_t kind, const int32_t *vertices, int32_t n, uint32_t a,
                                          uint32_t b, uint32_t tw, uint64_t *estimate, uint64_t *exact) {
    if (!g || (n > 0 && (!vertices || !estimate)) || n < 0)
        return fail(KAIROS_ERR_INVALID_ARG, "selectivity estimate: bad argument");
    const Csr *c = direction(g, kind);
    if (!c) return fail(KAIROS_ERR_INVALID_ARG, "selectivity estimate: kind must be KAIROS_EA, or KAIROS_LD with the reverse graph");
    for (int32_t i = 0; i < n; ++i)
        if (vertices[i] < 0 || vertices[i] >= g->n) return fail(KAIROS_ERR_INVALID_ARG, "selectivity estimate: vertex out of range");
    if (n == 0) return KAIROS_OK;
    std::lock_guard<std::mutex> lk(g->mu);
    cudaStream_t s = g->stream;
    int32_t *dv = (int32_t *)g->A.get((size_t)n * 4);
    unsigned long long *de = (unsigned long long *)g->A.get((size_t)n * 8);
    unsigned long long *dx = (unsigned long long *)g->A.get((size_t)n * 8);
    auto drop = [&]() {
        g->A.put(dv);
        g->A.put(de);
        g->A.put(dx);
    };
    if (!dv || !de || !dx) {
        drop();
        return fail(KAIROS_ERR_OOM, "selectivity estimate: device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(dv, vertices, (size_t)n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 4096);
        if (g->lam_bits == 16)
            estimate_kernel<uint16_t><<<grid, 256, 0, s>>>(n, dv, c->off, c->t, (const uint16_t *)c->lam, c->hidx, c->hhdr,
                                                           c->hcum, a, b, tw, de, dx);
        else
            estimate_kernel<uint32_t><<<grid, 256, 0, s>>>(n, dv, c->off, c->t, (const uint32_t *)c->lam, c->hidx, c->hhdr,
                                                           c->hcum, a, b, tw, de, dx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(estimate, de, (size_t)n * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && exact) e = cudaMemcpyAsync(exact, dx, (size_t)n * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    drop();
    if (e != cudaSuccess) return cuda_fail(e, "selectivity estimate");
    return KAIROS_OK;
}

kairos_status kairos_selectivity_histogram(kairos_graph *g, int32_t kind, int32_t vertex, uint64_t *meta4,
                                           uint32_t *counts) {
    if (!g || !meta4 || !counts) return fail(KAIROS_ERR_INVALID_ARG, "selectivity histogram: NULL argument");
    const Csr *c = direction(g, kind);
    if (!c) return fail(KAIROS_ERR_INVALID_ARG, "selectivity histogram: kind must be KAIROS_EA, or KAIROS_LD with the reverse graph");
    if (vertex < 0 || vertex >= g->n) return fail(KAIROS_ERR_INVALID_ARG, "selectivity histogram: vertex out of range");
    std::lock_guard<std::mutex> lk(g->mu);
    if (!c->hidx) return fail(KAIROS_ERR_INVALID_ARG, "selectivity histogram: no histograms built");
    cudaStream_t s = g->stream;
    uint32_t hx = NO_HIST;
    KAIROS_CUDA(cudaMemcpyAsync(&hx, c->hidx + vertex, 4, cudaMemcpyDeviceToHost, s), "selectivity histogram");
    KAIROS_CUDA(cudaStreamSynchronize(s), "selectivity histogram");
    if (hx == NO_HIST) return fail(KAIROS_ERR_INVALID_ARG, "selectivity histogram: the vertex has no histogram");
    HistHdr h;
    uint32_t *dc = (uint32_t *)g->A.get((size_t)HIST_B * HIST_B * 4);
    if (!dc) return fail(KAIROS_ERR_OOM, "selectivity histogram: device allocation failed");
    cudaError_t e = cudaMemcpyAsync(&h, c->hhdr + hx, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) {
        hist_counts_kernel<<<1, 256, 0, s>>>(c->hcum, hx, dc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dc, (size_t)HIST_B * HIST_B * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    g->A.put(dc);
    if (e != cudaSuccess) return cuda_fail(e, "selectivity histogram");
    meta4[0] = h.tmin;
    meta4[1] = h.S;
    meta4[2] = h.lmin;
    meta4[3] = h.D;
    return KAIROS_OK;
}

}  // extern "C"
