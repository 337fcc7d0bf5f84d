// Device build of the time-sorted CSR (the T-CSR of Sec. 4.2 with every adjacency list in
// departure-time order) and of the selective-index fence level (Sec. 3.2, Alg. 1).
//
// Sort: least-significant-digit radix sort of 64-bit keys (vertex << 32 | departure time)
// carrying a 32-bit edge index, 8-bit digits, one upsweep (per-tile digit histograms), one
// device-wide exclusive scan and one stable scatter per digit.  Alg. 1 sorts each indexed
// vertex's edges by start time; here every list is sorted once for the whole graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace kairos {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // keys per block
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- exclusive scan of uint32 (totals < 2^32) --------------------------------------------

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan of one value per thread; returns the block total in *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *total) {
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(x);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < nw ? wsum[lane] : 0;
        uint32_t vi = warp_incl_scan(v);
        if (lane < nw) wsum[lane] = vi - v;
        if (lane == nw - 1) wsum[31] = vi;
    }
    __syncthreads();
    uint32_t res = inc - x + wsum[warp];
    *total = wsum[31];
    __syncthreads();
    return res;
}

__global__ void scan_reduce_kernel(const uint32_t *in, int64_t n, uint32_t *sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t acc = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += in[i];
    }
    uint32_t tot;
    block_excl_scan(acc, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// out[i] = offset[block] + exclusive scan of in within the block's tile (blocked layout).
__global__ void scan_down_kernel(const uint32_t *in, int64_t n, const uint32_t *offset, uint32_t *out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t acc = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        acc += v[k];
    }
    uint32_t tot;
    uint32_t pre = block_excl_scan(acc, &tot) + (offset ? offset[blockIdx.x] : 0);
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = pre;
        pre += v[k];
    }
}

// Recursive device-wide exclusive scan; `tmp` must hold scan_tmp_words(n) words.
int64_t scan_tmp_words(int64_t n) {
    int64_t w = 0;
    while (n > SCAN_TILE) {
        n = cdiv(n, SCAN_TILE);
        w += 2 * n;
    }
    return w + 2;
}

cudaError_t excl_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t nb = cdiv(n, SCAN_TILE);
    if (nb == 1) {
        scan_down_kernel<<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out);
        return cudaGetLastError();
    }
    uint32_t *sums = tmp, *sums_scan = tmp + nb;
    scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums);
    cudaError_t e = excl_scan(sums, sums_scan, nb, tmp + 2 * nb, s);
    if (e != cudaSuccess) return e;
    scan_down_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums_scan, out);
    return cudaGetLastError();
}

// ---- radix sort --------------------------------------------------------------------------

__global__ void rs_upsweep(const uint64_t *keys, int64_t m, int shift, uint32_t *hist, int64_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = 0; k < RS_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
        if (i < m) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items of a tile keep their order among equal digits; tiles keep theirs
// through the digit-major, tile-minor scan of the histograms.
__global__ void rs_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout, int64_t m,
                           int shift, const uint32_t *offs, int64_t nblocks) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int sub = 0; sub < RS_ITEMS; ++sub) {
        int64_t i = base + (int64_t)sub * RS_THREADS + tid;
        bool valid = i < m;
        uint64_t key = valid ? kin[i] : 0;
        uint32_t val = valid ? vin[i] : 0;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) wc[w][tid] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wc[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) add += wc[w][tid];
        run[tid] += add;
        __syncthreads();
    }
}

// ---- CSR pieces ----------------------------------------------------------------------------

template <typename LamT>
__global__ void make_keys(int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t, const LamT *lam,
                          int mirror, uint64_t *keys, uint32_t *vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k;
        if (!mirror) {
            k = ((uint64_t)(uint32_t)src[i] << 32) | t[i];
        } else {  // reversed edge dst -> src, departing at TMAX - (t + lam)
            uint32_t tm = TMAX - (t[i] + (uint32_t)lam[i]);
            k = ((uint64_t)(uint32_t)dst[i] << 32) | tm;
        }
        keys[i] = k;
        vals[i] = (uint32_t)i;
    }
}

template <typename LamT>
__global__ void gather_edges(int64_t m, const uint64_t *keys, const uint32_t *vals, const int32_t *head_in,
                             const LamT *lam_in, int32_t *head_out, uint32_t *t_out, LamT *lam_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = vals[i];
        head_out[i] = head_in[e];
        t_out[i] = (uint32_t)keys[i];
        lam_out[i] = lam_in[e];
    }
}

// off[u] = first sorted position whose vertex is >= u (binary search on the sorted keys).
__global__ void csr_offsets(const uint64_t *keys, int64_t m, int64_t n, uint64_t *off) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= n; u += (int64_t)gridDim.x * blockDim.x) {
        uint64_t target = (uint64_t)u << 32;
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < target) lo = mid + 1; else hi = mid;
        }
        off[u] = (uint64_t)lo;
    }
}

template <typename LamT>
__global__ void validate_kernel(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                                const LamT *lam, int *flags) {
    int bad_v = 0, bad_t = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = src[i], v = dst[i];
        if (u < 0 || u >= n || v < 0 || v >= n) bad_v = 1;
        if ((uint64_t)t[i] + (uint64_t)lam[i] > (uint64_t)TMAX) bad_t = 1;
    }
    if (__any_sync(0xFFFFFFFFu, bad_v) && (threadIdx.x & 31) == 0) atomicOr(flags, 1);
    if (__any_sync(0xFFFFFFFFu, bad_t) && (threadIdx.x & 31) == 0) atomicOr(flags, 2);
}

__global__ void degree_stats(int64_t n, const uint64_t *off, int64_t x, int64_t chunk, unsigned long long *acc) {
    unsigned long long cnt = 0, ch = 0, mx = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d = off[u + 1] - off[u];
        if ((int64_t)d > x) {
            cnt += 1;
            ch += (d + chunk - 1) / chunk;
        }
        mx = d > mx ? d : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        ch += __shfl_xor_sync(0xFFFFFFFFu, ch, o);
        unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], cnt);
        atomicAdd(&acc[1], ch);
        atomicMax(&acc[2], mx);
    }
}

// ---- fence level ---------------------------------------------------------------------------

__global__ void fence_counts(int64_t n, const uint64_t *off, uint32_t threshold, uint32_t *cnt) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d = off[u + 1] - off[u];
        cnt[u] = (d > 0 && d >= threshold) ? (uint32_t)((d + FENCE_B - 1) >> FENCE_SHIFT) : 0u;
    }
}

// One warp per vertex: fence[fidx[u] + k] = t[off[u] + k * FENCE_B].
__global__ void fence_fill(int64_t n, const uint64_t *off, const uint32_t *t, const uint32_t *cnt,
                           uint32_t *fidx, uint32_t *fence) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < n; u += nw) {
        uint32_t c = cnt[u];
        uint32_t start = fidx[u];  // holds the exclusive scan of cnt on entry
        if (c == 0) {
            if (lane == 0) fidx[u] = NO_FENCE;
            continue;
        }
        uint64_t o = off[u];
        for (uint32_t k = lane; k < c; k += 32) fence[start + k] = t[o + ((uint64_t)k << FENCE_SHIFT)];
    }
}

int grid_for(int64_t items, int threads) {
    int64_t g = cdiv(items > 0 ? items : 1, threads);
    return (int)std::min<int64_t>(g, 65535LL * 16);
}

// src_of[i] = the vertex whose forward list holds position i (binary search over offsets).
__global__ void edge_sources(int64_t n, int64_t m, const uint64_t *off, int32_t *src_of) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;  // last u with off[u] <= i
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= (uint64_t)i) lo = mid; else hi = mid;
        }
        src_of[i] = (int32_t)lo;
    }
}

// slot[vals[j]] = j: the inverse of the sorted payload.
__global__ void invert_payload(int64_t m, const uint32_t *vals, uint32_t *slot) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        slot[vals[j]] = (uint32_t)j;
}

// ---- time-ordered stream ------------------------------------------------------------------

__global__ void time_keys(int64_t m, const uint32_t *t, uint64_t *keys, uint32_t *vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = t[i];
        vals[i] = (uint32_t)i;
    }
}

template <typename LamT>
__global__ void gather_records(int64_t m, const uint32_t *vals, const int32_t *src_of, const int32_t *dst,
                               const uint32_t *t, const LamT *lam, StreamRec *out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = vals[j];
        StreamRec r;
        r.src = src_of[e];
        r.dst = dst[e];
        r.t = t[e];
        r.lam = (uint32_t)lam[e];
        out[j] = r;
    }
}

// For k < nb: the block of records starting near k * eb begins at the first record departing at
// or after rec[k * eb].t (so that no instant is split); bnd[nb] = m.
__global__ void block_starts(const StreamRec *rec, int64_t m, int64_t eb, int64_t nb, uint64_t *bnd, uint32_t *bt) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= nb; k += (int64_t)gridDim.x * blockDim.x) {
        if (k == nb) {
            bnd[k] = (uint64_t)m;
            bt[k] = INF;
            continue;
        }
        const uint32_t key = rec[k * eb].t;
        int64_t lo = 0, hi = k * eb;  // rec[hi].t == key: the answer is in [lo, hi]
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rec[mid].t < key) lo = mid + 1; else hi = mid;
        }
        bnd[k] = (uint64_t)lo;
        bt[k] = key;
    }
}

// ---- selectivity histograms (Sec. 5.2) ------------------------------------------------------

__global__ void hist_flags(int64_t n, const uint64_t *off, uint32_t min_degree, uint32_t *flag) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        flag[u] = (off[u + 1] - off[u]) >= (uint64_t)min_degree && off[u + 1] > off[u] ? 1u : 0u;
}

__global__ void hist_number(int64_t n, const uint32_t *flag, const uint32_t *pos, uint32_t *hidx, int32_t *verts) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        hidx[u] = flag[u] ? pos[u] : NO_HIST;
        if (flag[u]) verts[pos[u]] = (int32_t)u;
    }
}

// One block per histogram: bucket counts in shared memory, then the row-wise prefix sums.
template <typename LamT>
__global__ void __launch_bounds__(256) hist_fill(int64_t nh, const int32_t *verts, const uint64_t *off, const uint32_t *t,
                                                 const LamT *lam, HistHdr *hdr, uint32_t *hcum, uint32_t *hrow) {
    extern __shared__ uint32_t cnt[];  // HIST_B * HIST_B counts, then HIST_B row totals
    __shared__ uint32_t lmn[8], lmx[8];
    for (int64_t h = blockIdx.x; h < nh; h += gridDim.x) {
        const int32_t u = verts[h];
        const uint64_t o0 = off[u], o1 = off[u + 1];
        const uint32_t tmin = t[o0], tmax = t[o1 - 1];  // each list is in departure order
        uint32_t mn = 0xFFFFFFFFu, mx = 0;
        for (uint64_t e = o0 + threadIdx.x; e < o1; e += blockDim.x) {
            const uint32_t x = (uint32_t)lam[e];
            mn = min(mn, x);
            mx = max(mx, x);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        }
        for (int i = threadIdx.x; i < HIST_B * HIST_B; i += blockDim.x) cnt[i] = 0;
        if ((threadIdx.x & 31) == 0) {
            lmn[threadIdx.x >> 5] = mn;
            lmx[threadIdx.x >> 5] = mx;
        }
        __syncthreads();
        mn = lmn[0];
        mx = lmx[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mn = min(mn, lmn[w]);
            mx = max(mx, lmx[w]);
        }
        const uint64_t S = (uint64_t)tmax - tmin + 1, D = (uint64_t)mx - mn + 1;
        for (uint64_t e = o0 + threadIdx.x; e < o1; e += blockDim.x) {
            const uint32_t i = (uint32_t)(((uint64_t)t[e] - tmin) * HIST_B / S);
            const uint32_t j = (uint32_t)(((uint64_t)(uint32_t)lam[e] - mn) * HIST_B / D);
            atomicAdd(&cnt[i * HIST_B + j], 1u);
        }
        __syncthreads();
        if (threadIdx.x < HIST_B) {
            uint32_t run = 0;
            uint32_t *row = hcum + ((size_t)h * HIST_B + threadIdx.x) * HIST_B;
            for (int j = 0; j < HIST_B; ++j) {
                run += cnt[threadIdx.x * HIST_B + j];
                row[j] = run;
            }
            cnt[HIST_B * HIST_B + threadIdx.x] = run;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t run = 0;
            uint32_t *rp = hrow + (size_t)h * (HIST_B + 1);
            for (int i = 0; i < HIST_B; ++i) {
                rp[i] = run;
                run += cnt[HIST_B * HIST_B + i];
            }
            rp[HIST_B] = run;
            HistHdr hh;
            hh.tmin = tmin;
            hh.lmin = mn;
            hh.S = S;
            hh.D = D;
            hdr[h] = hh;
        }
        __syncthreads();
    }
}

}  // namespace

kairos_status validate_edges(cudaStream_t s, int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                             const uint32_t *t, const void *lam, int lam_bits, int *flags_host,
                             const Allocator &A) {
    *flags_host = 0;
    if (m == 0) return KAIROS_OK;
    int *flags = (int *)A.get(sizeof(int));
    if (!flags) return fail(KAIROS_ERR_OOM, "validate: device allocation failed");
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        int g = grid_for(m, 256);
        if (lam_bits == 16)
            validate_kernel<uint16_t><<<g, 256, 0, s>>>(n, m, src, dst, t, (const uint16_t *)lam, flags);
        else
            validate_kernel<uint32_t><<<g, 256, 0, s>>>(n, m, src, dst, t, (const uint32_t *)lam, flags);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags_host, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    A.put(flags);
    if (e != cudaSuccess) return cuda_fail(e, "validate edges");
    return KAIROS_OK;
}

kairos_status build_csr(const Allocator &A, cudaStream_t s, int64_t n, int64_t m, const int32_t *src,
                        const int32_t *dst, const uint32_t *t, const void *lam, int lam_bits, int mirror,
                        Csr *out) {
    const size_t lam_sz = lam_bits == 16 ? 2 : 4;
    Csr c;
    c.off = (uint64_t *)A.get((size_t)(n + 1) * 8);
    c.dst = (int32_t *)A.get((size_t)std::max<int64_t>(m, 1) * 4);
    c.t = (uint32_t *)A.get((size_t)std::max<int64_t>(m, 1) * 4);
    c.lam = A.get((size_t)std::max<int64_t>(m, 1) * lam_sz);
    const int64_t nb = std::max<int64_t>(cdiv(m, RS_TILE), 1);
    const int64_t hist_n = 256 * nb;
    uint64_t *k0 = (uint64_t *)A.get((size_t)std::max<int64_t>(m, 1) * 8);
    uint64_t *k1 = (uint64_t *)A.get((size_t)std::max<int64_t>(m, 1) * 8);
    uint32_t *v0 = (uint32_t *)A.get((size_t)std::max<int64_t>(m, 1) * 4);
    uint32_t *v1 = (uint32_t *)A.get((size_t)std::max<int64_t>(m, 1) * 4);
    uint32_t *hist = (uint32_t *)A.get((size_t)hist_n * 4);
    uint32_t *offs = (uint32_t *)A.get((size_t)hist_n * 4);
    uint32_t *tmp = (uint32_t *)A.get((size_t)scan_tmp_words(hist_n) * 4);
    auto release_tmp = [&]() {
        A.put(k0); A.put(k1); A.put(v0); A.put(v1); A.put(hist); A.put(offs); A.put(tmp);
    };
    if (!c.off || !c.dst || !c.t || !c.lam || !k0 || !k1 || !v0 || !v1 || !hist || !offs || !tmp) {
        release_tmp();
        free_csr(A, &c);
        return fail(KAIROS_ERR_OOM, "graph build: device allocation failed");
    }
    cudaError_t e = cudaSuccess;
    const int g = grid_for(m, 256);
    if (m > 0) {
        if (lam_bits == 16)
            make_keys<uint16_t><<<g, 256, 0, s>>>(m, src, dst, t, (const uint16_t *)lam, mirror, k0, v0);
        else
            make_keys<uint32_t><<<g, 256, 0, s>>>(m, src, dst, t, (const uint32_t *)lam, mirror, k0, v0);
        e = cudaGetLastError();
        // digits cover 32 time bits plus the bits of the largest vertex id
        int vbits = 0;
        while (vbits < 63 && (1LL << vbits) < n) ++vbits;
        const int passes = (32 + vbits + 7) / 8;
        uint64_t *ki = k0, *ko = k1;
        uint32_t *vi = v0, *vo = v1;
        for (int p = 0; p < passes && e == cudaSuccess; ++p) {
            const int shift = 8 * p;
            rs_upsweep<<<(unsigned)nb, RS_THREADS, 0, s>>>(ki, m, shift, hist, nb);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = excl_scan(hist, offs, hist_n, tmp, s);
            if (e == cudaSuccess) {
                rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(ki, vi, ko, vo, m, shift, offs, nb);
                e = cudaGetLastError();
            }
            std::swap(ki, ko);
            std::swap(vi, vo);
        }
        if (e == cudaSuccess) {
            const int32_t *head = mirror ? src : dst;
            if (lam_bits == 16)
                gather_edges<uint16_t><<<g, 256, 0, s>>>(m, ki, vi, head, (const uint16_t *)lam, c.dst, c.t,
                                                         (uint16_t *)c.lam);
            else
                gather_edges<uint32_t><<<g, 256, 0, s>>>(m, ki, vi, head, (const uint32_t *)lam, c.dst, c.t,
                                                         (uint32_t *)c.lam);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            csr_offsets<<<grid_for(n + 1, 256), 256, 0, s>>>(ki, m, n, c.off);
            e = cudaGetLastError();
        }
    } else {
        e = cudaMemsetAsync(c.off, 0, (size_t)(n + 1) * 8, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release_tmp();
    if (e != cudaSuccess) {
        free_csr(A, &c);
        return cuda_fail(e, "graph build");
    }
    unsigned long long *acc = (unsigned long long *)A.get(3 * 8);
    if (!acc) {
        free_csr(A, &c);
        return fail(KAIROS_ERR_OOM, "graph build: device allocation failed");
    }
    unsigned long long h[3] = {0, 0, 0};
    e = cudaMemsetAsync(acc, 0, 24, s);
    if (e == cudaSuccess) {
        degree_stats<<<grid_for(n, 256), 256, 0, s>>>(n, c.off, 1LL << 62, 1, acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, 24, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    A.put(acc);
    if (e != cudaSuccess) {
        free_csr(A, &c);
        return cuda_fail(e, "graph build: degree scan");
    }
    c.max_deg = (int64_t)h[2];
    *out = c;
    return KAIROS_OK;
}

kairos_status build_reverse_slots(const Allocator &A, cudaStream_t s, int64_t n, int64_t m, const Csr &fwd,
                                  int lam_bits, uint32_t *fwd2rev) {
    if (m <= 0) return KAIROS_OK;
    const int64_t nb = std::max<int64_t>(cdiv(m, RS_TILE), 1);
    const int64_t hist_n = 256 * nb;
    int32_t *src_of = (int32_t *)A.get((size_t)m * 4);
    uint64_t *k0 = (uint64_t *)A.get((size_t)m * 8);
    uint64_t *k1 = (uint64_t *)A.get((size_t)m * 8);
    uint32_t *v0 = (uint32_t *)A.get((size_t)m * 4);
    uint32_t *v1 = (uint32_t *)A.get((size_t)m * 4);
    uint32_t *hist = (uint32_t *)A.get((size_t)hist_n * 4);
    uint32_t *offs = (uint32_t *)A.get((size_t)hist_n * 4);
    uint32_t *tmp = (uint32_t *)A.get((size_t)scan_tmp_words(hist_n) * 4);
    auto release_tmp = [&]() {
        A.put(src_of); A.put(k0); A.put(k1); A.put(v0); A.put(v1); A.put(hist); A.put(offs); A.put(tmp);
    };
    if (!src_of || !k0 || !k1 || !v0 || !v1 || !hist || !offs || !tmp) {
        release_tmp();
        return fail(KAIROS_ERR_OOM, "reverse slots: device allocation failed");
    }
    const int g = grid_for(m, 256);
    edge_sources<<<g, 256, 0, s>>>(n, m, fwd.off, src_of);
    cudaError_t e = cudaGetLastError();
    // keys of the reversed, time-mirrored edges (head << 32 | TMAX - (t + lam)), payload the
    // forward position: sorted exactly as the reverse list (ties in forward order)
    if (e == cudaSuccess) {
        if (lam_bits == 16)
            make_keys<uint16_t><<<g, 256, 0, s>>>(m, src_of, fwd.dst, fwd.t, (const uint16_t *)fwd.lam, 1, k0, v0);
        else
            make_keys<uint32_t><<<g, 256, 0, s>>>(m, src_of, fwd.dst, fwd.t, (const uint32_t *)fwd.lam, 1, k0, v0);
        e = cudaGetLastError();
    }
    int vbits = 0;
    while (vbits < 63 && (1LL << vbits) < n) ++vbits;
    const int passes = (32 + vbits + 7) / 8;
    uint64_t *ki = k0, *ko = k1;
    uint32_t *vi = v0, *vo = v1;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        const int shift = 8 * p;
        rs_upsweep<<<(unsigned)nb, RS_THREADS, 0, s>>>(ki, m, shift, hist, nb);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = excl_scan(hist, offs, hist_n, tmp, s);
        if (e == cudaSuccess) {
            rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(ki, vi, ko, vo, m, shift, offs, nb);
            e = cudaGetLastError();
        }
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    if (e == cudaSuccess) {
        invert_payload<<<g, 256, 0, s>>>(m, vi, fwd2rev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release_tmp();
    if (e != cudaSuccess) return cuda_fail(e, "reverse slots");
    return KAIROS_OK;
}

kairos_status split_capacity(const Allocator &A, cudaStream_t s, int64_t n, const uint64_t *off, int64_t x,
                             int64_t chunk, uint64_t *vertices, uint64_t *chunks) {
    unsigned long long *acc = (unsigned long long *)A.get(3 * 8);
    if (!acc) return fail(KAIROS_ERR_OOM, "workspace: device allocation failed");
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = cudaMemsetAsync(acc, 0, 24, s);
    if (e == cudaSuccess) {
        degree_stats<<<grid_for(n, 256), 256, 0, s>>>(n, off, x, chunk, acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, 24, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    A.put(acc);
    if (e != cudaSuccess) return cuda_fail(e, "workspace: degree scan");
    *vertices = h[0];
    *chunks = h[1];
    return KAIROS_OK;
}

kairos_status build_index(const Allocator &A, cudaStream_t s, int64_t n, uint32_t threshold, Csr *c) {
    free_index(A, c);
    if (threshold == KAIROS_NO_INDEX) return KAIROS_OK;
    uint32_t *cnt = (uint32_t *)A.get((size_t)n * 4);
    uint32_t *fidx = (uint32_t *)A.get((size_t)n * 4);
    uint32_t *tmp = (uint32_t *)A.get((size_t)scan_tmp_words(n) * 4);
    if (!cnt || !fidx || !tmp) {
        A.put(cnt); A.put(fidx); A.put(tmp);
        return fail(KAIROS_ERR_OOM, "index build: device allocation failed");
    }
    cudaError_t e;
    fence_counts<<<grid_for(n, 256), 256, 0, s>>>(n, c->off, threshold, cnt);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = excl_scan(cnt, fidx, n, tmp, s);
    uint32_t last[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[0], fidx + (n - 1), 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], cnt + (n - 1), 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int64_t total = (int64_t)last[0] + last[1];
    uint32_t *fence = nullptr;
    if (e == cudaSuccess) {
        fence = (uint32_t *)A.get((size_t)std::max<int64_t>(total, 1) * 4);
        if (!fence) {
            A.put(cnt); A.put(fidx); A.put(tmp);
            return fail(KAIROS_ERR_OOM, "index build: device allocation failed");
        }
        fence_fill<<<grid_for(n * 32, 256), 256, 0, s>>>(n, c->off, c->t, cnt, fidx, fence);
        e = cudaGetLastError();
    }
    // count indexed vertices (fence counts > 0) with the degree scan helper
    unsigned long long *acc = (unsigned long long *)A.get(3 * 8);
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess && acc) {
        e = cudaMemsetAsync(acc, 0, 24, s);
        if (e == cudaSuccess) {
            degree_stats<<<grid_for(n, 256), 256, 0, s>>>(n, c->off, (int64_t)threshold - 1, 1, acc);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, 24, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    A.put(acc);
    A.put(cnt);
    A.put(tmp);
    if (e != cudaSuccess || !acc) {
        A.put(fidx);
        A.put(fence);
        if (!acc && e == cudaSuccess) return fail(KAIROS_ERR_OOM, "index build: device allocation failed");
        return cuda_fail(e, "index build");
    }
    c->fidx = fidx;
    c->fence = fence;
    c->n_fence = total;
    c->indexed = (int64_t)h[0];
    return KAIROS_OK;
}

kairos_status build_time_stream(const Allocator &A, cudaStream_t s, int64_t n, int64_t m, const Csr &c, int lam_bits,
                                StreamRec *out) {
    if (m <= 0) return KAIROS_OK;
    const int64_t nb = std::max<int64_t>(cdiv(m, RS_TILE), 1);
    const int64_t hist_n = 256 * nb;
    int32_t *src_of = (int32_t *)A.get((size_t)m * 4);
    uint64_t *k0 = (uint64_t *)A.get((size_t)m * 8);
    uint64_t *k1 = (uint64_t *)A.get((size_t)m * 8);
    uint32_t *v0 = (uint32_t *)A.get((size_t)m * 4);
    uint32_t *v1 = (uint32_t *)A.get((size_t)m * 4);
    uint32_t *hist = (uint32_t *)A.get((size_t)hist_n * 4);
    uint32_t *offs = (uint32_t *)A.get((size_t)hist_n * 4);
    uint32_t *tmp = (uint32_t *)A.get((size_t)scan_tmp_words(hist_n) * 4);
    auto release_tmp = [&]() {
        A.put(src_of); A.put(k0); A.put(k1); A.put(v0); A.put(v1); A.put(hist); A.put(offs); A.put(tmp);
    };
    if (!src_of || !k0 || !k1 || !v0 || !v1 || !hist || !offs || !tmp) {
        release_tmp();
        return fail(KAIROS_ERR_OOM, "time stream: device allocation failed");
    }
    const int g = grid_for(m, 256);
    edge_sources<<<g, 256, 0, s>>>(n, m, c.off, src_of);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        time_keys<<<g, 256, 0, s>>>(m, c.t, k0, v0);
        e = cudaGetLastError();
    }
    // stable by departure time: equal departures keep the CSR order
    uint64_t *ki = k0, *ko = k1;
    uint32_t *vi = v0, *vo = v1;
    for (int p = 0; p < 4 && e == cudaSuccess; ++p) {
        rs_upsweep<<<(unsigned)nb, RS_THREADS, 0, s>>>(ki, m, 8 * p, hist, nb);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = excl_scan(hist, offs, hist_n, tmp, s);
        if (e == cudaSuccess) {
            rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(ki, vi, ko, vo, m, 8 * p, offs, nb);
            e = cudaGetLastError();
        }
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    if (e == cudaSuccess) {
        if (lam_bits == 16)
            gather_records<uint16_t><<<g, 256, 0, s>>>(m, vi, src_of, c.dst, c.t, (const uint16_t *)c.lam, out);
        else
            gather_records<uint32_t><<<g, 256, 0, s>>>(m, vi, src_of, c.dst, c.t, (const uint32_t *)c.lam, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release_tmp();
    if (e != cudaSuccess) return cuda_fail(e, "time stream");
    return KAIROS_OK;
}

__global__ void vertex_spans(int64_t n, const uint64_t *off, const uint32_t *t, uint64_t *span) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = off[v], b = off[v + 1];
        span[v] = a < b ? ((uint64_t)t[a] << 32) | t[b - 1] : ((uint64_t)INF << 32);
    }
}

kairos_status build_vertex_spans(const Allocator &A, cudaStream_t s, int64_t n, const Csr &c, TimeStream *ts) {
    if (ts->span) return KAIROS_OK;
    ts->span = (uint64_t *)A.get((size_t)std::max<int64_t>(n, 1) * 8);
    if (!ts->span) return fail(KAIROS_ERR_OOM, "time stream: device allocation failed");
    if (n > 0) vertex_spans<<<grid_for(n, 256), 256, 0, s>>>(n, c.off, c.t, ts->span);
    KAIROS_CUDA(cudaGetLastError(), "time stream: vertex spans");
    return KAIROS_OK;
}

void free_time_stream(const Allocator &A, TimeStream *ts) {
    A.put(ts->span);
    A.put(ts->rec);
    A.put(ts->bnd);
    A.put(ts->bt);
    delete[] ts->bt_host;
    *ts = TimeStream();
}

kairos_status cut_time_blocks(const Allocator &A, cudaStream_t s, int64_t m, int64_t block_edges, TimeStream *ts) {
    A.put(ts->bnd);
    A.put(ts->bt);
    delete[] ts->bt_host;
    ts->bnd = nullptr;
    ts->bt = nullptr;
    ts->bt_host = nullptr;
    ts->nblk = 0;
    const int64_t eb = std::max<int64_t>(block_edges, 1);
    const int64_t nb = m > 0 ? cdiv(m, eb) : 0;
    if (nb > (1 << 24)) return fail(KAIROS_ERR_INVALID_ARG, "time stream: too many blocks for this block size");
    uint64_t *dbnd = (uint64_t *)A.get((size_t)(nb + 1) * 8);
    uint32_t *dbt = (uint32_t *)A.get((size_t)(nb + 1) * 4);
    if (!dbnd || !dbt) {
        A.put(dbnd);
        A.put(dbt);
        return fail(KAIROS_ERR_OOM, "time stream: device allocation failed");
    }
    std::vector<uint64_t> hb(nb + 1);
    std::vector<uint32_t> ht(nb + 1);
    block_starts<<<grid_for(nb + 1, 256), 256, 0, s>>>(ts->rec, m, eb, nb, dbnd, dbt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), dbnd, (nb + 1) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ht.data(), dbt, (nb + 1) * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        A.put(dbnd);
        A.put(dbt);
        return cuda_fail(e, "time stream: blocks");
    }
    // an instant longer than a block merges the blocks it covers: drop repeated starts
    std::vector<uint64_t> ub;
    std::vector<uint32_t> ut;
    for (int64_t k = 0; k <= nb; ++k)
        if (ub.empty() || hb[k] != ub.back()) {
            ub.push_back(hb[k]);
            ut.push_back(ht[k]);
        }
    if (ub.size() == 1 && m == 0) {  // no edges: no block
        ub.assign(1, 0);
        ut.assign(1, INF);
    }
    const int nblk = (int)ub.size() - 1;
    e = cudaMemcpyAsync(dbnd, ub.data(), ub.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbt, ut.data(), ut.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        A.put(dbnd);
        A.put(dbt);
        return cuda_fail(e, "time stream: blocks");
    }
    ts->bnd = dbnd;
    ts->bt = dbt;
    ts->nblk = nblk;
    ts->block_edges = block_edges;
    ts->bt_host = new uint32_t[ut.size()];
    std::copy(ut.begin(), ut.end(), ts->bt_host);
    return KAIROS_OK;
}

void free_histograms(const Allocator &A, Csr *c) {
    A.put(c->hidx);
    A.put(c->hhdr);
    A.put(c->hcum);
    A.put(c->hrow);
    c->hidx = nullptr;
    c->hhdr = nullptr;
    c->hcum = nullptr;
    c->hrow = nullptr;
    c->n_hist = 0;
    c->hist_min_degree = 0;
}

kairos_status build_histograms(const Allocator &A, cudaStream_t s, int64_t n, uint32_t min_degree, int lam_bits,
                               Csr *c) {
    free_histograms(A, c);
    if (min_degree == KAIROS_NO_INDEX) return KAIROS_OK;
    if (min_degree == 0) min_degree = 1;
    uint32_t *flag = (uint32_t *)A.get((size_t)n * 4);
    uint32_t *pos = (uint32_t *)A.get((size_t)n * 4);
    uint32_t *tmp = (uint32_t *)A.get((size_t)scan_tmp_words(n) * 4);
    uint32_t *hidx = (uint32_t *)A.get((size_t)n * 4);
    auto drop = [&]() {
        A.put(flag);
        A.put(pos);
        A.put(tmp);
    };
    if (!flag || !pos || !tmp || !hidx) {
        drop();
        A.put(hidx);
        return fail(KAIROS_ERR_OOM, "histograms: device allocation failed");
    }
    hist_flags<<<grid_for(n, 256), 256, 0, s>>>(n, c->off, min_degree, flag);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = excl_scan(flag, pos, n, tmp, s);
    uint32_t last[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[0], pos + (n - 1), 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], flag + (n - 1), 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        drop();
        A.put(hidx);
        return cuda_fail(e, "histograms");
    }
    const int64_t nh = (int64_t)last[0] + last[1];
    int32_t *verts = (int32_t *)A.get((size_t)std::max<int64_t>(nh, 1) * 4);
    HistHdr *hdr = (HistHdr *)A.get((size_t)std::max<int64_t>(nh, 1) * sizeof(HistHdr));
    uint32_t *hcum = (uint32_t *)A.get((size_t)std::max<int64_t>(nh, 1) * HIST_B * HIST_B * 4);
    uint32_t *hrow = (uint32_t *)A.get((size_t)std::max<int64_t>(nh, 1) * (HIST_B + 1) * 4);
    if (!verts || !hdr || !hcum || !hrow) {
        drop();
        A.put(hidx);
        A.put(verts);
        A.put(hdr);
        A.put(hcum);
        A.put(hrow);
        return fail(KAIROS_ERR_OOM, "histograms: device allocation failed (lower the degree cutoff's count)");
    }
    hist_number<<<grid_for(n, 256), 256, 0, s>>>(n, flag, pos, hidx, verts);
    e = cudaGetLastError();
    const size_t smem = (size_t)(HIST_B * HIST_B + HIST_B) * 4;
    if (e == cudaSuccess && nh > 0) {
        const unsigned g = (unsigned)std::min<int64_t>(nh, 65535);
        if (lam_bits == 16) {
            e = cudaFuncSetAttribute(hist_fill<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                hist_fill<uint16_t><<<g, 256, smem, s>>>(nh, verts, c->off, c->t, (const uint16_t *)c->lam, hdr, hcum, hrow);
        } else {
            e = cudaFuncSetAttribute(hist_fill<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                hist_fill<uint32_t><<<g, 256, smem, s>>>(nh, verts, c->off, c->t, (const uint32_t *)c->lam, hdr, hcum, hrow);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    drop();
    A.put(verts);
    if (e != cudaSuccess) {
        A.put(hidx);
        A.put(hdr);
        A.put(hcum);
        A.put(hrow);
        return cuda_fail(e, "histograms");
    }
    c->hidx = hidx;
    c->hhdr = hdr;
    c->hcum = hcum;
    c->hrow = hrow;
    c->n_hist = nh;
    c->hist_min_degree = min_degree;
    return KAIROS_OK;
}

void free_index(const Allocator &A, Csr *c) {
    A.put(c->fidx);
    A.put(c->fence);
    c->fidx = nullptr;
    c->fence = nullptr;
    c->n_fence = 0;
    c->indexed = 0;
}

void free_csr(const Allocator &A, Csr *c) {
    free_index(A, c);
    free_histograms(A, c);
    A.put(c->off);
    A.put(c->dst);
    A.put(c->t);
    A.put(c->lam);
    *c = Csr();
}

}  // namespace kairos
