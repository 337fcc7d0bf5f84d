// The temporal edge-map (Table 2 TemporalEdgeMap, Sec. 4.4) behind earliest arrival
// (Alg. 2), as one persistent cooperative kernel per batch of W query lanes.
//
// State, vertex-major so that one edge feeds the W lanes of its head through contiguous
// words:  arr[v][q]  the label of v in lane q (Alg. 2's t[]), and
//         prev[v][q] the departure bound from which v's list was last scanned in lane q.
// Round r (Alg. 2's while loop): for every frontier vertex u, each lane q with
// thr = arr[u][q] (+1 under StrictlySucceeds, except at the lane's source) below
// lim = min(prev[u][q], tw_q + 1) relaxes exactly the edges (u, v, t, lam) with
// thr <= t < lim and t + lam <= tw_q: arr[v][q] = min(arr[v][q], t + lam) (Update's
// writeMin).  Since the relaxed value does not depend on arr[u], each edge is relaxed at
// most once per lane (prev[u][q] = thr afterwards).  The next frontier is every vertex
// whose label dropped in some lane (the label-correcting reading of Alg. 2's Visited
// flag), deduplicated by a bitmap and appended to a queue by warp ballots.
//
// Selective index (Sec. 3.2, Eqs. 1-3): a vertex with a fence level finds the first edge
// at or after min_q thr and the end of the window by binary search (fence keys, then one
// 32-edge block); an unindexed vertex scans its whole list, filtering by time.
//
// Work shapes: a warp takes 32 frontier vertices, gathers their lane states, computes
// their edge ranges, and walks the concatenated ranges 32 edges at a time (coalesced
// loads, a shuffle per lane group to share each edge with its W lanes).  Ranges longer
// than warp_max_edges are cut into chunk_edges chunks that every warp of the grid claims
// after a grid barrier.  Large frontiers are swept from the bitmap in vertex order.
#include <cuda_runtime.h>

#include "common.cuh"

namespace kairos {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr unsigned long long BARRIER_SPIN_LIMIT = 1ull << 24;  // with 128 ns sleeps: > 2 s

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch (all blocks resident).  Every wait is bounded:
// past the limit the block records KERR_BARRIER_TIMEOUT and leaves.  Returns true when the
// launch may go on (no error recorded anywhere).
__device__ __forceinline__ bool grid_sync(EdgeMapCtr *c, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(&c->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (ld_acquire(&c->bar_gen) == gen) {
                if (++spins > BARRIER_SPIN_LIMIT) {
                    atomicCAS(&c->err, 0, KERR_BARRIER_TIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        *s_flag = __ldcg(&c->err);
    }
    __syncthreads();
    return *s_flag == 0;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// First index i in [0, deg) with tl[i] >= x, through the fence keys F (F[k] = tl[32 k]).
__device__ __forceinline__ uint32_t lower_bound_fenced(const uint32_t *__restrict__ tl, uint32_t deg,
                                                       const uint32_t *__restrict__ F, uint32_t x) {
    uint32_t lo = 0, hi = (deg + FENCE_B - 1) >> FENCE_SHIFT;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&F[mid]) < x) lo = mid + 1; else hi = mid;
    }
    if (lo == 0) return 0;
    const uint32_t b = (lo - 1) << FENCE_SHIFT;  // tl[b] < x
    uint32_t l2 = b + 1, h2 = min(deg, b + FENCE_B);
    while (l2 < h2) {
        uint32_t mid = (l2 + h2) >> 1;
        if (__ldg(&tl[mid]) < x) l2 = mid + 1; else h2 = mid;
    }
    return l2;
}

template <int W>
struct WarpSmem {
    uint32_t thr[32][W];  // per slot and lane: first departure to scan
    uint32_t lim[32][W];  // per slot and lane: scan below this departure
    uint64_t base[32];    // per slot: first edge of its range
    uint32_t start[32];   // per slot: exclusive prefix of range lengths
    uint32_t L[32], H[32];
};

// Per-thread constants of its query lane q = lane % W.
struct LaneReg {
    int q, grp;
    bool on;
    uint32_t tw, lim_cap, strict;
    int32_t src;
};

// Warp-aggregated append of the lanes with `need` to the next frontier queue.
__device__ __forceinline__ void frontier_append(bool need, int32_t v, int lane, int32_t *queue, unsigned *count) {
    const unsigned mask = __ballot_sync(FULL, need);
    if (mask) {
        const int leader = __ffs(mask) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
        base = __shfl_sync(FULL, base, leader);
        if (need) queue[base + __popc(mask & ((1u << lane) - 1u))] = v;
    }
}

// Relax the 32 edges held one per thread (d < 0: none) for every lane: edge k*G + grp is
// taken by the W threads of group grp, thread q deciding for lane q with bounds thr/lim.
template <int W, typename BoundsF>
__device__ __forceinline__ void relax_edges(const EdgeMapArgs &a, const LaneReg &R, int lane, int32_t d, uint32_t tt,
                                            uint32_t ll, int slot, BoundsF bounds, int nxt, int n3,
                                            unsigned long long &relaxed) {
    constexpr int G = 32 / W;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const int ei = k * G + R.grp;
        const int32_t dv = (W == 1) ? d : __shfl_sync(FULL, d, ei);
        const uint32_t tv = (W == 1) ? tt : __shfl_sync(FULL, tt, ei);
        const uint32_t lv = (W == 1) ? ll : __shfl_sync(FULL, ll, ei);
        const int sl = (W == 1) ? slot : __shfl_sync(FULL, slot, ei);
        bool need = false;
        if (dv >= 0) {
            uint32_t th, li;
            bounds(sl, th, li);
            if (th <= tv && tv < li) {
                const uint32_t tau = tv + lv;  // <= TMAX: checked at graph build
                if (tau <= R.tw) {
                    ++relaxed;
                    uint32_t *p = a.arr + (size_t)dv * W + R.q;
                    if (tau < __ldcg(p)) {
                        const uint32_t old = atomicMin(p, tau);
                        if (tau < old) {
                            const uint32_t bit = 1u << (dv & 31);
                            const uint32_t ob = atomicOr(&a.bm[nxt][dv >> 5], bit);
                            need = !(ob & bit);
                        }
                    }
                }
            }
        }
        frontier_append(need, dv, lane, a.queue[nxt], &a.ctr->qcount[n3]);
    }
}

// Expand up to 32 frontier vertices (one per thread, u < 0 for none).
template <int W, typename LamT>
__device__ __forceinline__ void expand(const EdgeMapArgs &a, WarpSmem<W> &S, const LaneReg &R, int lane, int32_t u,
                                       int nxt, int c3, int n3, unsigned long long &relaxed,
                                       unsigned long long &scanned) {
    const LamT *__restrict__ lam = (const LamT *)a.lam;
    // 1. lane states of the 32 slots: thread (k, lane) handles slot (32k + lane) / W, lane q
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const int j = (k * 32 + lane) / W;
        const int32_t uj = (W == 1) ? u : __shfl_sync(FULL, u, j);
        uint32_t th = INF, li = 0;
        if (uj >= 0 && R.on) {
            const size_t idx = (size_t)uj * W + R.q;
            const uint32_t av = __ldcg(&a.arr[idx]);
            if (av != INF) {
                const uint32_t pv = __ldcg(&a.prev[idx]);
                const uint32_t t0 = av + ((R.strict && uj != R.src) ? 1u : 0u);
                const uint32_t l0 = pv < R.lim_cap ? pv : R.lim_cap;
                if (t0 < l0) {
                    th = t0;
                    li = l0;
                    __stcg(&a.prev[idx], t0);
                }
            }
        }
        S.thr[j][R.q] = th;
        S.lim[j][R.q] = li;
        uint32_t mn = th, mx = li;
#pragma unroll
        for (int o = 1; o < W; o <<= 1) {
            mn = min(mn, __shfl_xor_sync(FULL, mn, o));
            mx = max(mx, __shfl_xor_sync(FULL, mx, o));
        }
        if (R.q == 0) {
            S.L[j] = mn;
            S.H[j] = mx;
        }
    }
    __syncwarp();
    // 2. edge range of slot `lane`
    uint32_t len = 0;
    uint64_t base = 0;
    const uint32_t Lm = S.L[lane], Hm = S.H[lane];
    if (u >= 0 && Lm < Hm) {
        const uint64_t o0 = __ldg(&a.off[u]);
        const uint32_t deg = (uint32_t)(__ldg(&a.off[u + 1]) - o0);
        const uint32_t fi = a.fidx ? __ldg(&a.fidx[u]) : NO_FENCE;
        uint32_t lo = 0, hi = deg;
        if (fi != NO_FENCE) {
            lo = lower_bound_fenced(a.t + o0, deg, a.fence + fi, Lm);
            hi = lower_bound_fenced(a.t + o0, deg, a.fence + fi, Hm);
        }
        len = hi - lo;
        base = o0 + lo;
    }
    // 3. long ranges go to the grid-wide chunk list
    if (len > (uint32_t)a.warp_max_edges) {
        const uint32_t CH = (uint32_t)a.chunk_edges;
        const uint32_t nch = (len + CH - 1) / CH;
        const uint32_t e = atomicAdd(&a.ctr->bigcount[c3], 1u);
        const uint32_t cb = atomicAdd(&a.ctr->chunks[c3], nch);
        if (e < a.cap_big && (uint64_t)cb + nch <= a.cap_chunks) {
            a.big[e].base = base;
            a.big[e].len = len;
            a.big[e].chunk_base = cb;
            for (int qq = 0; qq < W; ++qq) {
                a.bigb[((size_t)e * W + qq) * 2] = S.thr[lane][qq];
                a.bigb[((size_t)e * W + qq) * 2 + 1] = S.lim[lane][qq];
            }
            for (uint32_t c = 0; c < nch; ++c) a.chunk_owner[cb + c] = e;
        } else {
            atomicCAS(&a.ctr->err, 0, KERR_CAPACITY);
        }
        len = 0;
    }
    // 4. walk the concatenated short ranges, 32 edges at a time
    const uint32_t incl = warp_incl_scan(len, lane);
    const uint32_t T = __shfl_sync(FULL, incl, 31);
    S.start[lane] = incl - len;
    S.base[lane] = base;
    __syncwarp();
    for (uint32_t c = 0; c < T; c += 32) {
        const uint32_t item = c + lane;
        int32_t d = -1;
        uint32_t tt = 0, ll = 0;
        int slot = 0;
        if (item < T) {
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                if (S.start[j + step] <= item) j += step;
            slot = j;
            const uint64_t e = S.base[j] + (item - S.start[j]);
            d = __ldg(&a.dst[e]);
            tt = __ldg(&a.t[e]);
            ll = (uint32_t)__ldg(&lam[e]);
            ++scanned;
        }
        relax_edges<W>(a, R, lane, d, tt, ll, slot,
                       [&](int sl, uint32_t &th, uint32_t &li) {
                           th = S.thr[sl][R.q];
                           li = S.lim[sl][R.q];
                       },
                       nxt, n3, relaxed);
    }
    __syncwarp();
}

template <int W, typename LamT>
__global__ void __launch_bounds__(EM_THREADS, 2) edgemap_kernel(const EdgeMapArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpSmem<W> &S = reinterpret_cast<WarpSmem<W> *>(smem_raw)[wib];
    const unsigned gw = blockIdx.x * (EM_THREADS / 32) + wib;
    const unsigned nw = gridDim.x * (EM_THREADS / 32);
    const size_t tid = (size_t)blockIdx.x * EM_THREADS + threadIdx.x;
    const size_t nthr = (size_t)gridDim.x * EM_THREADS;
    const int64_t n = a.n;
    const size_t nwords = (size_t)((n + 31) >> 5);
    EdgeMapCtr *C = a.ctr;
    const LamT *__restrict__ lam = (const LamT *)a.lam;

    LaneReg R;
    R.q = lane % W;
    R.grp = lane / W;
    R.on = R.q < a.lanes.nlanes;
    R.tw = a.lanes.tw[R.q];
    R.lim_cap = R.tw + 1u;
    R.strict = (a.lanes.strict_mask >> R.q) & 1u;
    R.src = a.lanes.src[R.q];
    unsigned long long relaxed = 0, scanned = 0;
    unsigned reached = 0;

    // ---- initial labels (Alg. 2: t[x] = window start, t[v] = infinity) ----
    for (size_t i = tid; i < (size_t)n * W; i += nthr) {
        a.arr[i] = INF;
        a.prev[i] = INF;
    }
    for (size_t i = tid; i < nwords; i += nthr) {
        a.bm[0][i] = 0u;
        a.bm[1][i] = 0u;
    }
    if (!grid_sync(C, &s_flag)) return;
    if (blockIdx.x == 0 && threadIdx.x < (unsigned)a.lanes.nlanes) {
        const int qq = threadIdx.x;
        const int32_t s = a.lanes.src[qq];
        a.arr[(size_t)s * W + qq] = a.lanes.ta[qq];
        const uint32_t bit = 1u << (s & 31);
        const uint32_t old = atomicOr(&a.bm[0][s >> 5], bit);
        if (!(old & bit)) a.queue[0][atomicAdd(&C->qcount[0], 1u)] = s;
    }
    if (!grid_sync(C, &s_flag)) return;

    // ---- rounds ----
    unsigned r = 0;
    for (;; ++r) {
        const int cur = r & 1, nxt = cur ^ 1;
        const int c3 = r % 3, n3 = (r + 1) % 3, p3 = (r + 2) % 3;
        const unsigned F = __ldcg(&C->qcount[c3]);
        if (F == 0) break;
        if (r >= a.max_rounds) {
            if (tid == 0) atomicCAS(&C->err, 0, KERR_ROUNDS);
            break;
        }
        if (tid == 0) {
            C->qcount[p3] = 0;
            C->bigcount[n3] = 0;
            C->chunks[n3] = 0;
            C->chunk_next[n3] = 0;
        }
        const bool dense = a.dense_div > 0 && (int64_t)F * a.dense_div > n;
        if (!dense) {
            for (unsigned b = gw * 32; b < F; b += nw * 32) {
                const unsigned i = b + lane;
                const int32_t u = (i < F) ? __ldcg(&a.queue[cur][i]) : -1;
                if (u >= 0) atomicAnd(&a.bm[cur][u >> 5], ~(1u << (u & 31)));
                expand<W, LamT>(a, S, R, lane, u, nxt, c3, n3, relaxed, scanned);
            }
        } else {
            // sweep the bitmap in vertex order; ballot-compact each 1024-vertex stripe
            for (size_t wb = (size_t)gw * 32; wb < nwords; wb += (size_t)nw * 32) {
                const size_t w = wb + lane;
                const uint32_t bits = (w < nwords) ? __ldcg(&a.bm[cur][w]) : 0u;
                if (bits) a.bm[cur][w] = 0u;
                const uint32_t cnt = __popc(bits);
                const uint32_t incl = warp_incl_scan(cnt, lane);
                const uint32_t pre = incl - cnt;
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                for (uint32_t b = 0; b < total; b += 32) {
                    const uint32_t k = b + lane;
                    int j = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const uint32_t pj = __shfl_sync(FULL, pre, j + step);
                        if (pj <= k) j += step;
                    }
                    const uint32_t bj = __shfl_sync(FULL, bits, j);
                    const uint32_t pj = __shfl_sync(FULL, pre, j);
                    int32_t u = -1;
                    if (k < total) u = (int32_t)((wb + j) * 32 + __fns(bj, 0, (int)(k - pj) + 1));
                    expand<W, LamT>(a, S, R, lane, u, nxt, c3, n3, relaxed, scanned);
                }
            }
        }
        if (!grid_sync(C, &s_flag)) return;

        // split ranges: every warp claims chunks
        const unsigned nch = __ldcg(&C->chunks[c3]);
        if (nch > 0) {
            for (;;) {
                unsigned c = 0;
                if (lane == 0) c = atomicAdd(&C->chunk_next[c3], 1u);
                c = __shfl_sync(FULL, c, 0);
                if (c >= nch || c >= a.cap_chunks) break;
                const uint32_t e = __ldcg(&a.chunk_owner[c]);
                if (e >= a.cap_big) continue;
                const uint64_t bbase = __ldcg((const unsigned long long *)&a.big[e].base);
                const uint32_t blen = __ldcg(&a.big[e].len);
                const uint32_t bcb = __ldcg(&a.big[e].chunk_base);
                if (c < bcb) continue;
                const uint32_t st = (c - bcb) * (uint32_t)a.chunk_edges;
                if (st >= blen) continue;
                const uint32_t cnt = min((uint32_t)a.chunk_edges, blen - st);
                const uint32_t th = __ldcg(&a.bigb[((size_t)e * W + R.q) * 2]);
                const uint32_t li = __ldcg(&a.bigb[((size_t)e * W + R.q) * 2 + 1]);
                for (uint32_t i = 0; i < cnt; i += 32) {
                    const uint32_t item = i + lane;
                    int32_t d = -1;
                    uint32_t tt = 0, ll = 0;
                    if (item < cnt) {
                        const uint64_t ed = bbase + st + item;
                        d = __ldg(&a.dst[ed]);
                        tt = __ldg(&a.t[ed]);
                        ll = (uint32_t)__ldg(&lam[ed]);
                        ++scanned;
                    }
                    relax_edges<W>(a, R, lane, d, tt, ll, 0,
                                   [&](int, uint32_t &x, uint32_t &y) {
                                       x = th;
                                       y = li;
                                   },
                                   nxt, n3, relaxed);
                }
            }
            if (!grid_sync(C, &s_flag)) return;
        }
    }

    // ---- read out: out[row_q][v] = label (mirrored back for latest departure) ----
    for (size_t i = tid; i < (size_t)n * W; i += nthr) {
        // nthr is a multiple of W, so this thread always sees lane R.q
        if (!R.on) continue;
        const size_t v = i / W;
        const uint32_t x = __ldcg(&a.arr[i]);
        reached += (x != INF);
        if (a.out) {
            const bool mir = (a.lanes.mirror_mask >> R.q) & 1u;
            const uint32_t y = (mir && x != INF) ? TMAX - x : x;
            if (!(a.out_is_arr && !mir)) a.out[a.lanes.row[R.q] * a.out_stride + (int64_t)v] = y;
        }
    }
    // ---- counters ----
#pragma unroll
    for (int o = W; o < 32; o <<= 1) {
        relaxed += __shfl_xor_sync(FULL, relaxed, o);
        reached += __shfl_xor_sync(FULL, reached, o);
    }
    unsigned long long sc = scanned;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) sc += __shfl_xor_sync(FULL, sc, o);
    if (lane < W && R.on) {
        atomicAdd(&C->relaxed[lane], relaxed);
        atomicAdd(&C->reached[lane], reached);
    }
    if (lane == 0) atomicAdd(&C->scanned, sc);
    if (tid == 0) C->rounds = r;
}

template <int W, typename LamT>
cudaError_t launch_t(const EdgeMapArgs &a, int grid, cudaStream_t s) {
    const size_t smem = sizeof(WarpSmem<W>) * (EM_THREADS / 32);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(edgemap_kernel<W, LamT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((void *)edgemap_kernel<W, LamT>, dim3(grid), dim3(EM_THREADS), args, smem, s);
}

template <int W, typename LamT>
int max_blocks_t() {
    const size_t smem = sizeof(WarpSmem<W>) * (EM_THREADS / 32);
    if (cudaFuncSetAttribute(edgemap_kernel<W, LamT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, edgemap_kernel<W, LamT>, EM_THREADS, smem) != cudaSuccess)
        return 0;
    return nb;
}

template <typename LamT>
cudaError_t launch_l(const EdgeMapArgs &a, int lanes, int grid, cudaStream_t s) {
    switch (lanes) {
        case 1: return launch_t<1, LamT>(a, grid, s);
        case 2: return launch_t<2, LamT>(a, grid, s);
        case 4: return launch_t<4, LamT>(a, grid, s);
        case 8: return launch_t<8, LamT>(a, grid, s);
        case 16: return launch_t<16, LamT>(a, grid, s);
        case 32: return launch_t<32, LamT>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename LamT>
int max_blocks_l(int lanes) {
    switch (lanes) {
        case 1: return max_blocks_t<1, LamT>();
        case 2: return max_blocks_t<2, LamT>();
        case 4: return max_blocks_t<4, LamT>();
        case 8: return max_blocks_t<8, LamT>();
        case 16: return max_blocks_t<16, LamT>();
        case 32: return max_blocks_t<32, LamT>();
        default: return 0;
    }
}

}  // namespace

size_t edgemap_smem_bytes(int lanes) {
    switch (lanes) {
        case 1: return sizeof(WarpSmem<1>) * (EM_THREADS / 32);
        case 2: return sizeof(WarpSmem<2>) * (EM_THREADS / 32);
        case 4: return sizeof(WarpSmem<4>) * (EM_THREADS / 32);
        case 8: return sizeof(WarpSmem<8>) * (EM_THREADS / 32);
        case 16: return sizeof(WarpSmem<16>) * (EM_THREADS / 32);
        case 32: return sizeof(WarpSmem<32>) * (EM_THREADS / 32);
        default: return 0;
    }
}

cudaError_t edgemap_launch(const EdgeMapArgs &a, int lanes, int lam_bits, int grid, cudaStream_t s) {
    return lam_bits == 16 ? launch_l<uint16_t>(a, lanes, grid, s) : launch_l<uint32_t>(a, lanes, grid, s);
}

int edgemap_max_grid(int lanes, int lam_bits, int *blocks_per_sm_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    int nb = lam_bits == 16 ? max_blocks_l<uint16_t>(lanes) : max_blocks_l<uint32_t>(lanes);
    if (blocks_per_sm_out) *blocks_per_sm_out = nb;
    return nb * sms;
}

}  // namespace kairos
