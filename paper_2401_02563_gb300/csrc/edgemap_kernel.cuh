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
// Work shapes: a warp takes 32 frontier vertices and gathers their W lane states with
// coalesced row loads (thread per lane), keeping per vertex the mask of lanes with work.
// Edges are then thread-per-edge, K_EDGES independent edges per thread per step (coalesced
// loads, several misses in flight), each looping over its source's active lanes only.
// Ranges up to warp_max_edges are walked by the warp that found them, concatenated;
// longer ones are cut into chunk_edges chunks.  Within a round, warps claim batches of 32
// frontier vertices from a counter and, once none is left, claim chunks as they are
// published (release/acquire on the chunk's owner word), so one grid barrier ends the
// round.  Large frontiers are swept from the bitmap in vertex order.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "grid_sync.cuh"
#include "hist.cuh"

namespace kairos {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;


__device__ __forceinline__ bool grid_sync(EdgeMapCtr *c, int *s_flag, unsigned long long limit) {
    return kairos::grid_sync(c, s_flag, limit, KERR_BARRIER_TIMEOUT);
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Lower bounds of two keys in one sorted array, 8-ary: each step loads 7 pivots per key (all
// in flight together) and keeps the eighth of the range that holds the answer, so a chain of
// about log8(n) dependent loads replaces log2(n).  On entry and throughout, the answer for x
// lies in [lx, hx]: A[i] < x for i < lx, and hx is the end or A[hx] >= x (same for y).  On
// return lx (ly) is the first index with A[i] >= x (y), or the end.
__device__ __forceinline__ void lower_bound2_kary(const uint32_t *__restrict__ A, uint32_t &lx, uint32_t hx, uint32_t x,
                                                  uint32_t &ly, uint32_t hy, uint32_t y) {
    while (hx - lx > 8 || hy - ly > 8) {
        const uint32_t nx = hx - lx, ny = hy - ly;
        const bool ax = nx > 8, ay = ny > 8;
        uint32_t cx = 0, cy = 0;
        uint32_t vx[7], vy[7];
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            vx[j - 1] = ax ? __ldg(&A[lx + (uint32_t)(((uint64_t)nx * j) >> 3)]) : 0u;
            vy[j - 1] = ay ? __ldg(&A[ly + (uint32_t)(((uint64_t)ny * j) >> 3)]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            cx += vx[j] < x;
            cy += vy[j] < y;
        }
        if (ax) {
            // pivots below x form a prefix: the answer is past pivot cx and at most pivot cx + 1
            const uint32_t l2 = cx ? lx + (uint32_t)(((uint64_t)nx * cx) >> 3) + 1u : lx;
            if (cx < 7) hx = lx + (uint32_t)(((uint64_t)nx * (cx + 1)) >> 3);
            lx = l2;
        }
        if (ay) {
            const uint32_t l2 = cy ? ly + (uint32_t)(((uint64_t)ny * cy) >> 3) + 1u : ly;
            if (cy < 7) hy = ly + (uint32_t)(((uint64_t)ny * (cy + 1)) >> 3);
            ly = l2;
        }
    }
    // at most 8 candidates per key: the answer is lx plus the count of those below x
    uint32_t cx = 0, cy = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool inx = lx + j < hx, iny = ly + j < hy;
        const uint32_t a = inx ? __ldg(&A[lx + j]) : 0u;
        const uint32_t b = iny ? __ldg(&A[ly + j]) : 0u;
        cx += (inx && a < x);
        cy += (iny && b < y);
    }
    lx += cx;
    ly += cy;
}

// First indices i in [0, deg) with tl[i] >= x and with tl[i] >= y (deg if none), through the
// fence keys F (F[k] = tl[32 k]): the fences first, then one 32-edge block.
__device__ __forceinline__ void lower_bound2_fenced(const uint32_t *__restrict__ tl, uint32_t deg,
                                                    const uint32_t *__restrict__ F, uint32_t x, uint32_t y,
                                                    uint32_t &rx, uint32_t &ry) {
    const uint32_t nf = (deg + FENCE_B - 1) >> FENCE_SHIFT;
    uint32_t lx = 0, ly = 0;
    lower_bound2_kary(F, lx, nf, x, ly, nf, y);
    // fence k = lx is the first at or above x: the answer lies in (32 (k - 1), min(32 k, deg)]
    // (k == 0: it is 0, the first edge)
    uint32_t bx = lx ? ((lx - 1) << FENCE_SHIFT) + 1 : 0, ex = lx ? min(deg, ((lx - 1) << FENCE_SHIFT) + FENCE_B) : 0;
    uint32_t by = ly ? ((ly - 1) << FENCE_SHIFT) + 1 : 0, ey = ly ? min(deg, ((ly - 1) << FENCE_SHIFT) + FENCE_B) : 0;
    lower_bound2_kary(tl, bx, ex, x, by, ey, y);
    rx = bx;
    ry = by;
}

template <int W>
struct WarpSmem {
    uint32_t thr[32][W];  // per slot and lane: first departure to scan
    uint32_t lim[32][W];  // per slot and lane: scan below this departure
    uint32_t act[32];     // per slot: lanes whose interval [thr, lim) is non-empty
    uint64_t base[32];    // per slot: first edge of its range
    uint32_t start[32];   // per slot: exclusive prefix of range lengths
    uint32_t L[32], H[32];
    uint32_t bthr[W], blim[W];  // lane bounds of the split range being walked
    // the same bounds as sorted breakpoints: lanes {q : thr_q <= t < lim_q} = bmask[i]
    // for bkey[i] <= t < bkey[i + 1] (bkey[-1] = -inf, mask 0)
    uint32_t bkey[2 * W], bmask[2 * W];
    unsigned long long phase[8];  // diagnostics: cycles per phase (lane 0)
};

// Per-warp phase timer (diagnostics): adds the cycles since the last mark to phase p.  The
// sums live in shared memory (lane 0 writes them), so that only the flag and the last
// timestamp occupy registers.
struct PhaseClock {
    bool on;
    long long last;
    unsigned long long *acc;  // 8 per warp, shared memory
    __device__ __forceinline__ void init(bool enable, unsigned long long *sacc, int lane) {
        on = enable;
        acc = sacc;
        last = on ? clock64() : 0;
        if (on && lane == 0)
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = 0;
    }
    __device__ __forceinline__ void mark(int p) {
        if (on) {
            const long long now = clock64();
            if ((threadIdx.x & 31) == 0) acc[p] += (unsigned long long)(now - last);
            last = now;
        }
    }
};

// Per-thread constants of its query lane q = lane % W.
struct LaneReg {
    int q, grp;
    bool on;
    uint32_t tw, lim_cap, strict;
    int32_t src;
};

struct BlockSmem {
    uint32_t tw[MAX_LANES];   // window end per lane
    uint32_t cnt[MAX_LANES];  // relaxations per lane (lanes > 1)
    uint32_t twmax;           // latest window end over the launch's lanes
    int flag;
};

constexpr int K_EDGES = 4;  // independent edges per thread per step

// Sorted breakpoints of the lane intervals [thr_q, lim_q) of the chunk being walked, and
// for each breakpoint the lanes whose interval contains it (so that for departure t the
// candidate lanes are bmask[i] with bkey[i] <= t < bkey[i+1]).  Inactive lanes contribute
// keys INF.  A bitonic sort of the 2W keys, W <= 32, two per thread.
template <int W>
__device__ __forceinline__ void build_breakpoints(WarpSmem<W> &S, int lane, uint32_t act) {
    constexpr int N = 2 * W;  // keys; thread `lane` holds keys lane and lane + 32 when present
    uint32_t k0 = INF, k1 = INF;
    if (lane < W) {
        const bool on = (act >> lane) & 1u;
        k0 = on ? S.bthr[lane] : INF;
        k1 = on ? S.blim[lane] : INF;
    }
    // element index e = lane (k0) for e < 32 or lane + 32 (k1); with N <= 32 both live in
    // k0 of lanes [0, N): rearrange so that element e sits in thread e % 32, slot e / 32
    uint32_t x0, x1;
    if constexpr (N <= 32) {
        // element e: e < W -> thr of lane e, else lim of lane e - W
        const uint32_t a0 = __shfl_sync(0xFFFFFFFFu, k0, lane % W);
        const uint32_t a1 = __shfl_sync(0xFFFFFFFFu, k1, lane % W);
        x0 = lane < W ? a0 : (lane < N ? a1 : INF);
        x1 = INF;
    } else {  // W == 32: thread lane holds thr (element lane) and lim (element lane + 32)
        x0 = k0;
        x1 = k1;
    }
    // bitonic sort of 64 slots (32 threads x 2), ascending by element index lane + 32 * slot
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride == 32) {  // partners are the two slots of the same thread
                const bool up = (lane & size) == 0 || size == 64;
                const uint32_t lo = min(x0, x1), hi = max(x0, x1);
                x0 = up ? lo : hi;
                x1 = up ? hi : lo;
            } else {
#pragma unroll
                for (int slot = 0; slot < 2; ++slot) {
                    uint32_t &x = slot ? x1 : x0;
                    const int e = lane + 32 * slot;
                    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, stride);
                    const bool up = (e & size) == 0;
                    const bool lower = (e & stride) == 0;
                    x = (lower == up) ? min(x, y) : max(x, y);
                }
            }
        }
    }
    // masks: lanes q with thr_q <= key < lim_q
    if constexpr (N <= 32) {
        if (lane < N) {
            uint32_t m = 0;
            for (int q = 0; q < W; ++q)
                if (((act >> q) & 1u) && S.bthr[q] <= x0 && x0 < S.blim[q]) m |= 1u << q;
            S.bkey[lane] = x0;
            S.bmask[lane] = m;
        }
    } else {
        uint32_t m0 = 0, m1 = 0;
        for (int q = 0; q < W; ++q) {
            if (!((act >> q) & 1u)) continue;
            const uint32_t th = S.bthr[q], li = S.blim[q];
            if (th <= x0 && x0 < li) m0 |= 1u << q;
            if (th <= x1 && x1 < li) m1 |= 1u << q;
        }
        S.bkey[lane] = x0;
        S.bmask[lane] = m0;
        S.bkey[lane + 32] = x1;
        S.bmask[lane + 32] = m1;
    }
    __syncwarp();
}

// Append the (up to K_EDGES) vertices this thread marked to the next frontier queue: one
// warp-wide prefix sum and one atomic per warp.
__device__ __forceinline__ void frontier_append_k(uint32_t needmask, const int32_t (&d)[K_EDGES], int lane,
                                                  int32_t *queue, unsigned *count) {
    const uint32_t c = __popc(needmask);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total == 0) return;
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(count, total);
    base = __shfl_sync(FULL, base, 31) + incl - c;
#pragma unroll
    for (int k = 0; k < K_EDGES; ++k)
        if ((needmask >> k) & 1u) queue[base++] = d[k];
}

// Relax K edges per thread (d < 0: none).  Edge k of this thread comes from a slot whose
// active lanes are act(k) and whose bounds for lane q are bounds(k, q, thr, lim).
// A lane whose (possibly stale, never too low) copy of the head's label is above the
// arrival issues a fire-and-forget atomic minimum; the head then gets one frontier-bitmap
// test-and-set per edge.  A head marked although another thread lowered it first is
// harmless: its next expansion finds every interval empty.
template <int W, int MODE, typename ActF, typename BoundsF>
__device__ __forceinline__ void relax_k(const EdgeMapArgs &a, const int32_t (&d)[K_EDGES], const uint32_t (&tt)[K_EDGES],
                                        const uint32_t (&ll)[K_EDGES], ActF actf, BoundsF bounds, BlockSmem &B,
                                        unsigned long long &cnt1, int lane, int nxt, int n3, uint32_t &hit) {
    uint32_t mark = 0;  // bit k: edge k lowered its head in some lane
    if constexpr (MODE == 1) {
        // every usable edge lowers its head unconditionally (fire-and-forget) and marks it
        // in the next bitmap (fire-and-forget): no load, no wait, no queue
#pragma unroll
        for (int k = 0; k < K_EDGES; ++k) {
            if (d[k] < 0) continue;
            const uint32_t tau = tt[k] + ll[k];
            uint32_t cand = 0;
            if constexpr (W == 1) {
                uint32_t th, li;
                bounds(k, 0, th, li);
                cand = (actf(k) && th <= tt[k] && tt[k] < li && tau <= B.tw[0]) ? 1u : 0u;
                cnt1 += cand;
            } else {
                uint32_t act = actf(k);
                while (act) {
                    const int q = __ffs(act) - 1;
                    act &= act - 1;
                    uint32_t th, li;
                    bounds(k, q, th, li);
                    if (th <= tt[k] && tt[k] < li && tau <= B.tw[q]) cand |= 1u << q;
                }
                if (a.count_relaxed)
                    for (uint32_t c2 = cand; c2; c2 &= c2 - 1) atomicAdd(&B.cnt[__ffs(c2) - 1], 1u);
            }
            if (cand) {
                uint32_t *row = a.arr + (size_t)d[k] * W;
                for (uint32_t c2 = cand; c2; c2 &= c2 - 1) atomicMin(row + (__ffs(c2) - 1), tau);
                atomicOr(&a.bm[nxt][d[k] >> 5], 1u << (d[k] & 31));
                hit |= cand;
            }
        }
        return;
    } else {
    if constexpr (W == 1) {
        bool ok[K_EDGES];
        uint32_t cur[K_EDGES];
#pragma unroll
        for (int k = 0; k < K_EDGES; ++k) {
            uint32_t th, li;
            bounds(k, 0, th, li);
            ok[k] = d[k] >= 0 && actf(k) && th <= tt[k] && tt[k] < li && tt[k] + ll[k] <= B.tw[0];
            cnt1 += ok[k];  // a register add: kept even when statistics are not requested
        }
#pragma unroll
        for (int k = 0; k < K_EDGES; ++k) cur[k] = ok[k] ? __ldcg(a.arr + d[k]) : 0u;
#pragma unroll
        for (int k = 0; k < K_EDGES; ++k) {
            const uint32_t tau = tt[k] + ll[k];
            if (ok[k] && tau < cur[k]) {
                atomicMin(a.arr + d[k], tau);  // result unused: a reduction
                mark |= 1u << k;
                hit = 1u;
            }
        }
    } else {
        if constexpr (MODE == 2) {
            // candidate lanes of each edge from the time bounds alone (shared memory)
            uint32_t cand_k[K_EDGES];
    #pragma unroll
            for (int k = 0; k < K_EDGES; ++k) {
                uint32_t cand = 0;
                const uint32_t tau = tt[k] + ll[k];
                if (d[k] >= 0) {
                    uint32_t act = actf(k);
                    while (act) {
                        const int q = __ffs(act) - 1;
                        act &= act - 1;
                        uint32_t th, li;
                        bounds(k, q, th, li);
                        if (th <= tt[k] && tt[k] < li && tau <= B.tw[q]) cand |= 1u << q;
                    }
                    if (a.count_relaxed)
                        for (uint32_t c2 = cand; c2; c2 &= c2 - 1) atomicAdd(&B.cnt[__ffs(c2) - 1], 1u);
                }
                cand_k[k] = cand;
            }
            // the head-row segments holding candidates, one per edge per pass: every edge of the
            // thread has a segment load in flight at once, and the passes stop when no edge has
            // candidates left (cost follows the candidates, not the lane width)
            constexpr int SEGL = (W >= 4) ? 4 : W;
            uint32_t rem[K_EDGES];
    #pragma unroll
            for (int k = 0; k < K_EDGES; ++k) rem[k] = cand_k[k];
            for (;;) {
                bool any = false;
                uint32_t v4[K_EDGES][SEGL];
                int sgk[K_EDGES];
    #pragma unroll
                for (int k = 0; k < K_EDGES; ++k) {
                    sgk[k] = -1;
                    if (rem[k]) {
                        any = true;
                        const int sg = (__ffs(rem[k]) - 1) / SEGL;
                        sgk[k] = sg;
                        const uint32_t *row = a.arr + (size_t)d[k] * W + sg * SEGL;
                        if constexpr (SEGL == 4) {
                            const uint4 v = *reinterpret_cast<const uint4 *>(row);  // may be stale: never below
                            v4[k][0] = v.x;
                            v4[k][1] = v.y;
                            v4[k][2] = v.z;
                            v4[k][3] = v.w;
                        } else {
                            const uint2 v = *reinterpret_cast<const uint2 *>(row);
                            v4[k][0] = v.x;
                            v4[k][1] = v.y;
                        }
                    }
                }
                if (!any) break;
    #pragma unroll
                for (int k = 0; k < K_EDGES; ++k) {
                    if (sgk[k] < 0) continue;
                    const uint32_t tau = tt[k] + ll[k];
                    uint32_t *row = a.arr + (size_t)d[k] * W + sgk[k] * SEGL;
    #pragma unroll
                    for (int j = 0; j < SEGL; ++j) {
                        const int q = sgk[k] * SEGL + j;
                        if (((rem[k] >> q) & 1u) && tau < v4[k][j]) {
                            atomicMin(row + j, tau);  // result unused: a reduction
                            mark |= 1u << k;
                            hit |= 1u << q;
                        }
                    }
                    const uint32_t segbits = (SEGL == 32) ? 0xFFFFFFFFu : (((1u << SEGL) - 1u) << (sgk[k] * SEGL));
                    rem[k] &= ~segbits;
                }
            }
        } else {
            // candidate lanes of each edge from the time bounds, then the head's state-row
            // segments holding them, fetched with independent vector loads
            constexpr int SEG = (W >= 4) ? 4 : W;  // lanes per load
            constexpr int NSEG = W / SEG;
            constexpr uint32_t SEGMASK = (SEG == 32) ? 0xFFFFFFFFu : ((1u << SEG) - 1u);
    #pragma unroll
            for (int k = 0; k < K_EDGES; ++k) {
                uint32_t cand = 0;
                const uint32_t tau = tt[k] + ll[k];
                if (d[k] >= 0) {
                    uint32_t act = actf(k);
                    while (act) {
                        const int q = __ffs(act) - 1;
                        act &= act - 1;
                        uint32_t th, li;
                        bounds(k, q, th, li);
                        if (th <= tt[k] && tt[k] < li && tau <= B.tw[q]) cand |= 1u << q;
                    }
                    if (a.count_relaxed)
                        for (uint32_t c2 = cand; c2; c2 &= c2 - 1) atomicAdd(&B.cnt[__ffs(c2) - 1], 1u);
                }
                if (cand) {
                    uint32_t *row = a.arr + (size_t)d[k] * W;
                    uint32_t cur[W];
    #pragma unroll
                    for (int sg = 0; sg < NSEG; ++sg) {
                        if ((cand >> (sg * SEG)) & SEGMASK) {
                            if constexpr (SEG == 4) {
                                const uint4 v = *reinterpret_cast<const uint4 *>(row + sg * 4);  // may be stale: never below
                                cur[sg * 4] = v.x;
                                cur[sg * 4 + 1] = v.y;
                                cur[sg * 4 + 2] = v.z;
                                cur[sg * 4 + 3] = v.w;
                            } else {
                                const uint2 v = *reinterpret_cast<const uint2 *>(row);
                                cur[0] = v.x;
                                cur[1] = v.y;
                            }
                        } else {
    #pragma unroll
                            for (int j = 0; j < SEG; ++j) cur[sg * SEG + j] = 0u;
                        }
                    }
    #pragma unroll
                    for (int q = 0; q < W; ++q)
                        if (((cand >> q) & 1u) && tau < cur[q]) {
                            atomicMin(row + q, tau);  // result unused: a reduction
                            mark |= 1u << k;
                            hit |= 1u << q;
                        }
                }
            }
        }
    }
    // one bitmap test-and-set per marked edge, all in flight together
    uint32_t old[K_EDGES];
#pragma unroll
    for (int k = 0; k < K_EDGES; ++k)
        old[k] = ((mark >> k) & 1u) ? atomicOr(&a.bm[nxt][d[k] >> 5], 1u << (d[k] & 31)) : 0xFFFFFFFFu;
    uint32_t need = 0;
#pragma unroll
    for (int k = 0; k < K_EDGES; ++k)
        if (!((old[k] >> (d[k] & 31)) & 1u)) need |= 1u << k;
    frontier_append_k(need, d, lane, a.queue[nxt], &a.ctr->qcount[n3].v);
    }
}

// Expand up to 32 frontier vertices (one per thread, u < 0 for none).
template <int W, int MODE, typename LamT>
__device__ __forceinline__ void expand(const EdgeMapArgs &a, WarpSmem<W> &S, BlockSmem &B, const LaneReg &R, int lane,
                                       int32_t u, int nxt, int c3, int n3, unsigned long long &cnt1,
                                       unsigned long long &scanned, PhaseClock &pc, uint32_t &hit) {
    const LamT *__restrict__ lam = (const LamT *)a.lam;
    // 1. lane states of the 32 slots: thread (k, lane) handles slot (32k + lane) / W, lane q.
    // G slots at a time: their label loads, then their bound loads, are in flight together.
    constexpr int G = W < 4 ? W : 4;
    const int nvalid = __popc(__ballot_sync(FULL, u >= 0));  // the valid slots form a prefix
#pragma unroll 1
    for (int k0 = 0; k0 < W; k0 += G) {  // kept rolled: measured faster than unrolled
        if ((k0 * 32) / W >= nvalid) break;  // the remaining slots are empty (never read)
        int32_t uj[G];
        uint32_t av[G], pv[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int j = ((k0 + i) * 32 + lane) / W;
            uj[i] = (W == 1) ? u : __shfl_sync(FULL, u, j);
            av[i] = (uj[i] >= 0 && R.on) ? __ldcg(&a.arr[(size_t)uj[i] * W + R.q]) : INF;
        }
#pragma unroll
        for (int i = 0; i < G; ++i) pv[i] = (av[i] != INF) ? __ldcg(&a.prev[(size_t)uj[i] * W + R.q]) : INF;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int j = ((k0 + i) * 32 + lane) / W;
            uint32_t th = INF, li = 0;
            if (av[i] != INF) {
                const uint32_t t0 = av[i] + ((R.strict && uj[i] != R.src) ? 1u : 0u);
                const uint32_t l0 = pv[i] < R.lim_cap ? pv[i] : R.lim_cap;
                if (t0 < l0) {
                    th = t0;
                    li = l0;
                    __stcg(&a.prev[(size_t)uj[i] * W + R.q], t0);
                }
            }
            S.thr[j][R.q] = th;
            S.lim[j][R.q] = li;
            const unsigned on = __ballot_sync(FULL, th < li);
            uint32_t mn = th, mx = li;
#pragma unroll
            for (int o = 1; o < W; o <<= 1) {
                mn = min(mn, __shfl_xor_sync(FULL, mn, o));
                mx = max(mx, __shfl_xor_sync(FULL, mx, o));
            }
            if (R.q == 0) {
                S.L[j] = mn;
                S.H[j] = mx;
                S.act[j] = (W == 32) ? on : ((on >> (lane & ~(W - 1))) & ((1u << W) - 1u));
            }
        }
    }
    __syncwarp();
    pc.mark(0);
    // 2. edge range of slot `lane`: [lower_bound(min thr), lower_bound(max lim)) when the
    // vertex is indexed, its whole list otherwise
    uint32_t len = 0;
    uint64_t base = 0;
    const uint32_t Lm = S.L[lane], Hm = S.H[lane];
    if (u >= 0 && Lm < Hm) {
        const uint64_t o0 = __ldg(&a.off[u]);
        const uint32_t deg = (uint32_t)(__ldg(&a.off[u + 1]) - o0);
        const uint32_t fi = a.fidx ? __ldg(&a.fidx[u]) : NO_FENCE;
        uint32_t lo = 0, hi = deg;
        bool search = fi != NO_FENCE;
        if (search && a.select_permille > 0 && a.hidx) {
            // Eq. 3: search the index when the estimated selectivity of the departure interval
            // (and the latest window end) is at most theta_sel, else scan the whole list
            const uint32_t hx = __ldg(&a.hidx[u]);
            if (hx != NO_HIST) {
                const uint64_t k = hist_estimate(a.hhdr[hx], a.hcum + (size_t)hx * HIST_B * HIST_B, Lm, (uint64_t)Hm - 1,
                                                 B.twmax);
                search = 1000ull * k <= (uint64_t)a.select_permille * deg;
            }
        }
        if (search) lower_bound2_fenced(a.t + o0, deg, a.fence + fi, Lm, Hm, lo, hi);
        len = hi - lo;
        base = o0 + lo;
    }
    pc.mark(1);
    // 3. ranges longer than warp_max_edges go to the grid-wide chunk list (one pair of
    // atomics per warp)
    const bool isbig = len > (uint32_t)a.warp_max_edges;
    const unsigned bmask = __ballot_sync(FULL, isbig);
    if (bmask) {
        const uint32_t CH = (uint32_t)a.chunk_edges;
        const uint32_t nch = isbig ? (len + CH - 1) / CH : 0u;
        const uint32_t chincl = warp_incl_scan(nch, lane);
        const uint32_t chtot = __shfl_sync(FULL, chincl, 31);
        unsigned e0 = 0, c0 = 0;
        if (lane == 0) {
            e0 = atomicAdd(&a.ctr->bigcount[c3].v, (unsigned)__popc(bmask));
            c0 = atomicAdd(&a.ctr->chunks[c3].v, chtot);
        }
        e0 = __shfl_sync(FULL, e0, 0);
        c0 = __shfl_sync(FULL, c0, 0);
        if (isbig) {
            const uint32_t e = e0 + __popc(bmask & ((1u << lane) - 1u));
            const uint32_t cb = c0 + chincl - nch;
            if (e < a.cap_big && (uint64_t)cb + nch <= a.cap_chunks) {
                BigEntry be;
                be.base = base;
                be.len = len;
                be.chunk_base = cb;
                be.act = S.act[lane];
                be.pad = 0;
                a.big[e] = be;
                for (int qq = 0; qq < W; ++qq) {
                    a.bigb[((size_t)e * W + qq) * 2] = S.thr[lane][qq];
                    a.bigb[((size_t)e * W + qq) * 2 + 1] = S.lim[lane][qq];
                }
                __threadfence();  // the entry is visible before any chunk names it
                for (uint32_t c = 0; c < nch; ++c) st_release(&a.chunk_owner[cb + c], e);
            } else {
                atomicCAS(&a.ctr->err, 0, KERR_CAPACITY);
            }
            len = 0;
        }
    }
    pc.mark(2);
    // 4. walk the concatenated short ranges, K_EDGES x 32 edges per step
    const uint32_t incl = warp_incl_scan(len, lane);
    const uint32_t T = __shfl_sync(FULL, incl, 31);
    S.start[lane] = incl - len;
    S.base[lane] = base;
    __syncwarp();
    for (uint32_t c = 0; c < T; c += 32 * K_EDGES) {
        int32_t d[K_EDGES];
        uint32_t tt[K_EDGES], ll[K_EDGES];
        int sl[K_EDGES];
#pragma unroll
        for (int k = 0; k < K_EDGES; ++k) {
            const uint32_t item = c + k * 32 + lane;
            d[k] = -1;
            tt[k] = 0;
            ll[k] = 0;
            sl[k] = 0;
            if (item < T) {
                int j = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1)
                    if (S.start[j + step] <= item) j += step;
                sl[k] = j;
                const uint64_t e = S.base[j] + (item - S.start[j]);
                d[k] = __ldg(&a.dst[e]);
                tt[k] = __ldg(&a.t[e]);
                ll[k] = (uint32_t)__ldg(&lam[e]);
                ++scanned;
            }
        }
        relax_k<W, MODE>(a, d, tt, ll, [&](int k) { return S.act[sl[k]]; },
                   [&](int k, int q, uint32_t &th, uint32_t &li) {
                       th = S.thr[sl[k]][q];
                       li = S.lim[sl[k]][q];
                   },
                   B, cnt1, lane, nxt, n3, hit);
    }
    __syncwarp();
    pc.mark(3);
}

template <int W, int MODE, typename LamT>
__global__ void __launch_bounds__(EM_THREADS, (W == 1 || W == 16) ? 4 : (W == 32 ? 2 : 3)) edgemap_kernel(const EdgeMapArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockSmem B;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpSmem<W> &S = reinterpret_cast<WarpSmem<W> *>(smem_raw)[wib];
    const size_t tid = (size_t)blockIdx.x * EM_THREADS + threadIdx.x;
    const size_t nthr = (size_t)gridDim.x * EM_THREADS;
    const int64_t n = a.n;
    const size_t nwords = (size_t)((n + 31) >> 5);
    EdgeMapCtr *C = a.ctr;
    const LamT *__restrict__ lam = (const LamT *)a.lam;

    LaneReg R;
    R.q = lane % W;
    R.grp = lane / W;
    R.on = R.q < a.lanes.nlanes && ((a.running_mask >> R.q) & 1u);
    R.tw = a.lanes.tw[R.q];
    R.lim_cap = R.tw + 1u;
    R.strict = (a.lanes.strict_mask >> R.q) & 1u;
    R.src = a.lanes.src[R.q];
    if (threadIdx.x < MAX_LANES) {
        B.tw[threadIdx.x] = a.lanes.tw[threadIdx.x];
        B.cnt[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        uint32_t m = 0;
        for (int q = 0; q < a.lanes.nlanes; ++q) m = max(m, a.lanes.tw[q]);
        B.twmax = m;
    }
    __syncthreads();  // the block's lane constants are read by every warp
    unsigned long long cnt1 = 0, scanned = 0;
    unsigned reached = 0;
    PhaseClock pc;
    pc.init(a.phase_clock != 0, S.phase, lane);

    // ---- initial labels (Alg. 2: t[x] = window start, t[v] = infinity) ----
    if (!a.resume) {
    for (size_t i = tid; i < (size_t)n * W; i += nthr) {
        a.arr[i] = INF;
        a.prev[i] = INF;
    }
    for (size_t i = tid; i < nwords; i += nthr) {
        a.bm[0][i] = 0u;
        a.bm[1][i] = 0u;
    }
    if (!grid_sync(C, &B.flag, a.spin_limit)) return;
    if (blockIdx.x == 0 && threadIdx.x < (unsigned)a.lanes.nlanes && ((a.running_mask >> threadIdx.x) & 1u)) {
        const int qq = threadIdx.x;
        const int32_t s = a.lanes.src[qq];
        a.arr[(size_t)s * W + qq] = a.lanes.ta[qq];
        const uint32_t bit = 1u << (s & 31);
        const uint32_t old = atomicOr(&a.bm[0][s >> 5], bit);
        if (!(old & bit)) a.queue[0][atomicAdd(&C->qcount[0].v, 1u)] = s;
    }
    if (!grid_sync(C, &B.flag, a.spin_limit)) return;
    }

    // ---- rounds ----
    unsigned r = a.round_begin;
    for (; r < a.round_end; ++r) {
        uint32_t hit = 0;  // lanes this thread lowered a label in, this round
        const int cur = r & 1, nxt = cur ^ 1;
        const int c3 = r % 3, n3 = (r + 1) % 3, p3 = (r + 2) % 3;
        // relax_mode 1 keeps no queue: after round 0 the bitmap is the frontier, and a round
        // without usable edges in any lane (active mask 0) ends the launch
        const unsigned F = (MODE == 1 && r > 0) ? (__ldcg(&C->active[p3].v) ? 1u : 0u)
                                                        : __ldcg(&C->qcount[c3].v);
        if (tid == 0 && r <= PROFILE_ROUNDS) {
            C->round_ns[r] = globaltimer();
            if (r > 0) C->round_chunks[r - 1] = __ldcg(&C->chunks[(r + 2) % 3].v);
            if (r < PROFILE_ROUNDS) C->round_frontier[r] = F;
        }
        if (F == 0) break;
        if (r >= a.max_rounds) {
            if (tid == 0) atomicCAS(&C->err, 0, KERR_ROUNDS);
            break;
        }
        if (tid == 0) {
            C->qcount[p3].v = 0;
            C->bigcount[n3].v = 0;
            C->chunks[n3].v = 0;
            C->chunk_next[n3].v = 0;
            C->bnext[n3].v = 0;
            C->bdone[n3].v = 0;
            C->active[n3].v = 0;
        }
        const bool dense = MODE == 1 || (a.dense_div > 0 && (int64_t)F * a.dense_div > n);
        // work of the round: batches of up to 32 queued vertices (or 1024-vertex bitmap
        // stripes), then the chunks that expanding them registered; both claimed dynamically.
        // A small frontier is spread thin (bs vertices per batch, about one batch per warp),
        // so that no warp walks many short ranges one after another while the others wait.
        const unsigned nwarps = gridDim.x * (EM_THREADS / 32);
        const unsigned per = (F + nwarps - 1) / nwarps;
        const unsigned bs = per >= 32 ? 32u : (per < 1 ? 1u : per);
        const unsigned nb = dense ? (unsigned)((nwords + 31) / 32) : (F + bs - 1) / bs;
        for (;;) {
            unsigned b = nb;
            if (lane == 0 && __ldcg(&C->bnext[c3].v) < nb) b = atomicAdd(&C->bnext[c3].v, 1u);
            b = __shfl_sync(FULL, b, 0);
            if (b < nb) {
                if (!dense) {
                    const unsigned i = b * bs + lane;
                    const int32_t u = ((unsigned)lane < bs && i < F) ? __ldcg(&a.queue[cur][i]) : -1;
                    if (u >= 0) atomicAnd(&a.bm[cur][u >> 5], ~(1u << (u & 31)));
                    expand<W, MODE, LamT>(a, S, B, R, lane, u, nxt, c3, n3, cnt1, scanned, pc, hit);
                } else {
                    // ballot-compact the 1024-vertex stripe, 32 vertices at a time
                    const size_t wb = (size_t)b * 32;
                    const size_t w = wb + lane;
                    const uint32_t bits = (w < nwords) ? __ldcg(&a.bm[cur][w]) : 0u;
                    if (bits) a.bm[cur][w] = 0u;
                    const uint32_t cnt = __popc(bits);
                    const uint32_t incl = warp_incl_scan(cnt, lane);
                    const uint32_t pre = incl - cnt;
                    const uint32_t total = __shfl_sync(FULL, incl, 31);
                    for (uint32_t b2 = 0; b2 < total; b2 += 32) {
                        const uint32_t k = b2 + lane;
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
                        expand<W, MODE, LamT>(a, S, B, R, lane, u, nxt, c3, n3, cnt1, scanned, pc, hit);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    __threadfence();  // chunk registrations of this batch precede its completion
                    atomicAdd(&C->bdone[c3].v, 1u);
                }
                continue;
            }
            // all batches are claimed: take the next chunk id, waiting (bounded) until it is
            // published, or until every batch is done and no chunk has that id
            unsigned c = 0, e = NO_OWNER;
            int state = 0;  // 0 wait, 1 work, 2 no more work
            if (lane == 0) {
                // no claim while every registered chunk is taken and no batch can add more
                unsigned backoff = 64;
                unsigned long long spins = 0;
                for (;;) {
                    const unsigned have = __ldcg(&C->chunks[c3].v);
                    if (__ldcg(&C->chunk_next[c3].v) < have) break;
                    if (ld_acquire(&C->bdone[c3].v) >= nb && __ldcg(&C->chunk_next[c3].v) >= __ldcg(&C->chunks[c3].v)) {
                        state = 2;
                        break;
                    }
                    if (__ldcg(&C->err) != 0 || ++spins > a.spin_limit) {
                        if (spins > a.spin_limit) atomicCAS(&C->err, 0, KERR_WAIT_TIMEOUT);
                        state = 2;
                        break;
                    }
                    __nanosleep(backoff);
                    backoff = backoff < 4096 ? 2 * backoff : 4096;
                }
                if (state == 0) c = atomicAdd(&C->chunk_next[c3].v, 1u);
                while (state == 0) {
                    if (c < __ldcg(&C->chunks[c3].v) && c < a.cap_chunks) {
                        e = ld_acquire(&a.chunk_owner[c]);
                        if (e != NO_OWNER) {
                            state = 1;
                            break;
                        }
                    } else if (ld_acquire(&C->bdone[c3].v) >= nb && c >= __ldcg(&C->chunks[c3].v)) {
                        state = 2;
                        break;
                    }
                    if (__ldcg(&C->err) != 0) {
                        state = 2;
                        break;
                    }
                    if (++spins > a.spin_limit) {
                        atomicCAS(&C->err, 0, KERR_WAIT_TIMEOUT);
                        state = 2;
                        break;
                    }
                    __nanosleep(backoff);
                    backoff = backoff < 4096 ? 2 * backoff : 4096;
                }
            }
            state = __shfl_sync(FULL, state, 0);
            pc.mark(4);
            if (state == 2) break;
            c = __shfl_sync(FULL, c, 0);
            e = __shfl_sync(FULL, e, 0);
            if (lane == 0) a.chunk_owner[c] = NO_OWNER;  // free the id for the next round
            if (e >= a.cap_big) continue;
            const uint64_t bbase = __ldcg((const unsigned long long *)&a.big[e].base);
            const uint32_t blen = __ldcg(&a.big[e].len);
            const uint32_t bcb = __ldcg(&a.big[e].chunk_base);
            const uint32_t bact = __ldcg(&a.big[e].act);
            if (c < bcb) continue;
            const uint32_t st = (c - bcb) * (uint32_t)a.chunk_edges;
            if (st >= blen) continue;
            const uint32_t cnt = min((uint32_t)a.chunk_edges, blen - st);
            if (lane < W) {
                S.bthr[lane] = __ldcg(&a.bigb[((size_t)e * W + lane) * 2]);
                S.blim[lane] = __ldcg(&a.bigb[((size_t)e * W + lane) * 2 + 1]);
            }
            __syncwarp();
            if (W > 1) build_breakpoints<W>(S, lane, bact);
            for (uint32_t i = 0; i < cnt; i += 32 * K_EDGES) {
                int32_t d[K_EDGES];
                uint32_t tt[K_EDGES], ll[K_EDGES];
#pragma unroll
                for (int k = 0; k < K_EDGES; ++k) {
                    const uint32_t item = i + k * 32 + lane;
                    d[k] = -1;
                    tt[k] = 0;
                    ll[k] = 0;
                    if (item < cnt) {
                        const uint64_t ed = bbase + st + item;
                        d[k] = __ldg(&a.dst[ed]);
                        tt[k] = __ldg(&a.t[ed]);
                        ll[k] = (uint32_t)__ldg(&lam[ed]);
                        ++scanned;
                    }
                }
                relax_k<W, MODE>(a, d, tt, ll,
                           [&](int k) -> uint32_t {
                               if (W == 1) return bact;
                               int lo = 0, hi = 2 * W;  // first breakpoint above t
                               while (lo < hi) {
                                   const int mid = (lo + hi) >> 1;
                                   if (S.bkey[mid] <= tt[k]) lo = mid + 1; else hi = mid;
                               }
                               return lo ? S.bmask[lo - 1] : 0u;
                           },
                           [&](int, int q, uint32_t &th, uint32_t &li) {
                               if (W == 1) {
                                   th = S.bthr[q];
                                   li = S.blim[q];
                               } else {  // the mask already holds exactly the lanes whose interval contains t
                                   th = 0u;
                                   li = INF;
                               }
                           },
                           B, cnt1, lane, nxt, n3, hit);
            }
            __syncwarp();
            pc.mark(5);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hit |= __shfl_xor_sync(FULL, hit, o);
        if (lane == 0 && hit) atomicOr(&C->active[c3].v, hit);
        pc.mark(7);
        if (!grid_sync(C, &B.flag, a.spin_limit)) return;
        pc.mark(6);
        if (tid == 0) C->last_active = __ldcg(&C->active[c3].v);
    }

    // ---- read out: out[row_q][v] = label (mirrored back for latest departure) ----
    for (size_t i = tid; !a.resume && i < (size_t)n * W; i += nthr) {
        // nthr is a multiple of W, so this thread always sees lane R.q
        if (!R.on) continue;
        const size_t v = i / W;
        const uint32_t x = __ldcg(&a.arr[i]);
        reached += (x != INF);
        if (a.out && W == 1) {
            const bool mir = (a.lanes.mirror_mask >> R.q) & 1u;
            const uint32_t y = (mir && x != INF) ? TMAX - x : x;
            if (!(a.out_is_arr && !mir)) a.out[a.lanes.row[R.q] * a.out_stride + (int64_t)v] = y;
        }
    }
    if (W > 1 && a.out && !a.resume) {
        // several lanes: 32 vertices x W lanes at a time through shared memory (the rounds are
        // over, so the warps' scratch is free once their phase sums are out), so that both the
        // [n][W] state and the output rows move in whole segments, also when the output is
        // host memory
        pc.mark(7);
        if (pc.on && lane == 0)
#pragma unroll
            for (int i = 0; i < 8; ++i) atomicAdd(&C->phase_cycles[i], S.phase[i]);
        pc.on = false;
        uint32_t *tile = reinterpret_cast<uint32_t *>(smem_raw);
        const int64_t ntile = (n + 31) / 32;
        for (int64_t tl = blockIdx.x; tl < ntile; tl += gridDim.x) {
            const int64_t v0 = tl * 32;
            const int nv = (int)(n - v0 < 32 ? n - v0 : 32);
            __syncthreads();
            for (int i = threadIdx.x; i < nv * W; i += EM_THREADS)
                tile[(i / W) * (W + 1) + i % W] = __ldcg(&a.arr[(size_t)v0 * W + i]);
            __syncthreads();
            for (int i = threadIdx.x; i < 32 * W; i += EM_THREADS) {
                const int q = i >> 5, vv = i & 31;
                if (q < a.lanes.nlanes && ((a.running_mask >> q) & 1u) && vv < nv) {
                    const uint32_t x = tile[vv * (W + 1) + q];
                    const bool mir = (a.lanes.mirror_mask >> q) & 1u;
                    a.out[a.lanes.row[q] * a.out_stride + v0 + vv] = (mir && x != INF) ? TMAX - x : x;
                }
            }
        }
    }
    // ---- counters ----
#pragma unroll
    for (int o = W; o < 32; o <<= 1) reached += __shfl_xor_sync(FULL, reached, o);
    unsigned long long sc = scanned;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        sc += __shfl_xor_sync(FULL, sc, o);
        cnt1 += __shfl_xor_sync(FULL, cnt1, o);
    }
    if (lane < W && R.on) atomicAdd(&C->reached[lane], reached);
    if (lane == 0) atomicAdd(&C->scanned, sc);
    if (W == 1) {
        if (lane == 0) atomicAdd(&C->relaxed[0], cnt1);
    } else {
        __syncthreads();
        if (threadIdx.x < (unsigned)W && B.cnt[threadIdx.x])
            atomicAdd(&C->relaxed[threadIdx.x], (unsigned long long)B.cnt[threadIdx.x]);
    }
    if (tid == 0) C->rounds = r;
    pc.mark(7);
    if (pc.on && lane == 0)
#pragma unroll
        for (int i = 0; i < 8; ++i) atomicAdd(&C->phase_cycles[i], S.phase[i]);
}

template <int W, int MODE, typename LamT>
cudaError_t launch_t(const EdgeMapArgs &a, int grid, cudaStream_t s) {
    const size_t smem = sizeof(WarpSmem<W>) * (EM_THREADS / 32);
    // the shared-memory attribute is per device: set it once on each device that launches
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(edgemap_kernel<W, MODE, LamT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((void *)edgemap_kernel<W, MODE, LamT>, dim3(grid), dim3(EM_THREADS), args, smem, s);
}

template <int W, int MODE, typename LamT>
int max_blocks_t() {
    const size_t smem = sizeof(WarpSmem<W>) * (EM_THREADS / 32);
    if (cudaFuncSetAttribute(edgemap_kernel<W, MODE, LamT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, edgemap_kernel<W, MODE, LamT>, EM_THREADS, smem) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace

// The kernels of lane width W for both edge-time widths and every relaxation mode (one
// translation unit per W instantiates them, so that the widths compile in parallel).  Lane
// width 1 has no candidate-segment variant: mode 2 runs mode 0's code there.
template <int W>
cudaError_t edgemap_launch_w(const EdgeMapArgs &a, int lam_bits, int grid, cudaStream_t s) {
    constexpr int M2 = (W == 1) ? 0 : 2;
    if (lam_bits == 16) {
        if (a.relax_mode == 1) return launch_t<W, 1, uint16_t>(a, grid, s);
        if (a.relax_mode == 2) return launch_t<W, M2, uint16_t>(a, grid, s);
        return launch_t<W, 0, uint16_t>(a, grid, s);
    }
    if (a.relax_mode == 1) return launch_t<W, 1, uint32_t>(a, grid, s);
    if (a.relax_mode == 2) return launch_t<W, M2, uint32_t>(a, grid, s);
    return launch_t<W, 0, uint32_t>(a, grid, s);
}

template <int W>
int edgemap_max_blocks_w(int lam_bits, int relax_mode) {
    constexpr int M2 = (W == 1) ? 0 : 2;
    if (lam_bits == 16) {
        if (relax_mode == 1) return max_blocks_t<W, 1, uint16_t>();
        if (relax_mode == 2) return max_blocks_t<W, M2, uint16_t>();
        return max_blocks_t<W, 0, uint16_t>();
    }
    if (relax_mode == 1) return max_blocks_t<W, 1, uint32_t>();
    if (relax_mode == 2) return max_blocks_t<W, M2, uint32_t>();
    return max_blocks_t<W, 0, uint32_t>();
}

}  // namespace kairos
