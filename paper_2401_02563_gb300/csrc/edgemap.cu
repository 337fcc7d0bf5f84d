// Launch dispatch of the temporal edge-map kernels (one instantiation file per lane width)
// and the small kernels of resumable launches: retiring lanes and seeding a lane.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace kairos {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// One warp per 32 vertices and lane (the lane loop is uniform); per-lane sums gather in
// shared memory and leave with one atomic per block.
__global__ void retire_lanes_kernel(uint32_t *arr, uint32_t *prev, int64_t n, int W, const RetireArgs ra,
                                    unsigned long long *stats) {
    __shared__ unsigned long long s_cnt[MAX_LANES], s_cs[MAX_LANES];
    if (threadIdx.x < MAX_LANES) {
        s_cnt[threadIdx.x] = 0;
        s_cs[threadIdx.x] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + threadIdx.x;
        for (uint32_t m = ra.mask; m; m &= m - 1) {
            const int q = __ffs(m) - 1;
            unsigned long long cnt = 0, cs = 0;
            if (v < n) {
                const size_t i = (size_t)v * W + q;
                const uint32_t x = arr[i];
                if ((ra.write_mask >> q) & 1u) {
                    const uint32_t y = (((ra.mirror_mask >> q) & 1u) && x != INF) ? TMAX - x : x;
                    ra.out[q][v] = y;
                    cnt = (x != INF);
                    cs = (unsigned long long)(v + 1) * y;
                }
                // only a vertex the query reached can hold a label or a scan bound (a bound
                // is set only when a reached vertex is expanded): reset just those
                if (x != INF) {
                    arr[i] = INF;
                    prev[i] = INF;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cnt += __shfl_xor_sync(FULL, cnt, o);
                cs += __shfl_xor_sync(FULL, cs, o);
            }
            if (lane == 0 && ((ra.write_mask >> q) & 1u)) {
                atomicAdd(&s_cnt[q], cnt);
                atomicAdd(&s_cs[q], cs);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < MAX_LANES && ((ra.write_mask >> threadIdx.x) & 1u)) {
        atomicAdd(&stats[2 * threadIdx.x], s_cnt[threadIdx.x]);
        atomicAdd(&stats[2 * threadIdx.x + 1], s_cs[threadIdx.x]);
    }
}

// Lane q's source enters the frontier of round r: its label, then the bitmap bit and a
// queue slot unless the vertex is already queued for that round.
__global__ void seed_lane_kernel(uint32_t *arr, uint32_t *bm, int32_t *queue, unsigned *count, int W, int q,
                                 int32_t src, uint32_t ta) {
    arr[(size_t)src * W + q] = ta;
    const uint32_t bit = 1u << (src & 31);
    if (!(atomicOr(&bm[src >> 5], bit) & bit)) queue[atomicAdd(count, 1u)] = src;
}

}  // namespace

cudaError_t retire_lanes(uint32_t *arr, uint32_t *prev, int64_t n, int W, const RetireArgs &ra,
                         unsigned long long *stats, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    retire_lanes_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(arr, prev, n, W, ra, stats);
    return cudaGetLastError();
}

cudaError_t seed_lane(const EdgeMapArgs &a, int W, int q, int32_t src, uint32_t ta, uint32_t r, cudaStream_t s) {
    seed_lane_kernel<<<1, 1, 0, s>>>(a.arr, a.bm[r & 1], a.queue[r & 1], &a.ctr->qcount[r % 3].v, W, q, src, ta);
    return cudaGetLastError();
}

cudaError_t edgemap_launch(const EdgeMapArgs &a, int lanes, int lam_bits, int grid, cudaStream_t s) {
    switch (lanes) {
        case 1: return edgemap_launch_w<1>(a, lam_bits, grid, s);
        case 2: return edgemap_launch_w<2>(a, lam_bits, grid, s);
        case 4: return edgemap_launch_w<4>(a, lam_bits, grid, s);
        case 8: return edgemap_launch_w<8>(a, lam_bits, grid, s);
        case 16: return edgemap_launch_w<16>(a, lam_bits, grid, s);
        case 32: return edgemap_launch_w<32>(a, lam_bits, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int edgemap_max_grid(int lanes, int lam_bits, int relax_mode, int *blocks_per_sm_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    int nb = 0;
    switch (lanes) {
        case 1: nb = edgemap_max_blocks_w<1>(lam_bits, relax_mode); break;
        case 2: nb = edgemap_max_blocks_w<2>(lam_bits, relax_mode); break;
        case 4: nb = edgemap_max_blocks_w<4>(lam_bits, relax_mode); break;
        case 8: nb = edgemap_max_blocks_w<8>(lam_bits, relax_mode); break;
        case 16: nb = edgemap_max_blocks_w<16>(lam_bits, relax_mode); break;
        case 32: nb = edgemap_max_blocks_w<32>(lam_bits, relax_mode); break;
        default: return 0;
    }
    if (blocks_per_sm_out) *blocks_per_sm_out = nb;
    return nb * sms;
}

}  // namespace kairos
