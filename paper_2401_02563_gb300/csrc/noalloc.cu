// Earliest arrival without any device allocation: the query's scratch (scan bounds,
// frontier bitmaps and queues, split-range lists, counters) lives in one file-scope
// __device__ array of fixed size, and the caller's output buffer holds the labels.
//
// Who needs this: code that must not allocate device memory while it runs, for example a
// process that has handed all of its device memory to its own pool up front, or one that
// calls in while another framework is capturing a CUDA graph and forbids new allocations.
// Such callers still build the graph beforehand (that allocates); each query afterwards
// allocates nothing.
//
// Limits: graphs of at most NA_MAX_VERTICES vertices whose long adjacency ranges fit the
// fixed split-range lists (checked per call).  The array is shared by every call in the
// process on a device: calls whose work overlaps on the GPU (different streams or threads
// without ordering) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.cuh"

namespace kairos {
namespace {

constexpr int64_t NA_MAX_VERTICES = 1 << 20;
constexpr uint32_t NA_MAX_SPLIT = 1u << 16;   // long ranges registered per round
constexpr uint32_t NA_MAX_CHUNKS = 1u << 18;  // grid-wide chunks per round
constexpr int NA_MAX_DEVICES = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t NA_OFF_CTR = 0;
constexpr size_t NA_OFF_CAP = NA_OFF_CTR + align256(sizeof(EdgeMapCtr));
constexpr size_t NA_OFF_PREV = NA_OFF_CAP + 256;
constexpr size_t NA_OFF_BM = NA_OFF_PREV + align256((size_t)NA_MAX_VERTICES * 4);
constexpr size_t NA_OFF_QUEUE = NA_OFF_BM + align256((size_t)(NA_MAX_VERTICES / 32) * 2 * 4);
constexpr size_t NA_OFF_BIG = NA_OFF_QUEUE + align256((size_t)NA_MAX_VERTICES * 2 * 4);
constexpr size_t NA_OFF_BIGB = NA_OFF_BIG + align256((size_t)NA_MAX_SPLIT * sizeof(BigEntry));
constexpr size_t NA_OFF_OWNER = NA_OFF_BIGB + align256((size_t)NA_MAX_SPLIT * 2 * 4);
constexpr size_t NA_BYTES = NA_OFF_OWNER + align256((size_t)NA_MAX_CHUNKS * 4);  // about 15.5 MB

static __device__ __align__(256) unsigned char na_scratch[NA_BYTES];

std::mutex na_mu;
void *na_addr[NA_MAX_DEVICES] = {};

// Device address of na_scratch on the current device (looked up once per device).
kairos_status scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation query: current device");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(KAIROS_ERR_INVALID_ARG, "no-allocation query: device index too large");
    std::lock_guard<std::mutex> lk(na_mu);
    if (!na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "no-allocation query: scratch address");
        na_addr[dev] = p;
    }
    *out = (unsigned char *)na_addr[dev];
    return KAIROS_OK;
}

// cap[0] = vertices whose degree exceeds x, cap[1] = sum of their ceil(degree / chunk).
__global__ void na_split_capacity(int64_t n, const uint64_t *off, int64_t x, int64_t chunk, unsigned long long *cap) {
    unsigned long long cnt = 0, ch = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t d = off[u + 1] - off[u];
        if ((int64_t)d > x) {
            cnt += 1;
            ch += (d + chunk - 1) / chunk;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        ch += __shfl_xor_sync(0xFFFFFFFFu, ch, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cap[0], cnt);
        atomicAdd(&cap[1], ch);
    }
}

}  // namespace
}  // namespace kairos

using namespace kairos;

extern "C" kairos_status kairos_earliest_arrival_noalloc(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw,
                                                         uint32_t *out) {
    if (!g || !out) return fail(KAIROS_ERR_INVALID_ARG, "no-allocation query: NULL argument");
    if (src < 0 || (int64_t)src >= g->n) return fail(KAIROS_ERR_INVALID_ARG, "no-allocation query: source out of range");
    if (ta > tw || tw > TMAX) return fail(KAIROS_ERR_INVALID_ARG, "no-allocation query: need ta <= tw <= KAIROS_TIME_MAX");
    if (g->n > NA_MAX_VERTICES)
        return fail(KAIROS_ERR_INVALID_ARG,
                    "no-allocation query: the graph has more than 2^20 vertices, the limit of the fixed scratch array");
    int dev = 0;
    KAIROS_CUDA(cudaGetDevice(&dev), "no-allocation query: current device");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(KAIROS_ERR_INVALID_ARG, "no-allocation query: out must be device memory");
    }
    if (at.device != dev)
        return fail(KAIROS_ERR_INVALID_ARG, "no-allocation query: out must be memory of the current device");
    std::lock_guard<std::mutex> lk(g->mu);
    unsigned char *base = nullptr;
    kairos_status st = scratch_address(&base);
    if (st != KAIROS_OK) return st;
    cudaStream_t s = g->stream;
    EdgeMapCtr *ctr = (EdgeMapCtr *)(base + NA_OFF_CTR);
    unsigned long long *cap = (unsigned long long *)(base + NA_OFF_CAP);
    uint32_t *owner = (uint32_t *)(base + NA_OFF_OWNER);
    const int64_t n = g->n, nwords = (n + 31) / 32;
    const int wm = g->tuning.warp_max_edges, ch = g->tuning.chunk_edges;

    // counters and chunk owners must start cleared; the kernel initialises the rest
    KAIROS_CUDA(cudaMemsetAsync(ctr, 0, sizeof(EdgeMapCtr), s), "no-allocation query: clear counters");
    KAIROS_CUDA(cudaMemsetAsync(cap, 0, 16, s), "no-allocation query: clear capacity");
    KAIROS_CUDA(cudaMemsetAsync(owner, 0xFF, (size_t)NA_MAX_CHUNKS * 4, s), "no-allocation query: clear chunk owners");
    na_split_capacity<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(n, g->fwd.off, wm, ch, cap);
    KAIROS_CUDA(cudaGetLastError(), "no-allocation query: capacity scan");
    unsigned long long hcap[2] = {0, 0};
    KAIROS_CUDA(cudaMemcpyAsync(hcap, cap, 16, cudaMemcpyDeviceToHost, s), "no-allocation query: capacity scan");
    KAIROS_CUDA(cudaStreamSynchronize(s), "no-allocation query: capacity scan");
    if (hcap[0] + 1 > NA_MAX_SPLIT || hcap[1] + 1 > NA_MAX_CHUNKS)
        return fail(KAIROS_ERR_INVALID_ARG,
                    "no-allocation query: the graph's long adjacency ranges exceed the fixed split-range lists");

    EdgeMapArgs a;
    std::memset(&a, 0, sizeof(a));
    a.off = g->fwd.off;
    a.dst = g->fwd.dst;
    a.t = g->fwd.t;
    a.lam = g->fwd.lam;
    a.fidx = g->fwd.fidx;
    a.fence = g->fwd.fence;
    a.n = n;
    a.arr = out;  // the caller's buffer holds the labels throughout
    a.prev = (uint32_t *)(base + NA_OFF_PREV);
    a.bm[0] = (uint32_t *)(base + NA_OFF_BM);
    a.bm[1] = a.bm[0] + nwords;
    a.queue[0] = (int32_t *)(base + NA_OFF_QUEUE);
    a.queue[1] = a.queue[0] + n;
    a.big = (BigEntry *)(base + NA_OFF_BIG);
    a.bigb = (uint32_t *)(base + NA_OFF_BIGB);
    a.chunk_owner = owner;
    a.cap_big = NA_MAX_SPLIT;
    a.cap_chunks = NA_MAX_CHUNKS;
    a.ctr = ctr;
    a.out = out;
    a.out_stride = n;
    a.out_is_arr = 1;
    a.lanes.nlanes = 1;
    a.lanes.src[0] = src;
    a.lanes.ta[0] = ta;
    a.lanes.tw[0] = tw;
    a.lanes.row[0] = 0;
    a.max_rounds = (uint32_t)std::min<int64_t>(n + 1, 0xFFFFFFF0LL);
    a.warp_max_edges = wm;
    a.chunk_edges = ch;
    a.dense_div = g->tuning.dense_div;
    a.round_end = 0xFFFFFFFFu;
    a.running_mask = 0xFFFFFFFFu;
    a.spin_limit = DEFAULT_SPIN_LIMIT;
    apply_test_hooks(a);
    int bps = 0;
    int grid = edgemap_max_grid(1, g->lam_bits, 0, &bps);
    if (grid <= 0) return fail(KAIROS_ERR_CUDA, "no-allocation query: no resident launch shape");
    if (g->tuning.blocks_per_sm > 0 && g->tuning.blocks_per_sm < bps) grid = g->tuning.blocks_per_sm * g->sm_count;
    KAIROS_CUDA(edgemap_launch(a, 1, g->lam_bits, grid, s), "no-allocation query: edge-map launch");
    int err = 0;
    KAIROS_CUDA(cudaMemcpyAsync(&err, &ctr->err, sizeof(int), cudaMemcpyDeviceToHost, s), "no-allocation query: status");
    KAIROS_CUDA(cudaStreamSynchronize(s), "no-allocation query");
    if (err == KERR_BARRIER_TIMEOUT || err == KERR_WAIT_TIMEOUT)
        return fail(KAIROS_ERR_TIMEOUT, "no-allocation query: a device wait ran past its limit");
    if (err == KERR_ROUNDS) return fail(KAIROS_ERR_TIMEOUT, "no-allocation query: round cap (n + 1) reached");
    if (err) return fail(KAIROS_ERR_INTERNAL, "no-allocation query: split-range capacity exceeded");
    return KAIROS_OK;
}
