// Internal declarations shared by the library's translation units (device helpers, the
// graph object, the edge-map launch record).  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "kairos.h"

namespace kairos {

constexpr uint32_t INF = 0xFFFFFFFFu;   // label of an unreached vertex
constexpr uint32_t TMAX = 0xFFFFFFFEu;  // largest finite time and mirror constant
constexpr uint32_t NO_FENCE = 0xFFFFFFFFu;
constexpr int FENCE_SHIFT = 5;          // one fence key every 32 edges
constexpr int FENCE_B = 1 << FENCE_SHIFT;
constexpr int EM_THREADS = 256;         // edge-map block size
constexpr int MAX_LANES = 32;
constexpr int PROFILE_ROUNDS = 256;
constexpr unsigned long long DEFAULT_SPIN_LIMIT = 1ull << 24;  // with backoff sleeps: seconds

// Device-side error codes reported through EdgeMapCtr::err.
enum : int { KERR_NONE = 0, KERR_BARRIER_TIMEOUT = 1, KERR_ROUNDS = 2, KERR_CAPACITY = 3, KERR_WAIT_TIMEOUT = 4 };
constexpr uint32_t NO_OWNER = 0xFFFFFFFFu;  // chunk_owner entry not yet published

// ---- status / error plumbing ---------------------------------------------------------

kairos_status fail(kairos_status st, const std::string &msg);
kairos_status cuda_fail(cudaError_t e, const char *what);

#define KAIROS_CUDA(call, what)                                 \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::kairos::cuda_fail(_e, what); \
    } while (0)

// ---- device memory -------------------------------------------------------------------

struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
    void *get(size_t bytes) const;   // nullptr on failure
    void put(void *p) const;
};

// Selectivity histogram of one vertex (Sec. 5.2): its edges' starts span [tmin, tmin + S) and
// durations [lmin, lmin + D), each cut into HIST_B equal buckets; bucket (i, j) holds the edges
// with (t - tmin) * HIST_B / S == i and (lam - lmin) * HIST_B / D == j.  Stored as row-wise
// inclusive prefix sums over j (cum[i][j] = edges in buckets (i, 0..j)) and the prefix of the
// row totals (row[i] = edges in rows 0..i-1).
constexpr int HIST_B = 100;
constexpr uint32_t NO_HIST = 0xFFFFFFFFu;
struct HistHdr {
    uint32_t tmin, lmin;
    uint64_t S, D;
};

// One direction of the time-sorted CSR plus its fence level.
struct Csr {
    uint64_t *off = nullptr;   // [n + 1] edge offsets
    int32_t *dst = nullptr;    // [m] head vertex
    uint32_t *t = nullptr;     // [m] departure time, ascending within each vertex
    void *lam = nullptr;       // [m] duration, uint16_t or uint32_t
    uint32_t *fidx = nullptr;  // [n] first fence key of the vertex, NO_FENCE if unindexed
    uint32_t *fence = nullptr; // fence keys: t of every FENCE_B-th edge of indexed vertices
    int64_t n_fence = 0;
    int64_t indexed = 0;
    int64_t max_deg = 0;
    // selectivity histograms of the vertices with degree >= hist_min_degree
    uint32_t *hidx = nullptr;  // [n] histogram number of the vertex, NO_HIST if none
    HistHdr *hhdr = nullptr;   // [n_hist]
    uint32_t *hcum = nullptr;  // [n_hist][HIST_B][HIST_B]
    uint32_t *hrow = nullptr;  // [n_hist][HIST_B + 1]
    int64_t n_hist = 0;
    uint32_t hist_min_degree = 0;
};

// Counters of one persistent edge-map launch (zeroed before each launch).  Counters that
// many warps update or poll in the same round sit on separate 128-byte lines.
struct __align__(128) PaddedU32 {
    unsigned int v;
    unsigned int pad[31];
};

struct EdgeMapCtr {
    unsigned int bar_count;
    unsigned int bar_gen;
    int err;
    unsigned int rounds;
    unsigned int pad0[28];
    PaddedU32 qcount[3];     // frontier queue lengths, indexed by round mod 3
    PaddedU32 bigcount[3];   // split ranges registered, by round mod 3
    PaddedU32 chunks[3];     // grid-wide chunks registered, by round mod 3
    PaddedU32 chunk_next[3]; // chunks claimed, by round mod 3
    PaddedU32 bnext[3];      // frontier batches claimed, by round mod 3
    PaddedU32 bdone[3];      // frontier batches finished, by round mod 3
    PaddedU32 active[3];     // lanes that lowered some label, by round mod 3
    unsigned int last_active;  // `active` of the last completed round
    unsigned long long scanned;
    unsigned long long relaxed[MAX_LANES];
    unsigned int reached[MAX_LANES];
    // per-round profile of the first PROFILE_ROUNDS rounds (block 0 after each barrier)
    unsigned long long round_ns[PROFILE_ROUNDS + 1];
    unsigned int round_frontier[PROFILE_ROUNDS];
    unsigned int round_chunks[PROFILE_ROUNDS];
    // SM cycles summed over warps per phase when EdgeMapArgs::phase_clock is set:
    // 0 lane states, 1 range search, 2 chunk registration, 3 local walk, 4 chunk wait,
    // 5 chunk walk, 6 grid barrier, 7 other
    unsigned long long phase_cycles[8];
};

// A long per-vertex edge range split into grid-wide chunks.
struct BigEntry {
    uint64_t base;        // first edge index
    uint32_t len;         // edges in the range
    uint32_t chunk_base;  // first chunk id
    uint32_t act;         // lanes with a non-empty departure interval
    uint32_t pad;
};

// Per-lane query parameters of one launch (times already mirrored for latest departure).
struct LaneParams {
    int32_t src[MAX_LANES];
    uint32_t ta[MAX_LANES];
    uint32_t tw[MAX_LANES];
    int64_t row[MAX_LANES]; // output row of lane q
    uint32_t strict_mask;  // bit q: StrictlySucceeds
    uint32_t mirror_mask;  // bit q: output is KAIROS_TIME_MAX - label (latest departure)
    int32_t nlanes;
};

struct EdgeMapArgs {
    // graph (one direction)
    const uint64_t *off;
    const int32_t *dst;
    const uint32_t *t;
    const void *lam;
    const uint32_t *fidx;  // nullptr: no index
    const uint32_t *fence;
    int64_t n;
    // workspace
    uint32_t *arr;         // [n][W] labels
    uint32_t *prev;        // [n][W] departure bound already scanned
    uint32_t *bm[2];       // frontier bitmaps, ceil(n/32) words each
    int32_t *queue[2];     // frontier queues, n entries each
    BigEntry *big;
    uint32_t *bigb;        // [cap_big][W][2] lane bounds of split ranges
    uint32_t *chunk_owner; // [cap_chunks]
    uint32_t cap_big, cap_chunks;
    EdgeMapCtr *ctr;
    // output: out[q * out_stride + v] for q < nlanes; nullptr: none
    uint32_t *out;
    int64_t out_stride;
    int out_is_arr;        // lanes == 1 and out aliases arr
    // parameters
    LaneParams lanes;
    uint32_t max_rounds;
    int warp_max_edges, chunk_edges, dense_div;
    int count_relaxed;     // nonzero: count relaxations per lane (query statistics)
    int relax_mode;        // 0 checked minimum + queue, 1 unconditional reductions + bitmap frontier
    // resumable operation: resume != 0 keeps the state of an earlier launch (no init, no
    // seeding, no readout) and runs rounds [round_begin, round_end); lanes outside
    // running_mask take no part
    int resume;
    uint32_t round_begin, round_end;
    uint32_t running_mask;
    int phase_clock;       // nonzero: accumulate per-phase cycle counts (diagnostics)
    unsigned long long spin_limit;  // polls before a device wait gives up (KERR_*_TIMEOUT)
    // per-vertex access choice (Sec. 5.1, Eq. 3): for a vertex with a histogram, scan its whole
    // list when the estimated selectivity exceeds select_permille / 1000, else search the index
    // (select_permille 0: the degree threshold alone decides)
    const uint32_t *hidx;
    const HistHdr *hhdr;
    const uint32_t *hcum;
    const uint32_t *hrow;
    int select_permille;
};

// ---- time-ordered stream mode (relax_mode 3) ---------------------------------------------
//
// Every edge of one direction as a 16-byte record in ascending departure time (ties in edge
// order), cut into time blocks: block k holds the records [bnd[k], bnd[k+1]), all departing in
// [bt[k], bt[k+1]) (an instant is never split).  A launch sweeps the blocks in time order;
// edges inside a block are relaxed together, and chains that start and end inside one block
// are finished by frontier rounds restricted to the block ("fix-ups").
constexpr int STREAM_MAX_LANES = 64;
struct StreamRec {
    int32_t src, dst;
    uint32_t t, lam;
};
struct TimeStream {
    StreamRec *rec = nullptr;  // [m]
    uint64_t *bnd = nullptr;   // [nblk + 1] first record of each block; bnd[nblk] = m
    uint32_t *bt = nullptr;    // [nblk + 1] first departure of each block; bt[nblk] = INF
    int32_t nblk = 0;
    int64_t block_edges = 0;   // target records per block the cut was made for
    uint32_t *bt_host = nullptr;  // host copy of bt
    uint64_t *span = nullptr;  // [n] (first departure << 32) | last departure of each vertex's
                               // list (INF << 32 | 0 for an empty list)
};

enum : int { KERR_FIX_ROUNDS = 5 };

struct StreamLanes {
    int32_t src[STREAM_MAX_LANES];
    uint32_t ta[STREAM_MAX_LANES];
    uint32_t tw[STREAM_MAX_LANES];
    int64_t row[STREAM_MAX_LANES];     // output row of lane q
    unsigned long long strict_mask;    // bit q: StrictlySucceeds
    unsigned long long mirror_mask;    // bit q: output is KAIROS_TIME_MAX - label
    int32_t nlanes;
};

struct StreamCtr {
    unsigned int bar_count;
    unsigned int bar_gen;
    int err;
    unsigned int pad0[29];
    PaddedU32 fcount[3];  // fix-up queue lengths, by generation mod 3
    PaddedU32 claim[2];   // pass tiles claimed past the first gridDim.x, by time block parity
    unsigned long long scanned;     // stream records read plus fix-up edges read
    unsigned long long cand;        // records whose lanes were examined
    unsigned long long fix_edges;   // edges read by fix-ups
    unsigned long long fix_vertices;
    unsigned int fix_rounds;        // fix-up generations run
    unsigned int blocks;            // time blocks swept
    unsigned int err_block, err_round;  // where the launch stopped on an error (time block, round)
    // fix-up generation and round count within the time block after a one-block run of short
    // rounds, by run parity: a block may still read run e's pair while block 0 writes run e + 1's
    unsigned int gen_shared[2];
    unsigned int round_shared[2];
    unsigned long long fread;       // frontier-length reads done, one per block and round: a
                                    // one-block run reuses the read slot only after all of them
    // diagnostics (phase_clock): pass candidates by number of candidate lanes (1, 2-4, 5-16,
    // 17-64), and candidate lanes in all
    unsigned long long cand_lanes[4];
    unsigned long long cand_pairs;
    unsigned long long wall_ns[3];   // block 0's wall time in passes, grid-wide fix-up rounds and
    unsigned long long segments[3];  // one-block runs (with their grid barriers), and their counts
    unsigned long long cand_improving;  // candidates (pass and fix-ups) that lowered some label
    unsigned long long lanes_lowered;   // labels lowered
    // SM cycles summed over warps when StreamArgs::phase_clock is set: 0 block passes (reading
    // and filtering records), 1 fix-ups, 2 grid barriers, initialisation and read-out, 3 the
    // passes' candidate relaxations
    unsigned long long phase_cycles[4];
    unsigned long long relaxed[STREAM_MAX_LANES];
    unsigned int reached[STREAM_MAX_LANES];
};

struct StreamArgs {
    const StreamRec *rec;
    const uint64_t *bnd;
    const uint32_t *bt;
    const uint64_t *span;      // [n] first and last departure of each vertex (TimeStream::span)
    int32_t k_begin, k_end;  // blocks swept
    // the same direction as a time-sorted CSR (fix-ups walk one vertex's list)
    const uint64_t *off;
    const int32_t *dst;
    const uint32_t *t;
    const void *lam;
    int64_t n;
    uint32_t *arr;     // [n][W] labels
    uint32_t *minrow;  // [n] at most the least label of the vertex over the lanes
    unsigned long long *rsum;  // [n][2] per half of 32 lanes: (bound << 32) | lanes of the half in
                               // which the vertex has a finite label (may lag, never ahead); the
                               // bound >= every label of the vertex in those lanes
    uint32_t *fbm;     // fix-up dedupe bitmap, ceil(n/32) words (all clear between blocks)
    int32_t *fq[2];    // fix-up queues, n entries each
    StreamCtr *ctr;
    uint32_t *out;     // out[row_q * out_stride + v]; nullptr: none
    int64_t out_stride;
    StreamLanes lanes;
    uint32_t max_fix_rounds;  // per block; past it KERR_FIX_ROUNDS
    unsigned long long spin_limit;
    int count_relaxed;        // nonzero: count usable edges per lane under the final labels
    int phase_clock;          // nonzero: accumulate per-phase cycle counts (diagnostics)
};

// Launch one stream-mode edge-map of W in {32, 64} lanes (cooperative).
cudaError_t stream_launch(const StreamArgs &a, int W, int lam_bits, int grid, cudaStream_t s);
int stream_max_grid(int W, int lam_bits, int sm_count, int *blocks_per_sm_out);
template <int W>
cudaError_t stream_launch_w(const StreamArgs &a, int lam_bits, int grid, cudaStream_t s);
template <int W>
int stream_max_blocks_w(int lam_bits);
// Build the time-ordered records of one direction from its CSR, and cut them into blocks of
// about block_edges records.
kairos_status build_time_stream(const Allocator &A, cudaStream_t s, int64_t n, int64_t m, const Csr &c, int lam_bits,
                                StreamRec *out);
kairos_status cut_time_blocks(const Allocator &A, cudaStream_t s, int64_t m, int64_t block_edges, TimeStream *ts);
// The first and last departure of every vertex's time-sorted list.
kairos_status build_vertex_spans(const Allocator &A, cudaStream_t s, int64_t n, const Csr &c, TimeStream *ts);
void free_time_stream(const Allocator &A, TimeStream *ts);

// Between resumable launches (serving): column operations on the [n][W] state.
// Retire the lanes in mask in one pass over the vertices: lanes in write_mask get
// out[q][v] = label (mirrored back when mirror_mask has q) with reached count and checksum
// added to stats[2q], stats[2q+1]; every lane in mask is then reset to unreached.
struct RetireArgs {
    uint32_t *out[MAX_LANES];
    uint32_t mask, write_mask, mirror_mask;
};
cudaError_t retire_lanes(uint32_t *arr, uint32_t *prev, int64_t n, int W, const RetireArgs &ra,
                         unsigned long long *stats, cudaStream_t s);
// Seed lane q at source src with label ta into the frontier of round r (bitmap + queue).
cudaError_t seed_lane(const EdgeMapArgs &a, int W, int q, int32_t src, uint32_t ta, uint32_t r, cudaStream_t s);

// Test hooks read from the environment on every call: KAIROS_SPIN_LIMIT (polls of every
// bounded device wait) and KAIROS_ROUND_CAP (edge-map rounds) shrink the limits so that the
// TIMEOUT paths can be exercised without a fault or a hang.
void apply_test_hooks(EdgeMapArgs &a);

// Launch one persistent edge-map (cooperative: every block resident).
cudaError_t edgemap_launch(const EdgeMapArgs &a, int lanes, int lam_bits, int grid, cudaStream_t s);
// Largest co-resident grid for this lane width (blocks per SM * SMs), 0 on error.
int edgemap_max_grid(int lanes, int lam_bits, int relax_mode, int *blocks_per_sm_out);
// per lane width (defined in edgemap_kernel.cuh, instantiated in edgemap_w<W>.cu)
template <int W>
cudaError_t edgemap_launch_w(const EdgeMapArgs &a, int lam_bits, int grid, cudaStream_t s);
template <int W>
int edgemap_max_blocks_w(int lam_bits, int relax_mode);

// Run queries through the batched edge-map, `lanes` per launch (api.cu; shared by the query
// calls, the autotuner and fastest paths).  out == nullptr discards the labels.
kairos_status kairos_run_queries(kairos_graph *g, const kairos_query *qs, int32_t nq, uint32_t *out,
                                 kairos_query_stats *stats, int lanes);
// The device a server's graph lives on (serve.cpp; used by the router).
int kairos_server_device(const kairos_server *s);
// Free the fastest-path scratch of a graph (fastest.cu).
void release_fastest_scratch(kairos_graph *g);
// Free the shortest-duration state of a graph (duration.cu).
void release_duration_scratch(kairos_graph *g);
// fwd2rev[i] = the slot of forward edge i in the reverse list's order (per head by mirrored
// time TMAX - (t + lam), i.e. latest arrival first; ties in forward order).
kairos_status build_reverse_slots(const Allocator &A, cudaStream_t s, int64_t n, int64_t m, const Csr &fwd,
                                  int lam_bits, uint32_t *fwd2rev);

// ---- device build ------------------------------------------------------------------------

// Time-sorted CSR of (key_src -> key_dst) edges.  mirror != 0 builds the reversed,
// time-mirrored graph: edge dst -> src departing at TMAX - (t + lam).
kairos_status build_csr(const Allocator &A, cudaStream_t s, int64_t n, int64_t m, const int32_t *src,
                        const int32_t *dst, const uint32_t *t, const void *lam, int lam_bits, int mirror,
                        Csr *out);
kairos_status validate_edges(cudaStream_t s, int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                             const uint32_t *t, const void *lam, int lam_bits, int *flags_host,
                             const Allocator &A);
kairos_status build_index(const Allocator &A, cudaStream_t s, int64_t n, uint32_t threshold, Csr *c);
// Selectivity histograms of the vertices with degree >= min_degree (KAIROS_NO_INDEX: none).
kairos_status build_histograms(const Allocator &A, cudaStream_t s, int64_t n, uint32_t min_degree, int lam_bits,
                               Csr *c);
void free_histograms(const Allocator &A, Csr *c);
void free_index(const Allocator &A, Csr *c);
void free_csr(const Allocator &A, Csr *c);
// Count vertices with degree > x and the grid chunks their full ranges need.
kairos_status split_capacity(const Allocator &A, cudaStream_t s, int64_t n, const uint64_t *off, int64_t x,
                             int64_t chunk, uint64_t *vertices, uint64_t *chunks);

}  // namespace kairos

// The graph object behind the opaque C handle.
struct kairos_graph {
    int64_t n = 0, m = 0;
    int device = 0;  // the device current at build: every call on the graph uses it
    int lam_bits = 32;
    cudaStream_t stream = nullptr;
    kairos::Allocator A;
    kairos::Csr fwd, rev;
    int has_rev = 0;
    uint32_t theta = KAIROS_NO_INDEX;
    kairos_tuning tuning{};
    double build_ms = 0, index_ms = 0, last_kernel_ms = 0;
    int sm_count = 0;
    std::mutex mu;

    // query workspace (grown on demand)
    struct Work {
        int lanes = 0;
        uint32_t *arr = nullptr, *prev = nullptr, *bm = nullptr;
        int32_t *queue = nullptr;
        kairos::BigEntry *big = nullptr;
        uint32_t *bigb = nullptr, *chunk_owner = nullptr;
        uint32_t cap_big = 0, cap_chunks = 0;
        int warp_max = 0, chunk = 0;
        kairos::EdgeMapCtr *ctr_host = nullptr; // pinned copy of the last launch's counters (diagnostics)
        uint32_t *stage = nullptr;              // [lanes][n] output staging for host outputs
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        size_t bytes = 0;
        kairos::EdgeMapCtr *ctrs = nullptr;       // one counter slot per launch of a call
        kairos::EdgeMapCtr *ctrs_host = nullptr;  // pinned mirror
        size_t ctr_slots = 0;
        cudaGraphExec_t graph_exec = nullptr;     // the last captured call
        std::string graph_key;
        // the second workspace and stream of concurrent launches (tuning.concurrent == 2)
        uint32_t *arr2 = nullptr, *prev2 = nullptr, *bm2 = nullptr, *bigb2 = nullptr, *chunk_owner2 = nullptr;
        int32_t *queue2 = nullptr;
        kairos::BigEntry *big2 = nullptr;
        cudaStream_t side = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        // fastest paths: label rows of one pass of start-time lanes, the running minimum
        // (host outputs) and the start times of the pass
        uint32_t *fast_rows = nullptr, *fast_best = nullptr, *fast_d = nullptr;
        int64_t fast_rows_cap = 0;
        // shortest durations: reverse slot of every forward edge, per-slot edge labels and
        // their per-head suffix minima, per-vertex flags, round counters
        uint32_t *sd_slot = nullptr, *sd_d = nullptr, *sd_sm = nullptr;
        uint8_t *sd_changed = nullptr, *sd_active = nullptr;
        uint32_t *sd_from = nullptr;  // [5][n] + 4: change bounds, the long-list queue, counters (duration.cu)
        uint32_t *sd_pred[2] = {nullptr, nullptr};  // per predicate: each edge's first in-time in-list slot
        void *sd_chunks = nullptr;                  // relaxation work items
        unsigned long long *sd_ctr = nullptr, *sd_ctr_host = nullptr;
    } work;
    // time-ordered stream mode: records per direction (built on first use) and the launch
    // workspace (two sets when two launches are in flight)
    kairos::TimeStream ts_fwd, ts_rev;
    struct StreamWork {
        int lanes = 0;
        uint32_t *arr = nullptr, *minrow = nullptr, *fbm = nullptr;
        unsigned long long *rsum = nullptr;
        int32_t *fq = nullptr;
        uint32_t *stage = nullptr;  // [W][n] labels bound for host memory (copied by the copy engine)
        size_t bytes = 0;
    } sw[4];
    // up to three more streams for time-ordered launches in flight together, with their fork and
    // join events
    cudaStream_t sside[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t sfork = nullptr, sjoin[3] = {nullptr, nullptr, nullptr};
    kairos::StreamCtr *sctrs = nullptr, *sctrs_host = nullptr;
    kairos::StreamCtr last_sctr{};  // counters of the last stream-mode launch (diagnostics)
    size_t sctr_slots = 0;
    int last_launches = 0;
    int64_t graph_launches = 0;
};
