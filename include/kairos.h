/*
 * kairos.h -- C ABI of the GB300 temporal edge-map library.
 *
 * The library answers time-respecting path queries on a temporal graph resident in GPU
 * memory (one GPU, sm_103a): earliest arrival from a source and latest departure towards
 * a target, each inside a time window, one at a time, in batches, or through a
 * continuous-batching server.  Every step of a query runs in the library's own CUDA
 * kernels; there is no CPU fallback.
 *
 * Model (paper Sec. 2.1): vertices 0..n-1; a temporal edge (u, v, t, lambda) departs u at
 * time t and arrives at v at t + lambda (its validity interval [t, t + lambda]).  Times
 * are uint32; t + lambda must not exceed KAIROS_TIME_MAX.
 * Ordering predicates (Sec. 2.2): consecutive edges A, B of a path satisfy
 * end(A) <= start(B) ("Succeeds", strict = 0, the default) or end(A) < start(B)
 * ("StrictlySucceeds", strict = 1).  The first edge may depart exactly at the window start
 * and the last may arrive exactly at the window end under either predicate.
 * Window [ta, tw] is inclusive at both ends (the window test of Alg. 2).
 * Results (Alg. 2 and Sec. 2.3's minimal temporal paths):
 *   earliest arrival from s:  out[s] = ta; out[v] = least arrival time at v over
 *                             time-respecting paths from s within the window;
 *   latest departure to x:    out[x] = tw; out[u] = greatest departure time from u over
 *                             time-respecting paths from u to x within the window;
 *   KAIROS_UNREACHED where no such path exists.
 *
 * Conventions for every call:
 *   - returns a kairos_status; never aborts, traps or exits; on failure
 *     kairos_last_error() gives a message (thread-local, valid until the next call);
 *   - pointers documented as "host or device" are classified with
 *     cudaPointerGetAttributes; host memory may be pageable or pinned;
 *   - calls on one graph are serialised internally (a graph owns one query workspace);
 *     distinct graphs may be used from distinct threads.
 */
#ifndef KAIROS_H
#define KAIROS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KAIROS_OK = 0,
    KAIROS_ERR_INVALID_ARG = 1, /* bad pointer, size, vertex id, or ta > tw / tw > TIME_MAX */
    KAIROS_ERR_OOM = 2,         /* device or host allocation failed */
    KAIROS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    KAIROS_ERR_OVERFLOW = 4,    /* an edge has t + lambda > KAIROS_TIME_MAX */
    KAIROS_ERR_NOT_READY = 5,   /* a served query has not finished yet */
    KAIROS_ERR_BUSY = 6,        /* the server's admission queue is full */
    KAIROS_ERR_TIMEOUT = 7,     /* a device-side wait or the round cap (n + 1) ran out */
    KAIROS_ERR_INTERNAL = 8     /* a device-side consistency check failed */
} kairos_status;

#define KAIROS_UNREACHED 0xFFFFFFFFu /* label of a vertex with no valid path */
#define KAIROS_TIME_MAX 0xFFFFFFFEu  /* largest finite time; also the mirror constant */
#define KAIROS_NO_INDEX 0xFFFFFFFFu  /* index threshold meaning "scan every list linearly" */

enum { KAIROS_EA = 0, KAIROS_LD = 1 };

typedef struct kairos_graph kairos_graph;   /* opaque; freed with kairos_graph_free */
typedef struct kairos_server kairos_server; /* opaque; borrows a graph; kairos_serve_destroy */

/* A structure-of-arrays temporal edge list (Sec. 2.1).  Edge i is
 * (src[i], dst[i], t_dep[i], lambda[i]); lambda is uint16_t[] when lambda_bits == 16, else
 * uint32_t[].  All four arrays are host memory, or device memory of the current device
 * when on_device != 0.  The library copies them during kairos_graph_build and keeps no
 * reference; the caller keeps ownership. */
typedef struct {
    int64_t n_vertices; /* n >= 1, n < 2^31 */
    int64_t n_edges;    /* m >= 0, m < 2^32 */
    const int32_t *src;
    const int32_t *dst;
    const uint32_t *t_dep;
    const void *lambda;
    int32_t lambda_bits; /* 16 or 32 */
    int32_t on_device;
} kairos_edge_list;

/* Optional build options (NULL = defaults). */
typedef struct {
    void *stream;                           /* cudaStream_t for all work on this graph; NULL: legacy default stream */
    void *(*alloc)(size_t bytes, void *ctx); /* device allocator; NULL: cudaMalloc */
    void (*free)(void *ptr, void *ctx);      /* matching release; NULL: cudaFree */
    void *alloc_ctx;
    int32_t skip_reverse; /* nonzero: do not build the mirrored reverse graph (latest
                             departure then returns INVALID_ARG); saves half the graph memory */
} kairos_graph_opts;

/* One query.  vertex is the source for KAIROS_EA and the target for KAIROS_LD. */
typedef struct {
    int32_t vertex;
    uint32_t ta, tw; /* inclusive window, ta <= tw <= KAIROS_TIME_MAX */
    uint8_t kind;    /* KAIROS_EA or KAIROS_LD */
    uint8_t strict;  /* 0 Succeeds, 1 StrictlySucceeds */
    uint16_t reserved;
} kairos_query;

/* Work counters of one query, filled by the calls that take a stats array. */
typedef struct {
    uint64_t relaxed_edges; /* usable edges relaxed: each edge with a reached tail, departure
                               on or after the tail's label and arrival within the window,
                               counted once (the "traversed edges" of GTEPS) */
    uint64_t scanned_edges; /* edge records loaded for this query's batch (shared by its lanes) */
    uint32_t rounds;        /* edge-map rounds until the frontier emptied */
    uint32_t reached;       /* vertices with a finite label */
} kairos_query_stats;

/* Launch-shape knobs of the edge-map; kairos_autotune picks them per graph. */
typedef struct {
    int32_t lanes;          /* queries relaxed together per launch: 1, 2, 4, 8, 16, 32, or 64
                               (64 with relax_mode 3 only) */
    int32_t blocks_per_sm;  /* resident 256-thread blocks per SM of the persistent grid; 0: as many as fit */
    int32_t warp_max_edges; /* a vertex's range longer than this is split across the grid */
    int32_t chunk_edges;    /* edges per grid-wide chunk of a split range (multiple of 32) */
    int32_t dense_div;      /* sweep the frontier bitmap instead of the queue when
                               |frontier| > n / dense_div (0: never) */
    int32_t relax_mode;     /* 0: read the head's label and lower it only when the arrival is
                               earlier, queueing heads that changed, fetching every lane
                               segment of a head at once (suits many active lanes); 2: the same
                               check, fetching only segments with candidate lanes, pass by pass
                               (suits few active lanes); 1: lower it with a fire-and-forget
                               atomic for every usable edge and take the next frontier from the
                               bitmap of touched heads; 3 (lanes 32 or 64): sweep all edges once in
                               departure-time order, block by block, relaxing every lane whose
                               label at the tail allows the departure, and finish chains inside a
                               block with frontier rounds restricted to that block (the first
                               call builds a time-ordered copy of the edges, 16 bytes per edge
                               and direction, kept with the graph); calls with fewer lanes (single
                               queries) run mode 0 */
    int32_t concurrent;     /* launches of one call kept in flight together, each on its own stream
                               and workspace with 1/concurrent of the resident blocks (unless
                               blocks_per_sm is set): 1 or 2 (0 means 1), or 4 with relax_mode 3.
                               More lets one launch's sparse rounds overlap another's busy ones; it
                               applies when the call has two or more launches and its outputs are
                               device memory, or page-locked host memory with relax_mode 3 (each
                               launch's rows are then staged on the device and copied to the host
                               by the copy engine on the launch's stream) */
    int32_t block_edges;    /* relax_mode 3: edges per time block (an instant is never split);
                               0: max(4096, n_edges / 512) */
    int32_t select_permille; /* selective access (Sec. 5.1, Eq. 3) for the frontier modes 0-2:
                               with histograms built (kairos_selectivity_build), an indexed vertex
                               whose estimated selectivity for the departure interval being
                               expanded exceeds select_permille / 1000 has its whole list scanned
                               instead of searched; 0: the index threshold alone decides.  Results
                               never depend on it */
} kairos_tuning;

typedef struct {
    int64_t n_vertices, n_edges;
    int32_t lambda_bits;
    uint32_t index_threshold;    /* KAIROS_NO_INDEX when no index is built */
    int64_t indexed_vertices;    /* forward graph vertices with a fence level */
    int64_t device_bytes;        /* graph + index + query workspace currently held */
    double build_ms;             /* last kairos_graph_build, device time */
    double index_ms;             /* last kairos_index_build, device time */
    int64_t graph_launches;      /* query calls run as a captured CUDA graph (capture or replay) */
} kairos_graph_info;

/* ---- graph and index -------------------------------------------------------------- */

/* Build the device-resident time-sorted CSR of Sec. 2.4/4.2 from an edge list: each
 * vertex's out-edges sorted by departure time (the paper's T-CSR, whose per-vertex lists
 * the library keeps in time order), plus the reversed, time-mirrored graph used for
 * latest departure (edge v -> u departing at KAIROS_TIME_MAX - (t + lambda)).
 * Errors: INVALID_ARG (NULL, n < 1, m < 0, vertex id out of range, lambda_bits not 16/32),
 * OVERFLOW (some t + lambda > KAIROS_TIME_MAX), OOM, CUDA.  *out is set only on success. */
kairos_status kairos_graph_build(const kairos_edge_list *edges, const kairos_graph_opts *opts,
                                 kairos_graph **out);

/* Selective index (Sec. 3.2 "Vertex Indexer", Alg. 1 IndexVertices, cost model Eqs. 1-3):
 * vertices whose degree is >= threshold get a fence level (every 32nd departure time of
 * their sorted list) and are searched; shorter lists are scanned linearly.
 * KAIROS_NO_INDEX drops the index (every list scanned).  Results never depend on it.
 * Errors: INVALID_ARG (NULL graph), OOM, CUDA. */
kairos_status kairos_index_build(kairos_graph *g, uint32_t threshold);

/* Selectivity histograms (Sec. 5.2): for every vertex with degree >= min_degree, in both
 * directions, a 2D density histogram of its edges over start time and duration, each cut into
 * 100 equal buckets over the vertex's own span (bucket i of starts holds the edges with
 * (t - tmin) * 100 / (tmax - tmin + 1) == i; likewise durations).  A temporal predicate
 * "departure in [a, b], arrival by tw" is estimated by counting every edge of a bucket whose
 * centre satisfies it (the centre of a bucket is the floor of the mean of its first and last
 * integer).  The edge-map uses the estimate for the access choice of tuning.select_permille.
 * KAIROS_NO_INDEX drops the histograms.  Memory: about 40 KB per such vertex and direction.
 * Errors: INVALID_ARG (NULL graph), OOM, CUDA. */
kairos_status kairos_selectivity_build(kairos_graph *g, uint32_t min_degree);

/* For each of the n vertices (host array) of the forward lists (kind KAIROS_EA) or of the
 * reversed, time-mirrored lists (KAIROS_LD): estimate[i] = the histogram's estimate of the edges
 * departing in [a, b] and arriving by tw (UINT64_MAX for a vertex without a histogram), and, when
 * exact is not NULL, exact[i] = the true number of such edges.  Host outputs.  Synchronous.
 * Errors: INVALID_ARG (NULL, vertex out of range, LD without the reverse graph), OOM, CUDA. */
kairos_status kairos_selectivity_estimate(kairos_graph *g, int32_t kind, const int32_t *vertices, int32_t n,
                                          uint32_t a, uint32_t b, uint32_t tw, uint64_t *estimate, uint64_t *exact);

/* The stored histogram of one vertex: meta4 = {tmin, start span S, lmin, duration span D} and
 * counts[i * 100 + j] = edges in start bucket i and duration bucket j (host arrays).  Errors:
 * INVALID_ARG (NULL, no histogram for the vertex), OOM, CUDA. */
kairos_status kairos_selectivity_histogram(kairos_graph *g, int32_t kind, int32_t vertex, uint64_t *meta4,
                                           uint32_t *counts);

void kairos_graph_free(kairos_graph *g); /* NULL is ignored; waits for the graph's stream */

kairos_status kairos_graph_get_info(const kairos_graph *g, kairos_graph_info *info);

/* ---- queries ------------------------------------------------------------------------ */

/* Earliest arrival from src within [ta, tw] under Succeeds (Alg. 2).  out: uint32_t[n],
 * host or device, owned by the caller.  Synchronous.  Errors: INVALID_ARG, TIMEOUT,
 * OOM, CUDA. */
kairos_status kairos_earliest_arrival(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, uint32_t *out);

/* Latest departure towards dst within [ta, tw] under Succeeds (Sec. 2.3), computed as
 * earliest arrival on the mirrored reverse graph.  out: uint32_t[n], host or device. */
kairos_status kairos_latest_departure(kairos_graph *g, int32_t dst, uint32_t ta, uint32_t tw, uint32_t *out);

/* Answer n queries of either kind and predicate.  out: uint32_t[n][n_vertices], query-major
 * (row i is query i's labels), host or device.  stats: NULL or kairos_query_stats[n].
 * Queries are packed tuning.lanes at a time into one persistent launch that loads each
 * edge once for all of its lanes.  Synchronous.  Errors as above. */
kairos_status kairos_batch_query(kairos_graph *g, const kairos_query *queries, int32_t n, uint32_t *out,
                                 kairos_query_stats *stats);

/* Fastest paths from src within [ta, tw] (Sec. 2.3 names fastest paths among the minimal
 * temporal paths; the definition is that of the paper's reference on temporal path
 * problems): out[v] = the minimum over time-respecting paths P from src to v inside the
 * window of (arrival(P) - first departure(P)); out[src] = 0; KAIROS_UNREACHED otherwise.
 * strict: 0 Succeeds, 1 StrictlySucceeds between consecutive edges.
 * Method: one earliest-arrival lane per distinct departure time d of src's usable
 * out-edges (window [d, tw]), packed tuning.lanes per launch on the batched edge-map, then
 * out[v] = min over d of (EA_d[v] - d) on the device.  out: uint32_t[n], host or device,
 * owned by the caller.  stats (may be NULL): start times, edge-map launches and relaxed
 * edges summed over the lanes (asking for it counts relaxations, which costs some time).
 * Synchronous.  Errors: INVALID_ARG (NULL graph or out, src out of range, ta > tw,
 * tw > KAIROS_TIME_MAX, strict not 0/1), TIMEOUT, OOM, CUDA. */
typedef struct {
    uint64_t start_times;    /* distinct departure times of src's usable out-edges */
    uint64_t launches;       /* edge-map launches */
    uint64_t relaxed_edges;  /* sum over the start-time lanes of their relaxed edges */
} kairos_fastest_stats;

kairos_status kairos_fastest_path(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, int32_t strict,
                                  uint32_t *out, kairos_fastest_stats *stats);

/* Shortest durations from src within [ta, tw] (Sec. 2.3 names shortest paths among the
 * minimal temporal paths; the definition is that of the paper's reference on temporal path
 * problems): out[v] = the minimum over time-respecting paths P from src to v inside the
 * window of the sum of P's edge durations (waiting is free); out[src] = 0;
 * KAIROS_UNREACHED otherwise.  strict: 0 Succeeds, 1 StrictlySucceeds.
 * Method: label-correcting rounds over edge labels D(e) = lambda_e + f_u(t_e), where f_u(tau)
 * is the least label of u's in-edges arriving by tau, kept as suffix minima over u's in-edges
 * in the reversed graph's order; at most n rounds.  The first call builds the reverse-slot
 * map of the edges (one radix sort) and per-edge uint32 arrays (reverse slot, label, suffix
 * minimum, and per predicate used the in-time slot), kept with the graph and freed with it.
 * Needs the reverse graph (not built with skip_reverse: INVALID_ARG).  out: uint32_t[n], host
 * or device.  stats (may be NULL): rounds and usable edges examined.  Synchronous.
 * Errors: INVALID_ARG, TIMEOUT (round cap), OOM, CUDA. */
typedef struct {
    uint64_t rounds;          /* relaxation rounds run */
    uint64_t examined_edges;  /* usable out-edges of active vertices, summed over the rounds */
} kairos_duration_stats;

kairos_status kairos_shortest_duration(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, int32_t strict,
                                       uint32_t *out, kairos_duration_stats *stats);

/* Temporal BFS from src within [ta, tw] (Table 4's T. BFS, read over time-respecting paths; the
 * paper gives no definition): out[v] = the least number of edges of a time-respecting path
 * from src to v inside the window; out[src] = 0; KAIROS_UNREACHED otherwise.  The same
 * computation as kairos_shortest_duration with every edge costing 1; same arguments, state,
 * stats and errors. */
kairos_status kairos_temporal_bfs(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, int32_t strict,
                                  uint32_t *out, kairos_duration_stats *stats);

/* Temporal connected components within [ta, tw] (the temporal connectivity application of
 * Sec. 2.3 and Table 4, adapted to a start and end time as Sec. 6 describes; the paper gives no
 * further definition, and this reading is the components of the window's snapshot): the
 * connected components of the undirected graph formed by the edges usable in the window
 * (t >= ta and t + lambda <= tw), every vertex included.  out[v] = the smallest vertex id of
 * v's component (v itself when it has no usable edge); out: uint32_t[n], host or device.
 * Method: one pass of concurrent union-find over the usable edges (larger root linked under
 * the smaller by compare-and-swap, path halving), then every vertex takes its root.
 * Synchronous.  Errors: INVALID_ARG (NULL, ta > tw, tw > KAIROS_TIME_MAX), OOM, CUDA,
 * INTERNAL (a link retry loop ran past its bound). */
kairos_status kairos_temporal_cc(kairos_graph *g, uint32_t ta, uint32_t tw, uint32_t *out);

/* ---- launch shape ----------------------------------------------------------------- */

kairos_status kairos_get_tuning(const kairos_graph *g, kairos_tuning *t);
/* Errors: INVALID_ARG when a field is outside the documented set. */
kairos_status kairos_set_tuning(kairos_graph *g, const kairos_tuning *t);

/* Time a grid of launch shapes on `sample` (its queries are run, results discarded) and
 * install the fastest; *best (may be NULL) receives it.  The grid covers the frontier modes
 * (lane widths 1-32, split thresholds, queue or bitmap frontier, relaxation modes 0-2, then chunk
 * size, resident blocks and two launches in flight) and the time-ordered mode 3 (32 and 64
 * lanes, one, two or four launches in flight, three block sizes).  Errors as kairos_batch_query. */
kairos_status kairos_autotune(kairos_graph *g, const kairos_query *sample, int32_t n, kairos_tuning *best);

/* The same search over lane widths of at least min_lanes only (large batches on large graphs,
 * where narrow launches cannot win and take long to time).  Errors as kairos_autotune, and
 * INVALID_ARG for min_lanes < 1. */
kairos_status kairos_autotune_from(kairos_graph *g, const kairos_query *sample, int32_t n, int32_t min_lanes,
                                   kairos_tuning *best);

/* Selective-index threshold by measurement (the cost model of Sec. 5.1 sets the cutoff
 * experimentally): for each of the n_thetas candidates (KAIROS_NO_INDEX allowed) rebuild
 * the fence level, time `sample` with the current launch shape, and keep the fastest.
 * ms_out (may be NULL) receives each candidate's device time.  *best (may be NULL) gets the
 * chosen threshold, which stays built.  Errors as kairos_batch_query / kairos_index_build. */
kairos_status kairos_autotune_index(kairos_graph *g, const kairos_query *sample, int32_t n, const uint32_t *thetas,
                                    int32_t n_thetas, uint32_t *best, double *ms_out);

/* ---- continuous-batching server ------------------------------------------------------ */

typedef struct {
    int32_t max_slots;      /* queries resident at once per query kind (lanes of the running
                               edge-map): 2, 4, 8, 16 or 32; 0: 16.  Lowered at start while the
                               device cannot hold that many beside reserve_bytes */
    int32_t queue_capacity; /* pending submissions before submit returns BUSY; 0: 4096 */
    int64_t reserve_bytes;  /* device memory to leave free; no query is admitted while free
                               memory is below it; 0: 256 MiB */
    int32_t rounds_per_slice; /* edge-map rounds per launch between admissions; 0: 2 */
} kairos_serve_opts;

typedef struct {
    kairos_status status;     /* the query's own outcome */
    uint32_t reached;         /* vertices with a finite label */
    uint64_t relaxed_edges;   /* as in kairos_query_stats */
    uint64_t checksum;        /* sum over v of (v + 1) * out[v], mod 2^64 */
    double latency_ms;        /* submit to completion, host clock */
} kairos_result_info;

/* Start a server thread on g (which must outlive it).  It keeps one resumable batched
 * edge-map per query kind (earliest arrival on the forward graph, latest departure on the
 * mirrored one) and alternates launches of rounds_per_slice rounds between them.  Between
 * launches it retires every lane whose query finished (no label changed in its last
 * round: the labels are read out on the device into the ticket's buffer) and admits
 * waiting queries into free lanes (their column is reset and their source joins the
 * running frontier), so queries that arrive while others run share the device with them.
 * Every answer equals that of the same query run alone.  Errors: INVALID_ARG, OOM, CUDA. */
kairos_status kairos_serve_create(kairos_graph *g, const kairos_serve_opts *opts, kairos_server **out);

/* Enqueue one query; out: uint32_t[n], host or device, must stay valid until the ticket
 * is polled OK.  Non-blocking.  Thread-safe.  Errors: INVALID_ARG, BUSY (queue full). */
kairos_status kairos_serve_submit(kairos_server *s, const kairos_query *q, uint32_t *out, uint64_t *ticket);

/* Wait up to timeout_us (0: do not wait, < 0: forever) for a ticket.  OK with *info filled
 * (the ticket is then retired), NOT_READY if still running, INVALID_ARG for an unknown
 * ticket.  Thread-safe. */
kairos_status kairos_serve_poll(kairos_server *s, uint64_t ticket, int64_t timeout_us, kairos_result_info *info);

/* Finish in-flight work, stop the thread and release the server.  NULL is ignored. */
void kairos_serve_destroy(kairos_server *s);

/* ---- one query stream over several server replicas --------------------------------------- */

/* Queries are independent, so serving on several GPUs means one graph replica and one server
 * per GPU (each built and created with that GPU current) behind one submission point; the
 * replicas share nothing and nothing is exchanged between them (Sec. 8(e) of the plan: replicas,
 * no collective).  A submission whose out buffer is device memory goes to the least-loaded
 * replica on that buffer's device (its labels are written in place there); a host buffer goes
 * to the least-loaded replica of all.  Load is submitted minus completed queries; ties go to the
 * replica after the last one chosen; a replica whose queue is full passes the query on.  The
 * router borrows the servers, which must outlive it.  Thread-safe. */
typedef struct kairos_router kairos_router;

/* servers: n >= 1 server handles.  Errors: INVALID_ARG (NULL, n < 1), OOM. */
kairos_status kairos_router_create(kairos_server *const *servers, int32_t n, kairos_router **out);

/* As kairos_serve_submit, on the replica chosen as above; *ticket is the router's.  Errors:
 * INVALID_ARG (NULL, no replica on the device of a device buffer, or the replica's own checks),
 * BUSY (every eligible replica's queue is full). */
kairos_status kairos_router_submit(kairos_router *r, const kairos_query *q, uint32_t *out, uint64_t *ticket);

/* As kairos_serve_poll on the replica that took the ticket (waits without blocking other
 * callers).  Errors: INVALID_ARG (unknown ticket), NOT_READY. */
kairos_status kairos_router_poll(kairos_router *r, uint64_t ticket, int64_t timeout_us, kairos_result_info *info);

/* Per replica (in creation order, up to n): queries submitted to it and completed there (any
 * array may be NULL).  Returns the number of replicas, 0 on a NULL router. */
int32_t kairos_router_replica_counts(const kairos_router *r, uint64_t *submitted, uint64_t *completed, int32_t n);

void kairos_router_destroy(kairos_router *r); /* NULL is ignored; the servers stay */

/* ---- query without device allocation ------------------------------------------------------ */

/* Earliest arrival from src within [ta, tw] under Succeeds, like kairos_earliest_arrival,
 * but allocating no device memory at all.  The paper has no counterpart: this serves
 * callers that cannot allocate while they query, such as a process that hands all of
 * its device memory to its own pool at start-up, or code called while another library
 * captures a CUDA graph and forbids new allocations.  The graph itself must have been
 * built beforehand (building allocates).
 * out: uint32_t[n_vertices] in DEVICE memory, owned by the caller; it holds the labels
 * throughout the query.  All other scratch lives in one fixed array compiled into the
 * library (about 15.5 MB, held on every GPU that loads the library until the process
 * exits) and limits the graph to at most 2^20 vertices, with its long adjacency ranges
 * fitting 65536 split entries and 262144 chunks per round; larger graphs get
 * INVALID_ARG with a message saying so.
 * The first call on a device looks the array up (cudaGetSymbolAddress); make that first
 * call before any stream capture.  Every call on a device shares the array: calls whose
 * GPU work can overlap (other streams, other threads without ordering) race on it and
 * must be serialised by the caller.  Synchronous on the graph's stream: it enqueues
 * memsets, a launch and small reads there and waits for them.  A caller that runs it
 * while another thread captures a CUDA graph must have built the graph with its own
 * stream (kairos_graph_opts.stream, not the legacy default stream, whose work would
 * invalidate a capture elsewhere), and that stream must not be the one being captured.
 * Errors: INVALID_ARG (NULL, out not device memory of the current device, vertex or
 * window out of range, graph over the limits), TIMEOUT (a device wait or the round cap
 * ran out), CUDA. */
kairos_status kairos_earliest_arrival_noalloc(kairos_graph *g, int32_t src, uint32_t ta, uint32_t tw, uint32_t *out);

/* ---- diagnostics -------------------------------------------------------------------- */

const char *kairos_last_error(void);
const char *kairos_status_string(kairos_status s);
/* Device time (ms) of the last query call's edge-map launches on g (sum), measured with
 * CUDA events on the graph's stream. */
double kairos_last_kernel_ms(const kairos_graph *g);

/* Round profile of the last edge-map launch on g: per round (up to max_rounds, at most
 * 256) the frontier size, the number of grid-wide chunks its long ranges were cut into, and
 * the round's device time in ms (from the GPU's global timer).  Any output may be NULL.
 * Returns the number of rounds written.  Diagnostic only; not synchronised with other
 * threads using g. */
int32_t kairos_last_round_profile(const kairos_graph *g, int32_t max_rounds, uint32_t *frontier, uint32_t *chunks,
                                  double *ms);

/* Cycle counts of the last edge-map launch, summed over warps, for 8 phases: lane-state
 * gather, range search, chunk registration, local walk, chunk wait, chunk walk, grid
 * barrier, other.  Zero unless the process ran with KAIROS_PHASE_CLOCK=1 in its
 * environment.  Returns 8, or 0 on a NULL argument.  Diagnostic only. */
int32_t kairos_last_phase_cycles(const kairos_graph *g, uint64_t *cycles8);

/* Counters of the last time-ordered (relax_mode 3) launch on g: out23 = {time blocks swept,
 * fix-up rounds, fix-up vertices, edges read by fix-ups, records whose lanes were examined,
 * records and edges read in all, then SM cycles summed over warps in block passes (reading and
 * filtering records), fix-ups, grid barriers with initialisation and read-out, and the passes'
 * candidate relaxations, then the pass's candidate records with 1, 2-4, 5-16 and 17-64
 * candidate lanes, the candidate lanes in all, the candidates (pass and fix-ups) that lowered
 * some label, the labels lowered, then thread block 0's wall time (ns) in passes, grid-wide
 * fix-up rounds and one-block fix-up runs, each with its closing grid barrier, and the number
 * of each (the cycles and everything from the lane counts on are zero unless the process ran
 * with KAIROS_PHASE_CLOCK=1)}.  Returns 23, or 0 on a NULL argument.  Diagnostic only. */
int32_t kairos_last_stream_profile(const kairos_graph *g, uint64_t *out23);

#ifdef __cplusplus
}
#endif

#endif /* KAIROS_H */
