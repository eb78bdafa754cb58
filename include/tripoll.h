/*
 * tripoll.h -- C ABI of the B300 metadata triangle survey library (libtripoll.so).
 *
 * The library computes surveys of triangles in decorated temporal graphs, the
 * operation of TriPoll (Steil et al., arXiv 2107.12330): every triangle of an
 * undirected graph is found exactly once in the degree-ordered directed graph
 * G+ (Sec. 3) by intersecting out-lists (Sec. 4.3, Alg. 1), and the metadata of
 * each triangle -- three vertex labels, three edge timestamps, three edge
 * labels (meta(Delta_pqr), Sec. 3) -- is folded into exact integer tables, the
 * GPU-resident counterpart of the user callbacks of Sec. 4.5 (Alg. 2, 3, 4).
 *
 * Conventions shared by every entry point:
 *   - Pointers marked "device or host" may point to device memory or to host
 *     memory (pageable or pinned); the library detects which and copies host
 *     data itself.  The caller keeps ownership of every buffer it passes.
 *   - All GPU work is ordered on the caller's CUDA stream `cuda_stream`
 *     (a cudaStream_t; NULL = the legacy default stream).  Entry points that
 *     return graph statistics or write host memory synchronise that stream.
 *   - Every call returns a tripoll_status.  Arguments are validated before any
 *     kernel that writes caller memory runs; on failure nothing is left
 *     allocated and *out handles are not written.
 *   - All arithmetic is integer; results are bit-exact and independent of the
 *     schedule.
 *   - Vertex ids are uint32 in [0, num_vertices); timestamps are uint32;
 *     labels are uint8 in [0, L).
 *   - Environment: TRIPOLL_MIRROR_MOVE_LOG2 = k (0 <= k, read at each survey
 *     call) makes the survey kernels move their on-chip partial sums into the
 *     result after every 2^k work items instead of every 2^9 (block kernels)
 *     or 2^14 (warp kernel) -- slower, same result; it exists so that tests
 *     can exercise those moves on small graphs.  Values above the defaults
 *     are ignored.
 */
#ifndef TRIPOLL_H
#define TRIPOLL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tripoll_graph* tripoll_graph_t;
typedef struct tripoll_server* tripoll_server_t;

typedef enum {
    TRIPOLL_OK = 0,
    TRIPOLL_ERR_INVALID_ARG = -1,    /* null handle/pointer, zero label count, t_lo > t_hi, ... */
    TRIPOLL_ERR_VERTEX_RANGE = -2,   /* an edge endpoint >= num_vertices */
    TRIPOLL_ERR_LABEL_RANGE = -3,    /* a vertex label >= num_vlabels or edge label >= num_elabels */
    TRIPOLL_ERR_NO_MEMORY = -4,      /* device allocation failed or a scratch budget would be exceeded */
    TRIPOLL_ERR_CUDA = -5,           /* a CUDA runtime call failed; see tripoll_last_error() */
    TRIPOLL_ERR_TIMEOUT = -6,        /* a bounded wait ran out */
    TRIPOLL_ERR_NO_EDGE_LABELS = -7, /* an edge-label survey on a graph built without edge labels */
    TRIPOLL_ERR_NOT_FOUND = -8       /* unknown request or graph slot */
} tripoll_status;

/* Survey kinds (bit mask).  The result buffer holds the requested tables in
 * this order, each immediately after the previous one (uint64 words):
 *
 *   TRIPOLL_COUNT           1 word   number of triangles in the window (Alg. 2).
 *   TRIPOLL_CLOSURE_HIST   33 words  closing time t3 - t1 of the sorted edge
 *                                    timestamps t1 <= t2 <= t3, counted in bin
 *                                    ceil(log2(t3 - t1)); differences 0 and 1
 *                                    both land in bin 0 (Sec. 5.7, Alg. 4).
 *   TRIPOLL_VLABEL_TRIPLES Lv^3      sorted vertex-label triple a <= b <= c at
 *                                    index (a*Lv + b)*Lv + c; other entries 0.
 *   TRIPOLL_ELABEL_TRIPLES Le^3      the same over the three edge labels.
 *   TRIPOLL_OPEN_CLOSE_HIST 33*33    joint (open, close) table of Alg. 4 at
 *                                    index open*33 + close, open = ceil(log2(t2 - t1)).
 *   TRIPOLL_MAX_ELABEL     Le        Alg. 3: among triangles whose three vertex
 *                                    labels are pairwise distinct, the count per
 *                                    maximum edge label.
 *   TRIPOLL_DEGREE_TRIPLES 33^3      Sec. 5.9:  sorted triple of ceil(log2 d(v))
 *                                    of the three vertices (d = degree in the
 *                                    simple graph), indexed like the label triples.
 *   TRIPOLL_VERTEX_LOCAL   n         local triangle participation per vertex, by
 *                                    input vertex id (Sec. 5.3).
 *   TRIPOLL_EDGE_LOCAL     m         local triangle participation per edge of G+
 *                                    (Sec. 5.3), by the edge's CSR position:
 *                                    word off[p] + i is the i-th out-edge of the
 *                                    vertex at position p, whose endpoints are
 *                                    order[p] and order[col[off[p] + i]] (see
 *                                    tripoll_graph_export); m = num_edges.
 *
 * A triangle is surveyed iff its three edge timestamps all lie in the inclusive
 * window [t_lo, t_hi]; [0, 0xFFFFFFFF] surveys every triangle.  The window
 * selects triangles, not degrees: every table equals the survey of the
 * subgraph of the edges whose timestamp lies in the window, except
 * TRIPOLL_DEGREE_TRIPLES, whose d(v) stays the degree in the whole simple
 * graph (the window leaves the order <+ of Sec. 3 unchanged too). */
enum {
    TRIPOLL_COUNT = 1,
    TRIPOLL_CLOSURE_HIST = 2,
    TRIPOLL_VLABEL_TRIPLES = 4,
    TRIPOLL_ELABEL_TRIPLES = 8,
    TRIPOLL_OPEN_CLOSE_HIST = 16,
    TRIPOLL_MAX_ELABEL = 32,
    TRIPOLL_DEGREE_TRIPLES = 64,
    TRIPOLL_VERTEX_LOCAL = 128,
    TRIPOLL_EDGE_LOCAL = 256
};
#define TRIPOLL_ALL_KINDS 511u
#define TRIPOLL_HIST_BINS 33u

/* Statistics of a built graph (G+ of Sec. 3).  Sizes are counts, not bytes. */
typedef struct {
    uint64_t num_vertices;   /* n */
    uint64_t num_input_edges;/* records passed to create */
    uint64_t num_edges;      /* m = |E+|: unique undirected edges after loop removal and dedup */
    uint64_t wedges;         /* |W+| = sum_p C(d+(p), 2) (Sec. 3) */
    uint64_t dplus_max;      /* max_p d+(p) */
    uint64_t degree_max;     /* max_v d(v) */
    uint64_t q_list_words;   /* sum over directed edges (p,q) of d+(q): out-list entries read once per in-edge */
    uint64_t num_graphs;     /* 1, or the number of graphs of a batched build */
    uint32_t num_vlabels;
    uint32_t num_elabels;    /* 0 when the graph has no edge labels */
    uint64_t device_bytes;   /* HBM held by the graph */
} tripoll_graph_info;

/* The survey plan of a graph: how middle vertices q are split into work items
 * (the load balancing of the wedge checks; the paper's Sec. 4.2 notes hub
 * imbalance, which the degree order only partly removes) and how a window is
 * applied.  Results never depend on it; speed does, by workload.
 *   warp_max_dplus       out-lists up to this length are surveyed one item per
 *                        warp (32..256; larger ones one item per block).
 *   block_item_in_edges  in-edges (p,q) per block item (256..2048, a multiple
 *                        of 256).
 *   long_list_min_dplus  out-lists longer than this go to the long-list kernel
 *                        (2048-entry parts; 1024..65536).
 *   window_view          1: a window compacts G+ to its in-window edges first
 *                        (tripoll_survey); 0: out-of-window edges are skipped
 *                        where they are met (no extra memory).
 * The bounds keep every on-chip partial sum below 2^32.  Defaults: 128, 2048,
 * 4096, 1. */
typedef struct {
    uint32_t warp_max_dplus;
    uint32_t block_item_in_edges;
    uint32_t long_list_min_dplus;
    uint32_t window_view;
} tripoll_plan;

/* Build G+ on the device (Sec. 3, Sec. 4.2): drop records with src == dst; merge
 * all records of an unordered pair into one edge keeping the lexicographic
 * minimum (timestamp, then edge label) -- the chronologically first record of
 * Sec. 5.2; compute degrees of the simple graph; order vertices by
 * (degree, id) -- the order <+ of Sec. 3 with the vertex id as tie-break;
 * direct each edge from its <+ -smaller end; store sorted out-lists (CSR) with
 * timestamp and edge-label arrays aligned to them and vertex labels permuted
 * to <+ order.
 *
 *   src, dst, ts  device or host, uint32[num_edges]: edge records.
 *   elabel        device or host, uint8[num_edges], or NULL (no edge labels).
 *   vlabel        device or host, uint8[num_vertices], or NULL (all labels 0).
 *   num_vlabels   >= 1 (1 when vlabel is NULL); num_elabels >= 1 when elabel != NULL.
 *   Errors: VERTEX_RANGE / LABEL_RANGE when a record or label is out of range,
 *   NO_MEMORY, CUDA.  Synchronises cuda_stream. */
int tripoll_graph_create(const uint32_t* src, const uint32_t* dst, const uint32_t* ts,
                         const uint8_t* elabel, uint64_t num_edges, const uint8_t* vlabel,
                         uint32_t num_vertices, uint32_t num_vlabels, uint32_t num_elabels,
                         void* cuda_stream, tripoll_graph_t* out);

/* Build one G+ holding many independent graphs (the batched workload).  Graph
 * i owns input records [edge_offsets[i], edge_offsets[i+1]) with vertex ids
 * local to it in [0, num_vertices[i]), and vertex labels at
 * vlabel[sum_{j<i} num_vertices[j] + v].  Each graph is built exactly as
 * tripoll_graph_create would build it alone.
 *   edge_offsets  host, uint64[num_graphs + 1], edge_offsets[0] == 0.
 *   num_vertices  host, uint32[num_graphs].
 * Other arguments as in tripoll_graph_create.  Synchronises cuda_stream. */
int tripoll_batch_create(const uint32_t* src, const uint32_t* dst, const uint32_t* ts,
                         const uint8_t* elabel, const uint64_t* edge_offsets,
                         const uint8_t* vlabel, const uint32_t* num_vertices, uint32_t num_graphs,
                         uint32_t num_vlabels, uint32_t num_elabels, void* cuda_stream,
                         tripoll_graph_t* out);

/* Number of uint64 words of a result for kind_mask: the sizes of the tables
 * listed above (the folds of Alg. 2, 3, 4, Sec. 5.3 and Sec. 5.9), summed
 * (TRIPOLL_VERTEX_LOCAL adds num_vertices words, TRIPOLL_EDGE_LOCAL num_edges
 * -- the unique edges of G+, tripoll_graph_stats' num_edges).  Host-only; no
 * error status (an unknown bit adds nothing). */
uint64_t tripoll_result_words(uint32_t kind_mask, uint32_t num_vlabels, uint32_t num_elabels,
                              uint64_t num_vertices, uint64_t num_edges);

/* Run one survey (Alg. 1 with the fold of the requested kinds) over every
 * triangle of g whose edge timestamps lie in [t_lo, t_hi].  A window other
 * than [0, 0xFFFFFFFF] first compacts G+ and its in-edge records to the
 * in-window edges (about 26 bytes per in-window edge of stream-ordered pool
 * memory, 30 with per-edge counts, and 0.75 per edge of G+, released when
 * the survey ends), so that wedges through an out-of-window edge are never
 * checked.  Sizing that view reads the in-window edge count back: the call
 * then waits for cuda_stream's earlier work and the view's first kernels.
 *   result  device or host, uint64[tripoll_result_words(kinds, ...)]; overwritten.
 *           For a batched graph: uint64[num_graphs * words], graph i's tables
 *           at offset i * words.
 *   Errors: INVALID_ARG (t_lo > t_hi, kind_mask == 0 or unknown bits),
 *   NO_EDGE_LABELS, NO_MEMORY, CUDA.  Asynchronous for a device result
 *   (apart from that wait); synchronises cuda_stream for a host result. */
int tripoll_survey(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi,
                   uint64_t* result, void* cuda_stream);

/* The same survey restricted to the pivots p (the <+ -smallest vertex of each
 * triangle, Sec. 3) at positions [pivot_lo, pivot_hi) of the <+ order.  The
 * sum of the results over a partition of [0, n) equals tripoll_survey's
 * result: this is the unit a multi-GPU run shards (each rank one range, then
 * one elementwise sum, the all_reduce of Alg. 2). */
int tripoll_survey_range(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi,
                         uint64_t pivot_lo, uint64_t pivot_hi, uint64_t* result,
                         void* cuda_stream);

/* Several survey requests on one graph in one pass: the unit the server
 * batches, usable on its own.  Request k surveys kinds kind_masks[k] over the
 * window [t_lo[k], t_hi[k]] into results[k]; every result equals
 * tripoll_survey's for that request alone.  The wedge checks (Sec. 3, Alg. 1)
 * of the union of the windows are made once, and each triangle found is
 * folded once -- into the cell of the requests' window bounds that holds its
 * earliest and latest edge timestamps (Alg. 4 takes the same two times); a
 * request's tables are the sum of the cells inside its window.
 *   count        1..64.
 *   kind_masks, t_lo, t_hi   host, uint32[count]; no TRIPOLL_VERTEX_LOCAL or
 *                TRIPOLL_EDGE_LOCAL; the graph is not a batched one.
 *   results      host, array of count pointers, each device or host memory of
 *                tripoll_result_words(kind_masks[k], ...) words.
 *   Scratch: the union window's view (see tripoll_survey) plus (distinct lower
 *   bounds) x (distinct upper bounds) records of the union of the kinds.
 *   Errors: INVALID_ARG, NO_EDGE_LABELS, NO_MEMORY (also when that record grid
 *   would reach 2^31 words: split the requests), CUDA.  Asynchronous when every
 *   result is device memory, else synchronises cuda_stream. */
int tripoll_survey_many(tripoll_graph_t g, uint32_t count, const uint32_t* kind_masks,
                        const uint32_t* t_lo, const uint32_t* t_hi, uint64_t* const* results,
                        void* cuda_stream);

/* tripoll_survey_range with the device time of each phase, for measurement:
 * CUDA events recorded on cuda_stream around each phase give phase_ms[0]
 * (building the window view), [1] (the kernel of middle vertices with short
 * out-lists, one per warp), [2] (the block-per-item kernel) and [3] (the
 * kernel of the longest out-lists), in milliseconds; a phase that does not run
 * reads 0.  phase_ms: host, float[4].  The result is the same as
 * tripoll_survey_range's.  Errors: those of tripoll_survey_range, INVALID_ARG
 * for a NULL phase_ms.  Synchronises cuda_stream. */
int tripoll_survey_timed(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi,
                         uint64_t pivot_lo, uint64_t pivot_hi, uint64_t* result, float* phase_ms,
                         void* cuda_stream);

/* tripoll_survey for callers that cannot allocate device memory where they
 * survey -- loops that must never enter an allocator (an allocation may block
 * on the driver or on other streams), or hosts whose device memory belongs to
 * another framework.  The paper has no counterpart; this is a library
 * convenience.  Same arguments, kernels and result as tripoll_survey, but the
 * call allocates nothing: its scratch (the accumulation record and two work
 * counters) is a static 8 MiB device array that every GPU loading the library
 * holds until the process exits, and a window is applied in place (no window
 * view: out-of-window edges are skipped where they are met).
 *   - The first call on a device looks up that array's device address (kept
 *     for the life of the process, so the device's primary context must not
 *     be reset while the library is loaded); make that first call before any
 *     stream capture on the device.
 *   - Every call reuses the same array (each call clears the part it needs):
 *     calls whose GPU work overlaps -- on different streams, or from different
 *     threads -- race and corrupt each other's results.  Order them on one
 *     stream or with events.
 *   - The current device must be the graph's device.
 *   - Errors: NO_MEMORY when the result (tripoll_result_words x 8 bytes, times
 *     the graph count of a batched graph) exceeds 8 MiB less 256 bytes; the
 *     argument errors of tripoll_survey.  Synchronises cuda_stream for a host
 *     result. */
int tripoll_survey_static(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi,
                          uint64_t* result, void* cuda_stream);

/* The plan of g (*plan: host).  Errors: INVALID_ARG for NULL arguments. */
int tripoll_get_plan(tripoll_graph_t g, tripoll_plan* plan);

/* Give g another plan: its work items are rebuilt on cuda_stream (a few
 * kernels over the vertices; no survey may run on g meanwhile).  Errors:
 * INVALID_ARG for a plan outside the bounds above, NO_MEMORY, CUDA.
 * Synchronises cuda_stream. */
int tripoll_set_plan(tripoll_graph_t g, const tripoll_plan* plan, void* cuda_stream);

/* The plan graphs built from now on start with (process-wide; NULL restores
 * the defaults).  Errors: INVALID_ARG for a plan outside the bounds. */
int tripoll_set_default_plan(const tripoll_plan* plan);

/* The autotuner: time surveys of g (kinds, window) under candidate plans and
 * keep the fastest.  Coordinate descent from g's current plan: each field in
 * turn takes each of its candidate values (warp_max_dplus 32, 64, 128, 256;
 * block_item_in_edges 512, 1024, 2048; long_list_min_dplus 2048, 4096, 8192;
 * window_view 1, 0 when the window is not the full range) with the others
 * fixed; a plan's time is the median of `reps` surveys (device time, CUDA
 * events on cuda_stream, after one untimed survey).  g ends with the best plan,
 * which *best (host) receives with its time *best_ms and the starting plan's
 * time *start_ms (both host, may be NULL).  Errors: those of tripoll_survey
 * and tripoll_set_plan.  Synchronises cuda_stream. */
int tripoll_tune(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi, uint32_t reps,
                 tripoll_plan* best, float* best_ms, float* start_ms, void* cuda_stream);

/* Split [0, n) into `parts` pivot ranges of near-equal survey cost (the
 * out-list entries each pivot's wedge checks read).  bounds: host,
 * uint64[parts + 1], bounds[0] = 0, bounds[parts] = n.  Synchronises. */
int tripoll_partition_pivots(tripoll_graph_t g, uint32_t parts, uint64_t* bounds,
                             void* cuda_stream);

/* Statistics of g (Sec. 3: n, |E+|, |W+| = sum C(d+,2), max d+; the paper
 * reports the same figures per dataset in Table 2), in one struct rather
 * than separate out-parameters.  *info: host, written on success.  Errors:
 * INVALID_ARG for a NULL handle or info.  No device work. */
int tripoll_graph_stats(tripoll_graph_t g, tripoll_graph_info* info);

/* Number of wedge checks (Sec. 3: a wedge (p,q),(p,r) with q <+ r, checked for
 * the closing edge (q,r)) that a survey over the window [t_lo, t_hi] performs:
 * the wedges of the subgraph of in-window edges, i.e. both (p,q) and (p,r) in
 * the window (others cannot close into a surveyed triangle), sum over pivots p
 * of C(k, 2) with k the in-window edges of Adj+(p).  [0, 0xFFFFFFFF] gives
 * |W+|.  *out: host.  Synchronises. */
int tripoll_wedge_checks(tripoll_graph_t g, uint32_t t_lo, uint32_t t_hi, uint64_t* out, void* cuda_stream);

/* Copy out the built G+ (for checking the builder): any pointer may be NULL.
 *   offsets  uint64[n+1], col uint32[m] (targets as positions in <+), ts
 *   uint32[m], elabel uint8[m], order uint32[n] (input id at each position).
 *   All host pointers.  Synchronises cuda_stream. */
int tripoll_graph_export(tripoll_graph_t g, uint64_t* offsets, uint32_t* col, uint32_t* ts,
                         uint8_t* elabel, uint32_t* order, void* cuda_stream);

/* Release the graph's device memory: the arrays of G+ and Adj+^m (Sec. 4.2)
 * and the survey plan, each returned to the allocator that made it, ordered on
 * the legacy default stream.  The caller must not destroy a graph while
 * surveys on it may still run on some stream, nor while a server holds it.
 * NULL is ignored; no status. */
void tripoll_destroy(tripoll_graph_t g);

/* ---- serving: resident graphs, continuous batching of survey requests ----
 *
 * A server owns a dispatcher thread and a set of CUDA streams.  Requests
 * (graph slot, kinds, window) are admitted in arrival order in rounds, while
 * fewer than max_inflight requests are on the device and the round's device
 * scratch fits under scratch_cap_bytes.  In a round, the requests on one graph
 * form one batch (up to 64) that runs as one pass, as tripoll_survey_many
 * does; a batch of one request runs as tripoll_survey.  Batches of different
 * graphs run at once on different streams, every request that arrives
 * meanwhile joins a later round, and a batch on a graph of 2^25 edges or more
 * runs only when no other such batch does (the requests queue up and the next
 * round takes them in one pass).  A batch is charged its records, its results
 * and the window view of its (union) window when the budget holds that too;
 * otherwise it skips out-of-window edges in place.  Results are the same as
 * tripoll_survey's for each request alone.  Requests for local counts, and
 * requests on batched graphs, run one per batch. */
int tripoll_server_create(uint64_t scratch_cap_bytes, uint32_t max_inflight,
                          tripoll_server_t* out);
/* Make g resident in the server (the server does not take ownership).  The
 * first time a graph is added, a histogram of its timestamps is taken (a few
 * kernels on the current device, which must be g's, and a read-back; the
 * call synchronises) so that a request is charged the window view of the
 * edges its window can hold rather than of all of them. */
int tripoll_server_add_graph(tripoll_server_t s, tripoll_graph_t g, uint32_t* slot);
/* Queue a request; returns its id.  Thread-safe. */
int tripoll_server_submit(tripoll_server_t s, uint32_t slot, uint32_t kind_mask, uint32_t t_lo,
                          uint32_t t_hi, uint64_t* request_id);
/* Wait up to timeout_ms for a request; on success copy its result (host,
 * uint64[words]) and its latency in nanoseconds (submit to result on host).
 * TIMEOUT when it is not done in time (it stays queued). */
int tripoll_server_wait(tripoll_server_t s, uint64_t request_id, uint64_t* result,
                        uint64_t* latency_ns, uint32_t timeout_ms);
/* Counters of the server so far (for measurement; no counterpart in the paper):
 * stats[0] requests launched, [1] batches, [2] survey passes (a fused batch
 * is one pass, a batch run request by request is one pass each), [3] requests
 * surveyed in fused passes.  stats: host, uint64[4]. */
int tripoll_server_stats(tripoll_server_t s, uint64_t* stats);
void tripoll_server_destroy(tripoll_server_t s);

/* Number of the library's own kernels launched by this process so far (not
 * counting launches made inside CUB routines).  For launch accounting only. */
uint64_t tripoll_launch_count(void);

/* ---- device memory ----
 *
 * By default every device array and temporary of the library comes from a
 * stream-ordered memory pool private to the library (one per device; it keeps
 * up to a quarter of the device's memory, at most 64 GiB, cached between
 * calls).  The caller's default pool and its settings are not touched.
 *
 * tripoll_set_allocator installs the caller's allocator instead -- e.g. a
 * framework's caching allocator, so that the library draws from the memory the
 * framework already holds (a library hook; the paper, whose method runs on
 * host memory, has no counterpart).  alloc(bytes, stream, ctx) returns device memory of the
 * current device, at least 256-byte aligned, that work ordered on `stream`
 * after the call may use, or NULL when it cannot (the library then fails with
 * TRIPOLL_ERR_NO_MEMORY and returns everything it holds; memory that is not
 * 256-byte aligned is handed back to free_fn and treated the same way).  free_fn(ptr, bytes,
 * stream, ctx) takes back one allocation; work ordered on `stream` before the
 * call may still be using it.  Graph arrays are returned on the legacy default
 * stream (NULL) by tripoll_destroy.  Both functions may be called from any
 * thread, including the server's dispatcher thread.  Every allocation is
 * returned to the allocator that made it, even after another one has been
 * installed.  Passing alloc == NULL (with free_fn == NULL) restores the
 * library's pool.  Install the allocator before the calls that should use it;
 * changing it while other threads call the library is allowed but which
 * allocator an in-flight call uses is then unspecified.
 *   Errors: INVALID_ARG when exactly one of alloc, free_fn is NULL. */
typedef void* (*tripoll_alloc_fn)(size_t bytes, void* cuda_stream, void* ctx);
typedef void (*tripoll_free_fn)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
int tripoll_set_allocator(tripoll_alloc_fn alloc, tripoll_free_fn free_fn, void* ctx);

/* Human-readable text of a status, and the detail of the calling thread's
 * last error (static storage; never NULL). */
const char* tripoll_status_string(int status);
const char* tripoll_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TRIPOLL_H */
