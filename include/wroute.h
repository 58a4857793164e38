/*
 * wroute.h -- C ABI of the GB300 (sm_103a) exact warehouse pick-routing library.
 *
 * The routing hot path of arXiv 2504.20655:
 *   (a) multi-source Bellman-Ford over the warehouse graph (Sec. 4.7:
 *       min-plus relaxation d[v] = min(d[v], d[u] + w(u, v)) until nothing
 *       changes, at most V-1 rounds), giving each order its pick-location
 *       distance matrix D[i][j] = dist(P_i, P_j) with P_0 the depot;
 *   (b) exhaustive evaluation of the order's pick sequences over D
 *       (Sec. 4.6: all n! sequences, each costed over its transitions;
 *       a route is an ordering of the stops, Sec. 2.4), split into
 *       rank-range segments whose partial minima are reduced
 *       (the segmentation strategy of the abstract and Sec. 6).
 *
 * Result of an order with picks P_1..P_k (1 <= k <= WR_MAX_K):
 *   cost = min over permutations pi of
 *          D[0][pi_1] + D[pi_1][pi_2] + ... + D[pi_{k-1}][pi_k] + D[pi_k][0]
 *   perm = the lexicographically first minimiser, perm[j] = pi_{j+1} - 1,
 *          i.e. a 0-based index into the order's own pick list.
 * All arithmetic is int32 and bit-exact.
 *
 * Conventions for every call:
 *   - Memory: inputs are borrowed for the duration of the call (the graph
 *     is copied); outputs are allocated by the caller.  ptr_kind says
 *     whether the caller's pointers are host (WR_HOST) or device
 *     (WR_DEVICE) memory of the context's device.
 *   - Streams: work is enqueued on cuda_stream (a cudaStream_t, NULL =
 *     the legacy default stream).  With WR_DEVICE outputs the call returns
 *     once the work is enqueued; results are valid after that stream
 *     synchronises.  With WR_HOST outputs the call returns after the
 *     results have been copied back.
 *   - Errors: every entry point returns WR_OK or one of the WR_E* codes
 *     below and leaves the context usable.  Device-side failures (a
 *     bounded wait that timed out, the sweep cap) are recorded in the
 *     context and returned by the next wr_sync() or host-output call.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef WROUTE_H
#define WROUTE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define WR_OK        0
#define WR_EINVAL    1  /* bad argument, malformed CSR, negative weight, distances that could reach
                           WR_INF (see wr_load_graph), size out of range */
#define WR_ENOMEM    2  /* allocation failed, or the memory budget holds fewer than 32 rows */
#define WR_ECUDA     3  /* a CUDA runtime call failed */
#define WR_ETIMEOUT  4  /* a bounded device-side wait (grid barrier) ran out */
#define WR_ENOGRAPH  5  /* no graph loaded */
#define WR_EINTERNAL 6  /* an internal bound or check failed (Bellman-Ford past its sweep cap, a Held-Karp table without an optimal next pick): cannot happen with w >= 0 */

/* per-order status */
#define WR_ORDER_OK          0
#define WR_ORDER_UNREACHABLE 1  /* every sequence has an unreachable leg: cost WR_INF, perm identity */
#define WR_ORDER_BAD         2  /* k < 1, k > WR_MAX_K or a node id outside [0, V): cost WR_INF */
#define WR_ORDER_RANGE       3  /* a finite D entry exceeds WR_LEG_MAX: cost WR_INF, perm identity */

/* pointer kinds */
#define WR_HOST   0
#define WR_DEVICE 1

/* route shapes (wr_set_route_mode) */
#define WR_ROUTE_TOUR 0  /* closed tour: depot -> picks -> depot (default) */
#define WR_ROUTE_OPEN 1  /* open path through the picks: the entrance/exit is not part of the route
                            (Sec. 3), so the depot's legs are free; one of every reversed pair is
                            the lexicographically first, so the result is the same as over the
                            paper's n!/2 undirected routes when D is symmetric */

#define WR_MAX_K   12          /* exhaustive enumeration: 12! = 479001600 ranks fit int32 */
#define WR_MAX_K_EXACT 20      /* with max_k above WR_MAX_K, orders of 13..max_k picks are solved exactly by
                                  Held-Karp (same optimum, same tie rule), wr_route_orders only */
#define WR_INF     2147483647  /* unreachable distance */
#define WR_LEG_MAX 10324440    /* 13 legs of at most this stay below 2^27: exact int32 sums */

typedef struct wr_ctx wr_ctx;  /* opaque; owns all device memory it allocates */

typedef struct {
    int device;                   /* CUDA device ordinal */
    uint64_t mem_budget_bytes;    /* cap on the distance-row buffer of one source segment */
    int max_k;                    /* largest order size accepted, <= WR_MAX_K_EXACT (default WR_MAX_K) */
    uint64_t barrier_max_spins;   /* iteration limit of every device-side wait (0 = default) */
    const char* tune_path;        /* tuning table file: applied at creation when it exists, written by
                                     wr_autotune (NULL = built-in defaults, nothing written) */
} wr_config;

/* Tunables (picked by the autotuner; results never depend on them). */
typedef struct {
    int32_t run_target;     /* Bellman-Ford tile: target nodes per run (consecutive ids) */
    int32_t tile_cap;       /* nodes (run + halo) staged in shared memory per tile: 128, 256 or 512 */
    int32_t enum_units;     /* sequence units per thread per scheduled chunk (a unit: a prefix and the
                               5040 orderings of the last 7 picks; for k >= 11, a set of the first
                               k - 7 picks (k = 12: and its first pick), the next pick, and the
                               orderings of the set (24) and of the last 6 (720); an order of k <= 6
                               is one unit) */
    int32_t enum_max_units_per_launch; /* rank-range segment: units per enumeration launch (0 = all) */
    int32_t bf_warps;       /* CTA tiling: warps sharing one sweep tile, 4 or 8 (0 = 8 for 512-node tiles, else 4) */
    int32_t bf_tiling;      /* sweep tiling: 1 = one warp per tile (lane = source; tile_cap 128 or 256),
                               2 = one CTA per tile (quads of sources per warp), 3 = warp tiles driven by
                               an asynchronous worklist instead of sweeps (tile_cap 128 or 256; no sweep
                               trace, wr_stats.sweeps = 0), 4 = warp tiles of two 32-source groups
                               (lane = source of each; tile_cap 128); 0 = 1 up to 256-slot tiles, else 2.
                               Defaults: tile_cap 128, run_target 60, warp tiles */
} wr_tuning;

/* Counters of the last call (device-timed with CUDA events on its stream). */
typedef struct {
    int64_t n_orders;
    int64_t n_sources;        /* distinct Bellman-Ford sources (depot + distinct pick nodes) */
    int64_t n_segments;       /* source segments run */
    int64_t sweeps;           /* Bellman-Ford sweeps, summed over segments */
    int64_t tile_visits;      /* (run, 32-source group) tiles processed, summed over sweeps */
    int64_t node_visits;      /* node x 32-lane group visits */
    int64_t bytes_alg;        /* algorithmic bytes of the sweeps: per sweep, 8*32 per visited
                                 (node, 32-source group) (own lanes read + written), plus
                                 8*indeg + 8 (arcs, row pointer) once per node visited in any group */
    int64_t sequences;        /* pick sequences evaluated */
    int64_t kernel_launches;  /* kernels launched by the call */
    float ms_select, ms_init, ms_bf, ms_gather, ms_enum, ms_finish, ms_total;
    int64_t bytes_reread;     /* descriptor bytes read again for a node's further groups within a
                                 sweep (overhead, not in bytes_alg; the worklist tiling counts
                                 every visit's descriptors in bytes_alg and leaves this 0) */
} wr_stats;

/* Create a context on cfg->device (NULL cfg = defaults: device 0, 2 GiB budget, max_k 12). */
int wr_create(const wr_config* cfg, wr_ctx** out);
void wr_destroy(wr_ctx* ctx);
const char* wr_strerror(int code);

/* Wait for all work the context enqueued and return any recorded device-side error. */
int wr_sync(wr_ctx* ctx);

/* a1 -- Load the graph (Sec. 4.7 keeps it as arrays u, v, w; here out-arc CSR):
 * arcs of node u are [row_ptr[u], row_ptr[u+1]) with heads col[] and int32
 * weights w[] >= 0.  row_ptr has V+1 entries, row_ptr[0] = 0, row_ptr[V] = E.
 * depot in [0, V) is P_0 of every order.  Copies everything; replaces any
 * previous graph.  WR_EINVAL on malformed input or a negative weight.
 * Distances are int32 and WR_INF marks an unreachable node, so a finite distance
 * must stay below WR_INF.  Every shortest path is simple (w >= 0): it has at most
 * V - 1 arcs and uses no arc twice.  The graph is therefore accepted only when
 *   min((V - 1) * max w, sum of all w) < WR_INF     (over the arcs as given),
 * and WR_EINVAL otherwise; every finite distance is then exact. */
int wr_load_graph(wr_ctx* ctx, int32_t V, int64_t E, const int64_t* row_ptr, const int32_t* col,
                  const int32_t* w, int32_t depot, int ptr_kind);

/* a1-a7 -- Route a batch of orders.  Order i has picks picks[offs[i] .. offs[i+1]),
 * offs has n_orders+1 non-decreasing entries with offs[0] = 0 (checked for host
 * input, WR_EINVAL; with device input offs[0] != 0 or offs[n] < 0 is WR_EINVAL
 * and no pick is read, and an order whose range leaves [0, offs[n]] is
 * reported WR_ORDER_BAD and gets no perm writes).
 * Writes cost[i], status[i] and perm[offs[i] + j].
 * Sources (depot + distinct pick nodes) are deduplicated on the device and
 * processed in segments of at most mem_budget_bytes of rows. */
int wr_route_orders(wr_ctx* ctx, int32_t n_orders, const int64_t* offs, const int32_t* picks,
                    int32_t* cost, int32_t* perm, int32_t* status, int ptr_kind, void* cuda_stream);

/* a3 -- Distance rows: rows[i * ld + v] = dist(src[i], v) for i < n_src, v < V
 * (WR_INF when unreachable), ld >= V.  src entries must lie in [0, V). */
int wr_bf_rows(wr_ctx* ctx, int32_t n_src, const int32_t* src, int32_t* rows, int64_t ld,
               int ptr_kind, void* cuda_stream);

/* a2+a3 at scale -- Produce the rows of n_src sources segment by segment under the
 * memory budget.  For each segment, consume(user, first, count, dev_rows, ld) is
 * called on the host once the segment's kernels are enqueued on cuda_stream;
 * dist(src[first + b], v) = dev_rows[v * ld + b] for b < count (node-major,
 * device memory, valid for work the consumer enqueues on the same stream).  The
 * buffer is reused after consume returns.  A non-zero return from consume stops
 * the call and is returned. */
typedef int (*wr_consume_fn)(void* user, int32_t first, int32_t count, const int32_t* dev_rows,
                             int64_t ld);
int wr_distance_rows(wr_ctx* ctx, int32_t n_src, const int32_t* src, int ptr_kind,
                     wr_consume_fn consume, void* user, void* cuda_stream);

/* Built-in consumer of wr_distance_rows for the scale workload: sub[i * n_dst + j] =
 * dist(src[i], dst[j]) and a per-row checksum
 *   check[i] = sum over v of (uint64)(uint32)dist(src[i], v) * (2v + 1)   (mod 2^64). */
int wr_submatrix(wr_ctx* ctx, int32_t n_src, const int32_t* src, int32_t n_dst, const int32_t* dst,
                 int32_t* sub, uint64_t* check, int ptr_kind, void* cuda_stream);

/* a5-a7 on given matrices -- D is n_orders blocks of 13 x 13 int32 (row-major,
 * the top-left (k+1) x (k+1) used, index 0 = depot, WR_INF = unreachable);
 * k[i] picks per order (k[i] <= WR_MAX_K: larger orders are WR_ORDER_BAD here).  Writes cost[i],
 * status[i] and perm[i * WR_MAX_K + j]. */
int wr_tour_eval(wr_ctx* ctx, int32_t n_orders, const int32_t* k, const int32_t* D, int32_t* cost,
                 int32_t* perm, int32_t* status, int ptr_kind, void* cuda_stream);

/* Tour evaluation that allocates no device memory (the paper has no counterpart).
 * For callers that cannot call cudaMalloc: a process whose device memory is owned
 * by another allocator (a framework's caching allocator, a fixed arena) that must
 * not be grown or fragmented behind its back, or a latency-critical loop that
 * cannot take the device-wide synchronisation cudaMalloc/cudaFree may imply.
 * Same results as wr_tour_eval on a context with the default max_k (orders of
 * 1..WR_MAX_K picks are evaluated, others are WR_ORDER_BAD), with the same
 * arguments and no context, computed on the current device.  All pointers must be device-accessible (device memory, or
 * managed/mapped memory); the work is enqueued on cuda_stream.
 * Scratch: a file-scope device array sized for WR_STATIC_MAX_ORDERS orders
 * (about 2.9 MB), held by every device that loads the library until the
 * process exits.  n_orders > WR_STATIC_MAX_ORDERS returns WR_EINVAL.
 * Set-up: a call outside any stream capture looks up the array's device address
 * on the current device, every time, so the address stays right after a
 * cudaDeviceReset; make the first call on a device, and the first call after a
 * cudaDeviceReset, before any stream capture.  Every call shares
 * the one array, so calls that overlap on the GPU (other streams, other host
 * threads) race: order them on one stream or synchronise between them. */
#define WR_STATIC_MAX_ORDERS 4096
int wr_tour_eval_static(int32_t n_orders, const int32_t* k, const int32_t* D, int32_t* cost,
                        int32_t* perm, int32_t* status, void* cuda_stream);

int wr_get_stats(wr_ctx* ctx, wr_stats* out);

/* Sweep trace (observability; the paper has no counterpart).  With max_sweeps > 0
 * every Bellman-Ford segment records, for each sweep t < max_sweeps, the number of
 * (run, 32-source group) tiles in its frontier and the device clock (ns) at which it
 * started; one more entry with 0 tiles marks the end.  Each segment overwrites the
 * previous segment's trace.  0 turns tracing off.  WR_EINVAL above 2^20. */
int wr_set_trace(wr_ctx* ctx, int32_t max_sweeps);
/* Copies up to max_entries (tiles, ns) pairs of the last segment's trace to
 * out[2i], out[2i+1] and sets *n_out to the number recorded (0 when tracing is off). */
int wr_get_trace(wr_ctx* ctx, int64_t* out, int32_t max_entries, int32_t* n_out);
/* Batching (the paper has no counterpart).  A plan captures the whole path (a1-a7) for
 * one batch of n_orders orders into a CUDA graph that is launched again and again on new
 * batch contents.  offs (n_orders + 1 entries), picks (max_picks), cost (n_orders), perm
 * (max_picks) and status (n_orders) are DEVICE buffers owned by the caller; every launch
 * reads offs/picks and writes cost/perm/status exactly as wr_route_orders would.  Each
 * batch must have offs[0] = 0 and offs[n_orders] <= max_picks (an order whose range leaves
 * [0, max_picks] comes back WR_ORDER_BAD).  A smaller batch is padded with empty orders
 * (offs[i+1] = offs[i]), which come back WR_ORDER_BAD.  The plan keeps a private copy of
 * the context's graph and tuning (taken at creation) and its own work buffers, so later
 * calls on the context do not disturb it; enum_max_units_per_launch is not used (one
 * enumeration launch).  Creation runs the path once uncaptured to size every buffer.
 * Launches of one plan must not overlap on the GPU (they share its work buffers). */
typedef struct wr_plan wr_plan;
int wr_plan_create(wr_ctx* ctx, int32_t n_orders, int64_t max_picks, const int64_t* offs, const int32_t* picks,
                   int32_t* cost, int32_t* perm, int32_t* status, wr_plan** out);
int wr_plan_launch(wr_plan* plan, void* cuda_stream);
/* Waits for the plan's last launch and returns any recorded device-side error. */
int wr_plan_sync(wr_plan* plan);
/* Counters and phase times of the last launch (the graph holds event-record nodes). */
int wr_plan_get_stats(wr_plan* plan, wr_stats* out);
void wr_plan_destroy(wr_plan* plan);

/* Autotuner (the paper has no counterpart).  Times wr_route_orders on the given batch
 * (median device time of `reps` calls after a warm-up, CUDA events) for each candidate
 * sweep tiling (warp or CTA tiles, tile_cap, run_target), then for each enumeration
 * chunk size with the best tiling, and applies the fastest tuning to the context.
 * Results never depend on the tuning, only the speed does.  When the context was
 * created with cfg.tune_path, the chosen tuning is written there ("name value"
 * lines) and read back by wr_create.  Writes the choice to *out when out != NULL.
 * Each candidate re-partitions the graph on the host. */
int wr_autotune(wr_ctx* ctx, int32_t n_orders, const int64_t* offs, const int32_t* picks, int ptr_kind,
                int32_t reps, wr_tuning* out);

/* Serving (the paper has no counterpart).  A server routes a stream of orders that
 * arrive over time, in real time, with the graph and a cache of distance rows
 * resident on the device.  Continuous batching: whenever one of n_slots slots is
 * free, the orders that have arrived (up to max_batch orders and max_batch_picks
 * picks) form a batch; the rows of its sources the cache lacks are computed by
 * multi-source Bellman-Ford straight into cache columns (least-recently-used groups
 * of 32 columns are evicted, never one the batch reads), every order's matrix is
 * gathered from the cache, and the enumeration runs on the slot's own stream, so
 * batches overlap on the GPU.  Admission stops growing a batch when its new sources
 * would not fit the cache.  Every result equals that of wr_route_orders on the
 * order alone.  The server keeps a private copy of the context's graph and tuning.
 * It routes orders of up to WR_MAX_K picks (larger ones come back WR_ORDER_BAD). */
typedef struct {
    int32_t max_batch;        /* orders per batch, >= 1 */
    int64_t max_batch_picks;  /* picks per batch, >= WR_MAX_K; also the largest order accepted */
    int32_t n_slots;          /* batches in flight, 1..8 */
    uint64_t cache_bytes;     /* device budget of the row cache: at least 512 rows of V int32 */
    int32_t plain;            /* 1 = the baseline: one order at a time, rows from scratch, no cache
                                 (the other fields are ignored) */
} wr_serve_config;

typedef struct {
    int64_t orders, batches;
    int64_t cache_hits;      /* sources of admitted orders found in the cache */
    int64_t rows_computed;   /* sources whose rows were computed */
    int64_t evicted_groups;  /* 32-column groups reused */
    int64_t bf_launches;
    double wall_s;           /* duration of the last run */
} wr_serve_stats;

typedef struct wr_server wr_server;
int wr_serve_create(wr_ctx* ctx, const wr_serve_config* cfg, wr_server** out);
/* Routes n_orders orders; order i (picks[offs[i] .. offs[i+1])) arrives arrival_s[i]
 * seconds after the call starts (non-decreasing).  All pointers are host memory.
 * Writes cost[i], status[i], perm[offs[i] + j] as wr_route_orders does, and done_s[i]
 * = when its result was on the host (seconds since the call started).  Returns when
 * every order is done. */
int wr_serve_run(wr_server* sv, int32_t n_orders, const double* arrival_s, const int64_t* offs, const int32_t* picks,
                 int32_t* cost, int32_t* perm, int32_t* status, double* done_s);
int wr_serve_get_stats(wr_server* sv, wr_serve_stats* out);
/* While a server runs, its batches overlap on the GPU and share the context's device
 * counters, so wr_get_stats on that context reports mixed figures then; wr_serve_stats
 * (host-side counts of the last wr_serve_run) is the server's own record. */
void wr_serve_destroy(wr_server* sv);

/* Node-level routes (the nodes a route passes; the paper has no API for them).  For each
 * order (picks[offs[i] .. offs[i+1])) and its pick sequence perm[offs[i] + j] (0-based indices
 * into the order's picks, e.g. from wr_route_orders), the route's nodes: the depot, then the
 * nodes of each leg after its first, ending at the depot (WR_ROUTE_TOUR), or in WR_ROUTE_OPEN
 * mode the first pick and then the legs between consecutive picks.  A leg s -> t is the
 * shortest path whose nodes read backward from t are lexicographically smallest: walking back
 * from t, the predecessor of v is the smallest node id u with an arc u -> v and
 * dist(s,u) + w(u,v) = dist(s,v).
 * Writes node_offs (n_orders + 1 entries; order i's nodes are nodes[node_offs[i] ..
 * node_offs[i+1])); an order that is invalid (status WR_ORDER_BAD, or perm not a permutation
 * of 0..k-1) or has an unreachable leg gets no nodes.  With nodes == NULL only node_offs is
 * written; if node_offs[n_orders] > max_nodes nothing more is written and WR_ENOMEM is
 * returned (node_offs is valid: call again with a larger buffer).  Requires every arc weight
 * > 0 (with zero-weight arcs the walk may cycle): WR_EINVAL otherwise.  Recomputes the rows of
 * the sources (twice for batches needing more than one segment). */
int wr_route_nodes(wr_ctx* ctx, int32_t n_orders, const int64_t* offs, const int32_t* picks, const int32_t* perm,
                   int64_t* node_offs, int32_t* nodes, int64_t max_nodes, int ptr_kind, void* cuda_stream);

/* Cluster-patched approximate routing (Sec. 3; the paper's own method for large orders).
 * With m > 0, wr_route_orders and plans created afterwards route every order of at most
 * WR_MAX_K picks by: k-means (at most m clusters) on the picks' plan coordinates
 * (wr_set_node_coords), the first optimal open route inside every cluster (at most 10
 * picks, else WR_ORDER_BAD), and the cheapest patching over every order and direction of
 * the clusters (depot legs included for WR_ROUTE_TOUR), ties to the lexicographically
 * first sequence.  cost is the patched route's cost (not the optimum).  m = 0 (the
 * default) routes exactly.  1 <= m <= 6, WR_EINVAL otherwise; wr_route_orders returns
 * WR_EINVAL while m > 0 and no coordinates are set; servers refuse m > 0. */
int wr_set_clusters(wr_ctx* ctx, int32_t m);
/* Plan coordinates of the nodes, xy[2v], xy[2v+1] (int32, |x|, |y| <= 2^20), for the
 * clustered routing; copied; cleared by wr_load_graph. */
int wr_set_node_coords(wr_ctx* ctx, const int32_t* xy, int ptr_kind);

/* Route shape of wr_route_orders, plans and servers created afterwards (WR_ROUTE_TOUR or
 * WR_ROUTE_OPEN); wr_tour_eval uses the matrices as given.  WR_EINVAL otherwise. */
int wr_set_route_mode(wr_ctx* ctx, int mode);

int wr_get_tuning(wr_ctx* ctx, wr_tuning* out);
/* Changing run_target or tile_cap re-partitions the loaded graph. */
int wr_set_tuning(wr_ctx* ctx, const wr_tuning* t);

#ifdef __cplusplus
}
#endif
#endif /* WROUTE_H */
