/*
 * CPU oracle for exact warehouse pick routing -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C.  It shares no code with the CUDA
 * path.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never calls it.
 *
 * What it computes (arXiv 2504.20655):
 *   - single-source shortest path distances by round-based Bellman-Ford
 *     over the arc list (Sec. 4.7, GPU Implementation: every round relaxes
 *     every arc u->v with weight w, at most V-1 rounds), cross-checked by
 *     Dijkstra as in the Remark of Sec. 4.7, by a FIFO Bellman-Ford-Moore
 *     queue, and by Floyd-Warshall on small graphs;
 *   - for one order (depot P_0, picks P_1..P_k): D[i][j] = dist(P_i, P_j)
 *     and the minimum over all k! pick sequences pi of
 *         cost(pi) = D[0][pi_1] + sum_{i<k} D[pi_i][pi_{i+1}] + D[pi_k][0]
 *     (Sec. 4.6: n! routes, each evaluated over its transitions; routes are
 *     orderings of the stops, Sec. 2.4), keeping the lexicographically
 *     first minimiser, by brute force in lexicographic order and by
 *     Held-Karp (Sec. 3 reference point) with lexicographic reconstruction.
 *
 * Conventions (readings of points the paper leaves open):
 *   - distances are int32, unreachable = OR_INF (INT32_MAX); weights >= 0;
 *     a graph whose distances could reach OR_INF is refused (or_graph_check),
 *     and no distance at or above OR_INF is ever cast to int32 (OR_EDIST);
 *   - a tour with an unreachable leg is not a candidate; if every tour has
 *     one the order is OR_UNREACHABLE (cost OR_INF, perm = identity);
 *   - any finite off-diagonal D entry above OR_LEG_MAX makes the order
 *     OR_RANGE (cost OR_INF, perm = identity): 13 legs of at most
 *     OR_LEG_MAX stay below 2^27, so exact sums fit int32;
 *   - k < 1, k above the solver's limit (OR_MAX_K for brute force, OR_MAX_K_HK
 *     for Held-Karp) or a node id outside [0, V) is OR_BADORDER;
 *   - 21 legs of at most OR_LEG_MAX stay below 2^31, so Held-Karp sums for
 *     k <= 20 are exact in int32 as well;
 *   - perm[j] is the 0-based index into the order's own pick list.
 */
#ifndef WROUTE_ORACLE_H
#define WROUTE_ORACLE_H
#include <stdint.h>

#define OR_INF INT32_MAX
#define OR_MAX_K 12      /* brute force: 12! = 479,001,600 sequences, ranks fit int32 */
#define OR_MAX_K_HK 20   /* Held-Karp: 2^20 x 20 table entries */
#define OR_LEG_MAX 10324440
#define OR_OK 0
#define OR_UNREACHABLE 1
#define OR_BADORDER 2
#define OR_RANGE 3
/* error return: a finite distance would reach OR_INF (see or_graph_check) */
#define OR_EDIST (-4)

#define OR_SSSP_ROUNDS 0
#define OR_SSSP_FIFO 1
#define OR_SSSP_DIJKSTRA 2
#define OR_TOUR_BRUTE 0
#define OR_TOUR_HELDKARP 1
/* or-ed into tour_kind of the route functions: the route is an open path through the
 * picks, the entrance/exit (depot) not part of it (Sec. 3): every depot leg costs 0. */
#define OR_OPEN_PATH 16

#ifdef __cplusplus
extern "C" {
#endif

/* Out-arc CSR: arcs of u are [row_ptr[u], row_ptr[u+1]) with head col[] and weight w[].
 * The shortest-path functions return OR_EDIST instead of a distance at or above OR_INF. */
int or_bf_rounds(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                 int32_t src, int32_t* dist, int32_t* rounds_out);
int or_bf_fifo(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
               int32_t src, int32_t* dist);
int or_dijkstra(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                int32_t src, int32_t* dist);
/* dist is V*V, row-major dist[s*V + t]. */
int or_floyd_warshall(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                      int32_t* dist);

/* 0 when every finite distance of the graph must stay below OR_INF, by the bound
 * min((V-1) * max w, sum of w) over the arcs as given; OR_EDIST when the bound
 * reaches OR_INF; -1 on a malformed CSR.  or_route_orders refuses such graphs. */
int or_graph_check(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w);

/* Rows for n_src sources: rows[i*V + v] = dist(src[i], v).  kind = OR_SSSP_*. */
int or_sssp_rows(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                 int32_t n_src, const int32_t* src, int kind, int n_threads, int32_t* rows);

/* Tours over a (k+1)x(k+1) matrix D (row-major, index 0 = depot). */
int or_tour_brute(int32_t k, const int32_t* D, int32_t* cost, int32_t* perm);
int or_tour_held_karp(int32_t k, const int32_t* D, int32_t* cost, int32_t* perm);

/* Cluster-patched approximate route of Sec. 3 over a (k+1)x(k+1) matrix D; xy holds
 * the k stops' plan coordinates (x0, y0, x1, y1, ...); at most m clusters of at most
 * 10 stops (more: OR_BADORDER); open_path != 0 leaves the depot legs out. */
int or_tour_clustered(int32_t k, const int32_t* D, const int32_t* xy, int32_t m, int open_path,
                      int32_t* cost, int32_t* perm);

/* The k-means step of the cluster-patched route (Sec. 3): farthest-first initial
 * centres, Lloyd steps until no assignment changes (at most 64).  Returns the number
 * of centres nc; assign[i] in [0, nc) is stop i's cluster; centre c's mean is
 * (Sx[c]/cnt[c], Sy[c]/cnt[c]) (arrays of at least min(m, k) entries); *steps (may be
 * NULL) = assignment passes run.  -1 on bad arguments (k outside 1..OR_MAX_K, m < 1). */
int or_kmeans(int32_t k, const int32_t* xy, int32_t m, int32_t* assign, int64_t* Sx, int64_t* Sy,
              int64_t* cnt, int32_t* steps);

/* Whole path for a batch of orders; picks of order i are picks[offs[i]..offs[i+1]). */
int or_route_orders(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                    int32_t depot, int32_t n_orders, const int64_t* offs, const int32_t* picks,
                    int sssp_kind, int tour_kind, int n_threads,
                    int32_t* cost, int32_t* perm, int32_t* status);

/* Routing of orders whose distance rows are given: rows[r*V + v] for the
 * source node src_nodes[r] (sorted ascending, must contain every node used). */
int or_route_with_rows(int32_t V, int32_t depot, int32_t n_rows, const int32_t* src_nodes,
                       const int32_t* rows, int32_t n_orders, const int64_t* offs,
                       const int32_t* picks, int tour_kind, int n_threads,
                       int32_t* cost, int32_t* perm, int32_t* status);

/* Counting helpers used by the pins: n!, and the Theorem of Sec. 3:
 * m! * 2^(m-1) + (n_1! + ... + n_m!)/2. */
int64_t or_factorial(int32_t n);
int64_t or_patched_route_count(int32_t m, const int32_t* n_j);

#ifdef __cplusplus
}
#endif
#endif
