/*
 * CPU oracle for exact warehouse pick routing -- TEST INFRASTRUCTURE ONLY.
 * See oracle.h for what is computed and the conventions taken.  Nothing in
 * the product path calls this file; it shares no code with the CUDA path.
 */
#include "oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;
#define BIG ((i64)1 << 62)

/* ------------------------------------------------------------------ */
/* Single-source shortest paths                                        */
/* ------------------------------------------------------------------ */

/* Distances are int32 with OR_INF (2^31 - 1) meaning unreachable: a finite
 * distance (below BIG) at or above OR_INF has no int32 value and is an
 * error, never a cast. */
static int fits_int32(const i64* d, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (d[i] < BIG && d[i] >= (i64)OR_INF) return 0;
    return 1;
}

/* The graph rule: a shortest path is simple (w >= 0), so it has at most V-1
 * arcs and uses no arc twice; its length is at most min((V-1) max w, sum w),
 * taken over the arcs as given.  The graph is accepted when that bound is below
 * OR_INF, so every finite distance fits int32. */
int or_graph_check(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w) {
    if (V <= 0 || row_ptr[0] != 0) return -1;
    i64 max_w = 0, sum_w = 0;
    for (int32_t u = 0; u < V; ++u) {
        if (row_ptr[u + 1] < row_ptr[u]) return -1;
        for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a) {
            if (col[a] < 0 || col[a] >= V || w[a] < 0) return -1;
            if (w[a] > max_w) max_w = w[a];
            if (sum_w < BIG) sum_w += w[a];
        }
    }
    i64 bound = (i64)(V - 1) * max_w;
    if (sum_w < bound) bound = sum_w;
    return bound < (i64)OR_INF ? 0 : OR_EDIST;
}

/* Sec. 4.7: Bellman-Ford relaxes every arc of the arc list per round and
 * needs at most V-1 rounds.  Each round here reads the previous round's
 * distances (a Jacobi round); the loop stops at the first round that
 * changes nothing, which leaves the same fixpoint. */
int or_bf_rounds(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                 int32_t src, int32_t* dist, int32_t* rounds_out) {
    if (V <= 0 || src < 0 || src >= V) return -1;
    i64* cur = (i64*)malloc(sizeof(i64) * (size_t)V);
    i64* nxt = (i64*)malloc(sizeof(i64) * (size_t)V);
    if (!cur || !nxt) { free(cur); free(nxt); return -2; }
    for (int32_t v = 0; v < V; ++v) cur[v] = BIG;
    cur[src] = 0;
    int32_t rounds = 0;
    for (int32_t r = 0; r < V - 1; ++r) {
        int changed = 0;
        memcpy(nxt, cur, sizeof(i64) * (size_t)V);
        for (int32_t u = 0; u < V; ++u) {
            if (cur[u] >= BIG) continue;
            for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a) {
                i64 cand = cur[u] + (i64)w[a];
                if (cand < nxt[col[a]]) { nxt[col[a]] = cand; changed = 1; }
            }
        }
        i64* t = cur; cur = nxt; nxt = t;
        if (!changed) break;
        ++rounds;
    }
    if (!fits_int32(cur, (size_t)V)) { free(cur); free(nxt); return OR_EDIST; }
    for (int32_t v = 0; v < V; ++v) dist[v] = cur[v] >= BIG ? OR_INF : (int32_t)cur[v];
    if (rounds_out) *rounds_out = rounds;
    free(cur); free(nxt);
    return 0;
}

/* Bellman-Ford-Moore: a FIFO queue of vertices whose distance dropped. */
int or_bf_fifo(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
               int32_t src, int32_t* dist) {
    if (V <= 0 || src < 0 || src >= V) return -1;
    i64* d = (i64*)malloc(sizeof(i64) * (size_t)V);
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
    char* inq = (char*)calloc((size_t)V, 1);
    if (!d || !q || !inq) { free(d); free(q); free(inq); return -2; }
    for (int32_t v = 0; v < V; ++v) d[v] = BIG;
    d[src] = 0;
    int64_t head = 0, count = 1;
    q[0] = src; inq[src] = 1;
    while (count > 0) {
        int32_t u = q[head]; head = (head + 1) % V; --count; inq[u] = 0;
        for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a) {
            int32_t v = col[a];
            i64 cand = d[u] + (i64)w[a];
            if (cand < d[v]) {
                d[v] = cand;
                if (!inq[v]) { q[(head + count) % V] = v; ++count; inq[v] = 1; }
            }
        }
    }
    if (!fits_int32(d, (size_t)V)) { free(d); free(q); free(inq); return OR_EDIST; }
    for (int32_t v = 0; v < V; ++v) dist[v] = d[v] >= BIG ? OR_INF : (int32_t)d[v];
    free(d); free(q); free(inq);
    return 0;
}

/* Dijkstra with a binary heap of (key, vertex) and lazy deletion. */
typedef struct { i64 key; int32_t v; } hitem;

static void heap_push(hitem* h, int64_t* n, hitem x) {
    int64_t i = (*n)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].key <= x.key) break;
        h[i] = h[p]; i = p;
    }
    h[i] = x;
}

static hitem heap_pop(hitem* h, int64_t* n) {
    hitem top = h[0];
    hitem last = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && h[c + 1].key < h[c].key) ++c;
        if (last.key <= h[c].key) break;
        h[i] = h[c]; i = c;
    }
    if (*n > 0) h[i] = last;
    return top;
}

int or_dijkstra(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                int32_t src, int32_t* dist) {
    if (V <= 0 || src < 0 || src >= V) return -1;
    int64_t E = row_ptr[V];
    i64* d = (i64*)malloc(sizeof(i64) * (size_t)V);
    char* done = (char*)calloc((size_t)V, 1);
    hitem* h = (hitem*)malloc(sizeof(hitem) * (size_t)(E + 1));
    if (!d || !done || !h) { free(d); free(done); free(h); return -2; }
    for (int32_t v = 0; v < V; ++v) d[v] = BIG;
    d[src] = 0;
    int64_t n = 0;
    hitem s0 = {0, src};
    heap_push(h, &n, s0);
    while (n > 0) {
        hitem it = heap_pop(h, &n);
        int32_t u = it.v;
        if (done[u]) continue;
        done[u] = 1;
        for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a) {
            int32_t v = col[a];
            i64 cand = d[u] + (i64)w[a];
            if (cand < d[v]) { d[v] = cand; hitem x = {cand, v}; heap_push(h, &n, x); }
        }
    }
    if (!fits_int32(d, (size_t)V)) { free(d); free(done); free(h); return OR_EDIST; }
    for (int32_t v = 0; v < V; ++v) dist[v] = d[v] >= BIG ? OR_INF : (int32_t)d[v];
    free(d); free(done); free(h);
    return 0;
}

int or_floyd_warshall(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                      int32_t* dist) {
    if (V <= 0 || V > 4096) return -1;
    size_t n = (size_t)V;
    i64* d = (i64*)malloc(sizeof(i64) * n * n);
    if (!d) return -2;
    for (size_t i = 0; i < n * n; ++i) d[i] = BIG;
    for (size_t i = 0; i < n; ++i) d[i * n + i] = 0;
    for (int32_t u = 0; u < V; ++u)
        for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a)
            if ((i64)w[a] < d[(size_t)u * n + (size_t)col[a]]) d[(size_t)u * n + (size_t)col[a]] = w[a];
    for (size_t m = 0; m < n; ++m)
        for (size_t i = 0; i < n; ++i) {
            if (d[i * n + m] >= BIG) continue;
            for (size_t j = 0; j < n; ++j) {
                if (d[m * n + j] >= BIG) continue;
                i64 c = d[i * n + m] + d[m * n + j];
                if (c < d[i * n + j]) d[i * n + j] = c;
            }
        }
    if (!fits_int32(d, n * n)) { free(d); return OR_EDIST; }
    for (size_t i = 0; i < n * n; ++i) dist[i] = d[i] >= BIG ? OR_INF : (int32_t)d[i];
    free(d);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Threaded drivers (static split of independent work items)           */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t V; const int64_t* row_ptr; const int32_t* col; const int32_t* w;
    int32_t n_src; const int32_t* src; int kind; int32_t* rows;
    int tid, nthr; int rc;
} rows_job;

static void* rows_worker(void* p) {
    rows_job* j = (rows_job*)p;
    j->rc = 0;
    for (int32_t i = j->tid; i < j->n_src; i += j->nthr) {
        int32_t* out = j->rows + (size_t)i * (size_t)j->V;
        int rc;
        if (j->kind == OR_SSSP_ROUNDS) rc = or_bf_rounds(j->V, j->row_ptr, j->col, j->w, j->src[i], out, 0);
        else if (j->kind == OR_SSSP_FIFO) rc = or_bf_fifo(j->V, j->row_ptr, j->col, j->w, j->src[i], out);
        else rc = or_dijkstra(j->V, j->row_ptr, j->col, j->w, j->src[i], out);
        if (rc) { j->rc = rc; return 0; }
    }
    return 0;
}

int or_sssp_rows(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                 int32_t n_src, const int32_t* src, int kind, int n_threads, int32_t* rows) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    rows_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < n_threads; ++t) {
        rows_job j = {V, row_ptr, col, w, n_src, src, kind, rows, t, n_threads, 0};
        jobs[t] = j;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], 0, rows_worker, &jobs[t]);
    rows_worker(&jobs[0]);
    int rc = jobs[0].rc;
    for (int t = 1; t < n_threads; ++t) { pthread_join(th[t], 0); if (jobs[t].rc) rc = jobs[t].rc; }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Tours                                                               */
/* ------------------------------------------------------------------ */

/* Cost of the closed tour 0 -> p[0] -> ... -> p[k-1] -> 0 over D, where p
 * holds pick indices 1..k; BIG if a leg is unreachable. */
static i64 tour_cost(int32_t k, const int32_t* D, const int32_t* p) {
    int32_t n = k + 1;
    i64 c = 0;
    int32_t prev = 0;
    for (int32_t i = 0; i <= k; ++i) {
        int32_t nx = (i < k) ? p[i] : 0;
        int32_t leg = D[prev * n + nx];
        if (leg == OR_INF) return BIG;
        c += leg;
        prev = nx;
    }
    return c;
}

/* Next permutation in lexicographic order; 0 when p was the last one. */
static int next_perm(int32_t* p, int32_t k) {
    int32_t i = k - 2;
    while (i >= 0 && p[i] >= p[i + 1]) --i;
    if (i < 0) return 0;
    int32_t j = k - 1;
    while (p[j] <= p[i]) --j;
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    for (int32_t a = i + 1, b = k - 1; a < b; ++a, --b) { t = p[a]; p[a] = p[b]; p[b] = t; }
    return 1;
}

static int range_check(int32_t k, const int32_t* D) {
    int32_t n = k + 1;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j)
            if (i != j && D[i * n + j] != OR_INF && (D[i * n + j] < 0 || D[i * n + j] > OR_LEG_MAX))
                return 0;
    return 1;
}

static void identity(int32_t k, int32_t* perm) {
    for (int32_t i = 0; i < k; ++i) perm[i] = i;
}

/* Sec. 4.6: every one of the k! sequences is evaluated, in lexicographic
 * order; a strict '<' keeps the first (lowest-rank) minimiser. */
int or_tour_brute(int32_t k, const int32_t* D, int32_t* cost, int32_t* perm) {
    if (k < 1 || k > OR_MAX_K) return OR_BADORDER;
    if (!range_check(k, D)) { *cost = OR_INF; identity(k, perm); return OR_RANGE; }
    int32_t p[OR_MAX_K], best_p[OR_MAX_K];
    for (int32_t i = 0; i < k; ++i) p[i] = i + 1;
    i64 best = BIG;
    do {
        i64 c = tour_cost(k, D, p);
        if (c < best) { best = c; memcpy(best_p, p, sizeof(int32_t) * (size_t)k); }
    } while (next_perm(p, k));
    if (best >= BIG) { *cost = OR_INF; identity(k, perm); return OR_UNREACHABLE; }
    *cost = (int32_t)best;
    for (int32_t i = 0; i < k; ++i) perm[i] = best_p[i] - 1;
    return OR_OK;
}

/* Held-Karp (Sec. 3 reference point): h(S, c) = cheapest way to start at
 * pick c having visited the pick set S (c in S), visit the rest and return
 * to the depot.  Reconstruction takes the smallest pick index attaining
 * the optimum at every step, which gives the lexicographically first
 * optimal sequence. */
int or_tour_held_karp(int32_t k, const int32_t* D, int32_t* cost, int32_t* perm) {
    if (k < 1 || k > OR_MAX_K_HK) return OR_BADORDER;
    if (!range_check(k, D)) { *cost = OR_INF; identity(k, perm); return OR_RANGE; }
    int32_t n = k + 1;
    uint32_t full = (1u << k) - 1u;
    size_t ns = (size_t)1 << k;
    i64* h = (i64*)malloc(sizeof(i64) * ns * (size_t)k);
    if (!h) return -2;
#define H(S, c) h[(size_t)(S) * (size_t)k + (size_t)(c)]
#define LEG(a, b) (D[(a) * n + (b)] == OR_INF ? BIG : (i64)D[(a) * n + (b)])
    for (uint32_t S = full + 1; S-- > 0;) {
        for (int32_t c = 0; c < k; ++c) {
            if (!(S & (1u << c))) continue;
            if (S == full) { H(S, c) = LEG(c + 1, 0); continue; }
            i64 best = BIG;
            for (int32_t j = 0; j < k; ++j) {
                if (S & (1u << j)) continue;
                i64 l = LEG(c + 1, j + 1);
                i64 r = H(S | (1u << j), j);
                if (l >= BIG || r >= BIG) continue;
                if (l + r < best) best = l + r;
            }
            H(S, c) = best;
        }
    }
    i64 best = BIG;
    for (int32_t j = 0; j < k; ++j) {
        i64 l = LEG(0, j + 1), r = H(1u << j, j);
        if (l < BIG && r < BIG && l + r < best) best = l + r;
    }
    if (best >= BIG) { free(h); *cost = OR_INF; identity(k, perm); return OR_UNREACHABLE; }
    /* reconstruct */
    uint32_t S = 0;
    int32_t cur = 0; /* matrix index of the current stop (0 = depot) */
    i64 remaining = best;
    for (int32_t pos = 0; pos < k; ++pos) {
        for (int32_t j = 0; j < k; ++j) {
            if (S & (1u << j)) continue;
            i64 l = LEG(cur, j + 1), r = H(S | (1u << j), j);
            if (l < BIG && r < BIG && l + r == remaining) {
                perm[pos] = j;
                S |= 1u << j;
                remaining = r;
                cur = j + 1;
                break;
            }
        }
    }
#undef H
#undef LEG
    free(h);
    *cost = (int32_t)best;
    return OR_OK;
}

/* Cluster-patched approximate route (Sec. 3): the k stops are grouped into
 * at most m clusters by k-means on their plan coordinates, an optimal open
 * route is found inside every cluster, and the cluster routes are patched
 * into one global route by trying every order of the clusters and every
 * travel direction of each (m! x 2^m candidates; the theorem of Sec. 3
 * counts m! x 2^(m-1) undirected ones).
 *
 * k-means: centres start at stop 0 and then, one by one, at the stop
 * farthest (squared Euclidean) from the centres so far, ties to the lowest
 * stop index, up to m centres (fewer if every remaining stop sits on a
 * centre).  Lloyd steps assign every stop to its nearest centre (ties to the
 * lowest centre) and move each non-empty centre to the mean of its stops,
 * until no assignment changes (at most 64 steps).  Distances to a mean
 * (Sx/c, Sy/c) are compared exactly as (c x - Sx)^2 + (c y - Sy)^2 over c^2.
 * Cluster route: the lexicographically first optimal open route over the
 * cluster's stops (legs between stops only).  Patching: the cheapest global
 * route, the depot legs included for closed tours (free for open paths),
 * ties to the lexicographically first stop sequence.  Clusters above 10
 * stops make the order OR_BADORDER. */
#define CL_MAX 10
static i64 leg64(const int32_t* D, int32_t n, int32_t a, int32_t b) {
    return D[a * n + b] == OR_INF ? BIG : (i64)D[a * n + b];
}
static int frac_less(i64 num1, i64 den1, i64 num2, i64 den2) { return num1 * den2 < num2 * den1; }

/* k-means on the stops' plan coordinates (Sec. 3 clusters the stops with
 * K-means): farthest-first initial centres, then Lloyd steps (assign every stop
 * to its nearest centre, move every non-empty centre to the mean of its stops)
 * until no assignment changes, at most 64 steps.  A centre is kept as the sums
 * (Sx, Sy) of its stops' coordinates and their count cnt, so the mean is
 * (Sx/cnt, Sy/cnt) without rounding; an initial centre is one stop (cnt = 1).
 * Returns the number of centres nc (assign[i] in [0, nc)); *steps = the number
 * of assignment passes run, the last one changing nothing unless the 64-step cap
 * was reached. */
int or_kmeans(int32_t k, const int32_t* xy, int32_t m, int32_t* assign, int64_t* Sx, int64_t* Sy,
              int64_t* cnt, int32_t* steps) {
    if (k < 1 || k > OR_MAX_K || m < 1) return -1;
    int32_t nc = 0;
    Sx[nc] = xy[0]; Sy[nc] = xy[1]; cnt[nc] = 1; ++nc;
    while (nc < m && nc < k) {
        int32_t best_i = -1;
        i64 best_d = -1;
        for (int32_t i = 0; i < k; ++i) {
            i64 dmin = -1;
            for (int32_t c = 0; c < nc; ++c) {
                i64 dx = (i64)xy[2 * i] - Sx[c], dy = (i64)xy[2 * i + 1] - Sy[c];
                i64 d = dx * dx + dy * dy;
                if (dmin < 0 || d < dmin) dmin = d;
            }
            if (dmin > best_d) { best_d = dmin; best_i = i; }
        }
        if (best_d <= 0) break;
        Sx[nc] = xy[2 * best_i]; Sy[nc] = xy[2 * best_i + 1]; cnt[nc] = 1; ++nc;
    }
    for (int32_t i = 0; i < k; ++i) assign[i] = -1;
    int32_t it = 0;
    while (it < 64) {
        ++it;
        int changed = 0;
        for (int32_t i = 0; i < k; ++i) {
            int32_t bc = 0;
            i64 bnum = 0, bden = 1;
            for (int32_t c = 0; c < nc; ++c) {
                i64 dx = cnt[c] * (i64)xy[2 * i] - Sx[c], dy = cnt[c] * (i64)xy[2 * i + 1] - Sy[c];
                i64 num = dx * dx + dy * dy, den = cnt[c] * cnt[c];
                if (c == 0 || frac_less(num, den, bnum, bden)) { bc = c; bnum = num; bden = den; }
            }
            if (assign[i] != bc) { assign[i] = bc; changed = 1; }
        }
        if (!changed) break;
        for (int32_t c = 0; c < nc; ++c) {
            i64 sx = 0, sy = 0, ct = 0;
            for (int32_t i = 0; i < k; ++i)
                if (assign[i] == c) { sx += xy[2 * i]; sy += xy[2 * i + 1]; ++ct; }
            if (ct > 0) { Sx[c] = sx; Sy[c] = sy; cnt[c] = ct; }
        }
    }
    if (steps) *steps = it;
    return nc;
}

int or_tour_clustered(int32_t k, const int32_t* D, const int32_t* xy, int32_t m, int open_path,
                      int32_t* cost, int32_t* perm) {
    if (k < 1 || k > OR_MAX_K || m < 1) return OR_BADORDER;
    if (!range_check(k, D)) { *cost = OR_INF; identity(k, perm); return OR_RANGE; }
    const int32_t n = k + 1;
    int32_t assign[OR_MAX_K];
    i64 Sx[OR_MAX_K], Sy[OR_MAX_K], cnt[OR_MAX_K];
    const int32_t nc = or_kmeans(k, xy, m, assign, Sx, Sy, cnt, 0);
    /* clusters in centre order, stops in increasing index */
    int32_t members[OR_MAX_K][OR_MAX_K], size[OR_MAX_K], M = 0;
    for (int32_t c = 0; c < nc; ++c) {
        int32_t sz = 0;
        for (int32_t i = 0; i < k; ++i)
            if (assign[i] == c) members[M][sz++] = i;
        if (sz == 0) continue;
        if (sz > CL_MAX) { *cost = OR_INF; identity(k, perm); return OR_BADORDER; }
        size[M++] = sz;
    }
    /* the first optimal open route inside every cluster */
    int32_t route[OR_MAX_K][OR_MAX_K];
    i64 fwd[OR_MAX_K], rev[OR_MAX_K];
    for (int32_t c = 0; c < M; ++c) {
        int32_t sz = size[c], p[OR_MAX_K], best_p[OR_MAX_K];
        for (int32_t i = 0; i < sz; ++i) p[i] = i;
        i64 best = BIG + 1;
        do {
            i64 t = 0;
            for (int32_t i = 0; i + 1 < sz && t < BIG; ++i) {
                i64 l = leg64(D, n, members[c][p[i]] + 1, members[c][p[i + 1]] + 1);
                t = l >= BIG ? BIG : t + l;
            }
            if (t < best) { best = t; memcpy(best_p, p, sizeof(int32_t) * (size_t)sz); }
        } while (next_perm(p, sz));
        for (int32_t i = 0; i < sz; ++i) route[c][i] = members[c][best_p[i]];
        fwd[c] = best;
        i64 r = 0;
        for (int32_t i = sz - 1; i > 0 && r < BIG; --i) {
            i64 l = leg64(D, n, route[c][i] + 1, route[c][i - 1] + 1);
            r = l >= BIG ? BIG : r + l;
        }
        rev[c] = r;
    }
    /* patching: every order of the clusters, every direction of each */
    int32_t order[OR_MAX_K], seq[OR_MAX_K], best_seq[OR_MAX_K];
    for (int32_t c = 0; c < M; ++c) order[c] = c;
    i64 best = BIG;
    int have = 0;
    do {
        for (uint32_t dir = 0; dir < (1u << M); ++dir) {
            int32_t len = 0;
            i64 t = 0;
            for (int32_t q = 0; q < M && t < BIG; ++q) {
                int32_t c = order[q], r = (dir >> q) & 1u;
                int32_t head = r ? route[c][size[c] - 1] : route[c][0];
                i64 inner = r ? rev[c] : fwd[c];
                i64 link = q == 0 ? (open_path ? 0 : leg64(D, n, 0, head + 1)) : leg64(D, n, seq[len - 1] + 1, head + 1);
                if (inner >= BIG || link >= BIG) { t = BIG; break; }
                t += link + inner;
                for (int32_t i = 0; i < size[c]; ++i) seq[len++] = r ? route[c][size[c] - 1 - i] : route[c][i];
            }
            if (t < BIG && !open_path) {
                i64 back = leg64(D, n, seq[k - 1] + 1, 0);
                t = back >= BIG ? BIG : t + back;
            }
            if (t >= BIG) continue;
            int better = !have || t < best;
            if (!better && t == best) {
                for (int32_t i = 0; i < k; ++i)
                    if (seq[i] != best_seq[i]) { better = seq[i] < best_seq[i]; break; }
            }
            if (better) { best = t; have = 1; memcpy(best_seq, seq, sizeof(int32_t) * (size_t)k); }
        }
    } while (next_perm(order, M));
    if (!have) { *cost = OR_INF; identity(k, perm); return OR_UNREACHABLE; }
    *cost = (int32_t)best;
    for (int32_t i = 0; i < k; ++i) perm[i] = best_seq[i];
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Whole path                                                          */
/* ------------------------------------------------------------------ */

static int32_t find_row(int32_t n_rows, const int32_t* src_nodes, int32_t node) {
    int32_t lo = 0, hi = n_rows - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (src_nodes[mid] == node) return mid;
        if (src_nodes[mid] < node) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

typedef struct {
    int32_t V, depot, n_rows; const int32_t* src_nodes; const int32_t* rows;
    int32_t n_orders; const int64_t* offs; const int32_t* picks; int tour_kind;
    int32_t* cost; int32_t* perm; int32_t* status; int tid, nthr; int rc;
} tour_job;

static void* tour_worker(void* p) {
    tour_job* j = (tour_job*)p;
    int32_t D[(OR_MAX_K_HK + 1) * (OR_MAX_K_HK + 1)];
    int32_t pts[OR_MAX_K_HK + 1];
    const int kind = j->tour_kind & ~OR_OPEN_PATH;
    const int open_path = (j->tour_kind & OR_OPEN_PATH) != 0;
    const int32_t kmax = kind == OR_TOUR_HELDKARP ? OR_MAX_K_HK : OR_MAX_K;
    j->rc = 0;
    for (int32_t o = j->tid; o < j->n_orders; o += j->nthr) {
        int64_t b = j->offs[o], e = j->offs[o + 1];
        int64_t k64 = e - b;
        int32_t* perm = j->perm + b;
        if (k64 < 1 || k64 > kmax) {
            j->cost[o] = OR_INF; j->status[o] = OR_BADORDER;
            for (int64_t i = 0; i < k64; ++i) perm[i] = (int32_t)i;
            continue;
        }
        int32_t k = (int32_t)k64, bad = 0;
        pts[0] = j->depot;
        for (int32_t i = 0; i < k; ++i) {
            pts[i + 1] = j->picks[b + i];
            if (pts[i + 1] < 0 || pts[i + 1] >= j->V) bad = 1;
        }
        if (bad) { j->cost[o] = OR_INF; j->status[o] = OR_BADORDER; identity(k, perm); continue; }
        int32_t n = k + 1;
        for (int32_t a = 0; a < n; ++a) {
            int32_t r = find_row(j->n_rows, j->src_nodes, pts[a]);
            if (r < 0) { j->rc = -3; return 0; }
            for (int32_t c = 0; c < n; ++c)
                D[a * n + c] = j->rows[(size_t)r * (size_t)j->V + (size_t)pts[c]];
        }
        if (open_path)
            for (int32_t a = 0; a < n; ++a) D[a * n] = D[a] = 0;
        int st = (kind == OR_TOUR_HELDKARP) ? or_tour_held_karp(k, D, &j->cost[o], perm)
                                            : or_tour_brute(k, D, &j->cost[o], perm);
        if (st < 0) { j->rc = st; return 0; }
        j->status[o] = st;
    }
    return 0;
}

int or_route_with_rows(int32_t V, int32_t depot, int32_t n_rows, const int32_t* src_nodes,
                       const int32_t* rows, int32_t n_orders, const int64_t* offs,
                       const int32_t* picks, int tour_kind, int n_threads,
                       int32_t* cost, int32_t* perm, int32_t* status) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    tour_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < n_threads; ++t) {
        tour_job j = {V, depot, n_rows, src_nodes, rows, n_orders, offs, picks, tour_kind,
                      cost, perm, status, t, n_threads, 0};
        jobs[t] = j;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], 0, tour_worker, &jobs[t]);
    tour_worker(&jobs[0]);
    int rc = jobs[0].rc;
    for (int t = 1; t < n_threads; ++t) { pthread_join(th[t], 0); if (jobs[t].rc) rc = jobs[t].rc; }
    return rc;
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int or_route_orders(int32_t V, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                    int32_t depot, int32_t n_orders, const int64_t* offs, const int32_t* picks,
                    int sssp_kind, int tour_kind, int n_threads,
                    int32_t* cost, int32_t* perm, int32_t* status) {
    if (V <= 0 || depot < 0 || depot >= V || n_orders < 0) return -1;
    int grc = or_graph_check(V, row_ptr, col, w);
    if (grc) return grc;
    int64_t np = offs[n_orders];
    int32_t* nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np + 1));
    if (!nodes) return -2;
    int32_t cnt = 0;
    nodes[cnt++] = depot;
    for (int32_t o = 0; o < n_orders; ++o) {
        int64_t k = offs[o + 1] - offs[o];
        if (k < 1 || k > OR_MAX_K_HK) continue;
        int bad = 0;
        for (int64_t i = offs[o]; i < offs[o + 1]; ++i) if (picks[i] < 0 || picks[i] >= V) bad = 1;
        if (bad) continue;
        for (int64_t i = offs[o]; i < offs[o + 1]; ++i) nodes[cnt++] = picks[i];
    }
    qsort(nodes, (size_t)cnt, sizeof(int32_t), cmp_i32);
    int32_t u = 0;
    for (int32_t i = 0; i < cnt; ++i) if (i == 0 || nodes[i] != nodes[i - 1]) nodes[u++] = nodes[i];
    int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)u * (size_t)V);
    if (!rows) { free(nodes); return -2; }
    int rc = or_sssp_rows(V, row_ptr, col, w, u, nodes, sssp_kind, n_threads, rows);
    if (rc == 0)
        rc = or_route_with_rows(V, depot, u, nodes, rows, n_orders, offs, picks, tour_kind, n_threads,
                                cost, perm, status);
    free(rows); free(nodes);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Counting                                                            */
/* ------------------------------------------------------------------ */

int64_t or_factorial(int32_t n) {
    int64_t f = 1;
    for (int32_t i = 2; i <= n; ++i) f *= i;
    return f;
}

/* Theorem of Sec. 3: m! 2^(m-1) orderings of m cluster routes with their
 * boundary-node choices, plus (n_1! + ... + n_m!)/2 undirected routes
 * inside the clusters. */
int64_t or_patched_route_count(int32_t m, const int32_t* n_j) {
    int64_t s = 0;
    for (int32_t j = 0; j < m; ++j) s += or_factorial(n_j[j]);
    return or_factorial(m) * ((int64_t)1 << (m - 1)) + s / 2;
}
