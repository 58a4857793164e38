"""CPU oracle -- test infrastructure only.

ctypes binding of oracle.c (plain C, built with gcc).  Only the tests,
the smoke check and the benchmark's CPU-baseline leg may import this
package; the routing library never does.  It shares no code with the
CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")

INF = 2**31 - 1
MAX_K = 12
MAX_K_HK = 20
LEG_MAX = 10324440
OK, UNREACHABLE, BADORDER, RANGE = 0, 1, 2, 3
EDIST = -4  # a finite distance would reach INF
SSSP = {"rounds": 0, "fifo": 1, "dijkstra": 2}
TOUR = {"brute": 0, "heldkarp": 1}
OPEN_PATH = 16

_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "oracle.c")
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, src,
                               "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


def _configure(L):
    P = ctypes.c_void_p
    i32, i64, I = ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    L.or_bf_rounds.argtypes = [i32, P, P, P, i32, P, P]
    L.or_bf_fifo.argtypes = [i32, P, P, P, i32, P]
    L.or_dijkstra.argtypes = [i32, P, P, P, i32, P]
    L.or_floyd_warshall.argtypes = [i32, P, P, P, P]
    L.or_sssp_rows.argtypes = [i32, P, P, P, i32, P, I, I, P]
    L.or_tour_brute.argtypes = [i32, P, P, P]
    L.or_tour_held_karp.argtypes = [i32, P, P, P]
    L.or_route_orders.argtypes = [i32, P, P, P, i32, i32, P, P, I, I, I, P, P, P]
    L.or_route_with_rows.argtypes = [i32, i32, i32, P, P, i32, P, P, I, I, P, P, P]
    L.or_factorial.argtypes = [i32]
    L.or_factorial.restype = i64
    L.or_tour_clustered.argtypes = [i32, P, P, i32, I, P, P]
    L.or_patched_route_count.argtypes = [i32, P]
    L.or_graph_check.argtypes = [i32, P, P, P]
    L.or_kmeans.argtypes = [i32, P, i32, P, P, P, P, P]
    L.or_patched_route_count.restype = i64
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(LIB))
    return _lib


class using:
    """Context manager that points this module at another build of oracle.c
    (the mutation tests compile deliberately broken copies)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    return (np.ascontiguousarray(g.row_ptr, dtype=np.int64), np.ascontiguousarray(g.col, dtype=np.int32),
            np.ascontiguousarray(g.w, dtype=np.int32))


class DistanceRangeError(RuntimeError):
    """A finite distance would reach INF (2^31 - 1): the graph breaks the int32 rule."""


def _check(rc, what):
    if rc == EDIST:
        raise DistanceRangeError(f"oracle {what}: a finite distance would reach INF")
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with {rc}")


def graph_check(g) -> bool:
    """True when every finite distance of g must stay below INF, by the bound
    min((V-1) * max w, sum of w) over the arcs as given."""
    rp, c, w = _csr(g)
    rc = lib().or_graph_check(g.V, _p(rp), _p(c), _p(w))
    if rc not in (0, EDIST):
        raise RuntimeError(f"oracle graph_check failed with {rc}")
    return rc == 0


def bf_rounds(g, src: int):
    rp, c, w = _csr(g)
    d = np.empty(g.V, dtype=np.int32)
    r = np.zeros(1, dtype=np.int32)
    _check(lib().or_bf_rounds(g.V, _p(rp), _p(c), _p(w), int(src), _p(d), _p(r)), "bf_rounds")
    return d, int(r[0])


def bf_fifo(g, src: int):
    rp, c, w = _csr(g)
    d = np.empty(g.V, dtype=np.int32)
    _check(lib().or_bf_fifo(g.V, _p(rp), _p(c), _p(w), int(src), _p(d)), "bf_fifo")
    return d


def dijkstra(g, src: int):
    rp, c, w = _csr(g)
    d = np.empty(g.V, dtype=np.int32)
    _check(lib().or_dijkstra(g.V, _p(rp), _p(c), _p(w), int(src), _p(d)), "dijkstra")
    return d


def floyd_warshall(g):
    rp, c, w = _csr(g)
    d = np.empty((g.V, g.V), dtype=np.int32)
    _check(lib().or_floyd_warshall(g.V, _p(rp), _p(c), _p(w), _p(d)), "floyd_warshall")
    return d


def sssp_rows(g, src, kind: str = "dijkstra", n_threads: int = 1):
    rp, c, w = _csr(g)
    src = np.ascontiguousarray(src, dtype=np.int32)
    rows = np.empty((src.shape[0], g.V), dtype=np.int32)
    _check(lib().or_sssp_rows(g.V, _p(rp), _p(c), _p(w), src.shape[0], _p(src), SSSP[kind],
                              int(n_threads), _p(rows)), "sssp_rows")
    return rows


def tour(D, kind: str = "brute"):
    """(status, cost, perm) of the best closed tour over the (k+1)x(k+1) matrix D."""
    D = np.ascontiguousarray(D, dtype=np.int32)
    k = D.shape[0] - 1
    cost = np.zeros(1, dtype=np.int32)
    perm = np.zeros(max(k, 1), dtype=np.int32)
    f = lib().or_tour_brute if kind == "brute" else lib().or_tour_held_karp
    st = f(k, _p(D), _p(cost), _p(perm))
    if st < 0:
        raise RuntimeError(f"oracle tour failed with {st}")
    return int(st), int(cost[0]), perm[:k].copy()


def route_orders(g, orders, sssp: str = "dijkstra", tour_kind: str = "brute", n_threads: int = 1, max_k=None,
                 open_path: bool = False):
    """(cost, perm, status) per order.  Orders above max_k (default: the solver's own
    limit, 12 for brute force and 20 for Held-Karp) are OR_BADORDER, as in a library
    context created with that max_k."""
    rp, c, w = _csr(g)
    offs = np.ascontiguousarray(orders.offs, dtype=np.int64)
    picks = np.ascontiguousarray(orders.picks, dtype=np.int32)
    n = offs.shape[0] - 1
    cost = np.zeros(n, dtype=np.int32)
    perm = np.zeros(max(int(offs[-1]), 1), dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    _check(lib().or_route_orders(g.V, _p(rp), _p(c), _p(w), int(g.depot), n, _p(offs), _p(picks),
                                 SSSP[sssp], TOUR[tour_kind] | (OPEN_PATH if open_path else 0), int(n_threads),
                                 _p(cost), _p(perm), _p(status)), "route_orders")
    if max_k is not None:
        for o in np.nonzero(np.diff(offs) > max_k)[0]:
            cost[o], status[o] = INF, BADORDER
            perm[offs[o]:offs[o + 1]] = np.arange(offs[o + 1] - offs[o])
    return cost, perm[:int(offs[-1])], status


def route_with_rows(V, depot, src_nodes, rows, orders, tour_kind: str = "brute", n_threads: int = 1):
    src_nodes = np.ascontiguousarray(src_nodes, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    offs = np.ascontiguousarray(orders.offs, dtype=np.int64)
    picks = np.ascontiguousarray(orders.picks, dtype=np.int32)
    n = offs.shape[0] - 1
    cost = np.zeros(n, dtype=np.int32)
    perm = np.zeros(max(int(offs[-1]), 1), dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    _check(lib().or_route_with_rows(int(V), int(depot), src_nodes.shape[0], _p(src_nodes), _p(rows), n,
                                    _p(offs), _p(picks), TOUR[tour_kind], int(n_threads), _p(cost),
                                    _p(perm), _p(status)), "route_with_rows")
    return cost, perm[:int(offs[-1])], status


def factorial(n: int) -> int:
    return int(lib().or_factorial(int(n)))


def patched_route_count(n_j) -> int:
    a = np.ascontiguousarray(n_j, dtype=np.int32)
    return int(lib().or_patched_route_count(a.shape[0], _p(a)))


def route_nodes(g, orders, perm, open_path: bool = False, n_threads: int = 1):
    """Node-level routes (plain Python over the oracle's Dijkstra rows): for each order and
    its pick sequence, the depot and then each leg's nodes after its first (open path: the
    first pick, then the legs between picks).  Leg s -> t is walked back from t, taking as
    the predecessor of v the smallest node id u with an arc u -> v and
    dist(s,u) + w(u,v) = dist(s,v).  An order with an unreachable leg, an invalid sequence
    or a bad order gets no nodes.  Returns (node_offs, nodes)."""
    offs = np.asarray(orders.offs, dtype=np.int64)
    picks = np.asarray(orders.picks, dtype=np.int64)
    V = g.V
    # in-arcs with node ids, the lightest arc per (u, v), no self loops
    src = np.repeat(np.arange(V), np.diff(g.row_ptr))
    best = {}
    for u, v, w in zip(src.tolist(), np.asarray(g.col).tolist(), np.asarray(g.w).tolist()):
        if u != v and ((u, v) not in best or w < best[(u, v)]):
            best[(u, v)] = w
    into = [[] for _ in range(V)]
    for (u, v), w in best.items():
        into[v].append((u, w))
    nodes_needed = np.unique(np.concatenate([[g.depot], picks[(picks >= 0) & (picks < V)]])).astype(np.int32)
    rows = sssp_rows(g, nodes_needed, "dijkstra", n_threads)
    row_of = {int(x): i for i, x in enumerate(nodes_needed)}

    def leg(s, t):
        d = rows[row_of[s]]
        if d[t] == INF:
            return None
        out, v = [], t
        while v != s:
            out.append(v)
            v = min(u for u, w in into[v] if d[u] != INF and int(d[u]) + w == int(d[v]))
        return out[::-1]

    node_offs, nodes = [0], []
    for o in range(len(offs) - 1):
        b, e = int(offs[o]), int(offs[o + 1])
        k = e - b
        seq = [int(x) for x in perm[b:e]]
        route = []
        ok = 1 <= k <= MAX_K_HK and all(0 <= p < V for p in picks[b:e]) and sorted(seq) == list(range(k))
        if ok:
            pts = [int(picks[b + j]) for j in seq]
            stops = pts if open_path else [g.depot] + pts + [g.depot]
            route = [stops[0]]
            for s, t in zip(stops[:-1], stops[1:]):
                part = leg(s, t)
                if part is None:
                    route = []
                    break
                route += part
        nodes += route
        node_offs.append(len(nodes))
    return np.array(node_offs, np.int64), np.array(nodes, np.int32)


def tour_clustered(D, xy, m: int, open_path: bool = False):
    """(status, cost, perm) of the cluster-patched route (Sec. 3) over D, with the k stops'
    plan coordinates xy (k x 2) and at most m clusters."""
    D = np.ascontiguousarray(D, dtype=np.int32)
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    k = D.shape[0] - 1
    cost = np.zeros(1, dtype=np.int32)
    perm = np.zeros(max(k, 1), dtype=np.int32)
    st = lib().or_tour_clustered(k, _p(D), _p(xy), int(m), int(bool(open_path)), _p(cost), _p(perm))
    if st < 0:
        raise RuntimeError(f"oracle clustered tour failed with {st}")
    return int(st), int(cost[0]), perm[:k].copy()


def kmeans(xy, m: int):
    """The k-means step of the cluster-patched route (Sec. 3) on the k stops' plan
    coordinates xy (k x 2), at most m clusters.  Returns (assign, Sx, Sy, cnt, steps):
    stop i's cluster assign[i], centre c's coordinate sums Sx[c], Sy[c] over its cnt[c]
    stops (the mean is Sx/cnt, Sy/cnt), and the number of assignment passes run."""
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    k = xy.shape[0]
    assign = np.zeros(max(k, 1), np.int32)
    sx, sy, cnt = (np.zeros(max(k, 1), np.int64) for _ in range(3))
    steps = np.zeros(1, np.int32)
    nc = lib().or_kmeans(k, _p(xy), int(m), _p(assign), _p(sx), _p(sy), _p(cnt), _p(steps))
    if nc < 0:
        raise RuntimeError(f"oracle kmeans failed with {nc}")
    return assign[:k].copy(), sx[:nc].copy(), sy[:nc].copy(), cnt[:nc].copy(), int(steps[0])


def route_orders_clustered(g, orders, xy, m: int, open_path: bool = False, n_threads: int = 1):
    """The cluster-patched route of every order (rows by the oracle's Dijkstra); xy is the
    (V, 2) plan coordinate array of the graph's nodes.  Orders above MAX_K picks or with a
    node out of range are BADORDER."""
    offs = np.asarray(orders.offs, dtype=np.int64)
    picks = np.asarray(orders.picks, dtype=np.int64)
    n = len(offs) - 1
    cost = np.full(n, INF, np.int32)
    status = np.full(n, BADORDER, np.int32)
    perm = np.zeros(max(int(offs[-1]), 1), np.int32)
    ok_nodes = picks[(picks >= 0) & (picks < g.V)]
    nodes = np.unique(np.concatenate([[g.depot], ok_nodes])).astype(np.int32)
    rows = sssp_rows(g, nodes, "dijkstra", n_threads)
    for o in range(n):
        b, e = int(offs[o]), int(offs[o + 1])
        k = e - b
        perm[b:e] = np.arange(k)
        pts = picks[b:e]
        if k < 1 or k > MAX_K or (pts < 0).any() or (pts >= g.V).any():
            continue
        allp = np.concatenate([[g.depot], pts])
        idx = np.searchsorted(nodes, allp)
        D = rows[idx][:, allp]
        st, c, p = tour_clustered(D, np.asarray(xy)[pts], m, open_path)
        status[o], cost[o] = st, c
        perm[b:e] = p
    return cost, perm[:int(offs[-1])], status
