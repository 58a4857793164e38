"""Pins of the oracle's shortest-path distances (CPU only).

Round-based Bellman-Ford (Sec. 4.7) is checked against things other than
itself: Dijkstra and Floyd-Warshall (independent algorithms, the Remark of
Sec. 4.7 validates BF by Dijkstra), SciPy's csgraph Dijkstra (a library
routine), closed-form distances on a uniform rectangular layout, the
round count on a path graph, and the fixpoint certificate.
"""
import numpy as np
import pytest

from paper_2504_20655_gb300 import synth
from tests.graphs import path_graph, random_graph

INF = 2**31 - 1


@pytest.mark.parametrize("seed", range(6))
def test_bf_equals_dijkstra_fifo_random(orc, seed):
    V = [5, 17, 40, 64, 120, 200][seed]
    g = random_graph(V, 3 * V, seed)
    for s in range(0, V, max(1, V // 7)):
        d, _ = orc.bf_rounds(g, s)
        assert (d == orc.dijkstra(g, s)).all()
        assert (d == orc.bf_fifo(g, s)).all()


@pytest.mark.parametrize("seed", range(3))
def test_bf_equals_floyd_warshall(orc, seed):
    g = random_graph(60 + 40 * seed, 250, seed + 100)
    fw = orc.floyd_warshall(g)
    for s in range(g.V):
        d, _ = orc.bf_rounds(g, s)
        assert (d == fw[s]).all()


def test_bf_equals_floyd_warshall_tiny_layout(orc):
    g = synth.tiny_layout().build()
    assert g.V <= 500
    fw = orc.floyd_warshall(g)
    rows = orc.sssp_rows(g, np.arange(g.V), "rounds", n_threads=4)
    assert (rows == fw).all()


def test_bf_equals_scipy_dijkstra(orc):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    for seed in range(3):
        g = random_graph(150, 600, seed + 7, w_lo=1, w_hi=90, allow_multi=False, allow_loops=False)
        m = sp.csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr), shape=(g.V, g.V))
        ref = csg.dijkstra(m, directed=True)
        for s in range(0, g.V, 13):
            d, _ = orc.bf_rounds(g, s)
            exp = np.where(np.isinf(ref[s]), INF, ref[s]).astype(np.int64)
            assert (d.astype(np.int64) == exp).all()


def test_scipy_on_medium_layout(orc):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    g = synth.medium_layout().build()
    m = sp.csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr), shape=(g.V, g.V))
    src = np.array([0, 777, 5050, 19999, g.depot], dtype=np.int32)
    ref = csg.dijkstra(m, directed=True, indices=src)
    rows = orc.sssp_rows(g, src, "fifo")
    assert (rows.astype(np.int64) == ref.astype(np.int64)).all()
    d, rounds = orc.bf_rounds(g, int(src[1]))
    assert (d == rows[1]).all() and 0 < rounds < g.V - 1


def test_closed_form_uniform_layout(orc):
    """F = 1, C = 2, every chain edge a, cross links c: between slots of
    different aisles the distance is min((s1+1)+(s2+1), (S-s1)+(S-s2))*a
    + |a1-a2|*c, within one aisle |s1-s2|*a (a detour through a third
    aisle costs at least (S+1)*a more)."""
    A, S, a, c, dw = 7, 9, 13, 41, 300
    lay = synth.Layout(A=A, S=S, F=1, C=2, step_lo=a, step_hi=a, cross_w=c, depot_w=dw)
    g = lay.build()
    slots = np.arange(lay.n_slots)
    rows = orc.sssp_rows(g, slots, "rounds")
    for p in slots:
        a1, s1 = divmod(int(p), S)
        for q in slots:
            a2, s2 = divmod(int(q), S)
            if a1 == a2:
                exp = abs(s1 - s2) * a
            else:
                exp = min((s1 + 1) + (s2 + 1), (S - s1) + (S - s2)) * a + abs(a1 - a2) * c
            assert rows[p, q] == exp
    d, _ = orc.bf_rounds(g, g.depot)
    for p in slots:
        a1, s1 = divmod(int(p), S)
        assert d[p] == dw + a1 * c + (s1 + 1) * a


def test_rounds_on_path(orc):
    for n in (2, 3, 10, 57):
        g = path_graph(n, w=3)
        d, rounds = orc.bf_rounds(g, 0)
        assert rounds == n - 1
        assert (d == 3 * np.arange(n)).all()
        d, rounds = orc.bf_rounds(g, n - 1)
        assert rounds == 0 and (d[:-1] == INF).all() and d[-1] == 0


def test_fixpoint_certificate_and_invariants(orc):
    g = synth.medium_layout().build()
    u, v, w = g.arcs()
    src = synth.distinct_sources(12, g.n_slots, 5)
    rows = orc.sssp_rows(g, src, "dijkstra", n_threads=4).astype(np.int64)
    for i, s in enumerate(src):
        d = rows[i]
        assert d[s] == 0
        fin = d[u] < INF
        # d[v] <= d[u] + w(u, v) on every arc
        assert (d[v[fin]] <= d[u[fin]] + w[fin]).all()
        # every finite d[v], v != s, is attained by some in-arc (weights > 0)
        best = np.full(g.V, np.iinfo(np.int64).max)
        np.minimum.at(best, v[fin], d[u[fin]] + w[fin])
        mask = (d < INF) & (np.arange(g.V) != s)
        assert (best[mask] == d[mask]).all()
    # triangle inequality on the pick submatrix
    sub = rows[:, src]
    for m in range(len(src)):
        assert (sub <= sub[:, m:m + 1] + sub[m:m + 1, :]).all()


def test_symmetry_undirected_layout(orc):
    g = synth.tiny_layout().build()
    fw = orc.floyd_warshall(g)
    assert (fw == fw.T).all()


def test_one_way_aisles_are_asymmetric(orc):
    g = synth.medium_layout().build()
    src = synth.distinct_sources(40, g.n_slots, 9)
    rows = orc.sssp_rows(g, src, "dijkstra", n_threads=4)
    sub = rows[:, src]
    assert (sub != sub.T).any()


def _graph(V, arcs):
    u, v, w = (np.array(x, np.int64) for x in zip(*arcs))
    rp, col, wt = synth.csr_from_arcs(V, u, v, w)
    return synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0, n_slots=V)


def _all_sssp(orc, g, s):
    return [orc.bf_rounds(g, s)[0], orc.bf_fifo(g, s), orc.dijkstra(g, s), orc.floyd_warshall(g)[s]]


def test_int32_rule_refuses_and_accepts(orc):
    """Distances are int32 with INF = 2^31 - 1 for unreachable.  A graph is accepted when
    min((V-1) max w, sum w) < INF; every shortest path is simple, so that bounds every
    finite distance.  Hand-worked cases for both sides of each term of the bound, and no
    shortest-path routine ever returns a distance at or above INF."""
    # two arcs of 1.5e9 in a row: the bound (3e9) and the true distance reach INF
    g = _graph(3, [(0, 1, 1_500_000_000), (1, 2, 1_500_000_000)])
    assert not orc.graph_check(g)
    for f in (lambda: orc.bf_rounds(g, 0), lambda: orc.bf_fifo(g, 0), lambda: orc.dijkstra(g, 0),
              lambda: orc.floyd_warshall(g)):
        with pytest.raises(orc.DistanceRangeError):
            f()
    with pytest.raises(orc.DistanceRangeError):
        orc.route_orders(g, synth.Orders(np.array([0, 1], np.int64), np.array([2], np.int32)))
    # one heavy arc: (V-1) max w = 4e9 but sum w = 2e9 + 5 < INF, so accepted; exact values
    g = _graph(3, [(0, 1, 2_000_000_000), (1, 2, 5)])
    assert orc.graph_check(g)
    for d in _all_sssp(orc, g, 0):
        assert d.tolist() == [0, 2_000_000_000, 2_000_000_005]
    # a complete graph of 4 nodes, every arc 5e8: sum w = 6e9 but (V-1) max w = 1.5e9 < INF
    g = _graph(4, [(a, b, 500_000_000) for a in range(4) for b in range(4) if a != b])
    assert orc.graph_check(g)
    for d in _all_sssp(orc, g, 2):
        assert d.tolist() == [500_000_000, 500_000_000, 0, 500_000_000]
    # the edge of the rule: one arc of INF - 1 is a finite distance; one arc of INF is not
    g = _graph(2, [(0, 1, INF - 1)])
    assert orc.graph_check(g)
    for d in _all_sssp(orc, g, 0):
        assert d.tolist() == [0, INF - 1]
    g = _graph(2, [(0, 1, INF)])
    assert not orc.graph_check(g)
    with pytest.raises(orc.DistanceRangeError):
        orc.dijkstra(g, 0)


@pytest.mark.parametrize("seed", range(4))
def test_int32_rule_is_sound(orc, seed):
    """On random small graphs with weights up to 2^31 - 1: whenever the rule accepts a
    graph, every source's distances come back (none reaches INF); whenever a distance
    reaches INF, the rule has refused the graph."""
    for t in range(40):
        V = 2 + (t % 6)
        n = 1 + (7 * t + seed) % (2 * V)
        hi = [INF, 1 << 30, 700_000_000, 300_000_000][(t + seed) % 4]
        g = random_graph(V, n, 4000 + 97 * seed + t, w_lo=0, w_hi=hi)
        ok = orc.graph_check(g)
        for s in range(V):
            try:
                orc.dijkstra(g, s)
            except orc.DistanceRangeError:
                assert not ok
