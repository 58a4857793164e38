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
