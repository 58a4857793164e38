"""Pins of the oracle's node-level routes (CPU only).

The leg rule (walk back from t taking the smallest predecessor id on a shortest
path) is checked against a brute-force enumeration of every shortest path on
small graphs (the rule must return the one whose reversed node sequence is
lexicographically smallest), and whole routes against the tour costs: every
step is an arc, the route visits the picks in the given order, and its length
is the tour cost.
"""
import numpy as np
import pytest

from paper_2504_20655_gb300 import synth
from tests.graphs import random_graph


def _arcs(g):
    src = np.repeat(np.arange(g.V), np.diff(g.row_ptr))
    best = {}
    for u, v, w in zip(src.tolist(), np.asarray(g.col).tolist(), np.asarray(g.w).tolist()):
        if u != v and ((u, v) not in best or w < best[(u, v)]):
            best[(u, v)] = w
    return best


def all_shortest_paths(g, d, s, t, arcs):
    """Every shortest s -> t path as a node list (positive weights: the tight arcs form a DAG)."""
    into = {}
    for (u, v), w in arcs.items():
        if d[u] < 2**31 - 1 and d[u] + w == d[v]:
            into.setdefault(v, []).append(u)
    out = []

    def back(v, acc):
        if v == s:
            out.append([s] + acc[::-1])
            return
        for u in into.get(v, []):
            back(u, acc + [v])
    back(t, [])
    return out


@pytest.mark.parametrize("seed", range(6))
def test_leg_rule_against_all_shortest_paths(orc, seed):
    g = random_graph(14, 40, 900 + seed, w_lo=1, w_hi=3)  # small weights: many ties
    arcs = _arcs(g)
    rows = orc.sssp_rows(g, np.arange(g.V, dtype=np.int32), "dijkstra")
    for s in range(g.V):
        for t in range(g.V):
            if s == t or rows[s, t] == 2**31 - 1:
                continue
            paths = all_shortest_paths(g, rows[s], s, t, arcs)
            want = min(paths, key=lambda p: p[::-1])
            # an open path through the picks (s, t) in this order is exactly the leg s -> t
            o = synth.Orders(np.array([0, 2], np.int64), np.array([s, t], np.int32))
            node_offs, nodes = orc.route_nodes(g, o, np.array([0, 1], np.int32), open_path=True)
            assert nodes.tolist() == want


def test_routes_walk_arcs_and_cost_the_tour(orc):
    g, o = synth.medium_workload(n_orders=60)
    arcs = _arcs(g)
    cost, perm, status = orc.route_orders(g, o, "dijkstra", "brute", 4)
    for open_path in (False, True):
        if open_path:
            cost, perm, status = orc.route_orders(g, o, "dijkstra", "brute", 4, open_path=True)
        node_offs, nodes = orc.route_nodes(g, o, perm, open_path=open_path)
        for i in range(o.n):
            r = nodes[node_offs[i]:node_offs[i + 1]].tolist()
            assert status[i] == 0 and len(r) > 0
            assert sum(arcs[(a, b)] for a, b in zip(r[:-1], r[1:])) == cost[i]
            picks_in_order = [int(o.order(i)[j]) for j in perm[o.offs[i]:o.offs[i + 1]]]
            it = iter(r)
            assert all(any(x == p for x in it) for p in picks_in_order)  # the picks, in this order
            if not open_path:
                assert r[0] == g.depot and r[-1] == g.depot


def test_invalid_sequences_get_no_nodes(orc):
    g, o = synth.medium_workload(n_orders=3)
    _, perm, _ = orc.route_orders(g, o, "dijkstra", "brute", 2)
    bad = perm.copy()
    bad[o.offs[1]] = bad[o.offs[1] + 1]  # not a permutation
    node_offs, _ = orc.route_nodes(g, o, bad)
    assert node_offs[2] == node_offs[1] and node_offs[1] > 0 and node_offs[3] > node_offs[2]
