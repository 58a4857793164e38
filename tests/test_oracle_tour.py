"""Pins of the oracle's tour search (CPU only).

Brute force over all k! sequences in lexicographic order (Sec. 4.6) is
checked against: hand-worked cases (tests/golden/tours_by_hand.json),
Held-Karp with lexicographic reconstruction (Sec. 3 reference point),
an independent itertools enumeration written here, the reversal symmetry
of undirected instances, and the status rules.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2504_20655_gb300 import synth

INF = 2**31 - 1
GOLD = os.path.join(os.path.dirname(__file__), "golden", "tours_by_hand.json")


def py_tour(D):
    """Independent enumeration: itertools yields permutations in lexicographic order."""
    k = D.shape[0] - 1
    best, arg = None, None
    for p in itertools.permutations(range(1, k + 1)):
        seq = (0,) + p + (0,)
        legs = [int(D[a, b]) for a, b in zip(seq[:-1], seq[1:])]
        if any(x == INF for x in legs):
            continue
        c = sum(legs)
        if best is None or c < best:
            best, arg = c, [x - 1 for x in p]
    return best, arg


def rand_D(k, seed, lo=0, hi=30, p_inf=0.0, sym=False):
    n = k + 1
    D = synth.uniform_int(seed, n * n, lo, hi).reshape(n, n)
    if p_inf > 0:
        D = np.where(synth.uniform01(seed ^ 99, n * n).reshape(n, n) < p_inf, INF, D)
    if sym:
        D = np.minimum(D, D.T)
    np.fill_diagonal(D, 0)
    return D.astype(np.int32)


def rank_of(perm):
    """Lexicographic rank of a permutation of 0..k-1 (factorial number system)."""
    k = len(perm)
    rest = sorted(perm)
    r = 0
    for i, x in enumerate(perm):
        j = rest.index(x)
        r = r * (k - i) + j
        rest.pop(j)
    return r


@pytest.mark.parametrize("case", json.load(open(GOLD))["cases"], ids=lambda c: c["name"])
def test_hand_worked(orc, case):
    D = np.array(case["D"], dtype=np.int32)
    for kind in ("brute", "heldkarp"):
        st, cost, perm = orc.tour(D, kind)
        assert st == case["status"] and cost == case["cost"] and perm.tolist() == case["perm"], kind


@pytest.mark.parametrize("k", range(1, 8))
def test_brute_equals_itertools(orc, k):
    for seed in range(5):
        for p_inf, hi in ((0.0, 3), (0.0, 1000), (0.3, 50)):
            D = rand_D(k, seed * 31 + k, hi=hi, p_inf=p_inf)
            st, cost, perm = orc.tour(D, "brute")
            best, arg = py_tour(D)
            if best is None:
                assert st == 1 and cost == INF and perm.tolist() == list(range(k))
            else:
                assert st == 0 and cost == best and perm.tolist() == arg


@pytest.mark.parametrize("k", range(1, 11))
def test_brute_equals_held_karp(orc, k):
    n_cases = 12 if k <= 8 else 3
    for seed in range(n_cases):
        hi = (2, 9, 500)[seed % 3]
        D = rand_D(k, seed * 7 + 1000 * k, hi=hi, p_inf=0.1 if seed % 4 == 0 else 0.0)
        assert orc.tour(D, "brute")[:2] == orc.tour(D, "heldkarp")[:2]
        b, h = orc.tour(D, "brute"), orc.tour(D, "heldkarp")
        assert (b[2] == h[2]).all()


def test_reversal_symmetry(orc):
    for k in range(2, 8):
        D = rand_D(k, 4242 + k, hi=20, sym=True)
        st, cost, perm = orc.tour(D, "brute")
        rev = perm[::-1]
        Dl = D.astype(np.int64)
        seq = [0] + [p + 1 for p in rev] + [0]
        assert sum(Dl[a, b] for a, b in zip(seq[:-1], seq[1:])) == cost
        assert rank_of(perm.tolist()) <= rank_of(rev.tolist())


def test_duplicate_picks_give_zero_legs(orc):
    x = np.array([0, 4, 4, 10, 4])
    D = np.abs(np.subtract.outer(x, x)).astype(np.int32)
    st, cost, perm = orc.tour(D, "brute")
    assert st == 0 and cost == 20
    assert py_tour(D) == (cost, perm.tolist())


def test_range_and_bad_orders(orc):
    D = rand_D(4, 5, hi=50)
    D[1, 2] = 10324441
    st, cost, perm = orc.tour(D, "brute")
    assert st == 3 and cost == INF and perm.tolist() == [0, 1, 2, 3]
    D[1, 2] = 10324440
    assert orc.tour(D, "brute")[0] == 0
    assert orc.tour(np.zeros((14, 14), dtype=np.int32), "brute")[0] == 2  # k = 13 > 12


def test_route_orders_statuses(orc):
    g = synth.tiny_layout().build()
    offs = np.array([0, 2, 2, 4, 17, 19], dtype=np.int64)
    picks = np.array([1, 2, 3, g.V, *range(13), 5, 5], dtype=np.int32)
    o = synth.Orders(offs, picks)
    cost, perm, status = orc.route_orders(g, o)
    assert status.tolist() == [0, 2, 2, 2, 0]
    assert cost[1] == INF and cost[2] == INF and cost[3] == INF
    assert perm[2:4].tolist() == [0, 1]
    assert perm[4:17].tolist() == list(range(13))
    assert cost[4] == 2 * orc.dijkstra(g, g.depot)[5]


# --- Held-Karp above the brute-force limit (k = 13 .. 20) -------------------------------

def line_lex_tour(pos):
    """Points on a line (depot at 0, pick j at pos[j] > 0, all distinct): a closed tour
    costs 2 * max(pos) exactly when its positions rise to the maximum and then fall, so
    the first optimal sequence in lexicographic order is found greedily, taking the
    smallest pick that still allows such a rise-and-fall completion."""
    k = len(pos)
    rest = set(range(k))
    cur, up, seq = 0, True, []
    while rest:
        for j in sorted(rest):
            others = rest - {j}
            if up and pos[j] > cur:
                ok = True  # keep rising: whatever is left below comes on the way down
            else:          # fall: everything left must lie below j
                ok = pos[j] < cur and all(pos[q] < pos[j] for q in others)
            if ok:
                if pos[j] < cur:
                    up = False
                seq.append(j)
                cur = pos[j]
                rest.remove(j)
                break
        else:
            raise AssertionError("no feasible step")
    return 2 * max(pos), seq


def line_D(pos):
    x = np.array([0] + list(pos), dtype=np.int64)
    return np.abs(x[:, None] - x[None, :]).astype(np.int32)


@pytest.mark.parametrize("k", [6, 9, 13, 16, 20])
def test_held_karp_points_on_a_line(orc, k):
    """Held-Karp against the closed form and the greedy rule of the line, beyond brute force."""
    rng = np.random.default_rng(1000 + k)
    pos = list(rng.choice(np.arange(1, 500), size=k, replace=False) * 3)
    cost, seq = line_lex_tour(pos)
    st, c, p = orc.tour(line_D(pos), "heldkarp")
    assert st == 0 and c == cost and p.tolist() == seq
    if k <= 9:  # the greedy rule itself against brute force
        st, c, p = orc.tour(line_D(pos), "brute")
        assert c == cost and p.tolist() == seq


@pytest.mark.parametrize("k", [13, 17, 20])
def test_held_karp_large_k_consistency(orc, k):
    """Random asymmetric instances: the returned sequence costs exactly the returned
    optimum, no random or shifted sequence beats it, and equal legs give the identity."""
    D = rand_D(k, 500 + k, lo=1, hi=1000)
    st, c, p = orc.tour(D, "heldkarp")
    seq = [0] + [x + 1 for x in p.tolist()] + [0]
    assert st == 0 and sorted(p.tolist()) == list(range(k))
    assert c == sum(int(D[a, b]) for a, b in zip(seq[:-1], seq[1:]))
    rng = np.random.default_rng(k)
    for _ in range(300):
        q = [0] + list(rng.permutation(k) + 1) + [0]
        assert c <= sum(int(D[a, b]) for a, b in zip(q[:-1], q[1:]))
    flat = np.full((k + 1, k + 1), 7, np.int32)
    np.fill_diagonal(flat, 0)
    st, c, p = orc.tour(flat, "heldkarp")
    assert st == 0 and c == 7 * (k + 1) and p.tolist() == list(range(k))


def test_held_karp_limits(orc):
    st, _, _ = orc.tour(rand_D(21, 3), "heldkarp")
    assert st == 2  # above the Held-Karp limit: bad order
    st, _, _ = orc.tour(rand_D(13, 3), "brute")
    assert st == 2  # above the brute-force limit


# --- open paths: the entrance/exit is not part of the route (Sec. 3) ---------------------

@pytest.mark.parametrize("k", [2, 5, 8, 14, 20])
def test_open_path_on_a_line(orc, k):
    """Open paths through points on a line cost the span exactly when they are monotone,
    so the first optimal sequence is the lexicographically smaller of the ascending and
    the descending order.  Brute force (k <= 8) and Held-Karp against that rule; the
    route functions' open mode gives the same as a matrix with free depot legs."""
    rng = np.random.default_rng(77 + k)
    pos = rng.choice(np.arange(1, 900), size=k, replace=False)
    up = list(np.argsort(pos, kind="stable"))
    want = min(up, up[::-1])
    span = int(pos.max() - pos.min())
    D = line_D(list(pos))
    D[0, :] = 0
    D[:, 0] = 0
    kinds = ["brute", "heldkarp"] if k <= 8 else ["heldkarp"]
    for kind in kinds:
        st, c, p = orc.tour(D, kind)
        assert st == 0 and c == span and p.tolist() == [int(x) for x in want], kind


def test_open_path_route_mode(orc):
    """The route functions' open mode equals closed tours over matrices whose depot legs
    are free, for brute force and Held-Karp, on a directed layout (one-way aisles)."""
    g, o = synth.medium_workload(n_orders=40)
    c1, p1, s1 = orc.route_orders(g, o, "dijkstra", "brute", 4, open_path=True)
    c2, p2, s2 = orc.route_orders(g, o, "dijkstra", "heldkarp", 4, open_path=True)
    assert (c1 == c2).all() and (p1 == p2).all() and (s1 == s2).all()
    cc, _, _ = orc.route_orders(g, o, "dijkstra", "brute", 4)
    assert (c1 <= cc).all() and (c1 < cc).any()  # dropping the depot legs never costs more
    rows = orc.sssp_rows(g, np.unique(np.concatenate([[g.depot], o.picks])).astype(np.int32), "dijkstra", 4)
    nodes = np.unique(np.concatenate([[g.depot], o.picks]))
    for i in range(0, o.n, 7):
        pts = np.concatenate([[g.depot], o.order(i)])
        idx = np.searchsorted(nodes, pts)
        D = rows[idx][:, pts].astype(np.int64)
        D[0, :] = 0
        D[:, 0] = 0
        st, c, p = orc.tour(D.astype(np.int32), "brute")
        assert c == c1[i] and p.tolist() == p1[o.offs[i]:o.offs[i + 1]].tolist()
