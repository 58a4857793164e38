"""Pins of the oracle's cluster-patched approximate route (Sec. 3), CPU only.

With as many clusters as stops every stop is its own cluster and the patching
tries every order of the stops, so the result must be the exact optimum (cost
and first optimal sequence) of brute force, for closed tours and open paths;
with one cluster the open route is the exact open path.  Three well separated
groups of stops are found as the three clusters, the route never beats the
exact optimum, and the counts of the theorem are pinned in test_golden_counts.
"""
import numpy as np
import pytest

from paper_2504_20655_gb300 import synth
from tests.test_oracle_tour import rand_D


def _xy(k, seed):
    return synth.uniform_int(seed, 2 * k, 0, 60).reshape(k, 2).astype(np.int32)


@pytest.mark.parametrize("k", [1, 2, 4, 6, 7])
@pytest.mark.parametrize("open_path", [False, True])
def test_one_stop_per_cluster_is_exact(orc, k, open_path):
    for seed in range(4):
        D = rand_D(k, 300 + 10 * k + seed, lo=1, hi=40)
        xy = _xy(k, 70 + seed)
        xy[:, 0] += 100 * np.arange(k)  # distinct positions: k non-empty clusters
        Dx = D.copy()
        if open_path:
            Dx[0, :] = 0
            Dx[:, 0] = 0
        st, c, p = orc.tour_clustered(D, xy, k, open_path)
        st2, c2, p2 = orc.tour(Dx, "brute")
        assert (st, c, p.tolist()) == (st2, c2, p2.tolist())


@pytest.mark.parametrize("k", [3, 6, 8])
def test_one_cluster_open_route_is_exact(orc, k):
    D = rand_D(k, 900 + k, lo=1, hi=40)
    Dx = D.copy()
    Dx[0, :] = 0
    Dx[:, 0] = 0
    st, c, p = orc.tour_clustered(D, _xy(k, 5), 1, True)
    st2, c2, p2 = orc.tour(Dx, "brute")
    assert (st, c, p.tolist()) == (st2, c2, p2.tolist())


def test_separated_groups_and_bounds(orc):
    """Three far-apart groups of stops on a line: the clusters are the groups, each is
    routed in position order, and the patched route equals the exact one here."""
    pos = [1, 2, 3, 50, 51, 52, 53, 100, 101]
    k = len(pos)
    x = np.array([0] + pos)
    D = np.abs(x[:, None] - x[None, :]).astype(np.int32)
    xy = np.stack([np.array(pos), np.zeros(k, int)], axis=1).astype(np.int32)
    st, c, p = orc.tour_clustered(D, xy, 3, False)
    assert st == 0 and c == 2 * 101 and p.tolist() == list(range(k))
    for seed in range(6):  # never below the exact optimum
        D = rand_D(9, 40 + seed, lo=1, hi=50)
        xy = _xy(9, seed)
        st, c, _ = orc.tour_clustered(D, xy, 3, False)
        _, c_exact, _ = orc.tour(D, "brute")
        assert st == 0 and c >= c_exact


def test_cluster_limit(orc):
    D = rand_D(12, 5, lo=1, hi=9)
    xy = np.zeros((12, 2), np.int32)  # every stop on one spot: a single cluster of 12
    st, _, _ = orc.tour_clustered(D, xy, 3, False)
    assert st == 2


def test_pairs_patch_to_the_best_contiguous_sequence(orc):
    """Clusters of two stops: the cluster route and its reverse are the only two inner
    orders, so the patched route must be the best of all k! sequences that keep every
    cluster together (first such sequence on ties), for tours and open paths."""
    import itertools
    k = 6
    xy = np.array([[0, 0], [1, 0], [200, 0], [201, 0], [400, 0], [401, 0]], np.int32)
    cl = [0, 0, 1, 1, 2, 2]
    for seed in range(8):
        D = rand_D(k, 4000 + seed, lo=1, hi=30)
        for open_path in (False, True):
            best = None
            for p in itertools.permutations(range(k)):
                groups = [cl[i] for i in p]
                if any(groups.index(g) + groups.count(g) - 1 != len(groups) - 1 - groups[::-1].index(g)
                       for g in set(groups)):
                    continue  # a cluster split apart
                seq = list(p)
                legs = list(zip(seq[:-1], seq[1:]))
                c = sum(int(D[a + 1, b + 1]) for a, b in legs)
                if not open_path:
                    c += int(D[0, seq[0] + 1]) + int(D[seq[-1] + 1, 0])
                if best is None or c < best[0]:
                    best = (c, seq)
            st, c, pm = orc.tour_clustered(D, xy, 3, open_path)
            assert st == 0 and (c, pm.tolist()) == best, (seed, open_path)
