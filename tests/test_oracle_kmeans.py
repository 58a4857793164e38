"""Pins of the oracle's k-means step (the clustering of Sec. 3's cluster-patched route), CPU only.

Hand-worked cases (tests/golden/kmeans_by_hand.json) fix the initialisation, the tie
rules and the stopping rule, including cases where Lloyd steps move a centre and change
assignments twice.  On random stops the result must be a fixed point of the Lloyd map,
checked here with exact rational arithmetic: every non-empty centre is the mean of its
stops, every stop sits with its nearest centre (ties to the lowest index), and the number
of centres is min(m, number of distinct stop positions).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2504_20655_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kmeans_by_hand.json")))


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_kmeans_by_hand(case):
    a, sx, sy, cnt, steps = oracle.kmeans(np.array(case["xy"]), case["m"])
    assert a.tolist() == case["assign"]
    assert (sx.tolist(), sy.tolist(), cnt.tolist()) == (case["Sx"], case["Sy"], case["cnt"])
    assert steps == case["steps"]


def _fixed_point(xy, m, a, sx, sy, cnt):
    k = len(xy)
    nc = len(cnt)
    if nc != min(m, len({tuple(p) for p in xy.tolist()})):
        return False
    for c in range(nc):
        members = [i for i in range(k) if a[i] == c]
        if members:
            if cnt[c] != len(members) or sx[c] != sum(int(xy[i, 0]) for i in members) \
                    or sy[c] != sum(int(xy[i, 1]) for i in members):
                return False
    means = [(Fraction(int(sx[c]), int(cnt[c])), Fraction(int(sy[c]), int(cnt[c]))) for c in range(nc)]
    for i in range(k):
        d = [(xy[i, 0] - mx) ** 2 + (xy[i, 1] - my) ** 2 for mx, my in means]
        if a[i] != d.index(min(d)):
            return False
    return True


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
def test_kmeans_fixed_point(m):
    for seed in range(60):
        k = 1 + seed % 12
        xy = synth.uniform_int(900 + 31 * m + seed, 2 * k, 0, 9 if seed % 3 else 40).reshape(k, 2).astype(np.int64)
        a, sx, sy, cnt, steps = oracle.kmeans(xy, m)
        assert steps < 64
        assert _fixed_point(xy, m, a, sx, sy, cnt), (m, seed, xy.tolist(), a.tolist())


def test_kmeans_initial_centres_are_farthest_first():
    """With one Lloyd pass that changes nothing (stops on the centres themselves) the
    centres are the initial ones: stop 0, then the farthest, then the farthest from both."""
    xy = np.array([[0, 0], [0, 0], [10, 0], [10, 0], [4, 3], [4, 3]])
    a, sx, sy, cnt, steps = oracle.kmeans(xy, 3)
    # stop 2 (distance 100) is the second centre; stop 4 (min(25, 45) = 25) the third
    assert a.tolist() == [0, 0, 1, 1, 2, 2] and cnt.tolist() == [2, 2, 2] and steps == 2
