"""Counts printed in the paper (tests/golden/paper_counts.json)."""
import json
import math
import os

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


def test_permutation_capacity(orc):
    g = GOLD["permutation_capacity"]
    assert orc.factorial(g["n"]) * (g["n"] - 1) == g["value"]
    g = GOLD["full_combinatorial_after_reorganisation"]
    assert orc.factorial(g["n"]) == g["value"]
    g = GOLD["factorial_12"]
    assert orc.factorial(g["n"]) == g["value"] < 2**31


def test_theorem_counts(orc):
    for c in GOLD["theorem_n12"]["cases"]:
        assert orc.patched_route_count(c["n_j"]) == c["value"]
    g = GOLD["theorem_n15"]
    assert orc.patched_route_count(g["n_j"]) == g["value"]


def test_bf_instance_arithmetic():
    from bench import paper_mteps
    g = GOLD["bf_instance"]
    assert math.ceil(g["E"] / g["threads_per_block"]) == g["blocks"]
    assert (g["V"] - 1) * g["E"] == g["relaxations"]
    # the paper's MTEPS convention: (V-1) * E per source over the run time
    mteps = paper_mteps(g["V"], g["E"], 1, g["ms_approx"] / 1e3)
    assert abs(mteps - g["mteps"]) / g["mteps"] < 0.01
