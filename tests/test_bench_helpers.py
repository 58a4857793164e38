"""Host-side helpers of bench.py: the operation counts its roofline objects divide by,
checked against explicit enumeration, and the oracle's baseline runners in every mode
on a small batch (no GPU)."""
import itertools
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

from paper_2504_20655_gb300 import synth  # noqa: E402


@pytest.mark.parametrize("k", range(2, 10))
def test_hk_transitions_by_enumeration(k):
    """Every (visited set S, last pick c in S, next pick j outside S), plus k first legs
    from the depot and k legs back."""
    n = 0
    for size in range(1, k):
        for S in itertools.combinations(range(k), size):
            n += len(S) * (k - len(S))
    assert bench.hk_transitions(k) == n + 2 * k


@pytest.mark.parametrize("k", range(1, 9))
def test_enum_ops_by_enumeration(k):
    """Prefix-sharing count: one add per node of the prefix tree below the depot, then a
    return leg and a compare per full sequence."""
    nodes = sum(len(list(itertools.permutations(range(k), l))) for l in range(1, k + 1))
    assert bench.enum_ops(k) == nodes + 2 * math.factorial(k)


@pytest.mark.parametrize("mode", ["exact", "heldkarp", "open", "clustered", "nodes"])
def test_oracle_runners_all_modes(mode):
    g, o = synth.medium_workload(n_orders=6)
    if mode == "heldkarp":
        g, o = synth.large_order_workload(n_orders=2, k_lo=13, k_hi=13)
    run = bench.oracle_runner(g, o, mode, 2)
    out = run(o.subset(np.arange(2)))
    assert out is not None


@pytest.mark.parametrize("k", range(2, 12))
def test_hk_table_bytes_by_levels(k):
    """Each level L writes C(k, L) subsets x L last picks and reads, once, the C(k, L+1)
    x (L+1) words of the level above: summed over the levels, k 2^(k-1) words each way."""
    words = sum(math.comb(k, L) * L for L in range(1, k + 1))
    assert bench.hk_table_bytes(k) == 2 * 4 * words
