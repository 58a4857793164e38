"""Small graph builders shared by the tests (inputs only, no routing arithmetic)."""
import numpy as np

from paper_2504_20655_gb300 import synth


def random_graph(V, n_arcs, seed, w_lo=0, w_hi=50, allow_multi=True, allow_loops=True):
    u = synth.uniform_int(seed ^ 11, n_arcs, 0, V - 1)
    v = synth.uniform_int(seed ^ 12, n_arcs, 0, V - 1)
    w = synth.uniform_int(seed ^ 13, n_arcs, w_lo, w_hi)
    keep = np.ones(n_arcs, dtype=bool)
    if not allow_loops:
        keep &= u != v
    u, v, w = u[keep], v[keep], w[keep]
    if not allow_multi:
        key = u * V + v
        _, first = np.unique(key, return_index=True)
        u, v, w = u[first], v[first], w[first]
    rp, col, wt = synth.csr_from_arcs(V, u, v, w)
    return synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0, n_slots=V)


def path_graph(n, w=1):
    u = np.arange(n - 1)
    v = np.arange(1, n)
    rp, col, wt = synth.csr_from_arcs(n, u, v, np.full(n - 1, w))
    return synth.Graph(V=n, row_ptr=rp, col=col, w=wt, depot=0, n_slots=n)
