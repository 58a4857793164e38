"""Host logic of the Bellman-Ford path, on the CPU.

tests/model/bf_model.cpp runs the library's graph preprocessing
(wr_graph.cpp) and replays the sweep kernel's tile passes and frontier
rules sequentially.  The tests check the partition's invariants and that
the replayed sweeps reach the oracle's distances for several tilings.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2504_20655_gb300 import synth
from tests.graphs import random_graph

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def model(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("bfm") / "libbfm.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2504_20655_gb300", "csrc"), "-I", CUDA_INC,
                           os.path.join(HERE, "model", "bf_model.cpp"),
                           os.path.join(ROOT, "paper_2504_20655_gb300", "csrc", "wr_graph.cpp"), "-o", so])
    lib = ctypes.CDLL(so)
    lib.bfm_fast_fraction.restype = ctypes.c_double
    return lib


def _arrs(g):
    return (np.ascontiguousarray(g.row_ptr, np.int64), np.ascontiguousarray(g.col, np.int32),
            np.ascontiguousarray(g.w, np.int32))


def model_rows(model, g, src, run_target, tile_cap):
    P = ctypes.c_void_p
    rp, c, w = _arrs(g)
    src = np.ascontiguousarray(src, np.int32)
    out = np.empty((len(src), g.V), np.int32)
    sw = np.zeros(1, np.int32)
    rc = model.bfm_rows(g.V, ctypes.c_longlong(g.E), rp.ctypes.data_as(P), c.ctypes.data_as(P), w.ctypes.data_as(P),
                        len(src), src.ctypes.data_as(P), run_target, tile_cap, out.ctypes.data_as(P),
                        sw.ctypes.data_as(P))
    assert rc == 0, rc
    return out, int(sw[0])


def check_partition(model, g, run_target, tile_cap):
    P = ctypes.c_void_p
    rp, c, w = _arrs(g)
    nr = np.zeros(1, np.int32)
    rc = model.bfm_check_partition(g.V, ctypes.c_longlong(g.E), rp.ctypes.data_as(P), c.ctypes.data_as(P),
                                   w.ctypes.data_as(P), run_target, tile_cap, nr.ctypes.data_as(P))
    return rc, int(nr[0])


def fast_path_fraction(model, g, run_target, tile_cap):
    P = ctypes.c_void_p
    rp, c, w = _arrs(g)
    return float(model.bfm_fast_fraction(g.V, ctypes.c_longlong(g.E), rp.ctypes.data_as(P), c.ctypes.data_as(P),
                                         w.ctypes.data_as(P), run_target, tile_cap))


TILINGS = [(96, 128), (32, 128), (200, 256), (1, 128), (128, 128), (400, 512)]


@pytest.mark.parametrize("rt,tc", TILINGS)
def test_partition_invariants(model, rt, tc):
    graphs = [random_graph(V, 3 * V, V + 5, w_lo=0, w_hi=100) for V in (1, 5, 100, 700)]
    graphs += [synth.tiny_layout().build(), synth.medium_layout().build()]
    for g in graphs:
        rc, n_runs = check_partition(model, g, rt, tc)
        assert rc == 0, (g.V, rc)
        assert n_runs >= (g.V + 2 * rt - 1) // (2 * rt)  # a run holds at most two segments
    # the layouts run entirely on the fast path
    for g in graphs[-2:]:
        assert fast_path_fraction(model, g, rt, tc) == 1.0


@pytest.mark.parametrize("seed", range(8))
def test_model_sweeps_random(model, orc, seed):
    V = [1, 2, 7, 33, 100, 257, 600, 1500][seed]
    g = random_graph(V, max(1, 3 * V), seed + 300, w_lo=0, w_hi=20 if seed % 2 else 1000)
    src = np.arange(0, V, max(1, V // 70), dtype=np.int32)
    ref = orc.sssp_rows(g, src, "dijkstra", 4)
    for rt, tc in TILINGS:
        out, sweeps = model_rows(model, g, src, rt, tc)
        assert (out == ref).all(), (rt, tc)
        assert sweeps <= V + 1


def test_model_sweeps_medium_layout(model, orc):
    g = synth.medium_layout().build()
    src = synth.distinct_sources(64, g.n_slots, 17)
    ref = orc.sssp_rows(g, src, "dijkstra", 4)
    for rt, tc in ((96, 128), (200, 256)):
        out, sweeps = model_rows(model, g, src, rt, tc)
        assert (out == ref).all()
        # far fewer sweeps than the hop diameter a Jacobi round count needs
        _, rounds = orc.bf_rounds(g, int(src[0]))
        assert sweeps < rounds


def test_high_in_degree_spills_to_global(model, orc):
    V = 700
    u = np.concatenate([np.arange(1, V), np.zeros(V - 1, np.int64)])
    v = np.concatenate([np.zeros(V - 1, np.int64), np.arange(1, V)])
    w = synth.uniform_int(77, u.shape[0], 1, 50)
    rp, col, wt = synth.csr_from_arcs(V, u, v, w)
    g = synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0)
    src = np.array([0, 5, 699, 350], np.int32)
    out, _ = model_rows(model, g, src, 96, 128)
    assert (out == orc.sssp_rows(g, src)).all()


def test_faces_share_tiles(model):
    """On a two-level aisle layout the two faces of an aisle stretch pair up: most runs
    hold two segments and the halo per own node drops well below the one-to-one of
    unpaired face chains."""
    g = synth.Layout(A=20, S=100, F=2, C=2, step_lo=50, step_hi=150, face_w=400).build()
    P = ctypes.c_void_p
    rp, c, w = _arrs(g)
    out = np.zeros(3, np.float64)
    model.bfm_pair_stats(g.V, ctypes.c_longlong(g.E), rp.ctypes.data_as(P), c.ctypes.data_as(P), w.ctypes.data_as(P),
                         60, 128, out.ctypes.data_as(P))
    paired, halo_per_node, compact = out
    assert paired > 0.8 and halo_per_node < 0.25 and compact == 1.0


def model_rows_worklist(model, g, src, run_target, tile_cap, order=0, seed_fed=1):
    P = ctypes.c_void_p
    rp, c, w = _arrs(g)
    src = np.ascontiguousarray(src, np.int32)
    out = np.empty((len(src), g.V), np.int32)
    visits = np.zeros(1, np.int64)
    rc = model.bfm_rows_worklist(g.V, ctypes.c_longlong(g.E), rp.ctypes.data_as(P), c.ctypes.data_as(P),
                                 w.ctypes.data_as(P), len(src), src.ctypes.data_as(P), run_target, tile_cap,
                                 ctypes.c_ulonglong(order), seed_fed, out.ctypes.data_as(P), visits.ctypes.data_as(P))
    assert rc == 0, rc
    return out, int(visits[0])


@pytest.mark.parametrize("seed", range(8))
def test_worklist_random_graphs_any_order(model, orc, seed):
    """The asynchronous worklist's rules -- seeds are each source's run and the runs it
    feeds, a visit that drops a row requests itself and the runs it feeds -- reach the
    oracle's rows whatever order the waiting visits are taken in."""
    V = [1, 2, 7, 33, 100, 257, 600, 1500][seed]
    g = random_graph(V, max(1, 3 * V), seed + 300, w_lo=0, w_hi=20 if seed % 2 else 1000)
    src = np.arange(0, V, max(1, V // 70), dtype=np.int32)
    ref = orc.sssp_rows(g, src, "dijkstra", 4)
    for rt, tc in TILINGS:
        for order in (0, 0x9E3779B97F4A7C15 + seed, 12345 + seed):
            out, _ = model_rows_worklist(model, g, src, rt, tc, order)
            assert (out == ref).all(), (rt, tc, order)


def test_worklist_medium_layout(model, orc):
    g = synth.medium_layout().build()
    src = synth.distinct_sources(64, g.n_slots, 17)
    ref = orc.sssp_rows(g, src, "dijkstra", 4)
    for order in (0, 7):
        out, visits = model_rows_worklist(model, g, src, 60, 128, order)
        assert (out == ref).all()
        assert visits > 0


def test_worklist_needs_the_fed_runs_in_its_seeds(model, orc):
    """Planted omission: with one node per run a source's own visit changes nothing, so
    without the runs it feeds among the seeds no distance beyond the sources is found."""
    g = random_graph(100, 300, 301, w_lo=1, w_hi=20)
    src = np.arange(0, 100, 7, dtype=np.int32)
    ref = orc.sssp_rows(g, src, "dijkstra", 4)
    out, _ = model_rows_worklist(model, g, src, 1, 128, 0, seed_fed=0)
    assert not (out == ref).all()
    out, _ = model_rows_worklist(model, g, src, 1, 128, 0, seed_fed=1)
    assert (out == ref).all()


def model_rows_warp(model, g, src, run_target, tile_cap):
    P = ctypes.c_void_p
    rp, c, w = _arrs(g)
    src = np.ascontiguousarray(src, np.int32)
    out = np.empty((len(src), g.V), np.int32)
    sw = np.zeros(1, np.int32)
    share = np.zeros(1, np.float64)
    rc = model.bfm_rows_warp(g.V, ctypes.c_longlong(g.E), rp.ctypes.data_as(P), c.ctypes.data_as(P),
                             w.ctypes.data_as(P), len(src), src.ctypes.data_as(P), run_target, tile_cap,
                             out.ctypes.data_as(P), sw.ctypes.data_as(P), share.ctypes.data_as(P))
    assert rc == 0, rc
    return out, int(sw[0]), float(share[0])


WARP_TILINGS = [(60, 128), (96, 128), (32, 128), (1, 128), (120, 256), (200, 256)]


@pytest.mark.parametrize("seed", range(8))
def test_warp_model_random_graphs(model, orc, seed):
    """The warp tiling replayed lane by lane (compact descriptors, extras folded before
    each pass, blocks of 4 nodes loaded before the previous block's carry chain, the
    generic path for runs that do not stage every source) reaches the oracle's rows."""
    V = [1, 2, 7, 33, 100, 257, 600, 1500][seed]
    g = random_graph(V, max(1, 3 * V), seed + 300, w_lo=0, w_hi=20 if seed % 2 else 1000)
    src = np.arange(0, V, max(1, V // 70), dtype=np.int32)
    ref = orc.sssp_rows(g, src, "dijkstra", 4)
    for rt, tc in WARP_TILINGS:
        out, sweeps, _ = model_rows_warp(model, g, src, rt, tc)
        assert (out == ref).all(), (rt, tc)
        assert sweeps <= V + 1


def test_warp_model_layouts_all_compact(model, orc):
    """On the aisle layouts every run takes the compact path: the cross-aisle nodes'
    aisle arcs beyond two per pass are the runs' extras.  Rows equal the oracle's."""
    for lay, n in ((synth.medium_layout(), 64), (synth.Layout(A=20, S=100, F=2, C=2, step_lo=50, step_hi=150,
                                                              face_w=400), 40)):
        g = lay.build()
        src = synth.distinct_sources(n, g.n_slots, 5)
        ref = orc.sssp_rows(g, src, "dijkstra", 4)
        for rt, tc in ((60, 128), (120, 256)):
            out, _, share = model_rows_warp(model, g, src, rt, tc)
            assert (out == ref).all(), (rt, tc)
            assert share == 1.0


def test_warp_model_high_in_degree(model, orc):
    """A hub with 699 in-arcs: its run overflows the tile and takes the generic path."""
    V = 700
    u = np.concatenate([np.arange(1, V), np.zeros(V - 1, np.int64)])
    v = np.concatenate([np.zeros(V - 1, np.int64), np.arange(1, V)])
    w = synth.uniform_int(77, u.shape[0], 1, 50)
    rp, col, wt = synth.csr_from_arcs(V, u, v, w)
    g = synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0)
    src = np.array([0, 5, 699, 350], np.int32)
    out, _, share = model_rows_warp(model, g, src, 96, 128)
    assert (out == orc.sssp_rows(g, src)).all()
    assert share < 1.0
