"""Warp-exact CPU model of the sweep kernel's fast path (tests/model/bf_warp_model.cpp).

The model replays the kernel's lanes, 4-source quads, shuffle scans and
32-bit wrap-around, with adversarial stale shared memory before every tile.
It must reach the oracle's distances; and with the kernel's INF fill of the
unstaged tile slots removed (a planted omission), it must not.
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


@pytest.fixture(scope="module")
def wm(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("bwm") / "libbwm.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2504_20655_gb300", "csrc"), "-I", "/usr/local/cuda/include",
                           os.path.join(HERE, "model", "bf_warp_model.cpp"),
                           os.path.join(ROOT, "paper_2504_20655_gb300", "csrc", "wr_graph.cpp"), "-o", so])
    return ctypes.CDLL(so)


def rows(wm, g, src, run_target=200, stale=1, inf_fill=1):
    P = ctypes.c_void_p
    rp, c, w = (np.ascontiguousarray(g.row_ptr, np.int64), np.ascontiguousarray(g.col, np.int32),
                np.ascontiguousarray(g.w, np.int32))
    src = np.ascontiguousarray(src, np.int32)
    out = np.empty((len(src), g.V), np.int32)
    sw = np.zeros(1, np.int32)
    rc = wm.bwm_rows(g.V, ctypes.c_longlong(g.E), rp.ctypes.data_as(P), c.ctypes.data_as(P), w.ctypes.data_as(P),
                     len(src), src.ctypes.data_as(P), run_target, stale, inf_fill, out.ctypes.data_as(P),
                     sw.ctypes.data_as(P))
    assert rc == 0, rc
    return out, int(sw[0])


def test_medium_orders_with_stale_shared_memory(wm, orc):
    g, o = synth.medium_workload(n_orders=64)
    src = np.unique(np.concatenate([[g.depot], o.picks])).astype(np.int32)
    out, sweeps = rows(wm, g, src)
    assert (out == orc.sssp_rows(g, src, "dijkstra", 4)).all()
    assert sweeps <= 12


@pytest.mark.parametrize("seed", range(4))
def test_random_graphs(wm, orc, seed):
    V = [40, 257, 600, 1500][seed]
    g = random_graph(V, 3 * V, seed + 900, w_lo=0, w_hi=1000, allow_multi=False)
    src = np.arange(0, V, max(1, V // 40), dtype=np.int32)
    for rt in (200, 64, 1):
        out, _ = rows(wm, g, src, run_target=rt)
        assert (out == orc.sssp_rows(g, src, "dijkstra", 4)).all(), rt


def test_planted_missing_inf_fill_is_caught(wm, orc):
    g, o = synth.medium_workload(n_orders=64)
    src = np.unique(np.concatenate([[g.depot], o.picks])).astype(np.int32)
    out, _ = rows(wm, g, src, inf_fill=0)
    assert (out < orc.sssp_rows(g, src, "dijkstra", 4)).any()
