"""The sharded path's host logic on CPU with the gloo backend (world size 2): every rank
routes its contiguous slice of the orders and the gathered results equal the whole
batch routed at once; every rank produces its slice of the scale sources' submatrix rows
and one all-gather gives the whole submatrix.  The oracle stands in for the per-rank
router here (no GPU); on GPUs the library routes each slice."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_even_slice_covers_once():
    from paper_2504_20655_gb300.shard import even_slice
    for n in (0, 1, 5, 1024, 1027):
        for world in (1, 2, 3, 8):
            parts = [even_slice(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    from paper_2504_20655_gb300 import shard, synth
    dist.init_process_group("gloo")
    # orders: each rank routes its slice, the results come together in batch order
    g, o = synth.medium_workload(n_orders=37)
    sub, lo, hi = shard.shard_orders(o, world, rank)
    c, p, s = oracle.route_orders(g, sub, "dijkstra", "heldkarp")
    cost, perm, status = shard.gather_order_results(torch.from_numpy(c), torch.from_numpy(p), torch.from_numpy(s),
                                                    world, rank)
    # scale-style rows: each rank its slice of the sources, one all-gather of the submatrix rows
    lay = synth.Layout(A=6, S=8, F=2, C=2, step_lo=5, step_hi=9, cross_w=30)
    gs = lay.build()
    src = synth.distinct_sources(21, gs.n_slots, 5)
    a, b = shard.even_slice(len(src), world, rank)
    rows = oracle.sssp_rows(gs, src[a:b], "dijkstra")
    subm = shard.all_gather_rows(torch.from_numpy(np.ascontiguousarray(rows[:, src])), world)
    out[rank] = (cost.numpy(), perm.numpy(), status.numpy(), subm.numpy(), (lo, hi))
    dist.destroy_process_group()


def test_two_ranks_gather_equals_whole_batch(orc):
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    got = dict(out)
    from paper_2504_20655_gb300 import synth
    g, o = synth.medium_workload(n_orders=37)
    c, p, s = orc.route_orders(g, o, "dijkstra", "heldkarp")
    lay = synth.Layout(A=6, S=8, F=2, C=2, step_lo=5, step_hi=9, cross_w=30)
    gs = lay.build()
    src = synth.distinct_sources(21, gs.n_slots, 5)
    full = orc.sssp_rows(gs, src, "dijkstra")[:, src]
    assert got[0][4] == (0, 19) and got[1][4] == (19, 37)
    for r in (0, 1):
        cost, perm, status, subm, _ = got[r]
        assert (cost == c).all() and (perm == p).all() and (status == s).all()
        assert (subm == full).all()
