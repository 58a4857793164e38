"""The benchmark's multi-rank host logic on CPU with the gloo backend (world size 2):
rank setup from the environment, the barrier, the max over ranks of the step time,
replica throughput, and the reference arm's rule that only rank 0 works."""
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    args = types.SimpleNamespace(impl="ours", backend="gloo")
    w, r, local = bench.dist_setup(args)
    bench.barrier(w)
    ms = bench.max_over_ranks(10.0 + 5.0 * r, w)  # the slower rank decides
    ref_args = types.SimpleNamespace(impl="reference", workload="tiny", warmup=0, steps=1, ref_budget=1.0)
    rc = bench.run_reference(ref_args) if r != 0 else 0  # ranks other than 0 exit without work
    out[r] = (w, r, local, ms, bench.replica_value(100, ms, w), rc)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    got = dict(out)
    assert sorted(got) == [0, 1]
    for r in (0, 1):
        w, rank, local, ms, value, rc = got[r]
        assert (w, rank, local) == (2, r, r)
        assert ms == 15.0                      # max over ranks, same on both
        assert value == pytest.approx(2 * 100 / 0.015)  # units of both replicas / slowest time
        assert rc == 0
