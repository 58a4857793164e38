"""Benchmark: exact-routed orders/s of the routing hot path on synthetic workloads.

One step = one call of the whole path (source selection, Bellman-Ford rows,
D gather, exhaustive sequence evaluation, reduction, decode) over one batch
of orders.  Default workload: the medium layout (100 aisles x 100 slots x 2
sides, 4 cross-aisles, 10% one-way aisles; V = 20,401) with 1024 orders of
k ~ U{4..10} Zipf(1.1) picks.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
launching stream, inputs resident in HBM, the L2 flushed (a 512 MiB write)
between steps outside the timed region; barrier + synchronize around the
timed region; max over ranks.  `e2e` repeats the measurement through the C
ABI with pinned host buffers (H2D of the orders and D2H of the results
inside the timed region).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def paper_mteps(V, E, n_src, seconds):
    """Sec. 4.7's throughput convention: (V-1) * E relaxations per source over the run time."""
    return (V - 1) * E * n_src / seconds / 1e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured", "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}


# GB300: 152 SMs.  Integer min and fused add-min instructions issue on the ALU
# pipe, 64 lanes per SM per clock (half the 128 INT32 lanes of the SM); every
# evaluated sequence costs one of them, so the enumeration's roofline counts
# sequences against that rate.
ALU_MIN_LANES_PER_SM = 64
N_SMS = 152


def alu_min_peak(pk):
    """T fused add-min ops/s: 152 SMs x 64 ALU-pipe lanes x the maximum SM clock."""
    return N_SMS * ALU_MIN_LANES_PER_SM * pk["sm_max_mhz"] * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index=0):
        self.proc = None
        self.index = index
        self.path = os.path.join(tempfile.gettempdir(), f"wroute_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()
        return False

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(name, n_orders=1024):
    from paper_2504_20655_gb300 import synth
    if name == "medium":
        g, o = synth.medium_workload(n_orders=n_orders)
        desc = "medium: 100 aisles x 100 slots x 2 sides, 4 cross-aisles, 10% one-way (V=20401); " \
               "1024 orders, k~U{4..10}, Zipf(1.1) over 50k SKUs"
    elif name == "batching":
        g, o = synth.batching_workload()
        desc = "batching: medium layout; 20000 orders, k=2+Geom(0.3) truncated at 12, Zipf(1.1) picks"
    elif name == "tiny":
        g, o = synth.tiny_workload()
        desc = "tiny: 10 aisles x 20 slots x 2 sides (V=421); one order of 6 picks"
    elif name == "heldkarp":
        g, o = synth.large_order_workload()
        desc = "large orders: medium layout (V=20401); 128 orders, k~U{13..20}, Zipf(1.1) over 50k SKUs"
    elif name in ("open", "clustered", "nodes"):
        g, o = synth.medium_workload()
        desc = {"open": "open paths (the entrance/exit not part of the route, Sec. 3): ",
                "clustered": "cluster-patched approximate routes (Sec. 3), at most 3 clusters: ",
                "nodes": "node-level routes of the exact sequences: "}[name] + \
            "medium layout (V=20401); 1024 orders, k~U{4..10}, Zipf(1.1) over 50k SKUs"
    else:
        raise ValueError(name)
    return g, o, desc


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = getattr(args, "backend", None) or ("nccl" if args.impl == "ours" else "gloo")
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


# DRAM traffic per launch of the default sweep kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum), from the captures summarised in profiles/bf_warp_kernel_*.txt.
# A figure holds only while the sources that shape the kernel's traffic are the ones
# it was taken on (hash below) and the tuning is the default one; otherwise null.
TRAFFIC_SOURCES = ["paper_2504_20655_gb300/csrc/wr_bf_warp.cu", "paper_2504_20655_gb300/csrc/wr_bf_common.cuh",
                   "paper_2504_20655_gb300/csrc/wr_graph.cpp"]
TRAFFIC_HASH = "84da2311a179ecb7"
TRAFFIC = {"medium": 724111104 + 453456896, "scale": 18794906000 + 9115479000}


def traffic_for(workload, tuned):
    import hashlib
    h = hashlib.sha1()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if tuned or h.hexdigest()[:16] != TRAFFIC_HASH:
        return None
    return TRAFFIC.get(workload)


def sweep_kernel_name(tuning):
    """The Bellman-Ford kernel a tuning selects (warp tiles, one or two source groups per warp;
    the warp worklist; CTA tiles)."""
    t = tuning["bf_tiling"]
    if t == 0:
        t = 1 if tuning["tile_cap"] <= 256 else 2
    return {1: "bf_warp_kernel", 4: "bf_warp_kernel", 3: "bf_warp_async_kernel"}.get(t, "bf_sweeps_kernel")


def cpu_oracle_rows_rate(g, src, budget_s=15.0, n_threads=None):
    """The oracle's Dijkstra rows on the host's cores for a bounded prefix of the
    sources; returns (E x sources / s, cores, sample)."""
    import oracle
    n_threads = n_threads or os.cpu_count() or 1
    m = n_threads
    while True:
        t0 = time.perf_counter()
        oracle.sssp_rows(g, src[:m], "dijkstra", n_threads)
        t = time.perf_counter() - t0
        if t > budget_s / 3 or m >= len(src):
            break
        m = min(len(src), m * max(2, int(budget_s / 3 / max(t, 1e-3))))
    return g.E * m / t / 1e9, n_threads, f"Dijkstra rows of the first {m} sources ({t:.1f} s on {n_threads} threads)"


def replica_value(units_per_rank, ms, world):
    """Whole-job throughput of `world` replicas that each processed units_per_rank
    units, timed by the slowest rank (ms = max over ranks)."""
    return world * units_per_rank / (ms / 1e3)


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_runner(g, o, mode, n_threads):
    """The oracle's whole path for a prefix of the batch o in the given mode, as it stands
    (node-level routes: the walk alone, over the oracle's own exact sequences)."""
    import oracle
    if mode == "heldkarp":
        return lambda sub: oracle.route_orders(g, sub, "rounds", "heldkarp", n_threads, max_k=20)
    if mode == "open":
        return lambda sub: oracle.route_orders(g, sub, "rounds", "brute", n_threads, open_path=True)
    if mode == "clustered":
        xy = synth_layout_coords()
        return lambda sub: oracle.route_orders_clustered(g, sub, xy, 3, False, n_threads)
    if mode == "nodes":
        _, perm_all, _ = oracle.route_orders(g, o, "dijkstra", "heldkarp", n_threads)  # untimed: the sequences

        def run(sub):
            return oracle.route_nodes(g, sub, perm_all[:int(sub.offs[-1])], False, n_threads)
        return run
    return lambda sub: oracle.route_orders(g, sub, "rounds", "brute", n_threads)


def synth_layout_coords():
    from paper_2504_20655_gb300 import synth
    return synth.medium_layout().coords()


def cpu_oracle_rate(g, o, budget_s=15.0, n_threads=None, mode="exact"):
    """The oracle (round-based Bellman-Ford + brute force over all k!, or the mode's own
    tour step) on the host's cores, on a bounded prefix of the batch; returns
    (orders/s, cores, sample)."""
    n_threads = n_threads or os.cpu_count() or 1
    run = oracle_runner(g, o, mode, n_threads)
    n = 8 if mode != "heldkarp" else 2
    t = 0.0
    while True:
        sub = o.subset(np.arange(min(n, o.n)))
        t0 = time.perf_counter()
        run(sub)
        t = time.perf_counter() - t0
        if t > budget_s / 3 or n >= o.n:
            break
        n = min(o.n, n * max(2, int(budget_s / 3 / max(t, 1e-3))))
    reps = 1
    if n >= o.n and t < budget_s / 3:  # the whole batch is quick: repeat it for a steadier rate
        reps = max(1, int(budget_s / 3 / max(t, 1e-3)))
        t0 = time.perf_counter()
        for _ in range(reps):
            run(sub)
        t = time.perf_counter() - t0
    what = f"first {n} orders of the batch" if reps == 1 else f"the whole batch of {n} orders x {reps}"
    return reps * n / t, n_threads, f"{what} ({t:.1f} s on {n_threads} threads)"


METRIC = {"clustered": "approximate-routed orders/s", "nodes": "node-routed orders/s"}


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    if args.workload == "scale":
        from paper_2504_20655_gb300 import synth
        g, src = synth.scale_workload(n_src=args.scale_sources)
        rates = []
        for i in range(args.warmup + args.steps):
            v, cores, sample = cpu_oracle_rows_rate(g, src, budget_s=args.ref_budget)
            if i >= args.warmup:
                rates.append(v)
        value = statistics.median(rates)
        line = {"impl": "reference", "metric": "BF Gedges/s (E x sources / step time)", "value": value,
                "unit": "Gedges/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * g.E * len(src) / (value * 1e9), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": "scale: rows of the 4096 sources, oracle Dijkstra"},
                "cpu_baseline": {"value": value, "unit": "Gedges/s", "cores": cores, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": "Gedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    g, o, desc = workload("medium" if args.workload == "serving" else args.workload)
    mode = args.workload if args.workload in ("heldkarp", "open", "clustered", "nodes") else "exact"
    rates = []
    for i in range(args.warmup + args.steps):
        r, cores, sample = cpu_oracle_rate(g, o, budget_s=args.ref_budget, mode=mode)
        if i >= args.warmup:
            rates.append(r)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC.get(args.workload, "exact-routed orders/s"), "value": value,
            "unit": "orders/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * o.n / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": "orders/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "orders/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def measure_scale(args):
    """Scale workload: rows of 4096 sources over the 1000 x 500 x 2-level layout
    (V = 1,002,001), produced segment by segment under the memory budget and
    consumed on the device (4096 x 4096 submatrix + per-row checksum).  Returns the
    line (rank 0) or None."""
    import torch

    from paper_2504_20655_gb300 import shard, synth, wroute
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # weak scaling: world x 4096 sources, every rank the rows of its contiguous slice of
    # them (as many as one GPU alone); one all-gather of the submatrix rows per step
    g, src_all = synth.scale_workload(n_src=args.scale_sources * world)
    s_lo, s_hi = shard.even_slice(len(src_all), world, rank)
    src = np.ascontiguousarray(src_all[s_lo:s_hi])
    n, n_all = len(src), len(src_all)
    r = wroute.Router(device=local, mem_budget_bytes=args.budget_gib << 30)
    if args.tune:
        r.set_tuning(**json.loads(args.tune))
    r.load_graph(g)
    stream = torch.cuda.current_stream(dev)
    d_src = torch.from_numpy(src).to(dev)
    d_dst = torch.from_numpy(np.ascontiguousarray(src_all)).to(dev)
    sub = torch.empty((n, n_all), dtype=torch.int32, device=dev)
    check = torch.empty(n, dtype=torch.int64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step():
        wroute.wr_submatrix(r.ctx, d_src, d_dst, sub, check, stream.cuda_stream)
        if world > 1:
            shard.all_gather_rows(sub, world)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    r.sync()
    stats_list = []
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            e0[i].record(stream)
            step()
            e1[i].record(stream)
            stats_list.append(r.stats())
        torch.cuda.synchronize()
    barrier(world)
    r.sync()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / args.steps, world, dev)
    st = stats_list[-1]
    bf_ms = statistics.median(s["ms_bf"] for s in stats_list)
    pk = peaks()
    achieved = st["bytes_alg"] / (bf_ms / 1e3) / 1e9
    gedges = g.E * n * world / (ms / 1e3) / 1e9
    line = {
        "metric": "BF Gedges/s (E x sources / step time)", "value": gedges, "unit": "Gedges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "scale: 1000 aisles x 500 slots x 2 levels, 2 cross-aisles (V=1002001, 3007998 arcs); "
                               f"rows of {n} distinct slot sources consumed as a {n}x{n_all} submatrix + checksums"
                               + (f"; sources split x{world}, one all-gather of the submatrix rows per step"
                                  if world > 1 else ""),
                   "budget_gib": args.budget_gib, "segments": st["n_segments"], "tuning": r.tuning(),
                   "l2": "rows (2 GiB per segment) exceed L2; 512 MiB flush between steps"},
        "roofline": {"kernel": sweep_kernel_name(r.tuning()), "bound": "hbm", "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     "traffic": traffic_for("scale", bool(args.tune)) if n == 4096 else None,
                     "peak_source": pk["source"], "bytes_alg_per_launch": st["bytes_alg"] / st["n_segments"],
                     "ms_per_launch": bf_ms / st["n_segments"], "launches": st["n_segments"],
                     "sweeps": st["sweeps"], "node_visits": st["node_visits"]},
        "phases_ms": {k[3:]: statistics.median(s[k] for s in stats_list) for k in
                      ("ms_init", "ms_bf", "ms_total")},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats_list)),
        "clocks": clk.summary(),
        "paper_convention_mteps": paper_mteps(g.V, g.E, n, ms / 1e3),
    }
    # end to end through the C ABI with host buffers: sources in, submatrix and checksums out
    h_sub = np.empty((n, n_all), np.int32)
    h_check = np.empty(n, np.uint64)
    e2e = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        wroute.wr_submatrix(r.ctx, src, src_all, h_sub, h_check)
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e) / len(e2e), world, dev)
    line["e2e"] = {"value": g.E * n * world / e2e_s / 1e9, "unit": "Gedges/s", "h2d_bytes_per_step": 4 * (n + n_all),
                   "d2h_bytes_per_step": 4 * n * n_all + 8 * n,
                   "matches_device_run": bool((h_sub == sub.cpu().numpy()).all())}
    if rank == 0 and not args.no_cpu:
        v, cores, sample = cpu_oracle_rows_rate(g, src, budget_s=args.ref_budget)
        line["cpu_baseline"] = {"value": v, "unit": "Gedges/s", "cores": cores, "kind": "oracle", "sample": sample}
    r.close()
    return line if rank == 0 else None


def enum_ops(k):
    """Prefix-sharing operation count of exhaustive enumeration for one order of k picks
    (every prefix of length l = 1..k extends a shorter one by one add, every full
    sequence adds its return leg and takes one compare): context only, the kernel
    shares suffix sums too and needs fewer."""
    f = math.factorial(k)
    return sum(f // math.factorial(k - l) for l in range(1, k + 1)) + 2 * f


def measure_batching(args):
    """Batching workload: 20,000 orders of k = 2..12 in one CUDA-graph launch per step
    (the whole path captured once by wr_plan_create), tuned by the library's autotuner on
    another batch of the same distribution (another seed); compared, bit for bit and in
    orders/s, with one plain wr_route_orders call per order.  Returns the line (rank 0)
    or None."""
    import torch

    from paper_2504_20655_gb300 import wroute
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g, o, desc = workload("batching")
    n, np_ = o.n, int(o.offs[-1])
    r = wroute.Router(device=local, mem_budget_bytes=args.budget_gib << 30)
    r.load_graph(g)
    offs_d = torch.from_numpy(o.offs).to(dev)
    picks_d = torch.from_numpy(o.picks).to(dev)
    if args.tune:
        r.set_tuning(**json.loads(args.tune))
        tuned_by = "fixed (--tune)"
        tuning_same_batch = None
    else:
        # tuned on a batch drawn with another seed, then timed on this one; the tuning the
        # timed batch itself would pick is reported beside it
        from paper_2504_20655_gb300 import synth
        _, o_t = synth.batching_workload(seed=synth.SEED_BASE + 1)
        t0 = time.perf_counter()
        r.autotune(torch.from_numpy(o_t.offs).to(dev), torch.from_numpy(o_t.picks).to(dev), reps=1)
        tuned_by = f"wr_autotune on another batch of the workload (seed {synth.SEED_BASE + 1}; " \
                   f"{time.perf_counter() - t0:.1f} s, untimed)"
        chosen = r.tuning()
        tuning_same_batch = r.autotune(offs_d, picks_d, reps=1)
        r.set_tuning(**chosen)
    plan = r.plan(n, np_)
    plan.set_batch(offs_d, picks_d)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        plan.launch(stream.cuda_stream)
    torch.cuda.synchronize()
    plan.sync()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stats_list = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            e0[i].record(stream)
            plan.launch(stream.cuda_stream)
            e1[i].record(stream)
            stats_list.append(plan.stats())  # syncs; outside the event pair
        torch.cuda.synchronize()
    barrier(world)
    plan.sync()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / args.steps, world, dev)
    value = replica_value(n, ms, world)
    g_cost, g_perm, g_status = plan.cost.cpu().numpy(), plan.perm.cpu().numpy(), plan.status.cpu().numpy()

    # the same batch through one direct call, and one plain call per order
    ref = r.route_orders(offs_d, picks_d)
    same_direct = bool((ref[0].cpu().numpy() == g_cost).all() and (ref[1].cpu().numpy()[:np_] == g_perm[:np_]).all()
                       and (ref[2].cpu().numpy() == g_status).all())
    k = o.k()
    offs1 = torch.zeros((n, 2), dtype=torch.int64, device=dev)
    offs1[:, 1] = torch.from_numpy(k).to(dev)
    c1 = torch.empty(n, dtype=torch.int32, device=dev)
    s1 = torch.empty(n, dtype=torch.int32, device=dev)
    p1 = torch.empty(max(np_, 1), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    m, t_plain = 0, 0.0
    t0 = time.perf_counter()
    while m < n and t_plain < args.plain_budget:
        lo, hi = int(o.offs[m]), int(o.offs[m + 1])
        wroute.wr_route_orders(r.ctx, offs1[m], picks_d[lo:hi], c1[m:m + 1], p1[lo:hi], s1[m:m + 1], stream.cuda_stream)
        m += 1
        if m % 64 == 0:
            torch.cuda.synchronize()
            t_plain = time.perf_counter() - t0
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    mp = int(o.offs[m])
    same_plain = bool((c1[:m].cpu().numpy() == g_cost[:m]).all() and (s1[:m].cpu().numpy() == g_status[:m]).all()
                      and (p1[:mp].cpu().numpy() == g_perm[:mp]).all())

    # end to end: pinned host batch in, results out, around every graph launch
    h_offs = torch.from_numpy(o.offs).pin_memory()
    h_picks = torch.from_numpy(o.picks).pin_memory()
    h_cost = torch.empty(n, dtype=torch.int32).pin_memory()
    h_perm = torch.empty(max(np_, 1), dtype=torch.int32).pin_memory()
    h_status = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.offs.copy_(h_offs, non_blocking=True)
        plan.picks[:np_].copy_(h_picks, non_blocking=True)
        plan.launch(stream.cuda_stream)
        h_cost.copy_(plan.cost, non_blocking=True)
        h_perm[:np_].copy_(plan.perm[:np_], non_blocking=True)
        h_status.copy_(plan.status, non_blocking=True)
        stream.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), world, dev)
    e2e_ok = bool((h_cost.numpy() == g_cost).all() and (h_perm.numpy()[:np_] == g_perm[:np_]).all())

    st = stats_list[-1]
    enum_ms = statistics.median(s["ms_enum"] for s in stats_list)
    bf_ms = statistics.median(s["ms_bf"] for s in stats_list)
    ops = float(sum(enum_ops(int(kk)) for kk in k))
    pk = peaks()
    alu_peak = alu_min_peak(pk)
    achieved = st["sequences"] / (enum_ms / 1e3) / 1e12  # one fused add-min per sequence
    line = {
        "metric": "exact-routed orders/s", "value": value, "unit": "orders/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": desc, "orders_per_step": n, "sources": st["n_sources"],
                   "l2": "flushed (512 MiB write) between steps", "launch": "one CUDA graph per step (wr_plan_launch)",
                   "parallelism": f"replicas x{world} (orders are independent)", "tuning": r.tuning(),
                   "tuned_by": tuned_by, "tuning_if_tuned_on_this_batch": tuning_same_batch},
        "roofline": {"kernel": "enum_kernel", "bound": "alu", "achieved": achieved, "peak": alu_peak,
                     "unit": "Tops/s", "frac": achieved / alu_peak, "traffic": None,
                     "peak_source": "derived: 152 SMs x 64 ALU-pipe lanes (min / add-min) x max SM clock",
                     "ops": "one fused add-min per sequence", "ops_per_launch": st["sequences"],
                     "ms_per_launch": enum_ms, "sequences": st["sequences"],
                     "prefix_sharing_ops_per_launch": ops},
        "phases_ms": {kk[3:]: statistics.median(s[kk] for s in stats_list) for kk in
                      ("ms_select", "ms_init", "ms_bf", "ms_gather", "ms_enum", "ms_finish", "ms_total")},
        "plain_per_order": {"value": m / t_plain, "unit": "orders/s", "orders": m,
                            "how": "one wr_route_orders call per order (n=1, device buffers), host wall clock",
                            "bit_exact_vs_graph": same_plain},
        "direct_call_bit_exact_vs_graph": same_direct,
        "e2e": {"value": world * n / e2e_s, "unit": "orders/s", "h2d_bytes_per_step": 8 * (n + 1) + 4 * np_,
                "d2h_bytes_per_step": 8 * n + 4 * np_, "matches_device_run": e2e_ok},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats_list)),
        "clocks": clk.summary(),
        "bf_ms": bf_ms,
    }
    if rank == 0 and not args.no_cpu:
        v, cores, sample = cpu_oracle_rate(g, o, budget_s=args.ref_budget)
        line["cpu_baseline"] = {"value": v, "unit": "orders/s", "cores": cores, "kind": "oracle", "sample": sample}
    plan.close()
    r.close()
    return line if rank == 0 else None


EPOCH = 100_000  # orders between two relocations of the top 5% SKUs


def serving_stream(n, rate, seed=None):
    """Orders of the serving workload (synth.serving_workload): relocation of the top 5%
    SKUs every EPOCH orders, Poisson arrivals at `rate` orders/s."""
    from paper_2504_20655_gb300 import synth
    lay, o, arr, _ = synth.serving_workload(n, rate, synth.SEED_BASE if seed is None else seed, EPOCH)
    return lay, o, arr


def serving_batch_roofline(r, args, reps=5):
    """Sweep and enumeration rooflines of one serving batch (max_batch orders of the stream),
    routed directly with every row computed; medians of reps calls after one warm-up."""
    import torch

    _, o, _ = serving_stream(args.serve_batch, 1000.0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stats = []
    for i in range(reps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        r.route_orders(o.offs, o.picks)
        if i:
            stats.append(r.stats())
    pk = peaks()
    bf_ms = statistics.median(s["ms_bf"] for s in stats)
    enum_ms = statistics.median(s["ms_enum"] for s in stats)
    st = stats[-1]
    achieved = st["bytes_alg"] / (bf_ms / 1e3) / 1e9 if bf_ms > 0 else 0.0
    alu_peak = alu_min_peak(pk)
    tops = st["sequences"] / (enum_ms / 1e3) / 1e12 if enum_ms > 0 else 0.0
    how = (f"one batch of {args.serve_batch} orders of the stream through wr_route_orders, every row computed "
           f"(a served batch computes only its cache misses); L2 flushed before each of {reps} calls, medians")
    return {"bf": {"kernel": sweep_kernel_name(r.tuning()), "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                   "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_source": pk["source"],
                   "bytes_alg_per_launch": st["bytes_alg"], "ms_per_launch": bf_ms, "sources": st["n_sources"],
                   "measured_on": how},
            "enum": {"kernel": "enum_kernel", "bound": "alu", "achieved": tops, "peak": alu_peak, "unit": "Tops/s",
                     "frac": tops / alu_peak, "sequences": st["sequences"], "ms": enum_ms, "measured_on": how}}


def measure_serving(args, rates=None, seconds=None, max_orders=None, plain_max=None, plain_seconds=None):
    """Serving workload: real-time arrivals, continuous batching with a resident row
    cache (wr_serve_*), p50/p99 arrival-to-result latency and orders/s per arrival rate,
    next to the plain mode (one order at a time, rows from scratch).  Each rate's stream
    runs as one server call per relocation epoch (EPOCH orders; the server and its row
    cache persist across calls), so the cache hit rate is reported per epoch; the first
    arrival of an epoch follows the last result of the one before.  Returns the line
    (rank 0) or None."""
    import torch

    from paper_2504_20655_gb300 import synth, wroute
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    rates = rates or [float(x) for x in args.rates.split(",")]
    seconds = args.serve_seconds if seconds is None else seconds
    max_orders = args.serve_max_orders if max_orders is None else max_orders
    plain_max = args.plain_max_orders if plain_max is None else plain_max
    plain_seconds = args.plain_seconds if plain_seconds is None else plain_seconds
    lay = None
    r = wroute.Router(device=local, mem_budget_bytes=args.budget_gib << 30)
    results = []
    with ClockSampler(local) as clk:
        for rate in rates:
            n = int(min(max_orders, max(2000, rate * seconds)))
            lay_r, o, arr = serving_stream(n, rate)
            if lay is None:
                lay = lay_r
                r.load_graph(lay.build())
            row = {"rate": rate, "orders": n}
            for mode in ("batched", "plain"):
                m = n if mode == "batched" else int(min(n, plain_max, max(500, rate * plain_seconds)))
                sv = r.server(plain=(mode == "plain"), max_batch=args.serve_batch, max_batch_picks=12 * args.serve_batch,
                              n_slots=args.serve_slots, cache_bytes=args.serve_cache_gib << 30)
                lat, epochs, t_end = [], [], 0.0
                cost = np.empty(m, np.int32)
                status = np.empty(m, np.int32)
                try:
                    # warm-up on a short prefix (kernels, cache)
                    w = min(200, m)
                    sv.run(arr[:w] - arr[0], o.offs[:w + 1], o.picks[:o.offs[w]])
                    for lo in range(0, m, EPOCH):
                        hi = min(m, lo + EPOCH)
                        sub = o.subset(np.arange(lo, hi))
                        a = arr[lo:hi] - arr[lo]
                        c, _, s_, done = sv.run(a, sub.offs, sub.picks)
                        st = sv.stats()
                        cost[lo:hi], status[lo:hi] = c, s_
                        lat.append((done - a) * 1e3)
                        t_end += max(float(done.max()), float(a[-1]))
                        looked_up = st["cache_hits"] + st["rows_computed"]
                        epochs.append({"epoch": lo // EPOCH, "orders": hi - lo, "batches": st["batches"],
                                       "cache_hit_rate": st["cache_hits"] / looked_up if looked_up else None,
                                       "rows_computed": st["rows_computed"], "evicted_groups": st["evicted_groups"]})
                finally:
                    sv.close()
                lat = np.concatenate(lat)
                row[mode] = {"orders": m, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "orders_per_s": m / t_end, "epochs": len(epochs), "relocations": (m - 1) // EPOCH,
                             "batches": sum(e["batches"] for e in epochs)}
                if mode == "batched":
                    row[mode]["per_epoch"] = epochs
                    chk = min(m, 2000)
                    ref = r.route_orders(o.offs[:chk + 1], o.picks[:o.offs[chk]])
                    row[mode]["bit_exact_vs_direct_first_%d" % chk] = bool(
                        (ref[0] == cost[:chk]).all() and (ref[2] == status[:chk]).all())
                    batched_cost = cost.copy()
                else:
                    row[mode]["bit_exact_vs_batched"] = bool((cost[:m] == batched_cost[:m]).all())
            row["plain"]["keeps_up"] = row["plain"]["orders_per_s"] >= 0.95 * rate
            results.append(row)
    # batched against plain at equal p99: for each rate plain keeps up with, the highest
    # arrival rate the batched server kept up with at a p99 no higher than plain's there
    matched = []
    for row in results:
        if not row["plain"]["keeps_up"]:
            continue
        p99 = row["plain"]["p99_ms"]
        ok = [x["rate"] for x in results if x["batched"]["p99_ms"] <= p99 and x["batched"]["orders_per_s"] >= 0.95 * x["rate"]]
        matched.append({"plain_rate": row["rate"], "plain_p99_ms": p99, "plain_orders_per_s": row["plain"]["orders_per_s"],
                        "batched_max_rate_at_that_p99": max(ok) if ok else None})
    # roofline of the serving batches' dominant kernels, on one batch of max_batch orders of the
    # stream through wr_route_orders with every row computed (a served batch computes only the rows
    # its row cache lacks): the sweep kernel against HBM, the enumeration against the ALU pipe
    roof = serving_batch_roofline(r, args)
    top = results[-1]["batched"]
    line = {
        "metric": "served orders/s (p50/p99 latency)", "value": top["orders_per_s"], "unit": "orders/s",
        "n_gpus": world, "steps": len(rates), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "serving: 200 aisles x 200 slots x 2 sides, 4 cross-aisles (V=80801); Poisson arrivals; "
                               "k=2+Geom(0.3)<=12; Zipf(1.1) over 50k SKUs, top 5% relocated every 1e5 orders",
                   "rates": rates, "orders_per_rate": [x["orders"] for x in results], "max_batch": args.serve_batch,
                   "slots": args.serve_slots, "row_cache_gib": args.serve_cache_gib, "tuning": r.tuning()},
        "serving": results,
        "batched_vs_plain_at_equal_p99": matched,
        "e2e": {"value": top["orders_per_s"], "unit": "orders/s", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": None, "note": "host arrays in and out of every batch: the serving loop is end to end"},
        "clocks": clk.summary(),
        "roofline": roof["bf"],
        "roofline_enum": roof["enum"],
    }
    if rank == 0 and not args.no_cpu:
        _, o, _ = serving_stream(2000, rates[0])
        v, cores, sample = cpu_oracle_rate(lay.build(), o, budget_s=args.ref_budget)
        line["cpu_baseline"] = {"value": v, "unit": "orders/s", "cores": cores, "kind": "oracle", "sample": sample}
    r.close()
    return line if rank == 0 else None


def measure_medium(args):
    """The default workload: one wr_route_orders call over the medium batch per step.
    Returns the line (rank 0) or None."""
    import torch

    from paper_2504_20655_gb300 import wroute
    from paper_2504_20655_gb300 import shard
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # weak scaling: every rank routes its own contiguous slice of 1024 orders of one
    # stream of world x 1024 orders, with no exchange on the data path
    g, o_all, desc = workload(args.workload, n_orders=1024 * world)
    o, o_lo, o_hi = shard.shard_orders(o_all, world, rank)
    r = wroute.Router(device=local, mem_budget_bytes=args.budget_gib << 30)
    if args.tune:
        r.set_tuning(**json.loads(args.tune))
    r.load_graph(g)
    stream = torch.cuda.current_stream(dev)
    offs = torch.from_numpy(o.offs).to(dev)
    picks = torch.from_numpy(o.picks).to(dev)
    n, np_ = o.n, int(o.offs[-1])
    cost = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(max(np_, 1), dtype=torch.int32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step():
        wroute.wr_route_orders(r.ctx, offs, picks, cost, perm, status, stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    r.sync()
    stats_list = []
    times = []
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            e0[i].record(stream)
            step()
            e1[i].record(stream)
            stats_list.append(r.stats())  # syncs; outside the event pair
        torch.cuda.synchronize()
    barrier(world)
    r.sync()
    times = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    ms = sum(times) / len(times)
    ms = max_over_ranks(ms, world, dev)
    value = replica_value(n, ms, world)
    if world > 1:  # the slices' results in batch order (after the timed region)
        g_cost, _, _ = shard.gather_order_results(cost, perm[:np_], status, world, rank)
        gathered = int(g_cost.shape[0])

    # end to end through the C ABI with pinned host buffers
    h_offs = torch.from_numpy(o.offs).pin_memory()
    h_picks = torch.from_numpy(o.picks).pin_memory()
    h_cost = torch.empty(n, dtype=torch.int32).pin_memory()
    h_perm = torch.empty(max(np_, 1), dtype=torch.int32).pin_memory()
    h_status = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        wroute.wr_route_orders(r.ctx, h_offs, h_picks, h_cost, h_perm, h_status, stream.cuda_stream)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), world, dev)
    ok = bool((h_cost.numpy() == cost.cpu().numpy()).all() and (h_perm.numpy()[:np_] == perm.cpu().numpy()[:np_]).all())

    st = stats_list[-1]
    bf_ms = statistics.median(s["ms_bf"] for s in stats_list)
    bytes_alg = st["bytes_alg"]
    pk = peaks()
    achieved = bytes_alg / (bf_ms / 1e3) / 1e9 if bf_ms > 0 else 0.0
    enum_ms = statistics.median(s["ms_enum"] for s in stats_list)
    seqs = st["sequences"]
    clocks = clk.summary()
    alu_peak = alu_min_peak(pk)
    traffic = float(args.traffic) if args.traffic else traffic_for(args.workload, bool(args.tune))
    line = {
        "metric": "exact-routed orders/s", "value": value, "unit": "orders/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": desc, "orders_per_step": n, "sources": st["n_sources"], "l2": "flushed (512 MiB write) between steps",
                   "parallelism": (f"orders split x{world} (contiguous slices of {1024 * world} orders, gathered after "
                                   f"timing: {gathered})" if world > 1 else "one GPU (orders are independent)"),
                   "tuning": r.tuning()},
        "roofline": {"kernel": sweep_kernel_name(r.tuning()), "bound": "hbm", "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "peak_source": pk["source"], "bytes_alg_per_launch": bytes_alg, "ms_per_launch": bf_ms,
                     "sweeps": st["sweeps"]},
        "roofline_enum": {"kernel": "enum_kernel", "bound": "alu", "sequences": seqs, "ms": enum_ms,
                          "gseq_per_s": seqs / (enum_ms / 1e3) / 1e9 if enum_ms > 0 else 0.0,
                          "alu_min_peak_tops": alu_peak,
                          "frac": (seqs / (enum_ms / 1e3) / 1e12) / alu_peak if enum_ms > 0 else 0.0},
        "phases_ms": {k[3:]: statistics.median(s[k] for s in stats_list) for k in
                      ("ms_select", "ms_init", "ms_bf", "ms_gather", "ms_enum", "ms_finish", "ms_total")},
        "e2e": {"value": world * n / e2e_s, "unit": "orders/s", "h2d_bytes_per_step": 8 * (n + 1) + 4 * np_,
                "d2h_bytes_per_step": 8 * n + 4 * np_, "matches_device_run": ok},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats_list)),
        "clocks": clocks,
        "paper_convention_mteps": paper_mteps(g.V, g.E, st["n_sources"], bf_ms / 1e3),
    }
    if args.trace:
        # one more call, untimed, with the sweep trace on: per sweep its frontier tiles and the
        # microseconds until the next sweep starts (the last: until the kernel's exit check)
        r.set_trace(4096)
        flush.zero_()
        torch.cuda.synchronize()
        step()
        r.sync()
        tr = r.trace()
        r.set_trace(0)
        line["sweep_trace"] = [[int(tr[i][0]), (int(tr[i + 1][1]) - int(tr[i][1])) / 1e3 if i + 1 < len(tr) else None]
                               for i in range(len(tr))]
    if rank == 0 and not args.no_cpu:
        v, cores, sample = cpu_oracle_rate(g, o, budget_s=args.ref_budget)
        line["cpu_baseline"] = {"value": v, "unit": "orders/s", "cores": cores, "kind": "oracle", "sample": sample}
    r.close()
    return line if rank == 0 else None


def hk_transitions(k):
    """Held-Karp transitions of one order of k picks: a set S of visited picks with its
    last pick c and a next pick j outside S (k(k-1)2^(k-2) of them), plus the k legs
    from the depot and the k legs back.  Each is one saturating add and one min."""
    return k * (k - 1) * (1 << (k - 2)) + 2 * k


def hk_table_bytes(k):
    """Algorithmic table traffic of Held-Karp for one order of k picks: every word
    h(S, c) of the 2^k x k table written once, and read once by the level below
    (h(S + j, j) for each S without j), 4 bytes each: k 2^(k-1) words each way."""
    return 2 * 4 * k * (1 << (k - 1))


def run_next(args):
    """The rows past the core of the path, each to the same bar as the medium line:
    Held-Karp for orders of 13..20 picks, open paths, cluster-patched approximate routes
    and node-level routes.  Timing (CUDA events on the launching stream, L2 flushed
    between steps), end to end through the C ABI with host buffers, the oracle in the
    same mode on the host's cores, the dominant kernel against its roofline."""
    import torch

    from paper_2504_20655_gb300 import synth, wroute
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = args.workload
    g, o, desc = workload(w)
    r = wroute.Router(device=local, mem_budget_bytes=args.budget_gib << 30, max_k=20 if w == "heldkarp" else 12)
    if args.tune:
        r.set_tuning(**json.loads(args.tune))
    r.load_graph(g)
    if w == "open":
        r.set_route_mode(True)
    if w == "clustered":
        r.set_clusters(3, synth.medium_layout().coords())
    stream = torch.cuda.current_stream(dev)
    n, np_ = o.n, int(o.offs[-1])
    offs = torch.from_numpy(o.offs).to(dev)
    picks = torch.from_numpy(o.picks).to(dev)
    cost = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(max(np_, 1), dtype=torch.int32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    if w == "nodes":
        # the exact sequences first (untimed), then their node-level routes
        wroute.wr_route_orders(r.ctx, offs, picks, cost, perm, status, stream.cuda_stream)
        node_offs = torch.zeros(n + 1, dtype=torch.int64, device=dev)
        wroute.wr_route_nodes(r.ctx, offs, picks, perm, node_offs, None, 0, stream.cuda_stream)
        torch.cuda.synchronize()
        n_nodes = int(node_offs[-1].item())
        nodes = torch.empty(max(n_nodes, 1), dtype=torch.int32, device=dev)

        def step():
            wroute.wr_route_nodes(r.ctx, offs, picks, perm, node_offs, nodes, n_nodes, stream.cuda_stream)
    else:
        def step():
            wroute.wr_route_orders(r.ctx, offs, picks, cost, perm, status, stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    r.sync()
    stats_list = []
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            e0[i].record(stream)
            step()
            e1[i].record(stream)
            stats_list.append(r.stats())  # syncs; outside the event pair
        torch.cuda.synchronize()
    barrier(world)
    r.sync()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / args.steps, world, dev)
    value = replica_value(n, ms, world)

    # end to end with pinned host buffers
    h_offs = torch.from_numpy(o.offs).pin_memory()
    h_picks = torch.from_numpy(o.picks).pin_memory()
    if w == "nodes":
        h_perm_in = perm[:max(np_, 1)].cpu().pin_memory()
        h_noffs = torch.zeros(n + 1, dtype=torch.int64).pin_memory()
        h_nodes = torch.empty(max(n_nodes, 1), dtype=torch.int32).pin_memory()

        def e2e_step():
            wroute.wr_route_nodes(r.ctx, h_offs, h_picks, h_perm_in, h_noffs, h_nodes, n_nodes, stream.cuda_stream)
        h2d, d2h = 8 * (n + 1) + 8 * np_, 8 * (n + 1) + 4 * n_nodes
    else:
        h_cost = torch.empty(n, dtype=torch.int32).pin_memory()
        h_perm = torch.empty(max(np_, 1), dtype=torch.int32).pin_memory()
        h_status = torch.empty(n, dtype=torch.int32).pin_memory()

        def e2e_step():
            wroute.wr_route_orders(r.ctx, h_offs, h_picks, h_cost, h_perm, h_status, stream.cuda_stream)
        h2d, d2h = 8 * (n + 1) + 4 * np_, 8 * n + 4 * np_
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), world, dev)
    if w == "nodes":
        ok = bool((h_noffs.numpy() == node_offs.cpu().numpy()).all()
                  and (h_nodes.numpy()[:n_nodes] == nodes.cpu().numpy()[:n_nodes]).all())
    else:
        ok = bool((h_cost.numpy() == cost.cpu().numpy()).all() and (h_status.numpy() == status.cpu().numpy()).all())

    st = stats_list[-1]
    pk = peaks()
    phases = {k[3:]: statistics.median(s[k] for s in stats_list) for k in
              ("ms_select", "ms_init", "ms_bf", "ms_gather", "ms_enum", "ms_finish", "ms_total")}
    bf_ms = phases["bf"]
    bf_gbs = st["bytes_alg"] / (bf_ms / 1e3) / 1e9 if bf_ms > 0 else 0.0
    bf_roof = {"kernel": sweep_kernel_name(r.tuning()), "bound": "hbm", "achieved": bf_gbs, "peak": pk["hbm_gbs"],
               "unit": "GB/s", "frac": bf_gbs / pk["hbm_gbs"], "traffic": None, "peak_source": pk["source"],
               "bytes_alg_per_launch": st["bytes_alg"], "ms_per_launch": bf_ms, "sweeps": st["sweeps"]}
    alu_peak = alu_min_peak(pk)
    extra = {}
    if w == "heldkarp":
        # the solve kernel dominates; its tables (2^k x k words per order) stream through HBM
        # once each way, which binds before the ALU pipe does (2 operations per transition)
        k = o.k()
        trans = float(sum(hk_transitions(int(kk)) for kk in k))
        tbytes = float(sum(hk_table_bytes(int(kk)) for kk in k))
        hk_ms = phases["enum"]
        achieved = tbytes / (hk_ms / 1e3) / 1e9 if hk_ms > 0 else 0.0
        roof = {"kernel": "hk_solve_kernel", "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_source": pk["source"],
                "bytes_alg_per_launch": tbytes, "ms_per_launch": hk_ms, "transitions_per_launch": trans,
                "transitions_per_s": trans / (hk_ms / 1e3) if hk_ms > 0 else 0.0,
                "alu_frac": (2 * trans / (hk_ms / 1e3) / 1e12) / alu_peak if hk_ms > 0 else 0.0}
        extra["roofline_bf"] = bf_roof
        metric = "exact-routed orders/s"
    else:
        roof = bf_roof
        metric = METRIC.get(w, "exact-routed orders/s")
        if w == "clustered":
            extra["cluster_kernel_ms"] = phases["enum"]
            # context: the approximate costs against the exact ones (same GPU, exact routing)
            rx = wroute.Router(device=local, mem_budget_bytes=args.budget_gib << 30)
            rx.load_graph(g)
            cx, _, sx = rx.route_orders(o.offs, o.picks)
            rx.close()
            ca = cost.cpu().numpy()
            okm = (sx == 0) & (status.cpu().numpy() == 0)
            extra["cost_ratio_vs_exact"] = {"mean": float(np.mean(ca[okm] / cx[okm])),
                                            "max": float(np.max(ca[okm] / cx[okm])),
                                            "exact_share": float(np.mean(ca[okm] == cx[okm]))}
        if w == "nodes":
            extra["nodes_per_step"] = n_nodes
            extra["walk_ms"] = phases["finish"]
    line = {
        "metric": metric, "value": value, "unit": "orders/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": desc, "orders_per_step": n, "sources": st["n_sources"],
                   "l2": "flushed (512 MiB write) between steps",
                   "parallelism": f"replicas x{world} (orders are independent)", "tuning": r.tuning()},
        "roofline": roof,
        "phases_ms": phases,
        "e2e": {"value": world * n / e2e_s, "unit": "orders/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "matches_device_run": ok},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats_list)),
        "clocks": clk.summary(),
    }
    line.update(extra)
    if rank == 0 and not args.no_cpu:
        mode = w
        v, cores, sample = cpu_oracle_rate(g, o, budget_s=args.ref_budget, mode=mode)
        line["cpu_baseline"] = {"value": v, "unit": "orders/s", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line))
    r.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="medium",
                    choices=["medium", "batching", "tiny", "scale", "serving", "heldkarp", "open", "clustered", "nodes"])
    ap.add_argument("--budget-gib", type=int, default=2)
    ap.add_argument("--tune", default="")
    ap.add_argument("--traffic", default="")
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--scale-sources", type=int, default=4096, help="sources of the scale workload")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--trace", action="store_true",
                    help="medium line: add the sweep trace of one more, untimed call (frontier tiles, us per sweep)")
    ap.add_argument("--plain-budget", type=float, default=3.0, help="seconds of plain per-order calls (batching)")
    ap.add_argument("--rates", default="1000,5000,20000,50000", help="serving: arrival rates, orders/s")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="serving: seconds of arrivals per rate")
    ap.add_argument("--serve-max-orders", type=int, default=100_000)
    ap.add_argument("--plain-max-orders", type=int, default=3000)
    ap.add_argument("--plain-seconds", type=float, default=1.5, help="serving: seconds of arrivals for the plain mode")
    ap.add_argument("--only", action="store_true",
                    help="default workload: the medium line alone, without the scale, batching and serving parts")
    ap.add_argument("--serve-batch", type=int, default=256)
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--serve-cache-gib", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    from paper_2504_20655_gb300 import build
    build.build()
    measure = {"scale": measure_scale, "batching": measure_batching, "serving": measure_serving}.get(args.workload)
    if args.workload in ("heldkarp", "open", "clustered", "nodes"):
        return run_next(args)
    if measure is not None:
        line = measure(args)
    else:
        line = measure_medium(args)
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if line is not None and world == 1 and not args.only and args.workload == "medium":
            # the rest of the headline metric from the same run: BF Gedges/s at scale against
            # HBM, the batching plan against plain per-order calls, served p50/p99 against plain
            line["workloads"] = {
                "scale": measure_scale(args),
                "batching": measure_batching(args),
                "serving": measure_serving(args, rates=[1000, 2000, 5000, 10000, 20000, 50000], seconds=1.0,
                                           max_orders=50_000, plain_max=1500, plain_seconds=0.75),
            }
    if line is not None:
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
