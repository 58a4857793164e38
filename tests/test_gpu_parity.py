"""GPU path vs the CPU oracle, element by element, through the C ABI.

All results are integers, so the bar is bit-exact equality: distance rows,
tour costs, argmin permutations (the lexicographically first minimiser)
and per-order statuses.
"""
import os

import numpy as np
import pytest

from paper_2504_20655_gb300 import synth
from tests.graphs import random_graph

pytestmark = pytest.mark.gpu
INF = 2**31 - 1
NT = os.cpu_count() or 4


@pytest.fixture(scope="module")
def wr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2504_20655_gb300 import build, wroute
    build.build()
    return wroute


@pytest.fixture(scope="module")
def router(wr):
    r = wr.Router(device=0)
    yield r
    r.close()


def test_bf_rows_tiny_all_sources(router, orc):
    g = synth.tiny_layout().build()
    router.load_graph(g)
    rows = router.bf_rows(np.arange(g.V, dtype=np.int32))
    assert (rows == orc.floyd_warshall(g)).all()
    st = router.stats()
    assert st["sweeps"] >= 1 and st["bytes_alg"] > 0


@pytest.fixture(params=[2, 1, 3, 4], ids=["cta_tiles", "warp_tiles", "warp_worklist", "warp_pairs"])
def tiling(request, router):
    saved = router.tuning()
    router.set_tuning(bf_tiling=request.param)
    yield request.param
    router.set_tuning(**saved)


@pytest.mark.parametrize("seed", range(8))
def test_bf_rows_random_graphs(router, orc, seed, tiling):
    V = [1, 2, 7, 33, 100, 257, 600, 1500][seed]
    g = random_graph(V, max(1, 3 * V), seed + 300, w_lo=0, w_hi=20 if seed % 2 else 1000)
    router.load_graph(g)
    src = np.arange(0, V, max(1, V // 70), dtype=np.int32)
    rows = router.bf_rows(src)
    ref = orc.sssp_rows(g, src, "dijkstra", NT)
    assert (rows == ref).all()


def test_bf_rows_chains_both_tilings(router, orc, tiling):
    """Long chains with sparse extra arcs (mostly compact runs for the warp tiling),
    directed and with zero weights, many sources."""
    V = 3000
    u = np.arange(V - 1, dtype=np.int64)
    v = u + 1
    extra_u = synth.uniform_int(91, 400, 0, V - 1)
    extra_v = synth.uniform_int(92, 400, 0, V - 1)
    w = np.concatenate([synth.uniform_int(93, V - 1, 0, 30), synth.uniform_int(94, V - 1, 0, 30),
                        synth.uniform_int(95, 400, 0, 500)])
    uu = np.concatenate([u, v, extra_u])
    vv = np.concatenate([v, u[: V - 1] * 0 + u, extra_v])
    keep = uu != vv
    rp, col, wt = synth.csr_from_arcs(V, uu[keep], vv[keep], w[keep])
    g = synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0)
    router.load_graph(g)
    src = np.arange(0, V, 23, dtype=np.int32)
    assert (router.bf_rows(src) == orc.sssp_rows(g, src, "dijkstra", NT)).all()


def test_bf_rows_high_in_degree(router, orc, tiling):
    # a node with more in-neighbours than a tile holds: its halo spills to global reads
    V = 700
    u = np.concatenate([np.arange(1, V), np.zeros(V - 1, np.int64)])
    v = np.concatenate([np.zeros(V - 1, np.int64), np.arange(1, V)])
    w = synth.uniform_int(77, u.shape[0], 1, 50)
    rp, col, wt = synth.csr_from_arcs(V, u, v, w)
    g = synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0)
    router.load_graph(g)
    src = np.array([0, 5, 699, 350], np.int32)
    assert (router.bf_rows(src) == orc.sssp_rows(g, src)).all()


@pytest.mark.parametrize("tune", [dict(run_target=96, tile_cap=128), dict(run_target=32, tile_cap=128),
                                  dict(run_target=200, tile_cap=256), dict(run_target=1, tile_cap=128),
                                  dict(run_target=400, tile_cap=512), dict(run_target=256, tile_cap=256),
                                  dict(run_target=200, tile_cap=256, bf_tiling=2),
                                  dict(run_target=200, tile_cap=256, bf_tiling=2, bf_warps=8),
                                  dict(run_target=100, tile_cap=128, bf_tiling=2, bf_warps=8),
                                  dict(run_target=96, tile_cap=128, bf_tiling=2),
                                  dict(run_target=1, tile_cap=128, bf_tiling=2),
                                  dict(run_target=200, tile_cap=256, bf_tiling=1),
                                  dict(run_target=256, tile_cap=256, bf_tiling=1),
                                  dict(run_target=96, tile_cap=128, bf_tiling=1),
                                  dict(run_target=1, tile_cap=128, bf_tiling=1),
                                  dict(run_target=60, tile_cap=128, bf_tiling=3),
                                  dict(run_target=200, tile_cap=256, bf_tiling=3),
                                  dict(run_target=1, tile_cap=128, bf_tiling=3),
                                  dict(run_target=60, tile_cap=128, bf_tiling=4),
                                  dict(run_target=96, tile_cap=128, bf_tiling=4),
                                  dict(run_target=1, tile_cap=128, bf_tiling=4)])
def test_bf_rows_medium_tuning_invariant(router, orc, tune):
    g = synth.medium_layout().build()
    saved = router.tuning()
    router.set_tuning(**tune)
    try:
        router.load_graph(g)
        src = synth.distinct_sources(200, g.n_slots, 17)
        src = np.concatenate([src, [g.depot]]).astype(np.int32)
        rows = router.bf_rows(src)
    finally:
        router.set_tuning(**saved)
    ref = orc.sssp_rows(g, src, "dijkstra", NT)
    assert (rows == ref).all()


def test_bf_segments_small_budget(wr, orc):
    g = synth.medium_layout().build()
    r = wr.Router(device=0, mem_budget_bytes=g.V * 4 * 64)  # 64 lanes per segment
    r.load_graph(g)
    src = synth.distinct_sources(150, g.n_slots, 3)
    rows = r.bf_rows(src)
    assert r.stats()["n_segments"] == 3
    assert (rows == orc.sssp_rows(g, src, "dijkstra", NT)).all()
    r.close()


def test_budget_too_small(wr):
    g = synth.tiny_layout().build()
    r = wr.Router(device=0, mem_budget_bytes=g.V * 4 * 16)
    r.load_graph(g)
    with pytest.raises(wr.WrError) as e:
        r.bf_rows(np.array([1, 2], np.int32))
    assert e.value.code == wr.WR_ENOMEM
    r.close()


def test_route_tiny(router, orc):
    g, o = synth.tiny_workload()
    router.load_graph(g)
    cost, perm, status = router.route_orders(o.offs, o.picks)
    c, p, s = orc.route_orders(g, o, "rounds", "brute")
    assert (cost == c).all() and (perm == p).all() and (status == s).all()
    st = router.stats()
    assert st["sequences"] == 720 and st["n_sources"] == 7


def test_route_medium_full(router, orc):
    """The benchmark's workload: 1024 orders, k in [4, 10], Zipf picks, medium layout."""
    g, o = synth.medium_workload()
    router.load_graph(g)
    cost, perm, status = router.route_orders(o.offs, o.picks)
    c, p, s = orc.route_orders(g, o, "dijkstra", "brute", NT)
    assert (status == s).all()
    assert (cost == c).all()
    assert (perm[:len(p)] == p).all()
    st = router.stats()
    assert st["sequences"] == sum(int(np.prod(np.arange(1, k + 1))) for k in o.k())


def test_route_device_pointers_and_stream(router, orc):
    import torch
    g, o = synth.medium_workload(n_orders=64)
    router.load_graph(g)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        offs = torch.from_numpy(o.offs).cuda()
        picks = torch.from_numpy(o.picks).cuda()
        cost, perm, status = router.route_orders(offs, picks)
    s.synchronize()
    router.sync()
    c, p, st = orc.route_orders(g, o, "dijkstra", "brute", NT)
    _assert_same(o, (cost.cpu().numpy(), perm.cpu().numpy(), status.cpu().numpy()), (c, p, st))


def test_route_device_pointers_default_stream(router, orc):
    import torch
    g, o = synth.medium_workload(n_orders=64)
    router.load_graph(g)
    offs = torch.from_numpy(o.offs).cuda()
    picks = torch.from_numpy(o.picks).cuda()
    cost, perm, status = router.route_orders(offs, picks)
    torch.cuda.synchronize()
    router.sync()
    c, p, st = orc.route_orders(g, o, "dijkstra", "brute", NT)
    _assert_same(o, (cost.cpu().numpy(), perm.cpu().numpy(), status.cpu().numpy()), (c, p, st))


def _assert_same(o, got, want):
    cost, perm, status = got
    c, p, st = want
    bad_st = np.nonzero(status != st)[0]
    bad_c = np.nonzero(cost != c)[0]
    bad_p = sorted({int(np.searchsorted(o.offs, i, side="right") - 1) for i in np.nonzero(perm[:len(p)] != p)[0]})
    msg = (f"status differs at {bad_st[:10].tolist()}, cost differs at {bad_c[:10].tolist()} "
           f"(got {cost[bad_c[:5]].tolist()} want {c[bad_c[:5]].tolist()}), perm differs in orders {bad_p[:10]}")
    assert len(bad_st) == 0 and len(bad_c) == 0 and len(bad_p) == 0, msg


def test_route_statuses_and_edge_cases(router, orc):
    g = synth.medium_layout().build()
    router.load_graph(g)
    V = g.V
    orders = [[5], [5, 5], list(range(100, 112)), list(range(200, 213)), [], [3, V], [-1, 2],
              [g.depot, 7, g.depot], [19999, 0, 10000, 15000, 5000, 12345, 54, 9999, 1, 2, 3]]
    offs = np.zeros(len(orders) + 1, np.int64)
    offs[1:] = np.cumsum([len(x) for x in orders])
    picks = np.array([x for od in orders for x in od], np.int32)
    o = synth.Orders(offs, picks)
    cost, perm, status = router.route_orders(o.offs, o.picks)
    c, p, s = orc.route_orders(g, o, "dijkstra", "heldkarp", NT, max_k=12)  # the context's default max_k
    assert status.tolist() == s.tolist() == [0, 0, 0, 2, 2, 2, 2, 0, 0]
    assert (cost == c).all() and (perm[:len(p)] == p).all()


def test_route_unreachable(router, orc):
    # directed chain 0 -> 1 -> 2 -> 3, depot 0: picks behind the depot cannot return
    V = 6
    u = np.array([0, 1, 2, 3, 4]); v = np.array([1, 2, 3, 0, 5]); w = np.array([3, 4, 5, 6, 1])
    rp, col, wt = synth.csr_from_arcs(V, u, v, w)
    g = synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0)
    router.load_graph(g)
    o = synth.Orders(np.array([0, 2, 3, 5], np.int64), np.array([1, 2, 5, 3, 1], np.int32))
    cost, perm, status = router.route_orders(o.offs, o.picks)
    c, p, s = orc.route_orders(g, o, "rounds", "brute")
    assert status.tolist() == s.tolist() == [0, 1, 0]
    assert cost.tolist() == c.tolist() and perm.tolist() == p.tolist()


def _rand_D(n, k, seed, hi, p_inf=0.0):
    m = k + 1
    D = synth.uniform_int(seed, n * 169, 0, hi).reshape(n, 13, 13).astype(np.int64)
    if p_inf:
        D = np.where(synth.uniform01(seed ^ 5, n * 169).reshape(n, 13, 13) < p_inf, INF, D)
    for i in range(13):
        D[:, i, i] = 0
    return D.astype(np.int32), m


@pytest.mark.parametrize("k", range(1, 11))
def test_tour_eval_vs_brute(router, orc, k):
    n = 24 if k <= 8 else 6
    for hi, p_inf in ((3, 0.0), (500, 0.0), (40, 0.15)):
        D, m = _rand_D(n, k, 1000 * k + hi, hi, p_inf)
        kk = np.full(n, k, np.int32)
        cost, perm, status = router.tour_eval(kk, D)
        for i in range(n):
            st, c, p = orc.tour(D[i, :m, :m], "brute")
            assert status[i] == st and cost[i] == c and perm[i, :k].tolist() == p.tolist(), (k, hi, i)


@pytest.mark.parametrize("k", [11, 12])
def test_tour_eval_vs_held_karp(router, orc, k):
    n = 3
    for hi in (2, 1000):
        D, m = _rand_D(n, k, 77 * k + hi, hi)
        cost, perm, status = router.tour_eval(np.full(n, k, np.int32), D)
        for i in range(n):
            st, c, p = orc.tour(D[i, :m, :m], "heldkarp")
            assert status[i] == st and cost[i] == c and perm[i, :k].tolist() == p.tolist()


def test_enumeration_batch_and_single_calls(router, orc):
    """36 orders of 7..12 picks with legs in 0..3 (ties everywhere, so the tie rule decides every
    result), in one call and one order per call: the same bits, equal to the oracle's Held-Karp
    with the same tie rule.  The call holds 34 orders of 11 or 12 picks, enough for set units
    (a set of the first picks walked in every order after one table build); one order alone
    takes prefix units."""
    kk = np.array([12] * 32 + [7, 11, 9, 11], np.int32)
    D, _ = _rand_D(len(kk), 12, 5150, 3)
    cost, perm, status = router.tour_eval(kk, D)
    for i, k in enumerate(kk):
        st, c, p = orc.tour(D[i, :k + 1, :k + 1], "heldkarp")
        assert status[i] == st == 0 and cost[i] == c and perm[i, :k].tolist() == p.tolist(), i
        c1, p1, s1 = router.tour_eval(kk[i:i + 1], D[i:i + 1])
        assert c1[0] == cost[i] and s1[0] == status[i] and (p1[0, :k] == perm[i, :k]).all(), i


def test_tour_eval_large_legs(router, orc):
    """Legs up to 10^6 (sequence costs up to 1.3e7): the 32-bit sums stay exact."""
    for k in (6, 8, 10, 12):
        D, m = _rand_D(3, k, 991 * k, 10**6)
        cost, perm, status = router.tour_eval(np.full(3, k, np.int32), D)
        for i in range(3):
            st, c, p = orc.tour(D[i, :m, :m], "brute" if k <= 8 else "heldkarp")
            assert status[i] == st == 0 and cost[i] == c and perm[i, :k].tolist() == p.tolist(), (k, i)


def test_tour_eval_statuses(router, orc):
    D, _ = _rand_D(4, 6, 9, 100)
    kk = np.array([0, 13, 6, 6], np.int32)
    D[3, 1, 2] = 10324441
    cost, perm, status = router.tour_eval(kk, D)
    assert status.tolist() == [2, 2, 0, 3]
    assert cost[3] == INF and perm[3, :6].tolist() == list(range(6))


@pytest.mark.parametrize("units,per_launch", [(1, 0), (16, 0), (4, 7), (2, 1000)])
def test_enumeration_segment_invariance(router, orc, units, per_launch):
    D, m = _rand_D(6, 9, 4242, 4)  # heavy ties
    kk = np.array([9, 8, 7, 9, 5, 3], np.int32)
    base = router.tour_eval(kk, D)
    router.set_tuning(enum_units=units, enum_max_units_per_launch=per_launch)
    try:
        got = router.tour_eval(kk, D)
    finally:
        router.set_tuning(enum_units=4, enum_max_units_per_launch=0)
    for a, b in zip(base, got):
        assert (a == b).all()
    for i, k in enumerate(kk):
        st, c, p = orc.tour(D[i, :k + 1, :k + 1], "brute")
        assert got[0][i] == c and got[1][i, :k].tolist() == p.tolist()


def test_batching_sample(router, orc):
    """Orders of uneven size (k = 2..12) from the batching workload, Held-Karp-lex oracle."""
    g, o = synth.batching_workload()
    k = o.k()
    idx = np.concatenate([np.nonzero(k == kk)[0][:6] for kk in range(2, 13)])
    sub = o.subset(idx)
    router.load_graph(g)
    cost, perm, status = router.route_orders(sub.offs, sub.picks)
    c, p, s = orc.route_orders(g, sub, "dijkstra", "heldkarp", NT)
    assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all()


def test_scale_submatrix_full_size(wr, orc):
    """Scale workload at full size, as the benchmark runs it: 4096 sources over
    V = 1,002,001 under the 2 GiB budget (8 segments).  Sampled rows and their
    checksums against the oracle; symmetry of the whole 4096 x 4096 submatrix
    (the layout is undirected) and the triangle inequality on a sample."""
    import torch
    g, src = synth.scale_workload()
    r = wr.Router(device=0, mem_budget_bytes=2 << 30)
    try:
        r.load_graph(g)
        d_src = torch.from_numpy(src).cuda()
        sub = torch.empty((len(src), len(src)), dtype=torch.int32, device="cuda")
        check = torch.empty(len(src), dtype=torch.int64, device="cuda")
        wr.wr_submatrix(r.ctx, d_src, d_src, sub, check)
        torch.cuda.synchronize()
        r.sync()
        assert r.stats()["n_segments"] == 8
    finally:
        r.close()
    sub = sub.cpu().numpy()
    check = check.cpu().numpy().view(np.uint64)
    assert (sub == sub.T).all() and (np.diag(sub) == 0).all()
    pick = [0, 511, 512, 2047, 3000, 4095]  # across segment boundaries
    rows = orc.sssp_rows(g, src[pick], "dijkstra", NT)
    weights = (2 * np.arange(g.V, dtype=np.uint64) + 1)
    for i, p in enumerate(pick):
        assert (sub[p] == rows[i][src]).all()
        assert check[p] == np.uint64((rows[i].astype(np.uint64) * weights).sum(dtype=np.uint64))
    s = synth.distinct_sources(64, len(src), 99)
    m = sub[np.ix_(s, s)].astype(np.int64)
    for k in range(len(s)):
        assert (m <= m[:, k:k + 1] + m[k:k + 1, :]).all()


def test_sweep_trace(router, orc):
    """The sweep trace of a one-segment call: one entry per sweep plus the end marker,
    frontiers summing to the tile visits, non-decreasing device times; tracing off
    leaves results unchanged."""
    g, o = synth.medium_workload(n_orders=64)
    saved = router.tuning()
    router.set_tuning(bf_tiling=1)  # the trace records sweeps: a sweep tiling
    router.load_graph(g)
    ref = router.route_orders(o.offs, o.picks)
    router.set_trace(4096)
    try:
        got = router.route_orders(o.offs, o.picks)
        st = router.stats()
        tr = router.trace()
    finally:
        router.set_trace(0)
        router.set_tuning(**saved)
    for a, b in zip(ref, got):
        assert (np.asarray(a) == np.asarray(b)).all()
    assert st["n_segments"] == 1
    assert len(tr) == st["sweeps"] + 1
    assert tr[-1, 0] == 0 and (tr[:-1, 0] > 0).all()
    assert int(tr[:, 0].sum()) == st["tile_visits"]
    assert (np.diff(tr[:, 1]) >= 0).all()
    assert len(router.trace()) == 0


def _plan_run(plan, offs, picks):
    import torch
    plan.set_batch(offs, picks)
    plan.launch()
    plan.sync()
    torch.cuda.synchronize()
    return plan.cost.cpu().numpy(), plan.perm.cpu().numpy(), plan.status.cpu().numpy()


def test_plan_graph_matches_direct_calls(router, orc):
    """A captured plan replays the whole path on new batch contents: each launch equals
    a direct wr_route_orders call on the same batch, padding orders come back BAD, and
    loading another graph into the context afterwards does not disturb the plan."""
    g, o = synth.batching_workload(n_orders=700)
    router.load_graph(g)
    a = o.subset(np.arange(0, 500))
    b = o.subset(np.arange(699, 199, -1))  # other contents, other size
    np_cap = int(max(a.offs[-1], b.offs[-1])) + 7
    plan = router.plan(520, np_cap)
    try:
        ref_a = router.route_orders(a.offs, a.picks)
        ref_b = router.route_orders(b.offs, b.picks)
        tiny = synth.tiny_layout().build()
        router.load_graph(tiny)  # the plan keeps its own copy of the medium graph
        for batch, ref in ((a, ref_a), (b, ref_b), (a, ref_a)):
            cost, perm, status = _plan_run(plan, batch.offs, batch.picks)
            n, npk = batch.n, int(batch.offs[-1])
            assert (cost[:n] == ref[0]).all() and (status[:n] == ref[2]).all()
            assert (perm[:npk] == ref[1][:npk]).all()
            assert (status[n:] == 2).all()  # padding: empty orders are WR_ORDER_BAD
        st = plan.stats()
        assert st["n_orders"] == 520 and st["sequences"] > 0
        assert st["n_sources"] == len(np.unique(np.append(a.picks, g.depot)))  # depot + distinct picks
    finally:
        plan.close()
    c, p, s = orc.route_orders(g, a.subset(np.arange(0, 60)), "dijkstra", "heldkarp", NT)
    assert (ref_a[0][:60] == c).all() and (ref_a[2][:60] == s).all()


def test_plan_batching_full_size(router, orc):
    """The batching workload at full size through the captured graph the benchmark
    launches: 20,000 orders, k = 2..12.  Every order against the Held-Karp-lex oracle
    (cost, argmin, status); brute force on a seeded 5% of the k >= 10 orders."""
    g, o = synth.batching_workload()
    router.load_graph(g)
    plan = router.plan(o.n, int(o.offs[-1]))
    try:
        cost, perm, status = _plan_run(plan, o.offs, o.picks)
    finally:
        plan.close()
    c, p, s = orc.route_orders(g, o, "dijkstra", "heldkarp", NT)
    assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all()
    k = o.k()
    big = np.nonzero(k >= 10)[0]
    rng = np.random.default_rng(2504)
    pick = np.sort(rng.choice(big, size=max(1, len(big) // 20), replace=False))
    sub = o.subset(pick)
    cb, pb, sb = orc.route_orders(g, sub, "dijkstra", "brute", NT)
    assert (cb == cost[pick]).all() and (sb == status[pick]).all()
    for j, i in enumerate(pick):
        lo, hi = o.offs[i], o.offs[i + 1]
        assert (perm[lo:hi] == pb[sub.offs[j]:sub.offs[j + 1]]).all()


def test_autotune_keeps_results(wr, orc, tmp_path):
    """The autotuner only changes speed: the tuned context routes bit-identically, writes
    its choice to the tuning file, and a new context reads that file back."""
    g, o = synth.medium_workload(n_orders=96)
    path = str(tmp_path / "wroute.tune")
    r = wr.Router(device=0, tune_path=path)
    try:
        r.load_graph(g)
        ref = r.route_orders(o.offs, o.picks)
        best = r.autotune(o.offs, o.picks, reps=1)
        assert r.tuning() == best
        got = r.route_orders(o.offs, o.picks)
        for a, b in zip(ref, got):
            assert (np.asarray(a) == np.asarray(b)).all()
    finally:
        r.close()
    text = open(path).read()
    assert f"tile_cap {best['tile_cap']}" in text and f"bf_tiling {best['bf_tiling']}" in text
    r2 = wr.Router(device=0, tune_path=path)
    try:
        assert r2.tuning() == best
    finally:
        r2.close()
    c, p, s = orc.route_orders(g, o, "dijkstra", "brute", NT)
    assert (ref[0] == c).all() and (ref[2] == s).all()


def _serve_orders(n, seed=2504, rate=20000.0):
    lay = synth.serve_layout(seed)
    g = lay.build()
    smap = synth.sku_slot_map(50_000, lay.n_slots, seed)
    k = synth.geometric_k(n, 0.3, 2, 12, seed)
    o = synth.zipf_orders(n, k, smap, 1.1, seed)
    return g, o, synth.poisson_arrivals(n, rate, seed)


def test_serve_mix_equals_alone(router, orc):
    """Serving loop with a small row cache (evictions happen) over a stream whose top 5%
    SKUs move to new slots twice inside the run (every 1000 orders): every order's result
    is the same in the mix as alone, bad orders are reported, completion follows arrival."""
    lay, o, arr, relocations = synth.serving_workload(3000, 20000.0, 2504, epoch=1000)
    assert relocations == 2
    g = lay.build()
    # two bad orders: a node out of range, an empty order
    picks = o.picks.copy()
    picks[o.offs[7]] = g.V + 5
    offs = o.offs.copy()
    offs[12:] -= offs[12] - offs[11]
    picks = np.delete(picks, np.arange(o.offs[11], o.offs[12]))
    router.load_graph(g)
    sv = router.server(max_batch=128, max_batch_picks=2048, n_slots=3, cache_bytes=200 << 20)
    try:
        cost, perm, status, done = sv.run(arr, offs, picks)
        st = sv.stats()
    finally:
        sv.close()
    assert st["orders"] == 3000 and st["batches"] > 1
    assert st["evicted_groups"] > 0 and st["cache_hits"] > 0
    assert (done >= arr - 1e-9).all()
    assert status[7] == 2 and status[11] == 2
    ref = router.route_orders(offs, picks)
    assert (cost == ref[0]).all() and (status == ref[2]).all() and (perm[:offs[-1]] == ref[1][:offs[-1]]).all()
    for i in range(0, 3000, 75):  # each alone
        lo, hi = offs[i], offs[i + 1]
        c1, p1, s1 = router.route_orders(np.array([0, hi - lo], np.int64), picks[lo:hi])
        assert c1[0] == cost[i] and s1[0] == status[i] and (p1[:hi - lo] == perm[lo:hi]).all()
    sub = [i for i in range(0, 3000, 15) if i not in (7, 11)]
    so = synth.Orders(offs, picks).subset(sub)
    c, p, s = orc.route_orders(g, so, "dijkstra", "heldkarp", NT)
    assert (cost[sub] == c).all() and (status[sub] == s).all()


def test_serve_plain_baseline(router):
    """The plain mode (one order at a time, rows from scratch) gives the same results."""
    g, o, arr = _serve_orders(200, rate=5000.0)
    router.load_graph(g)
    sv = router.server(plain=True)
    try:
        cost, perm, status, done = sv.run(arr, o.offs, o.picks)
        st = sv.stats()
    finally:
        sv.close()
    ref = router.route_orders(o.offs, o.picks)
    assert (cost == ref[0]).all() and (status == ref[2]).all() and (perm == ref[1][:len(perm)]).all()
    assert st["batches"] == 200 and (done >= arr - 1e-9).all()


def _big_orders(g, ks, seed):
    """Orders of the given sizes, distinct uniform slots each."""
    parts = [synth.uniform_slot_orders(1, int(k), g.n_slots, seed + i) for i, k in enumerate(ks)]
    offs = np.zeros(len(ks) + 1, np.int64)
    offs[1:] = np.cumsum(ks)
    return synth.Orders(offs, np.concatenate([p.picks for p in parts]).astype(np.int32))


def test_route_held_karp_large_orders(wr, orc):
    """Orders of 13..20 picks in a context created with max_k = 20: exact Held-Karp on the
    GPU against the oracle's Held-Karp (cost, first optimal sequence, status), mixed with
    exhaustive orders; the same orders are WR_ORDER_BAD under the default max_k = 12,
    and a captured plan gives the same results."""
    g = synth.medium_layout().build()
    ks = [13, 5, 14, 9, 15, 16, 3, 13, 17, 12, 18, 20, 14, 13, 6, 15]
    o = _big_orders(g, ks, 4242)
    r = wr.Router(device=0, max_k=20)
    try:
        r.load_graph(g)
        cost, perm, status = r.route_orders(o.offs, o.picks)
        plan = r.plan(o.n, int(o.offs[-1]))
        try:
            pc, pp, ps = _plan_run(plan, o.offs, o.picks)
        finally:
            plan.close()
    finally:
        r.close()
    c, p, s = orc.route_orders(g, o, "dijkstra", "heldkarp", NT, max_k=20)
    assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all()
    assert (pc == c).all() and (ps == s).all() and (pp[:len(p)] == p).all()
    assert (s == 0).all()
    r12 = wr.Router(device=0)
    try:
        r12.load_graph(g)
        c12, _, s12 = r12.route_orders(o.offs, o.picks)
    finally:
        r12.close()
    big = np.array(ks) > 12
    assert (s12[big] == 2).all() and (s12[~big] == s[~big]).all() and (c12[~big] == c[~big]).all()


def test_route_held_karp_unreachable_and_range(wr, orc):
    """Held-Karp statuses: an order with an unreachable pick, and one with a leg above
    WR_LEG_MAX, on a small directed graph with heavy arcs."""
    V = 60
    u = np.arange(V - 1, dtype=np.int64)
    w = synth.uniform_int(71, V - 1, 1, 40)
    w[20] = 20_000_000  # legs across this arc exceed WR_LEG_MAX
    rp, col, wt = synth.csr_from_arcs(V, np.concatenate([u, u + 1]), np.concatenate([u + 1, u]),
                                      np.concatenate([w, w]))
    g = synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0)
    # node 59 cut off from the depot: drop its arcs
    keep = (np.repeat(np.arange(V), np.diff(rp)) != 59) & (col != 59)
    src = np.repeat(np.arange(V), np.diff(rp))[keep]
    rp2, col2, wt2 = synth.csr_from_arcs(V, src, col[keep], wt[keep])
    g = synth.Graph(V=V, row_ptr=rp2, col=col2, w=wt2, depot=0)
    offs = np.array([0, 14, 28, 42], np.int64)
    picks = np.concatenate([np.arange(1, 15), np.arange(5, 18), [59], np.arange(10, 24) + 1]).astype(np.int32)
    o = synth.Orders(offs, picks)
    r = wr.Router(device=0, max_k=16)
    try:
        r.load_graph(g)
        cost, perm, status = r.route_orders(o.offs, o.picks)
    finally:
        r.close()
    c, p, s = orc.route_orders(g, o, "dijkstra", "heldkarp", NT, max_k=16)
    assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all()
    assert sorted(s.tolist()) == [0, 1, 3]


def test_route_open_paths(wr, orc):
    """Open paths (the entrance/exit not part of the route): exhaustive and Held-Karp
    orders against the oracle's open mode, directly, through a captured plan and through
    the serving loop (all created after the mode was set)."""
    g, o = synth.medium_workload(n_orders=200)
    big = _big_orders(g, [13, 15, 14], 99)
    offs = np.concatenate([o.offs, o.offs[-1] + big.offs[1:]])
    picks = np.concatenate([o.picks, big.picks]).astype(np.int32)
    ob = synth.Orders(offs, picks)
    r = wr.Router(device=0, max_k=16)
    try:
        r.load_graph(g)
        r.set_route_mode(True)
        cost, perm, status = r.route_orders(ob.offs, ob.picks)
        plan = r.plan(ob.n, int(ob.offs[-1]))
        try:
            pc, pp, ps = _plan_run(plan, ob.offs, ob.picks)
        finally:
            plan.close()
        sv = r.server(max_batch=64, max_batch_picks=1024, n_slots=2, cache_bytes=256 << 20)
        try:
            arr = synth.poisson_arrivals(o.n, 20000.0, 5)
            sc, sp, ss, _ = sv.run(arr, o.offs, o.picks)
        finally:
            sv.close()
    finally:
        r.close()
    c, p, s = orc.route_orders(g, ob, "dijkstra", "heldkarp", NT, max_k=16, open_path=True)
    assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all()
    assert (pc == c).all() and (ps == s).all() and (pp[:len(p)] == p).all()
    n = o.n
    assert (sc == c[:n]).all() and (ss == s[:n]).all() and (sp[:o.offs[-1]] == p[:o.offs[-1]]).all()
    cc, _, _ = orc.route_orders(g, o, "dijkstra", "heldkarp", NT)
    assert (c[:n] <= cc).all() and (c[:n] < cc).any()


def test_route_nodes_against_oracle(wr, orc):
    """Node-level routes (closed tours and open paths, one segment and several) against
    the oracle's walk of the same predecessor rule, element by element; an invalid
    sequence gets no nodes; zero-weight arcs are refused."""
    g, o = synth.medium_workload(n_orders=150)
    for open_path, budget in ((False, 2 << 30), (True, 2 << 30), (False, 64 * g.V * 4)):
        r = wr.Router(device=0, mem_budget_bytes=budget)
        try:
            r.load_graph(g)
            r.set_route_mode(open_path)
            cost, perm, status = r.route_orders(o.offs, o.picks)
            perm = perm[:o.offs[-1]].copy()
            perm[o.offs[5]] = perm[o.offs[5] + 1]  # order 5: not a permutation
            node_offs, nodes = r.route_nodes(o.offs, o.picks, perm)
        finally:
            r.close()
        want_offs, want_nodes = orc.route_nodes(g, o, perm, open_path=open_path, n_threads=NT)
        assert (node_offs == want_offs).all() and (nodes == want_nodes).all(), (open_path, budget)
        assert node_offs[6] == node_offs[5]
    zg = random_graph(50, 150, 7, w_lo=0, w_hi=3)
    r = wr.Router(device=0)
    try:
        r.load_graph(zg)
        with pytest.raises(wr.WrError):
            r.route_nodes(np.array([0, 1], np.int64), np.array([3], np.int32), np.array([0], np.int32))
    finally:
        r.close()


def test_route_nodes_long_legs_several_segments(wr, orc):
    """Node-level routes whose legs outgrow the 256-node leg cache (aisle faces of 300 slots:
    a leg along a face and back along another passes 300 to 600 nodes) mixed with short
    legs, in one segment and in several small ones, closed and open: the cached legs are
    copied and the long ones walked again, element by element against the oracle."""
    lay = synth.Layout(A=3, S=300, F=2, C=2, step_lo=80, step_hi=120, seed=synth.SEED_BASE + 41)
    g = lay.build()
    o = synth.uniform_slot_orders(40, 5, lay.n_slots, synth.SEED_BASE + 42)
    for open_path, budget in ((False, 2 << 30), (False, 32 * g.V * 4), (True, 32 * g.V * 4)):
        r = wr.Router(device=0, mem_budget_bytes=budget)
        try:
            r.load_graph(g)
            r.set_route_mode(open_path)
            cost, perm, status = r.route_orders(o.offs, o.picks)
            perm = np.ascontiguousarray(perm[:o.offs[-1]])
            node_offs, nodes = r.route_nodes(o.offs, o.picks, perm)
        finally:
            r.close()
        want_offs, want_nodes = orc.route_nodes(g, o, perm, open_path=open_path, n_threads=NT)
        assert (node_offs == want_offs).all() and (nodes == want_nodes).all(), (open_path, budget)
        # the batch really holds legs past the cache and legs within it
        leg_lens = []
        for i in range(o.n):
            route = want_nodes[want_offs[i]:want_offs[i + 1]]
            seq = o.picks[o.offs[i] + perm[o.offs[i]:o.offs[i + 1]]]
            stops = list(seq[1:]) if open_path else list(seq) + [g.depot]
            pos = 0
            for t in stops:
                nxt = pos + 1 + int(np.flatnonzero(route[pos + 1:] == t)[0])
                leg_lens.append(nxt - pos)
                pos = nxt
        assert max(leg_lens) > 256 and min(leg_lens) <= 256, (max(leg_lens), min(leg_lens))


def test_route_clustered_against_oracle(wr, orc):
    """Cluster-patched approximate routing (Sec. 3) against the oracle's restatement of
    the same steps, element by element, for closed tours and open paths and several m;
    through a captured plan as well; never cheaper than the exact optimum."""
    lay = synth.medium_layout()
    g, o = synth.medium_workload(n_orders=300)
    xy = lay.coords()
    exact_c, _, _ = orc.route_orders(g, o, "dijkstra", "heldkarp", NT)
    for m, open_path in ((3, False), (3, True), (2, False), (6, True)):
        r = wr.Router(device=0)
        try:
            r.load_graph(g)
            r.set_route_mode(open_path)
            r.set_clusters(m, xy)
            cost, perm, status = r.route_orders(o.offs, o.picks)
            if m == 3 and not open_path:
                plan = r.plan(o.n, int(o.offs[-1]))
                try:
                    pc, pp, ps = _plan_run(plan, o.offs, o.picks)
                finally:
                    plan.close()
                assert (pc == cost).all() and (pp[:o.offs[-1]] == perm[:o.offs[-1]]).all() and (ps == status).all()
        finally:
            r.close()
        c, p, s = orc.route_orders_clustered(g, o, xy, m, open_path, NT)
        assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all(), (m, open_path)
        if not open_path:
            assert (c >= exact_c).all()


@pytest.mark.parametrize("tiling", [1, 2, 3, 4], ids=["warp_sweeps", "cta_sweeps", "warp_worklist", "warp_pairs"])
def test_wait_limit_reports_timeout_and_device_stays_usable(wr, orc, tiling):
    """Failure detection without a GPU fault: with a one-spin wait limit the sweep
    kernel's grid barriers (or worklist waits) give up, every block returns, and the call
    reports WR_ETIMEOUT; a new context on the same device then computes the oracle's rows."""
    g = synth.medium_layout().build()
    src = synth.distinct_sources(64, g.n_slots, 3)
    r = wr.Router(device=0, barrier_max_spins=1)
    try:
        r.set_tuning(bf_tiling=tiling)
        r.load_graph(g)
        with pytest.raises(wr.WrError) as e:
            r.bf_rows(src)
        assert e.value.code == wr.WR_ETIMEOUT
    finally:
        r.close()
    r2 = wr.Router(device=0)
    try:
        r2.set_tuning(bf_tiling=tiling)
        r2.load_graph(g)
        assert (r2.bf_rows(src) == orc.sssp_rows(g, src, "dijkstra", NT)).all()
    finally:
        r2.close()


def test_route_clustered_kmeans_by_hand(wr, orc):
    """The hand-worked k-means cases (tests/golden/kmeans_by_hand.json: Lloyd steps that
    move centres and change assignments, ties, fewer spots than clusters) through the
    GPU's clustered routing: stops at the cases' coordinates on a complete graph of
    seeded asymmetric weights, the picks given in several orders, tours and open paths;
    equal to the oracle element by element."""
    import itertools
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kmeans_by_hand.json")))
    for ci, case in enumerate(gold["cases"]):
        xy_stops = np.array(case["xy"], np.int32)
        k = len(xy_stops)
        V = k + 1  # node k is the depot
        u, v = np.nonzero(~np.eye(V, dtype=bool))
        w = synth.uniform_int(7100 + ci, u.shape[0], 1, 60)
        rp, col, wt = synth.csr_from_arcs(V, u, v, w)
        g = synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=k, n_slots=k)
        xy = np.vstack([xy_stops, [[0, 0]]]).astype(np.int32)
        orders = [list(range(k)), list(range(k))[::-1]] + \
            [list(p) for p in itertools.islice(itertools.permutations(range(k)), 3, 40, 7)]
        offs = np.arange(len(orders) + 1, dtype=np.int64) * k
        o = synth.Orders(offs, np.array(sum(orders, []), np.int32))
        for open_path in (False, True):
            r = wr.Router(device=0)
            try:
                r.load_graph(g)
                r.set_route_mode(open_path)
                r.set_clusters(case["m"], xy)
                cost, perm, status = r.route_orders(o.offs, o.picks)
            finally:
                r.close()
            c, p, s_ = orc.route_orders_clustered(g, o, xy, case["m"], open_path, 1)
            assert (status == s_).all() and (cost == c).all() and (perm[:len(p)] == p).all(), \
                (case["name"], open_path)


def test_load_graph_int32_rule(wr, orc):
    """The int32 distance rule on both sides: graphs whose bound min((V-1) max w, sum w)
    reaches INF are refused by wr_load_graph (WR_EINVAL, context still usable) and by the
    oracle; accepted graphs with distances near 2^31 give the oracle's rows exactly, and
    orders over them the oracle's statuses (legs above WR_LEG_MAX are WR_ORDER_RANGE)."""
    def graph(V, arcs):
        u, v, w = (np.array(x, np.int64) for x in zip(*arcs))
        rp, col, wt = synth.csr_from_arcs(V, u, v, w)
        return synth.Graph(V=V, row_ptr=rp, col=col, w=wt, depot=0, n_slots=V)

    refused = [graph(3, [(0, 1, 1_500_000_000), (1, 2, 1_500_000_000)]), graph(2, [(0, 1, INF)]),
               graph(40, [(i, i + 1, 60_000_000) for i in range(39)])]
    accepted = [graph(3, [(0, 1, 2_000_000_000), (1, 2, 5), (2, 0, 7)]), graph(2, [(0, 1, INF - 1), (1, 0, 3)]),
                graph(4, [(a, b, 500_000_000 + 11 * a + b) for a in range(4) for b in range(4) if a != b]),
                graph(40, [(i, i + 1, 55_000_000) for i in range(39)] + [(39, 0, 1)])]
    r = wr.Router(device=0)
    try:
        for g in refused:
            assert not orc.graph_check(g)
            with pytest.raises(wr.WrError) as e:
                r.load_graph(g)
            assert e.value.code == wr.WR_EINVAL
        for g in accepted:
            assert orc.graph_check(g)
            r.load_graph(g)
            src = np.arange(g.V, dtype=np.int32)
            assert (r.bf_rows(src) == orc.sssp_rows(g, src, "dijkstra")).all()
            ks = [1, 2, min(3, g.V - 1)]
            picks = np.concatenate([np.arange(1, 1 + k) % g.V for k in ks]).astype(np.int32)
            o = synth.Orders(np.concatenate([[0], np.cumsum(ks)]).astype(np.int64), picks)
            cost, perm, status = r.route_orders(o.offs, o.picks)
            c, p, s_ = orc.route_orders(g, o, "dijkstra", "brute")
            assert (status == s_).all() and (cost == c).all() and (perm[:len(p)] == p).all()
    finally:
        r.close()


def test_route_orders_on_scale_layout(wr, orc):
    """Orders on the scale layout (V = 1,002,001): source selection over a graph larger than one
    block's compaction (the three-kernel path), against the oracle."""
    g, _ = synth.scale_workload(n_src=8)
    o = synth.uniform_slot_orders(6, 4, g.n_slots, 77)
    r = wr.Router(device=0)
    try:
        r.load_graph(g)
        cost, perm, status = r.route_orders(o.offs, o.picks)
    finally:
        r.close()
    c, p, s = orc.route_orders(g, o, "dijkstra", "brute", NT)
    assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all()


def test_route_clustered_uneven_orders(wr, orc):
    """Clustered routing of orders of 2..12 picks: with one cluster the orders above ten
    stops are WR_ORDER_BAD on both sides, with four clusters every order is routed; the
    results equal the oracle's element by element."""
    lay = synth.medium_layout()
    g, o = synth.batching_workload(n_orders=400)
    xy = lay.coords()
    assert (o.k() > 10).any()
    for m in (1, 4):
        r = wr.Router(device=0)
        try:
            r.load_graph(g)
            r.set_clusters(m, xy)
            cost, perm, status = r.route_orders(o.offs, o.picks)
        finally:
            r.close()
        c, p, s = orc.route_orders_clustered(g, o, xy, m, False, NT)
        assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all(), m
        if m == 1:
            assert (s[o.k() > 10] == 2).all()


def test_route_held_karp_full_batch_and_small_budget(wr, orc):
    """The large-order workload (128 orders of 13..20 picks) through batched Held-Karp
    against the oracle's Held-Karp; then again under a 64 MiB budget, where the tables
    are solved in many small batches and the rows in several segments: same results."""
    g, o = synth.large_order_workload()
    c, p, s = orc.route_orders(g, o, "dijkstra", "heldkarp", NT, max_k=20)
    assert (s == 0).all()
    for budget in (2 << 30, 64 << 20):
        r = wr.Router(device=0, max_k=20, mem_budget_bytes=budget)
        try:
            r.load_graph(g)
            cost, perm, status = r.route_orders(o.offs, o.picks)
        finally:
            r.close()
        assert (status == s).all() and (cost == c).all() and (perm[:len(p)] == p).all(), budget


def test_route_orders_device_buffers_bad_offsets(wr):
    """wr_route_orders with device buffers whose offsets do not start at 0, or decrease, or
    end below 0: WR_EINVAL, no pick read past the buffer, and the context still routes a
    valid batch afterwards with the same bits as before."""
    import torch
    g, o = synth.medium_workload(n_orders=16)
    dev = torch.device("cuda", 0)
    r = wr.Router(device=0)
    try:
        r.load_graph(g)
        want = r.route_orders(o.offs, o.picks)
        n = 3
        picks = torch.from_numpy(o.picks[:6].copy()).to(dev)  # 6 picks only
        cost = torch.empty(n, dtype=torch.int32, device=dev)
        perm = torch.empty(6, dtype=torch.int32, device=dev)
        status = torch.empty(n, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev).cuda_stream
        for bad in ([4, 6, 8, 10], [0, 2, 4, -1]):
            offs = torch.tensor(bad, dtype=torch.int64, device=dev)
            with pytest.raises(wr.WrError) as e:
                wr.wr_route_orders(r.ctx, offs, picks, cost, perm, status, stream)
            assert e.value.code == wr.WR_EINVAL, bad
        # a decreasing offset is a bad order, not a bad call: the other orders are routed
        offs = torch.tensor([0, 4, 2, 6], dtype=torch.int64, device=dev)
        wr.wr_route_orders(r.ctx, offs, picks, cost, perm, status, stream)
        torch.cuda.synchronize()
        st = status.cpu().numpy()
        assert st[1] == wr.WR_ORDER_BAD and st[0] == wr.WR_ORDER_OK and st[2] == wr.WR_ORDER_OK, st
        again = r.route_orders(o.offs, o.picks)
        for a, b in zip(want, again):
            assert (np.asarray(a) == np.asarray(b)).all()
    finally:
        r.close()


def test_route_nodes_device_buffers_one_call(wr):
    """wr_route_nodes with device buffers and a node buffer sized from a count-only call:
    one call writes the same nodes as the host path; a buffer one node short is ENOMEM."""
    import torch
    g, o = synth.medium_workload(n_orders=64)
    r = wr.Router(device=0)
    try:
        r.load_graph(g)
        _, perm, _ = r.route_orders(o.offs, o.picks)
        perm = np.ascontiguousarray(perm[:o.offs[-1]])
        h_offs, h_nodes = r.route_nodes(o.offs, o.picks, perm)
        dev = torch.device("cuda", 0)
        offs = torch.from_numpy(o.offs).to(dev)
        picks = torch.from_numpy(o.picks).to(dev)
        dperm = torch.from_numpy(perm).to(dev)
        node_offs = torch.zeros(o.n + 1, dtype=torch.int64, device=dev)
        wr.wr_route_nodes(r.ctx, offs, picks, dperm, node_offs, None, 0)
        torch.cuda.synchronize()
        total = int(node_offs[-1].item())
        assert total == len(h_nodes)
        nodes = torch.empty(total, dtype=torch.int32, device=dev)
        wr.wr_route_nodes(r.ctx, offs, picks, dperm, node_offs, nodes, total)
        torch.cuda.synchronize()
        assert (node_offs.cpu().numpy() == h_offs).all() and (nodes.cpu().numpy() == h_nodes).all()
        with pytest.raises(wr.WrError) as e:
            wr.wr_route_nodes(r.ctx, offs, picks, dperm, node_offs, nodes, total - 1)
        assert e.value.code == wr.WR_ENOMEM
    finally:
        r.close()
