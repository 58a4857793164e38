"""The pins catch plausible oracle mistakes.

Each case plants one mistake in a copy of oracle.c (on the CPU, in a
temporary directory), builds it, and checks that at least one pin from
the oracle test files fails against the broken build.
"""
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2504_20655_gb300 import synth
from tests.graphs import path_graph, random_graph

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tours_by_hand.json")))
KMEANS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kmeans_by_hand.json")))

MUTANTS = [
    ("bf dropped weight", "i64 cand = cur[u] + (i64)w[a];", "i64 cand = cur[u];"),
    ("bf extra term", "i64 cand = cur[u] + (i64)w[a];", "i64 cand = cur[u] + (i64)w[a] + 1;"),
    ("bf too few rounds", "for (int32_t r = 0; r < V - 1; ++r) {", "for (int32_t r = 0; r < V / 3; ++r) {"),
    ("bf reversed arcs", "if (cand < nxt[col[a]]) { nxt[col[a]] = cand; changed = 1; }",
     "if (cur[col[a]] < BIG && cur[col[a]] + (i64)w[a] < nxt[u]) { nxt[u] = cur[col[a]] + (i64)w[a]; changed = 1; }"),
    ("tour no return leg", "for (int32_t i = 0; i <= k; ++i) {", "for (int32_t i = 0; i < k; ++i) {"),
    ("tour transposed leg", "int32_t leg = D[prev * n + nx];", "int32_t leg = D[nx * n + prev];"),
    ("tour last minimiser", "if (c < best) { best = c; memcpy(best_p",
     "if (c <= best) { best = c; memcpy(best_p"),
    ("tour off-by-one perm", "for (int32_t i = 0; i < k; ++i) perm[i] = best_p[i] - 1;",
     "for (int32_t i = 0; i < k; ++i) perm[i] = best_p[i];"),
    ("heldkarp largest index", "for (int32_t j = 0; j < k; ++j) {\n            if (S & (1u << j)) continue;\n            i64 l = LEG(cur, j + 1)",
     "for (int32_t j = k - 1; j >= 0; --j) {\n            if (S & (1u << j)) continue;\n            i64 l = LEG(cur, j + 1)"),
    ("heldkarp no return", "if (S == full) { H(S, c) = LEG(c + 1, 0); continue; }",
     "if (S == full) { H(S, c) = 0; continue; }"),
    ("dijkstra no decrease", "if (cand < d[v]) { d[v] = cand; hitem x",
     "if (cand < d[v] && d[v] == BIG) { d[v] = cand; hitem x"),
    ("range limit off", "D[i * n + j] > OR_LEG_MAX", "D[i * n + j] > OR_LEG_MAX + 1"),
    ("patching forward only", "for (uint32_t dir = 0; dir < (1u << M); ++dir) {",
     "for (uint32_t dir = 0; dir < 1u; ++dir) {"),
    ("patching last minimiser", "int better = !have || t < best;", "int better = !have || t <= best;"),
    ("patching no return leg", "t = back >= BIG ? BIG : t + back;", "t = back >= BIG ? BIG : t;"),
    ("kmeans single pass", "while (it < 64) {", "while (it < 1) {"),
    ("kmeans centres never moved", "if (ct > 0) { Sx[c] = sx; Sy[c] = sy; cnt[c] = ct; }",
     "if (ct < 0) { Sx[c] = sx; Sy[c] = sy; cnt[c] = ct; }"),
    ("kmeans mean off by one", "if (ct > 0) { Sx[c] = sx; Sy[c] = sy; cnt[c] = ct; }",
     "if (ct > 0) { Sx[c] = sx; Sy[c] = sy; cnt[c] = ct + 1; }"),
    ("kmeans ties to highest centre", "if (c == 0 || frac_less(num, den, bnum, bden)) {",
     "if (c == 0 || !frac_less(bnum, bden, num, den)) {"),
    ("kmeans farthest tie to highest stop", "if (dmin > best_d) { best_d = dmin; best_i = i; }",
     "if (dmin >= best_d) { best_d = dmin; best_i = i; }"),
    ("int32 rule inclusive bound", "return bound < (i64)OR_INF ? 0 : OR_EDIST;",
     "return bound <= (i64)OR_INF ? 0 : OR_EDIST;"),
    ("int32 rule max term only", "if (sum_w < bound) bound = sum_w;", "(void)sum_w;"),
    ("int32 rule sum term only", "if (sum_w < bound) bound = sum_w;", "bound = sum_w;"),
    ("distance cast at INF", "if (d[i] < BIG && d[i] >= (i64)OR_INF) return 0;",
     "if (d[i] < BIG && d[i] > (i64)OR_INF) return 0;"),
    ("kmeans x only", "i64 num = dx * dx + dy * dy, den = cnt[c] * cnt[c];",
     "i64 num = dx * dx, den = cnt[c] * cnt[c];"),
]


def pins_pass() -> bool:
    """A compact run of the pins in test_oracle_sssp.py / test_oracle_tour.py."""
    try:
        A, S, a, c = 5, 6, 13, 41
        lay = synth.Layout(A=A, S=S, F=1, C=2, step_lo=a, step_hi=a, cross_w=c)
        g = lay.build()
        rows = oracle.sssp_rows(g, np.arange(lay.n_slots), "rounds")
        for p in range(lay.n_slots):
            a1, s1 = divmod(p, S)
            for q in range(lay.n_slots):
                a2, s2 = divmod(q, S)
                exp = abs(s1 - s2) * a if a1 == a2 else \
                    min(s1 + s2 + 2, 2 * S - s1 - s2) * a + abs(a1 - a2) * c
                if rows[p, q] != exp:
                    return False
        pg = path_graph(40, 2)
        d, r = oracle.bf_rounds(pg, 0)
        if r != 39 or (d != 2 * np.arange(40)).any():
            return False
        for seed in range(3):
            rg = random_graph(60, 200, seed + 50, w_lo=1)
            for s in range(0, 60, 11):
                if (oracle.bf_rounds(rg, s)[0] != oracle.dijkstra(rg, s)).any():
                    return False
        for case in GOLD["cases"]:
            D = np.array(case["D"], dtype=np.int32)
            for kind in ("brute", "heldkarp"):
                st, cost, perm = oracle.tour(D, kind)
                if st != case["status"] or cost != case["cost"] or perm.tolist() != case["perm"]:
                    return False
        for k in range(1, 8):
            for seed in range(4):
                n = k + 1
                D = synth.uniform_int(seed + 17 * k, n * n, 0, 9).reshape(n, n).astype(np.int32)
                np.fill_diagonal(D, 0)
                b, h = oracle.tour(D, "brute"), oracle.tour(D, "heldkarp")
                if b[:2] != h[:2] or (b[2] != h[2]).any():
                    return False
        # cluster-patched route: one stop per cluster is exact; pairs patch to the best
        # sequence that keeps every pair together
        import itertools
        for k in (3, 5):
            for seed in range(3):
                n = k + 1
                D = synth.uniform_int(seed + 31 * k, n * n, 1, 3).reshape(n, n).astype(np.int32)  # ties
                np.fill_diagonal(D, 0)
                xy = np.stack([100 * np.arange(k), np.zeros(k, int)], axis=1).astype(np.int32)
                c1, p1 = oracle.tour_clustered(D, xy, k, False)[1:]
                c2, p2 = oracle.tour(D, "brute")[1:]
                if c1 != c2 or p1.tolist() != p2.tolist():
                    return False
        xy = np.array([[0, 0], [1, 0], [200, 0], [201, 0]], np.int32)
        for seed in range(6):
            D = synth.uniform_int(seed + 77, 25, 1, 30 if seed % 2 else 2).reshape(5, 5).astype(np.int32)
            np.fill_diagonal(D, 0)
            best = None
            for p in itertools.permutations(range(4)):
                if abs(p.index(0) - p.index(1)) != 1 or abs(p.index(2) - p.index(3)) != 1:
                    continue
                c = int(D[0, p[0] + 1]) + sum(int(D[a + 1, b + 1]) for a, b in zip(p[:-1], p[1:])) + int(D[p[-1] + 1, 0])
                if best is None or c < best[0]:
                    best = (c, list(p))
            st, c, pm = oracle.tour_clustered(D, xy, 2, False)
            if (c, pm.tolist()) != best:
                return False
        # k-means step: the hand-worked cases and the fixed point of the Lloyd map
        from tests.test_oracle_kmeans import _fixed_point
        for case in KMEANS["cases"]:
            a, sx, sy, cnt, steps = oracle.kmeans(np.array(case["xy"]), case["m"])
            if a.tolist() != case["assign"] or cnt.tolist() != case["cnt"] or sx.tolist() != case["Sx"] \
                    or sy.tolist() != case["Sy"]:
                return False
        for seed in range(20):
            k = 3 + seed % 10
            xy = synth.uniform_int(500 + seed, 2 * k, 0, 12).reshape(k, 2).astype(np.int64)
            if not _fixed_point(xy, 3, *oracle.kmeans(xy, 3)[:4]):
                return False
        # the int32 distance rule and the refusal to cast a distance at or above INF
        from tests.test_oracle_sssp import test_int32_rule_refuses_and_accepts
        test_int32_rule_refuses_and_accepts(oracle)
        D = np.full((5, 5), 7, dtype=np.int32)
        np.fill_diagonal(D, 0)
        D[1, 2] = oracle.LEG_MAX + 1
        if oracle.tour(D, "brute")[0] != oracle.RANGE:
            return False
        return True
    except (Exception, pytest.fail.Exception):  # pytest.raises reports a miss with pytest.fail
        return False


def test_pins_pass_on_the_real_oracle():
    assert pins_pass()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    src = tmp_path / "oracle.c"
    src.write_text(text.replace(old, new))
    (tmp_path / "oracle.h").write_text(open(os.path.join(os.path.dirname(SRC), "oracle.h")).read())
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-w", "-o", str(so), str(src),
                           "-lpthread"])
    with oracle.using(str(so)):
        assert not pins_pass(), f"mutant survived: {name}"
