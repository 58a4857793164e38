"""Seeded synthetic inputs: warehouse aisle layouts and order batches.

This module only draws inputs. It holds none of the routing arithmetic
(no shortest paths, no tour costs), so both the CUDA path and the CPU
oracle can consume its output without sharing any of the method.

The paper's experiments (Sec. 4, Sec. 5 settings lists) use synthetic
rack lattices; the layouts here are synthetic stand-ins of that shape:
parallel aisles of slots, cross-aisles joining the aisles, one depot.

Randomness is a counter-based splitmix64 (Steele, Lea and Flood, 2014):
value i of stream s is mix64(s + (i + 1) * 0x9E3779B97F4A7C15), so every
draw is addressed by (stream, index) and results do not depend on the
order in which they are generated.  Each stream id is xor-ed into the
base seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 2504

# stream ids (xor-ed into the base seed)
STREAM_WEIGHTS = 1
STREAM_ONEWAY = 2
STREAM_SKUMAP = 3
STREAM_ORDER_K = 4
STREAM_ORDER_PICKS = 5
STREAM_ARRIVALS = 6
STREAM_RELOCATE = 7
STREAM_SOURCES = 8
STREAM_FACE = 9


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Values offset .. offset+n-1 of the splitmix64 stream keyed by seed."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_int(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """n integers in [lo, hi] (inclusive), multiply-shift on the top 32 bits."""
    span = np.uint64(hi - lo + 1)
    r = splitmix64(seed, n, offset) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return (np.int64(lo) + ((r * span) >> np.uint64(32)).astype(np.int64))


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits."""
    r = splitmix64(seed, n, offset) >> np.uint64(11)
    return r.astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------------------
# layouts
# ---------------------------------------------------------------------------

@dataclass
class Graph:
    """Directed graph in out-arc CSR form with int32 weights."""
    V: int
    row_ptr: np.ndarray  # int64[V+1]
    col: np.ndarray      # int32[E]
    w: np.ndarray        # int32[E]
    depot: int
    n_slots: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(self.col.shape[0])

    def arcs(self):
        """(u, v, w) arrays of all arcs."""
        u = np.repeat(np.arange(self.V, dtype=np.int32), np.diff(self.row_ptr))
        return u, self.col, self.w


def csr_from_arcs(V: int, u: np.ndarray, v: np.ndarray, w: np.ndarray) -> tuple:
    """Out-arc CSR, arcs sorted by (u, v)."""
    order = np.lexsort((v, u))
    u, v, w = u[order], v[order], w[order]
    row_ptr = np.zeros(V + 1, dtype=np.int64)
    np.add.at(row_ptr, u.astype(np.int64) + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, v.astype(np.int32), w.astype(np.int32)


@dataclass
class Layout:
    """Parallel-aisle warehouse.

    A aisles, S slot positions per aisle, F faces per position (two sides
    of an aisle, or two levels), C cross-aisles.  Slot node id(a, f, s) =
    (a*F + f)*S + s keeps consecutive slots of one aisle face at
    consecutive ids.  Cross-aisle node X(a, j) = A*F*S + j*A + a sits at
    boundary b_j = round(j*S/(C-1)) of aisle a (b_0 = 0 before the first
    slot, b_{C-1} = S after the last); numbering each cross-aisle along
    the aisles keeps it a run of consecutive ids too.  The depot is the
    last node and links to X(0, 0).

    Undirected edges:
      * chain of each (a, f): its slots in s order with X(a, j) inserted
        before slot b_j (after the last slot when b_j = S); weight
        U[step_lo, step_hi] per edge;
      * face links (a, f, s)-(a, f+1, s): U[step_lo, step_hi] when
        face_w is None (two sides of one aisle), else face_w (levels);
      * cross links X(a, j)-X(a+1, j): cross_w;
      * depot-X(0, 0): depot_w.
    A seeded fraction oneway_frac of the aisles keeps only the direction
    of increasing chain position on its chain arcs (one-way aisles).
    """
    A: int
    S: int
    F: int = 2
    C: int = 2
    step_lo: int = 80
    step_hi: int = 120
    face_w: int | None = None
    cross_w: int = 300
    depot_w: int = 300
    oneway_frac: float = 0.0
    seed: int = SEED_BASE

    @property
    def n_slots(self) -> int:
        return self.A * self.F * self.S

    @property
    def V(self) -> int:
        return self.A * self.F * self.S + self.A * self.C + 1

    def slot(self, a, f, s):
        return (np.asarray(a) * self.F + np.asarray(f)) * self.S + np.asarray(s)

    def xnode(self, a, j):
        return self.A * self.F * self.S + np.asarray(j) * self.A + np.asarray(a)

    @property
    def depot(self) -> int:
        return self.V - 1

    def boundaries(self) -> list[int]:
        if self.C < 2:
            raise ValueError("need at least two cross-aisles")
        d = 2 * (self.C - 1)
        return [(2 * j * self.S + (self.C - 1)) // d for j in range(self.C)]

    def oneway_aisles(self) -> np.ndarray:
        n = int(round(self.oneway_frac * self.A))
        if n == 0:
            return np.zeros(0, dtype=np.int64)
        key = splitmix64(self.seed ^ STREAM_ONEWAY, self.A)
        return np.sort(np.argsort(key, kind="stable")[:n])

    def chain_sequence(self) -> np.ndarray:
        """Node ids along one chain, for aisle 0 face 0, as offsets.

        Returned as (kind, index) pairs: kind 0 = slot s, kind 1 = X j.
        """
        b = self.boundaries()
        seq = []
        for s in range(self.S + 1):
            for j in range(self.C):
                if b[j] == s:
                    seq.append((1, j))
            if s < self.S:
                seq.append((0, s))
        return np.array(seq, dtype=np.int64)

    def coords(self) -> np.ndarray:
        """(V, 2) int32 plan coordinates: slot (a, f, s) at (a, s) -- both faces of a
        position share it --, cross-aisle node X(a, j) at (a, b_j) with the boundaries on
        the slot scale shifted by half a slot (2 b_j - 1 on a doubled scale), the depot
        next to X(0, 0).  Positions are doubled so every coordinate is an integer."""
        A, S, F, C = self.A, self.S, self.F, self.C
        xy = np.zeros((self.V, 2), dtype=np.int32)
        a = np.arange(A)[:, None, None]
        s = np.arange(S)[None, None, :]
        f = np.arange(F)[None, :, None]
        ids = ((a * F + f) * S + s).reshape(-1)
        xy[ids, 0] = np.broadcast_to(2 * a, (A, F, S)).reshape(-1)
        xy[ids, 1] = np.broadcast_to(2 * s, (A, F, S)).reshape(-1)
        b = np.array(self.boundaries())
        for j in range(C):
            xid = self.xnode(np.arange(A), j)
            xy[xid, 0] = 2 * np.arange(A)
            xy[xid, 1] = 2 * b[j] - 1
        xy[self.depot] = (0, -3)
        return xy

    def build(self) -> Graph:
        A, S, F, C = self.A, self.S, self.F, self.C
        seq = self.chain_sequence()                       # [S+C, 2]
        L = seq.shape[0]
        a = np.arange(A, dtype=np.int64)[:, None, None]
        f = np.arange(F, dtype=np.int64)[None, :, None]
        kind = seq[:, 0][None, None, :]
        idx = seq[:, 1][None, None, :]
        nodes = np.where(kind == 0, (a * F + f) * S + idx, A * F * S + idx * A + a)  # [A,F,L]
        cu = nodes[:, :, :-1].reshape(-1)
        cv = nodes[:, :, 1:].reshape(-1)
        n_chain = cu.shape[0]
        chain_aisle = np.broadcast_to(a, (A, F, L - 1)).reshape(-1)

        fu = []
        fv = []
        for ff in range(F - 1):
            s = np.arange(S, dtype=np.int64)
            fu.append(((np.arange(A)[:, None] * F + ff) * S + s[None, :]).reshape(-1))
            fv.append(((np.arange(A)[:, None] * F + ff + 1) * S + s[None, :]).reshape(-1))
        fu = np.concatenate(fu) if fu else np.zeros(0, np.int64)
        fv = np.concatenate(fv) if fv else np.zeros(0, np.int64)

        xa = np.arange(A - 1, dtype=np.int64)[:, None]
        xj = np.arange(C, dtype=np.int64)[None, :]
        xu = (A * F * S + xj * A + xa).reshape(-1)
        xv = (A * F * S + xj * A + xa + 1).reshape(-1)

        depot = self.V - 1
        ws = self.seed ^ STREAM_WEIGHTS
        w_chain = uniform_int(ws, n_chain, self.step_lo, self.step_hi, 0)
        if self.face_w is None:
            w_face = uniform_int(ws, fu.shape[0], self.step_lo, self.step_hi, n_chain)
        else:
            w_face = np.full(fu.shape[0], self.face_w, dtype=np.int64)
        w_x = np.full(xu.shape[0], self.cross_w, dtype=np.int64)

        oneway = np.zeros(A, dtype=bool)
        oneway[self.oneway_aisles()] = True
        chain_both = ~oneway[chain_aisle]

        x00 = A * F * S
        U = [cu, cv[chain_both], fu, fv, xu, xv, np.array([depot, x00])]
        Vv = [cv, cu[chain_both], fv, fu, xv, xu, np.array([x00, depot])]
        W = [w_chain, w_chain[chain_both], w_face, w_face, w_x, w_x,
             np.array([self.depot_w, self.depot_w], dtype=np.int64)]
        u = np.concatenate(U).astype(np.int64)
        v = np.concatenate(Vv).astype(np.int64)
        w = np.concatenate(W).astype(np.int64)
        row_ptr, col, wt = csr_from_arcs(self.V, u, v, w)
        n_und = n_chain + fu.shape[0] + xu.shape[0] + 1
        return Graph(V=self.V, row_ptr=row_ptr, col=col, w=wt, depot=depot,
                     n_slots=self.n_slots,
                     meta=dict(A=A, S=S, F=F, C=C, undirected_edges=int(n_und),
                               oneway_aisles=int(oneway.sum()), seed=self.seed))


# ---------------------------------------------------------------------------
# orders
# ---------------------------------------------------------------------------

@dataclass
class Orders:
    """A batch of orders: picks[offs[i]:offs[i+1]] are order i's pick nodes."""
    offs: np.ndarray   # int64[n+1]
    picks: np.ndarray  # int32[offs[n]]

    @property
    def n(self) -> int:
        return int(self.offs.shape[0] - 1)

    def k(self) -> np.ndarray:
        return np.diff(self.offs).astype(np.int64)

    def order(self, i: int) -> np.ndarray:
        return self.picks[self.offs[i]:self.offs[i + 1]]

    def subset(self, idx) -> "Orders":
        idx = np.asarray(idx, dtype=np.int64)
        ks = self.k()[idx]
        offs = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        offs[1:] = np.cumsum(ks)
        picks = np.concatenate([self.order(int(i)) for i in idx]) if idx.size else np.zeros(0, np.int32)
        return Orders(offs, picks.astype(np.int32))


def zipf_cdf(n_items: int, s: float) -> np.ndarray:
    """CDF of P(rank r) proportional to r^-s over ranks 1..n_items."""
    p = np.arange(1, n_items + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(p)
    return c / c[-1]


def sku_slot_map(n_sku: int, n_slots: int, seed: int) -> np.ndarray:
    """Uniform seeded assignment SKU -> slot (several SKUs may share a slot)."""
    return uniform_int(seed ^ STREAM_SKUMAP, n_sku, 0, n_slots - 1).astype(np.int32)


def _first_distinct(draws: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Per row, the first k[i] distinct entries of draws[i] (row-major output)."""
    n, m = draws.shape
    dup = np.zeros((n, m), dtype=bool)
    for j in range(1, m):
        dup[:, j] = (draws[:, :j] == draws[:, j:j + 1]).any(axis=1)
    keep = ~dup
    rank = np.cumsum(keep, axis=1)
    sel = keep & (rank <= k[:, None])
    if not (sel.sum(axis=1) == k).all():
        raise RuntimeError("not enough distinct draws; raise the draw width")
    return draws[sel]


def zipf_orders(n_orders: int, k: np.ndarray, sku_to_slot: np.ndarray, s: float,
                seed: int, width: int = 48) -> Orders:
    """Orders whose picks are distinct SKUs drawn by inverse CDF from Zipf(s)."""
    k = np.asarray(k, dtype=np.int64)
    cdf = zipf_cdf(sku_to_slot.shape[0], s)
    u = uniform01(seed ^ STREAM_ORDER_PICKS, n_orders * width).reshape(n_orders, width)
    sku = np.minimum(np.searchsorted(cdf, u, side="right"), cdf.shape[0] - 1)
    chosen = _first_distinct(sku, k)
    offs = np.zeros(n_orders + 1, dtype=np.int64)
    offs[1:] = np.cumsum(k)
    return Orders(offs, sku_to_slot[chosen].astype(np.int32))


def uniform_k(n_orders: int, lo: int, hi: int, seed: int) -> np.ndarray:
    return uniform_int(seed ^ STREAM_ORDER_K, n_orders, lo, hi)


def geometric_k(n_orders: int, p: float, k_min: int, k_max: int, seed: int,
                width: int = 64) -> np.ndarray:
    """k = k_min + Geom(p) failures, redrawn (next counter) while k > k_max."""
    u = uniform01(seed ^ STREAM_ORDER_K, n_orders * width).reshape(n_orders, width)
    u = np.maximum(u, 1e-300)
    f = np.floor(np.log(u) / np.log1p(-p)).astype(np.int64)
    k = k_min + f
    ok = k <= k_max
    first = np.argmax(ok, axis=1)
    if not ok.any(axis=1).all():
        raise RuntimeError("geometric draw width too small")
    return k[np.arange(n_orders), first]


def uniform_slot_orders(n_orders: int, k: int, n_slots: int, seed: int) -> Orders:
    draws = uniform_int(seed ^ STREAM_ORDER_PICKS, n_orders * 4 * k, 0, n_slots - 1)
    draws = draws.reshape(n_orders, 4 * k)
    kk = np.full(n_orders, k, dtype=np.int64)
    chosen = _first_distinct(draws, kk)
    offs = np.arange(n_orders + 1, dtype=np.int64) * k
    return Orders(offs, chosen.astype(np.int32))


def distinct_sources(n: int, n_slots: int, seed: int) -> np.ndarray:
    """n distinct slot ids, uniform, seeded."""
    key = splitmix64(seed ^ STREAM_SOURCES, n_slots)
    return np.sort(np.argsort(key, kind="stable")[:n]).astype(np.int32)


def poisson_arrivals(n: int, rate: float, seed: int, offset: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    u = uniform01(seed ^ STREAM_ARRIVALS, n, offset)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)


def relocate_top(sku_to_slot: np.ndarray, frac: float, n_slots: int, seed: int, epoch: int) -> np.ndarray:
    """Move the top frac of SKUs (by popularity rank) to new uniform slots."""
    m = int(round(frac * sku_to_slot.shape[0]))
    out = sku_to_slot.copy()
    out[:m] = uniform_int(seed ^ STREAM_RELOCATE, m, 0, n_slots - 1, offset=epoch * m).astype(np.int32)
    return out


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def tiny_layout(seed: int = SEED_BASE) -> Layout:
    return Layout(A=10, S=20, F=2, C=2, step_lo=80, step_hi=120, seed=seed)


def medium_layout(seed: int = SEED_BASE) -> Layout:
    return Layout(A=100, S=100, F=2, C=4, step_lo=80, step_hi=120, oneway_frac=0.1, seed=seed)


def scale_layout(seed: int = SEED_BASE) -> Layout:
    return Layout(A=1000, S=500, F=2, C=2, step_lo=50, step_hi=150, face_w=400, seed=seed)


def serve_layout(seed: int = SEED_BASE) -> Layout:
    return Layout(A=200, S=200, F=2, C=4, step_lo=80, step_hi=120, seed=seed)


def tiny_workload(seed: int = SEED_BASE):
    lay = tiny_layout(seed)
    g = lay.build()
    orders = uniform_slot_orders(1, 6, lay.n_slots, seed)
    return g, orders


def medium_workload(seed: int = SEED_BASE, n_orders: int = 1024, n_sku: int = 50_000):
    lay = medium_layout(seed)
    g = lay.build()
    smap = sku_slot_map(n_sku, lay.n_slots, seed)
    k = uniform_k(n_orders, 4, 10, seed)
    return g, zipf_orders(n_orders, k, smap, 1.1, seed)


def batching_workload(seed: int = SEED_BASE, n_orders: int = 20_000, n_sku: int = 50_000):
    lay = medium_layout(seed)
    g = lay.build()
    smap = sku_slot_map(n_sku, lay.n_slots, seed)
    k = geometric_k(n_orders, 0.3, 2, 12, seed)
    return g, zipf_orders(n_orders, k, smap, 1.1, seed)


def large_order_workload(seed: int = SEED_BASE, n_orders: int = 128, k_lo: int = 13, k_hi: int = 20,
                         n_sku: int = 50_000):
    """Medium layout; orders of k ~ U{k_lo..k_hi} distinct Zipf(1.1) picks: orders too large
    for exhaustive enumeration, routed exactly by Held-Karp."""
    lay = medium_layout(seed)
    g = lay.build()
    smap = sku_slot_map(n_sku, lay.n_slots, seed)
    k = uniform_k(n_orders, k_lo, k_hi, seed)
    return g, zipf_orders(n_orders, k, smap, 1.1, seed, width=160)


def serving_workload(n: int, rate: float, seed: int = SEED_BASE, epoch: int = 100_000):
    """Orders of the serving workload: 200 x 200 x 2-side layout, k = 2 + Geometric(0.3)
    failures (<= 12), Zipf(1.1) picks over 50,000 SKUs whose top 5% move to new slots
    every `epoch` orders (a seeded relocation); Poisson arrivals at `rate` orders/s.
    Returns (layout, orders, arrival times, relocations in the stream)."""
    lay = serve_layout(seed)
    smap = sku_slot_map(50_000, lay.n_slots, seed)
    k = geometric_k(n, 0.3, 2, 12, seed)
    parts, e = [], 0
    for lo in range(0, n, epoch):
        hi = min(n, lo + epoch)
        if lo > 0:
            e += 1
            smap = relocate_top(smap, 0.05, lay.n_slots, seed, e)
        parts.append(zipf_orders(hi - lo, k[lo:hi], smap, 1.1, seed + e))
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum(k)
    picks = np.concatenate([p.picks for p in parts]).astype(np.int32) if parts else np.zeros(0, np.int32)
    return lay, Orders(offs, picks), poisson_arrivals(n, rate, seed), e


def scale_workload(seed: int = SEED_BASE, n_src: int = 4096):
    lay = scale_layout(seed)
    g = lay.build()
    return g, distinct_sources(n_src, lay.n_slots, seed)
