"""Python binding of libwroute.so (include/wroute.h).

Argument marshalling only: every step of the routing path runs in the
library's CUDA kernels.  Functions keep the C names (wr_create,
wr_load_graph, wr_route_orders, ...); `Router` wraps a context for
convenience.  Arrays may be numpy arrays or torch tensors; CUDA tensors
are passed as device pointers (WR_DEVICE) on torch's current stream, host
arrays as WR_HOST.  There is no fallback: without the compiled library
every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwroute.so")

WR_OK, WR_EINVAL, WR_ENOMEM, WR_ECUDA, WR_ETIMEOUT, WR_ENOGRAPH, WR_EINTERNAL = range(7)
WR_ORDER_OK, WR_ORDER_UNREACHABLE, WR_ORDER_BAD, WR_ORDER_RANGE = range(4)
WR_HOST, WR_DEVICE = 0, 1
WR_MAX_K = 12
WR_INF = 2**31 - 1
WR_LEG_MAX = 10324440
DSTRIDE = 13

EXPORTS = ["wr_create", "wr_destroy", "wr_strerror", "wr_sync", "wr_load_graph", "wr_route_orders", "wr_bf_rows",
           "wr_distance_rows", "wr_submatrix", "wr_tour_eval", "wr_tour_eval_static", "wr_get_stats",
           "wr_get_tuning", "wr_set_tuning", "wr_set_trace", "wr_get_trace", "wr_autotune", "wr_set_route_mode", "wr_route_nodes", "wr_set_clusters",
           "wr_set_node_coords",
           "wr_serve_create", "wr_serve_run", "wr_serve_get_stats", "wr_serve_destroy",
           "wr_plan_create", "wr_plan_launch", "wr_plan_sync", "wr_plan_get_stats", "wr_plan_destroy"]
WR_STATIC_MAX_ORDERS = 4096


class wr_serve_config(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("max_batch_picks", ctypes.c_int64), ("n_slots", ctypes.c_int32),
                ("cache_bytes", ctypes.c_uint64), ("plain", ctypes.c_int32)]


class wr_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("orders", "batches", "cache_hits", "rows_computed", "evicted_groups",
                                              "bf_launches")] + [("wall_s", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class wr_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64), ("max_k", ctypes.c_int),
                ("barrier_max_spins", ctypes.c_uint64), ("tune_path", ctypes.c_char_p)]


class wr_tuning(ctypes.Structure):
    _fields_ = [("run_target", ctypes.c_int32), ("tile_cap", ctypes.c_int32), ("enum_units", ctypes.c_int32),
                ("enum_max_units_per_launch", ctypes.c_int32), ("bf_warps", ctypes.c_int32),
                ("bf_tiling", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class wr_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_orders", "n_sources", "n_segments", "sweeps", "tile_visits",
                                              "node_visits", "bytes_alg", "sequences", "kernel_launches")] + \
               [(n, ctypes.c_float) for n in ("ms_select", "ms_init", "ms_bf", "ms_gather", "ms_enum", "ms_finish",
                                              "ms_total")] + [("bytes_reread", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


CONSUME_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                              ctypes.c_int64)

_lib = None


class WrError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


def load_library(path: str = LIB_PATH):
    """Load libwroute.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libwroute.so not built at {path}; run paper_2504_20655_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, I, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64
    L.wr_create.argtypes = [ctypes.POINTER(wr_config), ctypes.POINTER(P)]
    L.wr_destroy.argtypes = [P]
    L.wr_destroy.restype = None
    L.wr_strerror.argtypes = [I]
    L.wr_strerror.restype = ctypes.c_char_p
    L.wr_sync.argtypes = [P]
    L.wr_load_graph.argtypes = [P, i32, i64, P, P, P, i32, I]
    L.wr_route_orders.argtypes = [P, i32, P, P, P, P, P, I, P]
    L.wr_bf_rows.argtypes = [P, i32, P, P, i64, I, P]
    L.wr_distance_rows.argtypes = [P, i32, P, I, CONSUME_FN, P, P]
    L.wr_submatrix.argtypes = [P, i32, P, i32, P, P, P, I, P]
    L.wr_tour_eval.argtypes = [P, i32, P, P, P, P, P, I, P]
    L.wr_tour_eval_static.argtypes = [i32, P, P, P, P, P, P]
    L.wr_get_stats.argtypes = [P, ctypes.POINTER(wr_stats)]
    L.wr_get_tuning.argtypes = [P, ctypes.POINTER(wr_tuning)]
    L.wr_set_tuning.argtypes = [P, ctypes.POINTER(wr_tuning)]
    L.wr_plan_create.argtypes = [P, i32, i64, P, P, P, P, P, ctypes.POINTER(P)]
    L.wr_plan_launch.argtypes = [P, P]
    L.wr_plan_sync.argtypes = [P]
    L.wr_plan_get_stats.argtypes = [P, ctypes.POINTER(wr_stats)]
    L.wr_plan_destroy.argtypes = [P]
    L.wr_plan_destroy.restype = None
    L.wr_autotune.argtypes = [P, i32, P, P, I, i32, ctypes.POINTER(wr_tuning)]
    L.wr_set_route_mode.argtypes = [P, I]
    L.wr_set_clusters.argtypes = [P, i32]
    L.wr_set_node_coords.argtypes = [P, P, I]
    L.wr_route_nodes.argtypes = [P, i32, P, P, P, P, P, i64, I, P]
    L.wr_serve_create.argtypes = [P, ctypes.POINTER(wr_serve_config), ctypes.POINTER(P)]
    L.wr_serve_run.argtypes = [P, i32, P, P, P, P, P, P, P]
    L.wr_serve_get_stats.argtypes = [P, ctypes.POINTER(wr_serve_stats)]
    L.wr_serve_destroy.argtypes = [P]
    L.wr_serve_destroy.restype = None
    L.wr_set_trace.argtypes = [P, i32]
    L.wr_get_trace.argtypes = [P, P, i32, ctypes.POINTER(ctypes.c_int32)]
    for name in EXPORTS:
        if name not in ("wr_destroy", "wr_strerror"):
            getattr(L, name).restype = I
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return load_library().wr_strerror(int(code)).decode()
    except ImportError:
        return f"error {code}"


def _check(rc, what):
    if rc != WR_OK:
        raise WrError(rc, what)


# ---------------------------------------------------------------------------
# argument marshalling
# ---------------------------------------------------------------------------

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, kind, keepalive) of an array-like; numpy/CPU arrays are made contiguous."""
    if x is None:
        return None, WR_HOST, None
    if _is_torch(x):
        import torch
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.int64}[dtype]
        if x.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (WR_DEVICE if x.is_cuda else WR_HOST), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, WR_HOST, a


def _stream(s):
    if s is not None:
        return int(s)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("mix of host and device arrays")
    return ks.pop() if ks else WR_HOST


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------

def wr_create(device=0, mem_budget_bytes=2 << 30, max_k=WR_MAX_K, barrier_max_spins=0, tune_path=None):
    L = load_library()
    cfg = wr_config(int(device), int(mem_budget_bytes), int(max_k), int(barrier_max_spins),
                    None if tune_path is None else os.fsencode(tune_path))
    ctx = ctypes.c_void_p()
    _check(L.wr_create(ctypes.byref(cfg), ctypes.byref(ctx)), "wr_create")
    return ctx


def wr_destroy(ctx):
    load_library().wr_destroy(ctx)


def wr_sync(ctx):
    _check(load_library().wr_sync(ctx), "wr_sync")


def wr_load_graph(ctx, V, row_ptr, col, w, depot):
    p_rp, k1, a1 = _ptr(row_ptr, np.int64)
    p_c, k2, a2 = _ptr(col, np.int32)
    p_w, k3, a3 = _ptr(w, np.int32)
    E = int(len(col))
    _check(load_library().wr_load_graph(ctx, int(V), E, p_rp, p_c, p_w, int(depot), _kind(k1, k2, k3)),
           "wr_load_graph")


def wr_route_orders(ctx, offs, picks, cost, perm, status, stream=None):
    n = int(len(offs)) - 1
    po, k1, a1 = _ptr(offs, np.int64)
    pp, k2, a2 = _ptr(picks, np.int32)
    pc, k3, a3 = _ptr(cost, np.int32)
    pm, k4, a4 = _ptr(perm, np.int32)
    ps, k5, a5 = _ptr(status, np.int32)
    for x, a in ((cost, a3), (perm, a4), (status, a5)):
        if isinstance(x, np.ndarray) and a is not x:
            raise ValueError("output numpy arrays must be contiguous int32")
    _check(load_library().wr_route_orders(ctx, n, po, pp, pc, pm, ps, _kind(k1, k2, k3, k4, k5), _stream(stream)),
           "wr_route_orders")


def wr_route_nodes(ctx, offs, picks, perm, node_offs, nodes=None, max_nodes=0, stream=None):
    """Node-level routes into caller buffers (numpy or torch, all host or all device):
    node_offs (n+1) always, nodes (max_nodes) unless None (count only)."""
    n = int(len(offs)) - 1
    po, k1, a1 = _ptr(offs, np.int64)
    pp, k2, a2 = _ptr(picks, np.int32)
    pm, k3, a3 = _ptr(perm, np.int32)
    pn, k4, a4 = _ptr(node_offs, np.int64)
    pd, k5, a5 = _ptr(nodes, np.int32)
    for x, a in ((node_offs, a4), (nodes, a5)):
        if isinstance(x, np.ndarray) and a is not x:
            raise ValueError("output numpy arrays must be contiguous")
    kinds = (k1, k2, k3, k4) + ((k5,) if nodes is not None else ())
    c = ctypes.c_void_p
    _check(load_library().wr_route_nodes(ctx, n, c(po), c(pp), c(pm), c(pn), c(pd) if pd else None,
                                         int(max_nodes), _kind(*kinds), _stream(stream)), "wr_route_nodes")


def wr_bf_rows(ctx, src, rows, ld, stream=None):
    p_s, k1, a1 = _ptr(src, np.int32)
    p_r, k2, a2 = _ptr(rows, np.int32)
    if isinstance(rows, np.ndarray) and a2 is not rows:
        raise ValueError("rows must be a contiguous int32 array")
    _check(load_library().wr_bf_rows(ctx, int(len(src)), p_s, p_r, int(ld), _kind(k1, k2), _stream(stream)),
           "wr_bf_rows")


def wr_distance_rows(ctx, src, consume, stream=None):
    """consume(first, count, dev_ptr, ld) -> int, called once per source segment."""
    p_s, k1, a1 = _ptr(src, np.int32)
    errors = []

    def cb(user, first, count, ptr, ld):
        try:
            return int(consume(int(first), int(count), int(ptr or 0), int(ld)) or 0)
        except Exception as e:  # noqa: BLE001 -- reported after the call
            errors.append(e)
            return -1

    fn = CONSUME_FN(cb)
    rc = load_library().wr_distance_rows(ctx, int(len(src)), p_s, k1, fn, None, _stream(stream))
    if errors:
        raise errors[0]
    if rc != WR_OK:
        raise WrError(rc, "wr_distance_rows")


def wr_submatrix(ctx, src, dst, sub, check, stream=None):
    p_s, k1, a1 = _ptr(src, np.int32)
    p_d, k2, a2 = _ptr(dst, np.int32)
    p_sub, k3, a3 = _ptr(sub, np.int32)
    p_chk, k4, a4 = _ptr(check, np.uint64)
    _check(load_library().wr_submatrix(ctx, int(len(src)), p_s, int(len(dst)), p_d, p_sub, p_chk,
                                       _kind(k1, k2, k3, k4), _stream(stream)), "wr_submatrix")


def wr_tour_eval(ctx, k, D, cost, perm, status, stream=None):
    n = int(len(k))
    p_k, k1, a1 = _ptr(k, np.int32)
    p_D, k2, a2 = _ptr(D, np.int32)
    p_c, k3, a3 = _ptr(cost, np.int32)
    p_p, k4, a4 = _ptr(perm, np.int32)
    p_s, k5, a5 = _ptr(status, np.int32)
    _check(load_library().wr_tour_eval(ctx, n, p_k, p_D, p_c, p_p, p_s, _kind(k1, k2, k3, k4, k5),
                                       _stream(stream)), "wr_tour_eval")


def wr_tour_eval_static(k, D, cost, perm, status, stream=None):
    """wr_tour_eval without a context and without allocating device memory
    (for callers whose device memory belongs to another allocator, or that
    cannot take cudaMalloc's synchronisation).  Device tensors only; uses
    the static scratch of the current device (at most WR_STATIC_MAX_ORDERS
    orders; calls that overlap on the GPU race on that scratch)."""
    n = int(len(k))
    ptrs = []
    for x, dt in ((k, np.int32), (D, np.int32), (cost, np.int32), (perm, np.int32), (status, np.int32)):
        p, kind, _ = _ptr(x, dt)
        if kind != WR_DEVICE:
            raise ValueError("wr_tour_eval_static takes device tensors only")
        ptrs.append(p)
    _check(load_library().wr_tour_eval_static(n, *ptrs, _stream(stream)), "wr_tour_eval_static")


def wr_get_stats(ctx) -> dict:
    st = wr_stats()
    _check(load_library().wr_get_stats(ctx, ctypes.byref(st)), "wr_get_stats")
    return st.as_dict()


def wr_get_tuning(ctx) -> dict:
    t = wr_tuning()
    _check(load_library().wr_get_tuning(ctx, ctypes.byref(t)), "wr_get_tuning")
    return t.as_dict()


def wr_set_tuning(ctx, **kw):
    t = wr_tuning()
    _check(load_library().wr_get_tuning(ctx, ctypes.byref(t)), "wr_get_tuning")
    for key, val in kw.items():
        setattr(t, key, int(val))
    _check(load_library().wr_set_tuning(ctx, ctypes.byref(t)), "wr_set_tuning")


def wr_autotune(ctx, offs, picks, reps=2) -> dict:
    """Pick and apply the fastest tuning for this batch (host or device arrays)."""
    po, kind_o, keep_o = _ptr(offs, np.int64)
    pp, kind_p, keep_p = _ptr(picks, np.int32)
    if kind_o != kind_p:
        raise ValueError("offs and picks must both be host or both device arrays")
    t = wr_tuning()
    _check(load_library().wr_autotune(ctx, len(offs) - 1, po, pp, kind_o, int(reps), ctypes.byref(t)), "wr_autotune")
    del keep_o, keep_p
    return t.as_dict()


def wr_set_trace(ctx, max_sweeps: int):
    _check(load_library().wr_set_trace(ctx, int(max_sweeps)), "wr_set_trace")


def wr_get_trace(ctx, max_entries: int = 1 << 16) -> np.ndarray:
    """[(frontier tiles, start ns), ...] per sweep of the last segment, then (0, end ns)."""
    out = np.zeros((max_entries, 2), dtype=np.int64)
    n = ctypes.c_int32(0)
    _check(load_library().wr_get_trace(ctx, out.ctypes.data_as(ctypes.c_void_p), max_entries, ctypes.byref(n)),
           "wr_get_trace")
    return out[:min(n.value, max_entries)].copy()


class Server:
    """A serving loop (wr_serve_*) over the context's graph: orders arrive over time,
    results come back with their completion times."""

    def __init__(self, ctx, max_batch=256, max_batch_picks=4096, n_slots=3, cache_bytes=4 << 30, plain=False):
        cfg = wr_serve_config(int(max_batch), int(max_batch_picks), int(n_slots), int(cache_bytes), int(bool(plain)))
        h = ctypes.c_void_p()
        _check(load_library().wr_serve_create(ctx, ctypes.byref(cfg), ctypes.byref(h)), "wr_serve_create")
        self.h = h

    def run(self, arrival_s, offs, picks):
        """Returns (cost, perm, status, done_s) for orders arriving at arrival_s (seconds)."""
        arrival = np.ascontiguousarray(arrival_s, dtype=np.float64)
        offs = np.ascontiguousarray(offs, dtype=np.int64)
        picks = np.ascontiguousarray(picks, dtype=np.int32)
        n = len(offs) - 1
        cost = np.empty(n, np.int32)
        status = np.empty(n, np.int32)
        perm = np.empty(max(int(offs[-1]), 1), np.int32)
        done = np.empty(n, np.float64)
        c = ctypes.c_void_p
        _check(load_library().wr_serve_run(self.h, n, c(arrival.ctypes.data), c(offs.ctypes.data), c(picks.ctypes.data),
                                           c(cost.ctypes.data), c(perm.ctypes.data), c(status.ctypes.data),
                                           c(done.ctypes.data)), "wr_serve_run")
        return cost, perm, status, done

    def stats(self) -> dict:
        st = wr_serve_stats()
        _check(load_library().wr_serve_get_stats(self.h, ctypes.byref(st)), "wr_serve_get_stats")
        return st.as_dict()

    def close(self):
        if self.h is not None:
            load_library().wr_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A batch of n_orders orders captured into a CUDA graph (wr_plan_*).

    The plan owns device tensors offs (n+1), picks (max_picks), cost, perm,
    status; fill offs/picks (set_batch), launch, then read the outputs."""

    def __init__(self, ctx, n_orders: int, max_picks: int, device=0):
        import torch
        dev = torch.device("cuda", device)
        self.n = int(n_orders)
        self.max_picks = int(max_picks)
        self.offs = torch.zeros(self.n + 1, dtype=torch.int64, device=dev)
        self.picks = torch.zeros(max(self.max_picks, 1), dtype=torch.int32, device=dev)
        self.cost = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.perm = torch.empty(max(self.max_picks, 1), dtype=torch.int32, device=dev)
        self.status = torch.empty(self.n, dtype=torch.int32, device=dev)
        torch.cuda.synchronize(dev)
        h = ctypes.c_void_p()
        _check(load_library().wr_plan_create(ctx, self.n, self.max_picks, self.offs.data_ptr(), self.picks.data_ptr(),
                                             self.cost.data_ptr(), self.perm.data_ptr(), self.status.data_ptr(),
                                             ctypes.byref(h)), "wr_plan_create")
        self.h = h

    def set_batch(self, offs, picks):
        """Copy a batch (numpy or torch) in; shorter batches are padded with empty orders."""
        import torch
        offs = torch.as_tensor(np.asarray(offs, dtype=np.int64) if not _is_torch(offs) else offs)
        picks = torch.as_tensor(np.asarray(picks, dtype=np.int32) if not _is_torch(picks) else picks)
        n = offs.shape[0] - 1
        if n > self.n or int(offs[-1]) > self.max_picks:
            raise ValueError("batch larger than the plan")
        self.offs[: n + 1].copy_(offs)
        self.offs[n + 1:].fill_(int(offs[-1]))
        if picks.shape[0]:
            self.picks[: picks.shape[0]].copy_(picks)

    def launch(self, stream=None):
        _check(load_library().wr_plan_launch(self.h, _stream(stream)), "wr_plan_launch")

    def sync(self):
        _check(load_library().wr_plan_sync(self.h), "wr_plan_sync")

    def stats(self) -> dict:
        st = wr_stats()
        _check(load_library().wr_plan_get_stats(self.h, ctypes.byref(st)), "wr_plan_get_stats")
        return st.as_dict()

    def close(self):
        if self.h is not None:
            load_library().wr_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Router:
    """One library context on one device."""

    def __init__(self, device=0, mem_budget_bytes=2 << 30, max_k=WR_MAX_K, barrier_max_spins=0, tune_path=None):
        self.ctx = wr_create(device, mem_budget_bytes, max_k, barrier_max_spins, tune_path)
        self.device = device
        self.V = None

    def close(self):
        if self.ctx is not None:
            wr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def load_graph(self, g):
        wr_load_graph(self.ctx, g.V, g.row_ptr, g.col, g.w, g.depot)
        self.V = g.V

    def route_orders(self, offs, picks, out=None, stream=None):
        """Returns (cost, perm, status) as arrays of the inputs' kind (numpy or torch)."""
        n = len(offs) - 1
        if out is None:
            if _is_torch(offs):
                import torch
                dev = offs.device
                np_ = int(offs[-1].item())
                out = (torch.empty(n, dtype=torch.int32, device=dev),
                       torch.empty(max(np_, 1), dtype=torch.int32, device=dev),
                       torch.empty(n, dtype=torch.int32, device=dev))
            else:
                np_ = int(offs[-1])
                out = (np.empty(n, np.int32), np.empty(max(np_, 1), np.int32), np.empty(n, np.int32))
        wr_route_orders(self.ctx, offs, picks, out[0], out[1], out[2], stream)
        return out

    def bf_rows(self, src, stream=None):
        src = np.ascontiguousarray(src, dtype=np.int32) if not _is_torch(src) else src
        if _is_torch(src) and src.is_cuda:
            import torch
            rows = torch.empty((len(src), self.V), dtype=torch.int32, device=src.device)
        else:
            rows = np.empty((len(src), self.V), dtype=np.int32)
        wr_bf_rows(self.ctx, src, rows, self.V, stream)
        return rows

    def tour_eval(self, k, D, stream=None):
        n = len(k)
        cost = np.empty(n, np.int32)
        perm = np.empty(n * WR_MAX_K, np.int32)
        status = np.empty(n, np.int32)
        wr_tour_eval(self.ctx, k, D, cost, perm, status, stream)
        return cost, perm.reshape(n, WR_MAX_K), status

    def submatrix(self, src, dst, stream=None):
        sub = np.empty((len(src), len(dst)), np.int32)
        check = np.empty(len(src), np.uint64)
        wr_submatrix(self.ctx, src, dst, sub, check, stream)
        return sub, check

    def stats(self):
        return wr_get_stats(self.ctx)

    def tuning(self):
        return wr_get_tuning(self.ctx)

    def autotune(self, offs, picks, reps=2):
        return wr_autotune(self.ctx, offs, picks, reps)

    def server(self, **kw):
        return Server(self.ctx, **kw)

    def plan(self, n_orders, max_picks):
        return Plan(self.ctx, n_orders, max_picks, self.device)

    def route_nodes(self, offs, picks, perm, stream=None):
        """Node-level routes of host orders and sequences: (node_offs, nodes)."""
        offs = np.ascontiguousarray(offs, dtype=np.int64)
        picks = np.ascontiguousarray(picks, dtype=np.int32)
        perm = np.ascontiguousarray(perm[: int(offs[-1])], dtype=np.int32)
        n = len(offs) - 1
        node_offs = np.zeros(n + 1, np.int64)
        c = ctypes.c_void_p
        L = load_library()
        _check(L.wr_route_nodes(self.ctx, n, c(offs.ctypes.data), c(picks.ctypes.data), c(perm.ctypes.data),
                                c(node_offs.ctypes.data), None, 0, WR_HOST, _stream(stream)), "wr_route_nodes")
        nodes = np.zeros(max(int(node_offs[-1]), 1), np.int32)
        _check(L.wr_route_nodes(self.ctx, n, c(offs.ctypes.data), c(picks.ctypes.data), c(perm.ctypes.data),
                                c(node_offs.ctypes.data), c(nodes.ctypes.data), int(node_offs[-1]), WR_HOST,
                                _stream(stream)), "wr_route_nodes")
        return node_offs, nodes[: int(node_offs[-1])]

    def set_clusters(self, m: int, coords=None):
        """Cluster-patched approximate routing with at most m clusters (0: exact); coords is
        the (V, 2) int32 plan coordinate array of the loaded graph's nodes."""
        if coords is not None:
            xy = np.ascontiguousarray(coords, dtype=np.int32)
            _check(load_library().wr_set_node_coords(self.ctx, xy.ctypes.data_as(ctypes.c_void_p), WR_HOST),
                   "wr_set_node_coords")
        _check(load_library().wr_set_clusters(self.ctx, int(m)), "wr_set_clusters")

    def set_route_mode(self, open_path: bool):
        """Closed tours through the depot (False, the default) or open paths through the picks (True)."""
        _check(load_library().wr_set_route_mode(self.ctx, 1 if open_path else 0), "wr_set_route_mode")

    def set_trace(self, max_sweeps):
        wr_set_trace(self.ctx, max_sweeps)

    def trace(self):
        return wr_get_trace(self.ctx)

    def set_tuning(self, **kw):
        wr_set_tuning(self.ctx, **kw)

    def sync(self):
        wr_sync(self.ctx)
