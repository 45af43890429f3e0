"""Python binding of libgamma (include/gamma.h): argument marshalling only.

The module-level functions carry the C-ABI names and take plain arrays:
numpy arrays (host) or torch tensors (host or CUDA); the library decides
where each pointer lives. Every step of the matching runs in the CUDA
library; if ``_build/libgamma.so`` cannot be loaded, importing the binding
raises instead of falling back to anything else. ``Context`` wraps the same
calls for convenience.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

GAMMA_OK, GAMMA_EINVAL, GAMMA_ENOMEM, GAMMA_ESTATE, GAMMA_EOVERFLOW, GAMMA_ETIMEOUT, GAMMA_ECUDA = (
    0, -1, -2, -3, -4, -5, -6)
GAMMA_F_PER_UPDATE, GAMMA_F_NO_FILTER, GAMMA_F_PER_QUERY, GAMMA_F_GRAPH, GAMMA_F_COUNT_BYTES, GAMMA_F_NO_LEAF = (
    0x1, 0x2, 0x4, 0x8, 0x10, 0x20)
GAMMA_F_NO_SHARE = 0x40
GAMMA_F_SEED_IN_ORDER = 0x80
GAMMA_F_SEED_BY_QUERY = 0x100

_NAMES = {0: "GAMMA_OK", -1: "GAMMA_EINVAL", -2: "GAMMA_ENOMEM", -3: "GAMMA_ESTATE",
          -4: "GAMMA_EOVERFLOW", -5: "GAMMA_ETIMEOUT", -6: "GAMMA_ECUDA"}


class gamma_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("work_budget", ctypes.c_uint64), ("warps_per_block", ctypes.c_int),
                ("frontier_tile", ctypes.c_int), ("steal_grain", ctypes.c_int),
                ("idle_limit_us", ctypes.c_uint32), ("handoff_limit_us", ctypes.c_uint32),
                ("hub_min_degree", ctypes.c_int32)]


class gamma_matches(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_void_p), ("capacity", ctypes.c_int64), ("stride", ctypes.c_int32),
                ("written", ctypes.c_int64), ("required", ctypes.c_int64)]


class gamma_stats(ctypes.Structure):
    _fields_ = [("ms_stage", ctypes.c_double), ("ms_seed", ctypes.c_double), ("ms_match", ctypes.c_double),
                ("ms_finalize", ctypes.c_double), ("ms_commit", ctypes.c_double), ("seeds", ctypes.c_int64),
                ("work_items", ctypes.c_int64), ("touched", ctypes.c_int64), ("pool_used", ctypes.c_int64),
                ("pool_cap", ctypes.c_int64), ("live_edges", ctypes.c_int64), ("expansions", ctypes.c_uint64),
                ("alg_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("graph_captures", ctypes.c_int64), ("donated_tasks", ctypes.c_int64)]


class gamma_server_options(ctypes.Structure):
    _fields_ = [("max_updates", ctypes.c_int64), ("max_requests", ctypes.c_int32), ("hbm_fraction", ctypes.c_double)]


class gamma_request_info(ctypes.Structure):
    _fields_ = [("arrival_ms", ctypes.c_double), ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("group_size", ctypes.c_int32), ("status", ctypes.c_int32)]


class gamma_server_stats(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int64), ("requests", ctypes.c_int64), ("updates", ctypes.c_int64),
                ("max_group", ctypes.c_int64), ("busy_ms", ctypes.c_double)]


class gamma_tune_point(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("frontier_tile", ctypes.c_int32),
                ("steal_grain", ctypes.c_int32), ("ms", ctypes.c_float)]


class GammaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (_NAMES.get(code, str(code)), msg))
        self.code = code


_P = ctypes.c_void_p
_SIGS = {
    "gamma_create": (ctypes.c_int, [ctypes.POINTER(gamma_options), ctypes.POINTER(ctypes.c_void_p)]),
    "gamma_destroy": (None, [_P]),
    "gamma_load_graph": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P]),
    "gamma_load_graph_el": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P]),
    "gamma_register_query_el": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P, _P]),
    "gamma_apply_batch_el": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int32, _P, _P, _P, _P]),
    "gamma_register_query": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "gamma_apply_batch": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, ctypes.c_int32, _P, _P, _P,
                                         ctypes.POINTER(gamma_matches)]),
    "gamma_apply_batches": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, _P, _P, _P]),
    "gamma_fetch_matches": (ctypes.c_int, [_P, ctypes.POINTER(gamma_matches)]),
    "gamma_update_counts": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "gamma_commit": (ctypes.c_int, [_P]),
    "gamma_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(gamma_stats)]),
    "gamma_export_adjacency": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64]),
    "gamma_reserve_vertices": (ctypes.c_int, [_P, ctypes.c_int32]),
    "gamma_plan_order": (ctypes.c_int, [ctypes.c_int32, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, _P, _P, _P]),
    "gamma_checkpoint": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "gamma_restore": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "gamma_add_vertices": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int32)]),
    "gamma_vertex_neighbors": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "gamma_set_options": (ctypes.c_int, [_P, ctypes.POINTER(gamma_options)]),
    "gamma_last_error": (ctypes.c_char_p, [_P]),
    "gamma_recount_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "gamma_probe_bandwidth": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P]),
    "gamma_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(gamma_tune_point), ctypes.c_int32,
                                      ctypes.POINTER(gamma_tune_point)]),
    "gamma_server_start": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(gamma_server_options),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "gamma_server_submit": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "gamma_server_wait": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(gamma_request_info)]),
    "gamma_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(gamma_server_stats)]),
    "gamma_server_stop": (ctypes.c_int, [_P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libgamma.so (building it first if needed); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libgamma.so is not built (%s); run paper_2401_17018_gb300.build" % _build.LIB)
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _as(a, dtype):
    if hasattr(a, "data_ptr"):
        import torch
        want = {np.int8: torch.int8, np.int32: torch.int32}[dtype]
        return a.to(want).contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def _check(ctx, rc: int):
    if rc != GAMMA_OK:
        msg = load_library().gamma_last_error(ctx) if ctx else b""
        raise GammaError(rc, (msg or b"").decode())


# ----------------------------------------------------------- C-ABI names
def gamma_create(options: Optional[gamma_options] = None) -> int:
    lib = load_library()
    out = ctypes.c_void_p()
    rc = lib.gamma_create(ctypes.byref(options) if options is not None else None, ctypes.byref(out))
    if rc != GAMMA_OK:
        raise GammaError(rc, "gamma_create failed")
    return out.value


def gamma_destroy(ctx: int) -> None:
    load_library().gamma_destroy(ctx)


def gamma_load_graph(ctx: int, n: int, labels, src, dst, elabels=None) -> None:
    """elabels (one per edge): an edge-labelled graph (gamma_load_graph_el)."""
    labels, src, dst = _as(labels, np.int32), _as(src, np.int32), _as(dst, np.int32)
    if elabels is None:
        _check(ctx, load_library().gamma_load_graph(ctx, int(n), _ptr(labels), int(src.shape[0]), _ptr(src),
                                                    _ptr(dst)))
    else:
        el = _as(elabels, np.int32)
        _check(ctx, load_library().gamma_load_graph_el(ctx, int(n), _ptr(labels), int(src.shape[0]), _ptr(src),
                                                       _ptr(dst), _ptr(el)))


def gamma_register_query(ctx: int, labels, src, dst, elabels=None) -> int:
    """elabels (one per query edge): edge labels (gamma_register_query_el)."""
    labels, src, dst = _as(labels, np.int32), _as(src, np.int32), _as(dst, np.int32)
    qid = ctypes.c_int32(-1)
    if elabels is None:
        _check(ctx, load_library().gamma_register_query(ctx, int(labels.shape[0]), _ptr(labels), int(src.shape[0]),
                                                        _ptr(src), _ptr(dst), ctypes.byref(qid)))
    else:
        el = np.ascontiguousarray(elabels, dtype=np.int32)
        _check(ctx, load_library().gamma_register_query_el(ctx, int(labels.shape[0]), _ptr(labels),
                                                           int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(el),
                                                           ctypes.byref(qid)))
    return qid.value


def gamma_apply_batch(ctx: int, op, src, dst, qids: Sequence[int], matches: Optional[gamma_matches] = None,
                      elab=None) -> Tuple[np.ndarray, np.ndarray, int]:
    """Returns (pos counts, neg counts, rc); rc is GAMMA_OK or GAMMA_EOVERFLOW
    (other codes raise).  elab: insertion labels (gamma_apply_batch_el)."""
    op, src, dst = _as(op, np.int8), _as(src, np.int32), _as(dst, np.int32)
    q = np.ascontiguousarray(qids, dtype=np.int32)
    pos = np.zeros(max(q.size, 1), np.uint64)
    neg = np.zeros(max(q.size, 1), np.uint64)
    mref = ctypes.byref(matches) if matches is not None else None
    if elab is None:
        rc = load_library().gamma_apply_batch(ctx, int(op.shape[0]), _ptr(op), _ptr(src), _ptr(dst), int(q.size),
                                              _ptr(q), _ptr(pos), _ptr(neg), mref)
    else:
        el = _as(elab, np.int32)
        rc = load_library().gamma_apply_batch_el(ctx, int(op.shape[0]), _ptr(op), _ptr(src), _ptr(dst), _ptr(el),
                                                 int(q.size), _ptr(q), _ptr(pos), _ptr(neg), mref)
    if rc not in (GAMMA_OK, GAMMA_EOVERFLOW):
        _check(ctx, rc)
    return pos[:q.size], neg[:q.size], rc


def gamma_load_graph_el(ctx: int, n: int, labels, src, dst, elabels) -> None:
    gamma_load_graph(ctx, n, labels, src, dst, elabels)


def gamma_register_query_el(ctx: int, labels, src, dst, elabels) -> int:
    return gamma_register_query(ctx, labels, src, dst, elabels)


def gamma_apply_batch_el(ctx: int, op, src, dst, elab, qids: Sequence[int],
                         matches: Optional[gamma_matches] = None) -> Tuple[np.ndarray, np.ndarray, int]:
    return gamma_apply_batch(ctx, op, src, dst, qids, matches, elab)


def gamma_apply_batches(ctx: int, req_off, op, src, dst, qids: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
    """Several requests staged together; returns (pos, neg) of shape [nreq, nq]."""
    off = np.ascontiguousarray(req_off, dtype=np.int64)
    nreq = off.size - 1
    op, src, dst = _as(op, np.int8), _as(src, np.int32), _as(dst, np.int32)
    q = np.ascontiguousarray(qids, dtype=np.int32)
    pos = np.zeros(max(nreq * q.size, 1), np.uint64)
    neg = np.zeros(max(nreq * q.size, 1), np.uint64)
    _check(ctx, load_library().gamma_apply_batches(ctx, nreq, _ptr(off), _ptr(op), _ptr(src), _ptr(dst), int(q.size),
                                                   _ptr(q), _ptr(pos), _ptr(neg)))
    return pos[:nreq * q.size].reshape(nreq, q.size), neg[:nreq * q.size].reshape(nreq, q.size)


def gamma_fetch_matches(ctx: int, matches: gamma_matches) -> int:
    rc = load_library().gamma_fetch_matches(ctx, ctypes.byref(matches))
    if rc not in (GAMMA_OK, GAMMA_EOVERFLOW):
        _check(ctx, rc)
    return rc


def gamma_update_counts(ctx: int, j: int, b: int) -> np.ndarray:
    out = np.zeros(max(b, 1), np.uint64)
    _check(ctx, load_library().gamma_update_counts(ctx, int(j), _ptr(out)))
    return out[:b]


def gamma_commit(ctx: int) -> None:
    _check(ctx, load_library().gamma_commit(ctx))


def gamma_get_stats(ctx: int) -> dict:
    st = gamma_stats()
    _check(ctx, load_library().gamma_get_stats(ctx, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in gamma_stats._fields_}


def gamma_export_adjacency(ctx: int, n: int, cap: int):
    """(off[n+1], nbr, tag) of the current (union) adjacency."""
    off = np.zeros(n + 1, np.int64)
    nbr = np.zeros(max(cap, 1), np.int32)
    tag = np.zeros(max(cap, 1), np.int32)
    _check(ctx, load_library().gamma_export_adjacency(ctx, _ptr(off), _ptr(nbr), _ptr(tag), int(cap)))
    return off, nbr[:off[-1]], tag[:off[-1]]


def gamma_checkpoint(ctx: int) -> bytes:
    """The committed graph and registered queries as bytes."""
    lib = load_library()
    need = ctypes.c_int64(0)
    rc = lib.gamma_checkpoint(ctx, None, 0, ctypes.byref(need))
    if rc not in (GAMMA_OK, GAMMA_EOVERFLOW):
        _check(ctx, rc)
    buf = np.zeros(max(int(need.value), 1), np.uint8)
    _check(ctx, lib.gamma_checkpoint(ctx, _ptr(buf), int(need.value), ctypes.byref(need)))
    return buf[:need.value].tobytes()


def gamma_restore(ctx: int, data: bytes) -> None:
    buf = np.frombuffer(data, np.uint8).copy()
    _check(ctx, load_library().gamma_restore(ctx, _ptr(buf), int(buf.size)))


def gamma_plan_order(labels, src, dst, a: int, b: int, label_freq=None):
    """(order, backward masks) of the matching order for seeded query edge (a, b); no GPU needed."""
    lab = _as(labels, np.int32)
    s = _as(src, np.int32)
    d = _as(dst, np.int32)
    freq = None if label_freq is None else np.ascontiguousarray(label_freq, np.int64)
    order = np.zeros(len(lab), np.int32)
    bwd = np.zeros(len(lab), np.uint16)
    rc = load_library().gamma_plan_order(int(len(lab)), _ptr(lab), int(len(s)), _ptr(s), _ptr(d), int(a), int(b),
                                         0 if freq is None else int(freq.size), _ptr(freq), _ptr(order), _ptr(bwd))
    if rc != GAMMA_OK:
        raise GammaError(rc, "gamma_plan_order: invalid query or seeded edge")
    return order, bwd


def gamma_reserve_vertices(ctx: int, n_max: int) -> None:
    _check(ctx, load_library().gamma_reserve_vertices(ctx, int(n_max)))


def gamma_add_vertices(ctx: int, labels) -> int:
    """Append len(labels) isolated vertices; returns the first new id."""
    lab = _as(labels, np.int32)
    first = ctypes.c_int32(0)
    _check(ctx, load_library().gamma_add_vertices(ctx, int(len(lab)), _ptr(lab), ctypes.byref(first)))
    return first.value


def gamma_vertex_neighbors(ctx: int, v: int, cap: int = 1024) -> np.ndarray:
    """Ids of v's current neighbours."""
    lib = load_library()
    while True:
        out = np.zeros(max(cap, 1), np.int32)
        cnt = ctypes.c_int64(0)
        rc = lib.gamma_vertex_neighbors(ctx, int(v), _ptr(out), int(cap), ctypes.byref(cnt))
        if rc == GAMMA_EOVERFLOW:
            cap = int(cnt.value)
            continue
        _check(ctx, rc)
        return out[:cnt.value]


def gamma_set_options(ctx: int, options: gamma_options) -> None:
    _check(ctx, load_library().gamma_set_options(ctx, ctypes.byref(options)))


def gamma_last_error(ctx: int) -> str:
    return (load_library().gamma_last_error(ctx) or b"").decode()


# ----------------------------------------------------------- convenience
def make_options(device: int = 0, stream=None, flags: int = 0, work_budget: int = 0, warps_per_block: int = 0,
                 frontier_tile: int = 0, steal_grain: int = 0, idle_limit_us: int = 0,
                 handoff_limit_us: int = 0, hub_min_degree: int = 0) -> gamma_options:
    s = stream
    if s is not None and hasattr(s, "cuda_stream"):
        s = s.cuda_stream
    return gamma_options(device, s, flags, work_budget, warps_per_block, frontier_tile, steal_grain, idle_limit_us,
                         handoff_limit_us, hub_min_degree)


class Context:
    """One libgamma context (see include/gamma.h for the state machine)."""

    def __init__(self, device: int = 0, stream=None, flags: int = 0, work_budget: int = 0,
                 warps_per_block: int = 0, frontier_tile: int = 0, steal_grain: int = 0, idle_limit_us: int = 0,
                 handoff_limit_us: int = 0, hub_min_degree: int = 0):
        self._opts = make_options(device, stream, flags, work_budget, warps_per_block, frontier_tile, steal_grain,
                                  idle_limit_us, handoff_limit_us, hub_min_degree)
        self.h = gamma_create(self._opts)
        self.b = 0
        self.qsizes = {}

    def close(self):
        if self.h:
            gamma_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        for k, v in kw.items():
            if k == "stream" and v is not None and hasattr(v, "cuda_stream"):
                v = v.cuda_stream
            setattr(self._opts, "cuda_stream" if k == "stream" else k, v)
        gamma_set_options(self.h, self._opts)

    def load_graph(self, n, labels, src, dst, elabels=None):
        gamma_load_graph(self.h, n, labels, src, dst, elabels)
        self.qsizes = {}

    def register_query(self, labels, src, dst, elabels=None) -> int:
        qid = gamma_register_query(self.h, labels, src, dst, elabels)
        self.qsizes[qid] = int(len(labels))
        return qid

    def apply_batch(self, op, src, dst, qids: Sequence[int], row_capacity: Optional[int] = None,
                    rows=None, elab=None):
        """Apply a batch. With row_capacity (host rows) or rows (a preallocated
        int32 buffer, host or device, shape [capacity, stride]) the match rows
        are returned too: (pos, neg, rows_written, required)."""
        self.b = int(op.shape[0])
        m = None
        buf = None
        if rows is not None or row_capacity is not None:
            stride = 3 + max([self.qsizes.get(int(q), 2) for q in qids] + [2])
            if rows is None:
                buf = np.full((max(int(row_capacity), 1), stride), -1, np.int32)
            else:
                buf = rows
                stride = int(buf.shape[1])
            m = gamma_matches(_ptr(buf), int(buf.shape[0]) if row_capacity is None else int(row_capacity), stride, 0, 0)
        pos, neg, rc = gamma_apply_batch(self.h, op, src, dst, qids, m, elab)
        if m is None:
            return pos, neg
        return pos, neg, buf[:m.written], m.required

    def apply_batches(self, req_off, op, src, dst, qids: Sequence[int]):
        self.b = int(op.shape[0])
        return gamma_apply_batches(self.h, req_off, op, src, dst, qids)

    def fetch_matches(self, rows):
        m = gamma_matches(_ptr(rows), int(rows.shape[0]), int(rows.shape[1]), 0, 0)
        gamma_fetch_matches(self.h, m)
        return rows[:m.written], m.required

    def update_counts(self, j: int) -> np.ndarray:
        return gamma_update_counts(self.h, j, self.b)

    def commit(self):
        gamma_commit(self.h)

    def stats(self) -> dict:
        return gamma_get_stats(self.h)

    def export_adjacency(self, n: int):
        st = self.stats()
        return gamma_export_adjacency(self.h, n, int(st["pool_used"]))

    def reserve_vertices(self, n_max: int):
        gamma_reserve_vertices(self.h, n_max)

    def checkpoint(self) -> bytes:
        return gamma_checkpoint(self.h)

    def restore(self, data: bytes):
        gamma_restore(self.h, data)
        # the query sizes, for the row stride of later applies (queries keep their ids)
        w = np.frombuffer(data, np.int32)
        n = int(w[2])
        m = int(np.frombuffer(data[16:24], np.int64)[0])
        k = 6 + n + 2 * m
        self.qsizes = {}
        for j in range(int(w[k])):
            q, eq = int(w[k + 1]), int(w[k + 2])
            self.qsizes[j] = q
            k += 2 + q + 2 * eq

    def add_vertices(self, labels) -> int:
        return gamma_add_vertices(self.h, labels)

    def vertex_neighbors(self, v: int) -> np.ndarray:
        return gamma_vertex_neighbors(self.h, v)


def gamma_autotune(ctx: int, grid, repeats: int = 1):
    """Sweep (warps_per_block, frontier_tile, steal_grain) points on the staged
    batch; returns (best point as a dict, list of every point with its ms)."""
    pts = (gamma_tune_point * len(grid))(*[gamma_tune_point(w, t, g, 0.0) for w, t, g in grid])
    best = gamma_tune_point()
    _check(ctx, load_library().gamma_autotune(ctx, len(grid), pts, int(repeats), ctypes.byref(best)))
    as_dict = lambda p: {k: getattr(p, k) for k, _ in gamma_tune_point._fields_}
    return as_dict(best), [as_dict(p) for p in pts]


def gamma_recount_noalloc(ctx: int, nslots: int) -> Tuple[np.ndarray, np.ndarray]:
    """Counts of the staged batch recomputed without allocating (see gamma.h):
    nslots = requests x queries of the staged batch.  The output arrays are
    sized for the library's 256-slot limit and their size is passed along,
    so a wrong nslots cannot make the library write past them."""
    cap = 256
    pos = np.zeros(cap, np.uint64)
    neg = np.zeros(cap, np.uint64)
    _check(ctx, load_library().gamma_recount_noalloc(ctx, cap, _ptr(pos), _ptr(neg)))
    return pos[:nslots], neg[:nslots]


def gamma_probe_bandwidth(device: int, nbytes: int, reps: int = 8, trials: int = 5) -> float:
    """Read bandwidth (GB/s) for a working set of nbytes (see gamma.h)."""
    out = ctypes.c_double(0.0)
    rc = load_library().gamma_probe_bandwidth(int(device), int(nbytes), int(reps), int(trials), ctypes.byref(out))
    if rc != GAMMA_OK:
        raise GammaError(rc, "gamma_probe_bandwidth failed")
    return out.value


# ----------------------------------------------------------- served form
def gamma_server_start(ctx: int, qids: Sequence[int], options: Optional[gamma_server_options] = None) -> int:
    q = np.ascontiguousarray(qids, dtype=np.int32)
    out = ctypes.c_void_p()
    rc = load_library().gamma_server_start(ctx, int(q.size), _ptr(q), ctypes.byref(options) if options else None,
                                           ctypes.byref(out))
    if rc != GAMMA_OK:
        raise GammaError(rc, "gamma_server_start failed")
    return out.value


def gamma_server_submit(srv: int, op, src, dst) -> int:
    op, src, dst = _as(op, np.int8), _as(src, np.int32), _as(dst, np.int32)
    t = ctypes.c_int64(-1)
    rc = load_library().gamma_server_submit(srv, int(op.shape[0]), _ptr(op), _ptr(src), _ptr(dst), ctypes.byref(t))
    if rc != GAMMA_OK:
        raise GammaError(rc, "gamma_server_submit failed")
    return t.value


def gamma_server_wait(srv: int, ticket: int, nq: int):
    """(status, pos[nq], neg[nq], info dict) of one finished request."""
    pos = np.zeros(max(nq, 1), np.uint64)
    neg = np.zeros(max(nq, 1), np.uint64)
    info = gamma_request_info()
    rc = load_library().gamma_server_wait(srv, int(ticket), _ptr(pos), _ptr(neg), ctypes.byref(info))
    return rc, pos[:nq], neg[:nq], {k: getattr(info, k) for k, _ in gamma_request_info._fields_}


def gamma_server_stats_get(srv: int) -> dict:
    st = gamma_server_stats()
    load_library().gamma_server_stats_get(srv, ctypes.byref(st))
    return {k: getattr(st, k) for k, _ in gamma_server_stats._fields_}


def gamma_server_stop(srv: int) -> None:
    load_library().gamma_server_stop(srv)


class Server:
    """Served form on a Context: submit requests, wait for their counts."""

    def __init__(self, ctx: Context, qids: Sequence[int], max_updates: int = 0, max_requests: int = 0,
                 hbm_fraction: float = 0.0):
        self.nq = len(qids)
        self.h = gamma_server_start(ctx.h, qids, gamma_server_options(max_updates, max_requests, hbm_fraction))

    def submit(self, op, src, dst) -> int:
        return gamma_server_submit(self.h, op, src, dst)

    def wait(self, ticket: int):
        return gamma_server_wait(self.h, ticket, self.nq)

    def stats(self) -> dict:
        return gamma_server_stats_get(self.h)

    def stop(self):
        if self.h:
            gamma_server_stop(self.h)
            self.h = None
