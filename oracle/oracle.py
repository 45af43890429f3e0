"""CPU oracle for batch-dynamic subgraph matching -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the library never does. It shares no code with the CUDA path: the
only import from the package is the seeded input generator module, which
holds no matching arithmetic.

Two independent programs compute the same thing, the plain definition of the
incremental matches of a batch (Sec. II-A, Def. 1, Def. 2, Problem Statement):

* ``bdsm`` (O2) calls ``bdsm_oracle.c``: per update, per query edge, per
  orientation, a backtracking search in the view of the update's sign
  (G' for insertions, G for deletions) that refuses image edges which are
  same-sign updates of smaller index, so each match is charged once, to its
  lowest-indexed update (Sec. IV-C, total order over updates).
* ``brute_bdsm`` (O1, pure Python, tiny inputs): enumerate Emb(Q, G) and
  Emb(Q, G') by trying every data vertex for every query vertex, take the two
  set differences, and charge each match to its lowest-indexed update.

Readings of points the paper leaves open are those listed in the oracle's C
header (batch validity) and: matches are embeddings (automorphic images are
distinct results); edges are undirected, so an update is tried in both
orientations on every query edge.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Dict, Iterable, List, Optional, Sequence, Set, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "bdsm_oracle.c")

OK, EINVAL, EBUDGET, ENOMEM = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags, no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        lib.oracle_bdsm.restype = ctypes.c_int
        lib.oracle_bdsm.argtypes = [
            ctypes.c_int32, p, ctypes.c_int64, p, p,
            ctypes.c_int32, p, ctypes.c_int32, p, p,
            ctypes.c_int64, p, p, p,
            ctypes.c_int64, p, p,
            p, ctypes.c_int64, p,
            ctypes.c_uint64, p]
        lib.oracle_bdsm_multi.restype = ctypes.c_int
        lib.oracle_bdsm_multi.argtypes = [
            ctypes.c_int32, p, ctypes.c_int64, p, p,
            ctypes.c_int32, p, p, p, p, p, p, p,
            ctypes.c_int64, p, p, p,
            ctypes.c_int64, p, p,
            p, ctypes.c_int64, p,
            ctypes.c_uint64, ctypes.c_uint64, p]
        lib.oracle_session_open.restype = ctypes.c_int
        lib.oracle_session_open.argtypes = [
            ctypes.c_int32, p, ctypes.c_int64, p, p, p,
            ctypes.c_int64, p, p, p, p, ctypes.POINTER(ctypes.c_void_p), p]
        lib.oracle_session_eval.restype = ctypes.c_int
        lib.oracle_session_eval.argtypes = [
            p, ctypes.c_int32, p, p, p, p, p, p, p, p,
            ctypes.c_int64, p, p, p, ctypes.c_int64, p,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_session_close.restype = None
        lib.oracle_session_close.argtypes = [p]
        lib.oracle_bdsm_multi_el.restype = ctypes.c_int
        lib.oracle_bdsm_multi_el.argtypes = [
            ctypes.c_int32, p, ctypes.c_int64, p, p, p,
            ctypes.c_int32, p, p, p, p, p, p, p, p,
            ctypes.c_int64, p, p, p, p,
            ctypes.c_int64, p, p,
            p, ctypes.c_int64, p,
            ctypes.c_uint64, ctypes.c_uint64, p]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, bad_index: int):
        super().__init__("oracle error %d (bad update index %d)" % (code, bad_index))
        self.code = code
        self.bad_index = bad_index


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _edge_labelled(elabels, queries, batch) -> bool:
    return (elabels is not None or getattr(batch, "elab", None) is not None or
            any(getattr(q, "elabels", None) is not None for q in queries))


def bdsm(n: int, labels, src, dst, query, batch, eval_idx: Optional[Sequence[int]] = None,
         want_tuples: bool = False, tuple_cap: int = 1 << 22, budget: int = 0, elabels=None):
    """O2: incremental matches of ``query`` for ``batch`` on graph (n, labels, src, dst).

    Returns (counts, tuples): counts[j] = matches charged to update eval_idx[j]
    (all updates when eval_idx is None); tuples is an int32 array of rows
    (update, sign, phi[0..q-1]) or None. Raises OracleError on invalid input
    or when ``budget`` (candidate tests) is exceeded.  Edge labels (Sec. II-A):
    ``elabels`` for the graph's edges, ``query.elabels`` and ``batch.elab``;
    absent ones mean label 0.
    """
    if _edge_labelled(elabels, [query], batch):
        c, t = _bdsm_el(n, labels, src, dst, [query], batch, eval_idx, want_tuples, tuple_cap, budget, 0, elabels)
        return c[0], t
    lib = _load()
    labels = np.ascontiguousarray(labels, np.int32)
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    ql = np.ascontiguousarray(query.labels, np.int32)
    qs = np.ascontiguousarray(query.src, np.int32)
    qd = np.ascontiguousarray(query.dst, np.int32)
    op = np.ascontiguousarray(batch.op, np.int8)
    us = np.ascontiguousarray(batch.src, np.int32)
    ud = np.ascontiguousarray(batch.dst, np.int32)
    b = op.size
    ev = None if eval_idx is None else np.ascontiguousarray(eval_idx, np.int64)
    ne = b if ev is None else ev.size
    counts = np.zeros(max(ne, 1), np.uint64)
    tup = np.zeros((tuple_cap, 2 + ql.size), np.int32) if want_tuples else None
    nt = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    rc = lib.oracle_bdsm(n, _ptr(labels), src.size, _ptr(src), _ptr(dst),
                         ql.size, _ptr(ql), qs.size, _ptr(qs), _ptr(qd),
                         b, _ptr(op), _ptr(us), _ptr(ud),
                         ne, _ptr(ev), _ptr(counts),
                         _ptr(tup), tuple_cap if want_tuples else 0,
                         ctypes.byref(nt) if want_tuples else None,
                         budget, ctypes.byref(bad))
    if rc != OK:
        raise OracleError(rc, bad.value)
    counts = counts[:ne]
    if want_tuples:
        if nt.value > tuple_cap:
            raise OracleError(ENOMEM, -1)
        tup = tup[:nt.value]
    return counts, tup


NOT_COMPUTED = np.iinfo(np.uint64).max


def _bdsm_el(n, labels, src, dst, queries, batch, eval_idx, want_tuples, tuple_cap, budget, update_budget,
             elabels):
    """O2 with edge labels: counts [nq, ne] (and rows for a single query)."""
    lib = _load()
    labels = np.ascontiguousarray(labels, np.int32)
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    el = None if elabels is None else np.ascontiguousarray(elabels, np.int32)
    qn = np.array([q.q for q in queries], np.int32)
    qe = np.array([q.eq for q in queries], np.int32)
    ql = np.ascontiguousarray(np.concatenate([q.labels for q in queries]), np.int32)
    qs = np.ascontiguousarray(np.concatenate([q.src for q in queries]), np.int32)
    qd = np.ascontiguousarray(np.concatenate([q.dst for q in queries]), np.int32)
    qel = np.ascontiguousarray(np.concatenate([q.elabels if q.elabels is not None else np.zeros(q.eq, np.int32)
                                               for q in queries]), np.int32)
    lo = np.concatenate([[0], np.cumsum(qn)[:-1]]).astype(np.int64)
    eo = np.concatenate([[0], np.cumsum(qe)[:-1]]).astype(np.int64)
    op = np.ascontiguousarray(batch.op, np.int8)
    us = np.ascontiguousarray(batch.src, np.int32)
    ud = np.ascontiguousarray(batch.dst, np.int32)
    uel = None if batch.elab is None else np.ascontiguousarray(batch.elab, np.int32)
    b = op.size
    ev = None if eval_idx is None else np.ascontiguousarray(eval_idx, np.int64)
    ne = b if ev is None else ev.size
    counts = np.zeros(max(len(queries) * ne, 1), np.uint64)
    tup = np.zeros((tuple_cap, 2 + int(qn[0])), np.int32) if want_tuples else None
    nt = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    rc = lib.oracle_bdsm_multi_el(n, _ptr(labels), src.size, _ptr(src), _ptr(dst), _ptr(el),
                                  len(queries), _ptr(qn), _ptr(ql), _ptr(lo), _ptr(qe), _ptr(qs), _ptr(qd),
                                  _ptr(eo), _ptr(qel), b, _ptr(op), _ptr(us), _ptr(ud), _ptr(uel),
                                  ne, _ptr(ev), _ptr(counts), _ptr(tup), tuple_cap if want_tuples else 0,
                                  ctypes.byref(nt) if want_tuples else None, budget, update_budget,
                                  ctypes.byref(bad))
    if rc != OK:
        raise OracleError(rc, bad.value)
    counts = counts[:len(queries) * ne].reshape(len(queries), ne)
    if want_tuples:
        if nt.value > tuple_cap:
            raise OracleError(ENOMEM, -1)
        tup = tup[:nt.value]
    return counts, tup


def bdsm_multi(n: int, labels, src, dst, queries, batch, eval_idx: Optional[Sequence[int]] = None,
               budget: int = 0, update_budget: int = 0, elabels=None) -> np.ndarray:
    """O2 for several queries in one call (G, G' and the batch map are built
    once). Returns counts[j, i] = matches of query j charged to update eval_idx[i].
    With update_budget, a (query, update) pair needing more candidate tests
    than that is skipped and reported as NOT_COMPUTED."""
    if queries and _edge_labelled(elabels, queries, batch):
        return _bdsm_el(n, labels, src, dst, queries, batch, eval_idx, False, 0, budget, update_budget, elabels)[0]
    lib = _load()
    labels = np.ascontiguousarray(labels, np.int32)
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    qn = np.array([q.q for q in queries], np.int32)
    qe = np.array([q.eq for q in queries], np.int32)
    ql = np.ascontiguousarray(np.concatenate([q.labels for q in queries]) if queries else np.zeros(1), np.int32)
    qs = np.ascontiguousarray(np.concatenate([q.src for q in queries]) if queries else np.zeros(1), np.int32)
    qd = np.ascontiguousarray(np.concatenate([q.dst for q in queries]) if queries else np.zeros(1), np.int32)
    lo = np.concatenate([[0], np.cumsum(qn)[:-1]]).astype(np.int64) if queries else np.zeros(1, np.int64)
    eo = np.concatenate([[0], np.cumsum(qe)[:-1]]).astype(np.int64) if queries else np.zeros(1, np.int64)
    op = np.ascontiguousarray(batch.op, np.int8)
    us = np.ascontiguousarray(batch.src, np.int32)
    ud = np.ascontiguousarray(batch.dst, np.int32)
    b = op.size
    ev = None if eval_idx is None else np.ascontiguousarray(eval_idx, np.int64)
    ne = b if ev is None else ev.size
    counts = np.zeros(max(len(queries) * ne, 1), np.uint64)
    bad = ctypes.c_int64(-1)
    rc = lib.oracle_bdsm_multi(n, _ptr(labels), src.size, _ptr(src), _ptr(dst),
                               len(queries), _ptr(qn), _ptr(ql), _ptr(lo), _ptr(qe), _ptr(qs), _ptr(qd), _ptr(eo),
                               b, _ptr(op), _ptr(us), _ptr(ud), ne, _ptr(ev), _ptr(counts),
                               None, 0, None, budget, update_budget, ctypes.byref(bad))
    if rc != OK:
        raise OracleError(rc, bad.value)
    return counts[:len(queries) * ne].reshape(len(queries), ne)


def _pack_queries(queries):
    qn = np.array([q.q for q in queries], np.int32)
    qe = np.array([q.eq for q in queries], np.int32)
    ql = np.ascontiguousarray(np.concatenate([q.labels for q in queries]), np.int32)
    qs = np.ascontiguousarray(np.concatenate([q.src for q in queries]), np.int32)
    qd = np.ascontiguousarray(np.concatenate([q.dst for q in queries]), np.int32)
    el = None
    if any(getattr(q, "elabels", None) is not None for q in queries):
        el = np.ascontiguousarray(np.concatenate([q.elabels if q.elabels is not None else np.zeros(q.eq, np.int32)
                                                  for q in queries]), np.int32)
    lo = np.concatenate([[0], np.cumsum(qn)[:-1]]).astype(np.int64)
    eo = np.concatenate([[0], np.cumsum(qe)[:-1]]).astype(np.int64)
    return qn, ql, lo, qe, qs, qd, eo, el


class Session:
    """O2 with G, the batch and G' built once and kept (the same program as
    ``bdsm_multi``, whose every call builds them afresh): for evaluating many
    (query, update) pairs of one batch, and for splitting one heavy pair over
    several processes (``part``, ``parts``: the candidates of the first
    searched query vertex are dealt round-robin, so the parts' counts add up
    to the whole)."""

    def __init__(self, n: int, labels, src, dst, batch, elabels=None):
        lib = _load()
        self._keep = [np.ascontiguousarray(labels, np.int32), np.ascontiguousarray(src, np.int32),
                      np.ascontiguousarray(dst, np.int32),
                      None if elabels is None else np.ascontiguousarray(elabels, np.int32),
                      np.ascontiguousarray(batch.op, np.int8), np.ascontiguousarray(batch.src, np.int32),
                      np.ascontiguousarray(batch.dst, np.int32),
                      None if getattr(batch, "elab", None) is None else np.ascontiguousarray(batch.elab, np.int32)]
        lab, s, d, el, op, us, ud, uel = self._keep
        self.b = op.size
        self.op = op
        h = ctypes.c_void_p()
        bad = ctypes.c_int64(-1)
        rc = lib.oracle_session_open(n, _ptr(lab), s.size, _ptr(s), _ptr(d), _ptr(el), op.size, _ptr(op), _ptr(us),
                                     _ptr(ud), _ptr(uel), ctypes.byref(h), ctypes.byref(bad))
        if rc != OK:
            raise OracleError(rc, bad.value)
        self._h = h

    def eval(self, queries, eval_idx: Optional[Sequence[int]] = None, budget: int = 0, update_budget: int = 0,
             part: int = 0, parts: int = 1) -> np.ndarray:
        """counts[j, i] = matches of queries[j] charged to update eval_idx[i]
        (within part ``part`` of ``parts``); NOT_COMPUTED where update_budget
        candidate tests did not suffice."""
        if self._h is None:
            raise OracleError(EINVAL, -1)
        qn, ql, lo, qe, qs, qd, eo, el = _pack_queries(queries)
        ev = None if eval_idx is None else np.ascontiguousarray(eval_idx, np.int64)
        ne = self.b if ev is None else ev.size
        counts = np.zeros(max(len(queries) * ne, 1), np.uint64)
        rc = _load().oracle_session_eval(self._h, len(queries), _ptr(qn), _ptr(ql), _ptr(lo), _ptr(qe), _ptr(qs),
                                         _ptr(qd), _ptr(eo), _ptr(el), ne, _ptr(ev), _ptr(counts), None, 0, None,
                                         budget, update_budget, part, parts)
        if rc != OK:
            raise OracleError(rc, -1)
        return counts[:len(queries) * ne].reshape(len(queries), ne)

    def close(self):
        if getattr(self, "_h", None) is not None:
            _load().oracle_session_close(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def totals(counts: np.ndarray, op: np.ndarray, eval_idx=None) -> Tuple[int, int]:
    """(positive, negative) totals from per-update charged counts."""
    sg = np.asarray(op)[np.arange(len(op)) if eval_idx is None else np.asarray(eval_idx)]
    c = counts.astype(np.uint64)
    return int(c[sg > 0].sum()), int(c[sg < 0].sum())


def canonical_tuples(tuples: np.ndarray) -> np.ndarray:
    """Rows (sign, phi...) sorted lexicographically, '+' before '-'; the update
    column is dropped (compared separately as per-update counts)."""
    if tuples is None or tuples.size == 0:
        return np.zeros((0, 0 if tuples is None else tuples.shape[1] - 1), np.int64)
    rows = tuples[:, 1:].astype(np.int64).copy()
    rows[:, 0] = np.where(rows[:, 0] > 0, 0, 1)
    order = np.lexsort(rows.T[::-1])
    return rows[order]


# ---------------------------------------------------------------------------
# O1: brute-force static difference (pure Python, tiny graphs only)
# ---------------------------------------------------------------------------

def _edge(a: int, b: int) -> Tuple[int, int]:
    return (a, b) if a < b else (b, a)


def brute_embeddings(n: int, labels, edges, query) -> Set[Tuple[int, ...]]:
    """Every injective label-preserving map V(Q) -> V(G) whose query edges are
    all data edges (Def. 2), by trying every data vertex for every query
    vertex in id order and checking edges as soon as both ends are placed.
    ``edges`` is a set of data edges, or a dict edge -> edge label, in which
    case every query edge must map onto an edge of its own label (a query
    without edge labels asks for label 0)."""
    q = query.q
    ql = [int(x) for x in query.labels]
    qe = [(int(a), int(b)) for a, b in zip(query.src, query.dst)]
    qel = [0] * len(qe) if getattr(query, "elabels", None) is None else [int(x) for x in query.elabels]
    lab = [int(x) for x in labels]
    labelled = isinstance(edges, dict)
    nbrs_before = [[] for _ in range(q)]  # (w, label) for query edges (u, w) with w < u
    for (a, b), l in zip(qe, qel):
        hi, lo = max(a, b), min(a, b)
        nbrs_before[hi].append((lo, l))
    out: Set[Tuple[int, ...]] = set()
    phi = [-1] * q

    def rec(u: int):
        if u == q:
            out.add(tuple(phi))
            return
        for v in range(n):
            if lab[v] != ql[u] or v in phi[:u]:
                continue
            if all((edges.get(_edge(v, phi[w])) == l) if labelled else (_edge(v, phi[w]) in edges)
                   for w, l in nbrs_before[u]):
                phi[u] = v
                rec(u + 1)
                phi[u] = -1

    rec(0)
    return out


def brute_bdsm(n: int, labels, src, dst, query, batch, elabels=None):
    """O1: (positive set, negative set, charge) by static enumeration on G and G'.

    charge maps each incremental match (sign, phi) to the lowest index among
    the same-sign updates whose edge is the image of a query edge. With edge
    labels (``elabels`` for G, ``batch.elab`` for insertions) the graphs are
    edge -> label maps and embeddings must preserve edge labels too.
    """
    upd: Dict[Tuple[int, int], int] = {}
    for k, (o, a, b) in enumerate(zip(batch.op, batch.src, batch.dst)):
        upd[_edge(int(a), int(b))] = k
    ins = {e for e, k in upd.items() if batch.op[k] > 0}
    dele = {e for e, k in upd.items() if batch.op[k] < 0}
    if elabels is None and getattr(batch, "elab", None) is None and getattr(query, "elabels", None) is None:
        g = {_edge(int(a), int(b)) for a, b in zip(src, dst)}
        gp = (g - dele) | ins
    else:
        gl = [0] * len(src) if elabels is None else [int(x) for x in elabels]
        g = {_edge(int(a), int(b)): l for a, b, l in zip(src, dst, gl)}
        bl = [0] * len(batch.op) if getattr(batch, "elab", None) is None else [int(x) for x in batch.elab]
        gp = {e: l for e, l in g.items() if e not in dele}
        gp.update({e: bl[upd[e]] for e in ins})
    e0 = brute_embeddings(n, labels, g, query)
    e1 = brute_embeddings(n, labels, gp, query)
    pos, neg = e1 - e0, e0 - e1
    qe = [(int(a), int(b)) for a, b in zip(query.src, query.dst)]
    charge: Dict[Tuple[int, Tuple[int, ...]], int] = {}
    for sign, s in ((1, pos), (-1, neg)):
        for phi in s:
            ks = [upd[_edge(phi[a], phi[b])] for a, b in qe
                  if _edge(phi[a], phi[b]) in upd and batch.op[upd[_edge(phi[a], phi[b])]] == sign]
            charge[(sign, phi)] = min(ks)
    return pos, neg, charge


if __name__ == "__main__":  # build only
    print(build(force="--force" in sys.argv))
