"""Seeded synthetic inputs for batch-dynamic subgraph matching (BDSM).

This module is the one piece of code shared by the CPU oracle (``oracle/``)
and the CUDA path: it draws graphs, labels, update batches and query graphs.
It holds none of the matching arithmetic. Everything is integer and
counter-based (splitmix64 of a per-stream key plus the element index), so the
same seed gives the same bytes on x86 and on Arm.

Workload shapes follow the paper's experimental setup (Sec. VI-A): power-law
graphs of average degree 12-18 with several vertex labels (Table II stand-ins),
update batches mixing insertions drawn from a held-out edge pool with uniform
deletions of existing edges (Sec. VI-A "insertion/deletion rate", mixed
workloads in Sec. VI-C), and query graphs extracted from the data graph by a
random walk, classed as sparse or dense by average degree (Sec. VI-A
"Queries").
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

U64 = np.uint64
_GOLD = U64(0x9E3779B97F4A7C15)
_M1 = U64(0xBF58476D1CE4E5B9)
_M2 = U64(0x94D049BB133111EB)

# stream identifiers (arbitrary distinct constants)
S_RMAT, S_PERM, S_LABEL, S_SHUF, S_DEL, S_MIX, S_QUERY, S_SIZE, S_ARRIVE = (
    11, 12, 13, 14, 15, 16, 17, 18, 19)
S_SRV_DEL, S_SRV_INS, S_SRV_MIX = 31, 32, 33
S_ELABEL = 41


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> U64(30))) * _M1
        z = (z ^ (z >> U64(27))) * _M2
        return z ^ (z >> U64(31))


def stream_key(seed: int, stream: int, sub: int = 0) -> np.uint64:
    k = np.array([(seed * 1000003 + stream * 7919 + sub * 104729) & 0xFFFFFFFFFFFFFFFF],
                 dtype=U64)
    return _mix(k + _GOLD)[0]


def rand_u64(seed: int, stream: int, idx, sub: int = 0) -> np.ndarray:
    """Counter-based uint64 draws: element i of ``idx`` -> splitmix64(key + (i+1)*gold)."""
    idx = np.asarray(idx, dtype=U64)
    key = stream_key(seed, stream, sub)
    with np.errstate(over="ignore"):
        return _mix(key + (idx + U64(1)) * _GOLD)


def rand_u32(seed: int, stream: int, idx, sub: int = 0) -> np.ndarray:
    return (rand_u64(seed, stream, idx, sub) >> U64(32)).astype(np.uint64)


def _prob_threshold(p: float) -> int:
    return min((1 << 32) - 1, int(math.floor(p * (1 << 32))))


# --------------------------------------------------------------------------
# graphs
# --------------------------------------------------------------------------

_RMAT_LIB = None


def _rmat_lib():
    """The C version of the R-MAT draw (rmat_gen.c), built with gcc on first
    use into the package's _build folder; None when it cannot be built."""
    global _RMAT_LIB
    if _RMAT_LIB is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "rmat_gen.c")
        so = os.path.join(here, "_build", "librmat.so")
        try:
            if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
                os.makedirs(os.path.dirname(so), exist_ok=True)
                tmp = so + ".tmp%d" % os.getpid()
                subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src])
                os.replace(tmp, so)
            lib = ctypes.CDLL(so)
        except (OSError, subprocess.CalledProcessError):
            _RMAT_LIB = False
            return None
        p = ctypes.c_void_p
        lib.rmat_draw.restype = ctypes.c_int64
        lib.rmat_draw.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32, p, p]
        _RMAT_LIB = lib
    return _RMAT_LIB or None


def _rmat_draw_numpy(scale: int, n_edges: int, seed: int, ta: int, tab: int, tabc: int):
    """First ``n_edges`` distinct non-loop candidates in draw order (numpy)."""
    keys_all: List[np.ndarray] = []
    drawn = 0
    need = n_edges
    uniq = None
    first = None
    while True:
        chunk = max(1 << 16, int(need * 1.25) + 1024)
        idx = np.arange(drawn, drawn + chunk, dtype=U64)
        src = np.zeros(chunk, dtype=np.int64)
        dst = np.zeros(chunk, dtype=np.int64)
        for lvl in range(scale):
            r = rand_u32(seed, S_RMAT, idx * U64(scale) + U64(lvl)).astype(np.int64)
            sbit = (r >= tab).astype(np.int64)
            dbit = ((r >= ta) & (r < tab)) | (r >= tabc)
            bit = 1 << (scale - 1 - lvl)
            src |= sbit * bit
            dst |= dbit.astype(np.int64) * bit
        lo = np.minimum(src, dst)
        hi = np.maximum(src, dst)
        keep = lo != hi
        key = (lo << 32) | hi
        key[~keep] = -1  # marks self-loops
        keys_all.append(key)
        drawn += chunk
        allk = np.concatenate(keys_all)
        uniq, first = np.unique(allk, return_index=True)
        if uniq.size and uniq[0] == -1:
            uniq, first = uniq[1:], first[1:]
        if uniq.size >= n_edges:
            break
        need = n_edges - uniq.size
    order = np.argsort(first, kind="stable")[:n_edges]
    sel = uniq[order]
    return (sel >> 32).astype(np.int64), (sel & 0xFFFFFFFF).astype(np.int64)


def rmat_edges(scale: int, n_edges: int, seed: int,
               a: float = 0.57, b: float = 0.19, c: float = 0.19,
               permute: bool = True, engine: str = "auto") -> Tuple[np.ndarray, np.ndarray]:
    """Undirected R-MAT edge list with exactly ``n_edges`` unique edges.

    Candidates are drawn in index order; self-loops are dropped, each edge is
    canonicalised to (min, max) and only its first occurrence is kept, until
    ``n_edges`` unique edges exist. Vertex ids are then relabelled by a seeded
    random permutation so that hubs are not clustered at low ids. Returns
    int32 arrays (src < dst), in first-draw order.  ``engine``: "numpy", "c"
    (rmat_gen.c, the same bytes, much faster) or "auto" (C when it builds).
    """
    n = 1 << scale
    ta, tab, tabc = (_prob_threshold(a), _prob_threshold(a + b),
                     _prob_threshold(a + b + c))
    lib = _rmat_lib() if engine in ("auto", "c") else None
    if engine == "c" and lib is None:
        raise RuntimeError("the C R-MAT generator could not be built")
    if lib is not None:
        import ctypes
        s32 = np.empty(n_edges, np.int32)
        d32 = np.empty(n_edges, np.int32)
        drawn = lib.rmat_draw(scale, n_edges, int(stream_key(seed, S_RMAT)), ta, tab, tabc,
                              s32.ctypes.data_as(ctypes.c_void_p), d32.ctypes.data_as(ctypes.c_void_p))
        if drawn < 0:
            raise MemoryError("rmat_draw")
        src, dst = s32.astype(np.int64), d32.astype(np.int64)
    else:
        src, dst = _rmat_draw_numpy(scale, n_edges, seed, ta, tab, tabc)
    if permute:
        perm_key = rand_u64(seed, S_PERM, np.arange(n, dtype=U64))
        newid = np.empty(n, dtype=np.int64)
        newid[np.argsort(perm_key, kind="stable")] = np.arange(n, dtype=np.int64)
        src, dst = newid[src], newid[dst]
    lo = np.minimum(src, dst).astype(np.int32)
    hi = np.maximum(src, dst).astype(np.int32)
    return lo, hi


def vertex_labels(n: int, n_labels: int, seed: int, zipf_s: Optional[float] = None,
                  stream: int = S_LABEL) -> np.ndarray:
    """iid vertex labels in [0, n_labels): uniform, or Zipf with P(k) ~ (k+1)^-s."""
    r = rand_u32(seed, stream, np.arange(n, dtype=U64)).astype(np.int64)
    if zipf_s is None:
        w = [1.0] * n_labels
    else:
        w = [(k + 1) ** (-zipf_s) for k in range(n_labels)]
    tot = sum(w)
    acc, thr = 0.0, []
    for k in range(n_labels - 1):
        acc += w[k]
        thr.append(_prob_threshold(acc / tot))
    return np.searchsorted(np.array(thr, dtype=np.int64), r, side="right").astype(np.int32)


def edge_labels(src: np.ndarray, dst: np.ndarray, n_labels: int, seed: int,
                zipf_s: Optional[float] = None) -> np.ndarray:
    """iid labels for undirected edges (the edge-labelled datasets of Table
    II, e.g. NF and LS), drawn per edge from its canonical (min, max) key so
    that an edge gets the same label wherever it appears (graph, pool,
    batch): uniform, or Zipf with P(k) ~ (k+1)^-s."""
    key = edge_keys(np.asarray(src), np.asarray(dst)).astype(np.uint64)
    r = (rand_u64(seed, S_ELABEL, key) >> U64(32)).astype(np.int64)
    w = [1.0] * n_labels if zipf_s is None else [(k + 1) ** (-zipf_s) for k in range(n_labels)]
    tot = sum(w)
    acc, thr = 0.0, []
    for k in range(n_labels - 1):
        acc += w[k]
        thr.append(_prob_threshold(acc / tot))
    return np.searchsorted(np.array(thr, dtype=np.int64), r, side="right").astype(np.int32)


def shuffle_order(m: int, seed: int, stream: int, sub: int = 0) -> np.ndarray:
    key = rand_u64(seed, stream, np.arange(m, dtype=U64), sub)
    return np.argsort(key, kind="stable")


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Symmetric CSR (row offsets int64, sorted neighbour ids int32)."""
    s = np.concatenate([src, dst]).astype(np.int64)
    d = np.concatenate([dst, src]).astype(np.int64)
    order = np.argsort(s * (1 << 32) + d, kind="stable")
    s, d = s[order], d[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(s, minlength=n), out=off[1:])
    return off, d.astype(np.int32)


def edge_keys(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    lo = np.minimum(src, dst).astype(np.int64)
    hi = np.maximum(src, dst).astype(np.int64)
    return (lo << 32) | hi


# --------------------------------------------------------------------------
# update batches
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Batch:
    op: np.ndarray   # int8, +1 insertion, -1 deletion
    src: np.ndarray  # int32
    dst: np.ndarray  # int32
    # int32 edge labels, None = unlabelled edges; an insertion's label, and
    # for a deletion the label the edge has (only the inverse batch uses it)
    elab: Optional[np.ndarray] = None

    def __len__(self) -> int:
        return int(self.op.size)

    def inverse(self) -> "Batch":
        """The batch that undoes this one (same order, opposite signs)."""
        return Batch((-self.op).astype(np.int8), self.src.copy(), self.dst.copy(),
                     None if self.elab is None else self.elab.copy())


def mixed_batch(ins_src, ins_dst, cur_src, cur_dst, n_del: int, seed: int, sub: int) -> Batch:
    """Insertions (given, in order) plus ``n_del`` uniform deletions sampled
    without replacement from the current edge list, interleaved by a seeded
    shuffle."""
    m = cur_src.size
    if n_del > m:
        raise ValueError("more deletions than edges")
    pick = shuffle_order(m, seed, S_DEL, sub)[:n_del]
    op = np.concatenate([np.ones(ins_src.size, np.int8), -np.ones(n_del, np.int8)])
    s = np.concatenate([ins_src, cur_src[pick]]).astype(np.int32)
    d = np.concatenate([ins_dst, cur_dst[pick]]).astype(np.int32)
    mix = shuffle_order(op.size, seed, S_MIX, sub)
    return Batch(op[mix], s[mix], d[mix])


def apply_batch_edges(src, dst, batch: Batch) -> Tuple[np.ndarray, np.ndarray]:
    """Edge list after a (valid) batch: deletions removed, insertions appended."""
    k = edge_keys(src, dst)
    dk = edge_keys(batch.src[batch.op < 0], batch.dst[batch.op < 0])
    keep = ~np.isin(k, dk)
    ins = batch.op > 0
    s = np.concatenate([src[keep], np.minimum(batch.src[ins], batch.dst[ins])])
    d = np.concatenate([dst[keep], np.maximum(batch.src[ins], batch.dst[ins])])
    return s.astype(np.int32), d.astype(np.int32)


# --------------------------------------------------------------------------
# query graphs
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Query:
    labels: np.ndarray  # int32 [q]
    src: np.ndarray     # int32 [eq]
    dst: np.ndarray     # int32 [eq]
    kind: str = ""
    elabels: Optional[np.ndarray] = None  # int32 [eq] edge labels, None = unlabelled edges

    @property
    def q(self) -> int:
        return int(self.labels.size)

    @property
    def eq(self) -> int:
        return int(self.src.size)

    def to_json(self) -> dict:
        d = {"labels": [int(x) for x in self.labels],
             "edges": [[int(a), int(b)] for a, b in zip(self.src, self.dst)],
             "kind": self.kind}
        if self.elabels is not None:
            d["elabels"] = [int(x) for x in self.elabels]
        return d

    @staticmethod
    def from_json(d: dict) -> "Query":
        e = np.array(d["edges"], dtype=np.int32).reshape(-1, 2)
        el = np.array(d["elabels"], np.int32) if "elabels" in d else None
        return Query(np.array(d["labels"], np.int32), e[:, 0].copy(), e[:, 1].copy(),
                     d.get("kind", ""), el)


def random_walk_query(off: np.ndarray, nbr: np.ndarray, labels: np.ndarray, q: int,
                      kind: str, seed: int, attempt: int) -> Optional[Query]:
    """One query-extraction attempt (Sec. VI-A: queries are random subgraphs
    of the data graph, classed by average degree as Dense, Sparse or Tree).

    "tree": a random walk from a uniform vertex of non-zero degree to uniform
    neighbours until ``q`` distinct vertices are seen; the query is the set
    of traversed edges, kept when it is a tree (|E| = |V| - 1).

    "dense" and "sparse": a growing walk. It starts at a uniformly drawn end
    of a uniformly drawn edge and repeatedly adds, among the neighbours of the
    vertices taken so far, one with the most neighbours inside the taken set
    (ties broken by the seeded generator), until ``q`` vertices are taken.
    "dense" keeps the induced subgraph when its average degree is > 3;
    "dense_ge3" when it is >= 3 (the paper's Dense class, Sec. VI-A).
    "sparse" keeps a random spanning tree of the induced subgraph plus random
    further induced edges up to |E| = min(#induced, q + r) with r in
    [0, q/2] drawn per attempt, so the average degree is <= 3 and the query
    has at least one cycle; it is None when the induced subgraph is a tree.
    "sparse_lt3": the same with average degree < 3, the complement of
    "dense_ge3" (a query of exactly 3 belongs to dense_ge3 only).
    Labels are inherited. Returns None when the class test fails.
    """
    n = off.size - 1
    step = 0

    def draw() -> int:
        nonlocal step
        v = int(rand_u64(seed, S_QUERY, np.array([step], dtype=U64), attempt)[0])
        step += 1
        return v

    def induced(order):
        edges = []
        for i in range(len(order)):
            row = nbr[off[order[i]]:off[order[i] + 1]]
            for j in range(i + 1, len(order)):
                pos = np.searchsorted(row, order[j])
                if pos < row.size and row[pos] == order[j]:
                    edges.append((i, j))
        return edges

    if kind == "tree":
        v = None
        for _ in range(64):
            c = draw() % n
            if off[c + 1] > off[c]:
                v = c
                break
        if v is None:
            return None
        order, seen, trav = [v], {v: 0}, set()
        for _ in range(60 * q):
            if len(order) == q:
                break
            d = int(off[v + 1] - off[v])
            w = int(nbr[off[v] + draw() % d])
            if w not in seen:
                seen[w] = len(order)
                order.append(w)
            a, b = seen[v], seen[w]
            trav.add((min(a, b), max(a, b)))
            v = w
        if len(order) < q or len(trav) != q - 1:
            return None
        edges = sorted(trav)
    else:
        m2 = int(off[-1])
        v = int(nbr[draw() % m2])
        order = [v]
        while len(order) < q:
            cand = np.concatenate([nbr[off[x]:off[x + 1]] for x in order])
            cand = cand[~np.isin(cand, np.array(order))]
            if cand.size == 0:
                return None
            u, cnt = np.unique(cand, return_counts=True)
            best = u[cnt == cnt.max()]
            order.append(int(best[draw() % best.size]))
        ind = induced(order)
        if kind in ("dense", "dense_ge3"):
            avg = 2.0 * len(ind) / q
            if not (avg > 3.0 if kind == "dense" else avg >= 3.0):
                return None
            edges = ind
        else:
            if len(ind) < q:
                return None
            ranked = sorted(ind, key=lambda e: (draw(), e))
            parent = list(range(q))

            def find(x):
                while parent[x] != x:
                    parent[x] = parent[parent[x]]
                    x = parent[x]
                return x
            tree, rest = [], []
            for a, b in ranked:
                ra, rb = find(a), find(b)
                if ra != rb:
                    parent[ra] = rb
                    tree.append((a, b))
                else:
                    rest.append((a, b))
            extra = 1 + draw() % (q // 2 + 1)
            extra = min(extra, len(rest), q // 2 + 1)
            edges = sorted(tree + rest[:extra])
            if not (len(edges) >= q and 2.0 * len(edges) / q <= 3.0):
                return None
            if kind == "sparse_lt3" and 2.0 * len(edges) / q >= 3.0:
                return None
    e = np.array(edges, dtype=np.int32).reshape(-1, 2)
    return Query(labels[np.array(order)].astype(np.int32), e[:, 0].copy(), e[:, 1].copy(), kind)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Graph:
    n: int
    labels: np.ndarray
    src: np.ndarray
    dst: np.ndarray
    elabels: Optional[np.ndarray] = None  # int32 edge labels, None = unlabelled edges

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.labels, self.src, self.dst) + (() if self.elabels is None else (self.elabels,)):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()[:16]


@dataclasses.dataclass
class Workload:
    name: str
    graph: Graph           # G0
    pool_src: np.ndarray   # held-out insertion pool
    pool_dst: np.ndarray
    seed: int


WORKLOADS = {
    # name: (scale, unique edges, labels, zipf s or None, seed)
    "tiny": (11, 10_000, 4, None, 1),
    "mid": (20, 8_388_608, 8, 1.2, 1),
    "large": (23, 67_108_864, 16, 1.0, 1),
    "served": (22, 33_554_432, 8, 1.2, 1),
}


def make_workload(name: str, scale: Optional[int] = None, n_edges: Optional[int] = None) -> Workload:
    """G0 plus insertion pool for a named workload; ``scale``/``n_edges``
    override the size (for scaled-down tests of the same shape)."""
    sc, ne, nl, zs, seed = WORKLOADS[name]
    sc = scale if scale is not None else sc
    ne = n_edges if n_edges is not None else ne
    src, dst = rmat_edges(sc, ne, seed)
    n = 1 << sc
    labels = vertex_labels(n, nl, seed, zs)
    order = shuffle_order(src.size, seed, S_SHUF)
    npool = int(round(src.size * 0.1))
    p, g = order[:npool], order[npool:]
    return Workload(name, Graph(n, labels, src[g].copy(), dst[g].copy()),
                    src[p].copy(), dst[p].copy(), seed)


def workload_batch(w: Workload, n_ins: int, n_del: int, sub: int = 0, pool_start: int = 0,
                   cur: Optional[Tuple[np.ndarray, np.ndarray]] = None) -> Batch:
    cs, cd = cur if cur is not None else (w.graph.src, w.graph.dst)
    return mixed_batch(w.pool_src[pool_start:pool_start + n_ins],
                       w.pool_dst[pool_start:pool_start + n_ins], cs, cd, n_del, w.seed, sub)


def consecutive_batches(w: Workload, count: int, n_ins: int, n_del: int) -> List[Batch]:
    """``count`` batches applied one after another to G0, each committed
    before the next (the large workload: five batches of 800,000 insertions
    and 200,000 deletions).  Batch k inserts the pool edges
    [k * n_ins, (k + 1) * n_ins) and deletes ``n_del`` edges drawn uniformly
    without replacement from the graph as it stands after batches 0..k-1;
    its updates are interleaved by a seeded shuffle."""
    cs, cd = w.graph.src, w.graph.dst
    out = []
    for k in range(count):
        isrc = w.pool_src[k * n_ins:(k + 1) * n_ins]
        idst = w.pool_dst[k * n_ins:(k + 1) * n_ins]
        if isrc.size < n_ins or n_del > cs.size:
            raise ValueError("the pool or the graph is too small for batch %d" % k)
        pick = sample_distinct(cs.size, n_del, w.seed, S_DEL, 100 + k)
        op = np.concatenate([np.ones(n_ins, np.int8), -np.ones(n_del, np.int8)])
        s = np.concatenate([isrc, cs[pick]]).astype(np.int32)
        d = np.concatenate([idst, cd[pick]]).astype(np.int32)
        mix = shuffle_order(op.size, w.seed, S_MIX, 100 + k)
        out.append(Batch(op[mix], s[mix], d[mix]))
        keep = np.ones(cs.size, bool)
        keep[pick] = False
        cs = np.concatenate([cs[keep], np.minimum(isrc, idst)]).astype(np.int32)
        cd = np.concatenate([cd[keep], np.maximum(isrc, idst)]).astype(np.int32)
    return out


def graph_after(src: np.ndarray, dst: np.ndarray, batches: Sequence[Batch]) -> Tuple[np.ndarray, np.ndarray]:
    """Edge list after applying ``batches`` in order (each valid on the graph
    the previous ones leave)."""
    for b in batches:
        src, dst = apply_batch_edges(src, dst, b)
    return src, dst


def served_sizes(n_batches: int, seed: int, lo_exp: float = 3.0, hi_exp: float = 6.0) -> np.ndarray:
    """Batch sizes floor(10^U(lo, hi)), U drawn from 32-bit integers."""
    r = rand_u32(seed, S_SIZE, np.arange(n_batches, dtype=U64)).astype(np.float64) / float(1 << 32)
    return np.floor(10.0 ** (lo_exp + (hi_exp - lo_exp) * r)).astype(np.int64)


def sample_distinct(n: int, k: int, seed: int, stream: int, sub: int = 0) -> np.ndarray:
    """k distinct uniform draws from range(n), in draw order: counter-based
    draws modulo n, repeats skipped (so the result is a uniform sample
    without replacement; the modulo bias is below n / 2^64)."""
    if k > n:
        raise ValueError("cannot draw %d distinct values from %d" % (k, n))
    got = np.empty(0, np.int64)
    ctr = 0
    while got.size < k:
        m = max(2 * (k - got.size), 1024)
        r = (rand_u64(seed, stream, np.arange(ctr, ctr + m, dtype=U64), sub) % U64(n)).astype(np.int64)
        ctr += m
        cand = np.concatenate([got, r])
        _, first = np.unique(cand, return_index=True)
        got = cand[np.sort(first)][:k]
    return got


def _take(pool: np.ndarray, size: int, pos: np.ndarray) -> Tuple[np.ndarray, int]:
    """Remove the entries at positions ``pos`` (distinct, < size) from the
    first ``size`` entries of ``pool`` in O(len(pos)): the holes below the
    new end are filled with the kept entries of the tail.  Returns the
    removed entries and the new size."""
    k = pos.size
    taken = pool[pos].copy()
    new = size - k
    holes = np.sort(pos[pos < new])
    mark = np.zeros(k, bool)
    mark[pos[pos >= new] - new] = True
    fill = new + np.flatnonzero(~mark)
    pool[holes] = pool[fill]
    return taken, new


def served_stream(w: "Workload", n_batches: int, seed: int, lo_exp: float = 3.0,
                  hi_exp: float = 6.0) -> List[Batch]:
    """The served workload's request stream: batches of floor(10^U(3, 6))
    updates (the exponents are parameters) with insertions : deletions = 1 : 1.  Deletions are drawn uniformly
    without replacement from the graph as it stands after the previous
    batches, insertions from the free pool (held-out edges and edges deleted
    earlier), so every batch is valid in order; the updates of a batch are
    interleaved by a seeded shuffle.  The present and free edge sets are kept
    as arrays with O(batch) removal, so a long stream costs time in
    proportion to its updates, not to the graph."""
    g = w.graph
    src = np.concatenate([g.src, w.pool_src])
    dst = np.concatenate([g.dst, w.pool_dst])
    m0, m = g.src.size, src.size
    pres = np.empty(m, np.int64)
    pres[:m0] = np.arange(m0)
    free = np.empty(m, np.int64)
    free[:m - m0] = np.arange(m0, m)
    npres, nfree = m0, m - m0
    out = []
    for k, n in enumerate(served_sizes(n_batches, seed, lo_exp, hi_exp)):
        nd = int(n) // 2
        ni = int(n) - nd
        d, npres = _take(pres, npres, sample_distinct(npres, nd, seed, S_SRV_DEL, k))
        i, nfree = _take(free, nfree, sample_distinct(nfree, ni, seed, S_SRV_INS, k))
        pres[npres:npres + ni] = i
        npres += ni
        free[nfree:nfree + nd] = d
        nfree += nd
        op = np.concatenate([np.ones(i.size, np.int8), -np.ones(d.size, np.int8)])
        e = np.concatenate([i, d])
        mix = shuffle_order(op.size, seed, S_SRV_MIX, k)
        out.append(Batch(op[mix], src[e][mix].astype(np.int32), dst[e][mix].astype(np.int32)))
    return out


def poisson_gaps(n: int, seed: int, rate_per_s: float) -> np.ndarray:
    """Exponential inter-arrival gaps (seconds) for a Poisson arrival process."""
    r = (rand_u32(seed, S_ARRIVE, np.arange(n, dtype=U64)).astype(np.float64) + 0.5) / float(1 << 32)
    return -np.log(r) / rate_per_s


def load_queries(path: str) -> List[Query]:
    import json
    with open(path) as f:
        d = json.load(f)
    return [Query.from_json(x) for x in d["queries"]]


def pattern_query(labels: Sequence[int], edges: Sequence[Tuple[int, int]], kind: str = "") -> Query:
    e = np.array(edges, dtype=np.int32).reshape(-1, 2)
    return Query(np.array(labels, np.int32), e[:, 0].copy(), e[:, 1].copy(), kind)


# The tiny workload's query: a 4-vertex labelled triangle with a tail, shaped
# like the running example's Q (u0 labelled A joined to u1 and u2, which share
# a label; u3 hangs on u1 with a third label) plus the u1-u2 edge.
TRIANGLE_WITH_TAIL = pattern_query([0, 1, 1, 2], [(0, 1), (0, 2), (1, 2), (1, 3)], "tiny")


def random_small_graph(n: int, p_edge_num: int, n_labels: int, seed: int, sub: int) -> Graph:
    """Erdos-Renyi style tiny graph for brute-force cross-checks."""
    iu, ju = np.triu_indices(n, 1)
    r = rand_u32(seed, S_RMAT, np.arange(iu.size, dtype=U64), sub).astype(np.int64)
    keep = r < (p_edge_num * (1 << 32)) // 100
    lab = (rand_u32(seed, S_LABEL, np.arange(n, dtype=U64), sub) % U64(n_labels)).astype(np.int32)
    return Graph(n, lab, iu[keep].astype(np.int32), ju[keep].astype(np.int32))
