"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every test here runs on the CPU. Each pin is independent of the oracle's own
code: the paper's running example (reconstructed, Sec. I Example 1), a
brute-force static difference (Def. 1 / Def. 2 written out), networkx's
subgraph-monomorphism enumerator, textbook closed forms (single edge, triangle
listing, wedge count from degrees) and invariants of the problem statement.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_17018_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _running():
    with open(os.path.join(GOLD, "running_example.json")) as f:
        d = json.load(f)
    e = np.array(d["edges"], np.int32)
    q = I.pattern_query(d["query"]["labels"], [tuple(x) for x in d["query"]["edges"]])
    b = I.Batch(np.array(d["batch"]["op"], np.int8), np.array(d["batch"]["src"], np.int32),
                np.array(d["batch"]["dst"], np.int32))
    return d, np.array(d["labels"], np.int32), e[:, 0].copy(), e[:, 1].copy(), q, b


def _tupset(t, sign=None):
    return {tuple(int(x) for x in r[2:]) for r in t if sign is None or r[1] == sign}


def test_running_example_bdsm():
    d, lab, s, t, q, b = _running()
    c, tup = O.bdsm(d["n"], lab, s, t, q, b, want_tuples=True)
    assert O.totals(c, b.op) == (d["bdsm"]["pos"], d["bdsm"]["neg"])
    assert c.tolist() == d["bdsm"]["per_update"]
    assert _tupset(tup, 1) == {tuple(x) for x in d["bdsm"]["pos_tuples"]}
    # the match quoted in the text exists in G (a static embedding)
    emb = O.brute_embeddings(d["n"], lab, {(min(a, bb), max(a, bb)) for a, bb in zip(s, t)}, q)
    assert tuple(d["static_match_in_G"]) in emb


def test_running_example_csm_sequence():
    """One update per batch, applied in order: +4, +2, -2 (Sec. I, Example 1)."""
    d, lab, s, t, q, b = _running()
    cs, ct = s.copy(), t.copy()
    for k in range(len(b)):
        one = I.Batch(b.op[k:k + 1], b.src[k:k + 1], b.dst[k:k + 1])
        c, tup = O.bdsm(d["n"], lab, cs, ct, q, one, want_tuples=True)
        want = d["csm"][k]
        assert O.totals(c, one.op) == (want["pos"], want["neg"])
        if "pos_tuples" in want:
            assert _tupset(tup, 1) == {tuple(x) for x in want["pos_tuples"]}
        if "neg_tuples" in want:
            assert _tupset(tup, -1) == {tuple(x) for x in want["neg_tuples"]}
        cs, ct = I.apply_batch_edges(cs, ct, one)
    # BDSM is not the concatenation of the CSM results (Sec. I)
    c, _ = O.bdsm(d["n"], lab, s, t, q, b)
    assert O.totals(c, b.op) != (4 + 2, 2)


def _random_batch(g: I.Graph, seed: int, n_ins: int, n_del: int) -> I.Batch:
    r = np.random.default_rng(seed)
    es = set(zip(g.src.tolist(), g.dst.tolist()))
    non = [(a, bb) for a in range(g.n) for bb in range(a + 1, g.n) if (a, bb) not in es]
    ni = min(len(non), n_ins)
    nd = min(len(es), n_del)
    ins = [non[i] for i in r.choice(len(non), ni, replace=False)] if ni else []
    el = sorted(es)
    dl = [el[i] for i in r.choice(len(el), nd, replace=False)] if nd else []
    ops = [1] * len(ins) + [-1] * len(dl)
    ed = ins + dl
    perm = r.permutation(len(ops))
    flip = r.integers(0, 2, len(ops))
    src = [ed[i][flip[j]] for j, i in enumerate(perm)]
    dst = [ed[i][1 - flip[j]] for j, i in enumerate(perm)]
    return I.Batch(np.array([ops[i] for i in perm], np.int8), np.array(src, np.int32), np.array(dst, np.int32))


SMALL_QUERIES = [
    I.pattern_query([0, 1], [(0, 1)]),
    I.pattern_query([0, 0, 0], [(0, 1), (1, 2)]),
    I.pattern_query([1, 0, 1], [(0, 1), (1, 2), (0, 2)]),
    I.pattern_query([0, 1, 1, 0], [(0, 1), (0, 2), (1, 2), (2, 3)]),
    I.pattern_query([0, 0, 0, 0], [(0, 1), (1, 2), (2, 3), (3, 0)]),
]


@pytest.mark.parametrize("trial", range(60))
def test_incremental_equals_static_difference(trial):
    """O2 (per-update search with charging) == O1 (Emb(G') - Emb(G) and back)."""
    g = I.random_small_graph(8, 45, 2, 3, trial)
    b = _random_batch(g, trial, 1 + trial % 4, trial % 3)
    for q in SMALL_QUERIES:
        pos, neg, charge = O.brute_bdsm(g.n, g.labels, g.src, g.dst, q, b)
        c, tup = O.bdsm(g.n, g.labels, g.src, g.dst, q, b, want_tuples=True)
        want = np.zeros(len(b), np.int64)
        for (_s, _phi), k in charge.items():
            want[k] += 1
        assert np.array_equal(c.astype(np.int64), want)
        got = {(int(r[1]), tuple(int(x) for x in r[2:])) for r in tup}
        assert len(got) == len(tup)  # no match found twice
        assert got == {(1, p) for p in pos} | {(-1, p) for p in neg}
        for r in tup:  # each row charged to its lowest same-sign update
            assert charge[(int(r[1]), tuple(int(x) for x in r[2:]))] == r[0]


def _nx_embeddings(n, labels, edges, q):
    nx = pytest.importorskip("networkx")
    from networkx.algorithms import isomorphism as iso
    G = nx.Graph()
    G.add_nodes_from((v, {"l": int(labels[v])}) for v in range(n))
    G.add_edges_from(edges)
    P = nx.Graph()
    P.add_nodes_from((u, {"l": int(q.labels[u])}) for u in range(q.q))
    P.add_edges_from(zip(q.src.tolist(), q.dst.tolist()))
    gm = iso.GraphMatcher(G, P, node_match=lambda a, b: a["l"] == b["l"])
    out = set()
    for mp in gm.subgraph_monomorphisms_iter():
        inv = {u: v for v, u in mp.items()}
        out.add(tuple(inv[u] for u in range(q.q)))
    return out


@pytest.mark.parametrize("trial", range(6))
def test_against_networkx_monomorphisms(trial):
    """Static embeddings from networkx (a library routine) differenced on G and G'."""
    g = I.random_small_graph(30, 18, 3, 11, trial)
    b = _random_batch(g, 100 + trial, 6, 4)
    ge = set(zip(g.src.tolist(), g.dst.tolist()))
    gp = set(ge)
    for o, s, t in zip(b.op, b.src, b.dst):
        e = (min(s, t), max(s, t))
        if o > 0:
            gp.add(e)
        else:
            gp.discard(e)
    for q in [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)]),
              I.pattern_query([0, 0, 1, 1], [(0, 1), (1, 2), (2, 3), (3, 0)])]:
        e0 = _nx_embeddings(g.n, g.labels, ge, q)
        e1 = _nx_embeddings(g.n, g.labels, gp, q)
        c, tup = O.bdsm(g.n, g.labels, g.src, g.dst, q, b, want_tuples=True)
        assert _tupset(tup, 1) == e1 - e0
        assert _tupset(tup, -1) == e0 - e1
        assert O.totals(c, b.op) == (len(e1 - e0), len(e0 - e1))


def test_single_edge_closed_form():
    """Q = one edge: each label-compatible update counts once per orientation."""
    w = I.make_workload("tiny")
    g = w.graph
    b = I.workload_batch(w, 200, 50)
    for la, lb in [(0, 1), (2, 2), (3, 0)]:
        q = I.pattern_query([la, lb], [(0, 1)])
        c, _ = O.bdsm(g.n, g.labels, g.src, g.dst, q, b)
        L = g.labels
        want = [int(L[s] == la and L[t] == lb) + int(L[t] == la and L[s] == lb) for s, t in zip(b.src, b.dst)]
        assert c.tolist() == want


def _triangles(n, edges):
    nx = pytest.importorskip("networkx")
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(edges)
    return {tuple(sorted(c)) for c in nx.enumerate_all_cliques(G) if len(c) == 3}


def test_unlabelled_triangle_closed_form():
    """6 embeddings per new / vanished triangle (triangle listing from networkx)."""
    g = I.random_small_graph(40, 22, 1, 5, 0)
    b = _random_batch(g, 7, 15, 10)
    ge = set(zip(g.src.tolist(), g.dst.tolist()))
    gp = set(ge)
    for o, s, t in zip(b.op, b.src, b.dst):
        e = (min(s, t), max(s, t))
        gp.add(e) if o > 0 else gp.discard(e)
    t0, t1 = _triangles(g.n, ge), _triangles(g.n, gp)
    q = I.pattern_query([0, 0, 0], [(0, 1), (1, 2), (0, 2)])
    c, _ = O.bdsm(g.n, g.labels, g.src, g.dst, q, b)
    assert O.totals(c, b.op) == (6 * len(t1 - t0), 6 * len(t0 - t1))


def test_unlabelled_wedge_closed_form():
    """Ordered 2-paths: Emb = sum_v d(v)(d(v)-1), so pos - neg is the difference."""
    w = I.make_workload("tiny")
    g = w.graph
    b = I.workload_batch(w, 300, 100)
    lab0 = np.zeros(g.n, np.int32)
    q = I.pattern_query([0, 0, 0], [(0, 1), (1, 2)])
    c, _ = O.bdsm(g.n, lab0, g.src, g.dst, q, b)
    pos, neg = O.totals(c, b.op)
    d0 = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n).astype(np.int64)
    s1, t1 = I.apply_batch_edges(g.src, g.dst, b)
    d1 = np.bincount(np.concatenate([s1, t1]), minlength=g.n).astype(np.int64)
    assert pos - neg == int((d1 * (d1 - 1)).sum() - (d0 * (d0 - 1)).sum())


def test_invariants_on_tiny_workload():
    w = I.make_workload("tiny")
    g = w.graph
    b = I.workload_batch(w, 256, 64)
    q = I.TRIANGLE_WITH_TAIL
    c, tup = O.bdsm(g.n, g.labels, g.src, g.dst, q, b, want_tuples=True)
    pos, neg = O.totals(c, b.op)
    assert pos + neg > 0
    # count equals the number of distinct rows; per-update sums equal totals
    rows = {(int(r[1]),) + tuple(int(x) for x in r[2:]) for r in tup}
    assert len(rows) == len(tup) == pos + neg
    assert int(c.sum()) == pos + neg
    # permuting the batch keeps the match sets (charges move with the updates)
    perm = np.random.default_rng(3).permutation(len(b))
    bp = I.Batch(b.op[perm], b.dst[perm], b.src[perm])
    cp, tp = O.bdsm(g.n, g.labels, g.src, g.dst, q, bp, want_tuples=True)
    assert O.totals(cp, bp.op) == (pos, neg)
    assert {(int(r[1]),) + tuple(int(x) for x in r[2:]) for r in tp} == rows
    # round trip: the inverse batch on G' removes exactly what the batch added
    s1, t1 = I.apply_batch_edges(g.src, g.dst, b)
    ci, ti = O.bdsm(g.n, g.labels, s1, t1, q, b.inverse(), want_tuples=True)
    assert _tupset(ti, -1) == _tupset(tup, 1)
    assert _tupset(ti, 1) == _tupset(tup, -1)


@pytest.mark.parametrize("case,bad", [
    ("dup_same", 3), ("insert_existing", 2), ("delete_missing", 1), ("self_loop", 0), ("bad_id", 2),
    ("ins_del_same_edge", 2)])
def test_batch_validation(case, bad):
    g = I.Graph(6, np.zeros(6, np.int32), np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32))
    q = I.pattern_query([0, 0], [(0, 1)])
    ops, src, dst = {
        "dup_same": ([1, 1, 1, 1], [0, 4, 0, 5], [4, 5, 5, 4]),
        "insert_existing": ([1, -1, 1], [0, 0, 2], [4, 1, 1]),
        "delete_missing": ([1, -1, 1], [0, 0, 3], [4, 5, 5]),
        "self_loop": ([1, 1], [2, 0], [2, 4]),
        "bad_id": ([1, 1, 1], [0, 1, 9], [4, 4, 0]),
        "ins_del_same_edge": ([1, 1, -1], [0, 1, 4], [4, 5, 0]),
    }[case]
    b = I.Batch(np.array(ops, np.int8), np.array(src, np.int32), np.array(dst, np.int32))
    with pytest.raises(O.OracleError) as e:
        O.bdsm(g.n, g.labels, g.src, g.dst, q, b)
    assert e.value.code == O.EINVAL and e.value.bad_index == bad


def test_planted_mistakes_are_caught():
    """A plausible bug in the charging or view logic changes these pins."""
    d, lab, s, t, q, b = _running()
    # ignoring the sign (treating the deletion as an insertion) changes the result
    b2 = I.Batch(np.array([1, 1, 1], np.int8), b.src, b.dst)
    with pytest.raises(O.OracleError):
        O.bdsm(d["n"], lab, s, t, q, b2)  # (4,5) exists: inserting it is invalid
    # dropping the deletion gives the CSM-like +6 instead of +4
    b3 = I.Batch(b.op[:2].copy(), b.src[:2].copy(), b.dst[:2].copy())
    c3, _ = O.bdsm(d["n"], lab, s, t, q, b3)
    assert O.totals(c3, b3.op) == (6, 0)


@pytest.mark.parametrize("trial", range(6))
def test_vertex_updates_as_edge_batches(trial):
    """Sec. II-A treats vertex updates as edge updates. Pinned by brute force:
    (1) deleting every edge of a vertex v makes exactly the embeddings of G
    that use v vanish (a connected query with >= 2 vertices uses one of v's
    edges whenever it uses v), and nothing appears; (2) inserting a new
    vertex's edges makes exactly the embeddings of G' that use it appear;
    (3) isolated extra vertices change no count."""
    g = I.random_small_graph(14, 40, 2, 7, trial)
    qs = [I.pattern_query([0, 1, 1], [(0, 1), (1, 2)]), I.TRIANGLE_WITH_TAIL if trial % 2 else
          I.pattern_query([0, 0, 1], [(0, 1), (1, 2), (0, 2)])]
    edges = {(min(int(a), int(b)), max(int(a), int(b))) for a, b in zip(g.src, g.dst)}
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n)
    v = int(np.argmax(deg))
    inc = sorted(e for e in edges if v in e)
    dele = I.Batch(-np.ones(len(inc), np.int8), np.array([a for a, _ in inc], np.int32),
                   np.array([b for _, b in inc], np.int32))
    # a new vertex n joined to the neighbours of v (and v), labelled like v
    n2 = g.n + 1
    lab2 = np.concatenate([g.labels, g.labels[v:v + 1]])
    new = sorted({(min(u, g.n), max(u, g.n)) for e in inc for u in e} )
    ins = I.Batch(np.ones(len(new), np.int8), np.array([a for a, _ in new], np.int32),
                  np.array([b for _, b in new], np.int32))
    for q in qs:
        emb = O.brute_embeddings(g.n, g.labels, edges, q)
        using_v = {m for m in emb if v in m}
        c, t = O.bdsm(g.n, g.labels, g.src, g.dst, q, dele, want_tuples=True)
        pos, neg = O.totals(c, dele.op)
        assert pos == 0 and neg == len(using_v)
        assert _tupset(t, -1) == using_v
        # (3) isolated extra vertex: same counts as on the original graph
        c3, _ = O.bdsm(n2, lab2, g.src, g.dst, q, dele)
        assert np.array_equal(c3, c)
        # (2) the new vertex's edges, on the graph with the vertex added
        emb2 = O.brute_embeddings(n2, lab2, edges | set(new), q)
        c2, t2 = O.bdsm(n2, lab2, g.src, g.dst, q, ins, want_tuples=True)
        pos2, neg2 = O.totals(c2, ins.op)
        assert neg2 == 0 and _tupset(t2, 1) == {m for m in emb2 if g.n in m}
        assert pos2 == len({m for m in emb2 if g.n in m})


def _is_valid_row(row, q, labels, g_edges, g2_edges, batch):
    """A row (charged update k, sign, phi) of the oracle, checked against the
    definitions directly: phi is injective and label-preserving, every query
    edge maps to an edge of the right view (G' for +, G for -), and k is the
    smallest index among the same-sign updates whose edge is a query-edge image."""
    k, sign = int(row[0]), int(row[1])
    phi = [int(x) for x in row[2:]]
    if len(set(phi)) != q.q or any(labels[phi[u]] != q.labels[u] for u in range(q.q)):
        return False
    view = g2_edges if sign > 0 else g_edges
    images = {(min(phi[a], phi[b]), max(phi[a], phi[b])) for a, b in zip(q.src.tolist(), q.dst.tolist())}
    if not images <= view:
        return False
    same = [i for i in range(len(batch)) if int(batch.op[i]) == sign and
            (min(int(batch.src[i]), int(batch.dst[i])), max(int(batch.src[i]), int(batch.dst[i]))) in images]
    return bool(same) and min(same) == k


BULK_QUERIES = SMALL_QUERIES + [
    I.pattern_query([0, 1, 0, 1, 0], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]),           # 5-cycle
    I.pattern_query([0, 0, 1, 1, 0], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 4)]),   # house
]


def test_incremental_equals_static_difference_bulk():
    """2,000 more random cases (6..12 vertices, 2..3 labels, 1..6 mixed
    updates, queries of 2..5 vertices): the oracle's counts and rows equal the
    static difference, and each row is valid under the definitions."""
    checked = 0
    for trial in range(2000):
        n = 6 + trial % 7
        g = I.random_small_graph(n, 30 + (trial * 7) % 40, 2 + trial % 2, 11, trial)
        b = _random_batch(g, 1000 + trial, 1 + trial % 4, trial % 3)
        if len(b) == 0:
            continue
        ge = {(min(a, c), max(a, c)) for a, c in zip(g.src.tolist(), g.dst.tolist())}
        s2, d2 = I.apply_batch_edges(g.src, g.dst, b)
        g2e = {(min(a, c), max(a, c)) for a, c in zip(s2.tolist(), d2.tolist())}
        for q in BULK_QUERIES:
            pos, neg, _ = O.brute_bdsm(g.n, g.labels, g.src, g.dst, q, b)
            c, tup = O.bdsm(g.n, g.labels, g.src, g.dst, q, b, want_tuples=True)
            assert O.totals(c, b.op) == (len(pos), len(neg))
            assert {(int(r[1]), tuple(int(x) for x in r[2:])) for r in tup} == \
                {(1, p) for p in pos} | {(-1, p) for p in neg}
            for r in tup:
                assert _is_valid_row(r, q, g.labels, ge, g2e, b)
            checked += len(tup)
    assert checked > 5000


def test_multi_query_oracle_with_samples_and_budgets():
    """bdsm_multi, which the full-size GPU tests use, against single-query
    runs: all queries at once give the same per-update charges; a sample of
    updates gives those updates' charges; with a per-(query, update) budget
    every pair it finishes is exact and the rest are marked NOT_COMPUTED."""
    w = I.make_workload("tiny")
    g = w.graph
    b = I.workload_batch(w, 300, 100, sub=9)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)]),
          I.pattern_query([1, 1, 2, 2], [(0, 1), (1, 2), (2, 3), (3, 0)])]
    single = np.stack([O.bdsm(g.n, g.labels, g.src, g.dst, q, b)[0] for q in qs])
    multi = O.bdsm_multi(g.n, g.labels, g.src, g.dst, qs, b)
    assert np.array_equal(multi, single) and int(single.sum()) > 0
    ev = np.array([3, 17, 18, 150, 399])
    assert np.array_equal(O.bdsm_multi(g.n, g.labels, g.src, g.dst, qs, b, eval_idx=ev), single[:, ev])
    tight = O.bdsm_multi(g.n, g.labels, g.src, g.dst, qs, b, update_budget=20)
    done = tight != O.NOT_COMPUTED
    assert 0 < done.sum() < done.size
    assert np.array_equal(tight[done], single[done])
    loose = O.bdsm_multi(g.n, g.labels, g.src, g.dst, qs, b, update_budget=1 << 40)
    assert np.array_equal(loose, single)


def test_incremental_equals_static_difference_property_based():
    """Property-based form of the O2 = O1 pin: Hypothesis draws the graph
    (4..9 vertices, 3 labels), the batch (distinct vertex pairs, each an
    insertion when absent and a deletion when present, in drawn order) and a
    connected query (random tree plus extra edges, 2..5 vertices)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @st.composite
    def case(draw):
        n = draw(st.integers(4, 9))
        labels = draw(st.lists(st.integers(0, 2), min_size=n, max_size=n))
        pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
        present = draw(st.lists(st.booleans(), min_size=len(pairs), max_size=len(pairs)))
        edges = [p for p, x in zip(pairs, present) if x]
        upd = draw(st.lists(st.sampled_from(pairs), min_size=1, max_size=6, unique=True))
        flip = draw(st.lists(st.booleans(), min_size=len(upd), max_size=len(upd)))
        q = draw(st.integers(2, 5))
        qlab = draw(st.lists(st.integers(0, 2), min_size=q, max_size=q))
        parent = [draw(st.integers(0, i - 1)) for i in range(1, q)]
        qe = {(parent[i - 1], i) for i in range(1, q)}
        extra = draw(st.lists(st.tuples(st.integers(0, q - 1), st.integers(0, q - 1)), max_size=3))
        qe |= {(min(a, b), max(a, b)) for a, b in extra if a != b}
        return n, labels, edges, upd, flip, qlab, sorted(qe)

    @hyp.settings(max_examples=400, deadline=None, derandomize=True)
    @hyp.given(case())
    def check(c):
        n, labels, edges, upd, flip, qlab, qe = c
        es = set(edges)
        op = np.array([-1 if p in es else 1 for p in upd], np.int8)
        src = np.array([p[1] if f else p[0] for p, f in zip(upd, flip)], np.int32)
        dst = np.array([p[0] if f else p[1] for p, f in zip(upd, flip)], np.int32)
        b = I.Batch(op, src, dst)
        lab = np.array(labels, np.int32)
        gs = np.array([a for a, _ in edges], np.int32)
        gd = np.array([x for _, x in edges], np.int32)
        query = I.pattern_query(qlab, qe)
        pos, neg, charge = O.brute_bdsm(n, lab, gs, gd, query, b)
        cnt, tup = O.bdsm(n, lab, gs, gd, query, b, want_tuples=True)
        assert O.totals(cnt, b.op) == (len(pos), len(neg))
        assert {(int(r[1]), tuple(int(x) for x in r[2:])) for r in tup} == \
            {(1, p) for p in pos} | {(-1, p) for p in neg}
        for r in tup:
            assert charge[(int(r[1]), tuple(int(x) for x in r[2:]))] == r[0]

    check()


def _labelled_case(trial):
    """A tiny graph with two edge labels, a mixed batch whose insertions carry
    labels (deletions carry the label the edge has), and edge-labelled queries."""
    g = I.random_small_graph(7 + trial % 4, 45, 2, 13, trial)
    r = np.random.default_rng(500 + trial)
    el = r.integers(0, 2, g.src.size).astype(np.int32)
    b = _random_batch(g, 700 + trial, 1 + trial % 4, trial % 3)
    have = {(min(a, c), max(a, c)): l for a, c, l in zip(g.src.tolist(), g.dst.tolist(), el.tolist())}
    bel = np.array([int(r.integers(0, 2)) if o > 0 else have[(min(a, c), max(a, c))]
                    for o, a, c in zip(b.op.tolist(), b.src.tolist(), b.dst.tolist())], np.int32)
    b = I.Batch(b.op, b.src, b.dst, bel)
    qs = []
    for q in SMALL_QUERIES + BULK_QUERIES[-2:]:
        qs.append(I.Query(q.labels, q.src, q.dst, "", r.integers(0, 2, q.eq).astype(np.int32)))
    return g, el, b, qs


def test_edge_labelled_incremental_equals_static_difference():
    """Edge labels (Sec. II-A: the label function also covers edges): O2 with
    edge labels equals the edge-labelled static difference on 600 random
    cases, rows and charges included."""
    checked = 0
    for trial in range(600):
        g, el, b, qs = _labelled_case(trial)
        if len(b) == 0:
            continue
        for q in qs:
            pos, neg, charge = O.brute_bdsm(g.n, g.labels, g.src, g.dst, q, b, elabels=el)
            c, tup = O.bdsm(g.n, g.labels, g.src, g.dst, q, b, want_tuples=True, elabels=el)
            assert O.totals(c, b.op) == (len(pos), len(neg))
            got = {(int(r[1]), tuple(int(x) for x in r[2:])) for r in tup}
            assert got == {(1, p) for p in pos} | {(-1, p) for p in neg}
            for r in tup:
                assert charge[(int(r[1]), tuple(int(x) for x in r[2:]))] == r[0]
            checked += len(tup)
        multi = O.bdsm_multi(g.n, g.labels, g.src, g.dst, qs, b, elabels=el)
        for j, q in enumerate(qs):
            assert np.array_equal(multi[j], O.bdsm(g.n, g.labels, g.src, g.dst, q, b, elabels=el)[0])
    assert checked > 1000


def test_edge_labels_reduce_to_vertex_labels():
    """Closed cases: all edge labels 0 give the unlabelled result; edge labels
    that are a function of the endpoint labels, asked for by the query with
    the same function, give the unlabelled result too, and asking one query
    edge for the other label gives no match at all; a repeated data edge with
    another label is rejected."""
    for trial in range(40):
        g = I.random_small_graph(9, 45, 3, 17, trial)
        b = _random_batch(g, 900 + trial, 3, 1)
        f = lambda a, c: int(g.labels[a] + g.labels[c]) % 2  # noqa: E731
        el = np.array([f(a, c) for a, c in zip(g.src.tolist(), g.dst.tolist())], np.int32)
        bel = np.array([f(a, c) for a, c in zip(b.src.tolist(), b.dst.tolist())], np.int32)
        bl = I.Batch(b.op, b.src, b.dst, bel)
        for q in SMALL_QUERIES:
            plain = O.bdsm(g.n, g.labels, g.src, g.dst, q, b, want_tuples=True)
            zero = O.bdsm(g.n, g.labels, g.src, g.dst,
                          I.Query(q.labels, q.src, q.dst, "", np.zeros(q.eq, np.int32)),
                          I.Batch(b.op, b.src, b.dst, np.zeros(len(b), np.int32)), want_tuples=True,
                          elabels=np.zeros(g.src.size, np.int32))
            assert np.array_equal(plain[0], zero[0]) and np.array_equal(plain[1], zero[1])
            qf = np.array([int(q.labels[a] + q.labels[c]) % 2 for a, c in zip(q.src.tolist(), q.dst.tolist())],
                          np.int32)
            same = O.bdsm(g.n, g.labels, g.src, g.dst, I.Query(q.labels, q.src, q.dst, "", qf), bl,
                          want_tuples=True, elabels=el)
            assert np.array_equal(plain[0], same[0]) and np.array_equal(plain[1], same[1])
            wrong = qf.copy()
            wrong[0] ^= 1
            none = O.bdsm(g.n, g.labels, g.src, g.dst, I.Query(q.labels, q.src, q.dst, "", wrong), bl, elabels=el)
            assert int(none[0].sum()) == 0
    g = I.Graph(4, np.zeros(4, np.int32), np.array([0, 1, 1], np.int32), np.array([1, 2, 0], np.int32))
    with pytest.raises(O.OracleError):
        O.bdsm(g.n, g.labels, g.src, g.dst, SMALL_QUERIES[0], I.Batch(np.ones(1, np.int8),
               np.array([2], np.int32), np.array([3], np.int32)), elabels=np.array([0, 0, 1], np.int32))


def _charges_by_update(charge, b):
    out = np.zeros(len(b), np.uint64)
    for (_, _phi), k in charge.items():
        out[k] += 1
    return out


def test_session_and_parts_equal_static_difference():
    """The oracle session (G, the batch and G' built once, many evaluations)
    and its split of each (query, update) search into parts: on 300 random
    small cases, with and without edge labels, the per-update charges of
    one session equal those of the static difference (O1), and for 2, 3 and
    7 parts the parts' counts add up to them."""
    checked = 0
    for trial in range(300):
        if trial % 2:
            g, el, b, qs = _labelled_case(trial)
        else:
            n = 6 + trial % 7
            g = I.random_small_graph(n, 30 + (trial * 7) % 40, 2 + trial % 2, 13, trial)
            b, el, qs = _random_batch(g, 3000 + trial, 1 + trial % 4, trial % 3), None, BULK_QUERIES
        if len(b) == 0:
            continue
        with O.Session(g.n, g.labels, g.src, g.dst, b, elabels=el) as S:
            whole = S.eval(qs)
            for j, q in enumerate(qs):
                _, _, charge = O.brute_bdsm(g.n, g.labels, g.src, g.dst, q, b, elabels=el)
                assert np.array_equal(whole[j], _charges_by_update(charge, b))
                checked += len(charge)
            for parts in (2, 3, 7):
                split = [S.eval(qs, part=p, parts=parts) for p in range(parts)]
                assert np.array_equal(sum(split), whole)
            ev = np.array([len(b) - 1, 0])
            assert np.array_equal(S.eval(qs, eval_idx=ev), whole[:, ev])
    assert checked > 1000
