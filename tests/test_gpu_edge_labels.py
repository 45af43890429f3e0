"""Edge labels on the CUDA path (Sec. II-A: the label function covers edges
too; the paper's NF and LS datasets, Table II, are edge-labelled).  An
embedding must map every query edge onto a data edge of the same label; an
insertion carries its label, a deletion removes the edge whatever its label.
The GPU's per-update charges and match rows are compared with the
edge-labelled oracle (pinned on the CPU against the edge-labelled static
difference)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_17018_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_17018_gb300 import gamma
    return gamma


def _run(G, g, el, qs, b, rows=True, flags=0, **opts):
    with G.Context(flags=flags | G.GAMMA_F_PER_UPDATE, **opts) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst, el)
        qids = [ctx.register_query(q.labels, q.src, q.dst, q.elabels) for q in qs]
        if rows:
            pos, neg, r, req = ctx.apply_batch(b.op, b.src, b.dst, qids, row_capacity=1 << 20, elab=b.elab)
            assert req == len(r)
        else:
            pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids, elab=b.elab)
            r = None
        per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
        ctx.commit()
    return pos, neg, per, r


def _labelled_case(trial):
    """A small random graph with two or three edge labels, a mixed batch whose
    insertions carry labels, and random connected queries with edge labels."""
    r = np.random.default_rng(4000 + trial)
    n = int(r.integers(8, 30))
    g = I.random_small_graph(n, int(r.integers(20, 60)), int(r.integers(1, 3)), 21, trial)
    nel = int(r.integers(2, 4))
    el = r.integers(0, nel, g.src.size).astype(np.int32)
    es = set(zip(g.src.tolist(), g.dst.tolist()))
    non = [(a, c) for a in range(n) for c in range(a + 1, n) if (a, c) not in es]
    ni = min(len(non), int(r.integers(1, 15)))
    nd = min(len(es), int(r.integers(0, 8)))
    ins = [non[i] for i in r.choice(len(non), ni, replace=False)] if ni else []
    dl = [sorted(es)[i] for i in r.choice(len(es), nd, replace=False)] if nd else []
    ed = ins + dl
    perm = r.permutation(len(ed))
    op = np.array([1 if i < ni else -1 for i in perm], np.int8)
    src = np.array([ed[i][0] for i in perm], np.int32)
    dst = np.array([ed[i][1] for i in perm], np.int32)
    have = {(int(a), int(c)): int(l) for a, c, l in zip(g.src, g.dst, el)}
    bel = np.array([int(r.integers(0, nel)) if o > 0 else have[(min(a, c), max(a, c))]
                    for o, a, c in zip(op.tolist(), src.tolist(), dst.tolist())], np.int32)
    b = I.Batch(op, src, dst, bel)
    nl = int(g.labels.max()) + 1
    qs = []
    for _ in range(4):
        q = int(r.integers(2, 6))
        edges = [(i, int(r.integers(0, i))) for i in range(1, q)]
        for _ in range(int(r.integers(0, 3))):
            a, c = sorted(r.choice(q, 2, replace=False).tolist())
            if (a, c) not in edges and (c, a) not in edges:
                edges.append((a, c))
        pq = I.pattern_query(r.integers(0, nl, q).tolist(), edges)
        qs.append(I.Query(pq.labels, pq.src, pq.dst, "", r.integers(0, nel, pq.eq).astype(np.int32)))
    return g, el, b, qs


@pytest.mark.parametrize("trial", range(24))
def test_fuzz_edge_labelled_graphs(G, trial):
    g, el, b, qs = _labelled_case(trial)
    rows = trial % 2 == 0
    pos, neg, per, r = _run(G, g, el, qs, b, rows=rows, steal_grain=[1, 3, 64][trial % 3])
    for j, q in enumerate(qs):
        c, t = O.bdsm(g.n, g.labels, g.src, g.dst, q, b, want_tuples=rows, elabels=el)
        assert np.array_equal(per[j], c), "query %d" % j
        assert (int(pos[j]), int(neg[j])) == O.totals(c, b.op)
        if rows:
            got = sorted((int(x[1]), int(x[2])) + tuple(int(v) for v in x[3:3 + q.q]) for x in r if x[0] == j)
            want = sorted((int(x[0]), int(x[1])) + tuple(int(v) for v in x[2:]) for x in t)
            assert got == want, "rows of query %d" % j


def test_power_law_graph_with_edge_labels_over_three_batches(G):
    """A power-law graph of the large workload's shape with three edge labels
    (a function of the edge, so an edge keeps its label wherever it appears),
    random-walk queries with edge labels, three consecutive batches with commits (labels move with relocated
    lists and survive commit): per-update charges equal the oracle's."""
    w = I.make_workload("large", scale=13, n_edges=80_000)
    g = w.graph
    lab = lambda s, d: I.edge_labels(s, d, 3, 5)
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    qs, att = [], 0
    while len(qs) < 6:
        q = I.random_walk_query(off, nbr, g.labels, 4 + att % 2, ["dense_ge3", "sparse", "tree"][att % 3], 31, att)
        att += 1
        if q is not None:  # query edge labels cycle through 0, 1, 2
            qs.append(I.Query(q.labels, q.src, q.dst, q.kind, (np.arange(q.eq) % 3).astype(np.int32)))
    batches = I.consecutive_batches(w, 3, 1500, 500)
    cs, cd = g.src, g.dst
    with G.Context(flags=G.GAMMA_F_PER_UPDATE, steal_grain=4) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst, lab(g.src, g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst, q.elabels) for q in qs]
        total = 0
        for b in batches:
            bel = lab(b.src, b.dst)
            bb = I.Batch(b.op, b.src, b.dst, bel)
            pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids, elab=bel)
            per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
            ctx.commit()
            want = O.bdsm_multi(g.n, g.labels, cs, cd, qs, bb, elabels=lab(cs, cd))
            assert np.array_equal(per, want)
            total += int(want.sum())
            cs, cd = I.apply_batch_edges(cs, cd, b)
    assert total > 0


def test_unlabelled_queries_on_a_labelled_graph_use_label_zero(G):
    """A query registered without edge labels asks for label 0 on every edge;
    on a graph without edge labels a query edge labelled 1 has no image."""
    g, el, b, qs = _labelled_case(3)
    plain = [I.Query(q.labels, q.src, q.dst) for q in qs]
    pos, neg, per, _ = _run(G, g, el, plain, b, rows=False)
    want = O.bdsm_multi(g.n, g.labels, g.src, g.dst, [I.Query(q.labels, q.src, q.dst, "", np.zeros(q.eq, np.int32))
                                                      for q in qs], b, elabels=el)
    assert np.array_equal(per, want)
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        q = qs[0]
        qid = ctx.register_query(q.labels, q.src, q.dst, np.ones(q.eq, np.int32))
        pos, neg = ctx.apply_batch(b.op, b.src, b.dst, [qid])
        assert int(pos[0]) == 0 and int(neg[0]) == 0
        ctx.commit()


def test_edge_label_errors(G):
    """Insertion labels on an unlabelled graph, a repeated edge with two labels,
    a label outside [0, 255], and several requests on a labelled graph are
    rejected with GAMMA_EINVAL; a rejected batch leaves the graph unchanged."""
    g, el, b, qs = _labelled_case(5)
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        with pytest.raises(G.GammaError) as e:
            ctx.apply_batch(b.op, b.src, b.dst, [], elab=b.elab)
        assert e.value.code == G.GAMMA_EINVAL
    with G.Context() as ctx:
        s2 = np.concatenate([g.src, g.src[:1]])
        d2 = np.concatenate([g.dst, g.dst[:1]])
        e2 = np.concatenate([el, (el[:1] + 1) % 3]).astype(np.int32)
        with pytest.raises(G.GammaError) as e:
            ctx.load_graph(g.n, g.labels, s2, d2, e2)
        assert e.value.code == G.GAMMA_EINVAL
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst, el)
        before = ctx.export_adjacency(g.n)
        bad = b.elab.copy()
        k = int(np.flatnonzero(b.op > 0)[0])
        bad[k] = 300
        with pytest.raises(G.GammaError) as e:
            ctx.apply_batch(b.op, b.src, b.dst, [], elab=bad)
        assert e.value.code == G.GAMMA_EINVAL and ("update %d " % k) in str(e.value)
        after = ctx.export_adjacency(g.n)
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        with pytest.raises(G.GammaError) as e:
            ctx.apply_batches(np.array([0, 1, len(b)]), b.op, b.src, b.dst, [])
        assert e.value.code == G.GAMMA_EINVAL
