"""Host-side checks of the seeded input generators (no GPU, no oracle).

The generators feed both the CUDA path and the oracle, so they must be
deterministic, produce valid batches in sequence, and give queries of the
class they were asked for.
"""
import numpy as np
import pytest

from paper_2401_17018_gb300 import inputs as I


def test_workload_is_deterministic_and_canonical():
    a = I.make_workload("served", scale=12, n_edges=20_000)
    b = I.make_workload("served", scale=12, n_edges=20_000)
    assert a.graph.digest() == b.graph.digest()
    g = a.graph
    assert np.all(g.src < g.dst)  # canonical (min, max), no self-loops
    k = I.edge_keys(np.concatenate([g.src, a.pool_src]), np.concatenate([g.dst, a.pool_dst]))
    assert np.unique(k).size == k.size == 20_000  # unique edges, exact count
    assert a.pool_src.size == round(0.1 * 20_000)


def test_sample_distinct_is_a_sample_without_replacement():
    x = I.sample_distinct(50, 50, 3, 7)
    assert sorted(x.tolist()) == list(range(50))
    y = I.sample_distinct(10_000, 2_000, 3, 7, 1)
    assert np.unique(y).size == 2_000 and y.min() >= 0 and y.max() < 10_000
    assert np.array_equal(y, I.sample_distinct(10_000, 2_000, 3, 7, 1))
    # roughly uniform: each tenth of the range gets about a tenth of the draws
    h = np.bincount(y // 1_000, minlength=10)
    assert np.all(np.abs(h - 200) < 60)
    with pytest.raises(ValueError):
        I.sample_distinct(5, 6, 1, 1)


def _replay(w, batches):
    keys = set(I.edge_keys(w.graph.src, w.graph.dst).tolist())
    for b in batches:
        k = I.edge_keys(b.src, b.dst).tolist()
        assert len(set(k)) == len(k)
        assert np.all(b.src != b.dst)
        for kk, o in zip(k, b.op.tolist()):
            if o > 0:
                assert kk not in keys
                keys.add(kk)
            else:
                assert kk in keys
                keys.remove(kk)
    return keys


def test_served_stream_batches_are_valid_in_order():
    w = I.make_workload("served", scale=13, n_edges=60_000)
    stream = I.served_stream(w, 6, w.seed, 2.0, 3.5)
    sizes = I.served_sizes(6, w.seed, 2.0, 3.5)
    assert [len(b) for b in stream] == sizes.tolist()
    assert all(100 <= s < 3163 for s in sizes)
    assert all(1_000 <= s < 1_000_000 for s in I.served_sizes(2_000, w.seed))
    for b in stream:  # insertions : deletions = 1 : 1 (the odd one is an insertion)
        ni = int((b.op > 0).sum())
        assert ni - (len(b) - ni) in (0, 1)
    _replay(w, stream)


def test_workload_batch_and_apply_agree():
    w = I.make_workload("mid", scale=12, n_edges=30_000)
    b = I.workload_batch(w, 900, 100)
    after = _replay(w, [b])
    s, d = I.apply_batch_edges(w.graph.src, w.graph.dst, b)
    assert set(I.edge_keys(s, d).tolist()) == after


@pytest.mark.parametrize("kind", ["tree", "dense", "dense_ge3", "sparse"])
def test_extracted_queries_have_their_class(kind):
    w = I.make_workload("mid", scale=12, n_edges=40_000)
    g = w.graph
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    got = 0
    for att in range(60):
        q = I.random_walk_query(off, nbr, g.labels, 6, kind, 5, att)
        if q is None:
            continue
        got += 1
        nq, ne = q.labels.size, q.src.size
        assert nq == 6
        avg = 2.0 * ne / nq
        if kind == "tree":
            assert ne == nq - 1
        elif kind == "dense":
            assert avg > 3
        elif kind == "dense_ge3":
            assert avg >= 3
        else:
            assert avg <= 3 and ne >= nq  # sparse: has a cycle
        # connected, and every query edge is an edge of the data graph between the stored labels
        adj = {i: set() for i in range(nq)}
        for a, b in zip(q.src.tolist(), q.dst.tolist()):
            adj[a].add(b)
            adj[b].add(a)
        seen, todo = {0}, [0]
        while todo:
            for v in adj[todo.pop()]:
                if v not in seen:
                    seen.add(v)
                    todo.append(v)
        assert len(seen) == nq
    assert got > 0


def test_edge_labels_follow_the_edge_not_its_position():
    w = I.make_workload("mid", scale=12, n_edges=30_000)
    g = w.graph
    el = I.edge_labels(g.src, g.dst, 4, 3, 1.2)
    # same edge, other orientation or position: same label
    assert np.array_equal(el, I.edge_labels(g.dst[::-1][::-1], g.src, 4, 3, 1.2))
    perm = np.random.default_rng(1).permutation(g.src.size)
    assert np.array_equal(el[perm], I.edge_labels(g.src[perm], g.dst[perm], 4, 3, 1.2))
    # Zipf(1.2) over 4 labels: label 0 most frequent, every label used
    h = np.bincount(el, minlength=4)
    assert h.argmax() == 0 and h.min() > 0 and el.max() < 4
    u = np.bincount(I.edge_labels(g.src, g.dst, 4, 3), minlength=4) / g.src.size
    assert np.all(np.abs(u - 0.25) < 0.02)


def test_c_rmat_draw_gives_the_numpy_bytes():
    """rmat_gen.c is the numpy R-MAT draw in C: the same edge lists, byte for
    byte, on several scales and seeds (including the tiny workload's graph)."""
    for scale, ne, seed in [(6, 100, 1), (11, 10_000, 1), (13, 50_000, 4), (15, 200_000, 2)]:
        a = I.rmat_edges(scale, ne, seed, engine="c")
        b = I.rmat_edges(scale, ne, seed, engine="numpy")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_consecutive_batches_are_valid_in_order():
    """Each of the consecutive batches is valid on the graph the previous ones
    leave: insertions absent, deletions present, no edge repeated."""
    w = I.make_workload("large", scale=12, n_edges=40_000)
    bs = I.consecutive_batches(w, 4, 800, 300)
    cur = {(int(a), int(b)) for a, b in zip(w.graph.src, w.graph.dst)}
    for b in bs:
        keys = [(min(int(x), int(y)), max(int(x), int(y))) for x, y in zip(b.src, b.dst)]
        assert len(set(keys)) == len(keys) and len(b) == 1100
        for o, k in zip(b.op, keys):
            assert (k in cur) == (o < 0)
        for o, k in zip(b.op, keys):
            (cur.discard if o < 0 else cur.add)(k)
