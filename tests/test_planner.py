"""The host planner (matching order, Alg. 1 input pi; Sec. IV-C) on the CPU.

Checks, for random connected queries of 2..16 vertices and every seeded edge
and orientation, that the order the library uses is valid (a permutation
starting with the seeded edge, every later vertex with a placed neighbour,
the backward masks equal to the query's adjacency) and follows its stated
preference: most placed neighbours, then higher degree, then the rarer data
label, then the smaller id.
"""
import numpy as np
import pytest

from paper_2401_17018_gb300 import gamma as G


def _random_connected(q, rng, n_labels=4):
    edges = {(int(rng.integers(0, i)), i) for i in range(1, q)}  # a random tree
    for _ in range(int(rng.integers(0, q + 2))):
        a, b = sorted(int(x) for x in rng.choice(q, 2, replace=False))
        edges.add((a, b))
    e = sorted(edges)
    return (rng.integers(0, n_labels, q).astype(np.int32), np.array([a for a, _ in e], np.int32),
            np.array([b for _, b in e], np.int32))


def _expected_order(lab, src, dst, a, b, freq):
    q = lab.size
    adj = np.zeros((q, q), bool)
    adj[src, dst] = adj[dst, src] = True
    deg = adj.sum(1)
    order = [a, b]
    while len(order) < q:
        cands = [u for u in range(q) if u not in order and adj[u, order].any()]
        key = lambda u: (int(adj[u, order].sum()), int(deg[u]), -int(freq[lab[u]]), -u)  # noqa: E731
        order.append(max(cands, key=key))
    return order, adj


@pytest.mark.parametrize("seed", range(30))
def test_plan_order_is_valid_and_follows_its_preferences(seed):
    rng = np.random.default_rng(seed)
    q = 2 + seed % 15
    lab, src, dst = _random_connected(q, rng)
    freq = rng.integers(1, 1000, 4).astype(np.int64)
    for a0, b0 in zip(src.tolist(), dst.tolist()):
        for a, b in ((a0, b0), (b0, a0)):
            order, bwd = G.gamma_plan_order(lab, src, dst, a, b, freq)
            want, adj = _expected_order(lab, src, dst, a, b, freq)
            assert order.tolist() == want
            assert sorted(order.tolist()) == list(range(q))
            for l in range(q):
                mask = sum(1 << k for k in range(l) if adj[order[l], order[k]])
                assert int(bwd[l]) == mask
                if l >= 2:
                    assert mask != 0


def test_plan_order_rejects_bad_queries():
    lab = np.zeros(4, np.int32)
    with pytest.raises(G.GammaError):  # disconnected
        G.gamma_plan_order(lab, np.array([0, 2], np.int32), np.array([1, 3], np.int32), 0, 1)
    with pytest.raises(G.GammaError):  # (0, 2) is not a query edge
        G.gamma_plan_order(lab, np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32), 0, 2)
    with pytest.raises(G.GammaError):  # repeated edge
        G.gamma_plan_order(lab[:2], np.array([0, 1], np.int32), np.array([1, 0], np.int32), 0, 1)
    order, bwd = G.gamma_plan_order(lab[:2], np.array([0], np.int32), np.array([1], np.int32), 1, 0)
    assert order.tolist() == [1, 0] and bwd.tolist() == [0, 1]
