"""Work donation under oracle comparison.  The DFS kernel's idle warps take
work that busy warps split off (the load balancing of Sec. V-A, here
grid-wide); the split must not change a single count.  A scaled-down
power-law graph of the large workload's shape, whose hub updates leave some
warps with far more work than others, is matched with small work items
(steal_grain 1) so that warps run dry early and take donated work; the test
checks that donation happened and that every update's charged count equals
the oracle's, for every query."""
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


def _queries(g, n, seed):
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    qs, att = [], 0
    while len(qs) < n:
        kind = ["sparse", "dense_ge3", "tree"][att % 3]
        q = I.random_walk_query(off, nbr, g.labels, 4 + att % 2, kind, seed, att)
        att += 1
        if q is not None:
            qs.append(q)
    return qs


@pytest.mark.parametrize("tile,flags", [(64, 0), (32, 0x20)])
def test_donated_work_gives_the_oracle_counts(G, tile, flags):
    w = I.make_workload("large", scale=14, n_edges=150_000)
    g = w.graph
    b = I.workload_batch(w, 1500, 500, sub=3)
    qs = _queries(g, 6, 23)
    with G.Context(flags=G.GAMMA_F_PER_UPDATE | flags, steal_grain=1, frontier_tile=tile) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids)
        st = ctx.stats()
        per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
        ctx.commit()
    assert st["donated_tasks"] > 0, "no work was donated; the case does not exercise donation"
    want = O.bdsm_multi(g.n, g.labels, g.src, g.dst, qs, b)
    assert np.array_equal(per, want)
    ins = b.op > 0
    assert np.array_equal(want[:, ins].sum(axis=1), pos) and np.array_equal(want[:, ~ins].sum(axis=1), neg)
    assert int(want.sum()) > 0
