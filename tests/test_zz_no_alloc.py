"""gamma_recount_noalloc: the DFS re-run over the staged batch with its
scratch in a static device array, for callers that must not allocate (for
example while capturing a CUDA graph in global mode, or when another
allocator owns the device memory).  Its counts must equal those that
gamma_apply_batch returned for the same staged batch, on two calls in a row.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2401_17018_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_17018_gb300 import gamma
    return gamma


def _queries(g, n):
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    att = 0
    while len(qs) < n:
        q = I.random_walk_query(off, nbr, g.labels, 4 + att % 2, ["dense", "sparse", "tree"][att % 3], 13, att)
        att += 1
        if q is not None:
            qs.append(q)
    return qs


@pytest.mark.parametrize("workload,scale,ne,nins,ndel", [("tiny", None, None, 256, 64),
                                                         ("large", 14, 120_000, 3000, 1000)])
def test_recount_without_allocation_matches_apply(G, workload, scale, ne, nins, ndel):
    w = I.make_workload(workload, scale=scale, n_edges=ne)
    g = w.graph
    b = I.workload_batch(w, nins, ndel)
    qs = _queries(g, 6)
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids)
        assert int(pos.sum() + neg.sum()) > 0
        for _ in range(2):  # the static scratch keeps the previous call's contents
            p2, n2 = G.gamma_recount_noalloc(ctx.h, len(qids))
            assert np.array_equal(p2, pos) and np.array_equal(n2, neg)
        ctx.commit()
