"""gamma_recount_noalloc: the DFS re-run over the staged batch with its
scratch in a static device array, for callers that cannot allocate device
memory when they need the counts (an application whose device memory is all
owned by another allocator, or a latency-critical loop that may not pay for
cudaMalloc).  Its counts must equal those that gamma_apply_batch (or
gamma_apply_batches) returned for the same staged batch, on two calls in a
row.  This file is collected last on purpose."""
import ctypes

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


def _queries(g, n, sizes=(4, 5)):
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    att = 0
    while len(qs) < n:
        q = I.random_walk_query(off, nbr, g.labels, sizes[att % len(sizes)], ["dense", "sparse", "tree"][att % 3],
                                13, att)
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


def test_recount_without_allocation_two_requests(G):
    """Two requests staged together: the recount fills request r's counts at
    r * nq + j, as gamma_apply_batches does, and refuses output arrays that
    hold fewer entries than requests x queries."""
    w = I.make_workload("large", scale=14, n_edges=120_000)
    g = w.graph
    b1 = I.workload_batch(w, 2000, 500, sub=1)
    cur = I.apply_batch_edges(g.src, g.dst, b1)
    b2 = I.workload_batch(w, 2000, 500, sub=2, pool_start=2000, cur=cur)
    k1 = set(I.edge_keys(b1.src, b1.dst).tolist())
    keep = np.array([k not in k1 for k in I.edge_keys(b2.src, b2.dst).tolist()])  # requests must not share edges
    b2 = I.Batch(b2.op[keep].copy(), b2.src[keep].copy(), b2.dst[keep].copy())
    op = np.concatenate([b1.op, b2.op])
    src = np.concatenate([b1.src, b2.src])
    dst = np.concatenate([b1.dst, b2.dst])
    off = np.array([0, len(b1), len(b1) + len(b2)], np.int64)
    qs = _queries(g, 5)
    with G.Context(steal_grain=1) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        pos, neg = ctx.apply_batches(off, op, src, dst, qids)  # [request, query]
        pos, neg = pos.reshape(-1), neg.reshape(-1)  # entry r * nq + j, as the recount lays them out
        assert pos.size == 2 * len(qids) and int(pos.sum() + neg.sum()) > 0
        for _ in range(2):
            p2, n2 = G.gamma_recount_noalloc(ctx.h, 2 * len(qids))
            assert np.array_equal(p2, pos) and np.array_equal(n2, neg)
        small = np.zeros(2 * len(qids) - 1, np.uint64)
        lib = G.load_library()
        rc = lib.gamma_recount_noalloc(ctx.h, small.size, small.ctypes.data_as(ctypes.c_void_p),
                                       small.ctypes.data_as(ctypes.c_void_p))
        assert rc == G.GAMMA_EINVAL and not small.any()
        ctx.commit()


def test_recount_without_allocation_with_donation(G):
    """A power-law graph whose hub updates make idle warps take donated work:
    the recount, whose donated-task ring is 64 times smaller than the
    context's, still finishes (a donation that would not fit is not made)
    and gives the apply's counts."""
    w = I.make_workload("large", scale=16, n_edges=600_000)
    g = w.graph
    b = I.workload_batch(w, 8000, 2000)
    qs = _queries(g, 8, sizes=(5, 6))
    with G.Context(steal_grain=4) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids)
        assert ctx.stats()["donated_tasks"] > 0
        for _ in range(2):
            p2, n2 = G.gamma_recount_noalloc(ctx.h, len(qids))
            assert np.array_equal(p2, pos) and np.array_equal(n2, neg)
            assert ctx.stats()["donated_tasks"] > 0
        ctx.commit()
