"""Parity at the benchmark's full sizes, on sampled outputs.

At these sizes the oracle cannot enumerate everything, so the CUDA path is
checked (a) on the per-update charged counts of a seeded sample of updates,
which the oracle computes one by one (pairs that would need more than a fixed
number of candidate tests are skipped, a rule that depends only on the oracle),
and (b) on properties that hold at any size: totals are the sums of the
per-update charges split by sign, and the inverse batch applied to G' swaps
the positive and negative totals.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_17018_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
# a bound on the DFS work of one apply (32-wide expansion steps, about 20 s of
# GPU time): a workload heavier than intended fails with GAMMA_ETIMEOUT
# instead of running for an hour
WORK_BUDGET = 30_000_000_000


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_17018_gb300 import gamma
    return gamma


def _load_queries(name, w):
    path = os.path.join(GOLD, "queries_%s.json" % name)
    if not os.path.exists(path):  # written by tests/golden/make_queries.py NAME
        pytest.skip("queries_%s.json has not been selected" % name)
    with open(path) as f:
        d = json.load(f)
    assert d["graph_digest"] == w.graph.digest()
    return [I.Query.from_json(x) for x in d["queries"]]


def _sample(b, k, seed):
    return np.sort(np.argsort(I.rand_u64(seed, 77, np.arange(b, dtype=np.uint64)))[:k])


def _check_workload(G, w, queries, batch, n_sample, update_budget, flags=0):
    import torch
    g = w.graph
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with G.Context(flags=flags | G.GAMMA_F_PER_UPDATE, stream=torch.cuda.Stream(), work_budget=WORK_BUDGET) as ctx:
        ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        pos, neg = ctx.apply_batch(dev(batch.op), dev(batch.src), dev(batch.dst), qids)
        per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
        ctx.commit()
        inv = batch.inverse()
        pos2, neg2 = ctx.apply_batch(dev(inv.op), dev(batch.src), dev(batch.dst), qids)
        ctx.commit()
    ins = batch.op > 0
    assert np.array_equal(per[:, ins].sum(axis=1), pos) and np.array_equal(per[:, ~ins].sum(axis=1), neg)
    assert np.array_equal(pos2, neg) and np.array_equal(neg2, pos)
    ev = _sample(len(batch), n_sample, 5)
    want = O.bdsm_multi(g.n, g.labels, g.src, g.dst, queries, batch, eval_idx=ev, update_budget=update_budget)
    done = want != O.NOT_COMPUTED
    assert done.mean() >= 0.5, "the oracle finished too few sampled pairs"
    got = per[:, ev]
    assert np.array_equal(got[done], want[done])
    return int(done.sum()), int(pos.sum() + neg.sum())


def test_mid_workload_fullsize_sampled(G):
    """The bench workload: scale-20 R-MAT, 20 six-vertex queries, 100k updates."""
    w = I.make_workload("mid")
    queries = _load_queries("mid", w)
    batch = I.workload_batch(w, 90_000, 10_000)
    checked, total = _check_workload(G, w, queries, batch, n_sample=32, update_budget=2_000_000)
    assert checked >= 320 and total > 0


def test_batched_workload_fullsize_sampled(G):
    """The batched workload: the mid graph and batch with 64 queries of 4..8
    vertices, in the batched form replayed as a CUDA graph."""
    w = I.make_workload("mid")
    queries = _load_queries("batched", w)
    assert len(queries) == 64
    batch = I.workload_batch(w, 90_000, 10_000)
    checked, total = _check_workload(G, w, queries, batch, n_sample=8, update_budget=1_000_000,
                                     flags=G.GAMMA_F_GRAPH)
    assert checked >= 256 and total > 0


def test_served_workload_fullsize_sampled(G):
    """The served workload: the first three requests of the served stream on
    the scale-22 graph.  Through the server each request gets the counts of
    applying the requests one after another; those equal the sums of the
    per-update charges, which the oracle checks on sampled updates against
    the graph each request meets."""
    import torch
    w = I.make_workload("served")
    queries = _load_queries("served", w)
    stream = I.served_stream(w, 3, w.seed)
    g = w.graph
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    alone, per = [], []
    with G.Context(flags=G.GAMMA_F_PER_UPDATE, work_budget=WORK_BUDGET) as ctx:
        ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        for b in stream:
            pos, neg = ctx.apply_batch(dev(b.op), dev(b.src), dev(b.dst), qids)
            per.append(np.stack([ctx.update_counts(j) for j in range(len(qids))]))
            alone.append((pos.tolist(), neg.tolist()))
            ctx.commit()
    with G.Context(work_budget=WORK_BUDGET) as ctx:
        ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        srv = G.Server(ctx, qids, max_requests=8)
        tickets = [srv.submit(b.op, b.src, b.dst) for b in stream]
        served = []
        for t in tickets:
            rc, pos, neg, info = srv.wait(t)
            assert rc == G.GAMMA_OK
            served.append((pos.tolist(), neg.tolist()))
        srv.stop()
    assert served == alone
    cur = (g.src, g.dst)
    checked = 0
    for k, b in enumerate(stream):
        ins = b.op > 0
        assert per[k][:, ins].sum(axis=1).tolist() == alone[k][0]
        assert per[k][:, ~ins].sum(axis=1).tolist() == alone[k][1]
        ev = _sample(len(b), 8, 11 + k)
        want = O.bdsm_multi(g.n, g.labels, cur[0], cur[1], queries, b, eval_idx=ev, update_budget=2_000_000)
        done = want != O.NOT_COMPUTED
        assert done.mean() >= 0.5
        assert np.array_equal(per[k][:, ev][done], want[done])
        checked += int(done.sum())
        cur = I.apply_batch_edges(cur[0], cur[1], b)
    assert checked >= 3 * 8 * 16 // 2


def test_large_workload_five_batches_sampled(G):
    """The large workload: the scale-23 graph (60.4M edges, 16 labels) and its
    8 queries, five consecutive batches of 800,000 insertions from the pool
    and 200,000 deletions from the current graph, with a commit after each.
    Every batch: totals split by sign equal the per-update charges, which the
    oracle checks on sampled updates against the graph that batch meets."""
    import torch
    w = I.make_workload("large")
    queries = _load_queries("large", w)
    g = w.graph
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cur = (g.src, g.dst)
    checked, total = 0, 0
    with G.Context(flags=G.GAMMA_F_PER_UPDATE, work_budget=WORK_BUDGET) as ctx:
        ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        for k in range(5):
            b = I.workload_batch(w, 800_000, 200_000, sub=k, pool_start=800_000 * k, cur=cur)
            pos, neg = ctx.apply_batch(dev(b.op), dev(b.src), dev(b.dst), qids)
            per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
            ctx.commit()
            ins = b.op > 0
            assert np.array_equal(per[:, ins].sum(axis=1), pos) and np.array_equal(per[:, ~ins].sum(axis=1), neg)
            ev = _sample(len(b), 4, 30 + k)
            want = O.bdsm_multi(g.n, g.labels, cur[0], cur[1], queries, b, eval_idx=ev, update_budget=2_000_000)
            done = want != O.NOT_COMPUTED
            assert done.mean() >= 0.5
            assert np.array_equal(per[:, ev][done], want[done])
            checked += int(done.sum())
            total += int(pos.sum() + neg.sum())
            cur = I.apply_batch_edges(cur[0], cur[1], b)
        st = ctx.stats()
    assert checked >= 5 * 4 * len(queries) // 2
    assert st["live_edges"] == 2 * cur[0].size  # directed entries
