"""Parity at the benchmark's full sizes.

At these sizes the oracle cannot enumerate everything, so the CUDA path is
checked on every pair of each query's check set -- a uniform sample of the
batch's updates and the updates whose endpoint labels match one of the
query's edges with the largest endpoint-degree product, which carry most of
the query's work on a power-law graph -- against per-update charged counts
the oracle computed without any budget (tests/golden/make_expected.py, which
calls only the oracle; no pair is skipped), and on properties that hold at
any size: totals are the sums of the per-update charges split by sign, and
the inverse batch applied to G' swaps the positive and negative totals.
"""
import json
import os
import sys

import numpy as np
import pytest

from paper_2401_17018_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLD)
import make_expected as ME  # noqa: E402  (batch construction only; the oracle is not run here)

# a bound on the DFS work of one apply (32-wide expansion steps, about a
# minute of GPU time): a workload heavier than intended fails with
# GAMMA_ETIMEOUT instead of running for an hour
WORK_BUDGET = 100_000_000_000


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_17018_gb300 import gamma
    return gamma


def _stored(name):
    if not os.path.exists(os.path.join(GOLD, "expected_%s.json" % name)):
        pytest.skip("no stored oracle counts for the %s workload (tests/golden/make_expected.py %s)" % (name, name))
    with open(os.path.join(GOLD, "queries_%s.json" % name)) as f:
        qd = json.load(f)
    with open(os.path.join(GOLD, "expected_%s.json" % name)) as f:
        ex = json.load(f)
    assert ex["queries_digest"] == ME.file_digest(os.path.join(GOLD, "queries_%s.json" % name)), \
        "expected values were computed for another query set"
    return [I.Query.from_json(x) for x in qd["queries"]], ex


def _compare(per, batch_expect, nq):
    """Every stored (query, update, count) equals the GPU's per-update charge."""
    j = np.array(batch_expect["query"], np.int64)
    u = np.array(batch_expect["update"], np.int64)
    want = np.array(batch_expect["count"], np.uint64)
    heavy = np.array(batch_expect["heavy"], bool)
    assert j.max() < nq
    got = per[j, u]
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, "first mismatches (query, update, gpu, oracle): %s" % [
        (int(j[i]), int(u[i]), int(got[i]), int(want[i])) for i in bad[:8]]
    return int(want.size), int(heavy.sum()), int(want[heavy].sum())


def _run_batches(G, name, flags=0):
    import torch
    queries, ex = _stored(name)
    w = I.make_workload(ME.MQ.SPECS[name]["workload"])
    assert ex["graph_digest"] == w.graph.digest()
    batches = ME.applied_batches(name, w)
    g = w.graph
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pairs = heavy = heavy_matches = 0
    totals = []
    with G.Context(flags=flags | G.GAMMA_F_PER_UPDATE, stream=torch.cuda.Stream(), work_budget=WORK_BUDGET) as ctx:
        ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        for k, b in enumerate(batches):
            pos, neg = ctx.apply_batch(dev(b.op), dev(b.src), dev(b.dst), qids)
            per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
            ins = b.op > 0
            assert np.array_equal(per[:, ins].sum(axis=1), pos) and np.array_equal(per[:, ~ins].sum(axis=1), neg)
            n, h, hm = _compare(per, ex["batches"][k], len(queries))
            pairs, heavy, heavy_matches = pairs + n, heavy + h, heavy_matches + hm
            totals.append((pos.copy(), neg.copy()))
            if len(batches) == 1:  # the inverse batch swaps the totals
                ctx.commit()
                inv = b.inverse()
                p2, n2 = ctx.apply_batch(dev(inv.op), dev(inv.src), dev(inv.dst), qids)
                assert np.array_equal(p2, neg) and np.array_equal(n2, pos)
            ctx.commit()
        st = ctx.stats()
    print("%s: %d (query, update) pairs equal the oracle's, %d of them heavy with %d matches" % (
        name, pairs, heavy, heavy_matches))
    return batches, totals, st, pairs, heavy


def test_large_workload_five_batches(G):
    """The headline workload: the scale-23 graph (60.4M edges, 16 labels) and
    its eight 6-vertex queries (4 sparse, 4 dense), five consecutive batches of 800,000
    insertions and 200,000 deletions, each committed before the next."""
    batches, totals, st, pairs, heavy = _run_batches(G, "large")
    assert heavy > 0 and sum(int(p.sum() + n.sum()) for p, n in totals) > 0
    w = I.make_workload("large")
    src, dst = I.graph_after(w.graph.src, w.graph.dst, batches)
    assert st["live_edges"] == 2 * src.size  # directed entries


def test_mid_workload(G):
    """The mid workload: scale-20 R-MAT, 20 six-vertex queries, 100k updates."""
    _, totals, _, pairs, heavy = _run_batches(G, "mid")
    assert heavy > 0 and int(totals[0][0].sum() + totals[0][1].sum()) > 0


def test_batched_workload(G):
    """The batched workload: the mid graph and batch with 64 queries of 4..7
    vertices (38 sparse of 4..6, 26 dense of 4..7), in the batched form
    replayed as a CUDA graph, its work created query by query."""
    queries, _ = _stored("batched")
    assert len(queries) == 64 and {q.q for q in queries} == set(range(4, 8))
    _, totals, _, pairs, heavy = _run_batches(G, "batched", flags=G.GAMMA_F_GRAPH | G.GAMMA_F_SEED_BY_QUERY)
    assert heavy > 0


def test_served_workload(G):
    """The served workload's first requests on the scale-22 graph: applied one
    after another they match the oracle on every check pair; through the
    server (continuous batching: the first two requests, staged together as
    one group) each request gets the same counts.  The work budget bounds
    one apply, and a group is one apply, so the server's context gets the
    budget of every request it may group."""
    batches, totals, _, pairs, heavy = _run_batches(G, "served")
    queries, _ = _stored("served")
    w = I.make_workload("served")
    g = w.graph
    reqs = batches[:2]
    with G.Context(work_budget=WORK_BUDGET * (len(reqs) + 1)) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        srv = G.Server(ctx, qids, max_requests=len(reqs))
        tickets = [srv.submit(b.op, b.src, b.dst) for b in reqs]
        for t, (p, n) in zip(tickets, totals):
            rc, pos, neg, info = srv.wait(t)
            assert rc == G.GAMMA_OK
            assert np.array_equal(pos, p) and np.array_equal(neg, n)
        srv.stop()
