"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Counts, per-update charges and sorted match rows must agree bit for bit
(everything on the path is integer).  Inputs are seeded and synthetic.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_17018_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_17018_gb300 import gamma
    return gamma


def gpu_run(G, graph, queries, batch, flags=0, rows=True, **opts):
    """Apply one batch on a fresh context; returns counts, per-update counts, rows."""
    with G.Context(flags=flags | G.GAMMA_F_PER_UPDATE, **opts) as ctx:
        ctx.load_graph(graph.n, graph.labels, graph.src, graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        if rows:
            pos, neg, r, req = ctx.apply_batch(batch.op, batch.src, batch.dst, qids, row_capacity=1 << 22)
            assert req == len(r)
        else:
            pos, neg = ctx.apply_batch(batch.op, batch.src, batch.dst, qids)
            r = None
        per = [ctx.update_counts(j) for j in range(len(qids))]
        st = ctx.stats()
        ctx.commit()
    return pos, neg, per, r, st


def oracle_run(graph, q, batch, rows=True):
    c, t = O.bdsm(graph.n, graph.labels, graph.src, graph.dst, q, batch, want_tuples=rows)
    return c, t


def rowset(r, qid):
    return sorted((int(x[1]), int(x[2])) + tuple(int(v) for v in x[3:]) for x in r if x[0] == qid)


def orowset(t, q):
    return sorted((int(x[0]), int(x[1])) + tuple(int(v) for v in x[2:]) for x in t)


def check(G, graph, queries, batch, rows=True, flags=0, **opts):
    pos, neg, per, r, st = gpu_run(G, graph, queries, batch, flags=flags, rows=rows, **opts)
    for j, q in enumerate(queries):
        c, t = oracle_run(graph, q, batch, rows)
        assert (int(pos[j]), int(neg[j])) == O.totals(c, batch.op), f"query {j}"
        assert np.array_equal(per[j], c), f"per-update counts, query {j}"
        if rows:
            got = [x[:2 + q.q] for x in rowset(r, j)]
            assert got == orowset(t, q), f"rows, query {j}"
    return pos, neg, st


def _golden_running():
    with open(os.path.join(GOLD, "running_example.json")) as f:
        d = json.load(f)
    e = np.array(d["edges"], np.int32)
    g = I.Graph(d["n"], np.array(d["labels"], np.int32), e[:, 0].copy(), e[:, 1].copy())
    q = I.pattern_query(d["query"]["labels"], [tuple(x) for x in d["query"]["edges"]])
    b = I.Batch(np.array(d["batch"]["op"], np.int8), np.array(d["batch"]["src"], np.int32),
                np.array(d["batch"]["dst"], np.int32))
    return d, g, q, b


def test_running_example(G):
    d, g, q, b = _golden_running()
    pos, neg, _ = check(G, g, [q], b)
    assert (int(pos[0]), int(neg[0])) == (d["bdsm"]["pos"], d["bdsm"]["neg"])


def test_running_example_csm_sequence(G):
    d, g, q, b = _golden_running()
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qid = ctx.register_query(q.labels, q.src, q.dst)
        got = []
        for k in range(len(b)):
            pos, neg = ctx.apply_batch(b.op[k:k + 1], b.src[k:k + 1], b.dst[k:k + 1], [qid])
            got.append((int(pos[0]), int(neg[0])))
            ctx.commit()
    assert got == [(c["pos"], c["neg"]) for c in d["csm"]]


def test_tiny_workload(G):
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 256, 0)
    check(G, w.graph, [I.TRIANGLE_WITH_TAIL], b)


def test_tiny_workload_mixed_many_queries(G):
    w = I.make_workload("tiny")
    g = w.graph
    b = I.workload_batch(w, 600, 300, sub=1)
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1], [(0, 1)]), I.pattern_query([2, 2], [(0, 1)]),
          I.pattern_query([1, 2, 3], [(0, 1), (1, 2)])]
    att = 0
    while len(qs) < 12:
        kind = ["dense", "sparse", "tree"][att % 3]
        q = I.random_walk_query(off, nbr, g.labels, 4 + att % 2, kind, 5, att)
        att += 1
        if q is not None:
            qs.append(q)
    check(G, g, qs, b)
    check(G, g, qs, b, rows=False)


@pytest.mark.parametrize("rows", [True, False])
@pytest.mark.parametrize("trial", range(40))
def test_fuzz_small_graphs(G, trial, rows):
    r = np.random.default_rng(1000 + trial)
    n = int(r.integers(6, 40))
    g = I.random_small_graph(n, int(r.integers(10, 60)), int(r.integers(1, 4)), 9, trial)
    es = set(zip(g.src.tolist(), g.dst.tolist()))
    non = [(a, b) for a in range(n) for b in range(a + 1, n) if (a, b) not in es]
    el = sorted(es)
    ni = min(len(non), int(r.integers(0, 20)))
    nd = min(len(el), int(r.integers(0, 10)))
    ins = [non[i] for i in r.choice(len(non), ni, replace=False)] if ni else []
    dl = [el[i] for i in r.choice(len(el), nd, replace=False)] if nd else []
    ed = ins + dl
    ops = [1] * ni + [-1] * nd
    perm = r.permutation(len(ed))
    if len(ed) == 0:
        pytest.skip("empty batch")
    b = I.Batch(np.array([ops[i] for i in perm], np.int8), np.array([ed[i][1] for i in perm], np.int32),
                np.array([ed[i][0] for i in perm], np.int32))
    nl = int(g.labels.max()) + 1
    qs = []
    for k in range(5):
        q = int(r.integers(2, 6))
        edges = [(i, int(r.integers(0, i))) for i in range(1, q)]
        for _ in range(int(r.integers(0, 3))):
            a, c = sorted(r.choice(q, 2, replace=False).tolist())
            if (a, c) not in edges and (c, a) not in edges:
                edges.append((a, c))
        qs.append(I.pattern_query(r.integers(0, nl, q).tolist(), edges))
    flags = [0, 2, 4][trial % 3]
    check(G, g, qs, b, rows=rows, flags=flags, frontier_tile=[32, 64, 128][trial % 3],
          steal_grain=[1, 3, 64][trial % 3])


def test_empty_batch_and_no_queries(G):
    w = I.make_workload("tiny")
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qid = ctx.register_query(I.TRIANGLE_WITH_TAIL.labels, I.TRIANGLE_WITH_TAIL.src, I.TRIANGLE_WITH_TAIL.dst)
        e = np.zeros(0, np.int32)
        pos, neg = ctx.apply_batch(np.zeros(0, np.int8), e, e, [qid])
        assert (int(pos[0]), int(neg[0])) == (0, 0)
        ctx.commit()
        b = I.workload_batch(w, 10, 0)
        pos, neg = ctx.apply_batch(b.op, b.src, b.dst, [])
        assert len(pos) == 0
        ctx.commit()


@pytest.mark.parametrize("case,bad", [
    ("dup_same", 3), ("insert_existing", 2), ("delete_missing", 1), ("self_loop", 0), ("bad_id", 2),
    ("ins_del_same_edge", 2), ("bad_op", 1)])
def test_invalid_batch_rejected_and_graph_unchanged(G, case, bad):
    g = I.Graph(6, np.zeros(6, np.int32), np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32))
    ops, src, dst = {
        "dup_same": ([1, 1, 1, 1], [0, 4, 0, 5], [4, 5, 5, 4]),
        "insert_existing": ([1, -1, 1], [0, 0, 2], [4, 1, 1]),
        "delete_missing": ([1, -1, 1], [0, 0, 3], [4, 5, 5]),
        "self_loop": ([1, 1], [2, 0], [2, 4]),
        "bad_id": ([1, 1, 1], [0, 1, 9], [4, 4, 0]),
        "ins_del_same_edge": ([1, 1, -1], [0, 1, 4], [4, 5, 0]),
        "bad_op": ([1, 2, 1], [0, 1, 2], [4, 4, 4]),
    }[case]
    q = I.pattern_query([0, 0, 0], [(0, 1), (1, 2)])
    good = I.Batch(np.array([1, -1], np.int8), np.array([3, 1], np.int32), np.array([4, 2], np.int32))
    c_ref, _ = O.bdsm(g.n, g.labels, g.src, g.dst, q, good)
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qid = ctx.register_query(q.labels, q.src, q.dst)
        with pytest.raises(G.GammaError) as e:
            ctx.apply_batch(np.array(ops, np.int8), np.array(src, np.int32), np.array(dst, np.int32), [qid])
        assert e.value.code == G.GAMMA_EINVAL
        assert ("update %d " % bad) in str(e.value)
        pos, neg = ctx.apply_batch(good.op, good.src, good.dst, [qid])
        assert (int(pos[0]), int(neg[0])) == O.totals(c_ref, good.op)


def test_state_machine(G):
    with G.Context() as ctx:
        with pytest.raises(G.GammaError) as e:
            ctx.commit()
        assert e.value.code == G.GAMMA_ESTATE
        g = I.Graph(4, np.zeros(4, np.int32), np.array([0], np.int32), np.array([1], np.int32))
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qid = ctx.register_query([0, 0], [0], [1])
        b = I.Batch(np.array([1], np.int8), np.array([2], np.int32), np.array([3], np.int32))
        ctx.apply_batch(b.op, b.src, b.dst, [qid])
        with pytest.raises(G.GammaError) as e:
            ctx.apply_batch(b.op, b.src, b.dst, [qid])
        assert e.value.code == G.GAMMA_ESTATE
        ctx.commit()
        with pytest.raises(G.GammaError):
            ctx.register_query([0, 0, 0], [0], [1])  # disconnected


def test_sequence_of_batches_with_commit(G):
    """Five consecutive mixed batches on a scaled-down large-workload graph."""
    w = I.make_workload("large", scale=14, n_edges=120_000)
    g = w.graph
    cs, cd = g.src, g.dst
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    qs = []
    att = 0
    while len(qs) < 4:
        q = I.random_walk_query(off, nbr, g.labels, 5, ["dense", "sparse"][att % 2], 3, att)
        att += 1
        if q is not None:
            qs.append(q)
    with G.Context(flags=G.GAMMA_F_PER_UPDATE) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        start = 0
        for it in range(5):
            b = I.workload_batch(w, 1600, 400, sub=it, pool_start=start, cur=(cs, cd))
            start += 1600
            pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids)
            for j, q in enumerate(qs):
                c, _ = O.bdsm(g.n, g.labels, cs, cd, q, b)
                assert (int(pos[j]), int(neg[j])) == O.totals(c, b.op), (it, j)
                assert np.array_equal(ctx.update_counts(j), c)
            ctx.commit()
            cs, cd = I.apply_batch_edges(cs, cd, b)
        st = ctx.stats()
        assert st["live_edges"] == 2 * cs.size


def test_options_do_not_change_results(G):
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 500, 200, sub=3)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 0, 1, 1], [(0, 1), (1, 2), (2, 3), (3, 0)])]
    ref = None
    for flags, tile, grain, wpb in [(0, 64, 64, 8), (2, 32, 1, 4), (4, 128, 7, 16), (6, 256, 1024, 2), (32, 64, 64, 8),
                                    (8, 64, 64, 8), (64, 64, 64, 8), (96, 32, 3, 8), (128, 64, 64, 8),
                                    (132, 32, 1, 4), (256, 64, 64, 8), (264, 64, 16, 4), (384, 64, 64, 8)]:
        pos, neg, _, _, _ = gpu_run(G, w.graph, qs, b, flags=flags, rows=False, frontier_tile=tile,
                                    steal_grain=grain, warps_per_block=wpb)
        got = (pos.tolist(), neg.tolist())
        if ref is None:
            ref = got
        assert got == ref


@pytest.mark.parametrize("flags", [0, 0x20, 0x40, 0x60, 0x80, 0xC0, 0x100])
def test_shared_last_position_equals_oracle(G, flags):
    """Queries whose last vertex (in the matching order) is not adjacent to the
    one before it: K(2,3) with the second side on one label (the sibling
    correction applies) and on two labels, a star, and a 5-cycle with a chord.
    The children of one partial match then share their last-position
    candidates (counted once per sibling); with GAMMA_F_NO_SHARE (0x40) and
    GAMMA_F_NO_LEAF (0x20) combinations, with work created in update order
    (GAMMA_F_SEED_IN_ORDER, 0x80) instead of grouped by hub, and query by
    query (GAMMA_F_SEED_BY_QUERY, 0x100), the
    per-update charges stay the oracle's, on a power-law graph with hubs and
    a mixed batch."""
    w = I.make_workload("large", scale=13, n_edges=90_000)
    g = w.graph
    b = I.workload_batch(w, 1200, 400, sub=2)
    k23 = [(0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4)]
    qs = [I.pattern_query([0, 0, 1, 1, 1], k23), I.pattern_query([0, 1, 2, 2, 3], k23),
          I.pattern_query([0, 1, 1, 1], [(0, 1), (0, 2), (0, 3)]),
          I.pattern_query([0, 1, 0, 1, 2], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 2)])]
    pos, neg, per, _, st = gpu_run(G, g, qs, b, flags=flags, rows=False, steal_grain=4)
    want = O.bdsm_multi(g.n, g.labels, g.src, g.dst, qs, b)
    assert np.array_equal(per, want)
    assert int(want.sum()) > 0


def test_row_overflow_and_fetch(G):
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 256, 0)
    q = I.TRIANGLE_WITH_TAIL
    c, t = oracle_run(w.graph, q, b)
    total = int(c.sum())
    assert total > 4
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qid = ctx.register_query(q.labels, q.src, q.dst)
        pos, neg, r, req = ctx.apply_batch(b.op, b.src, b.dst, [qid], row_capacity=3)
        assert int(pos[0]) + int(neg[0]) == total and req == total and len(r) == 3
        big = np.full((total, 3 + q.q), -1, np.int32)
        r2, req2 = ctx.fetch_matches(big)
        assert req2 == total
        assert [x[:2 + q.q] for x in rowset(r2, qid)] == orowset(t, q)
        ctx.commit()


def test_device_pointer_inputs(G):
    import torch
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 256, 50, sub=2)
    q = I.TRIANGLE_WITH_TAIL
    c, _ = oracle_run(w.graph, q, b, rows=False)
    with G.Context(stream=torch.cuda.current_stream()) as ctx:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        ctx.load_graph(w.graph.n, dev(w.graph.labels), dev(w.graph.src), dev(w.graph.dst))
        qid = ctx.register_query(q.labels, q.src, q.dst)
        pos, neg = ctx.apply_batch(dev(b.op), dev(b.src), dev(b.dst), [qid])
        assert (int(pos[0]), int(neg[0])) == O.totals(c, b.op)
        ctx.commit()


def test_work_budget_times_out_cleanly(G):
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 256, 0)
    with G.Context(work_budget=1) as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qid = ctx.register_query(I.TRIANGLE_WITH_TAIL.labels, I.TRIANGLE_WITH_TAIL.src, I.TRIANGLE_WITH_TAIL.dst)
        with pytest.raises(G.GammaError) as e:
            ctx.apply_batch(b.op, b.src, b.dst, [qid])
        assert e.value.code == G.GAMMA_ETIMEOUT
        ctx.commit()  # the graph is staged and still consistent
        ctx.set_options(work_budget=0)
        b2 = I.workload_batch(w, 10, 0, pool_start=300)
        ctx.apply_batch(b2.op, b2.src, b2.dst, [qid])
        ctx.commit()


def test_idle_wait_limit_times_out_cleanly(G):
    """The DFS kernel's waits for donated work are bounded: with a 1 us
    limit, the first warp that runs out of work while others still hold some
    gives up, the apply returns GAMMA_ETIMEOUT with the batch staged, and the
    context keeps working (commit, then the inverse batch with the default
    limit gives the counts of a context that never timed out).  No fault and
    no hang: the wait ends by its own limit."""
    w = I.make_workload("large", scale=15, n_edges=300_000)
    g = w.graph
    b = I.workload_batch(w, 4000, 1000)
    inv = b.inverse()
    off, nbr = I.csr_from_edges(g.n, g.src, g.dst)
    qs = [I.TRIANGLE_WITH_TAIL]
    att = 0
    while len(qs) < 4:
        q = I.random_walk_query(off, nbr, g.labels, 5, "sparse" if att % 2 else "dense", 17, att)
        att += 1
        if q is not None:
            qs.append(q)
    with G.Context() as ref:
        ref.load_graph(g.n, g.labels, g.src, g.dst)
        rq = [ref.register_query(q.labels, q.src, q.dst) for q in qs]
        ref.apply_batch(b.op, b.src, b.dst, rq)
        ref.commit()
        want = ref.apply_batch(inv.op, inv.src, inv.dst, rq)
        ref.commit()
    with G.Context(idle_limit_us=1) as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        with pytest.raises(G.GammaError) as e:
            ctx.apply_batch(b.op, b.src, b.dst, qids)
        assert e.value.code == G.GAMMA_ETIMEOUT
        ctx.commit()  # the batch was staged before the match phase gave up
        ctx.set_options(idle_limit_us=60_000_000)
        got = ctx.apply_batch(inv.op, inv.src, inv.dst, qids)
        ctx.commit()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_graph_mode_replays_and_matches(G):
    """GAMMA_F_GRAPH: the apply is captured once per shape and replayed; counts unchanged."""
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 300, 100, sub=4)
    inv = b.inverse()
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    ref = []
    for flags in [0, G.GAMMA_F_GRAPH]:
        got = []
        with G.Context(flags=flags) as ctx:
            ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
            qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
            for k in range(4):
                bb = b if k % 2 == 0 else inv
                pos, neg = ctx.apply_batch(bb.op, bb.src, bb.dst, qids)
                got.append((pos.tolist(), neg.tolist()))
                ctx.commit()
            st = ctx.stats()
        if flags:
            assert st["graph_captures"] == 1
            assert got == ref
        else:
            ref = got
    for j, q in enumerate(qs):
        c, _ = O.bdsm(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst, q, b)
        assert (ref[0][0][j], ref[0][1][j]) == O.totals(c, b.op)


def _requests(w, sizes, seed):
    """Consecutive requests on disjoint edges: insertions from the pool, deletions from G0."""
    g = w.graph
    reqs = []
    start, dstart = 0, 0
    order = np.random.default_rng(seed).permutation(g.src.size)
    for i, n in enumerate(sizes):
        ni = n * 3 // 4
        nd = n - ni
        s = np.concatenate([w.pool_src[start:start + ni], g.src[order[dstart:dstart + nd]]])
        d = np.concatenate([w.pool_dst[start:start + ni], g.dst[order[dstart:dstart + nd]]])
        op = np.concatenate([np.ones(ni, np.int8), -np.ones(nd, np.int8)])
        p = np.random.default_rng(seed + i).permutation(n)
        reqs.append(I.Batch(op[p], s[p].astype(np.int32), d[p].astype(np.int32)))
        start += ni
        dstart += nd
    return reqs


@pytest.mark.parametrize("flags", [0, 4, 8])
def test_requests_alone_equal_in_the_mix(G, flags):
    """Several requests staged together give each request the result it gets alone."""
    w = I.make_workload("tiny")
    reqs = _requests(w, [40, 1, 130, 75, 9, 200], 5)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)]), I.pattern_query([1, 1], [(0, 1)])]
    alone = []
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        for r in reqs:
            pos, neg = ctx.apply_batch(r.op, r.src, r.dst, qids)
            alone.append((pos.tolist(), neg.tolist()))
            ctx.commit()
        after_alone = ctx.export_adjacency(w.graph.n)
    with G.Context(flags=flags) as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        off = np.concatenate([[0], np.cumsum([len(r) for r in reqs])])
        cat = lambda f: np.concatenate([getattr(r, f) for r in reqs])
        pos, neg = ctx.apply_batches(off, cat("op"), cat("src"), cat("dst"), qids)
        ctx.commit()
        after_mix = ctx.export_adjacency(w.graph.n)
    assert [(pos[r].tolist(), neg[r].tolist()) for r in range(len(reqs))] == alone
    assert np.array_equal(after_alone[0], after_mix[0])
    # oracle, request by request
    cs, cd = w.graph.src, w.graph.dst
    for r, rb in enumerate(reqs):
        for j, q in enumerate(qs):
            c, _ = O.bdsm(w.graph.n, w.graph.labels, cs, cd, q, rb)
            assert (int(pos[r, j]), int(neg[r, j])) == O.totals(c, rb.op)
        cs, cd = I.apply_batch_edges(cs, cd, rb)


@pytest.mark.parametrize("flags", [0, 8])
def test_requests_sharing_edges_equal_one_at_a_time(G, flags):
    """Requests staged together may touch the same edges: the served stream's
    generator deletes edges earlier requests inserted and re-inserts deleted
    ones.  Each request gets its one-at-a-time counts (checked against the
    oracle on the graph the earlier requests leave) and the committed graph
    equals the one-at-a-time graph."""
    w = I.make_workload("tiny")
    reqs = I.served_stream(w, 12, 7, 0.5, 2.2)
    keys = [set(I.edge_keys(r.src, r.dst).tolist()) for r in reqs]
    assert any(keys[i] & keys[j] for i in range(len(keys)) for j in range(i))  # the case shares edges
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)]), I.pattern_query([1, 1], [(0, 1)])]
    alone = []
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        for r in reqs:
            pos, neg = ctx.apply_batch(r.op, r.src, r.dst, qids)
            alone.append((pos.tolist(), neg.tolist()))
            ctx.commit()
        after_alone = ctx.export_adjacency(w.graph.n)
    with G.Context(flags=flags | G.GAMMA_F_PER_UPDATE) as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        off = np.concatenate([[0], np.cumsum([len(r) for r in reqs])])
        cat = lambda f: np.concatenate([getattr(r, f) for r in reqs])
        pos, neg = ctx.apply_batches(off, cat("op"), cat("src"), cat("dst"), qids)
        per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
        ctx.commit()
        after_mix = ctx.export_adjacency(w.graph.n)
    assert [(pos[r].tolist(), neg[r].tolist()) for r in range(len(reqs))] == alone
    assert np.array_equal(after_alone[0], after_mix[0]) and np.array_equal(after_alone[1], after_mix[1])
    cs, cd = w.graph.src, w.graph.dst
    for r, rb in enumerate(reqs):
        c = O.bdsm_multi(w.graph.n, w.graph.labels, cs, cd, qs, rb)
        assert np.array_equal(per[:, off[r]:off[r + 1]], c)
        cs, cd = I.apply_batch_edges(cs, cd, rb)


def test_invalid_request_chains_are_rejected(G):
    """A request must be valid on the graph the earlier requests leave and may
    touch an edge once: inserting an edge an earlier request inserted, a
    request touching one edge twice, and deleting an edge no earlier request
    inserted are rejected with the offending index, the graph unchanged."""
    w = I.make_workload("tiny")
    e = (int(w.pool_src[0]), int(w.pool_dst[0]))  # not in G0
    f = (int(w.pool_src[1]), int(w.pool_dst[1]))
    cases = [
        ([0, 1, 2], [1, 1], [e, e], 1),                 # inserted twice, by two requests
        ([0, 2], [1, -1], [e, e], 1),                   # one request touches the edge twice
        ([0, 1, 2, 3], [1, -1, -1], [f, e, e], 1),      # deletes an edge that is absent
        ([0, 1, 2, 3], [1, -1, 1], [e, e, e], None),    # insert, delete, insert: valid
    ]
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qid = ctx.register_query([0, 1], [0], [1])
        before = ctx.export_adjacency(w.graph.n)
        for off, ops, edges, bad in cases:
            op = np.array(ops, np.int8)
            src = np.array([x[0] for x in edges], np.int32)
            dst = np.array([x[1] for x in edges], np.int32)
            if bad is None:
                ctx.apply_batches(np.array(off), op, src, dst, [qid])
                ctx.commit()
                after = ctx.export_adjacency(w.graph.n)
                assert after[0][-1] == before[0][-1] + 2  # e is in the graph once
                continue
            with pytest.raises(G.GammaError) as ex:
                ctx.apply_batches(np.array(off), op, src, dst, [qid])
            assert ex.value.code == G.GAMMA_EINVAL and ("update %d " % bad) in str(ex.value)
            now = ctx.export_adjacency(w.graph.n)
            assert np.array_equal(now[0], before[0]) and np.array_equal(now[1], before[1])


def test_server_results_equal_sequential(G):
    """Served form: every request's counts equal those of applying the requests
    one by one, and requests that queued while the GPU was busy were staged together."""
    w = I.make_workload("tiny")
    reqs = _requests(w, [int(x) for x in np.random.default_rng(9).integers(1, 30, 40)], 11)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    alone = []
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        for r in reqs:
            pos, neg = ctx.apply_batch(r.op, r.src, r.dst, qids)
            alone.append((pos.tolist(), neg.tolist()))
            ctx.commit()
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        srv = G.Server(ctx, qids, max_requests=16)
        tickets = [srv.submit(r.op, r.src, r.dst) for r in reqs]
        got, groups = [], []
        for t in tickets:
            rc, pos, neg, info = srv.wait(t)
            assert rc == G.GAMMA_OK
            got.append((pos.tolist(), neg.tolist()))
            groups.append(info["group_size"])
            assert info["done_ms"] >= info["start_ms"] >= info["arrival_ms"] - 1e-6
        st = srv.stats()
        srv.stop()
    assert got == alone
    assert max(groups) > 1 and st["requests"] == len(reqs) and st["groups"] < len(reqs)


def test_autotune_picks_a_point_and_keeps_counts(G):
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 400, 100, sub=6)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    with G.Context() as ctx:
        ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids)
        grid = [(4, 32, 1), (8, 64, 16), (16, 128, 4), (0, 64, 4)]  # the last point is invalid
        best, pts = G.gamma_autotune(ctx.h, grid, repeats=2)
        assert pts[-1]["ms"] < 0 and all(p["ms"] >= 0 for p in pts[:-1])
        assert best["ms"] == min(p["ms"] for p in pts[:-1])
        p2, n2 = G.gamma_recount_noalloc(ctx.h, len(qids))
        assert np.array_equal(p2, pos) and np.array_equal(n2, neg)
        ctx.commit()


def test_instrumented_build_counts_bytes_only(G):
    """GAMMA_F_COUNT_BYTES runs the DFS build that accounts algorithmic bytes:
    same counts and per-update charges as the timed build, and it is the only
    one that reports bytes."""
    w = I.make_workload("tiny")
    b = I.workload_batch(w, 400, 100, sub=5)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    res = {}
    for flags in (G.GAMMA_F_PER_UPDATE, G.GAMMA_F_PER_UPDATE | G.GAMMA_F_COUNT_BYTES):
        with G.Context(flags=flags) as ctx:
            ctx.load_graph(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst)
            qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
            pos, neg = ctx.apply_batch(b.op, b.src, b.dst, qids)
            per = [ctx.update_counts(j).tolist() for j in range(len(qids))]
            res[flags] = (pos.tolist(), neg.tolist(), per, ctx.stats()["alg_bytes"])
            ctx.commit()
    plain, counted = res[G.GAMMA_F_PER_UPDATE], res[G.GAMMA_F_PER_UPDATE | G.GAMMA_F_COUNT_BYTES]
    assert plain[:3] == counted[:3]
    assert plain[3] == 0 and counted[3] > 0


def _new_vertex_edges(n_old, k, seed):
    """Edges from each of k new vertices (ids n_old..n_old+k-1) to three old
    vertices, plus a path through the new ones; canonical and distinct."""
    e = set()
    r = I.rand_u64(seed, 72, np.arange(4 * k, dtype=np.uint64))
    for i in range(k):
        v = n_old + i
        for j in range(3):
            e.add((int(r[4 * i + j] % np.uint64(n_old)), v))
        if i:
            e.add((v - 1, v))
    e = sorted(e)
    return np.array([a for a, _ in e], np.int32), np.array([b for _, b in e], np.int32)


def test_vertex_insertions_and_deletions(G):
    """Vertex updates as edge batches (Sec. II-A): vertices added to a loaded
    graph (id space reserved before loading) join with no edges; a batch then
    inserts edges to them (mixed with ordinary updates), and deleting a vertex
    is the batch of its incident edges. Counts and per-update charges equal the
    oracle's on the grown graph, also with the apply replayed as a CUDA graph
    whose captured pointers the new vertices invalidate."""
    w = I.make_workload("tiny")
    g = w.graph
    k = 40
    new_labels = (I.rand_u32(3, 71, np.arange(k, dtype=np.uint64)) % np.uint64(4)).astype(np.int32)
    n2 = g.n + k
    labels2 = np.concatenate([g.labels, new_labels])
    ns, nd = _new_vertex_edges(g.n, k, 5)
    base = I.workload_batch(w, 200, 60, sub=4)
    op = np.concatenate([base.op, np.ones(ns.size, np.int8)])
    src = np.concatenate([base.src, ns])
    dst = np.concatenate([base.dst, nd])
    mix = I.shuffle_order(op.size, 9, 3)
    b1 = I.Batch(op[mix], src[mix], dst[mix])
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)]),
          I.pattern_query([0, 0, 1, 1], [(0, 1), (1, 2), (2, 3), (3, 0)])]
    for flags in (G.GAMMA_F_PER_UPDATE, G.GAMMA_F_PER_UPDATE | G.GAMMA_F_GRAPH):
        with G.Context(flags=flags) as ctx:
            ctx.reserve_vertices(n2)
            ctx.load_graph(g.n, g.labels, g.src, g.dst)
            qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
            # a batch of b1's size before the vertices arrive: in graph mode its
            # captured apply would be replayed for b1 unless adding vertices drops it
            pre = I.workload_batch(w, len(b1) - 10, 10, sub=8, pool_start=500)
            ctx.apply_batch(pre.op, pre.src, pre.dst, qids)
            ctx.commit()
            cur = I.apply_batch_edges(g.src, g.dst, pre)
            with pytest.raises(G.GammaError):
                ctx.add_vertices(np.full(k, 99, np.int32))  # label outside the graph's range
            assert ctx.add_vertices(new_labels) == g.n
            with pytest.raises(G.GammaError):
                ctx.add_vertices(np.zeros(1, np.int32))  # beyond the reserved vertex count
            pos, neg = ctx.apply_batch(b1.op, b1.src, b1.dst, qids)
            with pytest.raises(G.GammaError):
                ctx.add_vertices(np.ones(1, np.int32))  # a batch is staged
            per = np.stack([ctx.update_counts(j) for j in range(len(qids))])
            ctx.commit()
            want = O.bdsm_multi(n2, labels2, cur[0], cur[1], qs, b1)
            assert np.array_equal(per, want)
            assert pos.tolist() == want[:, b1.op > 0].sum(axis=1).tolist()
            assert neg.tolist() == want[:, b1.op < 0].sum(axis=1).tolist()
            cur = I.apply_batch_edges(cur[0], cur[1], b1)
            # delete a new vertex and an old one: the batch of their incident edges
            gone = [g.n + 7, int(ns[0])]
            e = set()
            for v in gone:
                for u in ctx.vertex_neighbors(v).tolist():
                    e.add((min(u, v), max(u, v)))
            e = sorted(e)
            assert len(e) >= 4
            b2 = I.Batch(-np.ones(len(e), np.int8), np.array([a for a, _ in e], np.int32),
                         np.array([c for _, c in e], np.int32))
            pos2, neg2 = ctx.apply_batch(b2.op, b2.src, b2.dst, qids)
            per2 = np.stack([ctx.update_counts(j) for j in range(len(qids))])
            ctx.commit()
            want2 = O.bdsm_multi(n2, labels2, cur[0], cur[1], qs, b2)
            assert np.array_equal(per2, want2) and int(pos2.sum()) == 0
            assert neg2.tolist() == want2.sum(axis=1).tolist()
            for v in gone:
                assert ctx.vertex_neighbors(v).size == 0
            cur = I.apply_batch_edges(cur[0], cur[1], b2)
            assert ctx.stats()["live_edges"] == 2 * cur[0].size


def _max_query_case():
    """16-vertex queries (the limit): a star whose centre has one neighbour per
    leaf label (two for labels 1..5 once the batch lands) and a path labelled
    0..15 that one inserted edge completes."""
    n = 64
    lab = np.zeros(n, np.int32)
    edges = set()
    for i in range(1, 16):
        lab[i] = i; edges.add((0, i))
    for i in range(16, 21):
        lab[i] = i - 15                       # second candidates for labels 1..5
    for k in range(16):                       # path 21..36 labelled 0..15
        lab[21 + k] = k
        if k: edges.add((20 + k, 21 + k))
    r = I.rand_u64(3, 91, np.arange(200, dtype=np.uint64))
    for j in range(37, 64):
        lab[j] = int(r[j] % np.uint64(16))
    for t in range(60):
        a, b = 37 + int(r[2 * t] % np.uint64(27)), 37 + int(r[2 * t + 1] % np.uint64(27))
        if a != b: edges.add((min(a, b), max(a, b)))
    edges.discard((28, 29))                   # the path is completed by the batch
    src = np.array([a for a, _ in sorted(edges)], np.int32); dst = np.array([b for _, b in sorted(edges)], np.int32)
    ins = [(0, 16), (0, 17), (0, 18), (28, 29), (37, 38) if (37, 38) not in edges else (39, 40)]
    dels = [(0, 3), sorted(e for e in edges if e[0] >= 37)[0]]
    op = np.array([1] * len(ins) + [-1] * len(dels), np.int8)
    bs = np.array([a for a, _ in ins + dels], np.int32); bd = np.array([b for _, b in ins + dels], np.int32)
    mix = I.shuffle_order(op.size, 4, 2)
    b = I.Batch(op[mix], bs[mix], bd[mix])
    star = I.pattern_query([0] + list(range(1, 16)), [(0, i) for i in range(1, 16)])
    path = I.pattern_query(list(range(16)), [(i, i + 1) for i in range(15)])
    return I.Graph(n, lab, src, dst), [star, path], b


def _wide_key_case():
    """The widest adjacency key: 2^23 vertices and labels up to 255 fill all 32
    bits (23 id bits, 8 label bits, the batch flag); the matches sit on the
    top ids and labels."""
    n = 1 << 23                                # 23 id bits + 8 label bits + flag = 32
    lab = np.zeros(n, np.int32)
    r = I.rand_u64(5, 92, np.arange(4000, dtype=np.uint64))
    hi = n - 1 - np.arange(40)                 # the top ids carry labels 254 / 255
    lab[hi] = np.where(np.arange(40) % 2 == 0, 255, 254)
    lab[7] = 128
    edges = set()
    for t in range(300):
        a, b = int(hi[r[2 * t] % np.uint64(40)]), int(hi[r[2 * t + 1] % np.uint64(40)])
        if a != b: edges.add((min(a, b), max(a, b)))
    for t in range(40):                        # a spread of low ids joined to the top ones
        a, b = int(r[1000 + t] % np.uint64(n - 64)), int(hi[t])
        edges.add((min(a, b), max(a, b)))
    edges.add((7, int(hi[0])))
    e = sorted(edges)
    keep, batch_e = e[:-30], e[-30:]
    src = np.array([a for a, _ in keep], np.int32); dst = np.array([b for _, b in keep], np.int32)
    dels = keep[:10]
    op = np.array([1] * len(batch_e) + [-1] * len(dels), np.int8)
    bs = np.array([a for a, _ in batch_e + dels], np.int32); bd = np.array([b for _, b in batch_e + dels], np.int32)
    mix = I.shuffle_order(op.size, 6, 2)
    b = I.Batch(op[mix], bs[mix], bd[mix])
    qs = [I.pattern_query([255, 254, 255], [(0, 1), (1, 2), (0, 2)]),
          I.pattern_query([128, 255, 254, 255], [(0, 1), (1, 2), (2, 3)]),
          I.pattern_query([0, 255, 254], [(0, 1), (1, 2)])]
    return I.Graph(n, lab, src, dst), qs, b


def test_sixteen_vertex_queries(G):
    g, qs, b = _max_query_case()
    pos, neg, _ = check(G, g, qs, b)
    assert (int(pos[0]), int(neg[0]), int(pos[1])) == (4, 1, 1)


def test_widest_adjacency_key(G):
    g, qs, b = _wide_key_case()
    pos, neg, _ = check(G, g, qs, b)
    assert int(pos.sum()) > 0 and int(neg.sum()) > 0


def test_server_isolates_an_invalid_request(G):
    """A request that deletes a missing edge fails alone: the requests staged
    with it get the results of serving the valid requests one at a time."""
    w = I.make_workload("tiny")
    reqs = _requests(w, [int(x) for x in np.random.default_rng(4).integers(1, 20, 24)], 13)
    g = w.graph
    have = set(I.edge_keys(g.src, g.dst).tolist())
    a = 0
    while True:  # a vertex pair that is never an edge during the stream
        u, v = 3 + a, 1000 + a
        touched = any(int(k) == (u << 32 | v) for r in reqs for k in I.edge_keys(r.src, r.dst))
        if (u << 32 | v) not in have and not touched:
            break
        a += 1
    bad_at = {5, 17}
    stream = []
    for i, r in enumerate(reqs):
        if i in bad_at:
            stream.append(I.Batch(np.array([-1], np.int8), np.array([u], np.int32), np.array([v], np.int32)))
        stream.append(r)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    alone = []
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        for r in reqs:
            pos, neg = ctx.apply_batch(r.op, r.src, r.dst, qids)
            alone.append((pos.tolist(), neg.tolist()))
            ctx.commit()
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        srv = G.Server(ctx, qids, max_requests=16)
        tickets = [srv.submit(r.op, r.src, r.dst) for r in stream]
        got, bad = [], 0
        for t, r in zip(tickets, stream):
            rc, pos, neg, info = srv.wait(t)
            if len(r) == 1 and int(r.src[0]) == u and int(r.dst[0]) == v:
                assert rc == G.GAMMA_EINVAL
                bad += 1
            else:
                assert rc == G.GAMMA_OK
                got.append((pos.tolist(), neg.tolist()))
        srv.stop()
    assert bad == len(bad_at) and got == alone


def test_checkpoint_and_restore(G):
    """A checkpoint taken after a commit restores the same graph (adjacency
    lists equal), the same queries under the same ids and the reserved
    vertex room; a batch applied after the restore, in the same or a fresh
    context, gives the counts and rows it gave the first time."""
    w = I.make_workload("tiny")
    g = w.graph
    b1 = I.workload_batch(w, 300, 80, sub=2)
    cur = I.apply_batch_edges(g.src, g.dst, b1)
    b2 = I.workload_batch(w, 300, 80, sub=3, pool_start=300, cur=cur)
    qs = [I.TRIANGLE_WITH_TAIL, I.pattern_query([0, 1, 2], [(0, 1), (1, 2)])]
    with G.Context() as ctx:
        ctx.reserve_vertices(g.n + 8)
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in qs]
        ctx.apply_batch(b1.op, b1.src, b1.dst, qids)
        with pytest.raises(G.GammaError):
            ctx.checkpoint()  # a batch is staged
        ctx.commit()
        ck = ctx.checkpoint()
        adj = ctx.export_adjacency(g.n)
        pos, neg, r, _ = ctx.apply_batch(b2.op, b2.src, b2.dst, qids, row_capacity=1 << 20)
        first = (pos.tolist(), neg.tolist(), sorted(map(tuple, r.tolist())))
        ctx.commit()
        ctx.restore(ck)
        for a, c in zip(ctx.export_adjacency(g.n), adj):
            assert np.array_equal(a, c)
        pos, neg, r, _ = ctx.apply_batch(b2.op, b2.src, b2.dst, qids, row_capacity=1 << 20)
        assert (pos.tolist(), neg.tolist(), sorted(map(tuple, r.tolist()))) == first
        ctx.commit()
        assert ctx.add_vertices(np.zeros(8, np.int32)) == g.n  # the reserve came back too
    with G.Context() as ctx2:
        with pytest.raises(G.GammaError):
            ctx2.restore(b"GMCK" + bytes(40))
        ctx2.restore(ck)
        pos, neg, r, _ = ctx2.apply_batch(b2.op, b2.src, b2.dst, qids, row_capacity=1 << 20)
        assert (pos.tolist(), neg.tolist(), sorted(map(tuple, r.tolist()))) == first
