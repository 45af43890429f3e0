"""The device-resident dynamic CSR (staging and commit) against a host
set model: after staging, every list is the union G u G' sorted by (label,
id) with update tags on the batch's edges; after commit, it is G'."""
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


def model_lists(n, labels, src, dst, batch=None):
    """Host model: {v: [(nbr, tag)]} sorted by (label, id)."""
    adj = {v: {} for v in range(n)}
    for a, b in zip(src.tolist(), dst.tolist()):
        adj[a][b] = -1
        adj[b][a] = -1
    if batch is not None:
        for k, (o, a, b) in enumerate(zip(batch.op.tolist(), batch.src.tolist(), batch.dst.tolist())):
            t = 2 * k + (1 if o < 0 else 0)
            adj[a][b] = t
            adj[b][a] = t
    return {v: sorted(((w, t) for w, t in d.items()), key=lambda x: (labels[x[0]], x[0])) for v, d in adj.items()}


def device_lists(ctx, n):
    off, nbr, tag = ctx.export_adjacency(n)
    return {v: list(zip(nbr[off[v]:off[v + 1]].tolist(), tag[off[v]:off[v + 1]].tolist())) for v in range(n)}


@pytest.mark.parametrize("name,scale,ne,nb", [("tiny", None, None, 288), ("large", 14, 120_000, 4000)])
def test_load_stage_commit_match_host_model(G, name, scale, ne, nb):
    w = I.make_workload(name, scale=scale, n_edges=ne)
    g = w.graph
    lab = g.labels.tolist()
    cs, cd = g.src, g.dst
    with G.Context() as ctx:
        ctx.load_graph(g.n, g.labels, g.src, g.dst)
        assert device_lists(ctx, g.n) == model_lists(g.n, lab, cs, cd)
        start = 0
        for it in range(3):
            nins = nb * 8 // 10
            b = I.workload_batch(w, nins, nb - nins, sub=it, pool_start=start, cur=(cs, cd))
            start += nins
            ctx.apply_batch(b.op, b.src, b.dst, [])
            got = device_lists(ctx, g.n)
            want = model_lists(g.n, lab, cs, cd, b)
            bad = [v for v in range(g.n) if got[v] != want[v]]
            assert not bad, (it, bad[:5], [(got[v], want[v]) for v in bad[:2]])
            ctx.commit()
            cs, cd = I.apply_batch_edges(cs, cd, b)
            assert device_lists(ctx, g.n) == model_lists(g.n, lab, cs, cd)
