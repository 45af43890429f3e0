"""Choose the query graphs of the benchmark workloads and store them as JSON.

Queries are extracted from G0 by the seeded extractor of
``paper_2401_17018_gb300.inputs.random_walk_query`` (Sec. VI-A: random
subgraphs of the data graph, classed by density). As in the paper, which
leaves queries over a 30-minute cap unsolved and out of its averages
(Sec. VI-A "Metrics"), a candidate is only kept when its work is bounded:
the CPU oracle must finish the candidate on a fixed sample of the batch's
updates (every ``stride``-th update) within ``budget`` candidate tests, and
the sample must contain at least one incremental match. Rejected candidates
are logged in the output with the reason. Nothing here touches the CUDA path.

Usage: python tests/golden/make_queries.py mid|batched|served|large [--workers 8]
"""
import argparse
import json
import os
import sys
import time
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2401_17018_gb300 import inputs as I  # noqa: E402

SPECS = {
    # name: (workload, batch inserts, batch deletions, plan of (kind, q) per query)
    "mid": ("mid", 90_000, 10_000, [("sparse", 6)] * 10 + [("dense", 6)] * 10),
    # 64 queries of 4..12 vertices (uneven sizes), alternating sparse and dense
    "batched": ("mid", 90_000, 10_000,
                [("sparse" if i % 2 == 0 else "dense_ge3", 4 + (i * 7) % 9) for i in range(64)]),
    # 16 queries of 6..8 vertices on the scale-22 graph (the served stream's first batch)
    "served": ("served", 3_000, 1_000, [("dense", 6 + i % 3) for i in range(16)]),
    # 8-vertex queries, 4 sparse and 4 dense, on the scale-23 graph (first batch)
    "large": ("large", 800_000, 200_000, [("sparse", 8)] * 4 + [("dense", 8)] * 4),
}
# (stride, budget) per query class: every stride-th update of the batch is
# evaluated, within budget candidate tests. Sparse queries on the power-law
# graphs are far costlier per update, so they get a thinner sample and a
# larger budget.
RULES = {"dense": (200, 10_000_000), "dense_ge3": (200, 10_000_000), "sparse": (2500, 40_000_000),
         "tree": (2500, 40_000_000)}

_W = None


def _init(name):
    global _W
    wl, ni, nd, _ = SPECS[name]
    w = I.make_workload(wl)
    b = I.workload_batch(w, ni, nd)
    off, nbr = I.csr_from_edges(w.graph.n, w.graph.src, w.graph.dst)
    _W = (w, b, off, nbr)


def _try(args):
    kind, q, attempt = args
    w, b, off, nbr = _W
    g = w.graph
    Q = I.random_walk_query(off, nbr, g.labels, q, kind, w.seed + 1000 * q, attempt)
    if Q is None:
        return attempt, None, "class test failed"
    stride, budget = RULES[kind]
    ev = np.arange(0, len(b), stride)
    t = time.time()
    try:
        c, _ = O.bdsm(g.n, g.labels, g.src, g.dst, Q, b, eval_idx=ev, budget=budget)
    except O.OracleError as e:
        return attempt, Q.to_json(), "oracle budget exceeded on the sample (code %d)" % e.code
    if int(c.sum()) == 0:
        return attempt, Q.to_json(), "no incremental match on the sample"
    d = Q.to_json()
    d["sample_matches"] = int(c.sum())
    d["sample_seconds"] = round(time.time() - t, 2)
    return attempt, d, None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(SPECS))
    ap.add_argument("--workers", type=int, default=8)
    args = ap.parse_args()
    wl, ni, nd, plan = SPECS[args.name]
    _init(args.name)
    w = _W[0]
    out = {"workload": wl, "graph_digest": w.graph.digest(), "batch": {"n_ins": ni, "n_del": nd, "sub": 0},
           "rule": "keep a candidate of class k when the CPU oracle finishes it on updates 0, s, 2s, ... of the "
                   "batch within B candidate tests and finds at least one incremental match there; (s, B) per "
                   "class: " + json.dumps(RULES),
           "queries": [], "rejected": []}
    want = {}
    for kind, q in plan:
        want[(kind, q)] = want.get((kind, q), 0) + 1
    chosen = {k: [] for k in want}
    seen = set()
    path = os.path.join(HERE, "queries_%s.json" % args.name)
    partial = path + ".partial"
    start_at = {}
    if os.path.exists(partial):  # resume: keep what an interrupted run chose
        with open(partial) as f:
            old = json.load(f)
        for d in old["chosen"]:
            key = (d["kind"], len(d["labels"]))
            if key in chosen and len(chosen[key]) < want[key]:
                chosen[key].append(d)
                seen.add(json.dumps([d["labels"], d["edges"]]))
        out["rejected"] = old["rejected"]
        start_at = {tuple(k.split(":")): v for k, v in old.get("next_attempt", {}).items()}

    def save_partial(next_attempt):
        with open(partial, "w") as f:
            json.dump({"chosen": [d for v in chosen.values() for d in v], "rejected": out["rejected"],
                       "next_attempt": {"%s:%d" % k: v for k, v in next_attempt.items()}}, f)
    ctx = get_context("fork")
    with ctx.Pool(args.workers) as pool:
        next_attempt = {}
        for (kind, q), need in sorted(want.items()):
            attempt = int(start_at.get((kind, str(q)), 0))
            while len(chosen[(kind, q)]) < need and attempt < 20000:
                jobs = [(kind, q, attempt + i) for i in range(args.workers * 2)]
                attempt += len(jobs)
                for att, d, why in pool.map(_try, jobs):
                    if len(chosen[(kind, q)]) >= need:
                        break
                    if why is None:
                        key = json.dumps([d["labels"], d["edges"]])
                        if key in seen:
                            continue
                        seen.add(key)
                        d["attempt"] = att
                        d["kind"] = kind
                        chosen[(kind, q)].append(d)
                        print("keep", kind, q, att, d["sample_matches"], flush=True)
                    elif d is not None:
                        out["rejected"].append({"kind": kind, "q": q, "attempt": att, "why": why})
                next_attempt[(kind, q)] = attempt
                save_partial(next_attempt)
            if len(chosen[(kind, q)]) < need:
                raise SystemExit("could not find %d %s queries of %d vertices" % (need, kind, q))
    # emit in the order of the plan
    used = {k: 0 for k in chosen}
    for kind, q in plan:
        out["queries"].append(chosen[(kind, q)][used[(kind, q)]])
        used[(kind, q)] += 1
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    if os.path.exists(partial):
        os.remove(partial)
    print("wrote", path, len(out["queries"]), "queries,", len(out["rejected"]), "rejected")


if __name__ == "__main__":
    main()
