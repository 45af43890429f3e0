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

Some workloads add to the sample the updates whose endpoints have the largest
degree product in G0: on a power-law graph those updates carry most of a
query's work, which a uniform sample misses. Such a workload may also cap the
attempts per (class, size); slots that the cap leaves empty fall to the next
smaller size of the same class, and each stored query records the size it
was planned with (``q_planned``).

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

# per-workload sampling that differs from the defaults above: (stride, budget)
# per class, the heavy updates added to the sample, the attempt cap per
# (class, size), and the smallest size a slot may fall to
SAMPLING = {
    "batched": {"rules": {"dense_ge3": (1000, 20_000_000), "sparse": (1000, 20_000_000)},
                "heavy": 8, "max_attempts": 60},
    "served": {"rules": {"dense": (100, 2_400_000)}, "heavy": 8, "max_attempts": 200, "min_q": 5},
    "large": {"rules": {"dense": (20000, 3_000_000), "sparse": (20000, 3_000_000)},
              "heavy": 8, "max_attempts": 40, "min_q": 5},
}
DEFAULT_SAMPLING = {"rules": RULES, "heavy": 0, "max_attempts": 20000}

_W = None


def _init(name):
    global _W
    wl, ni, nd, _ = SPECS[name]
    w = I.make_workload(wl)
    b = I.workload_batch(w, ni, nd)
    off, nbr = I.csr_from_edges(w.graph.n, w.graph.src, w.graph.dst)
    samp = SAMPLING.get(name, DEFAULT_SAMPLING)
    deg = np.diff(off).astype(np.float64)
    prod = deg[b.src] * deg[b.dst]
    heavy = np.sort(np.argsort(-prod, kind="stable")[:samp["heavy"]])
    _W = (w, b, off, nbr, samp, heavy)


def _try(args):
    kind, q, attempt = args
    w, b, off, nbr, samp, heavy = _W
    g = w.graph
    Q = I.random_walk_query(off, nbr, g.labels, q, kind, w.seed + 1000 * q, attempt)
    if Q is None:
        return attempt, None, "class test failed"
    stride, budget = samp["rules"][kind]
    ev = np.union1d(np.arange(0, len(b), stride), heavy)
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
    w, samp, heavy = _W[0], _W[4], _W[5]
    rule = ("keep a candidate of class k when the CPU oracle finishes it on updates 0, s, 2s, ... of the "
            "batch within B candidate tests and finds at least one incremental match there; (s, B) per "
            "class: " + json.dumps(samp["rules"]))
    if samp["heavy"]:
        rule += ("; the sample also holds the %d updates with the largest product of endpoint degrees in G0 "
                 "(%s)" % (samp["heavy"], ", ".join(str(int(x)) for x in heavy)))
    if samp["max_attempts"] < DEFAULT_SAMPLING["max_attempts"]:
        rule += ("; at most %d attempts per (class, size), the slots left empty fall to the next smaller "
                 "size of the class" % samp["max_attempts"])
        if "min_q" in samp:
            rule += " (down to %d vertices)" % samp["min_q"]
    out = {"workload": wl, "graph_digest": w.graph.digest(), "batch": {"n_ins": ni, "n_del": nd, "sub": 0},
           "rule": rule, "queries": [], "rejected": []}
    want = {}
    for kind, q in plan:
        want[(kind, q)] = want.get((kind, q), 0) + 1
    kinds = sorted({k for k, _ in want})
    qmax = {k: max(q for kk, q in want if kk == k) for k in kinds}
    qmin = {k: min([q for kk, q in want if kk == k] + [samp.get("min_q", 99)]) for k in kinds}
    # every size from the largest down to the smallest, so shortfalls can fall
    classes = [(k, q) for k in kinds for q in range(qmax[k], qmin[k] - 1, -1)]
    chosen = {c: [] for c in classes}
    seen = set()
    path = os.path.join(HERE, "queries_%s.json" % args.name)
    partial = path + ".partial"
    start_at = {}
    if os.path.exists(partial):  # resume: keep what an interrupted run chose
        with open(partial) as f:
            old = json.load(f)
        for d in old["chosen"]:
            key = (d["kind"], len(d["labels"]))
            if key in chosen:
                chosen[key].append(d)
                seen.add(json.dumps([d["labels"], d["edges"]]))
        out["rejected"] = old["rejected"]
        start_at = {(k.split(":")[0], int(k.split(":")[1])): v for k, v in old.get("next_attempt", {}).items()}
    next_attempt = dict(start_at)

    def save_partial():
        with open(partial, "w") as f:
            json.dump({"chosen": [d for v in chosen.values() for d in v], "rejected": out["rejected"],
                       "next_attempt": {"%s:%d" % k: v for k, v in next_attempt.items()}}, f)
    cap = samp["max_attempts"]
    carry = {k: 0 for k in kinds}
    ctx = get_context("fork")
    with ctx.Pool(args.workers) as pool:
        for kind, q in classes:
            need = want.get((kind, q), 0) + carry[kind]
            attempt = int(start_at.get((kind, q), 0))
            got = chosen[(kind, q)]
            del got[need:]
            while len(got) < need and attempt < cap:
                jobs = [(kind, q, a) for a in range(attempt, min(attempt + args.workers * 2, cap))]
                attempt += len(jobs)
                for att, d, why in pool.map(_try, jobs):
                    if len(got) >= need:
                        break
                    if why is None:
                        key = json.dumps([d["labels"], d["edges"]])
                        if key in seen:
                            continue
                        seen.add(key)
                        d["attempt"] = att
                        d["kind"] = kind
                        got.append(d)
                        print("keep", kind, q, att, d["sample_matches"], flush=True)
                    elif d is not None:
                        out["rejected"].append({"kind": kind, "q": q, "attempt": att, "why": why})
                next_attempt[(kind, q)] = attempt
                save_partial()
            carry[kind] = need - len(got)
            if carry[kind]:
                print("short", kind, q, carry[kind], flush=True)
            if carry[kind] and q == qmin[kind]:
                raise SystemExit("could not find %d %s queries of %d vertices" % (carry[kind], kind, q))
    # assign to the plan's slots: a size's own slots first, then those that fell from above
    avail = {c: list(v) for c, v in chosen.items()}
    slot_of = {}
    for kind in kinds:
        falling = []
        for q in range(qmax[kind], qmin[kind] - 1, -1):
            planned = [q] * want.get((kind, q), 0) + falling
            take = avail[(kind, q)]
            for j, pq in enumerate(planned[:len(take)]):
                d = dict(take[j])
                d["q_planned"] = pq
                slot_of.setdefault((kind, pq), []).append(d)
            falling = planned[len(take):]
    used = {}
    for kind, q in plan:
        i = used.get((kind, q), 0)
        out["queries"].append(slot_of[(kind, q)][i])
        used[(kind, q)] = i + 1
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    if os.path.exists(partial):
        os.remove(partial)
    print("wrote", path, len(out["queries"]), "queries,", len(out["rejected"]), "rejected")


if __name__ == "__main__":
    main()
