"""Expected per-update charged counts for the full-size parity tests, from
the CPU oracle alone.

For every batch a workload's test applies, and every stored query, the
check set is built as the query was selected (``make_queries.py``): every
``stride``-th update, and the ``heavy`` heaviest verifiable updates (going
down the updates whose endpoint labels match one of the query's edges by
decreasing product of endpoint degrees in the graph that batch meets, the
first ``heavy`` the oracle finishes within ``heavy_budget`` candidate tests
each; the walk stops after ``MAX_PASSED`` candidates were passed over).
Pairs the oracle cannot finish within their budget are passed over and
listed in the output; every pair of the check set is exact.  One worker
process per query, batch by batch.  Nothing here touches the CUDA path.

Batches: large -- the five consecutive batches of 800,000 insertions and
200,000 deletions; mid and batched -- the mid batch of 90,000 insertions
and 10,000 deletions; served -- the first ``SERVED_REQUESTS`` requests of the
served stream, each on the graph the previous ones leave.

Usage: python tests/golden/make_expected.py large|mid|batched|served [--workers 8]
Writes tests/golden/expected_NAME.json.  With --extend-passed, the pairs a
stored file lists as passed over are searched again, each split into
``PARTS`` parts run in parallel (their counts add up to the whole search,
pinned on the CPU), each part within the heavy budget; the pairs whose parts
all finish join the check set.
"""
import argparse
import hashlib
import json
import os
import sys
import time
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import make_queries as MQ  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2401_17018_gb300 import inputs as I  # noqa: E402

SERVED_REQUESTS = 4
# --extend-passed: a passed-over pair is searched again split into this many
# parts (the candidates of the first searched query vertex dealt
# round-robin), each within the heavy budget; when every part finishes the
# pair joins the check set with the parts' sum
PARTS = 8
# heavy candidates over budget passed over per (query, batch) before the walk
# stops (the check set then holds fewer heavy updates)
MAX_PASSED = 24

_S = None


def applied_batches(name, w):
    """(batches in order, each applied and committed before the next)."""
    wl = MQ.SPECS[name]["workload"]
    if wl == "large":
        return I.consecutive_batches(w, 5, 800_000, 200_000)
    if wl == "served":
        return I.served_stream(w, SERVED_REQUESTS, w.seed)
    return [I.workload_batch(w, 90_000, 10_000)]


def file_digest(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def _job(j):
    sess, queries, table, prod, sample, spec = _S
    got, heavy, passed, _ = MQ.check_pairs(sess, queries[j], table, prod, sample, spec, strict_sample=False,
                                           max_passed=MAX_PASSED)
    return j, got, heavy, passed


def _part(job):
    sess, queries, budget = _S
    j, u, p = job
    return j, u, p, int(sess.eval([queries[j]], eval_idx=[u], update_budget=budget, part=p, parts=PARTS)[0, 0])


def extend_passed(name, workers):
    """Search the passed-over pairs of the stored check sets again, each split
    into PARTS parts run in parallel, and move every pair whose parts all
    finish into the check set (marked heavy and extended)."""
    global _S
    spec = MQ.SPECS[name]
    path = os.path.join(HERE, "expected_%s.json" % name)
    with open(path) as f:
        out = json.load(f)
    qpath = os.path.join(HERE, "queries_%s.json" % name)
    assert out["queries_digest"] == file_digest(qpath)
    with open(qpath) as f:
        queries = [I.Query.from_json(x) for x in json.load(f)["queries"]]
    w = I.make_workload(spec["workload"])
    batches = applied_batches(name, w)
    src, dst = w.graph.src, w.graph.dst
    t0 = time.time()
    for k, b in enumerate(batches):
        rec = out["batches"][k]
        todo = [tuple(x) for x in rec["passed_over"]]
        if todo:
            _S = (O.Session(w.graph.n, w.graph.labels, src, dst, b), queries, spec["heavy_budget"])
            sums, bad = {}, set()
            with get_context("fork").Pool(workers) as pool:
                jobs = [(j, u, p) for j, u in todo for p in range(PARTS)]
                for j, u, p, c in pool.imap_unordered(_part, jobs):
                    if c == int(O.NOT_COMPUTED):
                        bad.add((j, u))
                    else:
                        sums[(j, u)] = sums.get((j, u), 0) + c
            _S[0].close()
            _S = None
            done = [x for x in todo if x not in bad]
            rec.setdefault("extended", [])
            for j, u in done:
                rec["query"].append(j)
                rec["update"].append(u)
                rec["count"].append(sums.get((j, u), 0))
                rec["heavy"].append(1)
                rec["extended"].append([j, u])
            rec["passed_over"] = [[j, u] for j, u in todo if (j, u) in bad]
            print("batch %d: %d of %d passed-over pairs verified in %d parts (%d matches), %d still passed over "
                  "[%.0f s]" % (k, len(done), len(todo), PARTS, sum(sums.get(x, 0) for x in done),
                                len(rec["passed_over"]), time.time() - t0), flush=True)
        src, dst = I.apply_batch_edges(src, dst, b)
    out["rule"] += ("; then every passed-over pair searched again in %d parts (the candidates of the first "
                    "searched query vertex dealt round-robin), each within %d candidate tests, joins the set "
                    "(listed under extended) when all parts finish" % (PARTS, spec["heavy_budget"]))
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


def main():
    global _S
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(MQ.SPECS))
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--extend-passed", action="store_true",
                    help="search the stored passed-over pairs again in parts and add those that finish")
    args = ap.parse_args()
    if args.extend_passed:
        return extend_passed(args.name, args.workers)
    spec = MQ.SPECS[args.name]
    qpath = os.path.join(HERE, "queries_%s.json" % args.name)
    with open(qpath) as f:
        qd = json.load(f)
    queries = [I.Query.from_json(x) for x in qd["queries"]]
    w = I.make_workload(spec["workload"])
    assert qd["graph_digest"] == w.graph.digest()
    batches = applied_batches(args.name, w)
    out = {"workload": spec["workload"], "queries_file": os.path.basename(qpath), "queries_digest": file_digest(qpath),
           "graph_digest": w.graph.digest(),
           "rule": "per batch and query: every %d-th update (within %d candidate tests each) and the %d heaviest "
                   "verifiable updates (going down the updates whose endpoint labels match one of the query's edges "
                   "by decreasing endpoint-degree product in the graph the batch meets, the first %d the oracle "
                   "finishes within %d candidate tests each, stopping after %d passed over); pairs over budget are "
                   "passed over and listed" % (spec["stride"], spec["sample_budget"], spec["heavy"], spec["heavy"],
                                               spec["heavy_budget"], MAX_PASSED),
           "batches": []}
    src, dst = w.graph.src, w.graph.dst
    t0 = time.time()
    for k, b in enumerate(batches):
        off, _ = I.csr_from_edges(w.graph.n, src, dst)
        deg = np.diff(off)
        table, prod = MQ.heavy_table(w.graph.labels, deg, b)
        sample = np.arange(0, len(b), spec["stride"], dtype=np.int64)
        _S = (O.Session(w.graph.n, w.graph.labels, src, dst, b), queries, table, prod, sample, spec)
        rec = {"index": k, "updates": len(b), "query": [], "update": [], "count": [], "heavy": [], "passed_over": []}
        with get_context("fork").Pool(args.workers) as pool:
            for j, got, heavy, passed in sorted(pool.imap_unordered(_job, range(len(queries))), key=lambda x: x[0]):
                hs = set(heavy)
                for u in sorted(got):
                    rec["query"].append(j)
                    rec["update"].append(u)
                    rec["count"].append(got[u])
                    rec["heavy"].append(1 if u in hs else 0)
                rec["passed_over"] += [[j, u] for u in passed]
        _S[0].close()
        _S = None
        out["batches"].append(rec)
        print("batch %d: %d pairs (%d heavy), %d matches, %d passed over [%.0f s]" % (
            k, len(rec["count"]), sum(rec["heavy"]), sum(rec["count"]), len(rec["passed_over"]), time.time() - t0),
            flush=True)
        src, dst = I.apply_batch_edges(src, dst, b)
    path = os.path.join(HERE, "expected_%s.json" % args.name)
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


if __name__ == "__main__":
    main()
