"""Choose the query graphs of the benchmark workloads and store them as JSON.

Queries are extracted from G0 by the seeded extractor of
``paper_2401_17018_gb300.inputs.random_walk_query`` (Sec. VI-A: random
subgraphs of the data graph, classed by density), attempt after attempt, in
the sizes and classes each workload asks for; a size never falls to a
smaller one.  As in the paper, which leaves queries over a 30-minute cap
unsolved and out of its averages (Sec. VI-A "Metrics"), a candidate is kept
only when every pair of its check set can be verified by the CPU oracle:

* the check set of query Q on a batch = a uniform sample of the batch's
  updates (every ``stride``-th) and the ``heavy`` heaviest verifiable
  updates: going down the updates whose endpoint labels match some edge of
  Q (in either orientation) by decreasing product of endpoint degrees in
  the graph the batch meets (on a power-law graph those carry most of Q's
  work), the first ``heavy`` that the oracle finishes within
  ``heavy_budget`` candidate tests each (those it cannot finish are passed
  over and counted; only the first ``TOP_PER_PAIR`` per label pair are
  tried);
* the oracle must finish each sampled pair within ``sample_budget``
  candidate tests, find ``heavy`` verifiable heavy updates (with
  ``max_passed``: before passing over more than that many), and the check
  set must hold at least one incremental match.

Rejections are counted per class and reason in the output.  Nothing here
touches the CUDA path: the oracle alone decides.  The check sets of every
batch are later evaluated without budgets by ``make_expected.py``.

Usage: python tests/golden/make_queries.py large|mid|batched|served [--workers 8]
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

def interleave(a, b):
    """a[0], b[0], a[1], b[1], ... and then the rest of the longer list."""
    out = []
    for i in range(max(len(a), len(b))):
        out += a[i:i + 1] + b[i:i + 1]
    return out


SPECS = {
    # 6-vertex queries (the paper's default size), 4 sparse and 4 dense, on
    # the scale-23 graph; selected on the first of the five consecutive
    # batches.  (8-vertex random-walk queries on this graph need more than
    # 2e10 DFS expansion steps of one GB300 per 1M-update batch for 10 of 11
    # measured candidates, and none of about 400 candidates had its heavy
    # updates verifiable by the oracle.)
    "large": {"workload": "large", "plan": [("sparse", 6)] * 4 + [("dense", 6)] * 4,
              "stride": 20_000, "sample_budget": 10_000_000, "heavy": 8, "heavy_budget": 100_000_000,
              "max_passed": 8, "max_attempts": 4000},
    # 20 six-vertex queries, 10 sparse and 10 dense, on the scale-20 graph
    "mid": {"workload": "mid", "plan": [("sparse", 6)] * 10 + [("dense", 6)] * 10,
            "stride": 1000, "sample_budget": 10_000_000, "heavy": 8, "heavy_budget": 100_000_000,
            "max_attempts": 4000},
    # 64 queries of 4..7 vertices, on the mid graph: 38 sparse (average
    # degree < 3) of 4..6 vertices and 26 dense (average degree >= 3, the
    # paper's Dense class) of 4..7, the two classes alternating while both
    # last.  Larger ones were not verifiable: of 20 dense 9-vertex, 264
    # sparse 9-vertex, 72 sparse 7-vertex and 32 dense 8-vertex candidates,
    # none had its sampled updates within the sample budget and eight heavy
    # updates verifiable (dense 8-vertex ones that were took 6 to 25 minutes
    # of oracle time each, without the passed-over cap).
    "batched": {"workload": "mid", "plan": interleave([("sparse_lt3", q) for q, n in ((4, 14), (5, 14), (6, 10))
                                                       for _ in range(n)],
                                                      [("dense_ge3", q) for q, n in ((4, 7), (5, 7), (6, 6), (7, 6))
                                                       for _ in range(n)]),
                "stride": 10_000, "sample_budget": 10_000_000, "heavy": 8, "heavy_budget": 100_000_000,
                "max_passed": 8, "max_passed_by_size": {7: 24, 8: 24}, "max_attempts": 6000},
    # 16 dense queries on the scale-22 served graph, 14 of 6 vertices and 2
    # of 7 (dense 7-vertex candidates verified at about one per 25 minutes of
    # oracle time, 2 of 20; none of 12 dense 8-vertex ones did); the
    # selection batch has the served stream's 1:1 mix of insertions and
    # deletions
    "served": {"workload": "served", "plan": [("dense", 7 if i in (7, 15) else 6) for i in range(16)],
               "stride": 10_000, "sample_budget": 10_000_000, "heavy": 8, "heavy_budget": 100_000_000,
               "max_passed": 8, "max_passed_by_size": {7: 24, 8: 24}, "max_attempts": 6000},
}
TOP_PER_PAIR = 64  # heavy candidates kept per endpoint-label pair

_S = None


def selection_batch(name, w):
    """The batch a workload's queries are chosen on."""
    wl = SPECS[name]["workload"]
    if wl == "large":
        return I.consecutive_batches(w, 1, 800_000, 200_000)[0]
    if wl == "served":
        return I.workload_batch(w, 50_000, 50_000)
    return I.workload_batch(w, 90_000, 10_000)


def heavy_table(labels, deg, b, top=TOP_PER_PAIR):
    """For every unordered endpoint-label pair, the batch's updates with that
    pair, by decreasing product of endpoint degrees (ties: smaller index)."""
    la, lb = labels[b.src], labels[b.dst]
    lo, hi = np.minimum(la, lb), np.maximum(la, lb)
    prod = deg[b.src].astype(np.float64) * deg[b.dst].astype(np.float64)
    order = np.lexsort((np.arange(len(b)), -prod))
    table = {}
    for k in order:
        key = (int(lo[k]), int(hi[k]))
        lst = table.setdefault(key, [])
        if len(lst) < top:
            lst.append(int(k))
    return table, prod


def heavy_candidates(q, table, prod):
    """The updates label-compatible with some edge of q (the first
    TOP_PER_PAIR of each endpoint-label pair), by decreasing endpoint-degree
    product (ties: smaller index)."""
    cand = set()
    for a, c in zip(q.src.tolist(), q.dst.tolist()):
        la, lc = int(q.labels[a]), int(q.labels[c])
        cand.update(table.get((min(la, lc), max(la, lc)), []))
    return sorted(cand, key=lambda k: (-prod[k], k))


def check_pairs(sess, Q, table, prod, sample, spec, strict_sample, max_passed=None):
    """Evaluate Q's check set on one batch, one pair at a time: the sampled
    updates within the sample budget, then the heaviest verifiable updates.
    Returns (counts by update, heavy updates, passed-over updates, reason):
    reason is None when the set is complete; with strict_sample a sampled
    update over budget is a reason (selection), else it is passed over.
    max_passed: stop looking for heavy updates after that many were passed
    over (the set then holds fewer)."""
    got, passed = {}, []
    for u in sample.tolist():
        c = int(sess.eval([Q], eval_idx=[u], update_budget=spec["sample_budget"])[0, 0])
        if c == int(O.NOT_COMPUTED):
            if strict_sample:
                return got, [], passed, "a sampled update needs more than the sample budget"
            passed.append(u)
            continue
        got[u] = c
    heavy = []
    for u in heavy_candidates(Q, table, prod):
        if len(heavy) == spec["heavy"]:
            break
        if u in got:
            heavy.append(u)
            continue
        if max_passed is not None and len(passed) >= max_passed:
            break
        c = int(sess.eval([Q], eval_idx=[u], update_budget=spec["heavy_budget"])[0, 0])
        if c == int(O.NOT_COMPUTED):
            passed.append(u)
            continue
        got[u] = c
        heavy.append(u)
    if len(heavy) < spec["heavy"]:
        return got, heavy, passed, "fewer verifiable heavy updates than required"
    return got, heavy, passed, None


def rule_text(spec):
    """The selection rule, in words, as stored with the queries."""
    return ("keep a candidate when the CPU oracle verifies its check set on the selection batch: every %d-th "
            "update within %d candidate tests each, and the %d heaviest verifiable updates (going down the updates "
            "whose endpoint labels match one of the query's edges by decreasing endpoint-degree product, the first "
            "%d finished within %d candidate tests each; heavier ones are passed over and counted%s); the check "
            "set must hold an incremental match; at most %d attempts per (class, size), no fall to smaller sizes" % (
                spec["stride"], spec["sample_budget"], spec["heavy"], spec["heavy"], spec["heavy_budget"],
                (", at most %d of them" % spec["max_passed"] +
                 "".join(", %d for %d vertices" % (v, k) for k, v in sorted(spec.get("max_passed_by_size", {}).items())))
                if spec.get("max_passed") else "",
                spec["max_attempts"]))


def max_passed_for(spec, q):
    """Heavy candidates a q-vertex query may pass over (None: no limit)."""
    return spec.get("max_passed_by_size", {}).get(q, spec.get("max_passed"))


def _init(name):
    global _S
    spec = SPECS[name]
    w = I.make_workload(spec["workload"])
    b = selection_batch(name, w)
    off, nbr = I.csr_from_edges(w.graph.n, w.graph.src, w.graph.dst)
    deg = np.diff(off)
    table, prod = heavy_table(w.graph.labels, deg, b)
    sess = O.Session(w.graph.n, w.graph.labels, w.graph.src, w.graph.dst, b)
    sample = np.arange(0, len(b), spec["stride"], dtype=np.int64)
    _S = (spec, w, b, off, nbr, table, prod, sess, sample)


def _try(args):
    kind, q, attempt = args
    spec, w, b, off, nbr, table, prod, sess, sample = _S
    g = w.graph
    Q = I.random_walk_query(off, nbr, g.labels, q, kind, w.seed + 1000 * q, attempt)
    if Q is None:
        return attempt, None, "class test failed"
    t = time.time()
    got, heavy, passed, why = check_pairs(sess, Q, table, prod, sample, spec, strict_sample=True,
                                          max_passed=max_passed_for(spec, q))
    if why is not None:
        return attempt, None, why
    if sum(got.values()) == 0:
        return attempt, None, "no incremental match in the check set"
    d = Q.to_json()
    d["kind"] = kind
    d["attempt"] = attempt
    d["sample_matches"] = int(sum(got[u] for u in sample.tolist()))
    d["heavy_matches"] = int(sum(got[u] for u in heavy))
    d["heavy_passed_over"] = len(passed)
    d["check_seconds"] = round(time.time() - t, 2)
    return attempt, d, None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(SPECS))
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--kind", default=None, help="select only this class (the partial results are merged by --merge)")
    ap.add_argument("--sizes", default=None, help="select only these sizes, e.g. 7,8 (with --kind)")
    ap.add_argument("--need", type=int, default=0,
                    help="with --kind: keep up to this many per size instead of the plan's count")
    ap.add_argument("--merge", action="store_true", help="merge the per-class partial files into the output")
    args = ap.parse_args()
    spec = SPECS[args.name]
    if args.merge:
        return merge(args.name)
    _init(args.name)
    w, b = _S[1], _S[2]
    rule = rule_text(spec)
    out = {"workload": spec["workload"], "graph_digest": w.graph.digest(), "selection_batch_updates": len(b),
           "rule": rule, "queries": [], "rejected": {}}
    want = {}
    sizes = {int(x) for x in args.sizes.split(",")} if args.sizes else None
    for kind, q in spec["plan"]:
        if (args.kind is None or kind == args.kind) and (args.sizes is None or q in sizes):
            want[(kind, q)] = want.get((kind, q), 0) + 1
    if args.need and args.kind is not None:
        want = {c: args.need for c in want}
    chosen = {c: [] for c in want}
    seen = set()
    ctx = get_context("fork")  # the workers share the parent's graph and oracle session
    t0 = time.time()
    partial = None
    if args.kind is not None:
        partial = os.path.join(HERE, "queries_%s.%s%s.partial" % (
            args.name, args.kind, ".q" + "-".join(str(q) for q in sorted(sizes)) if sizes else ""))
    rej_log = {}

    def write_partial(complete):
        # results arrive in attempt order, so the queries kept so far are the
        # first ones of their group among the attempts examined so far
        out["chosen"] = {"%s:%d" % k: v for k, v in chosen.items()}
        out["rejections"] = rej_log
        out["complete"] = complete
        with open(partial, "w") as f:
            json.dump(out, f, indent=1)

    with ctx.Pool(args.workers) as pool:
        for (kind, q), need in sorted(want.items()):
            got = chosen[(kind, q)]
            attempt = 0
            rej = out["rejected"].setdefault("%s:%d" % (kind, q), {})
            log = rej_log.setdefault("%s:%d" % (kind, q), [])
            while len(got) < need and attempt < spec["max_attempts"]:
                jobs = [(kind, q, a) for a in range(attempt, min(attempt + args.workers * 4, spec["max_attempts"]))]
                attempt += len(jobs)
                print("%s %d: attempts %d, kept %d, rejected %s [%.0fs]" % (kind, q, attempt - len(jobs), len(got),
                                                                         json.dumps(rej), time.time() - t0), flush=True)
                for att, d, why in pool.imap(_try, jobs):
                    if len(got) >= need:
                        break
                    if why is not None:
                        rej[why] = rej.get(why, 0) + 1
                        log.append([att, why])
                        continue
                    key = json.dumps([d["labels"], d["edges"]])
                    if key in seen:
                        log.append([att, "the same query as an earlier attempt"])
                        continue
                    seen.add(key)
                    got.append(d)
                    print("keep %s %d attempt %d: sample %d heavy %d (%.1fs) [%.0fs]" % (
                        kind, q, att, d["sample_matches"], d["heavy_matches"], d["check_seconds"],
                        time.time() - t0), flush=True)
                    if partial:
                        write_partial(False)
            rej["attempts"] = attempt
            if len(got) < need:
                if partial:
                    write_partial(False)
                raise SystemExit("found only %d of %d %s queries of %d vertices in %d attempts" % (
                    len(got), need, kind, q, attempt))
    if partial:  # one class: a partial file, merged later
        write_partial(True)
        print("wrote", partial, "in %.0f s" % (time.time() - t0))
        return
    used = {}
    for kind, q in spec["plan"]:
        i = used.get((kind, q), 0)
        out["queries"].append(chosen[(kind, q)][i])
        used[(kind, q)] = i + 1
    path = os.path.join(HERE, "queries_%s.json" % args.name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, len(out["queries"]), "queries in %.0f s" % (time.time() - t0))


def merge(name, here=HERE, spec=None):
    """Assemble queries_NAME.json from the partial files (one per class, or
    per class and sizes) in ``here``."""
    spec = spec or SPECS[name]
    chosen, rejected, logs, head = {}, {}, {}, None
    parts = sorted(f for f in os.listdir(here) if f.startswith("queries_%s." % name) and f.endswith(".partial"))
    for fn in parts:
        with open(os.path.join(here, fn)) as f:
            d = json.load(f)
        head = head or d
        rejected.update(d["rejected"])
        logs.update(d.get("rejections", {}))
        for key, v in d["chosen"].items():
            k, q = key.split(":")
            chosen[(k, int(q))] = v
    need = {}
    for kind, q in spec["plan"]:
        need[(kind, q)] = need.get((kind, q), 0) + 1
    for c, n in need.items():
        if len(chosen.get(c, [])) < n:
            raise SystemExit("the partial files hold %d %s queries of %d vertices, the plan needs %d" % (
                len(chosen.get(c, [])), c[0], c[1], n))
        chosen[c] = chosen[c][:n]
        key = "%s:%d" % c
        if key in logs:  # rejections among the attempts before the last query used
            last = chosen[c][-1]["attempt"]
            r = {}
            for att, why in logs[key]:
                if att < last:
                    r[why] = r.get(why, 0) + 1
            r["attempts"] = last + 1
            rejected[key] = r
    keys = [json.dumps([d["labels"], d["edges"]]) for c in need for d in chosen[c]]
    if len(set(keys)) != len(keys):
        raise SystemExit("the partial files hold the same query twice")
    out = {k: head[k] for k in ("workload", "graph_digest", "selection_batch_updates")}
    out["rule"] = rule_text(spec)
    out["queries"], out["rejected"] = [], {c: rejected[c] for c in sorted("%s:%d" % k for k in need)}
    used = {}
    for kind, q in spec["plan"]:
        i = used.get((kind, q), 0)
        out["queries"].append(chosen[(kind, q)][i])
        used[(kind, q)] = i + 1
    path = os.path.join(here, "queries_%s.json" % name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, len(out["queries"]), "queries")
    return out


if __name__ == "__main__":
    main()
