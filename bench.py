#!/usr/bin/env python3
"""Benchmark of batch-dynamic subgraph matching (BDSM) on GB300.

One step = one pass of the whole hot path over one update batch: stage the
batch into the device-resident dynamic CSR, seed, DFS extension with match
counting, counts back to the host, commit.

Default workload ("large"): R-MAT scale 23 (a, b, c = .57, .19, .19),
67,108,864 unique edges of which 90% form G0, 16 vertex labels Zipf(1.0),
8 eight-vertex queries (4 sparse, 4 dense) from tests/golden/queries_large.json,
five consecutive batches of 800,000 insertions from the held-out pool +
200,000 uniform deletions from the current graph, each committed before the
next.  Step k applies batch k mod 5; after the fifth batch G0 is restored
outside the timed region by applying the five inverse batches in reverse
order with no queries (stage and commit only).  Workload "mid": R-MAT scale
20, 8 labels Zipf(1.2), 20 six-vertex queries, one batch of 90,000
insertions + 10,000 deletions, steps alternating the batch and its inverse.
Inputs are synthetic (the paper's datasets are not available).  L2 is
flushed (a 256 MiB write) before every timed step, outside the timed events.

value   = updates/s with the batches already in HBM (device events per step)
e2e     = the same metric through the C-ABI with host (pinned) batch buffers
roofline: the DFS kernel's algorithmic bytes (per candidate slot, search
          step, probe and prepared entry; counted by an untimed launch of the
          instrumented build on the first batch) / that batch's timed DFS
          duration, against the measured HBM copy bandwidth; the L2 read
          bandwidth measured by the library's probe kernel is reported beside
cpu_baseline: the CPU oracle on a bounded sample of the first batch.
--impl reference times that oracle alone, as the reference arm.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "large": {"workload": "large", "queries": "tests/golden/queries_large.json", "n_ins": 800_000,
              "n_del": 200_000, "batches": 5},
    "mid": {"workload": "mid", "queries": "tests/golden/queries_mid.json", "n_ins": 90_000, "n_del": 10_000},
    # the same graph, queries and batch cut to its first 3,000 updates: a case
    # small enough for multi-pass profiler captures
    "mid_3k": {"workload": "mid", "queries": "tests/golden/queries_mid.json", "n_ins": 90_000, "n_del": 10_000,
               "first": 3000},
    # the first 20,000 updates: every warp stays busy for about a second, so a
    # profiler capture sees the steady state of the full batch
    "mid_20k": {"workload": "mid", "queries": "tests/golden/queries_mid.json", "n_ins": 90_000, "n_del": 10_000,
                "first": 20000},
    # the large graph and queries with the first 20,000 / 100,000 updates of
    # its first batch: profiling cases for the kernel on the large graph
    "large_20k": {"workload": "large", "queries": "tests/golden/queries_large.json", "n_ins": 800_000,
                  "n_del": 200_000, "batches": 1, "first": 20000},
    "large_100k": {"workload": "large", "queries": "tests/golden/queries_large.json", "n_ins": 800_000,
                   "n_del": 200_000, "batches": 1, "first": 100000},
    "tiny": {"workload": "tiny", "queries": None, "n_ins": 256, "n_del": 0},
}
DESCRIBE = {
    "large": "R-MAT scale 23, 60.4M edges, 16 labels Zipf(1.0), %d queries of %s vertices, five consecutive "
             "batches of 1,000,000 updates (800,000 ins + 200,000 del) with a commit after each, one batch per step",
    "large_20k": "R-MAT scale 23, 60.4M edges, 16 labels Zipf(1.0), %d queries of %s vertices, the first 20,000 "
                 "updates of the first large batch, batch and inverse alternating",
    "large_100k": "R-MAT scale 23, 60.4M edges, 16 labels Zipf(1.0), %d queries of %s vertices, the first 100,000 "
                  "updates of the first large batch, batch and inverse alternating",
    "mid": "R-MAT scale 20, 7.55M edges, 8 labels Zipf(1.2), %d queries of %s vertices, batch of 100,000 updates "
           "(90,000 ins + 10,000 del), batch and inverse alternating",
    "mid_3k": "R-MAT scale 20, 7.55M edges, 8 labels Zipf(1.2), %d queries of %s vertices, the first 3,000 updates "
              "of the mid batch, batch and inverse alternating",
    "mid_20k": "R-MAT scale 20, 7.55M edges, 8 labels Zipf(1.2), %d queries of %s vertices, the first 20,000 "
               "updates of the mid batch, batch and inverse alternating",
    "tiny": "R-MAT scale 11, 9k edges, 4 labels, %d query of %s vertices, 256 insertions, batch and inverse "
            "alternating",
}
METRIC = "updates/s & incremental matches/s per batch (1 GB300); p50/p99 batch latency"
STATUS_BYTES = 112  # the library's status block, read back after staging, matching and commit
# batched / served modes: a bound on one apply's DFS work (32-wide expansion
# steps, about a minute of GPU time), so a workload heavier than intended
# fails with GAMMA_ETIMEOUT instead of running on
WORK_BUDGET = 100_000_000_000


def load_workload(name):
    """(workload, queries, timed batches, restore batches): the timed steps
    cycle through the timed batches; after each full cycle the restore
    batches (applied untimed, with no queries) bring the graph back to G0."""
    from paper_2401_17018_gb300 import inputs as I
    spec = WORKLOADS[name]
    w = I.make_workload(spec["workload"])
    if spec["queries"]:
        with open(os.path.join(ROOT, spec["queries"])) as f:
            qd = json.load(f)
        if qd.get("graph_digest") not in (None, w.graph.digest()):
            raise SystemExit("stored queries were chosen on a different graph")
        queries = [I.Query.from_json(x) for x in qd["queries"]]
    else:
        queries = [I.TRIANGLE_WITH_TAIL]
    if "batches" in spec:
        batches = I.consecutive_batches(w, spec["batches"], spec["n_ins"], spec["n_del"])
    else:
        batches = [I.workload_batch(w, spec["n_ins"], spec["n_del"])]
    if "first" in spec:
        k = spec["first"]
        batches = [I.Batch(b.op[:k].copy(), b.src[:k].copy(), b.dst[:k].copy()) for b in batches[:1]]
    if len(batches) == 1:  # the batch and its inverse alternate; both are timed
        return w, queries, [batches[0], batches[0].inverse()], []
    return w, queries, batches, [b.inverse() for b in reversed(batches)]


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
                pw.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(pw) if pw else None,
                "other_gpu_processes": other_processes(self.device)}


def other_processes(device):
    """Compute processes on the device other than this one (contention evidence)."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(device), "--query-compute-apps=pid,process_name,used_memory",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20).stdout
    except (OSError, subprocess.SubprocessError):
        return None
    me = os.getpid()
    rows = []
    for ln in out.splitlines():
        p = [x.strip() for x in ln.split(",")]
        if len(p) >= 3 and p[0].isdigit() and int(p[0]) != me:
            rows.append({"pid": int(p[0]), "name": p[1], "mib": p[2]})
    return rows


def max_over_ranks(seconds, dist=None, device="cpu"):
    """The slowest rank's time: every rank receives the maximum of the ranks'
    local values (one all-reduce), so the reported rate is the whole job's."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units per second over the job: replicas each process the whole
    workload, so the job processes world x units in the slowest rank's time."""
    return world * units_per_rank / seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dfs_traffic(workload, kernel_file="paper_2401_17018_gb300/csrc/gm_match.cu"):
    """DRAM bytes per DFS launch from the committed ncu summary, if it was
    taken on this workload and on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "dfs_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256(open(os.path.join(ROOT, kernel_file), "rb").read()).hexdigest()[:16]
    if d.get("source_sha") != h or d.get("workload") != workload:
        return None
    return d.get("dram_bytes_per_launch")


def sample_order(n):
    """A seeded uniform order of the updates of a batch (the CPU samples)."""
    from paper_2401_17018_gb300 import inputs as I
    return np.argsort(I.rand_u64(7, 99, np.arange(n, dtype=np.uint64)), kind="stable")


def cpu_baseline(w, queries, batch, budget_s=15.0):
    """The oracle, single-threaded, on a sample of the batch's updates (all
    queries): G, the batch and G' are built once (timed apart and reported,
    not counted), then updates drawn in a seeded uniform order are evaluated
    in calls of k updates, k doubling while a call takes under half a second,
    until about budget_s seconds of search or the whole batch."""
    from oracle import oracle as O
    g = w.graph
    t = time.perf_counter()
    sess = O.Session(g.n, g.labels, g.src, g.dst, batch)
    build_s = time.perf_counter() - t
    order = sample_order(len(batch))
    done, total_s, k = 0, 0.0, 1
    while total_s < budget_s and done < len(batch):
        ev = np.sort(order[done:done + k])
        t = time.perf_counter()
        sess.eval(queries, eval_idx=ev)
        dt = time.perf_counter() - t
        total_s += dt
        done += ev.size
        if dt < 0.5:
            k *= 2
    sess.close()
    return {"value": done / max(total_s, 1e-9), "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": "%d updates of the first batch drawn uniformly (seeded), all %d queries, single thread, "
                      "%.2f s of search; building G, the batch and G' (%.1f s, once) excluded" % (
                          done, len(queries), total_s, build_s)}


def run_reference(args):
    """The reference arm: the CPU oracle on the same workload, rank 0 only.
    Each step evaluates, through one oracle session on G0 and the first
    batch (built before the timed steps), updates of that batch in a seeded
    uniform order until the step has searched for about step_s seconds."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    w, queries, timed, _ = load_workload(args.workload)
    batch = timed[0]
    g = w.graph
    t = time.perf_counter()
    sess = O.Session(g.n, g.labels, g.src, g.dst, batch)
    build_s = time.perf_counter() - t
    order = sample_order(len(batch))
    step_s = 1.0
    times, nupd, pos = [], [], 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        n = 0
        while True:
            sess.eval(queries, eval_idx=[int(order[pos % len(batch)])])
            pos += 1
            n += 1
            if time.perf_counter() - t0 >= step_s:
                break
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            nupd.append(n)
    sess.close()
    v = sum(nupd) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": config_of(args.workload, len(batch), queries, len(timed)),
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "sample": "per step about %.1f s of single-thread search over updates of the first "
                                       "batch in a seeded uniform order (%d updates in all), all %d queries; "
                                       "G, the batch and G' built once before the steps (%.1f s)" % (
                                           step_s, sum(nupd), len(queries), build_s)},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(workload, b, queries, nbatches):
    sizes = sorted({int(q.labels.size) for q in queries})
    qdesc = "%d" % sizes[0] if len(sizes) == 1 else "%d..%d" % (sizes[0], sizes[-1])
    return {"workload": "%s: %s" % (workload, DESCRIBE[workload] % (len(queries), qdesc)),
            "batch_updates": b, "queries": len(queries), "timed_batches": nbatches,
            "l2": "flushed before every timed step (256 MiB write)",
            "step": "apply one batch (stage+seed+DFS+counts to host) + commit"}


def run_batched(args):
    """Batched form: the same batch and the 64 stored batched queries,
    (1) plain: one seed + DFS launch sequence per query, (2) batched: one
    launch over all queries' seeds, autotuned and replayed as a CUDA graph.
    (3) the batched form with its work created query by query (the launch
    shape the autotuner chose for (2)). All must give identical counts."""
    import torch
    from paper_2401_17018_gb300 import gamma as G
    from paper_2401_17018_gb300 import inputs as I
    torch.cuda.set_device(0)
    w = I.make_workload("mid")
    with open(os.path.join(ROOT, "tests/golden/queries_batched.json")) as f:
        qd = json.load(f)
    if qd.get("graph_digest") not in (None, w.graph.digest()):
        raise SystemExit("stored queries were chosen on a different graph")
    queries = [I.Query.from_json(x) for x in qd["queries"]]
    batch = I.workload_batch(w, 90_000, 10_000)
    if args.first:
        batch = I.Batch(batch.op[:args.first].copy(), batch.src[:args.first].copy(), batch.dst[:args.first].copy())
    inv = batch.inverse()
    g = w.graph
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_b = (dev(batch.op), dev(batch.src), dev(batch.dst))
    d_i = (dev(inv.op), dev(batch.src), dev(batch.dst))
    grid = [(wpb, t, gr) for wpb in (4, 8, 16) for t in (32, 64, 128, 256, 512) for gr in (1, 2, 4, 8, 16)]
    if not args.full_grid:  # a frontier tile of 128 or more halves the resident warps: always slower here
        grid = [(wpb, 64, gr) for wpb in (4, 8, 16) for gr in (4, 16, 64)]
    out = {}
    counts = {}
    tuned = None
    for form, flags in (("plain", G.GAMMA_F_PER_QUERY), ("batched", G.GAMMA_F_GRAPH),
                        ("batched_by_query", G.GAMMA_F_GRAPH | G.GAMMA_F_SEED_BY_QUERY)):
        stream = torch.cuda.Stream()
        ctx = G.Context(stream=stream, flags=flags, work_budget=WORK_BUDGET)
        ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        sweep = None
        if form == "batched":
            ctx.apply_batch(*d_b, qids)
            tuned, sweep = G.gamma_autotune(ctx.h, grid, repeats=1)
            ctx.commit()
            ctx.apply_batch(*d_i, qids)
            ctx.commit()
        elif form == "batched_by_query":  # the launch shape the autotuner chose for the batched form
            ctx.set_options(warps_per_block=tuned["warps_per_block"], frontier_tile=tuned["frontier_tile"],
                            steal_grain=tuned["steal_grain"])
        applied = 0
        for k in range(args.warmup):
            ctx.apply_batch(*(d_b if applied % 2 == 0 else d_i), qids)
            ctx.commit()
            applied += 1
        if applied % 2:
            ctx.apply_batch(*d_i, qids)
            ctx.commit()
            applied += 1
        ms, res = [], []
        launches0 = ctx.stats()["kernel_launches"]
        for k in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pos, neg = ctx.apply_batch(*(d_b if applied % 2 == 0 else d_i), qids)
            ctx.commit()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            if applied % 2 == 0:
                res.append((pos.tolist(), neg.tolist()))
            applied += 1
        st = ctx.stats()
        out[form] = {"updates_per_s": len(batch) * len(ms) / (sum(ms) / 1e3), "ms_per_step": sum(ms) / len(ms),
                     "p50_ms": statistics.median(ms), "p99_ms": float(np.percentile(ms, 99)),
                     "gpu_launches_per_step": (st["kernel_launches"] - launches0) / len(ms),
                     "graph_captures": st["graph_captures"]}
        if form != "plain":
            out[form]["tuned"] = tuned
        if sweep:
            out[form]["sweep"] = sweep
        counts[form] = res[0] if res else None
        ctx.close()
    same = counts["plain"] == counts["batched"] == counts["batched_by_query"]
    line = {"metric": "batched vs plain per-query launches: updates/s and p99 batch latency (1 GB300)",
            "mode": "batched", "config": {"workload": "batched: R-MAT scale 20, %d queries of %d..%d vertices "
                                                      "(sparse and dense alternating), %s" % (
                                                          len(queries), min(q.labels.size for q in queries),
                                                          max(q.labels.size for q in queries),
                                                          "the first %d updates of the batch" % len(batch)
                                                          if args.first else "batch 100000 (90000 ins + 10000 del)"),
                                          "batch_updates": len(batch)},
            "steps": args.steps, "warmup": args.warmup, "identical_counts": same,
            "incremental_matches_per_step": int(sum(counts["plain"][0]) + sum(counts["plain"][1])) if counts["plain"] else None,
            "plain": out["plain"], "batched": out["batched"], "batched_by_query": out["batched_by_query"],
            "speedup": out["batched"]["updates_per_s"] / out["plain"]["updates_per_s"],
            "speedup_by_query": out["batched_by_query"]["updates_per_s"] / out["plain"]["updates_per_s"]}
    print(json.dumps(line), flush=True)
    if not same:
        raise SystemExit("batched and plain forms disagree")


def run_served(args):
    """Served form: a stream of uneven batches arriving as a Poisson
    process at a fraction of the closed-loop capacity; one request at a time
    ("plain") vs continuous batching ("served"); latency from arrival."""
    import threading as th
    import torch
    from paper_2401_17018_gb300 import gamma as G
    from paper_2401_17018_gb300 import inputs as I
    torch.cuda.set_device(0)
    w = I.make_workload("served")
    with open(os.path.join(ROOT, "tests/golden/queries_served.json")) as f:
        qd = json.load(f)
    if qd.get("graph_digest") not in (None, w.graph.digest()):
        raise SystemExit("stored queries were chosen on a different graph")
    queries = [I.Query.from_json(x) for x in qd["queries"]]
    stream_b = I.served_stream(w, args.batches, w.seed, args.size_exp[0], args.size_exp[1])
    total = sum(len(b) for b in stream_b)
    g = w.graph
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_graph = (dev(g.labels), dev(g.src), dev(g.dst))
    # the budget bounds one apply, and a served group of up to 64 requests is one apply
    ctx = G.Context(stream=torch.cuda.Stream(), work_budget=WORK_BUDGET * 64)

    def fresh():
        ctx.load_graph(g.n, *d_graph)
        return [ctx.register_query(q.labels, q.src, q.dst) for q in queries]

    # closed-loop capacity: every batch applied and committed back to back
    qids = fresh()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for b in stream_b:
        ctx.apply_batch(b.op, b.src, b.dst, qids)
        ctx.commit()
    cap = total / (time.perf_counter() - t)
    mean_b = total / len(stream_b)
    runs = {}
    for load in args.loads:
        gaps = I.poisson_gaps(len(stream_b), w.seed + int(load * 1000), load * cap / mean_b)
        arrive = np.cumsum(gaps)
        per_form = {}
        for form, maxreq in (("plain", 1), ("served", 64)):
            qids = fresh()
            srv = G.Server(ctx, qids, max_requests=maxreq)
            tickets = [None] * len(stream_b)
            t0 = time.perf_counter()

            def submit():
                for k, b in enumerate(stream_b):
                    dt = arrive[k] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    tickets[k] = srv.submit(b.op, b.src, b.dst)

            th_sub = th.Thread(target=submit)
            th_sub.start()
            th_sub.join()
            res, lat, groups, first, last = [], [], [], None, None
            for k in range(len(stream_b)):
                rc, pos, neg, info = srv.wait(tickets[k])
                if rc != G.GAMMA_OK:
                    raise SystemExit("request %d failed with %d" % (k, rc))
                res.append((pos.tolist(), neg.tolist()))
                lat.append(info["done_ms"] - info["arrival_ms"])
                groups.append(info["group_size"])
                first = info["arrival_ms"] if first is None else min(first, info["arrival_ms"])
                last = info["done_ms"] if last is None else max(last, info["done_ms"])
            sst = srv.stats()
            srv.stop()
            per_form[form] = {"p50_ms": statistics.median(lat), "p99_ms": float(np.percentile(lat, 99)),
                              "mean_ms": float(np.mean(lat)),
                              "sustained_updates_per_s": total / ((last - first) / 1e3),
                              "groups": sst["groups"], "max_group": sst["max_group"], "_res": res}
        same = per_form["plain"].pop("_res") == per_form["served"].pop("_res")
        if not same:
            raise SystemExit("served results differ from one-at-a-time results at load %.2f" % load)
        runs["%.2f" % load] = dict(per_form, identical_counts=same)
    line = {"metric": "served form: p50/p99 batch latency from arrival and sustained updates/s (1 GB300)",
            "mode": "served",
            "config": {"workload": "served: R-MAT scale 22, 8 labels Zipf(1.2), %d %s queries of %d..%d "
                                   "vertices, %d batches of floor(10^U(%g,%g)) updates (ins:del 1:1), Poisson "
                                   "arrivals" % (len(queries), "/".join(sorted({q.kind for q in queries})),
                                                 min(q.labels.size for q in queries),
                                                 max(q.labels.size for q in queries), len(stream_b),
                                                 args.size_exp[0], args.size_exp[1]),
                       "updates": total},
            "closed_loop_capacity_updates_per_s": cap, "loads": runs}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gamma", choices=["gamma", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hub-min-degree", type=int, default=0, help="lists that get a hash index (0: the library's default)")
    ap.add_argument("--tile", type=int, default=0, help="DFS frontier tile (0: default)")
    ap.add_argument("--wpb", type=int, default=0, help="DFS warps per block (0: default)")
    ap.add_argument("--grain", type=int, default=0, help="level-2 candidates per work item (0: default)")
    ap.add_argument("--per-query", action="store_true", help="plain form: one launch sequence per query")
    ap.add_argument("--mode", default="plain", choices=["plain", "batched", "served"],
                    help="plain: the metric's workload; batched / served: the batched and served forms")
    ap.add_argument("--full-grid", action="store_true", help="batched mode: sweep the whole autotuner grid")
    ap.add_argument("--first", type=int, default=0,
                    help="batched mode: keep only the first N updates of the batch (0 = all)")
    ap.add_argument("--batches", type=int, default=2000, help="served mode: batches in the stream")
    ap.add_argument("--size-exp", type=float, nargs=2, default=[3.0, 6.0],
                    help="served mode: batch sizes floor(10^U(a, b))")
    ap.add_argument("--loads", type=float, nargs="+", default=[0.5, 0.8, 0.95],
                    help="served mode: offered load as fractions of the closed-loop capacity")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "served":
        return run_served(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2401_17018_gb300 import gamma as G

    w, queries, timed, restore = load_workload(args.workload)
    g = w.graph
    stream = torch.cuda.Stream()
    flags = G.GAMMA_F_PER_QUERY if args.per_query else 0
    ctx = G.Context(device=local, stream=stream, flags=flags, hub_min_degree=args.hub_min_degree,
                    frontier_tile=args.tile, warps_per_block=args.wpb, steal_grain=args.grain)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
    qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
    d_timed = [(dev(b.op), dev(b.src), dev(b.dst)) for b in timed]
    h_timed = [(pin(b.op), pin(b.src), pin(b.dst)) for b in timed]
    d_restore = [(dev(b.op), dev(b.src), dev(b.dst)) for b in restore]
    sizes = [len(b) for b in timed]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    cur = [0]  # position in the cycle of timed batches (0: the graph is G0)

    def restore_if_cycle_done():
        if cur[0] == len(timed):
            for op, s_, d_ in d_restore:  # untimed, no queries: stage and commit only
                ctx.apply_batch(op, s_, d_, [])
                ctx.commit()
            cur[0] = 0

    def step(bufs):
        restore_if_cycle_done()
        k = cur[0]
        op, s_, d_ = bufs[k]
        pos, neg = ctx.apply_batch(op, s_, d_, qids)
        st = ctx.stats()
        ctx.commit()
        cur[0] += 1
        return k, int(pos.sum()) + int(neg.sum()), st

    # instrumented launch (untimed) on the first batch from G0: algorithmic bytes
    ctx.set_options(flags=flags | G.GAMMA_F_COUNT_BYTES)
    pos, neg = ctx.apply_batch(*d_timed[0], qids)
    alg_bytes = ctx.stats()["alg_bytes"]
    ctx.commit()
    ctx.set_options(flags=flags)
    inv0 = timed[0].inverse()
    ctx.apply_batch(dev(inv0.op), dev(inv0.src), dev(inv0.dst), [])
    ctx.commit()

    for k in range(args.warmup):
        step(d_timed)
    while cur[0] % len(timed):  # start the timed steps at the first batch of a cycle (the roofline's launch)
        step(d_timed)

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches = 0
    matches, phases, which = [], [], []
    t0 = time.perf_counter()
    for k in range(args.steps):
        restore_if_cycle_done()
        l0 = ctx.stats()["kernel_launches"]
        with torch.cuda.stream(stream):
            flush.zero_()
            evs[k][0].record(stream)
        j, m, st = step(d_timed)
        with torch.cuda.stream(stream):
            evs[k][1].record(stream)
        launches += ctx.stats()["kernel_launches"] - l0
        matches.append(m)
        phases.append(st)
        which.append(j)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms = [a.elapsed_time(bb) for a, bb in evs]
    units = sum(sizes[j] for j in which)
    tot_s = max_over_ranks(sum(ms) / 1e3, dist, "cuda")
    if dist:
        dist.barrier()

    # end to end through the C-ABI with host (pinned) batch buffers, on the
    # same batches as the timed steps (untimed steps first bring the cycle
    # back to its first batch)
    while cur[0] % len(timed):
        step(d_timed)
    e2e_t, e2e_units = [], 0
    for k in range(min(args.steps, len(timed))):  # the first batches of a cycle, as timed above
        restore_if_cycle_done()
        torch.cuda.synchronize()
        t = time.perf_counter()
        j, _, _ = step(h_timed)
        e2e_t.append(time.perf_counter() - t)
        e2e_units += sizes[j]
    e2e_v = whole_job_rate(e2e_units, world, max_over_ranks(sum(e2e_t), dist, "cuda"))

    dfs0 = [p["ms_match"] for p, j in zip(phases, which) if j == 0]
    dfs_ms = statistics.mean(dfs0) if dfs0 else 0.0
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (dfs_ms / 1e3) / 1e9 if dfs_ms > 0 else 0.0
    l2_gbs = G.gamma_probe_bandwidth(local, 64 << 20, reps=16, trials=5)
    phase_ms = {k: round(statistics.mean(p[k] for p in phases), 4)
                for k in ("ms_stage", "ms_seed", "ms_match", "ms_finalize", "ms_commit")}
    per_batch = {}
    for m_, j, t_ in zip(matches, which, ms):
        per_batch.setdefault(j, {"matches": m_, "ms": []})["ms"].append(round(t_, 3))
    line = {
        "metric": METRIC, "value": whole_job_rate(units, world, tot_s), "unit": "updates/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": config_of(args.workload, sizes[0], queries, len(timed)),
        "matches_per_s": whole_job_rate(sum(matches), world, tot_s),
        "incremental_matches_per_step": sum(matches) / len(matches),
        "p50_ms": statistics.median(ms), "p99_ms": float(np.percentile(ms, 99)), "step_ms": [round(x, 3) for x in ms],
        "per_batch": {str(j): v for j, v in sorted(per_batch.items())},
        "phase_ms": phase_ms, "wall_s": wall,
        "e2e": {"value": e2e_v, "unit": "updates/s", "h2d_bytes_per_step": 9 * sizes[0],
                "d2h_bytes_per_step": 16 * len(queries) + 3 * STATUS_BYTES},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "k_dfs", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": dfs_traffic(args.workload), "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": dfs_ms,
                     "launch": "the DFS launch of the first batch of the cycle",
                     "l2_read_gbs": l2_gbs, "l2_frac": achieved / l2_gbs if l2_gbs > 0 else None},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, queries, timed[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
