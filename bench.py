#!/usr/bin/env python3
"""Benchmark of batch-dynamic subgraph matching (BDSM) on GB300.

One step = one pass of the whole hot path over one update batch: stage the
batch into the device-resident dynamic CSR, seed, DFS extension with match
counting, counts back to the host, commit.
Steps alternate the batch and its inverse, so the graph cycles between G0
and G0 + batch and every step does the same amount of work.

Default workload ("mid"): R-MAT scale 20 (a, b, c = .57, .19, .19),
8,388,608 unique edges of which 90% form G0, 8 vertex labels Zipf(1.2),
20 six-vertex queries (10 sparse, 10 dense) from tests/golden/queries_mid.json,
one batch of 90,000 insertions from the held-out pool + 10,000 uniform
deletions, interleaved. Inputs are synthetic (the paper's datasets are not
available). The graph (about 60 MB of adjacency) fits in L2, so L2 is flushed
(a 256 MiB write) before every timed step, outside the timed events.

value   = updates/s with the batch already in HBM (device events per step)
e2e     = the same metric through the C-ABI with host (pinned) batch buffers
roofline: the DFS kernel's algorithmic bytes (per candidate slot, search
          step, probe and prepared entry; counted by an untimed launch of the
          instrumented build) / the timed launch's duration, against the
          measured HBM copy bandwidth
cpu_baseline: the CPU oracle on a bounded sample of the same batch.
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
    "mid": {"workload": "mid", "queries": "tests/golden/queries_mid.json", "n_ins": 90_000, "n_del": 10_000},
    # the same graph, queries and batch cut to its first 3,000 updates: a case
    # small enough for multi-pass profiler captures
    "mid_3k": {"workload": "mid", "queries": "tests/golden/queries_mid.json", "n_ins": 90_000, "n_del": 10_000,
               "first": 3000},
    # the first 20,000 updates: every warp stays busy for about a second, so a
    # profiler capture sees the steady state of the full batch
    "mid_20k": {"workload": "mid", "queries": "tests/golden/queries_mid.json", "n_ins": 90_000, "n_del": 10_000,
                "first": 20000},
    "tiny": {"workload": "tiny", "queries": None, "n_ins": 256, "n_del": 0},
}
METRIC = "updates/s & incremental matches/s per batch (1 GB300); p50/p99 batch latency"
STATUS_BYTES = 112  # the library's status block, read back after staging, matching and commit
# batched / served modes: a bound on one apply's DFS work (32-wide expansion
# steps, about a minute of GPU time), so a workload heavier than intended
# fails with GAMMA_ETIMEOUT instead of running on
WORK_BUDGET = 100_000_000_000


def load_workload(name):
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
    batch = I.workload_batch(w, spec["n_ins"], spec["n_del"])
    if "first" in spec:
        k = spec["first"]
        batch = I.Batch(batch.op[:k].copy(), batch.src[:k].copy(), batch.dst[:k].copy())
    return w, queries, batch


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


def dfs_traffic(kernel_file="paper_2401_17018_gb300/csrc/gm_match.cu"):
    """DRAM bytes per DFS launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "dfs_mid_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256(open(os.path.join(ROOT, kernel_file), "rb").read()).hexdigest()[:16]
    if d.get("source_sha") != h:
        return None
    return d.get("dram_bytes_per_launch")


def cpu_baseline(w, queries, batch, budget_s=15.0):
    """The oracle, single-threaded, on a sample of the batch's updates (all
    queries): calls of k uniformly drawn updates each, k doubling while a
    call's search is short next to its graph build, until about budget_s
    seconds of search (the sample wraps around the batch when the batch is
    cheap).  The graph build of a call is measured with empty calls and
    subtracted."""
    from oracle import oracle as O
    g = w.graph
    setup = float("inf")
    for _ in range(2):
        t = time.perf_counter()
        O.bdsm_multi(g.n, g.labels, g.src, g.dst, queries, batch, eval_idx=[])
        setup = min(setup, time.perf_counter() - t)
    order = np.argsort(I_rand(len(batch)))
    b = len(batch)
    total_upd, total_s, i, k, calls = 0, 0.0, 0, 2, 0
    while total_s < budget_s and calls < 5000 and (total_s < 1.0 or total_upd < b):
        ev = np.sort(order[np.arange(i, i + min(k, b)) % b])
        i += ev.size
        t = time.perf_counter()
        O.bdsm_multi(g.n, g.labels, g.src, g.dst, queries, batch, eval_idx=ev)
        dt = time.perf_counter() - t - setup
        total_s += max(dt, 0.0)
        total_upd += ev.size
        calls += 1
        if dt < 4 * setup:
            k *= 2
    return {"value": total_upd / max(total_s, 1e-6), "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": "%d updates of the batch drawn uniformly (seeded, wrapping around), all %d queries, single "
                      "thread, %.2f s of search; graph build (%.3f s per call) excluded" % (
                          total_upd, len(queries), total_s, setup)}


def I_rand(n):
    from paper_2401_17018_gb300 import inputs as I
    return I.rand_u64(7, 99, np.arange(n, dtype=np.uint64))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    w, queries, batch = load_workload(args.workload)
    g = w.graph
    order = np.argsort(I_rand(len(batch)))
    times, nupd = [], []
    for step in range(args.warmup + args.steps):
        ev = np.sort(order[2 * step:2 * step + 2])
        t = time.perf_counter()
        O.bdsm_multi(g.n, g.labels, g.src, g.dst, queries, batch, eval_idx=ev)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
            nupd.append(ev.size)
    v = sum(nupd) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": config_of(args.workload, len(batch), len(queries)),
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "sample": "per step 2 updates of the batch drawn uniformly (seeded), all %d "
                                       "queries, graph build included" % len(queries)},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(workload, b, nq):
    spec = WORKLOADS[workload]
    return {"workload": "%s: R-MAT %s, %d queries, batch %d (%d ins + %d del)" % (
        workload, {"mid": "scale 20, 7.55M edges, 8 labels Zipf(1.2)",
                   "mid_3k": "scale 20, 7.55M edges, 8 labels Zipf(1.2), first 3,000 updates of the mid batch",
                   "mid_20k": "scale 20, 7.55M edges, 8 labels Zipf(1.2), first 20,000 updates of the mid batch",
                   "tiny": "scale 11, 9k edges, 4 labels"}[workload], nq, b, spec["n_ins"], spec["n_del"]),
        "batch_updates": b, "queries": nq, "l2": "flushed before every timed step (256 MiB write)",
        "step": "apply batch (stage+seed+DFS+counts to host) + commit; batch and inverse alternate"}


def run_batched(args):
    """Batched form: the same batch and the 64 stored batched queries,
    (1) plain: one seed + DFS launch sequence per query, (2) batched: one
    launch over all queries' seeds, autotuned and replayed as a CUDA graph.
    Both must give identical counts."""
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
    if not args.full_grid:
        grid = [(wpb, t, gr) for wpb in (4, 8, 16) for t in (64, 128) for gr in (4, 16)]
    out = {}
    counts = {}
    for form, flags in (("plain", G.GAMMA_F_PER_QUERY), ("batched", G.GAMMA_F_GRAPH)):
        stream = torch.cuda.Stream()
        ctx = G.Context(stream=stream, flags=flags, work_budget=WORK_BUDGET)
        ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
        qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
        tuned = None
        if form == "batched":
            ctx.apply_batch(*d_b, qids)
            tuned, sweep = G.gamma_autotune(ctx.h, grid, repeats=1)
            ctx.commit()
            ctx.apply_batch(*d_i, qids)
            ctx.commit()
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
        if tuned:
            out[form]["tuned"] = tuned
            out[form]["sweep"] = sweep
        counts[form] = res[0] if res else None
        ctx.close()
    same = counts["plain"] == counts["batched"]
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
            "plain": out["plain"], "batched": out["batched"],
            "speedup": out["batched"]["updates_per_s"] / out["plain"]["updates_per_s"]}
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
    ctx = G.Context(stream=torch.cuda.Stream(), work_budget=WORK_BUDGET)

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
            "config": {"workload": "served: R-MAT scale 22, 8 uniform labels, %d dense queries of %d..%d "
                                   "vertices, %d batches of floor(10^U(%g,%g)) updates (ins:del 1:1), Poisson "
                                   "arrivals" % (len(queries), min(q.labels.size for q in queries),
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
    ap.add_argument("--workload", default="mid", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-query", action="store_true", help="plain form: one launch sequence per query")
    ap.add_argument("--mode", default="plain", choices=["plain", "batched", "served"],
                    help="plain: the metric's workload; batched / served: the batched and served forms")
    ap.add_argument("--full-grid", action="store_true", help="batched mode: sweep the whole autotuner grid")
    ap.add_argument("--first", type=int, default=0,
                    help="batched mode: keep only the first N updates of the batch (0 = all)")
    ap.add_argument("--batches", type=int, default=12, help="served mode: batches in the stream")
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

    w, queries, batch = load_workload(args.workload)
    inv = batch.inverse()
    g = w.graph
    stream = torch.cuda.Stream()
    flags = G.GAMMA_F_PER_QUERY if args.per_query else 0
    ctx = G.Context(device=local, stream=stream, flags=flags)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx.load_graph(g.n, dev(g.labels), dev(g.src), dev(g.dst))
    qids = [ctx.register_query(q.labels, q.src, q.dst) for q in queries]
    b = len(batch)
    d_b = (dev(batch.op), dev(batch.src), dev(batch.dst))
    d_i = (dev(inv.op), dev(batch.src), dev(batch.dst))
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_b = (pin(batch.op), pin(batch.src), pin(batch.dst))
    h_i = (pin(inv.op), pin(batch.src), pin(batch.dst))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    applied = [0]  # batches applied so far: even -> the graph is G0, odd -> G0 + batch

    def step(k, bufs_b, bufs_i):
        op, s, d = bufs_b if applied[0] % 2 == 0 else bufs_i
        pos, neg = ctx.apply_batch(op, s, d, qids)
        st = ctx.stats()
        ctx.commit()
        applied[0] += 1
        return int(pos.sum()) + int(neg.sum()), st

    for k in range(args.warmup):
        step(k, d_b, d_i)
    # instrumented step (untimed): algorithmic bytes of the DFS launch on the batch
    if applied[0] % 2:
        step(0, d_b, d_i)
    ctx.set_options(flags=flags | G.GAMMA_F_COUNT_BYTES)
    _, st_bytes = step(0, d_b, d_i)
    step(0, d_b, d_i)
    ctx.set_options(flags=flags)
    alg_bytes = st_bytes["alg_bytes"]

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ctx.stats()["kernel_launches"]
    matches, phases = [], []
    t0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            evs[k][0].record(stream)
        m, st = step(k, d_b, d_i)
        with torch.cuda.stream(stream):
            evs[k][1].record(stream)
        matches.append(m)
        phases.append(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = ctx.stats()["kernel_launches"] - launches0
    clk = clocks.stop()
    ms = [a.elapsed_time(bb) for a, bb in evs]
    tot_s = max_over_ranks(sum(ms) / 1e3, dist, "cuda")
    if dist:
        dist.barrier()

    # end to end through the C-ABI with host (pinned) batch buffers
    e2e_t = []
    for k in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        step(k, h_b, h_i)
        e2e_t.append(time.perf_counter() - t)
    e2e_v = whole_job_rate(b * args.steps, world, max_over_ranks(sum(e2e_t), dist, "cuda"))

    dfs_ms = statistics.mean(p["ms_match"] for p in phases)
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (dfs_ms / 1e3) / 1e9 if dfs_ms > 0 else 0.0
    phase_ms = {k: round(statistics.mean(p[k] for p in phases), 4)
                for k in ("ms_stage", "ms_seed", "ms_match", "ms_finalize", "ms_commit")}
    line = {
        "metric": METRIC, "value": whole_job_rate(b * args.steps, world, tot_s), "unit": "updates/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": config_of(args.workload, b, len(queries)),
        "matches_per_s": whole_job_rate(sum(matches), world, tot_s),
        "incremental_matches_per_step": matches[0],
        "p50_ms": statistics.median(ms), "p99_ms": float(np.percentile(ms, 99)), "step_ms": [round(x, 3) for x in ms],
        "phase_ms": phase_ms, "wall_s": wall,
        "e2e": {"value": e2e_v, "unit": "updates/s", "h2d_bytes_per_step": 9 * b,
                "d2h_bytes_per_step": 16 * len(queries) + 3 * STATUS_BYTES},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "k_dfs", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": dfs_traffic() if args.workload == "mid" else None,  # recorded on mid only
                     "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": dfs_ms},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, queries, batch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
