#!/usr/bin/env python
"""Benchmark: exact co-mining of the mid workload's 12 motifs on one B300.

Workload (named in the JSON line's ``config``): a seeded synthetic temporal
graph of 1M nodes and 20M edges (Zipf(1.6) endpoints, bursty Poisson
timestamps over 30 days), 12 motifs of 3-4 edges sharing 2-edge prefixes,
delta = 3600 s, counted exactly for a seeded uniform sample of root edges
(every motif's matches whose first edge is a sampled root).  One step is one
tm_count call over the sample; the metric is query root-edges per second =
roots x motifs / step time.  Under torchrun every rank mines its own root
sample (weak scaling, no collective on the data path).

``--impl reference`` times the CPU oracle (the plain recursion of
Algorithm 1 per motif, all host cores) on the same roots and motifs at a
window it finishes (CPU_SAMPLE_DELTA); the CPU-baseline leg of the default
run times the same sample on one core and on all cores, and the GPU on it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (graph spec, motifs, delta, default root sample)
    "mid": ("MID", "CONFIG2_MOTIFS", 3600, 64),
    "tiny": ("TINY", "CONFIG1_MOTIFS", 10_000, 50_000),
    "batched": (None, None, None, 65536),
    "probe": (None, None, None, 4),
    "serving": (None, None, None, 64),
    "ablation": (None, None, None, 64),
    "enumerate": (None, None, None, 50_000),
}


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def load_workload(name, n_roots, rank):
    from paper_2507_14813_b300 import synth
    gname, mname, delta, default_r = WORKLOADS[name]
    spec = getattr(synth, gname)
    src, dst, t = synth.make_graph(spec)
    motifs = getattr(synth, mname)
    R = n_roots or default_r
    roots = synth.root_sample(100 + rank, len(src), R)
    return spec, src, dst, t, motifs, delta, roots


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5 and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# Per-launch figures of the timed mining launch of the default benchmark from
# one ncu capture of that launch (profiles/), keyed by a hash of the kernel
# source they were taken on and by the schedule of the timed step; any other
# source reports null.  dram_bytes = dram__bytes_read.sum +
# dram__bytes_write.sum; l2_pct / dram_pct = ncu's L2 and DRAM throughput
# (percent of peak sustained).
PROFILE = {"5fa00b13a830d2c6": {"learned": {"dram_bytes": 334.66e6, "l2_pct": 6.12, "dram_pct": 0.01}}}


def kernel_hash():
    """Hash of the mining kernel's sources (the kernel and the device types)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("tm_kernel.cuh", "tm_device.h"):
        h.update(open(os.path.join(ROOT, "paper_2507_14813_b300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6400.0, "fallback"


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


# The CPU oracle does not finish the mid workload's hub roots at delta = 3600 s
# (a 4-edge star on one hub root has ~10^14 matches), so the CPU baseline and
# the reference arm run the same 64 roots and 12 motifs at this window, which
# the oracle finishes for every root in ~10 s on one core; the GPU step is
# timed on the same sample beside it.
CPU_SAMPLE_DELTA = 15


def cpu_sample(src, dst, t, motifs, roots, threads=1):
    """Oracle (Algorithm 1 per motif) over every root of the sample at
    CPU_SAMPLE_DELTA: (counts per motif, roots finished, wall seconds)."""
    import oracle
    t0 = time.perf_counter()
    counts, done = [], len(roots)
    for m in motifs:
        if threads == 1:
            _, pr = oracle.count_motif(src, dst, t, m, CPU_SAMPLE_DELTA, roots=roots, per_root=True)
        else:
            pr, _ = oracle.count_motif_timed(src, dst, t, m, CPU_SAMPLE_DELTA, roots, threads=threads,
                                             time_limit=0)
        done = min(done, int((pr >= 0).sum()))
        counts.append(int(pr[pr >= 0].sum()))
    return counts, done, time.perf_counter() - t0


def cpu_sample_text(n_roots, n_motifs, done, workload_delta):
    return ("the %d roots of the benchmark sample x %d motifs at delta = %d s instead of %d s (the oracle does not "
            "finish hub roots at the full window); %d of %d roots finished" %
            (n_roots, n_motifs, CPU_SAMPLE_DELTA, workload_delta, done, n_roots))


def plan_launches(n_roots):
    """Kernels of one learned plan: k_features, then tm_plan's k_mlp_fwd,
    k_plan_keys, four radix passes (k_rs_hist, the histogram scan, k_rs_scatter)
    and k_plan_apply.  The histogram scan is one k_scan_tile while the 256
    buckets x tiles fit one scan tile, else two more launches per level."""
    tiles = max(1, -(-n_roots // 4096))
    scan = 1
    n = 256 * tiles
    while n > 1024:                     # k_scan_tile + recursive scan + k_scan_add
        scan += 2
        n = -(-n // 1024)
    return 1 + 2 + 4 * (2 + scan) + 1


def train_cost_model(args, tmotif, g, tr, src, rank, d_roots):
    """Train the cost model (a11) on measured per-root work of a separate root
    sample, then score its predictions on the benchmark's own roots against
    their measured work.  Runs before any timed region: the trained model is
    an input of the step, like the graph."""
    import torch
    from paper_2507_14813_b300 import synth
    n_train = args.train_roots
    t0 = time.perf_counter()
    train = torch.from_numpy(synth.root_sample(200 + rank, len(src), n_train)).cuda()
    work = torch.zeros((n_train, tmotif.TM_WORK_FIELDS), dtype=torch.int64, device="cuda")
    tmotif.tm_count(g.h, tr.h, roots=train, per_root_work=work, mode=tmotif.TM_SCHED_DYNAMIC, stats=True)
    w = work.cpu().numpy()
    y = torch.from_numpy(np.log1p(w[:, 0] + w[:, 2]).astype(np.float32)).cuda()
    X = torch.zeros((n_train, tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, train, X)
    model = tmotif.Model(seed=1)
    model.fit_norm(X)
    hist = model.train(X, y, epochs=120, batch=256, lr=3e-3)
    t_train = time.perf_counter() - t0
    R = len(d_roots)
    wr = torch.zeros((R, tmotif.TM_WORK_FIELDS), dtype=torch.int64, device="cuda")
    tmotif.tm_count(g.h, tr.h, roots=d_roots, per_root_work=wr, mode=tmotif.TM_SCHED_DYNAMIC, stats=True)
    wb = wr.cpu().numpy()
    yb = np.log1p(wb[:, 0] + wb[:, 2])
    Xb = torch.zeros((R, tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, d_roots, Xb)
    pb = torch.zeros(R, dtype=torch.float32, device="cuda")
    model.predict(Xb, pb)
    p = pb.cpu().numpy()
    rmse = float(np.sqrt(np.mean((p - yb) ** 2)))
    rank_corr = float(np.corrcoef(np.argsort(np.argsort(p)), np.argsort(np.argsort(yb)))[0, 1]) if R > 2 else None
    return model, {"train_roots": n_train, "train_seconds": t_train, "final_train_loss": float(hist[-1]),
                   "label": "log1p(candidates + probes) per root", "rmse_log_work_on_bench_roots": rmse,
                   "spearman_on_bench_roots": rank_corr, "label_std_on_bench_roots": float(np.std(yb)),
                   "max_split": args.max_split, "unit_work": args.unit_work}


def run_batched(args):
    """64 random motif sets merged into one tree (each motif with its set's
    window), one persistent launch replayed from a CUDA graph, launch shape
    and split thresholds from the autotuner."""
    import torch
    from paper_2507_14813_b300 import build, synth, tmotif
    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    build.build()
    spec = synth.BATCHED_MILD
    src, dst, t = synth.make_graph(spec)
    sets = synth.batched_sets()
    motifs, deltas = [], []
    for ms, d in sets:
        motifs += ms
        deltas += [d] * len(ms)
    g = tmotif.Graph(src, dst, t, spec.n_nodes, presorted=True)
    tr = tmotif.Tree(motifs, deltas)
    R = args.roots or 65536
    roots = torch.from_numpy(synth.root_sample(100 + rank, len(src), R)).cuda()
    D = tmotif.TM_SCHED_DYNAMIC
    tune = tmotif.tm_autotune(g.h, tr.h, mode=D, roots=roots[:min(R, 8192)])
    counts = torch.zeros(len(motifs), dtype=torch.int64, device="cuda")
    ex = tmotif.Exec(g.h, tr.h, counts, mode=D, roots=roots, tune=tune)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ex.launch(stream)
    ex.status(stream)
    ref = counts.clone()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            ex.launch(stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    ex.status(stream)
    if not torch.equal(counts, ref):
        raise SystemExit("batched counts changed between replays")
    ms = statistics.median([a.elapsed_time(b) for a, b in ev])
    # the same sets launched one after another, each with its own tree
    seq_ms = None
    if not args.no_permotif:
        trees = [tmotif.Tree(ms_, d) for ms_, d in sets]
        outs = [torch.zeros(len(ms_), dtype=torch.int64, device="cuda") for ms_, _ in sets]
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for trx, o in zip(trees, outs):
            tmotif.tm_count(g.h, trx.h, mode=D, roots=roots, counts=o, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        seq_ms = a.elapsed_time(b)
        if not torch.equal(torch.cat(outs), ref):
            raise SystemExit("per-set counts differ from the batched launch")
    # the paper's sibling splitting and multi-offload in place of halving slices
    sib_ms = None
    if not args.no_permotif:
        S = tmotif.TM_SCHED_SIBLINGS
        tmotif.tm_count(g.h, tr.h, mode=S, roots=roots, counts=counts, tune=tune)
        ts = []
        for i in range(3):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tmotif.tm_count(g.h, tr.h, mode=S, roots=roots, counts=counts, stream=stream, tune=tune)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        if not torch.equal(counts, ref):
            raise SystemExit("sibling-split counts differ from the batched launch")
        sib_ms = statistics.median(ts)
    _, st = tmotif.tm_count(g.h, tr.h, mode=D, roots=roots, stats=True, tune=tune)
    peak, peak_kind = measured_peaks()
    achieved = st["algo_bytes_lists"] / (ms / 1000.0) / 1e9
    line = {
        "metric": "query root-edges/sec (roots x motifs / s), 64 motif sets in one batched launch",
        "value": R * len(motifs) / (ms / 1000.0), "unit": "root-edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "%s: %d nodes, %d edges, Zipf(%.1f), bursty; 64 random prefix-sharing sets "
                               "(%d motifs of 2-6 edges, windows 600/3600/86400 s) merged into one tree; %d roots"
                               % (spec.name, spec.n_nodes, spec.n_edges, spec.zipf_s, len(motifs), R),
                   "l2": "flushed between steps (256 MiB write)", "launch": "CUDA graph replay of one persistent launch"},
        "tree": tr.info(), "autotune": tune, "sets_one_by_one_ms": seq_ms, "siblings_ms": sib_ms,
        "batched_speedup_vs_one_by_one": (seq_ms / ms) if seq_ms else None,
        "work": {k: st[k] for k in ("candidates", "probes", "leaf_evals", "tasks_split", "algo_bytes", "warp_imbalance")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None},
        "gpu_launches": 3 * args.steps, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_serving(args):
    """Poisson arrivals of motif queries against a resident graph; continuous
    batching by the library's server; latency percentiles and throughput."""
    import torch
    from paper_2507_14813_b300 import build, synth, tmotif
    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    build.build()
    spec = synth.SERVING_MILD if not args.serving_small else synth.BATCHED_MILD
    t0 = time.perf_counter()
    src, dst, t = synth.make_graph(spec)
    t_gen = time.perf_counter() - t0
    g = tmotif.Graph(src, dst, t, spec.n_nodes, presorted=True)
    print("graph generated in %.1f s" % t_gen, file=sys.stderr, flush=True)
    rate = args.rate
    n_req = int(rate * args.duration)
    rng = np.random.default_rng(7 + rank)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    qs = [synth.serving_query(50_000 + i, len(src), args.query_roots) for i in range(n_req)]
    # warm-up requests
    srv = tmotif.Server(g, streams=args.streams, max_batch=args.max_batch, mem_budget=args.mem_budget)
    for i in range(4):
        tk = srv.submit(*qs[i])
        srv.poll(tk, wait=True)

    def phase(arr, queries):
        tickets = []
        t_start = time.perf_counter()
        for i, q in enumerate(queries):
            now = time.perf_counter() - t_start
            if arr[i] > now:
                time.sleep(arr[i] - now)
            tickets.append(srv.submit(*q))
        print("submitted %d requests in %.1f s" % (len(tickets), time.perf_counter() - t_start), file=sys.stderr,
              flush=True)
        out = [srv.poll(tk, wait=True) for tk in tickets]
        return out, time.perf_counter() - t_start

    with ClockSampler(local_rank) as clk:
        res, wall = phase(arrivals, qs)
    stress = None
    if args.stress_rate > 0:
        n_s = int(args.stress_rate * args.stress_duration)
        arr_s = np.cumsum(rng.exponential(1.0 / args.stress_rate, n_s))
        qs_s = [synth.serving_query(90_000 + i, len(src), args.query_roots) for i in range(n_s)]
        res_s, wall_s = phase(arr_s, qs_s)
        lat_s = np.array([st["latency_ms"] for _, st in res_s])
        stress = {"rate": args.stress_rate, "requests": n_s, "qps": n_s / wall_s,
                  "p50_ms": float(np.percentile(lat_s, 50)), "p99_ms": float(np.percentile(lat_s, 99)),
                  "mean_batch": float(np.mean([st["batch_size"] for _, st in res_s])),
                  "root_edges_per_s": sum(len(q[0]) * len(q[2]) for q in qs_s) / wall_s}
    info = srv.info()
    srv.close()
    lat = np.array([st["latency_ms"] for _, st in res])
    sizes = np.array([st["batch_size"] for _, st in res])
    # spot check: a few requests against tm_count alone
    for i in range(0, n_req, max(1, n_req // 8)):
        ms_, d, r = qs[i]
        alone = tmotif.count(g, tmotif.Tree(ms_, d), roots=r, mode=tmotif.TM_SCHED_DYNAMIC)
        if res[i][0].tolist() != alone.tolist():
            raise SystemExit("served counts differ from the request counted alone")
    units = sum(len(q[0]) * len(q[2]) for q in qs)
    line = {
        "metric": "serving: p99 request latency (ms) under Poisson arrivals, continuous batching",
        "value": float(np.percentile(lat, 99)), "unit": "ms", "n_gpus": world, "steps": n_req, "warmup": 4,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "qps": n_req / wall, "root_edges_per_s": units / wall,
        "mean_batch": float(sizes.mean()), "max_batch_seen": int(sizes.max()), "server": info, "stress": stress,
        "config": {"workload": "%s: %d nodes, %d edges, Zipf(%.1f), bursty; %d requests at %.0f/s (Poisson); "
                               "each 1-16 motifs of 2-5 edges, window log-uniform in [60, 86400] s, %d sampled roots"
                               % (spec.name, spec.n_nodes, spec.n_edges, spec.zipf_s, n_req, rate, args.query_roots),
                   "streams": args.streams, "max_batch": args.max_batch, "mem_budget": args.mem_budget,
                   "graph_generation_s": t_gen},
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_probe(args):
    """One co-mining launch on the mid workload's first --roots sampled roots
    (default 4): the small case the kernel profiles are taken on.  With
    --probe-learned, the benchmark step's own launch: the cost model trained
    as in the benchmark (two stats launches of k_mine), then features, plan
    and the planned launch over the 64 benchmark roots."""
    import torch
    from paper_2507_14813_b300 import build, synth, tmotif
    build.build()
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    tr = tmotif.Tree(synth.CONFIG2_MOTIFS, synth.MID_DELTA)
    if not args.generic:
        tr.compile()
    n = 64 if args.probe_learned else (args.roots or 4)
    r = torch.from_numpy(synth.root_sample(100, len(src), 64)[:n]).cuda()
    out = torch.zeros(len(synth.CONFIG2_MOTIFS), dtype=torch.int64, device="cuda")
    tune = {"ctas_per_sm": 0, "donate_seq": 0, "donate_leaf": args.donate_leaf, "poll_every": args.poll_every}
    mode = tmotif.TM_SCHED_DYNAMIC
    if args.probe_learned:
        model, _ = train_cost_model(args, tmotif, g, tr, src, 0, r)
        feats = torch.zeros((n, tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
        ro, sp = torch.zeros_like(r), torch.zeros_like(r)
        tmotif.tm_features(g.h, tr.h, r, feats)
        model.plan(feats, r, ro, sp, unit_work=args.unit_work, max_split=args.max_split)
        r, mode = ro, mode | tmotif.TM_SCHED_PLANNED
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tmotif.tm_count(g.h, tr.h, roots=r, counts=out, mode=mode, tune=tune,
                    root_split=sp if args.probe_learned else None)
    torch.cuda.synchronize()
    print(json.dumps({"probe": "mid, %d roots%s" % (n, ", learned plan" if args.probe_learned else ""),
                      "counts": out.cpu().tolist(), "seconds": time.perf_counter() - t0}))
    return 0


def run_ablation(args):
    """Section 6's window ablation on the GPU: co-mined and per-motif step
    times of the mid workload (same graph, motifs and root sample) at delta/2,
    delta and 2*delta, with the tree's SM, the graph's bipartiteness and the
    co-mining decision (Section 6, heuristic for co-mining)."""
    import torch
    from paper_2507_14813_b300 import build, synth, tmotif
    build.build()
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    motifs = synth.CONFIG2_MOTIFS
    R = args.roots or 64
    roots = torch.from_numpy(synth.root_sample(100, len(src), R)).cuda()
    counts = torch.zeros(len(motifs), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    bip = g.bipartite()

    def timed(tr, mode):
        for _ in range(args.warmup):
            tmotif.tm_count(g.h, tr.h, mode=mode, roots=roots, counts=counts, stream=stream)
        torch.cuda.synchronize()
        ms = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tmotif.tm_count(g.h, tr.h, mode=mode, roots=roots, counts=counts, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms), counts.cpu().tolist()

    rows = []
    with ClockSampler(0) as clk:
        for d in (synth.MID_DELTA // 2, synth.MID_DELTA, 2 * synth.MID_DELTA):
            tr = tmotif.Tree(motifs, d)
            co_ms, co = timed(tr, tmotif.TM_COMINE | tmotif.TM_SCHED_DYNAMIC)
            pm_ms, pm = timed(tr, tmotif.TM_PERMOTIF | tmotif.TM_SCHED_DYNAMIC)
            if co != pm:
                raise SystemExit("per-motif counts differ from co-mined counts at delta=%d" % d)
            rows.append({"delta": d, "comine_ms": co_ms, "permotif_ms": pm_ms, "speedup": pm_ms / co_ms,
                         "sm": tr.info()["similarity"], "advice_comine": tmotif.tm_comine_advice(g.h, tr.h),
                         "root_edges_per_s": R * len(motifs) / (co_ms / 1000.0), "counts": co})
            tr.close()
    print(json.dumps({
        "metric": "co-mining speedup over per-motif mining by window (Section 6 ablation)",
        "value": rows[1]["speedup"], "unit": "x", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "int64", "data": "synthetic", "rows": rows, "bipartite": bip,
        "config": {"workload": "mid-1m-20m at delta/2, delta, 2*delta; 12 motifs; %d sampled roots" % R,
                   "l2": "flushed between steps (256 MiB write)", "schedule": "TM_SCHED_DYNAMIC"},
        "clocks": clk.summary()}))
    return 0


def run_enumerate(args):
    """Enumeration throughput: every match of the tiny workload (2k nodes,
    50k edges, 4 motifs, delta = 10^4) from all 50k roots, written to a
    device buffer sized to hold them all."""
    import torch
    from paper_2507_14813_b300 import build, synth, tmotif
    build.build()
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    _, total, counts = tmotif.tm_enumerate(g.h, tr.h, cap=0)
    want = tmotif.tm_count(g.h, tr.h)
    if counts.tolist() != want.tolist():
        raise SystemExit("enumerated counts differ from tm_count")
    buf = torch.empty((total, tmotif.MATCH_FIELDS), dtype=torch.int32, device="cuda")
    import ctypes
    a, keep = tmotif._count_args(tmotif.TM_COMINE)
    nf = ctypes.c_int64(0)
    stream = torch.cuda.current_stream()

    def once():
        tmotif._check(tmotif.lib().tm_enumerate(g.h, tr.h, ctypes.byref(a), ctypes.c_void_p(buf.data_ptr()),
                                                ctypes.c_int64(total), ctypes.byref(nf), None,
                                                tmotif._stream(stream)))

    for _ in range(args.warmup):
        once()
    ms = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            once()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
    if nf.value != total:
        raise SystemExit("match total changed between runs")
    med = statistics.median(ms)
    written = total * tmotif.MATCH_FIELDS * 4
    peak, peak_kind = measured_peaks()
    print(json.dumps({
        "metric": "enumerated matches/sec (every match written to device memory)", "value": total / (med / 1000.0),
        "unit": "matches/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": med,
        "higher_is_better": True, "dtype": "int32", "data": "synthetic", "matches": total,
        "counts": counts.tolist(), "record_bytes": tmotif.MATCH_FIELDS * 4,
        "write_gbs": written / (med / 1000.0) / 1e9, "write_frac_of_hbm": written / (med / 1000.0) / 1e9 / peak,
        "peak_kind": peak_kind,
        "config": {"workload": "tiny-2k-50k: 2000 nodes, 50000 edges, Zipf(1.8); 4 motifs, delta=10000; all 50000 roots",
                   "note": "the call allocates its counters and synchronises; the records stay on the device"},
        "clocks": clk.summary()}))
    return 0


def run_reference(args):
    """The oracle on the host cores, each step the CPU sample (the benchmark's
    roots and motifs at CPU_SAMPLE_DELTA), timed by the wall clock."""
    rank, local_rank, world = env_rank()
    if rank != 0:
        return 0
    spec, src, dst, t, motifs, delta, roots = load_workload(args.workload, args.roots, 0)
    threads = os.cpu_count() or 1
    secs, done, counts = [], len(roots), None
    for i in range(args.warmup + args.steps):
        c, d, el = cpu_sample(src, dst, t, motifs, roots, threads=threads)
        if counts is not None and c != counts:
            raise SystemExit("oracle counts changed between steps")
        counts, done = c, min(done, d)
        if i >= args.warmup:
            secs.append(el)
    step_s = statistics.median(secs)
    units = len(roots) * len(motifs)
    value = units / step_s
    cfg = config_of(args, spec, motifs, delta, roots)
    cfg["sample_delta"] = CPU_SAMPLE_DELTA
    line = {
        "impl": "reference", "metric": "query root-edges/sec (roots x motifs / s), exact co-mining",
        "value": value, "unit": "root-edges/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * step_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": "root-edges/s", "cores": threads, "kind": "oracle",
                         "cpu": cpu_model(), "sample": cpu_sample_text(len(roots), len(motifs), done, delta),
                         "seconds_per_step": step_s},
        "counts": counts,
        "e2e": {"value": value, "unit": "root-edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_of(args, spec, motifs, delta, roots):
    return {"workload": "%s: %d nodes, %d edges, Zipf(%.1f), %s timestamps; %d motifs, delta=%d; "
                        "seeded uniform sample of %d root edges per rank"
                        % (spec.name, spec.n_nodes, spec.n_edges, spec.zipf_s, spec.times, len(motifs), delta,
                           len(roots)),
            "n_edges": spec.n_edges, "n_nodes": spec.n_nodes, "n_motifs": len(motifs), "delta": delta,
            "roots_per_rank": len(roots), "l2": "flushed between steps (256 MiB write)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid", choices=sorted(WORKLOADS))
    ap.add_argument("--roots", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true", help="skip the all-core oracle context figure")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-permotif", action="store_true")
    ap.add_argument("--static", action="store_true", help="one warp per root, no subtree splitting")
    ap.add_argument("--generic", action="store_true", help="the table-driven kernel only (no code generation)")
    ap.add_argument("--with-static", action="store_true",
                    help="also time the step with static scheduling (one warp per root; slow on hub roots)")
    ap.add_argument("--thread-work", type=float, default=100.0,
                    help="thread tier: roots predicted below this work run one per lane (0: no tier)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--train-roots", type=int, default=512)
    ap.add_argument("--unit-work", type=float, default=1e6)
    ap.add_argument("--max-split", type=int, default=4096)
    ap.add_argument("--poll-every", type=int, default=16, help="reactive splitting: chunk loads between polls")
    ap.add_argument("--donate-leaf", type=int, default=4096,
                    help="reactive splitting: shortest counting-only slice handed over")
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--duration", type=float, default=20.0)
    ap.add_argument("--query-roots", type=int, default=64)
    ap.add_argument("--streams", type=int, default=2)
    ap.add_argument("--max-batch", type=int, default=32)
    ap.add_argument("--mem-budget", type=int, default=4 << 30)
    ap.add_argument("--serving-small", action="store_true")
    ap.add_argument("--stress-rate", type=float, default=2000.0)
    ap.add_argument("--stress-duration", type=float, default=5.0)
    ap.add_argument("--mode", type=int, default=0, help="extra tm_count mode bits")
    ap.add_argument("--probe-learned", action="store_true",
                    help="probe workload: the benchmark step's planned launch over its 64 roots")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "probe":
        return run_probe(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "ablation":
        return run_ablation(args)
    if args.workload == "enumerate":
        return run_enumerate(args)

    import torch
    import torch.distributed as dist
    from paper_2507_14813_b300 import build, tmotif

    rank, local_rank, world = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    build.build()
    spec, src, dst, t, motifs, delta, roots = load_workload(args.workload, args.roots, rank)
    n_m = len(motifs)
    g = tmotif.Graph(src, dst, t, spec.n_nodes, presorted=True)
    tr = tmotif.Tree(motifs, delta)
    # kernels specialised to the tree and to each motif's chain (runtime code
    # generation), compiled before any timed region like the tree itself
    codegen = None
    if not args.generic:
        t0 = time.perf_counter()
        codegen = tr.compile(0 if args.no_permotif else tmotif.TM_COMPILE_CHAINS)
        codegen["seconds"] = time.perf_counter() - t0
    d_roots = torch.from_numpy(roots).cuda()
    counts = torch.zeros(n_m, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    mode = tmotif.TM_COMINE | args.mode | (0 if args.static else tmotif.TM_SCHED_DYNAMIC) | \
        (tmotif.TM_GENERIC if args.generic else 0)
    # learned scheduling (a11, a12): the model is trained before the timed
    # region; every step computes features, predicts, plans and counts
    model, learned = None, None
    if not args.no_learned and not args.static:
        model, learned = train_cost_model(args, tmotif, g, tr, src, rank, d_roots)
    R = len(roots)
    feats = torch.zeros((R, tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
    ro = torch.zeros_like(d_roots)
    sp = torch.zeros_like(d_roots)

    def plan(gh, th, r_dev, f, r_out, s_out, thread_work=0.0):
        tmotif.tm_features(gh, th, r_dev, f, stream=stream)
        model.plan(f, r_dev, r_out, s_out, unit_work=args.unit_work, max_split=args.max_split, stream=stream,
                   thread_work=thread_work)

    # reactive-splitting tunables (chunk loads between looks for idle warps, the
    # shortest counting-only slice worth handing over), from a sweep on this workload
    tune = {"ctas_per_sm": 0, "donate_seq": 0, "donate_leaf": args.donate_leaf, "poll_every": args.poll_every}

    def step(m, use_model, thread_work=0.0):
        if use_model:
            plan(g.h, tr.h, d_roots, feats, ro, sp, thread_work)
            tiers = tmotif.TM_SCHED_TIERS if thread_work > 0 else 0
            tmotif.tm_count(g.h, tr.h, mode=m | tmotif.TM_SCHED_PLANNED | tiers, roots=ro, counts=counts,
                            root_split=sp, stream=stream, tune=tune)
        else:
            tmotif.tm_count(g.h, tr.h, mode=m, roots=d_roots, counts=counts, stream=stream, tune=tune)

    def timed(m, use_model, n, thread_work=0.0):
        ts = []
        for i in range(n):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(m, use_model, thread_work)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
            if not torch.equal(counts, ref_counts):
                raise SystemExit("counts differ between schedules or modes")
        return statistics.median(ts)

    use_model = model is not None
    for _ in range(args.warmup):
        step(mode, use_model)
    torch.cuda.synchronize()
    ref_counts = counts.clone()

    # stats of one untimed launch of the same schedule: algorithmic bytes and work counters
    if use_model:
        _, st = tmotif.tm_count(g.h, tr.h, mode=mode | tmotif.TM_SCHED_PLANNED, roots=ro, root_split=sp,
                                stats=True, stream=stream, tune=tune)
    else:
        _, st = tmotif.tm_count(g.h, tr.h, mode=mode, roots=roots, stats=True, stream=stream, tune=tune)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            step(mode, use_model)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    if not torch.equal(counts, ref_counts):
        raise SystemExit("counts changed between steps")
    total_ms = sum(ms)
    if world > 1:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_step = total_ms / args.steps
    units = len(roots) * n_m * world
    value = units / (ms_step / 1000.0)
    n_cmp = max(1, min(args.steps, 3))

    # the same step without the model: reactive splitting alone
    reactive = timed(mode, False, n_cmp) if use_model else None
    # the same step with the table-driven kernel in place of the tree's own
    generic = timed(mode | tmotif.TM_GENERIC, use_model, n_cmp) if codegen else None
    # the same step with the paper's sibling splitting and multi-offload in
    # place of halving slices for idle warps
    siblings = timed(mode | tmotif.TM_SCHED_SIBLINGS, use_model, n_cmp) if not args.static else None
    # the same step with a thread tier: roots predicted below --thread-work one per lane
    tiers = tier_hist = None
    if use_model and args.thread_work > 0:
        tiers = timed(mode, True, n_cmp, args.thread_work)
        plan(g.h, tr.h, d_roots, feats, ro, sp, args.thread_work)
        _, st_t = tmotif.tm_count(g.h, tr.h, mode=mode | tmotif.TM_SCHED_PLANNED | tmotif.TM_SCHED_TIERS, roots=ro,
                                  root_split=sp, stats=True, stream=stream, tune=tune)
        tier_hist = {"thread": st_t["roots_thread_tier"], "split": st_t["roots_split"],
                     "warp": st_t["n_roots"] - st_t["roots_thread_tier"] - st_t["roots_split"]}
    # the same step, static: one warp per root, no plan, no queue
    static = timed(mode & ~tmotif.TM_SCHED_DYNAMIC, False, n_cmp) if args.with_static and not args.static else None
    # the per-motif comparator with static scheduling too
    perm_static = (timed((mode & ~tmotif.TM_SCHED_DYNAMIC) | tmotif.TM_PERMOTIF, False, n_cmp)
                   if args.with_static and not args.static and not args.no_permotif else None)

    # per-motif comparator on the same roots (one chain tree per motif), same schedule
    perm = perm_reactive = None
    if not args.no_permotif:
        step(mode | tmotif.TM_PERMOTIF, use_model)
        torch.cuda.synchronize()
        if not torch.equal(counts, ref_counts):
            raise SystemExit("per-motif counts differ from co-mined counts")
        perm = timed(mode | tmotif.TM_PERMOTIF, use_model, n_cmp)
        if use_model:
            perm_reactive = timed(mode | tmotif.TM_PERMOTIF, False, n_cmp)

    # end to end through the C-ABI with host buffers: load, build, (plan,) count, read back
    e2e = None
    if not args.no_e2e:
        # the caller's inputs live in pinned host memory (page-locked once,
        # outside the timed region); each step copies them to the device
        pins = [torch.from_numpy(a).pin_memory() for a in (src, dst, t, roots)]
        h_src, h_dst, h_t, h_roots = (x.numpy() for x in pins)
        times = []
        for i in range(2):
            t0 = time.perf_counter()
            g2 = tmotif.Graph(h_src, h_dst, h_t, spec.n_nodes, presorted=True)
            tr2 = tmotif.Tree(motifs, delta)
            if codegen:
                tr2.compile()                   # the process cache holds this tree's program
            if use_model:
                r2 = torch.from_numpy(h_roots).cuda()
                f2 = torch.empty((R, tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
                ro2, sp2 = torch.empty_like(r2), torch.empty_like(r2)
                plan(g2.h, tr2.h, r2, f2, ro2, sp2)
                c2 = tmotif.tm_count(g2.h, tr2.h, mode=mode | tmotif.TM_SCHED_PLANNED, roots=ro2, root_split=sp2,
                                     tune=tune)
            else:
                c2 = tmotif.tm_count(g2.h, tr2.h, mode=mode, roots=h_roots, tune=tune)
            g2.close()
            tr2.close()
            times.append(time.perf_counter() - t0)
            if not np.array_equal(c2, ref_counts.cpu().numpy()):
                raise SystemExit("end-to-end counts differ")
        e2e_s = min(times)
        e2e = {"value": len(roots) * n_m * world / e2e_s, "unit": "root-edges/s",
               "h2d_bytes_per_step": int(src.nbytes + dst.nbytes + t.nbytes + h_roots.nbytes),
               "d2h_bytes_per_step": 8 * n_m, "seconds_per_step": e2e_s, "host_memory": "pinned"}

    peak, peak_kind = measured_peaks()
    # algorithmic bytes per launch by list accounting: 16 per root, 8 per
    # candidate scanned, 12 per binary-search step of each list opened
    achieved = st["algo_bytes_lists"] / (ms_step / 1000.0) / 1e9
    achieved_probes = st["algo_bytes"] / (ms_step / 1000.0) / 1e9
    prof = PROFILE.get(kernel_hash(), {}).get("learned" if use_model else "reactive", {}) \
        if args.workload == "mid" and len(roots) == 64 and not args.static else {}
    line = {
        "metric": "query root-edges/sec (roots x motifs / s), exact co-mining",
        "value": value, "unit": "root-edges/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": config_of(args, spec, motifs, delta, roots),
        "roots_per_s": len(roots) * world / (ms_step / 1000.0),
        "counts_per_s": float(ref_counts.sum().item()) * world / (ms_step / 1000.0),
        "counts": ref_counts.cpu().tolist(),
        "schedule": ("learned plan (features, MLP, sorted slices) + reactive splitting" if use_model
                     else ("static, one warp per root" if args.static else "reactive splitting")),
        "tunables": {"unit_work": args.unit_work, "max_split": args.max_split, "poll_every": args.poll_every,
                     "donate_leaf": args.donate_leaf},
        "reactive_ms_per_step": reactive,
        "learned_speedup_vs_reactive": (reactive / ms_step) if reactive else None,
        "kernel": ("specialised to the tree (runtime code generation)" if codegen else "table-driven"),
        "codegen": codegen,
        "generic_ms_per_step": generic,
        "specialised_speedup_vs_generic": (generic / ms_step) if generic else None,
        "siblings_ms_per_step": siblings,
        "tiers_ms_per_step": tiers, "thread_work": args.thread_work, "tier_histogram": tier_hist,
        "static_ms_per_step": static, "permotif_static_ms_per_step": perm_static,
        "schedule_siblings": "the same step with sibling splitting and multi-offload (TM_SCHED_SIBLINGS)",
        "permotif_ms_per_step": perm,
        "comine_speedup_vs_permotif": (perm / ms_step) if perm else None,
        "permotif_reactive_ms_per_step": perm_reactive,
        "work": {k: st[k] for k in ("candidates", "expansions", "probes", "leaf_evals", "algo_bytes",
                                     "algo_bytes_lists", "warp_imbalance", "idle_expired", "tasks_split")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": prof.get("dram_bytes"),
                     "bytes_per_launch": st["algo_bytes_lists"],
                     "accounting": "16 B per root + 8 B per candidate scanned + 12 B per binary-search step "
                                   "(ceil(log2(len + 1))) of each candidate list opened",
                     "achieved_probe_accounting": achieved_probes,
                     "frac_probe_accounting": achieved_probes / peak,
                     "probe_accounting": "16 B per root + 8 B per candidate + 8 B per list probe + 16 B per hash "
                                         "probe + 4 B per pair-run probe",
                     "l2_throughput_pct_ncu": prof.get("l2_pct"), "dram_throughput_pct_ncu": prof.get("dram_pct"),
                     "kernel": "k_mine", "kernel_source": kernel_hash(),
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind},
        "gpu_launches": (plan_launches(len(roots)) + 2 if use_model else 2) * args.steps,
        "clocks": clk.summary(),
    }
    if learned:
        line["cost_model"] = learned
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        units = len(roots) * n_m
        c1, done, el = cpu_sample(src, dst, t, motifs, roots, threads=1)
        # the GPU on the same sample: same roots and motifs, same window
        tr_s = tmotif.Tree(motifs, CPU_SAMPLE_DELTA)
        gs = tmotif.count(g, tr_s, roots=d_roots, mode=mode)
        if gs.tolist() != c1:
            raise SystemExit("GPU counts differ from the oracle's on the CPU sample")
        ts = []
        for i in range(max(args.steps, 3)):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tmotif.tm_count(g.h, tr_s.h, mode=mode, roots=d_roots, counts=counts, stream=stream, tune=tune)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        gms = statistics.median(ts)
        sample = cpu_sample_text(len(roots), n_m, done, delta)
        line["cpu_baseline"] = {"value": units / el, "unit": "root-edges/s", "cores": 1, "kind": "oracle",
                                "cpu": cpu_model(), "sample": sample, "seconds": el,
                                "counts_equal_gpu": True}
        line["gpu_on_cpu_sample"] = {"value": units / (gms / 1000.0), "unit": "root-edges/s", "ms_per_step": gms,
                                     "delta": CPU_SAMPLE_DELTA, "schedule": "reactive splitting",
                                     "speedup_vs_cpu_one_core": el / (gms / 1000.0)}
        if not args.no_cpu_all_cores:
            n = os.cpu_count() or 1
            cn, done_n, el_n = cpu_sample(src, dst, t, motifs, roots, threads=n)
            if cn != c1:
                raise SystemExit("multithreaded oracle counts differ")
            line["cpu_baseline_all_cores"] = {
                "value": units / el_n, "unit": "root-edges/s", "cores": n, "kind": "oracle", "cpu": cpu_model(),
                "context": "the same oracle with a dynamic OpenMP loop over roots on every host core",
                "sample": cpu_sample_text(len(roots), n_m, done_n, delta), "seconds": el_n}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
