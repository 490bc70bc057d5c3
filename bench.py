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
Algorithm 1 per motif, all host cores) on a bounded part of the same sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (graph spec, motifs, delta, default root sample)
    "mid": ("MID", "CONFIG2_MOTIFS", 3600, 64),
    "tiny": ("TINY", "CONFIG1_MOTIFS", 10_000, 50_000),
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
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6400.0, "fallback"


def cpu_baseline(src, dst, t, motifs, delta, roots, seconds=20.0, threads=1):
    """Oracle (Algorithm 1 per motif) on a bounded part of the root sample."""
    import oracle
    per_motif = seconds / len(motifs)
    t_root = 0.0
    done_min = len(roots)
    for m in motifs:
        t0 = time.perf_counter()
        _, done = oracle.count_motif_timed(src, dst, t, m, delta, roots, threads=threads, time_limit=per_motif)
        el = time.perf_counter() - t0
        done_min = min(done_min, done)
        t_root += el / max(done, 1)            # seconds per root for this motif
    value = len(motifs) / t_root               # query root-edges per second
    return value, done_min


def run_reference(args):
    rank, local_rank, world = env_rank()
    if rank != 0:
        return 0
    spec, src, dst, t, motifs, delta, roots = load_workload(args.workload, args.roots, 0)
    threads = os.cpu_count() or 1
    steps = []
    for i in range(args.warmup + args.steps):
        v, done = cpu_baseline(src, dst, t, motifs, delta, roots, seconds=args.ref_seconds, threads=threads)
        if i >= args.warmup:
            steps.append(v)
    value = statistics.median(steps)
    sample = ("first roots of the %d-root sample reached within %.0f s per step (%d of %d for the slowest motif)"
              % (len(roots), args.ref_seconds, done, len(roots)))
    line = {
        "impl": "reference", "metric": "query root-edges/sec (roots x motifs / s), exact co-mining",
        "value": value, "unit": "root-edges/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * len(roots) * len(motifs) / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": config_of(args, spec, motifs, delta, roots),
        "cpu_baseline": {"value": value, "unit": "root-edges/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
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
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-permotif", action="store_true")
    ap.add_argument("--static", action="store_true", help="one warp per root, no subtree splitting")
    ap.add_argument("--mode", type=int, default=0, help="extra tm_count mode bits")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

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
    d_roots = torch.from_numpy(roots).cuda()
    counts = torch.zeros(n_m, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    mode = tmotif.TM_COMINE | args.mode | (0 if args.static else tmotif.TM_SCHED_DYNAMIC)

    def step(m):
        tmotif.tm_count(g.h, tr.h, mode=m, roots=d_roots, counts=counts, stream=stream)

    for _ in range(args.warmup):
        step(mode)
    torch.cuda.synchronize()
    ref_counts = counts.clone()

    # stats of one untimed launch: algorithmic bytes and work counters
    _, st = tmotif.tm_count(g.h, tr.h, mode=mode, roots=roots, stats=True, stream=stream)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            step(mode)
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

    # per-motif comparator on the same roots (one chain tree per motif)
    perm = None
    if not args.no_permotif:
        step(mode | tmotif.TM_PERMOTIF)
        torch.cuda.synchronize()
        if not torch.equal(counts, ref_counts):
            raise SystemExit("per-motif counts differ from co-mined counts")
        pm = []
        for i in range(max(1, min(args.steps, 3))):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(mode | tmotif.TM_PERMOTIF)
            b.record(stream)
            torch.cuda.synchronize()
            pm.append(a.elapsed_time(b))
        perm = statistics.median(pm)

    # end to end through the C-ABI with host buffers: load, build, count, read back
    e2e = None
    if not args.no_e2e:
        h_roots = roots.copy()
        times = []
        for i in range(2):
            t0 = time.perf_counter()
            g2 = tmotif.Graph(src, dst, t, spec.n_nodes, presorted=True)
            tr2 = tmotif.Tree(motifs, delta)
            c2 = tmotif.tm_count(g2.h, tr2.h, mode=mode, roots=h_roots)
            g2.close()
            tr2.close()
            times.append(time.perf_counter() - t0)
            if not np.array_equal(c2, ref_counts.cpu().numpy()):
                raise SystemExit("end-to-end counts differ")
        e2e_s = min(times)
        e2e = {"value": len(roots) * n_m * world / e2e_s, "unit": "root-edges/s",
               "h2d_bytes_per_step": int(src.nbytes + dst.nbytes + t.nbytes + h_roots.nbytes),
               "d2h_bytes_per_step": 8 * n_m, "seconds_per_step": e2e_s}

    peak, peak_kind = measured_peaks()
    achieved = st["algo_bytes"] / (ms_step / 1000.0) / 1e9
    line = {
        "metric": "query root-edges/sec (roots x motifs / s), exact co-mining",
        "value": value, "unit": "root-edges/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": config_of(args, spec, motifs, delta, roots),
        "roots_per_s": len(roots) * world / (ms_step / 1000.0),
        "counts_per_s": float(ref_counts.sum().item()) * world / (ms_step / 1000.0),
        "counts": ref_counts.cpu().tolist(),
        "permotif_ms_per_step": perm,
        "comine_speedup_vs_permotif": (perm / ms_step) if perm else None,
        "work": {k: st[k] for k in ("candidates", "expansions", "probes", "leaf_evals", "algo_bytes")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind},
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        v, done = cpu_baseline(src, dst, t, motifs, delta, roots, seconds=args.cpu_seconds, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "root-edges/s", "cores": 1, "kind": "oracle",
                                "sample": "first roots of the same sample reached in %.0f s (%d of %d for the "
                                          "slowest motif), Algorithm 1 per motif" % (args.cpu_seconds, done, len(roots))}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
