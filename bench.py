#!/usr/bin/env python3
"""Harmonic-mean GTEPS of the compressed + sieved BFS on one GB300 (and N replicas).

One step = one breadth-first search from each of the workload's roots (64 by
default) on the resident graph, with the L2 flushed (a 256 MiB write) before
every search.  TEPS_r = m_r / t_r, where m_r is the number of input tuples in
the component reached from root r (self-loops and duplicates counted, Sec.
VII-A) and t_r the CUDA-event time of search r; the reported value is the
harmonic mean N_roots / sum_r (1 / TEPS_r).  The same graph is then searched
with the raw-bitmap exchange (BIT, Alg. 1) for the comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload s22|s26|s26er|s20|s12]
  python bench.py --impl reference      # the CPU oracle on the host cores

Under torchrun (N > 1) every rank searches its own replica of the graph from
its own seeded roots (weak scaling, no data-path collective); rank 0 prints the
JSON line with the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (scale, edgefactor, grid p, kind, roots, description)
    "s12": (12, 16, 2, 0, 16, "kronecker-s12-ef16-grid2x2"),
    "s20": (20, 16, 8, 0, 64, "kronecker-s20-ef16-grid8x8"),
    "s22": (22, 16, 8, 0, 64, "kronecker-s22-ef16-grid8x8"),
    "s24": (24, 16, 16, 0, 64, "kronecker-s24-ef16-grid16x16"),
    "s26": (26, 16, 16, 0, 64, "kronecker-s26-ef16-grid16x16"),
    "s26er": (26, 16, 16, 1, 64, "erdos-renyi-s26-ef16-grid16x16"),
}
METRIC = "harmonic-mean GTEPS on 1 GB300 (compressed+sieved vs plain GPU BFS) at bit-exact levels"
MODE_NAMES = {0: "plain", 1: "compress", 2: "compress_sieve"}
DIRECTIONS = {"top_down": 0, "hybrid": 1, "bottom_up": 2}
KERNEL_SOURCES = ["paper_1208_5542_gb300/csrc/bfs_level.cu", "paper_1208_5542_gb300/csrc/wah.cuh",
                  "paper_1208_5542_gb300/csrc/common.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="s26", choices=sorted(WORKLOADS) + ["msbfs20", "serve"],
                    help="s12..s26er: single searches; msbfs20: one 64-root batch on scale 20; "
                         "serve: Poisson query stream over 8 resident graphs")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="length of the serving stream")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="mean arrivals per second of the serving stream")
    ap.add_argument("--mode", type=int, default=2, help="0 plain, 1 compress, 2 compress+sieve")
    ap.add_argument("--wah-bits", type=int, default=32)
    ap.add_argument("--direction", default="top_down", choices=sorted(DIRECTIONS),
                    help="top_down: the paper's algorithms; hybrid: top-down / bottom-up levels chosen per level")
    ap.add_argument("--alpha", type=int, default=4, help="hybrid: bottom-up once m_f > m_u / alpha")
    ap.add_argument("--beta", type=int, default=24, help="hybrid: top-down again once the frontier < n / beta")
    ap.add_argument("--row-exchange", default="on", choices=["on", "off"],
                    help="compress_sieve: the fold of each block-row as a compressed exchange of row buffers")
    ap.add_argument("--roots", type=int, default=0, help="override the number of roots")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--profile-run", action="store_true",
                    help="build the graph and run one search per mode, untimed (for ncu)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers --
def kernel_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(workload, mode_name, algorithmic_bytes):
    """Per-launch DRAM bytes of the expansion kernel: the DRAM / algorithmic byte
    ratio of the committed ncu summary times this launch's algorithmic bytes, or
    None if none was taken for this workload or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
    except OSError:
        return None
    ent = data.get(f"{workload}:{mode_name}")
    if not ent or ent.get("kernel_hash") != kernel_hash():
        return None
    return round(ent["dram_over_algorithmic"] * algorithmic_bytes)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        # the raw samples (summarised in the JSON line) go to BFS_BENCH_LOG_DIR, else the temp dir
        log_dir = os.environ.get("BFS_BENCH_LOG_DIR") or tempfile.gettempdir()
        os.makedirs(log_dir, exist_ok=True)
        self.path = os.path.join(log_dir, f"clocks_{os.getpid()}.csv")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_value(inv, ms_step, n_roots, dist=None, device=None):
    """Whole-job harmonic-mean GTEPS over replicas: the roots searched by all
    ranks divided by the slowest rank's sum of t_r / m_r (every rank searches
    n_roots roots of its own replica; no data-path collective, only this
    timing reduction).  Returns (GTEPS, the slowest rank's ms per step)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        x = torch.tensor([inv, ms_step], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        inv, ms_step = float(x[0]), float(x[1])
    return ((n_roots * world / inv) / 1e9 if inv > 0 else 0.0), ms_step


def compression_factor(exch, mode):
    """C (Alg. 2) or C' (Alg. 3) of Sec. VI-A: the mean over the levels of the
    compressed-to-raw size of the exchange, 1 / C_i at level i.  None for
    PLAIN (nothing is compressed) or when no level was recorded."""
    r = [e["wah_over_raw"] for e in exch if e.get("wah_over_raw") is not None]
    if mode == 0 or not r:
        return None
    return {"symbol": "C'" if mode == 2 else "C", "value": round(sum(r) / len(r), 6), "levels": len(r)}


def hm_gteps(m, t):
    """Harmonic mean of m_r / t_r in GTEPS (t in seconds)."""
    s = sum(tr / mr for mr, tr in zip(m, t) if mr > 0)
    n = sum(1 for mr in m if mr > 0)
    return (n / s) / 1e9 if s > 0 else 0.0


# ---------------------------------------------------------- reference arm --
def workload_config(args, n, tuples, nroots):
    """The workload keys both arms report (so that their lines pair up)."""
    scale, ef, p, _, _, desc = WORKLOADS[args.workload]
    return {"workload": desc + f"-{MODE_NAMES[args.mode]}-{nroots}roots" +
            ("" if args.direction == "top_down" else f"-{args.direction}"), "scale": scale,
            "edgefactor": ef, "vertices": n, "tuples": int(tuples), "grid": f"{p}x{p}",
            "mode": MODE_NAMES[args.mode], "wah_word_bits": args.wah_bits, "roots": nroots,
            "direction": args.direction if args.direction != "hybrid"
            else f"hybrid (alpha {args.alpha}, beta {args.beta})"}


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores (one core)."""
    import numpy as np  # noqa: F401

    import graphgen
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    scale, ef, _, kind, nroots, _ = WORKLOADS[args.workload]
    if args.roots:
        nroots = args.roots
    if rank != 0:
        return
    n, src, dst = graphgen.edges(scale, ef, kind=kind)
    roots = graphgen.pick_roots(n, src, dst, nroots, seed=7)
    deg = graphgen.degrees(n, src, dst)
    g = oracle.csr(n, src, dst)
    ms, ts = [], []
    k = 0
    total_steps = args.warmup + args.steps
    step_times = []
    for step in range(total_steps):
        r = int(roots[k % len(roots)])
        k += 1
        t0 = time.perf_counter()
        level, parent = oracle.bfs(g, r)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            ms.append(graphgen.traversed_tuples(deg, level))
            ts.append(dt)
            step_times.append(dt)
    value = hm_gteps(ms, ts)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(step_times) / len(step_times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {**workload_config(args, n, len(src), nroots),
                   "step": "one search (plain single-threaded CPU oracle: queue BFS + smallest-parent pass)",
                   "parallelism": "one host core"},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} roots of the {nroots}, one per step"},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- our arm --

# ------------------------------------------------------- batch and serving --
def bench_batch(args, bfs, graphgen, torch, dev):
    """64 roots as one bit-parallel batch (bfs_run_batch, one CUDA-graph launch)
    on Kronecker scale 20, 8x8 grid: aggregate GTEPS = sum of m_r / batch time,
    beside the same 64 roots searched one by one."""
    n, src, dst = graphgen.edges(20, 16)
    roots = graphgen.pick_roots(n, src, dst, 64)
    g = bfs.Graph.from_edges(n, src, dst, p=8, mode=2)
    deg = (torch.bincount(torch.from_numpy(src).to(dev).long(), minlength=n)
           + torch.bincount(torch.from_numpy(dst).to(dev).long(), minlength=n))
    shape = g.batch_autotune(roots)
    levels = torch.empty((64, n), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        g.run_batch(roots, levels=levels)
    times = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.run_batch(roots, levels=levels)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    m = [int((deg * (levels[r] >= 0)).sum().item()) // 2 for r in range(64)]
    t_batch = sum(times) / len(times)
    # the same roots one by one (device outputs, no statistics)
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    level = torch.empty(n, dtype=torch.int32, device=dev)
    for r in roots[:4]:
        g.run(int(r), parent, level)
    t_single = 0.0
    for r in roots:
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.run(int(r), parent, level)
        e1.record()
        e1.synchronize()
        t_single += e0.elapsed_time(e1) / 1e3
    # the batch's level rows equal the single searches' (both bit-exact with the
    # oracle in the -m gpu tests)
    exact = 0
    for k in range(0, 64, 16):
        g.run(int(roots[k]), parent, level)
        exact += int(bool(torch.equal(level, levels[k])))
    line = {"metric": "aggregate GTEPS of one 64-root bit-parallel batch", "value": round(sum(m) / t_batch / 1e9, 3),
            "unit": "GTEPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t_batch, 3), "higher_is_better": True, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "kronecker-s20-ef16-grid8x8-batch64", "launch": "one CUDA graph per batch",
                       "autotuned_shape": {"threads": shape[0], "ctas_per_sm": shape[1]},
                       "l2": "flushed (256 MiB write) before every batch"},
            "single_searches": {"value": round(sum(m) / t_single / 1e9, 3), "unit": "GTEPS",
                                "ms_for_64": round(1e3 * t_single, 3)},
            "validation": {"batch_rows_equal_single_searches": exact, "checked": 4}}
    print(json.dumps(line), flush=True)
    return 0


def bench_serve(args, bfs, graphgen, torch, dev):
    """Continuous batching: a seeded Poisson stream (2,000 queries/s) of
    single-root searches over 8 resident Kronecker graphs (scales 16-22 and 24),
    each graph with up to 64 lanes; latency percentiles from the server and
    aggregate GTEPS over the stream."""
    import numpy as np
    scales = [16, 17, 18, 19, 20, 21, 22, 24]
    srv = bfs.Server(hbm_budget_bytes=48 << 30, max_lanes=64)
    graphs = []
    for sc in scales:
        n, src, dst = graphgen.edges(sc, 16)
        p = 4 if sc <= 18 else (8 if sc <= 22 else 16)
        g = bfs.Graph.from_edges(n, src, dst, p=p)
        deg = (torch.bincount(torch.from_numpy(src).to(dev).long(), minlength=n)
               + torch.bincount(torch.from_numpy(dst).to(dev).long(), minlength=n))
        graphs.append((srv.add_graph(g), n, g, deg, graphgen.pick_roots(n, src, dst, 256, seed=7 + sc)))
    rng = np.random.default_rng(11)
    rate = args.serve_rate
    # warm-up: a few queries per graph
    for gid, n, _, _, rts in graphs:
        for r in rts[:4]:
            srv.wait(srv.submit(gid, int(r)), n)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * args.serve_seconds * 1.2) + 16))
    arrivals = arrivals[arrivals < args.serve_seconds]
    which = rng.integers(0, len(graphs), size=len(arrivals))
    pick = rng.integers(0, 256, size=len(arrivals))
    base = srv.stats()
    # one client thread per graph collects that graph's results as soon as they
    # are done, so that results do not pile up against the HBM budget
    import queue
    import threading
    tqs = [queue.Queue() for _ in graphs]
    edges = [0] * len(graphs)

    def collect(k):
        gid, n, _, deg, _ = graphs[k]
        while True:
            t = tqs[k].get()
            if t is None:
                return
            lv = srv.wait(t, n, timeout_s=120.0)
            edges[k] += int((deg * (lv >= 0)).sum().item()) // 2

    ths = [threading.Thread(target=collect, args=(k,)) for k in range(len(graphs))]
    for th in ths:
        th.start()
    nsub = 0
    t0 = time.perf_counter()
    for a_t, k, q in zip(arrivals, which, pick):
        now = time.perf_counter() - t0
        if a_t > now:
            time.sleep(a_t - now)
        gid, n, _, _, rts = graphs[k]
        tqs[k].put(srv.submit(gid, int(rts[q])))
        nsub += 1
    for tq in tqs:
        tq.put(None)
    for th in ths:
        th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    line = {"metric": f"serving: p50/p99 query latency and aggregate GTEPS (Poisson {rate:,.0f} queries/s)",
            "value": round(sum(edges) / wall / 1e9, 3), "unit": "GTEPS", "n_gpus": 1, "higher_is_better": True,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "kronecker-s16..s22,s24-serving", "graphs": len(graphs), "rate_per_s": rate,
                       "seconds": args.serve_seconds, "queries": nsub, "lanes_per_graph": 64,
                       "client": "one thread per graph collects its results as they finish"},
            "latency_us": {"p50": st["p50_us"], "p99": st["p99_us"], "max": st["max_us"]},
            "server": {"completed": st["completed"] - base["completed"], "rejected": st["rejected"],
                       "iterations": st["iterations"], "peak_lanes": st["peak_lanes"],
                       "hbm_used_bytes": st["hbm_used_bytes"]},
            "wall_s": round(wall, 3)}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import graphgen
    from paper_1208_5542_gb300 import build as libbuild
    from paper_1208_5542_gb300 import bfs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        libbuild.build()
    if world > 1:
        dist.barrier()

    if args.workload == "msbfs20":
        return bench_batch(args, bfs, graphgen, torch, dev)
    if args.workload == "serve":
        return bench_serve(args, bfs, graphgen, torch, dev)

    scale, ef, p, kind, nroots, desc = WORKLOADS[args.workload]
    if args.roots:
        nroots = args.roots
    t_setup = time.perf_counter()
    n, src, dst = graphgen.edges(scale, ef, kind=kind)
    roots = graphgen.pick_roots(n, src, dst, nroots, seed=7 + 1000 * rank)
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=args.mode, wah_bits=args.wah_bits)
    g.set_row_exchange(args.row_exchange == "on")
    if args.direction != "top_down":
        g.set_direction(DIRECTIONS[args.direction], args.alpha, args.beta)
    src_d = torch.from_numpy(src).to(dev)
    dst_d = torch.from_numpy(dst).to(dev)
    deg = (torch.bincount(src_d.long(), minlength=n) + torch.bincount(dst_d.long(), minlength=n))
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    level = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    if args.profile_run:
        # one untimed search per mode from the first root, with the per-level
        # algorithmic bytes of the expansion (to set against ncu's DRAM bytes)
        out = {"profile_run": True, "workload": desc, "root": int(roots[0]), "kernel_hash": kernel_hash()}
        for mode in (args.mode, 0):
            g.set_mode(mode, args.wah_bits)
            _, _, st = g.run(int(roots[0]), parent, level, stats=True)
            alg = []
            for k, ls in enumerate(st.levels):
                nxt = st.levels[k + 1]["frontier_vertices"] if k + 1 < len(st.levels) else 0
                alg.append(4 * ls["edges_scanned"] + 12 * ls["column_hits"] + ls["wah_bytes"] + 4 * nxt)
            out[MODE_NAMES[mode]] = {"levels": st.n_levels, "expand_algorithmic_bytes": alg}
        torch.cuda.synchronize()
        print(json.dumps(out))
        return

    def step(record=False):
        """One search per root; returns per-root device times (s), m_r, and stats."""
        times, ms_, sts = [], [], []
        for r in roots:
            flush.fill_(1)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, _, st = g.run(int(r), parent, level, stats=record, timing=record, stream=stream)
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
            ms_.append(int((deg * (level >= 0)).sum().item()) // 2)
            sts.append(st)
        return times, ms_, sts

    def timed(mode):
        g.set_mode(mode, args.wah_bits)
        for _ in range(args.warmup):
            step()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        per_root = [[] for _ in roots]
        wall0 = time.perf_counter()
        m_r = None
        for _ in range(args.steps):
            t, m_r, _ = step()
            for i, x in enumerate(t):
                per_root[i].append(x)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - wall0
        t_mean = [sum(x) / len(x) for x in per_root]
        # one more pass, outside the timed steps, with per-level statistics and
        # phase events (the library's stepwise loop) for the roofline and the report
        _, _, sts = step(record=True)
        return t_mean, m_r, [sts], wall

    clocks = ClockSampler(local)
    clocks.start()
    t_cs, m_r, stats_cs, wall_cs = timed(args.mode)
    clk = clocks.stop()

    # whole-job value: roots of all ranks over the slowest rank's sum of t_r/m_r
    inv = sum(t / m for t, m in zip(t_cs, m_r) if m > 0)
    value, ms_step = job_value(inv, 1e3 * sum(t_cs), len(roots), dist if world > 1 else None, dev)

    # roofline of the expansion kernel (algorithmic bytes per launch / event time per launch)
    ex_bytes = ex_ms = 0.0
    ex_entries = 0
    launches = 0
    levels_tot = 0
    per_level = {}
    for sts in stats_cs:
        for st in sts:
            levels_tot += st.n_levels
            for k, ls in enumerate(st.levels):
                wah_read = ls["wah_bytes"]
                discovered = st.levels[k + 1]["frontier_vertices"] if k + 1 < len(st.levels) else 0
                # entries read (4 B) + rank word and column-pointer pair per item (12 B)
                # + streams decoded + one parent word per discovered vertex
                ex_bytes += 4 * ls["edges_scanned"] + 12 * ls["column_hits"] + wah_read + 4 * discovered
                ex_ms += ls["ms_traversing"]
                ex_entries += ls["edges_scanned"]
                launches += 1
                agg = per_level.setdefault(k, {"frontier": 0, "exchanged": 0, "raw_bytes": 0, "wah_bytes": 0,
                                                "hits": 0, "n": 0})
                agg["frontier"] += ls["frontier_vertices"]
                agg["exchanged"] += ls["exchanged_vertices"]
                agg["raw_bytes"] += ls["raw_bytes"]
                agg["wah_bytes"] += ls["wah_bytes"]
                agg["hits"] += ls["column_hits"]
                agg["n"] += 1
    # kernels of the timed steps: per level the sum, scan and write passes of the
    # encoder, expansion, hub pieces, reduction and the level step (PLAIN: expansion,
    # hub pieces, reduction, level step); per search the init, root and first-level
    # kernels.  The levels of every root are those of the recording pass.
    launches_per_level = {0: 4, 1: 7, 2: 7}[args.mode]
    if args.direction != "top_down":     # bottom-up expansion (+ clear and decode of the streams)
        launches_per_level += 1 if args.mode == 0 else 3
    gpu_launches = args.steps * sum(3 + launches_per_level * st.n_levels for st in stats_cs[0])
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (ex_bytes / launches) / (ex_ms / launches / 1e3) / 1e9 if launches and ex_ms > 0 else 0.0
    # the bound that binds the expansion on its L1/L2 path: one scattered read
    # (the visited test) per entry, against this GPU's measured scattered-read
    # rate on a region the size of one block-row's visited bits
    scatter_region = max(4096, (n // p + 7) // 8)
    scatter_peak = bfs.measure_scatter_reads(scatter_region) / 1e9
    scatter_achieved = ex_entries / (ex_ms / 1e3) / 1e9 if ex_ms > 0 else 0.0
    nb_range = -(-n // p)
    window = 8 * -(-nb_range // 32) + 4096 <= 227 * 1024      # the library's row-window rule
    traffic = None
    if args.direction == "top_down":     # the counters were taken on top-down levels
        traffic = ncu_traffic(args.workload, MODE_NAMES[args.mode], ex_bytes / launches if launches else 0)
    exch = []
    for k in sorted(per_level):
        a = per_level[k]
        f = a["frontier"] / a["n"]
        exch.append({"level": k, "frontier": round(f, 1),
                     "wah_over_raw": round(a["wah_bytes"] / a["raw_bytes"], 6) if a["raw_bytes"] else None,
                     "sieve_drop": round(1 - a["exchanged"] / (p * a["frontier"]), 4) if a["frontier"] else None})

    # phase breakdown (Table 6 labels), summed over the timed searches
    phases = {"compression_sieve": 0.0, "communication": 0.0, "traversing": 0.0, "row_compression_sieve": 0.0,
              "row_fold": 0.0, "reducing": 0.0}
    for sts in stats_cs:
        for st in sts:
            for ls in st.levels:
                phases["compression_sieve"] += ls["ms_compress_sieve"]
                phases["communication"] += ls["ms_communication"]
                phases["traversing"] += ls["ms_traversing"]
                phases["row_compression_sieve"] += ls["ms_row_compress"]
                phases["row_fold"] += ls["ms_row_fold"]
                phases["reducing"] += ls["ms_reducing"]
    nsearch = sum(len(s) for s in stats_cs)
    phases = {k: round(v / nsearch, 4) for k, v in phases.items()}

    # validation: BFS-tree invariants and the smallest-parent rule for every root
    # (torch over the edge list), bit-exact oracle comparison on the CPU-baseline sample
    g.set_mode(args.mode, args.wah_bits)
    invariant_ok = 0
    for r in roots:
        g.run(int(r), parent, level, stream=stream)
        lv = level.long()
        pa = parent.long()
        u, v = src_d.long(), dst_d.long()
        r = int(r)
        ok = bool(lv[r] == 0) and bool(pa[r] == r)
        lu, lvv = lv[u], lv[v]
        ok &= not bool(((lu >= 0) ^ (lvv >= 0)).any())
        both = (lu >= 0) & (lvv >= 0)
        ok &= not bool(((lu - lvv).abs()[both] > 1).any())
        best = torch.full((n,), 2**62, dtype=torch.int64, device=dev)
        m1 = (lvv == lu + 1) & (lu >= 0)
        best.scatter_reduce_(0, v[m1], u[m1], reduce="amin")
        m2 = (lu == lvv + 1) & (lvv >= 0)
        best.scatter_reduce_(0, u[m2], v[m2], reduce="amin")
        reached = (lv > 0)
        ok &= bool((pa[reached] == best[reached]).all())
        ok &= bool((pa[lv < 0] == -1).all())
        invariant_ok += int(ok)

    # PLAIN (BIT, Alg. 1) on the same graph
    plain = None
    if not args.no_plain and args.mode != 0:
        t_pl, m_pl, stats_pl, _ = timed(0)
        plain = {"value": hm_gteps(m_pl, t_pl), "ms_per_step": round(1e3 * sum(t_pl), 3)}
        g.set_mode(args.mode, args.wah_bits)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hp = torch.empty(n, dtype=torch.int32).pin_memory()
        hl = torch.empty(n, dtype=torch.int32).pin_memory()
        ts_e2e, m_e2e = [], []
        for r in roots:
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.run(int(r), hp, hl, stream=stream)
            ts_e2e.append(time.perf_counter() - t0)
            m_e2e.append(int(deg[torch.from_numpy(hl.numpy() >= 0).to(dev)].sum().item()) // 2)
        e2e = {"value": hm_gteps(m_e2e, ts_e2e), "unit": "GTEPS", "h2d_bytes_per_step": 4 * len(roots),
               "d2h_bytes_per_step": 8 * n * len(roots)}

    # CPU oracle on the host cores, bounded sample (rank 0, N = 1 only)
    cpu = None
    oracle_exact = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        go = oracle.csr(n, src, dst)
        m_c, t_c = [], []
        oracle_exact = 0
        t_start = time.perf_counter()
        for r in roots:
            t0 = time.perf_counter()
            lv_o, pa_o = oracle.bfs(go, int(r))
            t_c.append(time.perf_counter() - t0)
            m_c.append(int(deg[torch.from_numpy(lv_o >= 0).to(dev)].sum().item()) // 2)
            g.run(int(r), parent, level, stream=stream)
            oracle_exact += int(bool((level.cpu().numpy() == lv_o).all() and (parent.cpu().numpy() == pa_o).all()))
            if time.perf_counter() - t_start > args.cpu_seconds:
                break
        cpu = {"value": hm_gteps(m_c, t_c), "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": f"{len(t_c)} of the {len(roots)} roots (single-threaded queue BFS + smallest-parent pass)"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {**workload_config(args, n, len(src), len(roots)),
                   "step": "one search per root", "l2": "flushed (256 MiB write) before every search",
                   "parallelism": f"replicas x{world}"},
        "plain_gpu": plain,
        "roofline": {"kernel": ("expand_wah" if args.mode else "expand_plain") + " + expand_pieces" +
                     ("" if args.direction == "top_down" else " + expand_bottom_up"), "bound": "hbm",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4) if peak else None,
                     "peak_source": peak_src, "traffic": traffic,
                     "traffic_source": ("DRAM/algorithmic ratio of an ncu capture at scale 24 (same 16x16 grid and "
                                        "visiting path) times this launch's algorithmic bytes") if traffic else None,
                     "algorithmic_bytes_per_launch": round(ex_bytes / launches) if launches else 0,
                     "avg_launch_ms": round(ex_ms / launches, 5) if launches else 0, "launches": launches,
                     "scattered": {"bound": "scattered 4-byte reads (one visited test per entry)",
                                   "achieved": round(scatter_achieved, 1), "peak": round(scatter_peak, 1),
                                   "unit": "G entries/s vs G reads/s", "frac": round(scatter_achieved / scatter_peak, 4)
                                   if scatter_peak else None, "region_bytes": scatter_region,
                                   "peak_source": "measured in this run (bfs_measure_scatter_reads)",
                                   "visited_test": "shared-memory row window (this bound does not apply)" if window
                                   else "through L1/L2, one scattered read per entry"}},
        "phases_ms_per_search": phases,
        "exchange_per_level": exch,
        "compression_factor": compression_factor(exch, args.mode),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": gpu_launches,
        "validation": {"invariant_and_min_parent_roots": invariant_ok, "roots": len(roots),
                       "oracle_bit_exact_roots": oracle_exact},
        "setup_s": round(setup_s, 2), "timed_wall_s": round(wall_cs, 3),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
