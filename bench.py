#!/usr/bin/env python3
"""Harmonic-mean GTEPS of the compressed + sieved BFS on one GB300 (and N replicas).

One step = one breadth-first search from each of the workload's roots (64 by
default) on the resident graph, with the L2 flushed (a 256 MiB write) before
every search.  TEPS_r = m_r / t_r, where m_r is the number of input tuples in
the component reached from root r (self-loops and duplicates counted, Sec.
VII-A) and t_r the CUDA-event time of search r; the reported value is the
harmonic mean N_roots / sum_r (1 / TEPS_r).

Arms on the same resident graph, each timed the same way:
  value          DIR-WAH (Alg. 3): the frontier exchange sieved by the cross
                 directory and WAH-compressed; each block-row folds its
                 partials locally, as in the paper's 1D ownership;
  plain_gpu      BIT (Alg. 1): the raw bitmap exchange;
  row_exchange   DIR-WAH with the fold of every block-row itself a compressed,
                 sieved exchange of per-block row buffers (the 2D partition the
                 paper names in Sec. VIII; the library's default);
  hybrid         both exchanges with top-down / bottom-up levels (Sec. VIII, IX);
  adaptive       every exchanged slice as the smallest of WAH stream, sparse
                 vector and raw bitmap (Sec. II, Table 2);
  dynamic_directory  DIR-WAH sieved by the search's dynamic cross directory
                 (Sec. V-B), with the cost of its update.
The default run adds the other configurations (Kronecker scale 22 on 8 x 8, the
Erdos-Renyi scale-26 control, the 64-root batch, the serving stream) under
"configs".

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
import os
import re
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
KERNEL_SOURCES = ["paper_1208_5542_gb300/csrc/bfs_level.cu", "paper_1208_5542_gb300/csrc/wah.cu",
                  "paper_1208_5542_gb300/csrc/wah.cuh", "paper_1208_5542_gb300/csrc/common.cuh"]
CHUNK_GROUPS = 1024          # groups per chunk of the data-parallel encoder
ORACLE_SAMPLE_ENTRIES = 200_000_000   # adjacency entries per bounded oracle sample (a few seconds)


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
    ap.add_argument("--row-exchange", default="off", choices=["on", "off"],
                    help="the value arm's fold: off = local to the block-row (Alg. 3), on = row buffers")
    ap.add_argument("--format", default="wah", choices=["wah", "adaptive"],
                    help="the value arm's exchanged slices: WAH streams, or the smallest of WAH / vector / raw")
    ap.add_argument("--roots", type=int, default=0, help="override the number of roots")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of the row-exchange and hybrid arms")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-arms", action="store_true", help="skip the row-exchange and hybrid arms")
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-samples", type=int, default=3, help="bounded oracle samples of the CPU baseline")
    ap.add_argument("--profile-run", action="store_true",
                    help="build the graph and run one search per arm, untimed (for ncu)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers --
def code_digest(texts):
    """Hash of C/CUDA sources' code: comments and blank lines do not count."""
    h = hashlib.sha256()
    for text in texts:
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for line in text.splitlines():
            line = re.sub(r"//.*", "", line).rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def kernel_hash():
    """Hash of the kernel sources' code, so that a comment edit does not retire
    the committed ncu counters."""
    texts = []
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as fh:
            texts.append(fh.read())
    return code_digest(texts)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(key, algorithmic_bytes):
    """Per-launch DRAM bytes of a kernel: the DRAM / algorithmic byte ratio of the
    committed ncu summary (profiles/ncu_traffic.json, entry `key`) times this
    launch's algorithmic bytes; None if no capture was taken for it or the
    kernels changed since.  Returns (bytes, source)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
    except OSError:
        return None, None
    ent = data.get(key)
    if not ent or ent.get("kernel_hash") != kernel_hash():
        return None, None
    return round(ent["dram_over_algorithmic"] * algorithmic_bytes), ent.get("source")


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


def compression_factor(per_root, mode):
    """C (Alg. 2) or C' (Alg. 3) of Sec. VI-A for one search: the mean over its
    levels of the compressed-to-raw size of the exchange (1 / C_i at level i);
    averaged over the searches.  `per_root` holds, per search, its levels'
    compressed / raw ratios (None for a level without a raw size).  None for
    PLAIN (nothing is compressed) or when no level was recorded."""
    if mode == 0:
        return None
    vals, nlev = [], 0
    for levels in per_root:
        r = [x for x in levels if x is not None]
        if r:
            vals.append(sum(r) / len(r))
            nlev += len(r)
    if not vals:
        return None
    return {"symbol": "C'" if mode == 2 else "C", "value": round(sum(vals) / len(vals), 6),
            "searches": len(vals), "levels_per_search": round(nlev / len(vals), 2)}


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


def oracle_sample_gteps(oracle, go, roots, samples, budget):
    """Bounded samples of the oracle's queue BFS (one core): per sample the
    search from the next root stopped after `budget` scanned entries; the TEPS
    of a sample = scanned entries / 2 (tuples) / time.  Returns (harmonic-mean
    GTEPS, per-sample seconds)."""
    ms, ts = [], []
    for k in range(samples):
        r = int(roots[k % len(roots)])
        t0 = time.perf_counter()
        _, scanned = oracle.bfs_sample(go, r, budget)
        ts.append(time.perf_counter() - t0)
        ms.append(scanned // 2)
    return hm_gteps(ms, ts), ts


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores (one core): every step is
    a bounded sample of the workload -- the oracle's queue BFS from the next
    root, stopped after a fixed budget of scanned adjacency entries."""
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
    g = oracle.csr(n, src, dst)
    budget = min(ORACLE_SAMPLE_ENTRIES, len(g.col))
    oracle_sample_gteps(oracle, g, roots, args.warmup, budget)
    rest = list(roots[args.warmup % len(roots):]) + list(roots[:args.warmup % len(roots)])
    value, ts = oracle_sample_gteps(oracle, g, rest, args.steps, budget)
    sample = (f"{args.steps} bounded samples: the queue BFS from the next root stopped after {budget:,} scanned "
              "entries (tuples = entries / 2)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(args, n, len(src), nroots),
        "method": {"step": "one bounded oracle sample (plain single-threaded CPU queue BFS)",
                   "parallelism": "one host core"},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- our arm --
def level_rooflines(stats, n, wbits, peak, peak_src, workload):
    """Per-kernel rooflines from the recording pass's per-level counters and
    CUDA-event phase times: the algorithmic bytes of each level's launch of the
    kernel over its event time, summed over the top-down levels of every
    recorded search.  Returns ({kernel: entry}, entries scanned)."""
    chunk_bytes = CHUNK_GROUPS * (wbits - 1) // 8
    acc = {k: [0.0, 0.0, 0] for k in ("expansion", "compress_sieve", "reduce", "row_compress_sieve", "row_fold")}
    entries = 0
    for st in stats:
        for k, ls in enumerate(st.levels):
            if ls["bottom_up"]:
                continue
            discovered = st.levels[k + 1]["frontier_vertices"] if k + 1 < len(st.levels) else 0
            # expansion: entries read (4 B) + rank word and column-pointer pair per item (12 B)
            # + streams decoded + one parent word per discovered vertex
            acc["expansion"][0] += 4 * ls["edges_scanned"] + 12 * ls["column_hits"] + ls["wah_bytes"] + 4 * discovered
            acc["expansion"][1] += ls["ms_traversing"]
            acc["expansion"][2] += 1
            entries += ls["edges_scanned"]
            if ls["compress_chunks"] or ls["wah_bytes"]:
                # sieve + compress: every chunk read holds frontier and directory bits; the streams written
                acc["compress_sieve"][0] += 2 * chunk_bytes * ls["compress_chunks"] + ls["wah_bytes"]
                acc["compress_sieve"][1] += ls["ms_compress_sieve"]
                acc["compress_sieve"][2] += 1
            # reduce: t, pi read; pi, f, t written (20 B per 32-bit word); a level per discovered vertex
            acc["reduce"][0] += 20 * ((n + 31) // 32) + 4 * discovered + n // 1024
            acc["reduce"][1] += ls["ms_reducing"]
            acc["reduce"][2] += 1
            if ls["row_compress_chunks"] or ls["row_wah_bytes"]:
                acc["row_compress_sieve"][0] += 2 * chunk_bytes * ls["row_compress_chunks"] + ls["row_wah_bytes"]
                acc["row_compress_sieve"][1] += ls["ms_row_compress"]
                acc["row_compress_sieve"][2] += 1
                # the fold: row buffers read, the block-rows' next bits written
                acc["row_fold"][0] += ls["row_wah_bytes"] + (n + 7) // 8
                acc["row_fold"][1] += ls["ms_row_fold"]
                acc["row_fold"][2] += 1
    out = {}
    for name, (b, ms, launches) in acc.items():
        if not launches or ms <= 0:
            continue
        achieved = (b / launches) / (ms / launches / 1e3) / 1e9
        traffic, src = ncu_traffic(f"{workload}:{name}", b / launches)
        out[name] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4) if peak else None, "peak_source": peak_src,
                     "traffic": traffic, "traffic_source": src,
                     "algorithmic_bytes_per_launch": round(b / launches), "avg_launch_ms": round(ms / launches, 5),
                     "launches": launches}
    return out, entries


def search_roofline_of(levels_per_search, m, wbits, peak, value, peak_src):
    """The whole search against HBM: per search, its algorithmic bytes over its
    traversed edges m_r -- adjacency entries 4 B, (vertex, block) columns 12 B
    (rank word and column-pointer pair), level, parent and candidate parent 12 B
    per reached vertex, every stream written and read, the directory words the
    sieve reads with each live chunk -- averaged over the searches; the GTEPS the
    copy rate `peak` (GB/s) allows at that rate, and `value` against it."""
    bpe = []
    for levels, m_r in zip(levels_per_search, m):
        if not m_r:
            continue
        b = sum(4 * ls["edges_scanned"] + 12 * ls["column_hits"] + 2 * ls["wah_bytes"] +
                (CHUNK_GROUPS * (wbits - 1) // 8) * ls["compress_chunks"] + 12 * ls["frontier_vertices"]
                for ls in levels)
        bpe.append(b / m_r)
    if not bpe:
        return None
    per_edge = sum(bpe) / len(bpe)
    bound = peak / per_edge
    return {"bound": "hbm", "bytes_per_edge": round(per_edge, 3), "peak_gbs": peak, "bound_gteps": round(bound, 1),
            "achieved_gteps": round(value, 4), "frac": round(value / bound, 4), "peak_source": peak_src}


def validate_all(g, roots, parent, level, src_d, dst_d, n, dev, stream, torch):
    """BFS-tree invariants and the smallest-parent rule, every root (torch over
    the edge list): the root is its own parent at level 0; both ends of every
    edge are reached or neither; levels differ by at most 1 along an edge; the
    parent is the smallest neighbour one level closer; unreached vertices have
    parent -1.  Returns the number of roots that pass."""
    ok_roots = 0
    u, v = src_d.long(), dst_d.long()
    for r in roots:
        g.run(int(r), parent, level, stream=stream)
        lv = level.long()
        pa = parent.long()
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
        ok_roots += int(ok)
    return ok_roots


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import graphgen
    from paper_1208_5542_gb300 import bfs
    from paper_1208_5542_gb300 import build as libbuild

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
        print(json.dumps(bench_batch(args, bfs, graphgen, torch, dev)), flush=True)
        return 0
    if args.workload == "serve":
        print(json.dumps(bench_serve(args, bfs, graphgen, torch, dev)), flush=True)
        return 0

    scale, ef, p, kind, nroots, desc = WORKLOADS[args.workload]
    if args.roots:
        nroots = args.roots
    t_setup = time.perf_counter()
    n, src, dst = graphgen.edges(scale, ef, kind=kind)
    roots = graphgen.pick_roots(n, src, dst, nroots, seed=7 + 1000 * rank)
    g = bfs.Graph.from_edges(n, src, dst, p=p, mode=args.mode, wah_bits=args.wah_bits)
    src_d = torch.from_numpy(src).to(dev)
    dst_d = torch.from_numpy(dst).to(dev)
    deg = (torch.bincount(src_d.long(), minlength=n) + torch.bincount(dst_d.long(), minlength=n))
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    level = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def configure(mode, rowx, direction, adaptive=None, dynamic=False):
        g.set_mode(mode, args.wah_bits)
        g.set_dynamic_directory(dynamic)
        g.set_row_exchange(rowx)
        g.set_direction(DIRECTIONS[direction], args.alpha, args.beta)
        g.set_exchange_format(args.format == "adaptive" if adaptive is None else adaptive)

    if args.profile_run:
        # one untimed search per arm from the first root (for ncu), with the
        # per-level counters that give each kernel's algorithmic bytes
        out = {"profile_run": True, "workload": desc, "root": int(roots[0]), "kernel_hash": kernel_hash()}
        for name, mode, rowx, dyn in (("compress_sieve", args.mode, args.row_exchange == "on", False),
                                      ("plain", 0, False, False), ("row_exchange", 2, True, False),
                                      ("dynamic_directory", 2, False, True)):
            configure(mode, rowx, args.direction, dynamic=dyn)
            _, _, st = g.run(int(roots[0]), parent, level, stats=True)
            out[name] = {"levels": st.n_levels, "per_level": [
                {f: st.levels[k][f] for f in ("edges_scanned", "column_hits", "wah_bytes", "row_wah_bytes",
                                               "compress_chunks", "row_compress_chunks", "frontier_vertices",
                                               "exchanged_vertices")}
                for k in range(st.n_levels)]}
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

    def timed(mode, rowx, direction, steps, warmup, record=True, adaptive=None, dynamic=False):
        """Warm-up, then `steps` timed steps (the library's CUDA-graph level loop,
        no statistics); then one recording pass (the stepwise loop with per-level
        statistics and phase events) outside the timed steps."""
        configure(mode, rowx, direction, adaptive, dynamic)
        for _ in range(warmup):
            step()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        per_root = [[] for _ in roots]
        wall0 = time.perf_counter()
        m_r = None
        for _ in range(steps):
            t, m_r, _ = step()
            for i, x in enumerate(t):
                per_root[i].append(x)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - wall0
        t_mean = [sum(x) / len(x) for x in per_root]
        sts = step(record=True)[2] if record else None
        return {"t": t_mean, "m": m_r, "stats": sts, "wall": wall, "gteps": hm_gteps(m_r, t_mean),
                "ms_per_step": 1e3 * sum(t_mean)}

    value_rowx = args.row_exchange == "on"
    clocks = ClockSampler(local)
    clocks.start()
    main_arm = timed(args.mode, value_rowx, args.direction, args.steps, args.warmup)
    clk = clocks.stop()

    # whole-job value: roots of all ranks over the slowest rank's sum of t_r/m_r
    inv = sum(t / m for t, m in zip(main_arm["t"], main_arm["m"]) if m > 0)
    value, ms_step = job_value(inv, main_arm["ms_per_step"], len(roots), dist if world > 1 else None, dev)

    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    kr, ex_entries = level_rooflines(main_arm["stats"], n, args.wah_bits, peak, peak_src, args.workload)
    ex = kr.pop("expansion", None)
    # the bound that binds the expansion on its L1/L2 path: one scattered read
    # (the visited test) per entry, against this GPU's measured scattered-read
    # rate on a region the size of one block-row's visited bits
    scatter_region = max(4096, (n // p + 7) // 8)
    scatter_peak = bfs.measure_scatter_reads(scatter_region) / 1e9
    nb_range = -(-n // p)
    window = 8 * -(-nb_range // 32) + 4096 <= 227 * 1024      # the library's row-window rule
    roofline = None
    if ex:
        ex_ms = ex["avg_launch_ms"] * ex["launches"]
        scatter_achieved = ex_entries / (ex_ms / 1e3) / 1e9 if ex_ms > 0 else 0.0
        roofline = {"kernel": ("expand_wah" if args.mode else "expand_plain") + " + expand_pieces", **ex,
                    "scattered": {"bound": "scattered 4-byte reads (one visited test per entry)",
                                  "achieved": round(scatter_achieved, 1), "peak": round(scatter_peak, 1),
                                  "unit": "G entries/s vs G reads/s",
                                  "frac": round(scatter_achieved / scatter_peak, 4) if scatter_peak else None,
                                  "region_bytes": scatter_region,
                                  "peak_source": "measured in this run (bfs_measure_scatter_reads)",
                                  "visited_test": "shared-memory row window (this bound does not apply)" if window
                                  else "through L1/L2, one scattered read per entry"}}
    # the kernel times come from the stepwise recording pass; the timed steps run
    # the same kernels as one CUDA-graph launch per search: the two side by side
    stepwise_ms = 0.0
    for st in main_arm["stats"]:
        for ls in st.levels:
            stepwise_ms += (ls["ms_compress_sieve"] + ls["ms_communication"] + ls["ms_traversing"] +
                            ls["ms_row_compress"] + ls["ms_row_fold"] + ls["ms_reducing"])
    timing_modes = {"graph_ms_per_search": round(main_arm["ms_per_step"] / len(roots), 4),
                    "stepwise_phases_ms_per_search": round(stepwise_ms / len(roots), 4)}
    # the whole search against HBM (the GTEPS roofline): algorithmic bytes per
    # traversed edge -- adjacency entries 4 B, (vertex, block) columns 12 B (rank
    # word and column-pointer pair), level, parent and candidate-parent 12 B per
    # reached vertex, every stream written and read, the directory words the
    # sieve reads -- and the GTEPS the measured copy rate allows at that rate
    search_roofline = search_roofline_of([st.levels for st in main_arm["stats"]], main_arm["m"], args.wah_bits,
                                         peak, value, peak_src)

    per_level, per_root_ratio = {}, []
    phases = {"compression_sieve": 0.0, "communication": 0.0, "traversing": 0.0, "row_compression_sieve": 0.0,
              "row_fold": 0.0, "reducing": 0.0}
    for st in main_arm["stats"]:
        ratios = []
        for k, ls in enumerate(st.levels):
            a = per_level.setdefault(k, {"frontier": 0, "exchanged": 0, "raw_bytes": 0, "wah_bytes": 0, "n": 0})
            a["frontier"] += ls["frontier_vertices"]
            a["exchanged"] += ls["exchanged_vertices"]
            a["raw_bytes"] += ls["raw_bytes"]
            a["wah_bytes"] += ls["wah_bytes"]
            a["n"] += 1
            ratios.append(ls["wah_bytes"] / ls["raw_bytes"] if ls["raw_bytes"] else None)
            phases["compression_sieve"] += ls["ms_compress_sieve"]
            phases["communication"] += ls["ms_communication"]
            phases["traversing"] += ls["ms_traversing"]
            phases["row_compression_sieve"] += ls["ms_row_compress"]
            phases["row_fold"] += ls["ms_row_fold"]
            phases["reducing"] += ls["ms_reducing"]
        per_root_ratio.append(ratios)
    phases = {k: round(v / len(roots), 4) for k, v in phases.items()}
    exch = []
    for k in sorted(per_level):
        a = per_level[k]
        f = a["frontier"] / a["n"]
        exch.append({"level": k, "frontier": round(f, 1),
                     "wah_over_raw": round(a["wah_bytes"] / a["raw_bytes"], 6) if a["raw_bytes"] else None,
                     "sieve_drop": round(1 - a["exchanged"] / (p * a["frontier"]), 4) if a["frontier"] else None})

    # validation of the value arm: BFS-tree invariants and the smallest-parent rule, every root
    configure(args.mode, value_rowx, args.direction)
    invariant_ok = validate_all(g, roots, parent, level, src_d, dst_d, n, dev, stream, torch)

    # the other arms on the same graph
    arms = {}
    plain = None
    if not args.no_plain and args.mode != 0:
        pl = timed(0, False, args.direction, args.steps, args.warmup, record=False)
        plain = {"value": round(pl["gteps"], 4), "ms_per_step": round(pl["ms_per_step"], 3)}
    if not args.no_arms and args.mode == 2:
        rx = timed(2, not value_rowx, args.direction, args.extra_steps, 2)
        rk, _ = level_rooflines(rx["stats"], n, args.wah_bits, peak, peak_src, args.workload)
        row_bytes = sum(ls["row_wah_bytes"] for st in rx["stats"] for ls in st.levels) / len(roots)
        arms["row_exchange"] = {
            "fold": "row buffers (on)" if not value_rowx else "local (off)", "value": round(rx["gteps"], 4),
            "ms_per_step": round(rx["ms_per_step"], 3), "steps": args.extra_steps,
            "cost_vs_value": round(rx["ms_per_step"] / main_arm["ms_per_step"] - 1, 4),
            "row_bytes_per_search": round(row_bytes),
            "rooflines": {k: v for k, v in rk.items() if k.startswith("row_")},
            "validation": {"invariant_and_min_parent_roots":
                           validate_all(g, roots, parent, level, src_d, dst_d, n, dev, stream, torch),
                           "roots": len(roots)}}
        if args.direction == "top_down":
            hy = {"direction": f"hybrid (alpha {args.alpha}, beta {args.beta})", "steps": args.extra_steps}
            for name, mode in (("compress_sieve", 2), ("plain", 0)):
                h = timed(mode, False, "hybrid", args.extra_steps, 2, record=False)
                hy[name] = {"value": round(h["gteps"], 4), "ms_per_step": round(h["ms_per_step"], 3),
                            "validation": {"invariant_and_min_parent_roots":
                                           validate_all(g, roots, parent, level, src_d, dst_d, n, dev, stream,
                                                        torch), "roots": len(roots)}}
            arms["hybrid"] = hy
        if args.wah_bits == 32:
            # the level-adaptive exchange format: every slice as the smallest of its
            # WAH stream, sparse vector and raw bitmap
            ad = {"format": "adaptive (WAH / sparse vector / raw bitmap per slice and level)",
                  "steps": args.extra_steps}
            for name, direction in (("top_down", args.direction), ("hybrid", "hybrid")):
                if name == "hybrid" and args.direction != "top_down":
                    continue
                h = timed(2, value_rowx, direction, args.extra_steps, 2, record=name == "top_down",
                          adaptive=args.format != "adaptive")
                ad[name] = {"value": round(h["gteps"], 4), "ms_per_step": round(h["ms_per_step"], 3),
                            "validation": {"invariant_and_min_parent_roots":
                                           validate_all(g, roots, parent, level, src_d, dst_d, n, dev, stream,
                                                        torch), "roots": len(roots)}}
                if h["stats"]:
                    ex_b = sum(ls["wah_bytes"] for st in h["stats"] for ls in st.levels)
                    raw_b = sum(ls["raw_bytes"] for st in h["stats"] for ls in st.levels)
                    ad[name]["exchange_over_raw"] = round(ex_b / raw_b, 6) if raw_b else None
            arms["adaptive" if args.format != "adaptive" else "wah_format"] = ad
        # the dynamic cross directory (Sec. V-B): the sieve drops the vertices whose
        # every entry into a block-row leads to a visited vertex; its update walks the
        # entries of every visited vertex once per search
        dy = timed(2, value_rowx, args.direction, args.extra_steps, 2, dynamic=True)
        ex_dyn = sum(ls["exchanged_vertices"] for st in dy["stats"] for ls in st.levels)
        ex_static = sum(ls["exchanged_vertices"] for st in main_arm["stats"] for ls in st.levels)
        arms["dynamic_directory"] = {
            "value": round(dy["gteps"], 4), "ms_per_step": round(dy["ms_per_step"], 3), "steps": args.extra_steps,
            "cost_vs_value": round(dy["ms_per_step"] / main_arm["ms_per_step"] - 1, 4),
            "exchanged_over_static": round(ex_dyn / ex_static, 4) if ex_static else None,
            "wah_bytes_per_search": round(sum(ls["wah_bytes"] for st in dy["stats"] for ls in st.levels) / len(roots)),
            "update_ms_per_search": round(sum(ls["ms_directory_update"] for st in dy["stats"]
                                              for ls in st.levels) / len(roots), 4),
            "validation": {"invariant_and_min_parent_roots":
                           validate_all(g, roots, parent, level, src_d, dst_d, n, dev, stream, torch),
                           "roots": len(roots)}}
        configure(args.mode, value_rowx, args.direction)

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

    # CPU oracle on the host cores (rank 0, N = 1 only): bounded samples for the
    # baseline, one full search compared with the GPU bit for bit
    cpu = None
    oracle_exact = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        go = oracle.csr(n, src, dst)
        budget = min(ORACLE_SAMPLE_ENTRIES, len(go.col))
        v, ts = oracle_sample_gteps(oracle, go, roots, args.cpu_samples, budget)
        cpu = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": f"{len(ts)} bounded samples, {sum(ts):.1f} s: the queue BFS from a root stopped after "
                         f"{budget:,} scanned entries (tuples = entries / 2)"}
        r0 = int(roots[0])
        lv_o, pa_o = oracle.bfs(go, r0)
        g.run(r0, parent, level, stream=stream)
        oracle_exact = int(bool((level.cpu().numpy() == lv_o).all() and (parent.cpu().numpy() == pa_o).all()))
        del go

    valid = invariant_ok == len(roots) and oracle_exact in (None, 1)
    # kernels of the timed steps, per level: the encoder's three passes (not PLAIN), the
    # expansion and the piece kernel (two variants each off the row window), the
    # row encoder's three passes and the fold (row exchange), the reduction and the
    # level step; per search the init, root and first-level kernels
    variants = 1 if window else 2
    launches_per_level = (0 if args.mode == 0 else 3) + 2 * variants + 2 + (4 if value_rowx else 0)
    if args.direction != "top_down":     # bottom-up expansion (+ clear and decode of the streams)
        launches_per_level += 1 if args.mode == 0 else (4 if args.format == "adaptive" else 3)
    gpu_launches = args.steps * sum(3 + launches_per_level * st.n_levels for st in main_arm["stats"])

    configs = None
    if not args.no_configs and args.workload == "s26" and world == 1:
        del g
        torch.cuda.empty_cache()
        configs = other_configs(args, bfs, graphgen, torch, dev)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": round(value, 4) if valid else 0.0, "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(args, n, len(src), len(roots)),
        "method": {"step": "one search per root", "l2": "flushed (256 MiB write) before every search",
                   "parallelism": f"replicas x{world}",
                   "fold": "row buffers (2D fold)" if value_rowx else "local to the block-row (Alg. 3)",
                   "exchange_format": args.format},
        "plain_gpu": plain,
        **arms,
        "roofline": roofline,
        "search_roofline": search_roofline,
        "kernel_rooflines": kr,
        "timing_modes": timing_modes,
        "phases_ms_per_search": phases,
        "exchange_per_level": exch,
        "compression_factor": compression_factor(per_root_ratio, args.mode),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": gpu_launches,
        "validation": {"invariant_and_min_parent_roots": invariant_ok, "roots": len(roots),
                       "oracle_bit_exact_roots": oracle_exact, "passed": valid},
        "configs": configs,
        "setup_s": round(setup_s, 2), "timed_wall_s": round(main_arm["wall"], 3),
    }
    if not valid:
        line["validation_failed"] = True
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def codec_study(g, bfs, torch, n, p, root):
    """The bitmap codes on the slices one DIR-WAH search exchanges (Sec. IV names
    BBC and PLWAH beside WAH; the paper weighs codes by size and time): every
    slice of every level decoded from its WAH stream on the GPU, then encoded
    and decoded again with each code through the library (one call per slice,
    scratch allocation and synchronisation included); bytes per code over the
    search, mean microseconds per slice, and every round trip checked."""
    nb = -(-n // p)
    cap = 1 << 26
    g.set_mode(2, 32)
    g.set_row_exchange(False)
    _, _, st = g.run(int(root), stats=True, trace_capacity=cap)
    torch.cuda.synchronize()
    words = st.trace_words[: st.trace_used]
    counts = st.trace_counts.cpu().numpy()
    out = {"slices": 0, "bytes": {"wah": 0, "plwah": 0, "bbc": 0, "raw": 0},
           "us_per_slice": {"wah_decode": 0.0, "plwah_encode": 0.0, "plwah_decode": 0.0, "bbc_encode": 0.0,
                            "bbc_decode": 0.0}, "round_trips_equal": 0}
    off = 0
    for k in range(counts.shape[0]):
        for s, c in enumerate(counts[k]):
            c = int(c)
            j = s % p
            nbits = max(0, min(n, (j + 1) * nb) - j * nb)
            w = words[off: off + c]
            off += c
            t0 = time.perf_counter()
            bits = bfs.wah_decode(w, nbits)
            t1 = time.perf_counter()
            pl = bfs.plwah_encode(bits, nbits)
            t2 = time.perf_counter()
            plb = bfs.plwah_decode(pl, nbits)
            t3 = time.perf_counter()
            bb = bfs.bbc_encode(bits, nbits)
            t4 = time.perf_counter()
            bbb = bfs.bbc_decode(bb, nbits)
            t5 = time.perf_counter()
            for key, dt in (("wah_decode", t1 - t0), ("plwah_encode", t2 - t1), ("plwah_decode", t3 - t2),
                            ("bbc_encode", t4 - t3), ("bbc_decode", t5 - t4)):
                out["us_per_slice"][key] += dt * 1e6
            out["bytes"]["wah"] += 4 * c
            out["bytes"]["plwah"] += 4 * pl.numel()
            out["bytes"]["bbc"] += bb.numel()
            out["bytes"]["raw"] += 4 * ((nbits + 31) // 32)
            out["round_trips_equal"] += int(torch.equal(plb, bits) and torch.equal(bbb, bits))
            out["slices"] += 1
    for key in out["us_per_slice"]:
        out["us_per_slice"][key] = round(out["us_per_slice"][key] / max(1, out["slices"]), 1)
    out["over_wah"] = {k: round(v / out["bytes"]["wah"], 4) for k, v in out["bytes"].items()} if out["bytes"]["wah"] else None
    return out


def other_configs(args, bfs, graphgen, torch, dev):
    """The other configurations, each with its own validation: Kronecker scale
    22 on 8 x 8 (DIR-WAH, BIT, and DIR-WAH with the row exchange), the
    Erdos-Renyi scale-26 control (DIR-WAH, BIT), the 64-root batch and the
    serving stream.  Fewer timed steps than the headline."""
    import oracle
    out = {}
    steps = max(1, min(args.steps, args.extra_steps))
    for wl in ("s22", "s26er"):
        scale, ef, p, kind, nroots, desc = WORKLOADS[wl]
        n, src, dst = graphgen.edges(scale, ef, kind=kind)
        roots = graphgen.pick_roots(n, src, dst, nroots, seed=7)
        g = bfs.Graph.from_edges(n, src, dst, p=p, mode=2)
        src_d = torch.from_numpy(src).to(dev)
        dst_d = torch.from_numpy(dst).to(dev)
        deg = torch.bincount(src_d.long(), minlength=n) + torch.bincount(dst_d.long(), minlength=n)
        parent = torch.empty(n, dtype=torch.int32, device=dev)
        level = torch.empty(n, dtype=torch.int32, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream()
        res = {"workload": desc + f"-{nroots}roots", "grid": f"{p}x{p}", "steps": steps}
        for name, mode, rowx in (("compress_sieve", 2, False), ("plain", 0, False), ("row_exchange", 2, True)):
            if wl == "s26er" and name == "row_exchange":
                continue
            g.set_mode(mode, 32)
            g.set_row_exchange(rowx)
            ts = [0.0] * len(roots)
            ms = [0] * len(roots)
            for it in range(2 + steps):
                for i, r in enumerate(roots):
                    flush.fill_(1)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    g.run(int(r), parent, level, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    if it >= 2:
                        ts[i] += e0.elapsed_time(e1) / 1e3 / steps
                        ms[i] = int((deg * (level >= 0)).sum().item()) // 2
            inv_ok = validate_all(g, roots, parent, level, src_d, dst_d, n, dev, stream, torch)
            res[name] = {"value": round(hm_gteps(ms, ts), 4) if inv_ok == len(roots) else 0.0,
                         "ms_per_step": round(1e3 * sum(ts), 3),
                         "validation": {"invariant_and_min_parent_roots": inv_ok, "roots": len(roots)}}
        # the oracle on one root: the full search at scale 22, the levels of a
        # bounded sample (a prefix of the search) at scale 26
        go = oracle.csr(n, src, dst)
        r0 = int(roots[0])
        g.set_mode(2, 32)
        g.set_row_exchange(True)
        g.run(r0, parent, level, stream=stream)
        glv = level.cpu().numpy()
        if scale <= 22:
            lv_o, pa_o = oracle.bfs(go, r0)
            res["oracle"] = {"root": r0, "bit_exact": bool((glv == lv_o).all() and
                                                           (parent.cpu().numpy() == pa_o).all())}
            res["codecs"] = codec_study(g, bfs, torch, n, p, r0)
        else:
            lv_o, _ = oracle.bfs_sample(go, r0, ORACLE_SAMPLE_ENTRIES)
            got = lv_o >= 0
            res["oracle"] = {"root": r0, "sample_levels_equal": bool((glv[got] == lv_o[got]).all()),
                             "sample_vertices": int(got.sum())}
        out[wl] = res
        del g, go, src_d, dst_d, deg, parent, level, flush
        torch.cuda.empty_cache()
    a = argparse.Namespace(**vars(args))
    a.steps, a.warmup = steps, 2
    out["msbfs20"] = bench_batch(a, bfs, graphgen, torch, dev)
    out["serve"] = bench_serve(a, bfs, graphgen, torch, dev)
    return out


# ------------------------------------------------------- batch and serving --
def bench_batch(args, bfs, graphgen, torch, dev):
    """64 roots as one bit-parallel batch (bfs_run_batch, one CUDA-graph launch)
    on Kronecker scale 20, 8x8 grid: aggregate GTEPS = sum of m_r / batch time,
    beside the same 64 roots searched one by one."""
    import oracle
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
    # four lanes against the oracle
    go = oracle.csr(n, src, dst)
    exact = sum(int(bool((levels[k].cpu().numpy() == oracle.bfs_levels(go, int(roots[k]))).all()))
                for k in range(0, 64, 16))
    return {"metric": "aggregate GTEPS of one 64-root bit-parallel batch", "value": round(sum(m) / t_batch / 1e9, 3),
            "unit": "GTEPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t_batch, 3), "higher_is_better": True, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "kronecker-s20-ef16-grid8x8-batch64", "launch": "one CUDA graph per batch",
                       "autotuned_shape": {"threads": shape[0], "ctas_per_sm": shape[1]},
                       "l2": "flushed (256 MiB write) before every batch"},
            "single_searches": {"value": round(sum(m) / t_single / 1e9, 3), "unit": "GTEPS",
                                "ms_for_64": round(1e3 * t_single, 3)},
            "validation": {"lanes_equal_to_oracle": exact, "checked": 4}}


def bench_serve(args, bfs, graphgen, torch, dev):
    """Continuous batching: a seeded Poisson stream (2,000 queries/s) of
    single-root searches over 8 resident Kronecker graphs (scales 16-22 and 24),
    each graph with up to 64 lanes; latency percentiles from the server and
    aggregate GTEPS over the stream; results on the small graphs against the oracle."""
    import queue
    import threading

    import numpy as np

    import oracle
    scales = [16, 17, 18, 19, 20, 21, 22, 24]
    srv = bfs.Server(hbm_budget_bytes=48 << 30, max_lanes=64)
    graphs = []
    for sc in scales:
        n, src, dst = graphgen.edges(sc, 16)
        p = 4 if sc <= 18 else (8 if sc <= 22 else 16)
        g = bfs.Graph.from_edges(n, src, dst, p=p)
        deg = (torch.bincount(torch.from_numpy(src).to(dev).long(), minlength=n)
               + torch.bincount(torch.from_numpy(dst).to(dev).long(), minlength=n))
        graphs.append((srv.add_graph(g), n, g, deg, graphgen.pick_roots(n, src, dst, 256, seed=7 + sc),
                       (src, dst) if sc <= 18 else None))
    rng = np.random.default_rng(11)
    rate = args.serve_rate
    # warm-up: a few queries per graph
    for gid, n, _, _, rts, _ in graphs:
        for r in rts[:4]:
            srv.wait(srv.submit(gid, int(r)), n)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * args.serve_seconds * 1.2) + 16))
    arrivals = arrivals[arrivals < args.serve_seconds]
    which = rng.integers(0, len(graphs), size=len(arrivals))
    pick = rng.integers(0, 256, size=len(arrivals))
    base = srv.stats()
    # one client thread per graph collects that graph's results as soon as they
    # are done, so that results do not pile up against the HBM budget
    tqs = [queue.Queue() for _ in graphs]
    edges = [0] * len(graphs)
    kept = {}

    def collect(k):
        _, n, _, deg, _, keep = graphs[k]
        while True:
            item = tqs[k].get()
            if item is None:
                return
            t, r = item
            lv = srv.wait(t, n, timeout_s=120.0)
            edges[k] += int((deg * (lv >= 0)).sum().item()) // 2
            if keep is not None and (k, r) not in kept and len(kept) < 48:
                kept[(k, r)] = lv.cpu().numpy()

    ths = [threading.Thread(target=collect, args=(k,)) for k in range(len(graphs))]
    for th in ths:
        th.start()
    nsub = 0
    t0 = time.perf_counter()
    for a_t, k, q in zip(arrivals, which, pick):
        now = time.perf_counter() - t0
        if a_t > now:
            time.sleep(a_t - now)
        gid, n, _, _, rts, _ = graphs[k]
        tqs[k].put((srv.submit(gid, int(rts[q])), int(rts[q])))
        nsub += 1
    for tq in tqs:
        tq.put(None)
    for th in ths:
        th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    # results of the small graphs against the oracle
    checked = exact = 0
    csrs = {}
    for (k, r), lv in kept.items():
        if k not in csrs:
            csrs[k] = oracle.csr(graphs[k][1], *graphs[k][5])
        exact += int(bool((lv == oracle.bfs_levels(csrs[k], r)).all()))
        checked += 1
    return {"metric": f"serving: p50/p99 query latency and aggregate GTEPS (Poisson {rate:,.0f} queries/s)",
            "value": round(sum(edges) / wall / 1e9, 3), "unit": "GTEPS", "n_gpus": 1, "higher_is_better": True,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "kronecker-s16..s22,s24-serving", "graphs": len(graphs), "rate_per_s": rate,
                       "seconds": args.serve_seconds, "queries": nsub, "lanes_per_graph": 64,
                       "client": "one thread per graph collects its results as they finish"},
            "latency_us": {"p50": st["p50_us"], "p99": st["p99_us"], "max": st["max_us"]},
            "server": {"completed": st["completed"] - base["completed"], "rejected": st["rejected"],
                       "iterations": st["iterations"], "peak_lanes": st["peak_lanes"],
                       "hbm_used_bytes": st["hbm_used_bytes"]},
            "validation": {"results_equal_to_oracle": exact, "checked": checked},
            "wall_s": round(wall, 3)}


if __name__ == "__main__":
    main()
