#!/usr/bin/env python3
"""Benchmark: direction-optimising BFS GTEPS on one GB300 (and N replicas).

Workload (default): RMAT scale 22, edge factor 16, a=0.57 b=c=0.19 d=0.05,
symmetrised, self-loops and duplicates removed, int32 CSR; 64 seeded sources
of degree > 0 run one at a time with the plain push/pull direction switch.
A step = the 64 searches.  value = undirected edges in the reached components
summed over the sources / device time (GTEPS).  Also reported: the same 64
sources as one 64-lane MS-BFS launch (batched) and with the learned policy,
an end-to-end figure through the C ABI with host buffers, the roofline of the
BFS kernel, and the CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat-s22-ef16")
    ap.add_argument("--sources", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip batched / learned / ER extras")
    ap.add_argument("--no-rcm", action="store_true", help="skip the Reverse Cuthill-McKee reordered leg")
    ap.add_argument("--profile-batched", type=int, default=0, metavar="R",
                    help="only run R 64-lane batched launches of the workload's sources and exit (for ncu)")
    ap.add_argument("--profile-single", type=int, default=0, metavar="R",
                    help="only run the first R single-source searches of the workload and exit (for ncu); "
                         "the persistent drive runs them in one launch")
    ap.add_argument("--mode", choices=["persistent", "host-loop", "graph"], default="persistent",
                    help="drive of --profile-single: host-loop runs every level as its own launch")
    ap.add_argument("--profile-components", type=int, default=0, metavar="R",
                    help="only run R connected-components launches on the workload's graph and exit (for ncu)")
    ap.add_argument("--levels", action="store_true",
                    help="print a per-level time and byte breakdown of the single-source searches and exit")
    ap.add_argument("--policy-weights", default=os.path.join(ROOT, "paper_2607_17106_gb300", "policy_weights.npy"))
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_source_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's sources: every replica searches its own seeded sources (weak scaling)."""
    return base_seed + 1000 * rank


def replica_totals(dist, edges: float, seconds: float, device="cpu"):
    """Whole-job totals of a replicas-only run: the edges all ranks traversed
    (sum) and the slowest rank's time (max).  dist = None on one process."""
    if dist is None:
        return float(edges), float(seconds)
    import torch
    e = torch.tensor([float(edges)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(e.item()), float(t.item())


def describe(w) -> str:
    p = w.params
    if w.kind == "rmat":
        d = 1 - p["a"] - p["b"] - p["c"]
        return (f"RMAT scale {p['scale']}, edge factor {p['edge_factor']}, a={p['a']} b={p['b']} c={p['c']} "
                f"d={d:.2f}")
    if w.kind == "er":
        return f"Erdos-Renyi n={p['n']}, {p['m_pairs']} pairs (mean degree {2 * p['m_pairs'] / p['n']:.0f})"
    if w.kind == "grid":
        return f"{p['width']}x{p['height']} 4-neighbour grid, {int(100 * p['p_del'])}% edges deleted, relabelled"
    if w.kind == "ba":
        return f"Barabasi-Albert n={p['n']}, m={p['m']}"
    return w.kind


# ------------------------------------------------------------ roofline model
def level_bytes(stats: np.ndarray, n: int):
    """Per-level minimum DRAM bytes of one search, push and pull form.

    From the per-level statistics f, e_f, u, s_u, d_new (Cascade 1; the pull
    form of Section 5 reads s_u entries with early exit):
      push: queue 4f + row offsets 8f + columns 4e_f + depth/parent writes
            8d_new + next queue 4d_new + visited bitmap read and next bitmap
            written once each n/4
      pull: visited n/8 + row offsets 8u + scanned columns 4s_u + frontier
            n/8 + depth/parent writes 8d_new + next bitmap n/8
    """
    f, e_f, u, s_u, d_new, e_u = (stats[:, i].astype(np.float64) for i in range(6))
    push = 12 * f + 4 * e_f + 12 * d_new + n / 4
    pull = 3 * n / 8 + 8 * u + 4 * s_u + 8 * d_new
    return push, pull


def bytes_model(stats: np.ndarray, n: int):
    """B_min of one search: the cheaper form's bytes summed over its levels."""
    push, pull = level_bytes(stats, n)
    return float(np.minimum(push, pull).sum())


def rcm_leg(bg, torch, n, src, dst, sources, depth, parent, depth_h, stream, edges, plain_ms, batched_ms,
            extra_flags=0):
    """The paper's preprocessing (Section 7.1): the same graph renumbered in Reverse
    Cuthill-McKee order, the same sources under the renaming; plain (one source at
    a time) and batched device times, and the depths mapped back."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gr = bg.Graph.build(n, src, dst, flags=bg.BFS_DEFAULT_FLAGS | bg.BFS_REORDER_RCM | extra_flags)
    build_s = time.perf_counter() - t0
    newid = gr.permutation()
    rs = newid[np.asarray(sources)].astype(np.int32)
    k = len(rs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    single = bg.options(batch=0)
    batched = bg.options(batch=1)

    def plain():
        for j in range(k):
            gr.run(rs[j:j + 1], depth[j], parent[j], single)

    plain()
    torch.cuda.synchronize()
    e0.record(stream)
    plain()
    e1.record(stream)
    torch.cuda.synchronize()
    gr.sync()
    pms = e0.elapsed_time(e1)
    same = bool(np.array_equal(depth.cpu().numpy()[:, newid], depth_h))
    gr.run(rs, depth, parent, batched)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        gr.run(rs, depth, parent, batched)
    e1.record(stream)
    torch.cuda.synchronize()
    gr.sync()
    bms = e0.elapsed_time(e1) / 3
    same = same and bool(np.array_equal(depth.cpu().numpy()[:, newid], depth_h))
    gr.free()
    return {"build_s_with_reorder": build_s, "plain_gteps": edges / (pms * 1e-3) / 1e9, "plain_ms_per_step": pms,
            "plain_speedup_vs_input_order": plain_ms / pms, "batched_gteps": edges / (bms * 1e-3) / 1e9,
            "batched_ms_per_step": bms, "batched_speedup_vs_input_order": batched_ms / bms,
            "depth_equal_under_renaming": same}


def small_levels_active(bg, opt, info) -> bool:
    """Whether bfs_run drives each source's small levels in a thread-block
    cluster (a launch pair per source) under these options: the library's
    rule for the persistent drive (fused claiming, no frontier sort; the
    automatic choice for maximum degree <= 16)."""
    if opt.mode != bg.BFS_MODE_PERSISTENT or opt.frontier_sort != bg.BFS_SORT_NONE or opt.push_filter != bg.BFS_PUSH_FUSED:
        return False
    return opt.small_levels == bg.BFS_SMALL_CLUSTER or (opt.small_levels == bg.BFS_SMALL_AUTO and info.deg_max <= 16)


def teps_edges(stats: np.ndarray) -> float:
    """Undirected edges with both ends reached = (sum of degrees over reached vertices) / 2."""
    return float(stats[:, 1].sum()) / 2.0


# ------------------------------------------------------------ clock sampling
class ClockSampler:
    def __init__(self, device_index: int):
        self.idx = device_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi takes a moment to start: open the timed region only once it reports
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self) -> int:
        """Index of the next sample: samples from here on were taken in the timed region."""
        return len(self.samples)

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self, first: int = 0):
        """Summary of the samples from index `first` on (the last one before it if none)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        window = self.samples[first:] or self.samples[-1:]
        for s in window:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
                for nm, val in zip(names, s[4:8]):
                    if val.strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = ["common.cuh", "level.cuh", "policy_dev.cuh", "bfs_single.cu"]


def source_hash() -> str:
    """Hash of the single-source kernel's sources: recorded ncu traffic is valid only for this code."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2607_17106_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per launch of the BFS kernel from the committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(workload)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def measured_peak():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------ CPU baseline
def cpu_baseline(n, src, dst, sources, budget_s=20.0, gpu_depth=None):
    """The oracle as it stands, single-threaded, on a bounded sample of sources."""
    import oracle
    t0 = time.perf_counter()
    adj = oracle.build_adjacency(n, src, dst)
    build_s = time.perf_counter() - t0
    edges = 0.0
    t_bfs = 0.0
    used = 0
    parity = True
    for j, s in enumerate(sources):
        t1 = time.perf_counter()
        depth, parent = oracle.bfs(adj, int(s))
        t_bfs += time.perf_counter() - t1
        deg = np.diff(adj.row_ptr)
        edges += float(deg[depth >= 0].sum()) / 2.0
        if gpu_depth is not None and j < len(gpu_depth):
            parity = parity and bool(np.array_equal(depth, gpu_depth[j]))
        used += 1
        if t_bfs > budget_s:
            break
    return {"value": edges / t_bfs / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{used} of the workload's sources, FIFO queue BFS (adjacency build {build_s:.1f}s untimed)",
            "parity_on_sample": parity}


# ------------------------------------------------------------ reference arm
METRIC = "BFS GTEPS, plain single-source push/pull direction-optimising (batched+learned reported beside)"
METRIC_MIXED = "BFS GTEPS, mixed batch of 256 queries over RMAT scales 16-22 in one persistent launch"


def workload_desc(w, n: int, m: int) -> str:
    return f"{w.name}: {describe(w)}, symmetrised+dedup, n={n}, m={m} directed"


def mixed_queries():
    return graphgen.mixed_batch()


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    import oracle
    if args.workload == MIXED:  # one query of the batch per step, in query order
        scales, graphs, goq, srcs = mixed_queries()
        adjs = {}
        metric, wdesc = METRIC_MIXED, MIXED + ": 256 queries over RMAT scales 16..22; one query per step"
    else:
        w = graphgen.WORKLOADS[args.workload]
        n, src, dst = w.edges()
        sources = w.sources(n, src, dst)
        adj = oracle.build_adjacency(n, src, dst)
        metric, wdesc = METRIC, workload_desc(w, n, adj.m) + "; one of its seeded sources per step"
    times, edges = [], []
    for step in range(args.warmup + args.steps):
        if args.workload == MIXED:
            q = step % len(srcs)
            gi = int(goq[q])
            if gi not in adjs:
                adjs[gi] = oracle.build_adjacency(*graphs[gi])
            a, s = adjs[gi], int(srcs[q])
        else:
            a, s = adj, int(sources[step % len(sources)])
        t0 = time.perf_counter()
        depth, _ = oracle.bfs(a, s)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            edges.append(float(np.diff(a.row_ptr)[depth >= 0].sum()) / 2.0)
    value = sum(edges) / sum(times) / 1e9
    line = {"impl": "reference", "metric": metric, "value": value,
            "unit": "GTEPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": wdesc, "engine": "CPU oracle (FIFO queue BFS), single thread"},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} single-source searches"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ mixed batch
MIXED = "mixed-rmat16-22-q256"


def run_mixed_bench(args, bg, torch, dist=None, rank=0, ws=1):
    """256 queries over RMAT graphs of scales 16..22 (edge factor 16, seeds 16..22),
    the graph of each query drawn uniformly (seed 106): one bfs_run_mixed launch
    against the same queries as per-graph 64-lane batches and one at a time."""
    scales, edge_lists, goq, srcs = mixed_queries()
    graphs = [(n, bg.Graph.build(n, s, d)) for n, s, d in edge_lists]
    q = len(srcs)
    depth = [torch.empty(graphs[gi][0], dtype=torch.int32, device="cuda") for gi in goq]
    parent = [torch.empty(graphs[gi][0], dtype=torch.int32, device="cuda") for gi in goq]
    gl = [g for _, g in graphs]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def mixed_once():
        bg.run_mixed(gl, goq, srcs, depth, parent, bg.options())

    for _ in range(args.warmup):
        mixed_once()
    torch.cuda.synchronize()
    ref = [dd.cpu().numpy() for dd in depth]
    edges = 0.0
    for i, gi in enumerate(goq):
        st = gl[gi].level_stats(depth[i])
        edges += teps_edges(st)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        mixed_once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_mixed = e0.elapsed_time(e1) / args.steps
    # replicas: every rank runs the same 256 queries
    job_edges, ms_mixed = replica_totals(dist, edges, ms_mixed, "cuda")
    ok = all(np.array_equal(depth[i].cpu().numpy(), ref[i]) for i in range(q))
    # the same queries per graph as ordinary 64-lane batches, and one at a time
    e0.record(stream)
    for gi in range(len(scales)):
        idx = np.flatnonzero(goq == gi)
        n = graphs[gi][0]
        for c0 in range(0, len(idx), 64):
            part = idx[c0:c0 + 64]
            dd = torch.empty((len(part), n), dtype=torch.int32, device="cuda")
            gl[gi].run(srcs[part], dd, None, bg.options())
    e1.record(stream)
    torch.cuda.synchronize()
    ms_per_graph = e0.elapsed_time(e1)
    e0.record(stream)
    for i, gi in enumerate(goq):
        gl[gi].run(np.array([srcs[i]], np.int32), depth[i], parent[i], bg.options(batch=0))
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    tuned = None
    try:
        from paper_2607_17106_gb300 import tune
        ot = tune.tuned_options(tune.MIXED_KEY, 0, 0)
        bg.run_mixed(gl, goq, srcs, depth, parent, ot)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            bg.run_mixed(gl, goq, srcs, depth, parent, ot)
        e1.record(stream)
        torch.cuda.synchronize()
        tms = e0.elapsed_time(e1) / args.steps
        tuned = {"ms": tms, "gteps": edges / (tms * 1e-3) / 1e9, "speedup_vs_default": ms_mixed / tms,
                 "depth_repeatable": all(np.array_equal(depth[i].cpu().numpy(), ref[i]) for i in range(q)),
                 "options": {f: getattr(ot, f) for f in tune.BATCH_SPACE}}
    except Exception as exc:
        tuned = {"skipped": str(exc)[:120]}
    if rank != 0:
        return 0
    line = {"metric": METRIC_MIXED,
            "value": job_edges / (ms_mixed * 1e-3) / 1e9, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": MIXED + ": 256 queries, graph of each uniform over RMAT scales 16..22 (edge "
                                          "factor 16, a=0.57 b=c=0.19, seeds 16..22)", "edges_per_step": edges},
            "gpu_launches": args.steps, "depth_repeatable": ok,
            "per_graph_batches": {"ms": ms_per_graph, "gteps": edges / (ms_per_graph * 1e-3) / 1e9},
            "tuned": tuned,
            "one_at_a_time": {"ms": ms_single, "gteps": edges / (ms_single * 1e-3) / 1e9}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ per-level breakdown
DIR_NAMES = {0: "push-queue", 1: "push-bitmap", 2: "pull"}


def level_breakdown(args, bg, torch, g, w, n, sources, opt):
    """Per-level durations (device %globaltimer stamps of the level log) beside
    each level's minimum bytes, push and pull, for the single-source searches.
    Printed as markdown tables; levels are aggregated by index (short searches)
    and by form and frontier size."""
    k = len(sources)
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    cap = min(n + 2, 1 << 16)
    log = (bg.bfs_level_record * cap)()
    nlev = bg.ctypes.c_int32(0)
    o = bg.options(**{f: getattr(opt, f) for f in ("batch", "mode", "policy", "alpha", "beta", "gamma", "chunk",
                                                   "medium", "pull_serial", "block_threads")})
    o.level_log = bg.ctypes.cast(log, bg.ctypes.POINTER(bg.bfs_level_record))
    o.level_log_cap = cap
    o.levels_out = bg.ctypes.pointer(nlev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    rows = []       # (level, dir, f, e_f, u, s_u, d_new, us, push_B, pull_B)
    searches = []   # (levels, log µs, event µs)
    for _ in range(max(1, args.warmup)):
        g.run(np.array([sources[0]], np.int32), depth, parent, bg.options(batch=0))
    torch.cuda.synchronize()
    for j in range(k):
        e0.record(stream)
        g.run(np.array([sources[j]], np.int32), depth, parent, bg.options(batch=0))
        e1.record(stream)
        torch.cuda.synchronize()
        ev_us = e0.elapsed_time(e1) * 1e3
        g.run(np.array([sources[j]], np.int32), depth, parent, o)  # synchronises (level log)
        L = nlev.value
        st = g.level_stats(depth)
        if L + 1 > cap or log[L].dir != -1 or len(st) != L:
            raise RuntimeError(f"level log of source {j} incomplete ({L} levels, {len(st)} in the statistics)")
        push, pull = level_bytes(st, n)
        t = [log[i].t_ns for i in range(L + 1)]
        for i in range(L):
            rows.append((i, log[i].dir, *st[i, :5].tolist(), (t[i + 1] - t[i]) / 1e3, push[i], pull[i]))
        searches.append((L, (t[L] - t[0]) / 1e3, ev_us))
    R = np.array(rows, dtype=np.float64)
    out = [f"## Per-level breakdown: {w.name}, {k} sources one at a time (block_threads {opt.block_threads})", "",
           f"searches: mean {np.mean([x[0] for x in searches]):.1f} levels; mean time from the first level's "
           f"start to the closing record {np.mean([x[1] for x in searches]):.1f} us; mean event-timed launch "
           f"{np.mean([x[2] for x in searches]):.1f} us", ""]
    bmin = np.minimum(R[:, 8], R[:, 9])
    if int(R[:, 0].max()) < 40:
        out += ["| level | searches | forms taken | mean f | mean e_f | mean u | mean s_u | mean d_new | mean us | "
                "B_push MB | B_pull MB | B_min MB | GB/s at B_min |", "|" + "---|" * 13]
        for lv in range(int(R[:, 0].max()) + 1):
            sel = R[:, 0] == lv
            dirs = ", ".join(f"{DIR_NAMES[d]} {int((R[sel, 1] == d).sum())}" for d in (0, 1, 2) if (R[sel, 1] == d).any())
            us = R[sel, 7].mean()
            out.append(f"| {lv} | {int(sel.sum())} | {dirs} | {R[sel, 2].mean():.0f} | {R[sel, 3].mean():.0f} | "
                       f"{R[sel, 4].mean():.0f} | {R[sel, 5].mean():.0f} | {R[sel, 6].mean():.0f} | {us:.1f} | "
                       f"{R[sel, 8].mean() / 1e6:.2f} | {R[sel, 9].mean() / 1e6:.2f} | {bmin[sel].mean() / 1e6:.2f} | "
                       f"{bmin[sel].mean() / (us * 1e-6) / 1e9:.0f} |")
        out.append("")
    out += ["| form | frontier f | levels | total us (all searches) | mean us per level | B_min MB per level | "
            "GB/s at B_min |", "|---|---|---|---|---|---|---|"]
    lg = np.floor(np.log2(np.maximum(R[:, 2], 1)) / 4).astype(int)
    for d in (0, 1, 2):
        for b in sorted(set(lg[R[:, 1] == d].tolist())):
            sel = (R[:, 1] == d) & (lg == b)
            us = R[sel, 7].sum()
            out.append(f"| {DIR_NAMES[d]} | [{16 ** b}, {16 ** (b + 1)}) | {int(sel.sum())} | {us:.0f} | "
                       f"{us / sel.sum():.2f} | {bmin[sel].mean() / 1e6:.3f} | {bmin[sel].sum() / (us * 1e-6) / 1e9:.0f} |")
    print("\n".join(out))
    return 0


# ------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_2607_17106_gb300 as bg
    from paper_2607_17106_gb300 import build as bgbuild

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    bgbuild.build()
    bg.load()
    stream = torch.cuda.current_stream()
    if args.workload == MIXED:
        rc = run_mixed_bench(args, bg, torch, dist, rank, ws)
        if dist:
            dist.destroy_process_group()
        return rc

    w = graphgen.WORKLOADS[args.workload]
    n, src, dst = w.edges()
    # weak scaling: every rank searches its own 64 seeded sources on a replica
    sources = graphgen.sample_sources(n, src, dst, args.sources, rank_source_seed(w.source_seed, rank))
    g = bg.Graph.build(n, src, dst)
    info = g.info()
    k = len(sources)
    depth = torch.empty((k, n), dtype=torch.int32, device="cuda")
    parent = torch.empty((k, n), dtype=torch.int32, device="cuda")
    opt = bg.options(batch=0)
    if args.levels:
        return level_breakdown(args, bg, torch, g, w, n, sources, opt)
    if args.profile_components > 0:
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        for _ in range(args.profile_components):
            g.components(lab)
        print(json.dumps({"profile_components": args.profile_components, "workload": w.name}))
        return 0
    if args.profile_single > 0:
        mode = {"persistent": bg.BFS_MODE_PERSISTENT, "host-loop": bg.BFS_MODE_HOST_LOOP,
                "graph": bg.BFS_MODE_GRAPH}[args.mode]
        r = min(args.profile_single, k)
        if mode == bg.BFS_MODE_PERSISTENT:  # the r searches in one launch, as the timed step runs them
            g.run(sources[:r], depth[:r], parent[:r], bg.options(batch=0, mode=mode))
        else:
            for j in range(r):
                g.run(sources[j:j + 1], depth[j], parent[j], bg.options(batch=0, mode=mode))
        g.sync()
        torch.cuda.synchronize()
        print(json.dumps({"profile_single": args.profile_single, "mode": args.mode, "workload": w.name}))
        return 0
    if args.profile_batched > 0:
        for _ in range(args.profile_batched):
            g.run(sources, depth, parent, bg.options(batch=1))
        g.sync()
        torch.cuda.synchronize()
        print(json.dumps({"profile_batched": args.profile_batched, "workload": w.name, "sources": k}))
        return 0

    def plain_step(events=None):
        """The k searches one after another: one bfs_run call, which runs them
        in one persistent launch (a barrier between searches)."""
        if events is not None:
            events[0].record(stream)
        g.run(sources, depth, parent, opt)
        if events is not None:
            events[1].record(stream)

    for _ in range(args.warmup):
        plain_step()
    g.sync()
    torch.cuda.synchronize()

    # per-source work (from the finished search) for TEPS and the roofline
    depth_h = depth.cpu().numpy()
    stats = [g.level_stats(depth[j]) for j in range(k)]
    edges = sum(teps_edges(s) for s in stats)
    bmin = [bytes_model(s, n) for s in stats]

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ev = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    first_sample = clocks.mark()
    t_start.record(stream)
    for s in range(args.steps):
        plain_step(ev[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop(first_sample)
    g.sync()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [ev[s][0].elapsed_time(ev[s][1]) for s in range(args.steps)]
    # every rank searched its own sources: the job's edges over the slowest rank's time
    job_edges, total_ms = replica_totals(dist, edges, total_ms, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_edges / (ms_per_step * 1e-3) / 1e9

    peak, peak_kind = measured_peak()
    mean_launch_s = float(np.mean(launch_ms)) * 1e-3
    step_bmin = float(np.sum(bmin))  # the k searches of one launch
    achieved = step_bmin / mean_launch_s / 1e9
    # Graph500-style per-search TEPS, untimed pass: each search in a launch of
    # its own, its edges over its own event-timed launch; searches that reach
    # fewer than 1000 edges (a source in a tiny component) are reported apart,
    # since their launch time is mostly the fixed cost of a launch
    ev1 = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(k)]
    for j in range(k):
        ev1[j][0].record(stream)
        g.run(sources[j:j + 1], depth[j], parent[j], opt)
        ev1[j][1].record(stream)
    torch.cuda.synchronize()
    one_ms = np.array([ev1[j][0].elapsed_time(ev1[j][1]) for j in range(k)])
    big = np.array([teps_edges(stats[j]) >= 1000 for j in range(k)])
    per_src = np.array([teps_edges(stats[j]) for j in range(k)]) / (one_ms * 1e-3) / 1e9
    ps = per_src[big]
    teps_stats = {"median_gteps": float(np.median(ps)),
                  "harmonic_mean_gteps": float(len(ps) / np.sum(1.0 / np.maximum(ps, 1e-12))),
                  "min_gteps": float(ps.min()), "max_gteps": float(ps.max()), "searches": int(len(ps)),
                  "excluded_tiny_components": int((~big).sum()),
                  "us_per_search_one_launch_each": float(one_ms.mean() * 1e3),
                  "timer": "one launch per search (untimed pass); searches reaching < 1000 edges excluded"}
    small = small_levels_active(bg, opt, info)
    launches_per_step = 2 * k if small else 1
    kernel = ("bfs1_kernel (per source: a one-cluster launch for the small levels, then the grid-wide launch; "
              "figures per step of k searches)" if small else
              "bfs1_kernel (persistent; one launch runs the k searches in turn)")
    roof = {"bound": "hbm", "kernel": kernel,
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
            "frac_of_nominal_8TBs": achieved / NOMINAL_HBM_GBS, "bytes_per_launch": step_bmin / launches_per_step,
            "bytes_per_step": step_bmin, "searches_per_step": k, "launches_per_step": launches_per_step,
            "launch_us": mean_launch_s * 1e6 / launches_per_step, "step_us": mean_launch_s * 1e6,
            "us_per_search": mean_launch_s * 1e6 / k,
            "traffic": None if small else recorded_traffic(w.name)}

    extra = {}
    if not args.no_extra:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def time_batched(o, reps=3):
            """ms per launch of the k sources as 64-lane MS-BFS batches (device time)."""
            g.run(sources, depth, parent, o)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                g.run(sources, depth, parent, o)
            e1.record(stream)
            torch.cuda.synchronize()
            g.sync()
            return e0.elapsed_time(e1) / reps

        def time_single(o, count=None):
            """ms for the first `count` sources one at a time (device time)."""
            js = range(k if count is None else min(count, k))
            for j in js:
                g.run(np.array([sources[j]], np.int32), depth[j], parent[j], o)
            torch.cuda.synchronize()
            e0.record(stream)
            for j in js:
                g.run(np.array([sources[j]], np.int32), depth[j], parent[j], o)
            e1.record(stream)
            torch.cuda.synchronize()
            g.sync()
            return e0.elapsed_time(e1), len(js)

        def same_depths():
            return bool(np.array_equal(depth.cpu().numpy(), depth_h))

        bms = time_batched(bg.options(batch=1))
        # the same searches' minimum bytes (sum of B_min over the k sources)
        # over the batched time: the roofline fraction of the batched form
        extra["batched_msbfs"] = {"gteps": edges / (bms * 1e-3) / 1e9, "ms_per_step": bms,
                                  "speedup_vs_plain": ms_per_step / bms, "depth_equal_to_plain": same_depths(),
                                  "roofline_frac": float(np.sum(bmin)) / (bms * 1e-3) / 1e9 / peak}
        try:
            from paper_2607_17106_gb300 import tune
            ot = tune.tuned_options(w.kind, n, info.m, batch=True)
            tms = time_batched(ot)
            extra["batched_tuned"] = {"gteps": edges / (tms * 1e-3) / 1e9, "ms_per_step": tms,
                                      "speedup_vs_plain": ms_per_step / tms, "depth_equal_to_plain": same_depths(),
                                      "options": {f: getattr(ot, f) for f in ("chunk", "medium", "pull_serial",
                                                                              "batch_alpha", "batch_beta")}}
        except Exception as exc:  # no cache entry for this device/graph class
            extra["batched_tuned"] = {"skipped": str(exc)[:120]}
        try:
            from paper_2607_17106_gb300 import tune
            ots = tune.tuned_options(w.kind, n, info.m, batch=False)
            dms, _ = time_single(bg.options(batch=0))
            tms, _ = time_single(ots)
            extra["single_tuned"] = {"ms_per_step": tms, "default_ms_same_timer": dms, "speedup_vs_default": dms / tms,
                                     "depth_equal_to_plain": same_depths(),
                                     "options": {f: getattr(ots, f) for f in tune.SINGLE_SPACE}}
        except Exception as exc:
            extra["single_tuned"] = {"skipped": str(exc)[:120]}
        # push advance / visited update arrangements (Variants 13/14 and 20/23
        # against the fused claim), all 64 sources, heuristic directions
        fms, _ = time_single(bg.options(batch=0))
        pv = {"fused_ms_per_step": fms}
        for name, pf in (("filter", bg.BFS_PUSH_FILTER), ("filter_predicated", bg.BFS_PUSH_FILTER_PREDICATED)):
            vms, _ = time_single(bg.options(batch=0, push_filter=pf))
            pv[name] = {"gteps": edges / (vms * 1e-3) / 1e9, "ms_per_step": vms, "speedup_vs_fused": fms / vms,
                        "depth_equal_to_plain": same_depths()}
        extra["push_variants"] = pv
        # frontier order of push-queue levels (Variants 6 and 7 against claim order)
        fsv = {"claim_order_ms_per_step": fms}
        for name, fs in (("device_sort", bg.BFS_SORT_DEVICE), ("tile_sort", bg.BFS_SORT_TILE)):
            vms, _ = time_single(bg.options(batch=0, frontier_sort=fs))
            fsv[name] = {"gteps": edges / (vms * 1e-3) / 1e9, "ms_per_step": vms, "speedup_vs_claim_order": fms / vms,
                         "depth_equal_to_plain": same_depths()}
        extra["frontier_sort"] = fsv
        gms, cnt = time_single(bg.options(batch=0, mode=bg.BFS_MODE_GRAPH), 8)
        pms, _ = time_single(bg.options(batch=0), 8)
        extra["graph_mode_single"] = {"sources": cnt, "ms_graph_mode": gms, "ms_persistent": pms,
                                      "graph_over_persistent": gms / pms}
        if os.path.exists(args.policy_weights):
            pol = bg.Policy(np.load(args.policy_weights))
            lms, _ = time_single(bg.options(batch=0, policy=bg.BFS_POLICY_MLP, mlp=pol))
            hms, _ = time_single(bg.options(batch=0))  # the heuristic on the same timer, for a like-for-like ratio
            extra["learned_single"] = {"gteps": edges / (lms * 1e-3) / 1e9, "ms_per_step": lms,
                                       "speedup_vs_plain": ms_per_step / lms, "heuristic_same_timer_ms": hms,
                                       "speedup_vs_heuristic_same_timer": hms / lms,
                                       "depth_equal_to_plain": same_depths()}
            blms = time_batched(bg.options(batch=1, policy=bg.BFS_POLICY_MLP, mlp=pol))
            extra["batched_learned"] = {"gteps": edges / (blms * 1e-3) / 1e9, "ms_per_step": blms,
                                        "speedup_vs_plain": ms_per_step / blms, "depth_equal_to_plain": same_depths(),
                                        "roofline_frac": float(np.sum(bmin)) / (blms * 1e-3) / 1e9 / peak}
        if not args.no_rcm:
            extra["rcm"] = rcm_leg(bg, torch, n, src, dst, sources, depth, parent, depth_h, stream, edges,
                                   ms_per_step, extra["batched_msbfs"]["ms_per_step"])
            # the same with pull rows ordered by degree, highest first
            extra["rcm_hubs_first"] = rcm_leg(bg, torch, n, src, dst, sources, depth, parent, depth_h, stream, edges,
                                              ms_per_step, extra["batched_msbfs"]["ms_per_step"],
                                              extra_flags=bg.BFS_PULL_HUBS_FIRST)

    if not args.no_extra:
        # connected components by min-label propagation on the same graph
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        g.components(lab)
        times, iters = [], 0
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, iters = g.components(lab)  # synchronises
            times.append(time.perf_counter() - t0)
        cms = float(np.median(times)) * 1e3
        extra["components"] = {"ms": cms, "iterations": iters,
                               "gteps": info.m / 2 / (cms * 1e-3) / 1e9,
                               "components": int(torch.unique(lab).numel()),
                               "timer": "host, around the synchronous bfs_components call"}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    src_host = torch.from_numpy(np.asarray(sources, np.int32)).pin_memory()
    depth_host = torch.empty((k, n), dtype=torch.int32).pin_memory()
    parent_host = torch.empty((k, n), dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    # context: a plain device-to-pinned-host copy of the same bytes on this
    # machine (before the runs below fill the host buffers with their results)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    depth_host.copy_(depth, non_blocking=True)
    parent_host.copy_(parent, non_blocking=True)
    torch.cuda.synchronize()
    copy_gbs = 8 * k * n / (time.perf_counter() - t1) / 1e9
    g.run(src_host, depth_host, parent_host, opt)  # untimed: first use of the path
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.run(src_host, depth_host, parent_host, opt)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    job_edges_e2e, e2e_s = replica_totals(dist, edges, e2e_s, "cuda")
    e2e = {"value": job_edges_e2e / e2e_s / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": 4 * k,
           "d2h_bytes_per_step": 8 * k * n, "ms_per_step": e2e_s * 1e3,
           "d2h_copy_gbs_plain": copy_gbs,
           "path": "bfs_run(k=64, host sources, host depth/parent, one source at a time)"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(n, src, dst, sources[:8], budget_s=15.0, gpu_depth=depth_host.numpy()[:8])

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_desc(w, n, info.m) + f"; {k} seeded sources one at a time",
                       "sources_per_step": k, "edges_per_step": edges,
                       "l2": "inputs larger than L2 (CSR col array %d MB)" % (4 * info.m // 2**20),
                       "parallelism": f"replicas x{ws}", "policy": "Beamer alpha=14 beta=48 (batched: alpha=4 beta=48)"},
            "roofline": roof, "per_search": teps_stats, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clk, **extra,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
