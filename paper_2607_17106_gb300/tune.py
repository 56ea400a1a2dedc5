"""Autotuner for the BFS launch and load-balance parameters.

Sweeps, on a given graph and seeded sources, the knobs of `bfs_options` that
change only the schedule (never the result): drive mode, CTA size, chunk-unit
size, warp threshold, pull flatten width, claim aggregation, the push
advance / visited-update arrangement (fused, or an edge frontier claimed by a
filter pass: Variants 13/14 and 20/23 of Section 7.2), the frontier order of
push-queue levels (claim order, or sorted device-wide or per tile: Variants 6
and 7), and the direction
thresholds alpha / beta / gamma; for batched (64-lane) searches the MS-BFS
knobs.  Each candidate's mean device time per search is measured with
CUDA events after warm-up; the best is stored in a JSON cache keyed by
(GPU name, SM count, graph class, log2 n, log2 m) and returned by
`tuned_options`.

Usage: python -m paper_2607_17106_gb300.tune --workload rmat-s22-ef16
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os
import sys

import numpy as np

from . import (BFS_MODE_GRAPH, BFS_MODE_PERSISTENT, BFS_PUSH_FILTER, BFS_PUSH_FILTER_PREDICATED, BFS_PUSH_FUSED,
               BFS_SMALL_AUTO, BFS_SMALL_CLUSTER, BFS_SMALL_OFF, BFS_SORT_DEVICE, BFS_SORT_NONE, BFS_SORT_TILE, Graph,
               options)

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(_HERE, "tune_cache.json")

SINGLE_SPACE = {
    "mode": [BFS_MODE_PERSISTENT, BFS_MODE_GRAPH],
    "block_threads": [256, 512, 1024],
    "chunk": [128, 256, 1024],
    "medium": [16, 32, 64],
    "pull_serial": [8, 16, 32],
    "claim_aggregate": [0, 1],
    "push_filter": [BFS_PUSH_FUSED, BFS_PUSH_FILTER, BFS_PUSH_FILTER_PREDICATED],
    "frontier_sort": [BFS_SORT_NONE, BFS_SORT_DEVICE, BFS_SORT_TILE],
    "small_levels": [BFS_SMALL_AUTO, BFS_SMALL_OFF, BFS_SMALL_CLUSTER],
    "alpha": [8.0, 14.0, 24.0],
    "beta": [12.0, 24.0, 48.0],
    "gamma": [8.0, 16.0, 64.0],
}

BATCH_SPACE = {
    "chunk": [128, 256, 1024],
    "medium": [16, 32],
    "pull_serial": [16, 32, 64],
    "batch_alpha": [2.0, 4.0, 8.0, 14.0, 64.0],
    "batch_beta": [24.0, 48.0],
}


def device_key() -> dict:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return {"gpu": p.name, "sms": p.multi_processor_count}


def graph_key(kind: str, n: int, m: int) -> str:
    d = device_key()
    return f"{d['gpu']}|{d['sms']}|{kind}|{int(round(math.log2(max(n, 1))))}|{int(round(math.log2(max(m, 1))))}"


def time_candidate(g: Graph, sources, opt, batch: bool, reps: int = 3) -> float:
    """Mean device microseconds per search (per 64-lane launch when batch)."""
    import torch
    n = g.n
    k = len(sources) if batch else 1
    depth = torch.empty((k, n), dtype=torch.int32, device="cuda")
    parent = torch.empty((k, n), dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()

    def once():
        if batch:
            g.run(np.asarray(sources, np.int32), depth, parent, opt)
        else:
            for s in sources:
                g.run(np.array([s], np.int32), depth[0], parent[0], opt)

    once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        once()
    e1.record(st)
    torch.cuda.synchronize()
    g.sync()
    per = reps * (1 if batch else len(sources))
    return e0.elapsed_time(e1) * 1e3 / per


def time_mixed(graphs, goq, srcs, depth, parent, opt, reps: int = 3) -> float:
    """Device microseconds of one bfs_run_mixed launch over the whole batch."""
    import torch
    from . import run_mixed
    st = torch.cuda.current_stream()
    run_mixed(graphs, goq, srcs, depth, parent, opt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        run_mixed(graphs, goq, srcs, depth, parent, opt)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / reps


def valid_candidate(cand: dict) -> bool:
    """Combinations the library accepts: the filter forms and the frontier sorts
    need the persistent or host-loop drive."""
    if cand.get("mode") != BFS_MODE_GRAPH:
        return True
    return cand.get("push_filter", BFS_PUSH_FUSED) == BFS_PUSH_FUSED and cand.get("frontier_sort", BFS_SORT_NONE) == BFS_SORT_NONE


def coordinate_search(g: Graph, sources, space: dict, batch: bool, rounds: int = 2, verbose=False, timer=None):
    """Coordinate descent over `space` from the library defaults (each knob in
    turn).  timer(opt) -> us replaces the per-search timing when given."""
    best = {}
    base = options(batch=1 if batch else 0)
    if timer is None:
        timer = lambda o: time_candidate(g, sources, o, batch)  # noqa: E731
    best_t = timer(base)
    trials = [({}, best_t)]
    for _ in range(rounds):
        improved = False
        for knob, values in space.items():
            for v in values:
                cand = dict(best)
                cand[knob] = v
                if cand == best or not valid_candidate(cand):
                    continue
                t = timer(options(batch=1 if batch else 0, **cand))
                trials.append((cand, t))
                if verbose:
                    print(f"  {cand}: {t:.1f} us", flush=True)
                if t < best_t * 0.99:
                    best, best_t, improved = cand, t, True
        if not improved:
            break
    return best, best_t, trials


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


MIXED_KEY = "mixed-rmat16-22-q256"


def tuned_options(kind: str, n: int, m: int, batch: bool = False, path: str = DEFAULT_CACHE, **extra):
    """bfs_options from the cache entry of this graph class (defaults if none).
    kind == MIXED_KEY selects the entry of the mixed multi-graph batch."""
    if kind == MIXED_KEY:
        d = device_key()
        entry = load_cache(path).get(f"{d['gpu']}|{d['sms']}|{MIXED_KEY}")
    else:
        entry = load_cache(path).get(graph_key(kind, n, m) + ("|batch" if batch else "|single"))
    kw = dict(entry["options"]) if entry else {}
    kw.update(extra)
    kw.setdefault("batch", 1 if batch else 0)
    return options(**kw)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="rmat-s22-ef16")
    ap.add_argument("--sources", type=int, default=8)
    ap.add_argument("--batch", action="store_true", help="tune 64-lane batched searches")
    ap.add_argument("--cache", default=DEFAULT_CACHE)
    ap.add_argument("--rounds", type=int, default=2)
    ap.add_argument("--mixed", action="store_true", help="tune the mixed batch of 256 queries over RMAT 16-22 "
                                                          "(one bfs_run_mixed launch)")
    args = ap.parse_args(argv)
    root = os.path.dirname(_HERE)
    if root not in sys.path:
        sys.path.insert(0, root)
    import graphgen
    from .build import build
    build()
    if args.mixed:
        return _tune_mixed(args, graphgen)
    w = graphgen.WORKLOADS[args.workload]
    n, src, dst = w.edges()
    g = Graph.build(n, src, dst)
    k = 64 if args.batch else args.sources
    sources = graphgen.sample_sources(n, src, dst, k, w.source_seed + 555)
    space = BATCH_SPACE if args.batch else SINGLE_SPACE
    best, best_t, trials = coordinate_search(g, sources, space, args.batch, args.rounds, verbose=True)
    default_t = trials[0][1]
    cache = load_cache(args.cache)
    key = graph_key(w.kind, n, g.m) + ("|batch" if args.batch else "|single")
    cache[key] = {"options": best, "us": best_t, "default_us": default_t, "workload": w.name,
                  "trials": len(trials)}
    with open(args.cache, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    print(json.dumps({"key": key, "best": best, "us": best_t, "default_us": default_t,
                      "speedup": default_t / best_t}))
    return 0


def _tune_mixed(args, graphgen):
    import torch
    scales, edge_lists, goq, srcs = graphgen.mixed_batch()
    graphs = [Graph.build(n, s, d) for n, s, d in edge_lists]
    ns = [n for n, _, _ in edge_lists]
    depth = [torch.empty(ns[gi], dtype=torch.int32, device="cuda") for gi in goq]
    parent = [torch.empty(ns[gi], dtype=torch.int32, device="cuda") for gi in goq]
    timer = lambda o: time_mixed(graphs, goq, srcs, depth, parent, o)  # noqa: E731
    best, best_t, trials = coordinate_search(None, None, BATCH_SPACE, True, args.rounds, verbose=True, timer=timer)
    default_t = trials[0][1]
    cache = load_cache(args.cache)
    d = device_key()
    key = f"{d['gpu']}|{d['sms']}|{MIXED_KEY}"
    cache[key] = {"options": best, "us": best_t, "default_us": default_t, "workload": MIXED_KEY,
                  "trials": len(trials)}
    with open(args.cache, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    print(json.dumps({"key": key, "best": best, "us": best_t, "default_us": default_t,
                      "speedup": default_t / best_t}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
