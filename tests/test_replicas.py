"""Replicas-only multi-GPU path, host side, on CPU: two gloo ranks.

Every rank searches its own seeded sources on a replica of the graph, with
no exchange on the data path; the bench reports the edges all ranks traversed
over the slowest rank's time, and only rank 0 prints or runs the reference
arm.  These tests run the reductions and the rank rules with world size 2.
"""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import graphgen  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        n, s, d = graphgen.rmat(10, 8, seed=2)
        srcs = graphgen.sample_sources(n, s, d, 16, bench.rank_source_seed(102, rank))
        edges, secs = 1000.0 * (rank + 1), 0.5 + rank  # a rank's own work and time
        e, t = bench.replica_totals(dist, edges, secs, "cpu")
        with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
            json.dump({"sources": [int(x) for x in srcs], "edges": e, "secs": t}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_edges_and_take_the_slowest_time(tmp_path):
    ws = 2
    mp.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    r = [json.load(open(tmp_path / f"r{i}.json")) for i in range(ws)]
    for x in r:
        assert x["edges"] == 3000.0  # 1000 + 2000: the job's edges
        assert x["secs"] == 1.5      # the slower rank
    assert r[0]["sources"] != r[1]["sources"]  # each replica searches its own sources


def test_one_process_totals_are_its_own():
    assert bench.replica_totals(None, 123.0, 4.5) == (123.0, 4.5)
    assert bench.rank_source_seed(102, 0) == 102 and bench.rank_source_seed(102, 3) == 3102


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload = "no-such-workload"  # rank 1 must return before touching it
        steps = 1
        warmup = 0

    assert bench.run_reference(Args()) == 0


def test_launch_pairs_counted_where_small_levels_run_in_a_cluster():
    # the bench's launch count follows the library's rule: a launch pair per
    # source for bounded-degree graphs under the persistent drive, else one
    # launch for all the sources of a step
    import types
    import paper_2607_17106_gb300 as bg
    from paper_2607_17106_gb300 import build
    build.build()  # bfs_options_init comes from the library (no GPU needed)
    bg.load()
    o = bg.options(batch=0)
    grid_like, rmat_like = types.SimpleNamespace(deg_max=4), types.SimpleNamespace(deg_max=5000)
    assert bench.small_levels_active(bg, o, grid_like)
    assert not bench.small_levels_active(bg, o, rmat_like)
    assert bench.small_levels_active(bg, bg.options(batch=0, small_levels=bg.BFS_SMALL_CLUSTER), rmat_like)
    assert not bench.small_levels_active(bg, bg.options(batch=0, small_levels=bg.BFS_SMALL_OFF), grid_like)
    assert not bench.small_levels_active(bg, bg.options(batch=0, mode=bg.BFS_MODE_GRAPH), grid_like)
    assert not bench.small_levels_active(bg, bg.options(batch=0, frontier_sort=bg.BFS_SORT_TILE), grid_like)
    assert not bench.small_levels_active(bg, bg.options(batch=0, push_filter=bg.BFS_PUSH_FILTER), grid_like)
