"""The autotuner with real GPU timings.

coordinate_search times candidates with CUDA events on the device; whatever it
picks only changes the schedule, so searches run with the chosen options must
still give the oracle's depths bit-exactly and valid parents.  The command-line
entry point writes a cache entry that tuned_options reads back.
"""
import json

import numpy as np
import pytest

import graphgen
import oracle
import paper_2607_17106_gb300 as bg
from paper_2607_17106_gb300 import tune

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat16():
    from paper_2607_17106_gb300 import build
    build.build()
    bg.load()
    n, s, d = graphgen.rmat(16, 16, seed=9)
    g = bg.Graph.build(n, s, d)
    adj = oracle.build_adjacency(n, s, d)
    yield n, s, d, g, adj
    g.free()


def _check_options(g, adj, n, srcs, opt):
    k = len(srcs)
    depth = torch.empty((k, n), dtype=torch.int32, device="cuda")
    parent = torch.empty((k, n), dtype=torch.int32, device="cuda")
    g.run(np.asarray(srcs, np.int32), depth, parent, opt)
    g.sync()
    dd, pp = depth.cpu().numpy(), parent.cpu().numpy()
    for j in range(0, k, max(1, k // 4)):
        ref, _ = oracle.bfs(adj, int(srcs[j]), with_parent=False)
        assert np.array_equal(dd[j], ref), j
        assert oracle.validate(adj, int(srcs[j]), dd[j], pp[j]) == 0, j


def test_single_source_search_with_real_timings(rmat16):
    n, s, d, g, adj = rmat16
    srcs = graphgen.sample_sources(n, s, d, 4, seed=77)
    space = {"chunk": [128, 1024], "pull_serial": [8, 16], "frontier_sort": tune.SINGLE_SPACE["frontier_sort"],
             "push_filter": tune.SINGLE_SPACE["push_filter"], "alpha": [8.0, 14.0]}
    best, t, trials = tune.coordinate_search(g, srcs, space, batch=False, rounds=1)
    assert len(trials) >= 1 + len(space) and all(tt > 0 for _, tt in trials)
    assert t <= trials[0][1]  # never worse than the library defaults as measured
    assert set(best) <= set(space)
    _check_options(g, adj, n, srcs, bg.options(batch=0, **best))


def test_batched_search_with_real_timings(rmat16):
    n, s, d, g, adj = rmat16
    srcs = graphgen.sample_sources(n, s, d, 64, seed=78)
    space = {"pull_serial": [16, 32], "batch_alpha": [4.0, 8.0], "chunk": [256, 1024]}
    best, t, trials = tune.coordinate_search(g, srcs, space, batch=True, rounds=1)
    assert len(trials) >= 4 and t <= trials[0][1]
    _check_options(g, adj, n, srcs, bg.options(batch=1, **best))


def test_command_line_writes_a_cache_entry_that_tuned_options_reads(tmp_path):
    path = tmp_path / "cache.json"
    assert tune.main(["--workload", "rmat-s14-ef16", "--sources", "4", "--rounds", "1", "--cache", str(path)]) == 0
    cache = json.loads(path.read_text())
    (key, entry), = cache.items()
    assert key.endswith("|single") and "|rmat|14|" in key
    assert entry["us"] <= entry["default_us"] and entry["workload"] == "rmat-s14-ef16"
    w = graphgen.WORKLOADS["rmat-s14-ef16"]
    n, s, d = w.edges()
    g = bg.Graph.build(n, s, d)
    opt = tune.tuned_options("rmat", n, g.m, path=str(path))
    for f, v in entry["options"].items():
        assert getattr(opt, f) == pytest.approx(v), f
    _check_options(g, oracle.build_adjacency(n, s, d), n, w.sources(n, s, d), opt)
    g.free()
