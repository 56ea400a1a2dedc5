"""Autotuner host logic (no GPU): coordinate search and the JSON cache."""
import json

import pytest

import paper_2607_17106_gb300 as bg
from paper_2607_17106_gb300 import build as bgbuild
from paper_2607_17106_gb300 import tune


@pytest.fixture(scope="module", autouse=True)
def _lib():
    bgbuild.build()
    bg.load()


def test_coordinate_search_finds_the_separable_minimum(monkeypatch):
    best = {"chunk": 256, "medium": 16, "alpha": 24.0}  # every knob off its library default

    def fake_time(g, sources, opt, batch, reps=3):
        t = 100.0
        t += 10.0 * (opt.chunk != best["chunk"])
        t += 5.0 * (opt.medium != best["medium"])
        t += 3.0 * (opt.alpha != best["alpha"])
        return t

    monkeypatch.setattr(tune, "time_candidate", fake_time)
    space = {"chunk": [128, 256, 1024], "medium": [16, 32, 64], "alpha": [8.0, 14.0, 24.0]}
    found, t, trials = tune.coordinate_search(None, [0], space, batch=False, rounds=3)
    assert found == best and t == 100.0
    assert len(trials) >= 1 + 2 + 2 + 2


def test_coordinate_search_skips_rejected_combinations(monkeypatch):
    # the CUDA-graph drive rejects the filter forms: never time that pair
    def fake_time(g, sources, opt, batch, reps=3):
        assert not (opt.mode == bg.BFS_MODE_GRAPH and opt.push_filter != bg.BFS_PUSH_FUSED)
        return 100.0 - 20.0 * (opt.mode == bg.BFS_MODE_GRAPH) - 10.0 * (opt.push_filter == bg.BFS_PUSH_FILTER)

    monkeypatch.setattr(tune, "time_candidate", fake_time)
    space = {"mode": [bg.BFS_MODE_PERSISTENT, bg.BFS_MODE_GRAPH], "push_filter": tune.SINGLE_SPACE["push_filter"]}
    found, t, _ = tune.coordinate_search(None, [0], space, batch=False, rounds=3)
    assert found == {"mode": bg.BFS_MODE_GRAPH} and t == 80.0
    assert tune.valid_candidate({"push_filter": bg.BFS_PUSH_FILTER})
    assert not tune.valid_candidate({"mode": bg.BFS_MODE_GRAPH, "push_filter": bg.BFS_PUSH_FILTER_PREDICATED})
    assert tune.valid_candidate({"frontier_sort": bg.BFS_SORT_DEVICE})
    assert not tune.valid_candidate({"mode": bg.BFS_MODE_GRAPH, "frontier_sort": bg.BFS_SORT_TILE})


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "device_key", lambda: {"gpu": "TestGPU", "sms": 152})
    path = tmp_path / "cache.json"
    key = tune.graph_key("rmat", 1 << 22, 128312596) + "|single"
    path.write_text(json.dumps({key: {"options": {"chunk": 1024, "pull_serial": 8}, "us": 1.0}}))
    o = tune.tuned_options("rmat", 1 << 22, 128312596, path=str(path))
    assert o.chunk == 1024 and o.pull_serial == 8 and o.batch == 0
    o2 = tune.tuned_options("er", 1 << 22, 67108864, path=str(path))
    assert o2.chunk == bg.options().chunk  # no entry: library defaults
