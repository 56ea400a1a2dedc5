"""Host logic of the learned direction policy (no GPU): the training-graph
recipe, the regression targets, the cost-weighted resampling, the gate that
mirrors the device rule, and the regret measure."""
import math

import numpy as np
import pytest

from paper_2607_17106_gb300 import policy as pl


def test_training_recipe_is_seeded_and_has_the_stated_mix():
    a = pl.training_specs(200, 16, 22, seed=1000)
    b = pl.training_specs(200, 16, 22, seed=1000)
    assert a == b
    kinds = [s["kind"] for s in a]
    assert kinds.count("rmat") == 120 and kinds.count("er") == 40 and kinds.count("grid") == 40
    for s in a:
        if s["kind"] == "rmat":
            assert 16 <= s["scale"] <= 22 and 0.45 <= s["a"] <= 0.65 and s["edge_factor"] in (8, 16, 32)
            assert math.isclose(s["a"] + s["b"] + s["c"], 0.95) and s["b"] == s["c"]
        elif s["kind"] == "er":
            assert s["m_pairs"] == 8 * s["n"]  # mean degree 16 after symmetrising
        else:
            assert 512 <= s["width"] <= 2048 and s["width"] == s["height"] and 0 <= s["p_del"] <= 0.2
    assert len({s["seed"] for s in a}) == 200


def test_log_time_targets():
    T = np.array([[10.0, 20.0, 40.0], [5.0, 5.0, 1e9]], np.float32)
    t = pl.log_time_targets(T)
    assert t[0, 0] == 0 and np.isclose(t[0, 1], -math.log(2)) and np.isclose(t[0, 2], -math.log(4))
    assert t[1, 0] == 0 and t[1, 1] == 0 and t[1, 2] == pl.LOG_TIME_FLOOR  # clipped


def test_resampling_follows_the_cost_of_a_wrong_choice():
    # level 0: a wrong choice costs 1000 us; level 1: nothing (only the floor)
    T = np.array([[10.0, 1010.0, 20.0], [7.0, 7.0, 7.0]], np.float32)
    idx = pl.resample_index(T, n_rows=20000, seed=3, floor_us=0.5)
    assert idx.min() >= 0 and idx.max() <= 1
    share = np.mean(idx == 1)
    assert share < 0.002  # 0.5 / 1000.5 expected
    assert np.array_equal(idx, pl.resample_index(T, n_rows=20000, seed=3, floor_us=0.5))


def test_gate_mirrors_the_device_rule():
    alpha, trust, margin = 8.0, 8.0, 1.0
    K = np.array([0, 0, 2, 0, 0], np.int64)  # the heuristic's choices
    # feature 0 = log2(e_f / m_u); the band is 1/trust < alpha * e_f / m_u < trust
    x0 = np.array([math.log2(1 / 8),      # ratio 1: in the band
                   math.log2(1 / 8),      # in the band, but the margin is not met
                   math.log2(1 / 8),      # in the band, heuristic already best
                   math.log2(2.0),        # ratio 16: outside
                   math.log2(1 / 80)])    # ratio 0.1: outside
    X = np.zeros((5, 10)); X[:, 0] = x0
    Z = np.array([[0.0, 0.0, 1.5],   # pull beats push by 1.5 > margin -> 2
                  [0.0, 0.0, 0.9],   # by 0.9 <= margin -> heuristic 0
                  [0.0, 0.5, 0.2],   # argmax 1 but heuristic 2: 0.5 - 0.2 <= margin -> 2
                  [0.0, 0.0, 9.0],   # outside the band -> heuristic
                  [0.0, 9.0, 0.0]])
    got = pl.gate(Z, X, K, alpha=alpha, trust=trust, margin=margin)
    assert got.tolist() == [2, 0, 2, 0, 0]


def test_regret():
    T = np.array([[10.0, 20.0, 30.0], [4.0, 1.0, 2.0]])
    r = pl.regret(np.array([0, 1]), T)
    assert r["regret"] == 0 and r["agree_best"] == 1
    r = pl.regret(np.array([2, 0]), T)
    assert math.isclose(r["time_us"], 34.0) and math.isclose(r["regret"], 34.0 / 11.0 - 1) and r["agree_best"] == 0
