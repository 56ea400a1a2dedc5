"""Input generators: Philox known answers, determinism, and recipe shapes."""
import os

import numpy as np

import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        c0, c1, c2, c3, k0, k1, *out = [int(x, 16) for x in r]
        seed = (k1 << 32) | k0
        index = (c1 << 32) | c0
        got = [graphgen.philox_word(seed, index, c2, c3, i) for i in range(4)]
        assert got == out


def test_generators_are_deterministic_and_in_range():
    for fn in (lambda: graphgen.rmat(12, 4, seed=3), lambda: graphgen.erdos_renyi(1000, 5000, 4),
               lambda: graphgen.grid(30, 20, 0.2, 5), lambda: graphgen.barabasi_albert(500, 4, 6)):
        n1, s1, d1 = fn()
        n2, s2, d2 = fn()
        assert n1 == n2 and np.array_equal(s1, s2) and np.array_equal(d1, d2)
        assert s1.min() >= 0 and d1.min() >= 0 and s1.max() < n1 and d1.max() < n1


def test_rmat_quadrant_frequencies():
    # top-level quadrant of each edge: (src >= n/2, dst >= n/2) ~ (a, b, c, d)
    n, s, d = graphgen.rmat(10, 64, a=0.57, b=0.19, c=0.19, seed=8)
    hs, hd = s >= n // 2, d >= n // 2
    freq = [np.mean(~hs & ~hd), np.mean(~hs & hd), np.mean(hs & ~hd), np.mean(hs & hd)]
    assert np.allclose(freq, [0.57, 0.19, 0.19, 0.05], atol=0.01)


def test_grid_deletion_rate_and_structure():
    n, s, d = graphgen.grid(200, 150, 0.1, seed=4, relabel=False)
    total = 150 * 199 + 149 * 200
    assert abs(len(s) / total - 0.9) < 0.01
    rs, cs = np.divmod(s, 200)
    rd, cd = np.divmod(d, 200)
    assert np.all(np.abs(rs - rd) + np.abs(cs - cd) == 1)


def test_permutation_is_a_permutation():
    p = graphgen.permutation(10007, 42)
    assert np.array_equal(np.sort(p), np.arange(10007))


def test_ba_shape():
    n, s, d = graphgen.barabasi_albert(2000, 5, seed=1)
    assert len(s) == 15 + (2000 - 6) * 5
    assert np.all(s[15:] == np.repeat(np.arange(6, 2000), 5))
    assert np.all(d[15:] <= s[15:])


def test_sources_distinct_with_degree():
    n, s, d = graphgen.rmat(12, 4, seed=3)
    src = graphgen.sample_sources(n, s, d, 64, seed=9)
    assert len(set(src.tolist())) == 64
    ok = np.zeros(n, bool)
    nz = s != d
    ok[s[nz]] = True
    ok[d[nz]] = True
    assert ok[src].all()
