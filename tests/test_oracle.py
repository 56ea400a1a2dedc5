"""Pins for the CPU oracle: it is checked here against things other than itself.

- brute force: hop distances by Boolean matrix powers on thousands of tiny graphs
- closed forms: grid (Manhattan), path, cycle, star, complete graph, disjoint pieces
- invariants: edge depth gap <= 1, reached set == connected component (union-find)
- validator: accepts oracle output, rejects each kind of corrupted parent/depth
- per-level statistics: closed forms on path and complete graphs, identities of Cascade 1
- MLP FP64 reference: central finite differences, zero-parameter closed form; Adam at step 1, under a
  constant gradient at every step, two steps by hand, momentum past a zero gradient
- regression loss: finite differences, constant-output closed form, exact-fit zero
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle


def _tiny_graph(rng, n):
    m = int(rng.integers(0, 3 * n + 1))
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    return src, dst


def test_bfs_matches_boolean_matrix_powers_on_random_tiny_graphs():
    rng = np.random.default_rng(20261202)
    checked = 0
    for g in range(10000):
        n = int(rng.integers(1, 65)) if g % 4 else int(rng.integers(1, 9))
        src, dst = _tiny_graph(rng, n)
        adj = oracle.build_adjacency(n, src, dst)
        dist = oracle.apsp_boolean(n, src, dst)
        for s in range(n) if n <= 16 else rng.choice(n, 4, replace=False):
            depth, parent = oracle.bfs(adj, int(s))
            assert np.array_equal(depth, dist[s]), (g, n, s)
            assert oracle.validate(adj, int(s), depth, parent) == 0
            checked += 1
    assert checked > 40000


def test_adjacency_is_the_deduplicated_symmetric_edge_set():
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = int(rng.integers(1, 40))
        src, dst = _tiny_graph(rng, n)
        adj = oracle.build_adjacency(n, src, dst)
        pairs = set()
        for s, d in zip(src.tolist(), dst.tolist()):
            if s != d:
                pairs.add((s, d))
                pairs.add((d, s))
        got = set()
        for u in range(n):
            row = adj.col[adj.row_ptr[u]:adj.row_ptr[u + 1]].tolist()
            assert row == sorted(set(row))
            got.update((u, v) for v in row)
        assert got == pairs
        assert adj.m == len(pairs)


def test_directed_adjacency_keeps_direction():
    src = np.array([0, 1, 1, 2, 2], np.int32)
    dst = np.array([1, 2, 2, 0, 2], np.int32)
    adj = oracle.build_adjacency(3, src, dst, symmetrize=False)
    assert adj.row_ptr.tolist() == [0, 1, 2, 3]
    assert adj.col.tolist() == [1, 2, 0]
    depth, _ = oracle.bfs(adj, 1)
    assert depth.tolist() == [2, 0, 1]


def test_grid_depth_is_manhattan_distance():
    w, h = 37, 23
    n, src, dst = graphgen.grid(w, h, 0.0, seed=9, relabel=False)
    adj = oracle.build_adjacency(n, src, dst)
    rr, cc = np.divmod(np.arange(n), w)
    for s in [0, w - 1, n - 1, (h // 2) * w + w // 3]:
        depth, parent = oracle.bfs(adj, s)
        sr, sc = divmod(s, w)
        assert np.array_equal(depth, np.abs(rr - sr) + np.abs(cc - sc))
        assert oracle.validate(adj, s, depth, parent) == 0


def test_relabelled_grid_is_the_permuted_grid():
    w, h = 19, 11
    n, s0, d0 = graphgen.grid(w, h, 0.0, seed=3, relabel=False)
    _, s1, d1 = graphgen.grid(w, h, 0.0, seed=3, relabel=True)
    perm = graphgen.permutation(n, 3)
    assert np.array_equal(perm[s0], s1) and np.array_equal(perm[d0], d1)
    a0 = oracle.build_adjacency(n, s0, d0)
    a1 = oracle.build_adjacency(n, s1, d1)
    depth0, _ = oracle.bfs(a0, 5)
    depth1, _ = oracle.bfs(a1, int(perm[5]))
    assert np.array_equal(depth1[perm], depth0)


def test_closed_forms_path_cycle_star_complete():
    n = 50
    i = np.arange(n)
    path = (np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32))
    adj = oracle.build_adjacency(n, *path)
    for s in [0, 17, n - 1]:
        assert np.array_equal(oracle.bfs(adj, s)[0], np.abs(i - s))
    cyc = (np.arange(n, dtype=np.int32), ((np.arange(n) + 1) % n).astype(np.int32))
    adj = oracle.build_adjacency(n, *cyc)
    for s in [0, 11]:
        d = np.abs(i - s)
        assert np.array_equal(oracle.bfs(adj, s)[0], np.minimum(d, n - d))
    star = (np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32))
    adj = oracle.build_adjacency(n, *star)
    assert np.array_equal(oracle.bfs(adj, 0)[0], np.where(i == 0, 0, 1))
    depth, parent = oracle.bfs(adj, 7)
    assert depth[7] == 0 and depth[0] == 1 and np.all(depth[(i != 0) & (i != 7)] == 2)
    assert parent[7] == 7 and parent[0] == 7 and np.all(parent[(i != 0) & (i != 7)] == 0)
    k = 12
    comp = np.array(list(itertools.combinations(range(k), 2)), np.int32)
    adj = oracle.build_adjacency(k, comp[:, 0], comp[:, 1])
    assert np.array_equal(oracle.bfs(adj, 3)[0], np.where(np.arange(k) == 3, 0, 1))


def test_disconnected_pieces_and_isolated_vertices_are_unreached():
    src = np.array([0, 1, 4, 5, 7], np.int32)
    dst = np.array([1, 2, 5, 6, 7], np.int32)  # 7 has only a self-loop; 3 is isolated
    adj = oracle.build_adjacency(8, src, dst)
    depth, parent = oracle.bfs(adj, 0)
    assert depth.tolist() == [0, 1, 2, -1, -1, -1, -1, -1]
    assert parent.tolist() == [0, 0, 1, -1, -1, -1, -1, -1]
    depth, parent = oracle.bfs(adj, 7)
    assert depth.tolist() == [-1] * 7 + [0] and parent.tolist() == [-1] * 7 + [7]


@pytest.mark.parametrize("kind", ["rmat", "er", "ba"])
def test_invariants_and_reached_set_equals_component(kind):
    if kind == "rmat":
        n, src, dst = graphgen.rmat(12, 8, seed=11)
    elif kind == "er":
        n, src, dst = graphgen.erdos_renyi(5000, 6000, seed=12)
    else:
        n, src, dst = graphgen.barabasi_albert(3000, 3, seed=13)
    adj = oracle.build_adjacency(n, src, dst)
    comp = oracle.components(n, src, dst)
    for s in graphgen.sample_sources(n, src, dst, 6, seed=5):
        depth, parent = oracle.bfs(adj, int(s))
        assert oracle.validate(adj, int(s), depth, parent) == 0
        reached = depth >= 0
        assert np.array_equal(reached, comp == comp[s])
        u = np.repeat(np.arange(n), np.diff(adj.row_ptr))
        du, dv = depth[u], depth[adj.col]
        both = (du >= 0) & (dv >= 0)
        assert np.all(np.abs(du[both] - dv[both]) <= 1)
        assert np.all((du >= 0) == (dv >= 0))


def test_validator_rejects_corruptions():
    n, src, dst = graphgen.rmat(10, 8, seed=21)
    adj = oracle.build_adjacency(n, src, dst)
    s = int(graphgen.sample_sources(n, src, dst, 1, seed=1)[0])
    depth, parent = oracle.bfs(adj, s)
    assert oracle.validate(adj, s, depth, parent) == 0
    reached = np.flatnonzero((depth >= 2))
    v = int(reached[0])
    # parent that is not a neighbour
    p = parent.copy()
    nbrs = set(adj.col[adj.row_ptr[v]:adj.row_ptr[v + 1]].tolist())
    far = next(int(x) for x in np.flatnonzero(depth == depth[v] - 1) if int(x) not in nbrs)
    p[v] = far
    assert oracle.validate(adj, s, depth, p) == 6
    # parent at the wrong level (a neighbour of the same depth or deeper)
    same = [x for x in nbrs if depth[x] >= depth[v]]
    if same:
        p = parent.copy()
        p[v] = same[0]
        assert oracle.validate(adj, s, depth, p) == 7
    # a two-cycle of parents
    p = parent.copy()
    a = v
    b = int(parent[v])
    p[b] = a
    assert oracle.validate(adj, s, depth, p) in (6, 7)
    # parent of an unreached vertex / reached vertex without parent
    p = parent.copy()
    p[v] = -1
    assert oracle.validate(adj, s, depth, p) == 2
    # wrong source entry
    p = parent.copy()
    p[s] = int(adj.col[adj.row_ptr[s]])
    assert oracle.validate(adj, s, depth, p) == 1
    # depth off by one on a vertex (edge gap > 1 or parent level breaks)
    d = depth.copy()
    d[v] += 2
    assert oracle.validate(adj, s, d, parent) in (3, 7)
    # a reached vertex marked unreached
    d = depth.copy()
    d[v] = -1
    assert oracle.validate(adj, s, d, None) == 4
    d = depth.copy()
    d[v] = 0
    assert oracle.validate(adj, s, d, None) == 8


def test_level_stats_closed_form_path():
    n = 9
    adj = oracle.build_adjacency(n, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32))
    depth, _ = oracle.bfs(adj, 0)
    st = oracle.level_stats(adj, depth)
    deg = np.diff(adj.row_ptr)
    assert st.shape == (n, 6)
    for i in range(n):
        f, e_f, u, s_u, d_new, e_u = st[i].tolist()
        assert f == 1 and e_f == deg[i]
        assert d_new == (1 if i < n - 1 else 0)
        assert u == n - 1 - i
        assert e_u == int(deg[i + 1:].sum())
        assert s_u == (1 + e_u - deg[i + 1] if i < n - 1 else 0)


def test_level_stats_closed_form_complete_graph_and_identities():
    k = 10
    pairs = np.array(list(itertools.combinations(range(k), 2)), np.int32)
    adj = oracle.build_adjacency(k, pairs[:, 0], pairs[:, 1])
    st = oracle.level_stats(adj, oracle.bfs(adj, 0)[0])
    assert st.tolist() == [[1, k - 1, k - 1, k - 1, k - 1, (k - 1) ** 2],
                           [k - 1, (k - 1) ** 2, 0, 0, 0, 0]]
    n, src, dst = graphgen.rmat(11, 8, seed=31)
    adj = oracle.build_adjacency(n, src, dst)
    s = int(graphgen.sample_sources(n, src, dst, 1, seed=2)[0])
    depth, _ = oracle.bfs(adj, s)
    st = oracle.level_stats(adj, depth)
    f, e_f, u, s_u, d_new, e_u = st.T
    assert f.sum() == np.count_nonzero(depth >= 0)
    assert np.array_equal(d_new[:-1], f[1:]) and d_new[-1] == 0
    assert np.array_equal(u[:-1] - u[1:], d_new[:-1])   # P_{i+1} = P_i OR F_{i+1}
    assert np.array_equal(e_u[:-1] - e_u[1:], e_f[1:])
    assert np.all(s_u <= e_u) and np.all(s_u >= 0)


def _random_params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.4, oracle.mlp_num_params())


def test_mlp_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(3)
    P = _random_params(4)
    X = rng.normal(0, 1, (17, oracle.N_IN))
    y = rng.integers(0, oracle.N_OUT, 17).astype(np.int32)
    loss, g = oracle.mlp_loss_grad(P, X, y)
    h = 1e-6
    num = np.empty_like(g)
    for i in range(len(P)):
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        num[i] = (oracle.mlp_loss_grad(Pp, X, y)[0] - oracle.mlp_loss_grad(Pm, X, y)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) / np.max(np.abs(g)) < 1e-7
    assert loss > 0


def test_mlp_closed_forms():
    P = np.zeros(oracle.mlp_num_params())
    b3 = np.array([0.5, -1.0, 2.0])
    P[-3:] = b3
    X = np.random.default_rng(1).normal(0, 1, (5, oracle.N_IN))
    assert np.allclose(oracle.mlp_forward(P, X), np.tile(b3, (5, 1)))
    P[-3:] = 0
    loss, g = oracle.mlp_loss_grad(P, X, np.array([0, 1, 2, 0, 1], np.int32))
    assert abs(loss - np.log(3)) < 1e-15
    # gradient wrt b3 is mean(softmax - onehot) = 1/3 - frequency of each class
    assert np.allclose(g[-3:], np.array([1 / 3 - 2 / 5, 1 / 3 - 2 / 5, 1 / 3 - 1 / 5]))
    # one hidden path: W1[0,0]=1, W2[0,0]=1, W3[j,0]=c_j gives z = c * relu(x0)
    P = np.zeros(oracle.mlp_num_params())
    P[0] = 1.0
    off_w2 = 32 * 10 + 32
    P[off_w2] = 1.0
    off_w3 = off_w2 + 32 * 32 + 32
    c = np.array([2.0, -3.0, 0.25])
    P[off_w3 + 0] = c[0]; P[off_w3 + 32] = c[1]; P[off_w3 + 64] = c[2]
    X = np.zeros((3, oracle.N_IN)); X[:, 0] = [1.5, -2.0, 0.0]
    Z = oracle.mlp_forward(P, X)
    assert np.allclose(Z, np.outer(np.maximum(X[:, 0], 0), c))


def test_mlp_regression_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(5)
    P = _random_params(6)
    X = rng.normal(0, 1, (13, oracle.N_IN))
    t = rng.normal(0, 2, (13, oracle.N_OUT))
    loss, g = oracle.mlp_regress_loss_grad(P, X, t)
    h = 1e-6
    num = np.empty_like(g)
    for i in range(len(P)):
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        num[i] = (oracle.mlp_regress_loss_grad(Pp, X, t)[0] - oracle.mlp_regress_loss_grad(Pm, X, t)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) / np.max(np.abs(g)) < 1e-7
    assert loss > 0


def test_mlp_regression_closed_forms():
    rng = np.random.default_rng(8)
    X = rng.normal(0, 1, (6, oracle.N_IN))
    t = rng.uniform(-5, 0, (6, oracle.N_OUT))
    # only the output bias set: z = b3 for every row, so L = mean |b3 - t|^2 / 2
    # and dL/db3 = b3 - mean(t); nothing reaches the zero weights
    P = np.zeros(oracle.mlp_num_params())
    b3 = np.array([0.5, -1.0, 2.0])
    P[-3:] = b3
    loss, g = oracle.mlp_regress_loss_grad(P, X, t)
    assert abs(loss - 0.5 * ((b3 - t) ** 2).sum(axis=1).mean()) < 1e-13
    assert np.allclose(g[-3:], b3 - t.mean(axis=0), atol=1e-14)
    assert np.all(g[:-3] == 0)
    # targets equal to the network's own outputs: zero loss, zero gradient
    P = _random_params(9)
    loss, g = oracle.mlp_regress_loss_grad(P, X, oracle.mlp_forward(P, X))
    assert loss < 1e-28 and np.max(np.abs(g)) < 1e-14


def test_adam_first_step_is_lr_times_sign():
    P = np.array([1.0, -2.0, 3.0]); m1 = np.zeros(3); m2 = np.zeros(3)
    g = np.array([0.3, -5.0, 1e-3])
    oracle.adam_step(P, m1, m2, g, t=1, lr=0.01, eps=1e-12)
    assert np.allclose(P, [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], atol=1e-9)


def test_adam_constant_gradient_moves_lr_per_step():
    # Kingma & Ba, Algorithm 1: with the same gradient g at every step the
    # bias-corrected moments are exactly g and g^2, so each step moves every
    # parameter by lr * g / (|g| + eps), at t = 1 and at every later t
    P0 = np.array([0.5, -1.5, 2.0, 0.0])
    g = np.array([0.2, -3.0, 1e-2, 7.0])
    P, m1, m2 = P0.copy(), np.zeros(4), np.zeros(4)
    lr, eps = 0.003, 1e-8
    for t in range(1, 11):
        oracle.adam_step(P, m1, m2, g, t=t, lr=lr, eps=eps)
        assert np.allclose(P, P0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12), t


def test_adam_two_steps_by_hand():
    # beta1 = 1/2, beta2 = 3/4, g1 = 1, g2 = 3, eps = 0, lr = 1.
    # step 1: m = 1/2, v = 1/4; corrections 1/2, 1/4 -> update 1 / sqrt(1) = 1
    # step 2: m = 1/4 + 3/2 = 7/4, v = 3/16 + 9/4 = 39/16; corrections 3/4 and
    #         7/16 -> m_hat = 7/3, v_hat = 39/7 -> update (7/3) / sqrt(39/7)
    P, m1, m2 = np.array([10.0]), np.zeros(1), np.zeros(1)
    oracle.adam_step(P, m1, m2, np.array([1.0]), t=1, lr=1.0, beta1=0.5, beta2=0.75, eps=0.0)
    assert np.allclose(P, [9.0], atol=1e-14)
    assert np.allclose([m1[0], m2[0]], [0.5, 0.25], atol=1e-15)
    oracle.adam_step(P, m1, m2, np.array([3.0]), t=2, lr=1.0, beta1=0.5, beta2=0.75, eps=0.0)
    assert np.allclose([m1[0], m2[0]], [7 / 4, 39 / 16], atol=1e-15)
    assert np.allclose(P, [9.0 - (7 / 3) / np.sqrt(39 / 7)], atol=1e-14)


def test_adam_momentum_carries_past_a_zero_gradient():
    # default betas: a step with g = 1 then one with g = 0.  The first moment
    # is then 0.9 * 0.1 = 0.09 over 1 - 0.81 = 0.19, i.e. 9/19, the second
    # 0.999 * 0.001 over 1 - 0.999^2 = 0.001999, i.e. 999/1999: the parameter
    # keeps moving although the gradient is zero
    P, m1, m2 = np.array([0.0]), np.zeros(1), np.zeros(1)
    lr = 0.01
    oracle.adam_step(P, m1, m2, np.array([1.0]), t=1, lr=lr, eps=0.0)
    oracle.adam_step(P, m1, m2, np.array([0.0]), t=2, lr=lr, eps=0.0)
    assert np.allclose(P, [-lr - lr * (9 / 19) / np.sqrt(999 / 1999)], atol=1e-15)


def test_directed_validation_follows_edge_direction():
    # 0 -> 1 -> 2 -> 0 cycle plus 2 -> 3: from 0, depth(0)=0 is reached again by 2 -> 0
    src = np.array([0, 1, 2, 2], np.int32)
    dst = np.array([1, 2, 0, 3], np.int32)
    adj = oracle.build_adjacency(4, src, dst, symmetrize=False)
    depth, parent = oracle.bfs(adj, 0)
    assert depth.tolist() == [0, 1, 2, 3]
    assert oracle.validate(adj, 0, depth, parent, directed=True) == 0
    assert oracle.validate(adj, 0, depth, parent, directed=False) == 3   # 2 -> 0 spans two levels
    d = depth.copy(); d[3] = -1
    assert oracle.validate(adj, 0, d, None, directed=True) == 4
    d = depth.copy(); d[3] = 5
    assert oracle.validate(adj, 0, d, None, directed=True) == 3


# ------------------------------------------------------------------ RCM
def _cm_rules_hold(adj, newid) -> bool:
    """Declarative check that n-1-newid numbers the vertices in a Cuthill-McKee
    sequence under the oracle's tie rules (rank = (degree, id)): components are
    contiguous and start at their lowest-ranked vertex, in the rank order of the
    starts; inside a component positions follow BFS depth from the start; inside
    a depth level, vertices are ordered by (lowest position of a neighbour one
    level up, rank).  Components and depths come from scipy, not from the oracle."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    n = adj.n
    pos = n - 1 - np.asarray(newid, np.int64)
    if sorted(pos.tolist()) != list(range(n)):
        return False
    deg = adj.degree()
    rank = np.empty(n, np.int64)
    rank[np.lexsort((np.arange(n), deg))] = np.arange(n)
    rows = np.repeat(np.arange(n), deg)
    A = sp.csr_matrix((np.ones(adj.m), (rows, adj.col)), shape=(n, n))
    ncomp, lab = cg.connected_components(A, directed=False)
    starts = []
    for c in range(ncomp):
        members = np.flatnonzero(lab == c)
        p = np.sort(pos[members])
        if p[-1] - p[0] != len(members) - 1:
            return False  # not contiguous
        start = members[np.argmin(rank[members])]
        if pos[start] != p[0]:
            return False
        starts.append((p[0], rank[start]))
        dist = cg.shortest_path(A, unweighted=True, indices=int(start))
        dm = dist[members].astype(np.int64)
        by_pos = members[np.argsort(pos[members])]
        if np.any(np.diff(dist[by_pos]) < 0):
            return False  # depth must not decrease along the sequence
        prev = None
        for v in by_pos[1:]:
            d = int(dist[v])
            nb = adj.col[adj.row_ptr[v]:adj.row_ptr[v + 1]]
            up = [pos[u] for u in nb if dist[u] == d - 1]
            key = (d, min(up), rank[v])
            if prev is not None and key <= prev:
                return False
            prev = key
        del dm
    starts.sort()
    return all(starts[i][1] < starts[i + 1][1] for i in range(len(starts) - 1))


def test_rcm_hand_derived_orders():
    # path 3-0-4-1-2: ends 2 and 3 have degree 1, 2 ranks first; Cuthill-McKee
    # 2,1,4,0,3 reversed
    adj = oracle.build_adjacency(5, np.array([3, 0, 4, 1], np.int32), np.array([0, 4, 1, 2], np.int32))
    assert oracle.rcm(adj).tolist() == [1, 3, 4, 0, 2]
    # star 0-{1..4} plus isolated 5: CM = 5 | 1, 0, 2, 3, 4 ; reversed
    adj = oracle.build_adjacency(6, np.zeros(4, np.int32), np.arange(1, 5, dtype=np.int32))
    assert oracle.rcm(adj).tolist() == [3, 4, 2, 1, 0, 5]
    # two parents: 0 (deg 1) - 1 - {2, 3}, 2 - 4, 3 - 4, 3 - 5.  CM from 0:
    # 0, 1, {2 (deg 2), 3 (deg 3)}, then 4 (first neighbour up = 2), 5 (up = 3)
    adj = oracle.build_adjacency(6, np.array([0, 1, 1, 2, 3, 3], np.int32), np.array([1, 2, 3, 4, 4, 5], np.int32))
    assert oracle.rcm(adj).tolist() == [5, 4, 3, 2, 1, 0]


def test_rcm_closed_form_path_in_natural_order():
    n = 50
    adj = oracle.build_adjacency(n, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32))
    assert np.array_equal(oracle.rcm(adj), n - 1 - np.arange(n))


@pytest.mark.parametrize("kind", ["er", "grid", "ba", "tree", "dense"])
def test_rcm_satisfies_the_cuthill_mckee_rules(kind):
    rng = np.random.default_rng(4)
    for t in range(6):
        if kind == "er":
            n = int(rng.integers(20, 200))
            s, d = rng.integers(0, n, (2, int(rng.integers(n // 2, 2 * n)))).astype(np.int32)
        elif kind == "grid":
            n, s, d = graphgen.grid(int(rng.integers(3, 12)), int(rng.integers(3, 12)), 0.15, seed=t)
        elif kind == "ba":
            n, s, d = graphgen.barabasi_albert(int(rng.integers(30, 300)), 3, seed=t)
        elif kind == "tree":
            n = int(rng.integers(20, 300))
            s = np.array([rng.integers(0, v) for v in range(1, n)], np.int32)
            d = np.arange(1, n, dtype=np.int32)
        else:
            n = 24
            s, d = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.5], np.int32).T
        adj = oracle.build_adjacency(n, s, d)
        newid = oracle.rcm(adj)
        assert _cm_rules_hold(adj, newid), (kind, t)
        # the renamed graph keeps the edge set
        padj = oracle.permute(adj, newid)
        assert padj.m == adj.m
        inv = np.argsort(newid)
        for v in range(0, n, max(1, n // 7)):
            got = np.sort(inv[padj.col[padj.row_ptr[newid[v]]:padj.row_ptr[newid[v] + 1]]])
            assert np.array_equal(got, adj.col[adj.row_ptr[v]:adj.row_ptr[v + 1]])


def test_rcm_rule_check_rejects_planted_mistakes():
    # the checker must catch an unreversed sequence, a swapped tie and a bad start
    n, s, d = graphgen.grid(6, 5, 0.1, seed=2)
    adj = oracle.build_adjacency(n, s, d)
    newid = oracle.rcm(adj)
    assert _cm_rules_hold(adj, newid)
    assert not _cm_rules_hold(adj, n - 1 - newid)  # Cuthill-McKee without the reversal
    pos = n - 1 - newid
    by_pos = np.argsort(pos)
    swapped = newid.copy()
    a, b = by_pos[3], by_pos[4]
    swapped[a], swapped[b] = newid[b], newid[a]
    assert not _cm_rules_hold(adj, swapped)
    rolled = (newid + 1) % n  # start moved off the lowest-ranked vertex
    assert not _cm_rules_hold(adj, rolled)


# ------------------------------------------------------------ min-label components
def test_min_label_closed_forms():
    # path, a cycle plus isolated vertices, two stars: smallest id per component
    adj = oracle.build_adjacency(6, np.array([5, 4, 3, 2, 1], np.int32), np.array([4, 3, 2, 1, 0], np.int32))
    assert oracle.min_label(adj).tolist() == [0] * 6
    adj = oracle.build_adjacency(8, np.array([3, 5, 7], np.int32), np.array([5, 7, 3], np.int32))
    assert oracle.min_label(adj).tolist() == [0, 1, 2, 3, 4, 3, 6, 3]
    adj = oracle.build_adjacency(7, np.array([6, 6, 2, 2], np.int32), np.array([4, 5, 0, 1], np.int32))
    assert oracle.min_label(adj).tolist() == [0, 0, 0, 3, 4, 4, 4]


@pytest.mark.parametrize("kind", ["er", "grid", "rmat", "ba"])
def test_min_label_equals_union_find_and_scipy(kind):
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    rng = np.random.default_rng(8)
    for t in range(4):
        if kind == "er":
            n = int(rng.integers(50, 3000))
            s, d = rng.integers(0, n, (2, int(rng.integers(n // 3, n)))).astype(np.int32)
        elif kind == "grid":
            n, s, d = graphgen.grid(int(rng.integers(5, 60)), int(rng.integers(5, 60)), 0.45, seed=t)
        elif kind == "rmat":
            n, s, d = graphgen.rmat(11, 2, seed=30 + t)
        else:
            n, s, d = graphgen.barabasi_albert(2000, 1, seed=t)
        adj = oracle.build_adjacency(n, s, d)
        lab = oracle.min_label(adj)
        assert np.array_equal(lab, oracle.components(n, s, d))  # union-find, separate code
        A = sp.csr_matrix((np.ones(adj.m), (np.repeat(np.arange(n), adj.degree()), adj.col)), shape=(n, n))
        _, comp = cg.connected_components(A, directed=False)
        first = np.full(comp.max() + 1, n)
        np.minimum.at(first, comp, np.arange(n))
        assert np.array_equal(lab, first[comp])  # scipy components, smallest id each
