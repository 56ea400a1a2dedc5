"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

Depths must match the oracle bit-exactly (depth is the unique hop distance of
Cascade 1); parents are not unique (ANY in Eq. advance), so they must pass the
oracle's validator instead.  Every direction schedule must give the same depths
(the paper's manipulations are semantics-preserving, Section 4.A).
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2607_17106_gb300 as bg

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_17106_gb300 import build
    build.build()
    bg.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _graph_pair(n, src, dst):
    adj = oracle.build_adjacency(n, src, dst)
    g = bg.Graph.build(n, src, dst)
    return adj, g


def _run(g, n, sources, opt=None, with_parent=True):
    k = len(sources)
    # a sentinel, so that an entry the run leaves unwritten cannot pass for an
    # earlier run's result left in reused memory
    depth = torch.full((k * n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    parent = torch.full((k * n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda") if with_parent else None
    src = np.asarray(sources, np.int32)
    g.run(src, depth, parent, opt)
    g.sync()
    torch.cuda.synchronize()
    d = depth.cpu().numpy().reshape(k, n)
    p = parent.cpu().numpy().reshape(k, n) if with_parent else None
    return d, p


def _check(adj, sources, d, p, directed=False):
    for j, s in enumerate(sources):
        ref, _ = oracle.bfs(adj, int(s), with_parent=False)
        assert np.array_equal(d[j], ref), f"depth mismatch for source {s}: {np.flatnonzero(d[j] != ref)[:10]}"
        if p is not None:
            assert oracle.validate(adj, int(s), d[j], p[j], directed=directed) == 0


# ------------------------------------------------------------------ builder
@pytest.mark.parametrize("kind", ["rmat", "er", "grid", "ba", "dups"])
def test_builder_csr_equals_oracle_adjacency(kind):
    if kind == "rmat":
        n, s, d = graphgen.rmat(14, 16, seed=1)
    elif kind == "er":
        n, s, d = graphgen.erdos_renyi(30000, 100000, seed=3)
    elif kind == "grid":
        n, s, d = graphgen.grid(300, 200, 0.1, seed=4)
    elif kind == "ba":
        n, s, d = graphgen.barabasi_albert(20000, 8, seed=8)
    else:
        rng = np.random.default_rng(1)
        n = 1000
        s = rng.integers(0, 50, 20000).astype(np.int32)  # many repeats and self-loops
        d = rng.integers(0, 50, 20000).astype(np.int32)
    adj, g = _graph_pair(n, s, d)
    rp, col = g.csr()
    assert np.array_equal(rp.astype(np.int64), adj.row_ptr)
    assert np.array_equal(col, adj.col)
    info = g.info()
    deg = np.diff(adj.row_ptr)
    assert info.m == adj.m and info.deg_max == deg.max() and info.n_isolated == int((deg == 0).sum())
    assert abs(info.deg_mean - deg.mean()) < 1e-9 * max(1, deg.mean())


def test_builder_directed_csc_is_the_transpose():
    n, s, d = graphgen.rmat(12, 8, seed=21)
    adj = oracle.build_adjacency(n, s, d, symmetrize=False)
    adjt = oracle.build_adjacency(n, d, s, symmetrize=False)
    g = bg.Graph.build(n, s, d, flags=bg.BFS_DEDUP | bg.BFS_DROP_SELF | bg.BFS_BUILD_CSC)
    rp, col = g.csr()
    assert np.array_equal(rp, adj.row_ptr) and np.array_equal(col, adj.col)
    rpt, colt = g.csr(csc=True)
    assert np.array_equal(rpt, adjt.row_ptr) and np.array_equal(colt, adjt.col)
    srcs = graphgen.sample_sources(n, s, d, 8, seed=3)
    for policy in (bg.BFS_POLICY_HEURISTIC, bg.BFS_POLICY_PULL, bg.BFS_POLICY_PUSH):
        dd, pp = _run(g, n, srcs, bg.options(policy=policy, batch=0))
        _check(adj, srcs, dd, pp, directed=True)
    dd, pp = _run(g, n, srcs, bg.options(batch=1))
    _check(adj, srcs, dd, pp, directed=True)


def test_builder_device_inputs_and_errors():
    n, s, d = graphgen.rmat(10, 8, seed=2)
    ts, td = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    g = bg.Graph.build(n, ts, td)
    adj = oracle.build_adjacency(n, s, d)
    rp, col = g.csr()
    assert np.array_equal(col, adj.col)
    bad = d.copy()
    bad[5] = n
    with pytest.raises(bg.BfsError) as e:
        bg.Graph.build(n, s, bad)
    assert e.value.status == bg.BFS_EINVAL


# ----------------------------------------------------------- single source
def _rmat14():
    w = graphgen.WORKLOADS["rmat-s14-ef16"]
    n, s, d = w.edges()
    return n, s, d, w.sources(n, s, d)


@pytest.fixture(scope="module")
def rmat14():
    n, s, d, srcs = _rmat14()
    adj, g = _graph_pair(n, s, d)
    return n, adj, g, srcs


def test_rmat14_push_only_matches_oracle(rmat14):
    n, adj, g, srcs = rmat14
    d, p = _run(g, n, srcs, bg.options(policy=bg.BFS_POLICY_PUSH, batch=0))
    _check(adj, srcs, d, p)


@pytest.mark.parametrize("policy", [bg.BFS_POLICY_HEURISTIC, bg.BFS_POLICY_PULL, bg.BFS_POLICY_PUSH])
@pytest.mark.parametrize("mode", [bg.BFS_MODE_PERSISTENT, bg.BFS_MODE_HOST_LOOP, bg.BFS_MODE_GRAPH])
def test_rmat14_policies_and_modes(rmat14, policy, mode):
    n, adj, g, srcs = rmat14
    d, p = _run(g, n, srcs[:6], bg.options(policy=policy, mode=mode, batch=0))
    _check(adj, srcs[:6], d, p)


@pytest.mark.parametrize("threads", [256, 512, 1024])
@pytest.mark.parametrize("aggregate", [0, 1])
def test_rmat14_launch_shapes_and_claiming(rmat14, threads, aggregate):
    n, adj, g, srcs = rmat14
    o = bg.options(block_threads=threads, claim_aggregate=aggregate, chunk=64, medium=8, batch=0)
    d, p = _run(g, n, srcs[:4], o)
    _check(adj, srcs[:4], d, p)


@pytest.mark.parametrize("mode", [bg.BFS_MODE_PERSISTENT, bg.BFS_MODE_GRAPH])
def test_random_schedules_give_identical_depths(rmat14, mode):
    n, adj, g, srcs = rmat14
    rng = np.random.default_rng(5)
    for t in range(12):
        sched = rng.integers(0, 3, 40).tolist()
        s = srcs[t % len(srcs)]
        d, p = _run(g, n, [s], bg.options(schedule=sched, chunk=128 if t % 2 else 2048, batch=0, mode=mode))
        _check(adj, [s], d, p)


def test_host_outputs_and_level_log(rmat14):
    n, adj, g, srcs = rmat14
    k = 3
    depth = np.empty(k * n, np.int32)
    parent = np.empty(k * n, np.int32)
    log = (bg.bfs_level_record * 64)()
    nlev = bg.ctypes.c_int32(0)
    o = bg.options(batch=0, level_log=log, level_log_cap=64, levels_out=bg.ctypes.pointer(nlev))
    g.run(np.asarray(srcs[:k], np.int32), depth, parent, o)
    d, p = depth.reshape(k, n), parent.reshape(k, n)
    _check(adj, srcs[:k], d, p)
    ref = oracle.level_stats(adj, d[k - 1])
    assert nlev.value == len(ref)
    for i in range(nlev.value):
        assert log[i].level == i and log[i].f == ref[i][0] and log[i].e_f == ref[i][1]
    # the graph-mode loop records the same levels
    log2 = (bg.bfs_level_record * 64)()
    o = bg.options(batch=0, mode=bg.BFS_MODE_GRAPH, level_log=log2, level_log_cap=64,
                   levels_out=bg.ctypes.pointer(nlev))
    g.run(np.asarray(srcs[k - 1:k], np.int32), depth[:n], parent[:n], o)
    assert nlev.value == len(ref)
    for i in range(nlev.value):
        assert log2[i].f == ref[i][0] and log2[i].e_f == ref[i][1]


@pytest.mark.parametrize("kind", ["er", "grid", "ba", "path", "star"])
def test_other_graph_families(kind):
    if kind == "er":
        n, s, d = graphgen.erdos_renyi(1 << 15, 8 << 15, seed=3)
    elif kind == "grid":
        n, s, d = graphgen.grid(256, 256, 0.1, seed=4)
    elif kind == "ba":
        n, s, d = graphgen.barabasi_albert(1 << 15, 8, seed=8)
    elif kind == "path":
        n = 5000
        s, d = np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)
    else:
        n = 70000
        s, d = np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32)
    adj, g = _graph_pair(n, s, d)
    srcs = graphgen.sample_sources(n, s, d, 4, seed=11)
    for o in (bg.options(batch=0), bg.options(batch=0, chunk=64, medium=4, pull_serial=2),
              bg.options(batch=0, mode=bg.BFS_MODE_GRAPH)):
        dd, pp = _run(g, n, srcs, o)
        _check(adj, srcs, dd, pp)


@pytest.mark.parametrize("serial", [1, 3, 32])
def test_pull_long_row_deferral(rmat14, serial):
    # forced pull with a tiny serial budget: nearly every scan is deferred to
    # the warp's long-row list, which fills and drains many times per block
    n, adj, g, srcs = rmat14
    for mode in (bg.BFS_MODE_PERSISTENT, bg.BFS_MODE_GRAPH):
        o = bg.options(batch=0, policy=bg.BFS_POLICY_PULL, pull_serial=serial, mode=mode)
        dd, pp = _run(g, n, srcs[:4], o)
        _check(adj, srcs[:4], dd, pp)


@pytest.mark.parametrize("pf", [bg.BFS_PUSH_FILTER, bg.BFS_PUSH_FILTER_PREDICATED])
def test_push_filter_forms_match_oracle(rmat14, pf):
    # the advance appends (target, source) pairs to an edge frontier and a
    # filter pass after a grid barrier claims them (Variants 13/14, 20/23):
    # push-only, the heuristic, random schedules, the host loop, small chunks
    n, adj, g, srcs = rmat14
    opts = [bg.options(batch=0, push_filter=pf, policy=bg.BFS_POLICY_PUSH),
            bg.options(batch=0, push_filter=pf),
            bg.options(batch=0, push_filter=pf, mode=bg.BFS_MODE_HOST_LOOP, chunk=64, medium=4),
            bg.options(batch=0, push_filter=pf, block_threads=512, claim_aggregate=1)]
    for o in opts:
        dd, pp = _run(g, n, srcs[:4], o)
        _check(adj, srcs[:4], dd, pp)
    rng = np.random.default_rng(17)
    for t in range(4):
        sched = rng.integers(0, 3, 30).tolist()
        s = srcs[t]
        dd, pp = _run(g, n, [s], bg.options(schedule=sched, batch=0, push_filter=pf))
        _check(adj, [s], dd, pp)


@pytest.mark.parametrize("kind", ["grid", "ba", "star", "tiny"])
def test_push_filter_other_families(kind):
    if kind == "grid":
        n, s, d = graphgen.grid(128, 96, 0.1, seed=4)
    elif kind == "ba":
        n, s, d = graphgen.barabasi_albert(1 << 14, 8, seed=8)
    elif kind == "star":
        n = 70000
        s, d = np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32)
    else:
        n = 77
        s = np.array([0, 1, 2, 40, 41, 76], np.int32)
        d = np.array([1, 2, 3, 41, 42, 76], np.int32)
    adj, g = _graph_pair(n, s, d)
    srcs = graphgen.sample_sources(n, s, d, 3, seed=12) if kind != "tiny" else [0, 5, 40, 76]
    for pf in (bg.BFS_PUSH_FILTER, bg.BFS_PUSH_FILTER_PREDICATED):
        for pol in (bg.BFS_POLICY_HEURISTIC, bg.BFS_POLICY_PUSH):
            dd, pp = _run(g, n, srcs, bg.options(batch=0, push_filter=pf, policy=pol))
            _check(adj, srcs, dd, pp)


def test_push_filter_option_errors(rmat14):
    n, adj, g, srcs = rmat14
    for o in (bg.options(batch=0, push_filter=3), bg.options(batch=0, push_filter=-1),
              bg.options(batch=0, push_filter=bg.BFS_PUSH_FILTER, mode=bg.BFS_MODE_GRAPH)):
        with pytest.raises(bg.BfsError) as e:
            _run(g, n, srcs[:1], o)
        assert e.value.status == bg.BFS_EINVAL


@pytest.mark.parametrize("fs", [bg.BFS_SORT_DEVICE, bg.BFS_SORT_TILE])
def test_frontier_sort_forms_match_oracle(rmat14, fs):
    # Variants 6 (device-wide sort through the bitmap) and 7 (per-tile
    # bitonic sort): push-only, the heuristic, random schedules (queue levels
    # after pull and after push levels), the host loop, small chunks, and the
    # other CTA sizes
    n, adj, g, srcs = rmat14
    opts = [bg.options(batch=0, frontier_sort=fs, policy=bg.BFS_POLICY_PUSH),
            bg.options(batch=0, frontier_sort=fs),
            bg.options(batch=0, frontier_sort=fs, mode=bg.BFS_MODE_HOST_LOOP, chunk=64, medium=4),
            bg.options(batch=0, frontier_sort=fs, block_threads=512),
            bg.options(batch=0, frontier_sort=fs, block_threads=256, push_filter=bg.BFS_PUSH_FILTER)]
    for o in opts:
        dd, pp = _run(g, n, srcs[:4], o)
        _check(adj, srcs[:4], dd, pp)
    rng = np.random.default_rng(23)
    for t in range(4):
        sched = rng.integers(0, 3, 30).tolist()
        s = srcs[t]
        dd, pp = _run(g, n, [s], bg.options(schedule=sched, batch=0, frontier_sort=fs))
        _check(adj, [s], dd, pp)


@pytest.mark.parametrize("kind", ["grid", "ba", "path", "tiny"])
def test_frontier_sort_other_families(kind):
    if kind == "grid":
        n, s, d = graphgen.grid(128, 96, 0.1, seed=4)
    elif kind == "ba":
        n, s, d = graphgen.barabasi_albert(1 << 14, 8, seed=8)
    elif kind == "path":
        n = 3000
        s, d = np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)
    else:
        n = 77
        s = np.array([0, 1, 2, 40, 41, 76], np.int32)
        d = np.array([1, 2, 3, 41, 42, 76], np.int32)
    adj, g = _graph_pair(n, s, d)
    srcs = graphgen.sample_sources(n, s, d, 3, seed=12) if kind != "tiny" else [0, 5, 40, 76]
    for fs in (bg.BFS_SORT_DEVICE, bg.BFS_SORT_TILE):
        for pol in (bg.BFS_POLICY_HEURISTIC, bg.BFS_POLICY_PUSH):
            dd, pp = _run(g, n, srcs, bg.options(batch=0, frontier_sort=fs, policy=pol))
            _check(adj, srcs, dd, pp)


def test_frontier_sort_option_errors(rmat14):
    n, adj, g, srcs = rmat14
    for o in (bg.options(batch=0, frontier_sort=3), bg.options(batch=0, frontier_sort=-1),
              bg.options(batch=0, frontier_sort=bg.BFS_SORT_TILE, mode=bg.BFS_MODE_GRAPH)):
        with pytest.raises(bg.BfsError) as e:
            _run(g, n, srcs[:1], o)
        assert e.value.status == bg.BFS_EINVAL


def _barbell():
    """A 3000-vertex path, an RMAT scale-14 component and a 2000-vertex path in
    a chain: searches from the path ends run long stretches of tiny levels with
    a burst of large levels in the middle."""
    nr, rs, rd = graphgen.rmat(14, 16, seed=21)
    deg = np.bincount(np.concatenate([rs, rd]), minlength=nr)
    hub = int(np.argmax(deg))
    leaf = int(np.flatnonzero(deg == deg[deg > 0].min())[0])
    a, b = 3000, 2000
    pa = np.arange(a, dtype=np.int32)
    pb = np.arange(a + nr, a + nr + b, dtype=np.int32)
    src = np.concatenate([pa[:-1], rs + a, pb[:-1], [a - 1, a + leaf]]).astype(np.int32)
    dst = np.concatenate([pa[1:], rd + a, pb[1:], [a + hub, a + nr]]).astype(np.int32)
    return a + nr + b, src, dst


@pytest.mark.parametrize("threads,small", [(1024, 0), (512, 0), (1024, 1), (512, 1)])
def test_long_runs_of_tiny_levels_around_a_burst(threads, small):
    # thousands of one-vertex levels along the paths, two large levels in the
    # RMAT component between them; with small=1 one thread-block cluster runs
    # the path levels until the burst and the grid-wide launch the rest
    n, s, d = _barbell()
    adj, g = _graph_pair(n, s, d)
    srcs = [0, n - 1, 3000 + 5, 1500]
    sl = bg.BFS_SMALL_CLUSTER if small else bg.BFS_SMALL_OFF
    for pol in (bg.BFS_POLICY_HEURISTIC, bg.BFS_POLICY_PUSH):
        dd, pp = _run(g, n, srcs, bg.options(batch=0, policy=pol, block_threads=threads, small_levels=sl))
        _check(adj, srcs, dd, pp)
    # the level log covers every level, across the two launches
    log = (bg.bfs_level_record * 8192)()
    nlev = bg.ctypes.c_int32(0)
    depth = np.empty(n, np.int32)
    g.run(np.array([0], np.int32), depth, None, bg.options(batch=0, level_log=log, level_log_cap=8192,
                                                          levels_out=bg.ctypes.pointer(nlev), small_levels=sl))
    ref = oracle.level_stats(adj, depth)
    assert nlev.value == len(ref)
    for i in range(nlev.value):
        assert log[i].level == i and log[i].f == ref[i][0] and log[i].e_f == ref[i][1], i
    assert log[nlev.value].dir == -1
    # the level limit is enforced in the middle of the first path
    with pytest.raises(bg.BfsError) as e:
        _run(g, n, [0], bg.options(batch=0, max_levels=100, small_levels=sl))
    assert e.value.status == bg.BFS_ERANGE
    dd, pp = _run(g, n, [0], bg.options(batch=0, small_levels=sl))
    _check(adj, [0], dd, pp)


@pytest.mark.parametrize("small", [bg.BFS_SMALL_AUTO, bg.BFS_SMALL_CLUSTER, bg.BFS_SMALL_OFF])
def test_small_levels_in_a_cluster_on_grids(small):
    # a relabelled grid with deletions (maximum degree 4: the automatic choice
    # runs it in one cluster), n not a multiple of 32, several sources in one
    # call, an isolated source; and an ER graph whose levels outgrow the
    # cluster after a few levels
    n, s, d = graphgen.grid(97, 83, 0.1, seed=41)
    adj, g = _graph_pair(n, s, d)
    deg = np.diff(adj.row_ptr)
    iso = np.flatnonzero(deg == 0)
    srcs = graphgen.sample_sources(n, s, d, 5, seed=42).tolist() + ([int(iso[0])] if len(iso) else [])
    dd, pp = _run(g, n, srcs, bg.options(batch=0, small_levels=small))
    _check(adj, srcs, dd, pp)
    g.free()
    n2, s2, d2 = graphgen.erdos_renyi(20000, 80000, seed=43)
    adj2, g2 = _graph_pair(n2, s2, d2)
    srcs2 = graphgen.sample_sources(n2, s2, d2, 3, seed=44).tolist()
    for pol in (bg.BFS_POLICY_HEURISTIC, bg.BFS_POLICY_PUSH):
        dd, pp = _run(g2, n2, srcs2, bg.options(batch=0, small_levels=small, policy=pol))
        _check(adj2, srcs2, dd, pp)
    g2.free()


def test_small_levels_option_errors():
    n, s, d = graphgen.grid(16, 16, 0.0, seed=1)
    g = bg.Graph.build(n, s, d)
    with pytest.raises(bg.BfsError) as e:
        _run(g, n, [0], bg.options(batch=0, small_levels=2))
    assert e.value.status == bg.BFS_EINVAL
    g.free()


def test_many_searches_in_one_launch_match_the_oracle():
    # k sources with batch = 0 and device outputs run one after another in one
    # persistent launch: an isolated source, a two-vertex component, the same
    # hub twice, a path end, mixed with ordinary sources; and the same sources
    # one call each
    # (with n % 4 != 0 most output rows start off a 16-byte boundary, where
    # the -1 stores of a row switch from 4-byte to 16-byte stores)
    nr, rs, rd = graphgen.rmat(13, 16, seed=31)
    a = 2500
    src = np.concatenate([rs, np.arange(nr, nr + a - 1), [nr + a + 1]]).astype(np.int32)
    dst = np.concatenate([rd, np.arange(nr + 1, nr + a), [nr + a + 2]]).astype(np.int32)
    for pad in (0, 1, 3):
        n = nr + a + 4 + pad  # nr + a + 3 and the padding stay isolated
        adj, g = _graph_pair(n, src, dst)
        deg = np.diff(adj.row_ptr)
        hub = int(np.argmax(deg))
        srcs = [nr + a + 3, nr + a + 1, hub, hub, nr, 7] + graphgen.sample_sources(n, src, dst, 6, seed=5).tolist()
        opts = [bg.options(batch=0)]
        if pad == 0:
            opts += [bg.options(batch=0, block_threads=512), bg.options(batch=0, policy=bg.BFS_POLICY_PULL)]
        for o in opts:
            dd, pp = _run(g, n, srcs, o)
            _check(adj, srcs, dd, pp)
        d1 = np.stack([_run(g, n, [s], bg.options(batch=0))[0][0] for s in srcs])
        assert np.array_equal(d1, dd)
        g.free()


def test_edge_cases_tiny_and_isolated():
    # one vertex, no edges
    g = bg.Graph.build(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    d, p = _run(g, 1, [0], bg.options(batch=0))
    assert d.tolist() == [[0]] and p.tolist() == [[0]]
    # isolated source and disconnected pieces, n not a multiple of 32
    n = 77
    s = np.array([0, 1, 2, 40, 41, 76], np.int32)
    dd = np.array([1, 2, 3, 41, 42, 76], np.int32)
    adj, g = _graph_pair(n, s, dd)
    for src in [0, 5, 40, 76]:
        for pol in (bg.BFS_POLICY_HEURISTIC, bg.BFS_POLICY_PULL, bg.BFS_POLICY_PUSH):
            for mode in (bg.BFS_MODE_PERSISTENT, bg.BFS_MODE_GRAPH):
                d1, p1 = _run(g, n, [src], bg.options(policy=pol, batch=0, mode=mode))
                _check(adj, [src], d1, p1)
    with pytest.raises(bg.BfsError) as e:
        _run(g, n, [n], bg.options(batch=0))
    assert e.value.status == bg.BFS_EINVAL
    with pytest.raises(bg.BfsError):
        _run(g, n, [-1], bg.options(batch=0))


def test_level_limit_and_barrier_timeout_report_errors(rmat14):
    n, adj, g, srcs = rmat14
    with pytest.raises(bg.BfsError) as e:
        _run(g, n, [srcs[0]], bg.options(batch=0, max_levels=1))
    assert e.value.status == bg.BFS_ERANGE
    with pytest.raises(bg.BfsError) as e:
        _run(g, n, [srcs[0]], bg.options(batch=0, max_levels=1, mode=bg.BFS_MODE_GRAPH))
    assert e.value.status == bg.BFS_ERANGE
    # a 1 ns limit makes every barrier wait run out: the kernel must give up
    # cleanly and report ETIMEOUT, and the next run must be unaffected
    with pytest.raises(bg.BfsError) as e:
        _run(g, n, [srcs[0]], bg.options(batch=0, barrier_timeout_ns=1))
    assert e.value.status == bg.BFS_ETIMEOUT
    d, p = _run(g, n, srcs[:2], bg.options(batch=0))
    _check(adj, srcs[:2], d, p)


def test_level_stats_match_oracle(rmat14):
    n, adj, g, srcs = rmat14
    d, _ = _run(g, n, srcs[:3], bg.options(batch=0), with_parent=False)
    for j in range(3):
        ref = oracle.level_stats(adj, d[j])
        got = g.level_stats(torch.from_numpy(d[j].copy()).cuda())
        assert np.array_equal(got, ref)
    n2 = 3000
    pth, g2 = _graph_pair(n2, np.arange(n2 - 1, dtype=np.int32), np.arange(1, n2, dtype=np.int32))
    d2, _ = _run(g2, n2, [0], bg.options(batch=0), with_parent=False)
    assert np.array_equal(g2.level_stats(d2[0]), oracle.level_stats(pth, d2[0]))


# ------------------------------------------------------------------ MS-BFS
@pytest.mark.parametrize("k", [1, 5, 64, 130])
def test_msbfs_lanes_match_single_source_oracle(rmat14, k):
    n, adj, g, srcs = rmat14
    w = graphgen.WORKLOADS["rmat-s14-ef16"]
    _, s, d = w.edges()
    sources = graphgen.sample_sources(n, s, d, k, seed=77)
    dd, pp = _run(g, n, sources, bg.options(batch=1))
    _check(adj, sources, dd, pp)


@pytest.mark.parametrize("policy", [bg.BFS_POLICY_PUSH, bg.BFS_POLICY_PULL])
def test_msbfs_forms_and_duplicate_sources(rmat14, policy):
    n, adj, g, srcs = rmat14
    sources = list(srcs[:10]) + list(srcs[:3])  # repeated sources are allowed
    dd, pp = _run(g, n, sources, bg.options(policy=policy, chunk=64, medium=8, pull_serial=2))
    _check(adj, sources, dd, pp)


def test_msbfs_other_families():
    for n, s, d in (graphgen.grid(128, 128, 0.1, seed=4), graphgen.erdos_renyi(20000, 80000, seed=5),
                    graphgen.barabasi_albert(20000, 4, seed=6)):
        adj, g = _graph_pair(n, s, d)
        sources = graphgen.sample_sources(n, s, d, 64, seed=2)
        dd, pp = _run(g, n, sources, bg.options())
        _check(adj, sources, dd, pp)


def test_mixed_batch_over_several_graphs():
    graphs, adjs, ns = [], [], []
    for sc in (10, 11, 12):
        n, s, d = graphgen.rmat(sc, 8, seed=100 + sc)
        adj, g = _graph_pair(n, s, d)
        graphs.append(g)
        adjs.append((adj, s, d))
        ns.append(n)
    rng = np.random.default_rng(4)
    q = 150
    goq = rng.integers(0, 3, q).astype(np.int32)
    srcs = np.array([graphgen.sample_sources(ns[gi], adjs[gi][1], adjs[gi][2], 1, seed=1000 + i)[0]
                     for i, gi in enumerate(goq)], np.int32)
    depth = [torch.empty(ns[gi], dtype=torch.int32, device="cuda") for gi in goq]
    parent = [torch.empty(ns[gi], dtype=torch.int32, device="cuda") for gi in goq]
    bg.run_mixed(graphs, goq, srcs, depth, parent, bg.options())
    torch.cuda.synchronize()
    for i, gi in enumerate(goq):
        adj = adjs[gi][0]
        ref, _ = oracle.bfs(adj, int(srcs[i]), with_parent=False)
        dd = depth[i].cpu().numpy()
        assert np.array_equal(dd, ref)
        assert oracle.validate(adj, int(srcs[i]), dd, parent[i].cpu().numpy()) == 0
