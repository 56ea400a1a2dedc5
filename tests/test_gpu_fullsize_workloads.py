"""GPU parity at full size on every benchmark workload beyond RMAT-22 and BA-22,
in the launch configurations the benchmark times.

- Erdos-Renyi n = 2^22, mean degree 16: single-source persistent searches and
  a 64-lane batch.
- 4096 x 4096 grid with 10% of its edges deleted and relabelled vertices: the
  long-diameter case (thousands of levels), single-source in the persistent
  and the CUDA-graph drive, and a 32-lane batch.
- RMAT scale 24: one 64-lane batch (scale-24 index arithmetic, 4.3 GB of
  depths) and one single-source search.
- The mixed batch of 256 queries over RMAT scales 16..22 in one
  bfs_run_mixed launch.
- Held-out RMAT scale 23, edge factor 32, a = 0.60, under the learned policy
  with the committed weights: single-source and batched.

Whole depth rows are compared with the oracle's FIFO BFS (Cascade 1)
bit-exactly and parents pass the oracle's validator.  For queries or lanes the
oracle does not recompute, properties that hold at any size are checked on the
device over every edge (reached ends differ by at most one level, no edge
joins a reached and an unreached vertex, the source has depth 0).
"""
import os

import numpy as np
import pytest

import graphgen
import oracle
import paper_2607_17106_gb300 as bg

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(bg.__file__), "policy_weights.npy")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_17106_gb300 import build
    build.build()
    bg.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _load(name):
    w = graphgen.WORKLOADS[name]
    n, s, d = w.edges()
    srcs = np.asarray(w.sources(n, s, d), np.int32)  # the benchmark's rank-0 sources
    g = bg.Graph.build(n, s, d)
    adj = oracle.build_adjacency(n, s, d)
    del s, d
    return n, srcs, g, adj


def _edge_checker(g):
    """Device check over every CSR entry (u, v) of one depth row: reached ends
    differ by at most one level, no edge joins a reached and an unreached
    vertex, and the source has depth 0."""
    rp, col = g.csr()
    n = len(rp) - 1
    row_ptr = torch.from_numpy(rp.astype(np.int64)).cuda()
    rows = torch.repeat_interleave(torch.arange(n, device="cuda", dtype=torch.int64), row_ptr[1:] - row_ptr[:-1])
    colt = torch.from_numpy(col).cuda().long()

    def holds(depth_row, s) -> bool:
        d = depth_row.long()
        du, dv = d[rows], d[colt]
        if bool(((du >= 0) != (dv >= 0)).any()):
            return False
        both = (du >= 0) & (dv >= 0)
        if bool(((du - dv).abs()[both] > 1).any()):
            return False
        return int(depth_row[s]) == 0

    return holds


def _check_row(adj, s, d_row, p_row, what):
    ref, _ = oracle.bfs(adj, int(s), with_parent=False)
    bad = np.flatnonzero(d_row != ref)
    assert bad.size == 0, f"{what}: {bad.size} depths differ, first at {bad[:5]}"
    if p_row is not None:
        assert oracle.validate(adj, int(s), d_row, p_row) == 0, f"{what}: parents rejected"


def _single(g, n, srcs, js, opt, adj, what):
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    for j in js:
        g.run(srcs[j:j + 1], depth, parent, opt)
        g.sync()
        _check_row(adj, srcs[j], depth.cpu().numpy(), parent.cpu().numpy(), f"{what} source #{j}")


def _batched(g, n, srcs, lanes, opt, adj, what, props_every=0):
    k = len(srcs)
    depth = torch.full((k, n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    parent = torch.full((k, n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    g.run(srcs, depth, parent, opt)
    g.sync()
    for j in lanes:
        _check_row(adj, srcs[j], depth[j].cpu().numpy(), parent[j].cpu().numpy(), f"{what} lane {j}")
    if props_every:
        holds = _edge_checker(g)
        for j in range(1, k, props_every):
            assert holds(depth[j], int(srcs[j])), f"{what} lane {j}: edge properties"
            assert int(parent[j][int(srcs[j])]) == int(srcs[j])
        del holds
    del depth, parent
    torch.cuda.empty_cache()


def test_er22_single_and_batched():
    n, srcs, g, adj = _load("er-n22-deg16")
    _single(g, n, srcs, (0, 31, 63), bg.options(batch=0), adj, "ER-22")
    _batched(g, n, srcs, (0, 31, 63), bg.options(batch=1), adj, "ER-22 batch", props_every=9)
    g.free()


def test_grid4096_persistent_graph_mode_and_batched():
    n, srcs, g, adj = _load("grid-4096-del10")
    _single(g, n, srcs, (0, 15, 31), bg.options(batch=0), adj, "grid persistent")
    _single(g, n, srcs, (0, 31), bg.options(batch=0, mode=bg.BFS_MODE_GRAPH), adj, "grid graph mode")
    _batched(g, n, srcs, (0, 16, 31), bg.options(batch=1), adj, "grid batch", props_every=5)
    g.free()


def test_rmat24_batched_64_lanes_and_single():
    n, srcs, g, adj = _load("rmat-s24-ef16")
    _batched(g, n, srcs, (0, 31, 63), bg.options(batch=1), adj, "RMAT-24 batch", props_every=16)
    _single(g, n, srcs, (0,), bg.options(batch=0), adj, "RMAT-24")
    g.free()


def test_rmat23_ef32_under_the_learned_policy():
    n, srcs, g, adj = _load("rmat-s23-ef32-a60")
    pol = bg.Policy(np.load(WEIGHTS))
    _single(g, n, srcs, (0, 31, 63), bg.options(batch=0, policy=bg.BFS_POLICY_MLP, mlp=pol), adj, "RMAT-23 MLP")
    _batched(g, n, srcs, (0, 31, 63), bg.options(batch=1, policy=bg.BFS_POLICY_MLP, mlp=pol), adj,
             "RMAT-23 MLP batch")
    pol.free()
    g.free()


def test_mixed_batch_256_queries_one_launch():
    scales, edge_lists, goq, srcs = graphgen.mixed_batch()
    graphs = [bg.Graph.build(n, s, d) for n, s, d in edge_lists]
    ns = [n for n, _, _ in edge_lists]
    depth = [torch.empty(ns[gi], dtype=torch.int32, device="cuda") for gi in goq]
    parent = [torch.empty(ns[gi], dtype=torch.int32, device="cuda") for gi in goq]
    bg.run_mixed(graphs, goq, srcs, depth, parent, bg.options())
    torch.cuda.synchronize()
    for g in graphs:
        g.sync()
    checked = 0
    for gi, sc in enumerate(scales):
        adj = oracle.build_adjacency(*edge_lists[gi])
        idx = np.flatnonzero(goq == gi)
        # every query on graphs up to scale 20; four on scales 21 and 22,
        # including the last query of the largest graph
        pick = idx if sc <= 20 else np.unique(np.concatenate([idx[:3], idx[-1:]]))
        for q in pick:
            _check_row(adj, srcs[q], depth[q].cpu().numpy(), parent[q].cpu().numpy(), f"query {q} (scale {sc})")
            checked += 1
        rest = np.setdiff1d(idx, pick)
        if len(rest):
            holds = _edge_checker(graphs[gi])
            for q in rest:
                assert holds(depth[q], int(srcs[q])), f"query {q}: edge properties"
    assert checked >= 3 * len(scales)
    for g in graphs:
        g.free()
