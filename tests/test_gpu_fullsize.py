"""GPU parity at the benchmark's full sizes, in the launch configurations
bench.py times (single-source persistent search with default options; 64-lane
batches with default options).

The oracle computes whole depth arrays for a sample of the sources, which must
match bit-exactly, and validates their parents.  For more lanes of a batch,
properties that hold at any size are checked on the device over every edge:
|depth u - depth v| <= 1 where both ends are reached, and no edge joins a
reached and an unreached vertex; the source has depth 0 and is its own parent.
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


def _edge_properties_hold(row_ptr, col, depth_row, s) -> bool:
    """Device check over every CSR entry (u, v) of one lane's depth row."""
    n = depth_row.numel()
    deg = row_ptr[1:] - row_ptr[:-1]
    rows = torch.repeat_interleave(torch.arange(n, device="cuda", dtype=torch.int64), deg)
    du = depth_row[rows]
    dv = depth_row[col]
    reached_u, reached_v = du >= 0, dv >= 0
    if bool((reached_u != reached_v).any()):
        return False
    both = reached_u & reached_v
    if bool(((du - dv).abs()[both] > 1).any()):
        return False
    return int(depth_row[s]) == 0


@pytest.fixture(scope="module", params=["rmat-s22-ef16", "ba-n22-m8"])
def full(request):
    w = graphgen.WORKLOADS[request.param]
    n, s, d = w.edges()
    srcs = np.asarray(w.sources(n, s, d), np.int32)  # the bench's rank-0 sources
    g = bg.Graph.build(n, s, d)
    adj = oracle.build_adjacency(n, s, d)
    yield w.name, n, s, d, srcs, g, adj
    g.free()


def test_single_source_full_size_sampled(full):
    # the bench's step: the 64 sources one after another in one persistent
    # launch, with no grid barrier between consecutive searches
    name, n, s, d, srcs, g, adj = full
    k = len(srcs)
    depth = torch.full((k, n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    parent = torch.full((k, n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    g.run(srcs, depth, parent, bg.options(batch=0))
    g.sync()
    for j in (0, 17, 63):
        dd, pp = depth[j].cpu().numpy(), parent[j].cpu().numpy()
        ref, _ = oracle.bfs(adj, int(srcs[j]), with_parent=False)
        assert np.array_equal(dd, ref), (name, j)
        assert oracle.validate(adj, int(srcs[j]), dd, pp) == 0, (name, j)
    rp, col = g.csr()
    row_ptr = torch.from_numpy(rp.astype(np.int64)).cuda()
    colt = torch.from_numpy(col.astype(np.int64)).cuda()
    for j in range(1, k, 5):
        assert _edge_properties_hold(row_ptr, colt, depth[j].long(), int(srcs[j])), (name, j)
        assert int(parent[j][int(srcs[j])]) == int(srcs[j])
        assert int((depth[j] == 0x5A5A5A5A).sum()) == 0 and int((parent[j] == 0x5A5A5A5A).sum()) == 0
    # one search per call gives the same depths
    one = torch.empty(n, dtype=torch.int32, device="cuda")
    for j in (5, 40):
        g.run(srcs[j:j + 1], one, None, bg.options(batch=0))
        g.sync()
        assert torch.equal(one, depth[j]), (name, j)


def test_batched_full_size_sampled_and_properties(full):
    name, n, s, d, srcs, g, adj = full
    k = len(srcs)
    depth = torch.full((k, n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    parent = torch.full((k, n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    g.run(srcs, depth, parent, bg.options(batch=1))
    g.sync()
    for j in (0, 31, 63):  # whole lanes against the oracle
        dd, pp = depth[j].cpu().numpy(), parent[j].cpu().numpy()
        ref, _ = oracle.bfs(adj, int(srcs[j]), with_parent=False)
        assert np.array_equal(dd, ref), (name, j)
        assert oracle.validate(adj, int(srcs[j]), dd, pp) == 0, (name, j)
    rp, col = g.csr()
    row_ptr = torch.from_numpy(rp.astype(np.int64)).cuda()
    colt = torch.from_numpy(col.astype(np.int64)).cuda()
    for j in range(1, k, 9):  # properties over every edge for more lanes
        assert _edge_properties_hold(row_ptr, colt, depth[j].long(), int(srcs[j])), (name, j)
        assert int(parent[j][int(srcs[j])]) == int(srcs[j])


def test_reordered_full_size_sampled(full):
    name, n, s, d, srcs, g, adj = full
    gr = bg.Graph.build(n, s, d, flags=bg.BFS_DEFAULT_FLAGS | bg.BFS_REORDER_RCM | bg.BFS_PULL_HUBS_FIRST)
    newid = gr.permutation()
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    j = 5
    gr.run(newid[srcs[j:j + 1]], depth, parent, bg.options(batch=0))
    gr.sync()
    ref, _ = oracle.bfs(adj, int(srcs[j]), with_parent=False)
    assert np.array_equal(depth.cpu().numpy()[newid], ref), name
    gr.free()


def test_components_full_size(full):
    name, n, s, d, srcs, g, adj = full
    got, iters = g.components()
    assert np.array_equal(got, oracle.min_label(adj)), name
    assert iters > 0

