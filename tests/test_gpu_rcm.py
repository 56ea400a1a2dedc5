"""GPU parity of the Reverse Cuthill-McKee reordering (Section 7.1 preprocessing).

The numbering is unique under the tie rules stated in include/bfs.h and in the
oracle (rank = (degree, id), components started at their lowest-ranked vertex),
so the device permutation must equal the oracle's element by element, and the
rebuilt CSR must equal the oracle's renamed adjacency exactly.  BFS on the
reordered graph is then checked like any other graph, and its depths must be the
input graph's depths under the renaming.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2607_17106_gb300 as bg

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

RCM_FLAGS = bg.BFS_DEFAULT_FLAGS | bg.BFS_REORDER_RCM


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_17106_gb300 import build
    build.build()
    bg.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _graph(kind):
    if kind == "rmat14":
        n, s, d = graphgen.rmat(14, 16, seed=1)
    elif kind == "rmat16":
        n, s, d = graphgen.rmat(16, 16, seed=3)
    elif kind == "er":
        n, s, d = graphgen.erdos_renyi(30000, 40000, seed=3)  # many small components and isolated vertices
    elif kind == "grid":
        n, s, d = graphgen.grid(200, 150, 0.2, seed=4)  # relabelled, with deletions
    elif kind == "ba":
        n, s, d = graphgen.barabasi_albert(20000, 4, seed=8)
    elif kind == "star":
        n = 9000
        s, d = np.zeros(n - 2, np.int32), np.arange(1, n - 1, dtype=np.int32)  # vertex n-1 isolated
    elif kind == "path":
        n = 3000
        perm = graphgen.permutation(n, seed=5)
        s, d = perm[:-1].astype(np.int32), perm[1:].astype(np.int32)
    elif kind == "one":
        n, s, d = 1, np.zeros(0, np.int32), np.zeros(0, np.int32)
    else:
        n, s, d = 2, np.array([1], np.int32), np.array([0], np.int32)
    return n, s, d


@pytest.mark.parametrize("kind", ["rmat14", "rmat16", "er", "grid", "ba", "star", "path", "one", "edge"])
def test_rcm_permutation_and_csr_equal_oracle(kind):
    n, s, d = _graph(kind)
    adj = oracle.build_adjacency(n, s, d)
    want = oracle.rcm(adj)
    g = bg.Graph.build(n, s, d, flags=RCM_FLAGS)
    got = g.permutation()
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]
    padj = oracle.permute(adj, want)
    rp, col = g.csr()
    assert np.array_equal(rp.astype(np.int64), padj.row_ptr)
    assert np.array_equal(col, padj.col)
    rp2, col2 = g.csr(csc=True)  # symmetric: the d-major copy is the CSR
    assert np.array_equal(rp2, rp) and np.array_equal(col2, col)
    info = g.info()
    assert info.m == adj.m and info.n_isolated == int(np.sum(adj.degree() == 0))


@pytest.mark.parametrize("kind", ["rmat14", "grid", "ba"])
def test_bfs_on_reordered_graph(kind):
    n, s, d = _graph(kind)
    adj = oracle.build_adjacency(n, s, d)
    g = bg.Graph.build(n, s, d, flags=RCM_FLAGS)
    newid = g.permutation()
    padj = oracle.permute(adj, newid)
    srcs = graphgen.sample_sources(n, s, d, 4, seed=21)
    nsrc = newid[np.asarray(srcs)]
    for o in (bg.options(batch=0), bg.options(batch=1), bg.options(batch=0, mode=bg.BFS_MODE_GRAPH)):
        depth = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        parent = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        g.run(nsrc, depth, parent, o)
        g.sync()
        dd, pp = depth.cpu().numpy(), parent.cpu().numpy()
        for j, sj in enumerate(srcs):
            ref, _ = oracle.bfs(padj, int(nsrc[j]), with_parent=False)
            assert np.array_equal(dd[j], ref)
            assert oracle.validate(padj, int(nsrc[j]), dd[j], pp[j]) == 0
            orig, _ = oracle.bfs(adj, int(sj), with_parent=False)
            assert np.array_equal(dd[j][newid], orig)  # depth of v is the depth of newid[v]


def test_rcm_errors_and_identity_permutation():
    n, s, d = _graph("path")
    with pytest.raises(bg.BfsError) as e:
        bg.Graph.build(n, s, d, flags=(bg.BFS_DEFAULT_FLAGS & ~bg.BFS_SYMMETRIZE) | bg.BFS_REORDER_RCM)
    assert e.value.status == bg.BFS_EINVAL
    g = bg.Graph.build(n, s, d)
    assert np.array_equal(g.permutation(), np.arange(n))
    # device destination
    gr = bg.Graph.build(n, s, d, flags=RCM_FLAGS)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    bg.load().bfs_graph_permutation(gr.handle, bg._ptr(out), bg._stream(None))
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), gr.permutation())


# ------------------------------------------------------- hubs-first pull rows
def _hubs_first_rows(adjt, outdeg):
    """Rows of the d-major adjacency ordered by the entry's out-degree, descending, ties by id."""
    cols = []
    for v in range(adjt.n):
        row = adjt.col[adjt.row_ptr[v]:adjt.row_ptr[v + 1]]
        cols.append(row[np.lexsort((row, -outdeg[row]))])
    return np.concatenate(cols) if cols else np.zeros(0, np.int32)


@pytest.mark.parametrize("kind", ["rmat14", "ba", "grid", "directed", "rcm"])
def test_pull_hubs_first_rows_and_bfs(kind):
    directed = kind == "directed"
    if directed:
        n, s, d = graphgen.rmat(12, 8, seed=21)
        flags = bg.BFS_DEDUP | bg.BFS_DROP_SELF | bg.BFS_BUILD_CSC | bg.BFS_PULL_HUBS_FIRST
        adj = oracle.build_adjacency(n, s, d, symmetrize=False)
        adjt = oracle.build_adjacency(n, d, s, symmetrize=False)
    else:
        n, s, d = _graph("rmat14" if kind == "rcm" else kind)
        flags = RCM_FLAGS | bg.BFS_PULL_HUBS_FIRST if kind == "rcm" else bg.BFS_DEFAULT_FLAGS | bg.BFS_PULL_HUBS_FIRST
        adj = oracle.build_adjacency(n, s, d)
        if kind == "rcm":
            adj = oracle.permute(adj, oracle.rcm(adj))
        adjt = adj
    g = bg.Graph.build(n, s, d, flags=flags)
    rp, col = g.csr()
    assert np.array_equal(rp.astype(np.int64), adj.row_ptr) and np.array_equal(col, adj.col)  # CSR ascending
    rpt, colt = g.csr(csc=True)
    assert np.array_equal(rpt.astype(np.int64), adjt.row_ptr)
    assert np.array_equal(colt, _hubs_first_rows(adjt, adj.degree()))
    newid = g.permutation()
    srcs = newid[np.asarray(graphgen.sample_sources(n, s, d, 4, seed=23))]
    opts = [bg.options(batch=0), bg.options(batch=0, policy=bg.BFS_POLICY_PULL),
            bg.options(batch=0, policy=bg.BFS_POLICY_PULL, mode=bg.BFS_MODE_GRAPH), bg.options(batch=1),
            bg.options(batch=1, policy=bg.BFS_POLICY_PULL)]
    for o in opts:
        depth = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        parent = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        g.run(srcs, depth, parent, o)
        g.sync()
        dd, pp = depth.cpu().numpy(), parent.cpu().numpy()
        for j, sj in enumerate(srcs):
            ref, _ = oracle.bfs(adj, int(sj), with_parent=False)
            assert np.array_equal(dd[j], ref)
            assert oracle.validate(adj, int(sj), dd[j], pp[j], directed=directed) == 0
    if directed:
        return  # the statistics' closed form for s_u is exact on symmetric graphs only
    # level statistics stay those of the ascending rows
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    g.run(srcs[:1], depth, None, bg.options(batch=0))
    g.sync()
    got = g.level_stats(depth)
    want = oracle.level_stats(adj, depth.cpu().numpy())
    assert np.array_equal(got, want)
