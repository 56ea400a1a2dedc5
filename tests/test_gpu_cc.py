"""GPU parity of connected components by min-label propagation.

The fixed point is unique (the smallest vertex id of each component), so the
device labels must equal the oracle's element by element.
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


def _case(kind):
    if kind == "rmat14":
        return graphgen.rmat(14, 16, seed=1)
    if kind == "rmat-sparse":
        return graphgen.rmat(15, 2, seed=9)  # many small components
    if kind == "er":
        return graphgen.erdos_renyi(40000, 30000, seed=3)
    if kind == "grid":
        return graphgen.grid(300, 200, 0.45, seed=4)  # near the percolation threshold
    if kind == "ba":
        return graphgen.barabasi_albert(30000, 1, seed=8)
    if kind == "star":
        n = 70001  # hub row of 70000 entries: chunk units
        return n, np.full(n - 2, 5, np.int32), np.array([v for v in range(n) if v not in (5, n - 1)], np.int32)
    if kind == "path":
        n = 5000  # ~n iterations of the propagation
        perm = graphgen.permutation(n, seed=5)
        return n, perm[:-1].astype(np.int32), perm[1:].astype(np.int32)
    if kind == "noedges":
        return 77, np.zeros(0, np.int32), np.zeros(0, np.int32)
    return 1, np.zeros(0, np.int32), np.zeros(0, np.int32)


@pytest.mark.parametrize("kind", ["rmat14", "rmat-sparse", "er", "grid", "ba", "star", "path", "noedges", "one"])
def test_components_equal_oracle(kind):
    n, s, d = _case(kind)
    adj = oracle.build_adjacency(n, s, d)
    want = oracle.min_label(adj)
    g = bg.Graph.build(n, s, d)
    got, iters = g.components()
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]
    assert iters >= (1 if adj.m else 0)
    dev = torch.empty(n, dtype=torch.int32, device="cuda")  # device destination
    g.components(dev)
    assert np.array_equal(dev.cpu().numpy(), want)


def test_components_on_reordered_graph_and_errors():
    n, s, d = _case("rmat-sparse")
    adj = oracle.build_adjacency(n, s, d)
    gr = bg.Graph.build(n, s, d, flags=bg.BFS_DEFAULT_FLAGS | bg.BFS_REORDER_RCM)
    got, _ = gr.components()
    assert np.array_equal(got, oracle.min_label(oracle.permute(adj, gr.permutation())))
    gd = bg.Graph.build(n, s, d, flags=bg.BFS_DEDUP | bg.BFS_BUILD_CSC)  # directed
    with pytest.raises(bg.BfsError) as e:
        gd.components()
    assert e.value.status == bg.BFS_EINVAL
