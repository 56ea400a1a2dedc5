"""The no-allocation variant of the level statistics, through the C ABI.

bfs_level_stats_noalloc serves callers that may not allocate memory while
they run (their device memory is reserved up front, or allocation is audited
after start-up): it keeps its scratch in a fixed-size device array of the
library.  Its table must equal the allocating bfs_level_stats exactly (the
statistics are integer counts), on two calls in a row -- the second call
starts from the scratch the first one left behind.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_2607_17106_gb300 as bg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(lib, g, depth, max_levels):
    out = np.full((max_levels, 6), -7, np.int64)
    lv = ctypes.c_int32(-1)
    rc = lib.bfs_level_stats_noalloc(g.handle, depth.data_ptr(), max_levels, out.ctypes.data, ctypes.byref(lv),
                                     torch.cuda.current_stream().cuda_stream)
    return rc, out[: max(lv.value, 0)].copy()


def test_no_alloc_level_stats_equal_the_allocating_call():
    from paper_2607_17106_gb300 import build
    build.build()
    lib = bg.load()
    n, s, d = graphgen.rmat(15, 16, seed=3)
    g = bg.Graph.build(n, s, d)
    srcs = graphgen.sample_sources(n, s, d, 2, seed=17)
    depth = torch.empty((2, n), dtype=torch.int32, device="cuda")
    g.run(srcs, depth, None, bg.options(batch=0))
    g.sync()
    for j in (0, 1):  # two calls in a row, different searches
        ref = g.level_stats(depth[j])
        rc, got = _noalloc(lib, g, depth[j], 4096)
        assert rc == bg.BFS_OK, lib.bfs_last_error()
        assert got.shape == ref.shape and np.array_equal(got, ref)
    # a longer search (a path: one level per vertex) and the size limit
    m = 3000
    gp = bg.Graph.build(m, np.arange(m - 1, dtype=np.int32), np.arange(1, m, dtype=np.int32))
    dp = torch.empty(m, dtype=torch.int32, device="cuda")
    gp.run(np.array([0], np.int32), dp, None, bg.options(batch=0))
    gp.sync()
    rc, got = _noalloc(lib, gp, dp, 4096)
    assert rc == bg.BFS_OK and np.array_equal(got, gp.level_stats(dp))
    rc, _ = _noalloc(lib, gp, dp, 4097)
    assert rc == bg.BFS_ERANGE
    rc, _ = _noalloc(lib, gp, dp, 100)  # 3000 levels do not fit in 100
    assert rc == bg.BFS_ERANGE
