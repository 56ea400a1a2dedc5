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


def _driver_pool():
    """The device's default stream-ordered memory pool through the driver API
    (the pool cudaMallocAsync draws from), or None where libcuda is absent."""
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return None, None
    dev = ctypes.c_int(0)
    pool = ctypes.c_void_p()
    if cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) != 0:
        return None, None
    if cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) != 0:
        return None, None
    return cu, pool


def _pool_attr(cu, pool, attr):
    v = ctypes.c_uint64(0)
    assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


USED_CURRENT, USED_HIGH = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH


def test_no_alloc_call_allocates_nothing():
    # around two calls: the default pool's high-water mark (reset before the
    # calls) stays at what was in use, device free memory is unchanged, and
    # torch's allocator saw no allocation; the allocating call, between the
    # same resets, does raise the mark (the probe is not blind)
    lib = bg.load()
    n, s, d = graphgen.rmat(14, 16, seed=5)
    g = bg.Graph.build(n, s, d)
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    g.run(graphgen.sample_sources(n, s, d, 1, seed=3), depth, None, bg.options(batch=0))
    g.sync()
    rc, ref = _noalloc(lib, g, depth, 64)  # first call on the device: symbol lookup
    assert rc == bg.BFS_OK
    cu, pool = _driver_pool()
    if cu is None:
        pytest.skip("driver API not loadable")
    zero = ctypes.c_uint64(0)
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    free0, _ = torch.cuda.mem_get_info()
    used0 = _pool_attr(cu, pool, USED_CURRENT)
    assert cu.cuMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
    for _ in range(2):
        rc, got = _noalloc(lib, g, depth, 64)
        assert rc == bg.BFS_OK and np.array_equal(got, ref)
    torch.cuda.synchronize()
    assert _pool_attr(cu, pool, USED_HIGH) <= used0
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
    # positive control: the allocating call draws scratch from that pool
    assert cu.cuMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
    assert np.array_equal(g.level_stats(depth, max_levels=64), ref)
    assert _pool_attr(cu, pool, USED_HIGH) > used0
    g.free()
