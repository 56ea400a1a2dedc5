"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

import paper_2607_17106_gb300 as bg
from paper_2607_17106_gb300 import build as bgbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfs.h")


@pytest.fixture(scope="module")
def lib():
    bgbuild.build()
    return bg.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(bfs_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    assert "bfs_build_graph" in names and "bfs_run" in names and "bfs_run_mixed" in names
    assert sorted(names) == sorted(bg.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_options_layout_matches_c(lib):
    o = bg.options()
    assert o.struct_size == ctypes.sizeof(bg.bfs_options)
    assert (o.alpha, o.beta, o.gamma) == (14.0, 48.0, 16.0)
    assert (o.batch_alpha, o.batch_beta) == (4.0, 48.0)
    assert o.chunk == 1024 and o.block_threads == 1024 and o.batch == 1 and o.claim_aggregate == 0
    assert o.push_filter == bg.BFS_PUSH_FUSED
    assert o.frontier_sort == bg.BFS_SORT_NONE
    assert o.small_levels == bg.BFS_SMALL_AUTO
    assert o.pull_serial == 16
    assert ctypes.sizeof(bg.bfs_level_record) == 40
    assert ctypes.sizeof(bg.bfs_graph_stats) == 48


def test_status_strings_and_argument_errors_need_no_gpu(lib):
    assert lib.bfs_status_string(bg.BFS_EINVAL) == b"invalid argument"
    assert lib.bfs_status_string(bg.BFS_ETIMEOUT) == b"device wait timed out"
    assert b"sm_103a" in lib.bfs_version()
    h = ctypes.c_void_p()
    # rejected before any CUDA call
    assert lib.bfs_build_graph(0, 0, None, None, 15, None, ctypes.byref(h)) == bg.BFS_EINVAL
    assert b"n must be positive" in lib.bfs_last_error()
    assert lib.bfs_build_graph(5, -1, None, None, 15, None, ctypes.byref(h)) == bg.BFS_EINVAL
    assert lib.bfs_run(None, None, 1, None, None, None, None) == bg.BFS_EINVAL
    with pytest.raises(bg.BfsError):
        bg._check(lib.bfs_run(None, None, 1, None, None, None, None))
    # the reordering flag needs a symmetric build; the later entry points check their arguments
    src = (ctypes.c_int32 * 2)(0, 1)
    dst = (ctypes.c_int32 * 2)(1, 2)
    assert lib.bfs_build_graph(3, 2, src, dst, bg.BFS_DEDUP | bg.BFS_REORDER_RCM, None, ctypes.byref(h)) == bg.BFS_EINVAL
    assert b"BFS_SYMMETRIZE" in lib.bfs_last_error()
    assert lib.bfs_components(None, None, None, None) == bg.BFS_EINVAL
    assert lib.bfs_graph_permutation(None, None, None) == bg.BFS_EINVAL


def test_library_has_no_oracle_dependency():
    # the product binding never imports the oracle package
    src = open(os.path.join(ROOT, "paper_2607_17106_gb300", "__init__.py")).read()
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)
    for f in os.listdir(os.path.join(ROOT, "paper_2607_17106_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2607_17106_gb300", "csrc", f)).read()
