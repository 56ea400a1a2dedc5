"""CPU oracle for the BFS hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library never loads it, and it shares no
code with the CUDA path: it is built from ``oracle.c`` alone by gcc.

Functions (each follows the passage cited in ``oracle.c``):
  build_adjacency  Cascade 1, Eq. G; Sections 3 and 4.C (CSR, symmetric edges)
  bfs              Cascade 1 (init, Eq. advance, Eq. update, stop rule)
  level_stats      per-level f, e_f, u, s_u, d_new, e_u of Cascade 1 / Section 5
  apsp_boolean     independent pin: Boolean matrix powers (n <= 64)
  components       independent pin: union-find
  validate         Graph500-style depth/parent checks
  min_label        connected components as the fixed point of min-label
                   propagation (the min operator in place of ANY)
  rcm, permute     Reverse Cuthill-McKee numbering (Section 7.1 preprocessing)
                   with fixed tie breaks, and the renamed adjacency
  mlp_*, adam_step FP64 reference of the learned direction policy (no paper
                   counterpart; pinned by finite differences in the tests)

Parity status: depth pinned (brute force, closed forms, invariants); RCM
pinned by hand-derived orders and a declarative check of the Cuthill-McKee rules;
parent pinned by validation (not unique); MLP pinned by finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

N_IN, N_HID, N_OUT = 10, 32, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc -O2, no vector intrinsics)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.or_build_adjacency.argtypes = [i64, i64, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
        lib.or_build_adjacency.restype = i64
        lib.or_bfs.argtypes = [i64, vp, vp, ctypes.c_int32, vp, vp]
        lib.or_bfs.restype = ctypes.c_int32
        lib.or_level_stats.argtypes = [i64, vp, vp, vp, ctypes.c_int32, vp]
        lib.or_level_stats.restype = ctypes.c_int32
        lib.or_apsp_boolean.argtypes = [ctypes.c_int32, vp, vp]
        lib.or_apsp_boolean.restype = ctypes.c_int
        lib.or_components.argtypes = [i64, i64, vp, vp, vp]
        lib.or_rcm.argtypes = [i64, vp, vp, vp]
        lib.or_min_label.argtypes = [i64, vp, vp, vp]
        lib.or_min_label.restype = ctypes.c_int
        lib.or_rcm.restype = ctypes.c_int
        lib.or_components.restype = ctypes.c_int
        lib.or_validate.argtypes = [i64, vp, vp, ctypes.c_int32, vp, vp, ctypes.c_int]
        lib.or_validate.restype = ctypes.c_int
        lib.or_mlp_num_params.argtypes = []
        lib.or_mlp_num_params.restype = ctypes.c_int32
        lib.or_mlp_forward.argtypes = [vp, vp, i64, vp]
        lib.or_mlp_forward.restype = ctypes.c_int
        lib.or_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp, vp]
        lib.or_mlp_loss_grad.restype = ctypes.c_int
        lib.or_mlp_regress_loss_grad.argtypes = [vp, vp, vp, i64, vp, vp]
        lib.or_mlp_regress_loss_grad.restype = ctypes.c_int
        lib.or_adam_step.argtypes = [vp, vp, vp, vp, i64, i64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double]
        lib.or_adam_step.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Adjacency:
    """Sorted CSR adjacency: row_ptr (int64, n+1) and col (int32)."""

    def __init__(self, n, row_ptr, col):
        self.n = int(n)
        self.row_ptr = row_ptr
        self.col = col

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def build_adjacency(n, src, dst, symmetrize=True, drop_self=True, dedup=True) -> Adjacency:
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    row_ptr = np.empty(n + 1, np.int64)
    col = np.empty(max(1, 2 * len(src)), np.int32)
    m = _load().or_build_adjacency(n, len(src), _ptr(src), _ptr(dst), int(symmetrize), int(drop_self),
                                   int(dedup), _ptr(row_ptr), _ptr(col))
    if m < 0:
        raise ValueError("bad edge list")
    return Adjacency(n, row_ptr, col[:m].copy())


def bfs(adj: Adjacency, s: int, with_parent=True):
    depth = np.empty(adj.n, np.int32)
    parent = np.empty(adj.n, np.int32) if with_parent else None
    lv = _load().or_bfs(adj.n, _ptr(adj.row_ptr), _ptr(adj.col), int(s), _ptr(depth), _ptr(parent))
    if lv < 0:
        raise ValueError("bad source")
    return depth, parent


def level_stats(adj: Adjacency, depth, max_levels=1 << 16) -> np.ndarray:
    """int64 [levels][6]: f, e_f, u, s_u, d_new, e_u per level (see oracle.c)."""
    depth = np.ascontiguousarray(depth, np.int32)
    out = np.zeros((max_levels, 6), np.int64)
    lv = _load().or_level_stats(adj.n, _ptr(adj.row_ptr), _ptr(adj.col), _ptr(depth), max_levels, _ptr(out))
    if lv < 0:
        raise ValueError("too many levels")
    return out[:lv].copy()


def apsp_boolean(n, src, dst, symmetrize=True) -> np.ndarray:
    """Hop distances for n <= 64 by Boolean matrix powers (self-loops ignored)."""
    adj = np.zeros(n, np.uint64)
    for s, d in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if s == d:
            continue
        adj[s] |= np.uint64(1) << np.uint64(d)
        if symmetrize:
            adj[d] |= np.uint64(1) << np.uint64(s)
    dist = np.empty(n * n, np.int32)
    if _load().or_apsp_boolean(n, _ptr(adj), _ptr(dist)):
        raise ValueError("n must be in 1..64")
    return dist.reshape(n, n)


def components(n, src, dst) -> np.ndarray:
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    comp = np.empty(n, np.int32)
    _load().or_components(n, len(src), _ptr(src), _ptr(dst), _ptr(comp))
    return comp


def min_label(adj: Adjacency) -> np.ndarray:
    """Fixed point of min-label propagation: smallest vertex id of each vertex's component (int32 [n])."""
    label = np.empty(adj.n, np.int32)
    if _load().or_min_label(adj.n, _ptr(adj.row_ptr), _ptr(adj.col), _ptr(label)) != 0:
        raise MemoryError("or_min_label")
    return label


def rcm(adj: Adjacency) -> np.ndarray:
    """Reverse Cuthill-McKee new id of every vertex (int32 [n]); tie rules in oracle.c."""
    newid = np.empty(adj.n, np.int32)
    if _load().or_rcm(adj.n, _ptr(adj.row_ptr), _ptr(adj.col), _ptr(newid)) != 0:
        raise MemoryError("or_rcm")
    return newid


def permute(adj: Adjacency, newid) -> Adjacency:
    """The same graph with vertex v renamed newid[v] (rows sorted ascending)."""
    newid = np.asarray(newid, np.int64)
    deg = adj.degree()
    rows = np.repeat(np.arange(adj.n, dtype=np.int64), deg)
    src = newid[rows].astype(np.int32)
    dst = newid[adj.col.astype(np.int64)].astype(np.int32)
    return build_adjacency(adj.n, src, dst, symmetrize=False, drop_self=False, dedup=False)


def validate(adj: Adjacency, s, depth, parent=None, directed=False) -> int:
    depth = np.ascontiguousarray(depth, np.int32)
    parent = None if parent is None else np.ascontiguousarray(parent, np.int32)
    return int(_load().or_validate(adj.n, _ptr(adj.row_ptr), _ptr(adj.col), int(s), _ptr(depth),
                                   _ptr(parent), int(directed)))


def mlp_num_params() -> int:
    return int(_load().or_mlp_num_params())


def mlp_forward(params, X) -> np.ndarray:
    params = np.ascontiguousarray(params, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, N_IN)
    out = np.empty((X.shape[0], N_OUT), np.float64)
    _load().or_mlp_forward(_ptr(params), _ptr(X), X.shape[0], _ptr(out))
    return out


def mlp_loss_grad(params, X, y):
    params = np.ascontiguousarray(params, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, N_IN)
    y = np.ascontiguousarray(y, np.int32)
    loss = np.zeros(1, np.float64)
    grad = np.empty(mlp_num_params(), np.float64)
    _load().or_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(y), X.shape[0], _ptr(loss), _ptr(grad))
    return float(loss[0]), grad


def mlp_regress_loss_grad(params, X, t):
    """Mean over rows of sum_j (z_j - t_j)^2 / 2 for the network outputs z, and its gradient."""
    params = np.ascontiguousarray(params, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, N_IN)
    t = np.ascontiguousarray(t, np.float64).reshape(-1, N_OUT)
    assert t.shape[0] == X.shape[0]
    loss = np.zeros(1, np.float64)
    grad = np.empty(mlp_num_params(), np.float64)
    _load().or_mlp_regress_loss_grad(_ptr(params), _ptr(X), _ptr(t), X.shape[0], _ptr(loss), _ptr(grad))
    return float(loss[0]), grad


def adam_step(params, m1, m2, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place FP64 Adam update of params, m1, m2 (all float64 arrays)."""
    g = np.ascontiguousarray(grad, np.float64)
    _load().or_adam_step(_ptr(params), _ptr(m1), _ptr(m2), _ptr(g), len(params), int(t), lr, beta1, beta2, eps)
