"""Thin Python binding of libbfsgb (the C ABI in include/bfs.h).

Argument marshalling only: every step of a search runs in the library's CUDA
kernels.  PyTorch supplies device memory (``tensor.data_ptr()``) and streams
(``torch.cuda.current_stream().cuda_stream``); plain NumPy arrays are accepted
as host buffers.  The library is loaded on first use and there is no fallback:
if ``libbfsgb.so`` is missing or fails to load, every call raises.

Level-synchronous BFS of the paper's Cascade 1 (Section 3): each level is a
masked Boolean SpMSpV, run in push form (CSR expand of the frontier) or pull
form (Section 5: unvisited vertices scan in-neighbours with early exit).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfsgb.so")

# status codes
BFS_OK, BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA, BFS_ETIMEOUT, BFS_ERANGE, BFS_EVALIDATE = range(7)
# build flags
BFS_SYMMETRIZE, BFS_DEDUP, BFS_DROP_SELF, BFS_BUILD_CSC, BFS_DEFAULT_FLAGS = 1, 2, 4, 8, 15
BFS_REORDER_RCM, BFS_PULL_HUBS_FIRST = 16, 32
# level forms
BFS_DIR_PUSH_QUEUE, BFS_DIR_PUSH_BITMAP, BFS_DIR_PULL = 0, 1, 2
# drive modes
BFS_MODE_PERSISTENT, BFS_MODE_HOST_LOOP, BFS_MODE_GRAPH = 0, 1, 2
# push advance / visited update arrangements
BFS_PUSH_FUSED, BFS_PUSH_FILTER, BFS_PUSH_FILTER_PREDICATED = 0, 1, 2
# frontier order of push-queue levels
BFS_SORT_NONE, BFS_SORT_DEVICE, BFS_SORT_TILE = 0, 1, 2
BFS_SMALL_AUTO, BFS_SMALL_OFF, BFS_SMALL_CLUSTER = -1, 0, 1
# policies
BFS_POLICY_HEURISTIC, BFS_POLICY_PUSH, BFS_POLICY_PULL, BFS_POLICY_SCHEDULE, BFS_POLICY_MLP = range(5)
BFS_MLP_IN, BFS_MLP_HIDDEN, BFS_MLP_OUT = 10, 32, 3
BFS_MLP_NPARAM, BFS_MLP_NNORM = 1507, 20

EXPORTED = [
    "bfs_build_graph", "bfs_graph_info", "bfs_graph_csr", "bfs_graph_permutation", "bfs_components",
    "bfs_free_graph", "bfs_options_init", "bfs_run",
    "bfs_sync", "bfs_run_mixed", "bfs_level_stats", "bfs_level_stats_noalloc", "bfs_profile_levels",
    "bfs_policy_features", "bfs_policy_load",
    "bfs_policy_weights", "bfs_policy_free", "bfs_policy_forward", "bfs_policy_train_step",
    "bfs_policy_train_step_regress",
    "bfs_policy_set_norm", "bfs_status_string", "bfs_last_error", "bfs_version",
]


class BfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class bfs_graph_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("symmetric", ctypes.c_int32),
                ("n_isolated", ctypes.c_int32), ("deg_max", ctypes.c_int32), ("deg_mean", ctypes.c_double),
                ("deg_var", ctypes.c_double)]


class bfs_level_record(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("dir", ctypes.c_int32), ("f", ctypes.c_int64), ("e_f", ctypes.c_int64),
                ("m_u", ctypes.c_int64), ("t_ns", ctypes.c_int64)]


class bfs_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("mode", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float), ("gamma", ctypes.c_float),
                ("chunk", ctypes.c_int32), ("medium", ctypes.c_int32), ("pull_serial", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("claim_aggregate", ctypes.c_int32), ("barrier_timeout_ns", ctypes.c_int64),
                ("schedule", ctypes.POINTER(ctypes.c_int8)), ("schedule_len", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("mlp", ctypes.c_void_p),
                ("level_log", ctypes.POINTER(bfs_level_record)), ("level_log_cap", ctypes.c_int32),
                ("levels_out", ctypes.POINTER(ctypes.c_int32)), ("batch", ctypes.c_int32),
                ("push_filter", ctypes.c_int32), ("frontier_sort", ctypes.c_int32),
                ("batch_alpha", ctypes.c_float), ("batch_beta", ctypes.c_float), ("small_levels", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libbfsgb.so and declare every exported signature.  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_2607_17106_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    st = ctypes.c_int
    sig = {
        "bfs_build_graph": (st, [i32, i64, vp, vp, u32, vp, ctypes.POINTER(vp)]),
        "bfs_graph_info": (st, [vp, ctypes.POINTER(bfs_graph_stats)]),
        "bfs_graph_csr": (st, [vp, i32, vp, vp, vp]),
        "bfs_graph_permutation": (st, [vp, vp, vp]),
        "bfs_components": (st, [vp, vp, vp, vp]),
        "bfs_free_graph": (None, [vp]),
        "bfs_options_init": (None, [ctypes.POINTER(bfs_options)]),
        "bfs_run": (st, [vp, vp, i32, vp, vp, ctypes.POINTER(bfs_options), vp]),
        "bfs_sync": (st, [vp, vp]),
        "bfs_run_mixed": (st, [ctypes.POINTER(vp), i32, vp, vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp),
                               ctypes.POINTER(bfs_options), vp]),
        "bfs_level_stats": (st, [vp, vp, i32, vp, ctypes.POINTER(i32), vp]),
        "bfs_level_stats_noalloc": (st, [vp, vp, i32, vp, ctypes.POINTER(i32), vp]),
        "bfs_profile_levels": (st, [vp, i32, ctypes.POINTER(bfs_options), i32, i32, vp, vp, vp,
                                    ctypes.POINTER(i32), vp]),
        "bfs_policy_features": (st, [vp, i32, i64, i64, i64, i64, i32, vp]),
        "bfs_policy_load": (st, [vp, i32, ctypes.POINTER(vp)]),
        "bfs_policy_weights": (st, [vp, vp, i32]),
        "bfs_policy_free": (None, [vp]),
        "bfs_policy_forward": (st, [vp, vp, i64, vp, vp]),
        "bfs_policy_train_step": (st, [vp, vp, vp, i64, ctypes.c_float, i32, vp, vp, vp]),
        "bfs_policy_train_step_regress": (st, [vp, vp, vp, i64, ctypes.c_float, i32, vp, vp, vp]),
        "bfs_policy_set_norm": (st, [vp, vp]),
        "bfs_status_string": (ctypes.c_char_p, [st]),
        "bfs_last_error": (ctypes.c_char_p, []),
        "bfs_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != BFS_OK:
        lib = load()
        raise BfsError(status, f"{lib.bfs_status_string(status).decode()}: {lib.bfs_last_error().decode()}")


def _ptr(x):
    """Address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def options(**kw) -> bfs_options:
    """bfs_options with library defaults, then the given fields overridden."""
    o = bfs_options()
    load().bfs_options_init(ctypes.byref(o))
    sched = kw.pop("schedule", None)
    for k, v in kw.items():
        if k == "mlp" and isinstance(v, Policy):
            v = v.handle
        setattr(o, k, v)
    if sched is not None:
        arr = (ctypes.c_int8 * len(sched))(*[int(s) for s in sched])
        o._sched_keep = arr  # keep alive
        o.schedule = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int8))
        o.schedule_len = len(sched)
        if "policy" not in kw:
            o.policy = BFS_POLICY_SCHEDULE
    return o


class Graph:
    """Owning handle of a bfs_graph (device CSR, optional CSC, workspaces)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    @classmethod
    def build(cls, n: int, src, dst, flags: int = BFS_DEFAULT_FLAGS, stream=None) -> "Graph":
        h = ctypes.c_void_p()
        m = len(src)
        _check(load().bfs_build_graph(int(n), int(m), _ptr(src), _ptr(dst), int(flags), _stream(stream),
                                      ctypes.byref(h)))
        return cls(h.value)

    def info(self) -> bfs_graph_stats:
        s = bfs_graph_stats()
        _check(load().bfs_graph_info(self.handle, ctypes.byref(s)))
        return s

    @property
    def n(self) -> int:
        return self.info().n

    @property
    def m(self) -> int:
        return self.info().m

    def csr(self, csc: bool = False):
        """(row_ptr int32[n+1], col int32[m]) copied to host numpy arrays."""
        s = self.info()
        rp = np.empty(s.n + 1, np.int32)
        col = np.empty(max(s.m, 1), np.int32)
        _check(load().bfs_graph_csr(self.handle, int(csc), _ptr(rp), _ptr(col), _stream(None)))
        return rp, col[: s.m]

    def components(self, label=None, stream=None):
        """bfs_components: (label [n] int32, iterations); label host numpy (default) or a device tensor."""
        out = np.empty(self.n, np.int32) if label is None else label
        it = ctypes.c_int32(0)
        _check(load().bfs_components(self.handle, _ptr(out), ctypes.byref(it), _stream(stream)))
        return out, it.value

    def permutation(self) -> np.ndarray:
        """bfs_graph_permutation: int32 [n], new id of every input vertex (identity unless RCM-reordered)."""
        out = np.empty(self.n, np.int32)
        _check(load().bfs_graph_permutation(self.handle, _ptr(out), _stream(None)))
        return out

    def run(self, sources, depth, parent=None, opt: bfs_options | None = None, stream=None):
        """bfs_run: sources (int seq / array / tensor), depth/parent [k][n] buffers."""
        if isinstance(sources, (int, np.integer)):
            sources = np.array([sources], np.int32)
        elif isinstance(sources, (list, tuple)):
            sources = np.array(sources, np.int32)
        k = sources.numel() if hasattr(sources, "numel") else len(sources)
        _check(load().bfs_run(self.handle, _ptr(sources), int(k), _ptr(depth), _ptr(parent),
                              ctypes.byref(opt) if opt is not None else None, _stream(stream)))

    def sync(self, stream=None):
        _check(load().bfs_sync(self.handle, _stream(stream)))

    def level_stats(self, depth, max_levels: int = 1 << 16, stream=None) -> np.ndarray:
        """int64 [levels][6] = f, e_f, u, s_u, d_new, e_u (bfs_level_stats)."""
        out = np.zeros((max_levels, 6), np.int64)
        lv = ctypes.c_int32(0)
        _check(load().bfs_level_stats(self.handle, _ptr(depth), int(max_levels), _ptr(out), ctypes.byref(lv),
                                      _stream(stream)))
        return out[: lv.value].copy()

    def profile_levels(self, source: int, opt: bfs_options | None = None, repeats: int = 3,
                       max_levels: int = 4096, stream=None):
        """(features[L][10], times_us[L][3], taken[L]) of bfs_profile_levels."""
        X = np.zeros((max_levels, BFS_MLP_IN), np.float32)
        T = np.zeros((max_levels, 3), np.float32)
        taken = np.zeros(max_levels, np.int32)
        lv = ctypes.c_int32(0)
        _check(load().bfs_profile_levels(self.handle, int(source), ctypes.byref(opt) if opt is not None else None,
                                         int(repeats), int(max_levels), _ptr(X), _ptr(T), _ptr(taken),
                                         ctypes.byref(lv), _stream(stream)))
        L = lv.value
        return X[:L].copy(), T[:L].copy(), taken[:L].copy()

    def features(self, level, f, e_f, m_u, f_prev, prev_dir) -> np.ndarray:
        x = np.empty(BFS_MLP_IN, np.float32)
        _check(load().bfs_policy_features(self.handle, int(level), int(f), int(e_f), int(m_u), int(f_prev),
                                          int(prev_dir), _ptr(x)))
        return x

    def free(self):
        if self.handle and self.handle.value:
            load().bfs_free_graph(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def run_mixed(graphs, graph_of_query, sources, depth_ptrs, parent_ptrs=None, opt=None, stream=None):
    """bfs_run_mixed over a list of Graph; depth_ptrs/parent_ptrs: device pointers (or tensors)."""
    ng = len(graphs)
    garr = (ctypes.c_void_p * ng)(*[g.handle.value for g in graphs])
    goq = np.ascontiguousarray(graph_of_query, np.int32)
    src = np.ascontiguousarray(sources, np.int32)
    nq = len(src)
    darr = (ctypes.c_void_p * nq)(*[_ptr(d) for d in depth_ptrs])
    parr = None
    if parent_ptrs is not None:
        parr = (ctypes.c_void_p * nq)(*[_ptr(p) for p in parent_ptrs])
    _check(load().bfs_run_mixed(garr, ng, _ptr(goq), _ptr(src), nq, darr, parr,
                                ctypes.byref(opt) if opt is not None else None, _stream(stream)))


class Policy:
    """Learned direction policy (FP32 MLP 10-32-32-3) held by the library."""

    def __init__(self, weights):
        w = np.ascontiguousarray(weights, np.float32)
        h = ctypes.c_void_p()
        _check(load().bfs_policy_load(_ptr(w), len(w), ctypes.byref(h)))
        self.handle = h

    def weights(self) -> np.ndarray:
        out = np.empty(BFS_MLP_NPARAM + BFS_MLP_NNORM, np.float32)
        _check(load().bfs_policy_weights(self.handle, _ptr(out), len(out)))
        return out

    def set_norm(self, mean, inv_std):
        a = np.ascontiguousarray(np.concatenate([mean, inv_std]), np.float32)
        _check(load().bfs_policy_set_norm(self.handle, _ptr(a)))

    def forward(self, X, logits, rows: int, stream=None):
        _check(load().bfs_policy_forward(self.handle, _ptr(X), int(rows), _ptr(logits), _stream(stream)))

    def train_step(self, X, y, rows: int, lr: float, step: int, grad_out=None, stream=None) -> float:
        loss = np.zeros(1, np.float32)
        _check(load().bfs_policy_train_step(self.handle, _ptr(X), _ptr(y), int(rows), float(lr), int(step),
                                            _ptr(loss), _ptr(grad_out), _stream(stream)))
        return float(loss[0])

    def train_step_regress(self, X, target, rows: int, lr: float, step: int, grad_out=None, stream=None) -> float:
        """One Adam step of least-squares regression of the outputs on target (device float [rows][3])."""
        loss = np.zeros(1, np.float32)
        _check(load().bfs_policy_train_step_regress(self.handle, _ptr(X), _ptr(target), int(rows), float(lr),
                                                    int(step), _ptr(loss), _ptr(grad_out), _stream(stream)))
        return float(loss[0])

    def free(self):
        if self.handle and self.handle.value:
            load().bfs_policy_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def version() -> str:
    return load().bfs_version().decode()
