"""Seeded synthetic graph inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only *generates* edge lists and source vertices; it contains no BFS
arithmetic (no symmetrising, deduplication, CSR construction or traversal).  All
randomness is Philox-4x32-10 keyed by (seed, stream, index), so outputs are
identical on every machine and thread count.

The named workloads in :data:`WORKLOADS` are the synthetic stand-ins for the
paper's dataset groups (Section 7.1): RMAT/Kronecker for high degree variance,
Barabasi-Albert for mid, Erdos-Renyi and perturbed grids for low variance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, no arch flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, i32p, i32p, ctypes.c_int]
        lib.gg_rmat.restype = ctypes.c_int
        lib.gg_erdos_renyi.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, i32p, i32p,
                                       ctypes.c_int]
        lib.gg_erdos_renyi.restype = ctypes.c_int
        lib.gg_grid_num_edges.argtypes = [ctypes.c_int64, ctypes.c_int64]
        lib.gg_grid_num_edges.restype = ctypes.c_int64
        lib.gg_grid.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                ctypes.c_int, i32p, i32p, ctypes.c_int]
        lib.gg_grid.restype = ctypes.c_int64
        lib.gg_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, i32p]
        lib.gg_permutation.restype = ctypes.c_int
        lib.gg_barabasi_albert.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
        lib.gg_barabasi_albert.restype = ctypes.c_int64
        lib.gg_sample_sources.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p, ctypes.c_int32,
                                          ctypes.c_uint64, i32p]
        lib.gg_sample_sources.restype = ctypes.c_int
        lib.gg_philox_word.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_int]
        lib.gg_philox_word.restype = ctypes.c_uint32
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def philox_word(seed: int, index: int, stream: int, sub: int, which: int) -> int:
    """One 32-bit output word of Philox-4x32-10 for counter (index, stream, sub)."""
    return int(_load().gg_philox_word(seed, index, stream, sub, which))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1):
    """RMAT edge list: edge_factor * 2**scale tuples, `scale` quadrant draws each."""
    m = edge_factor * (1 << scale)
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gg_rmat(scale, m, a, b, c, seed, _p(src), _p(dst), _threads())
    if rc:
        raise ValueError("bad RMAT parameters")
    return 1 << scale, src, dst


def erdos_renyi(n: int, m_pairs: int, seed: int):
    """G(n, M): M ordered pairs with endpoints uniform in [0, n)."""
    src = np.empty(m_pairs, np.int32)
    dst = np.empty(m_pairs, np.int32)
    if _load().gg_erdos_renyi(n, m_pairs, seed, _p(src), _p(dst), _threads()):
        raise ValueError("bad Erdos-Renyi parameters")
    return n, src, dst


def grid(width: int, height: int, p_del: float, seed: int, relabel: bool = True):
    """4-neighbour width x height grid, edges deleted with prob. p_del, vertices relabelled."""
    lib = _load()
    cap = lib.gg_grid_num_edges(width, height)
    src = np.empty(cap, np.int32)
    dst = np.empty(cap, np.int32)
    m = lib.gg_grid(width, height, p_del, seed, 1 if relabel else 0, _p(src), _p(dst), _threads())
    if m < 0:
        raise ValueError("bad grid parameters")
    return width * height, src[:m].copy(), dst[:m].copy()


def permutation(n: int, seed: int) -> np.ndarray:
    """The seeded Fisher-Yates permutation the grid generator relabels with."""
    perm = np.empty(n, np.int32)
    if _load().gg_permutation(n, seed, _p(perm)):
        raise ValueError("bad permutation size")
    return perm


def barabasi_albert(n: int, m: int, seed: int):
    """Preferential attachment (Batagelj-Brandes), m edges per new vertex, (m+1)-clique start."""
    cap = m * (m + 1) // 2 + (n - m - 1) * m
    src = np.empty(cap, np.int32)
    dst = np.empty(cap, np.int32)
    e = _load().gg_barabasi_albert(n, m, seed, _p(src), _p(dst))
    if e < 0:
        raise ValueError("bad Barabasi-Albert parameters")
    return n, src[:e], dst[:e]


def sample_sources(n: int, src: np.ndarray, dst: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k distinct seeded vertices that have at least one non-self-loop edge."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    out = np.empty(max(k, 1), np.int32)
    rc = _load().gg_sample_sources(n, len(src), _p(src), _p(dst), k, seed, _p(out))
    if rc == 2:
        raise ValueError("fewer than k vertices with degree > 0")
    if rc:
        raise ValueError("bad source-sampling arguments")
    return out[:k].copy()


@dataclass(frozen=True)
class Workload:
    """A named synthetic graph + source recipe."""
    name: str
    kind: str                    # "rmat" | "er" | "grid" | "ba"
    params: dict = field(default_factory=dict)
    seed: int = 1
    n_sources: int = 16
    source_seed: int = 101

    def edges(self):
        p = self.params
        if self.kind == "rmat":
            return rmat(p["scale"], p.get("edge_factor", 16), p.get("a", 0.57), p.get("b", 0.19),
                        p.get("c", 0.19), self.seed)
        if self.kind == "er":
            return erdos_renyi(p["n"], p["m_pairs"], self.seed)
        if self.kind == "grid":
            return grid(p["width"], p["height"], p.get("p_del", 0.0), self.seed, p.get("relabel", True))
        if self.kind == "ba":
            return barabasi_albert(p["n"], p["m"], self.seed)
        raise ValueError(self.kind)

    def sources(self, n, src, dst, k: int | None = None):
        return sample_sources(n, src, dst, self.n_sources if k is None else k, self.source_seed)


def _rmat_w(name, scale, ef=16, a=0.57, b=0.19, c=0.19, seed=1, ns=16, ss=101):
    return Workload(name, "rmat", dict(scale=scale, edge_factor=ef, a=a, b=b, c=c), seed, ns, ss)


WORKLOADS = {
    # small single-source push case (16,384 vertices)
    "rmat-s14-ef16": _rmat_w("rmat-s14-ef16", 14, seed=1, ns=16, ss=101),
    # direction-optimising pair, 64 sources each
    "rmat-s22-ef16": _rmat_w("rmat-s22-ef16", 22, seed=2, ns=64, ss=102),
    "er-n22-deg16": Workload("er-n22-deg16", "er", dict(n=1 << 22, m_pairs=8 << 22), 3, 64, 103),
    # long-diameter grid
    "grid-4096-del10": Workload("grid-4096-del10", "grid", dict(width=4096, height=4096, p_del=0.1),
                                4, 32, 104),
    # batched MS-BFS
    "rmat-s24-ef16": _rmat_w("rmat-s24-ef16", 24, seed=5, ns=64, ss=105),
    # held-out policy evaluation graphs
    "rmat-s23-ef32-a60": _rmat_w("rmat-s23-ef32-a60", 23, ef=32, a=0.60, b=0.175, c=0.175, seed=7,
                                 ns=64, ss=107),
    "ba-n22-m8": Workload("ba-n22-m8", "ba", dict(n=1 << 22, m=8), 8, 64, 108),
}


def mixed_batch(n_queries: int = 256, scales=tuple(range(16, 23)), seed: int = 106):
    """The mixed multi-graph workload: RMAT graphs of the given scales (edge
    factor 16, a=0.57 b=c=0.19, seed = scale) and n_queries queries whose graph
    is drawn uniformly (numpy PCG64, `seed`), sources sampled per graph with
    seed + graph index.  Returns (scales, [(n, src, dst)], graph_of_query, sources)."""
    scales = list(scales)
    graphs = [rmat(sc, 16, seed=sc) for sc in scales]
    goq = np.random.default_rng(seed).integers(0, len(scales), n_queries).astype(np.int32)
    srcs = np.zeros(n_queries, np.int32)
    for gi, (n, s, d) in enumerate(graphs):
        idx = np.flatnonzero(goq == gi)
        if len(idx):
            srcs[idx] = sample_sources(n, s, d, len(idx), seed + gi)
    return scales, graphs, goq, srcs
