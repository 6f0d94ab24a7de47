"""Seeded synthetic graph inputs shared by the oracle tests, the CUDA tests and the bench.

Input generation only: splitmix64 counter-based draws, RMAT / uniform edge
sampling, CSR assembly with self-loop and duplicate removal, symmetrisation,
edge weights and root selection.  Nothing in here computes any step of the
partition-centric method.

Seeds follow one fixed recipe so every consumer sees the same graph:
graph seed = 0x9E3779B97F4A7C15 ^ scale (RMAT) or ^ (scale | 1<<32) (uniform),
weights and roots draw from their own streams.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None

GRAPH_SEED = 0x9E3779B97F4A7C15
WEIGHT_SEED = 0x5EEDF00DCAFEBEEF
ROOT_SEED = 0x0123456789ABCDEF


def build(force: bool = False) -> str:
    """Compiles the generator shared object in place (gcc, OpenMP if available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O3", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _SO + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gg_splitmix64_at.restype = ctypes.c_uint64
            lib.gg_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_splitmix64_fill.restype = None
            lib.gg_splitmix64_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p]
            lib.gg_rmat_edges.restype = None
            lib.gg_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, u32p, u32p]
            lib.gg_uniform_edges.restype = None
            lib.gg_uniform_edges.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.gg_build_csr.restype = ctypes.c_uint64
            lib.gg_build_csr.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, u64p, u32p]
            lib.gg_weights.restype = None
            lib.gg_weights.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, i32p]
            lib.gg_roots.restype = ctypes.c_uint32
            lib.gg_roots.argtypes = [ctypes.c_uint32, u64p, ctypes.c_uint32, ctypes.c_uint64, u32p]
            lib.gg_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().gg_splitmix64_fill(seed & (2**64 - 1), start, count, _p(out, ctypes.c_uint64))
    return out


class CSR:
    """A directed graph in CSR form: row_ptr (uint64, V+1), col (uint32, E), optional weights (int32, E)."""

    def __init__(self, num_vertices: int, row_ptr: np.ndarray, col: np.ndarray, weights=None, name: str = ""):
        self.num_vertices = int(num_vertices)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        self.col = np.ascontiguousarray(col, dtype=np.uint32)
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.int32)
        self.name = name
        assert self.row_ptr.shape == (self.num_vertices + 1,)
        assert int(self.row_ptr[-1]) == self.col.shape[0]

    @property
    def num_edges(self) -> int:
        return int(self.col.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.uint64)

    def with_weights(self, hi: int = 255, seed: int = WEIGHT_SEED) -> "CSR":
        w = np.empty(self.num_edges, dtype=np.int32)
        if self.num_edges:
            _load().gg_weights(self.num_edges, seed, hi, _p(w, ctypes.c_int32))
        return CSR(self.num_vertices, self.row_ptr, self.col, w, self.name + "+w")

    def src(self) -> np.ndarray:
        return np.repeat(np.arange(self.num_vertices, dtype=np.uint32), np.diff(self.row_ptr).astype(np.int64))


def from_edges(n: int, src, dst, drop_self: bool = True, dedup: bool = True, symmetrize: bool = False,
               name: str = "") -> CSR:
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    m = src.shape[0]
    row_ptr = np.empty(n + 1, dtype=np.uint64)
    col = np.empty(max(1, m * (2 if symmetrize else 1)), dtype=np.uint32)
    e = _load().gg_build_csr(n, m, _p(src, ctypes.c_uint32), _p(dst, ctypes.c_uint32), int(drop_self),
                             int(dedup), int(symmetrize), _p(row_ptr, ctypes.c_uint64), _p(col, ctypes.c_uint32))
    return CSR(n, row_ptr, col[:e].copy(), name=name)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int | None = None, symmetrize: bool = False) -> CSR:
    """Directed RMAT graph with 2^scale vertices from edge_factor * 2^scale samples (self loops and duplicates removed)."""
    n = 1 << scale
    m = edge_factor * n
    if seed is None:
        seed = GRAPH_SEED ^ scale
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    _load().gg_rmat_edges(scale, m, a, b, c, seed & (2**64 - 1), _p(src, ctypes.c_uint32), _p(dst, ctypes.c_uint32))
    g = from_edges(n, src, dst, symmetrize=symmetrize, name=f"rmat{scale}_ef{edge_factor}" + ("_sym" if symmetrize else ""))
    return g


def uniform(num_vertices: int, num_samples: int, seed: int | None = None, symmetrize: bool = False,
            name: str | None = None) -> CSR:
    """Uniform random directed graph: num_samples (u, v) draws, self loops and duplicates removed."""
    if seed is None:
        seed = GRAPH_SEED ^ (num_vertices | (1 << 32))
    src = np.empty(num_samples, dtype=np.uint32)
    dst = np.empty(num_samples, dtype=np.uint32)
    _load().gg_uniform_edges(num_vertices, num_samples, seed & (2**64 - 1), _p(src, ctypes.c_uint32),
                             _p(dst, ctypes.c_uint32))
    return from_edges(num_vertices, src, dst, symmetrize=symmetrize,
                      name=name or f"uniform{num_vertices}_{num_samples}" + ("_sym" if symmetrize else ""))


def symmetrized(g: CSR) -> CSR:
    return from_edges(g.num_vertices, g.src(), g.col, symmetrize=True, name=g.name + "_sym")


def roots(g: CSR, count: int = 16, seed: int = ROOT_SEED) -> np.ndarray:
    """`count` distinct vertices with out-degree >= 1, drawn from a fixed stream."""
    out = np.empty(count, dtype=np.uint32)
    k = _load().gg_roots(g.num_vertices, _p(g.row_ptr, ctypes.c_uint64), count, seed, _p(out, ctypes.c_uint32))
    return out[:k].copy()


# Small hand graphs ---------------------------------------------------------------------------

def ring(n: int) -> CSR:
    """Directed cycle 0 -> 1 -> ... -> n-1 -> 0."""
    s = np.arange(n, dtype=np.uint32)
    return from_edges(n, s, (s + 1) % n, name=f"ring{n}")


def path(n: int) -> CSR:
    s = np.arange(n - 1, dtype=np.uint32)
    return from_edges(n, s, s + 1, name=f"path{n}")


def complete(n: int) -> CSR:
    """Complete digraph without self loops."""
    s, d = np.meshgrid(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32), indexing="ij")
    return from_edges(n, s.ravel(), d.ravel(), name=f"complete{n}")


def star(n: int, center: int = 0) -> CSR:
    """Symmetrised star: center <-> every other vertex."""
    leaves = np.array([v for v in range(n) if v != center], dtype=np.uint32)
    c = np.full(leaves.shape, center, dtype=np.uint32)
    return from_edges(n, np.concatenate([c, leaves]), np.concatenate([leaves, c]), name=f"star{n}")


def disjoint_rings(sizes) -> CSR:
    """Union of directed rings with consecutive vertex ranges (one component per ring)."""
    srcs, dsts, off = [], [], 0
    for n in sizes:
        s = np.arange(n, dtype=np.uint32)
        srcs.append(s + off)
        dsts.append((s + 1) % n + off)
        off += n
    return from_edges(off, np.concatenate(srcs), np.concatenate(dsts), name="rings" + "_".join(map(str, sizes)))


def multigraph(n: int, src, dst, name: str = "multi") -> CSR:
    """Keeps self loops and repeated edges (the engine treats them as parallel edges)."""
    return from_edges(n, src, dst, drop_self=False, dedup=False, name=name)
