"""ORACLE -- test infrastructure only.

Python access to the plain serial C oracle in ``oracle.c`` (FP64, one thread).
Only the test suite, ``__graft_entry__.smoke()`` and the bench's CPU-baseline /
reference leg may import this package; the CUDA library never calls it and
shares no code with it.

Tier 1 (plain definitions): ``pagerank``, ``ppr``, ``bfs``, ``msbfs``, ``cc``, ``sssp``.
Approximation following its algorithm's steps: ``nibble`` (Alg. 4).
Tier 2 (the serial GPOP engine of Alg. 2 / Alg. 3 / Eq. (mode)): ``gpop``.
Model helpers (Sec. 3.2): ``mode_decide``, ``mode_bytes``, ``partition_stats``.

Every function states the passage it follows; the C source spells out each step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

U32_INF = 0xFFFFFFFF
U64_INF = 0xFFFFFFFFFFFFFFFF

ALGOS = {"pagerank": 0, "bfs": 1, "cc": 2, "sssp": 3, "ppr": 4}
POLICIES = {"analytic": 0, "force_sc": 2, "force_pc": 3}


def build(force: bool = False) -> str:
    """Compiles the oracle shared object in place with gcc (-O2, no fast-math)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _SO + ".tmp", "-lm"],
                   check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp = ctypes.c_void_p
            u32, u64, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
            lib.orc_pagerank.argtypes = [u32, vp, vp, dbl, u32, dbl, vp, vp, vp, vp]
            lib.orc_ppr.argtypes = [u32, vp, vp, u32, dbl, u32, dbl, vp, vp, vp]
            lib.orc_nibble.argtypes = [u32, vp, vp, u32, dbl, u32, vp, vp, vp]
            lib.orc_bfs.argtypes = [u32, vp, vp, u32, vp, vp]
            lib.orc_cc.argtypes = [u32, vp, vp, vp]
            lib.orc_sssp.argtypes = [u32, vp, vp, vp, u32, vp]
            lib.orc_mode_decide.argtypes = [u64, u64, u64, u64, u64, u32, u32]
            lib.orc_mode_bytes.argtypes = [ctypes.c_int, u64, u64, u64, u64, u64]
            lib.orc_mode_bytes.restype = dbl
            lib.orc_partition_stats.argtypes = [u32, vp, vp, u32, vp, vp]
            lib.orc_gpop.argtypes = [u32, vp, vp, vp, u32, u32, u32, dbl, u32, dbl, u32, u32, u32,
                                     vp, vp, vp, vp, vp, vp, vp, vp, vp]
            for f in ("orc_pagerank", "orc_ppr", "orc_nibble", "orc_bfs", "orc_cc", "orc_sssp", "orc_mode_decide",
                      "orc_partition_stats", "orc_gpop"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(g.col, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.uint32)
    return g.num_vertices, rp, col


def pagerank(g, damping: float = 0.85, max_iters: int = 10, tol: float = 0.0, history: bool = False):
    """Alg. 6 as a power iteration in FP64; returns (x, iterations, last L1 change[, per-iteration changes])."""
    n, rp, col = _csr(g)
    x = np.zeros(max(n, 1), dtype=np.float64)
    it = ctypes.c_uint32()
    res = ctypes.c_double()
    hist = np.zeros(max(max_iters, 1), dtype=np.float64) if history else None
    rc = _load().orc_pagerank(n, _ptr(rp), _ptr(col), damping, max_iters, tol, _ptr(x), ctypes.byref(it),
                              ctypes.byref(res), _ptr(hist))
    assert rc == 0
    out = (x[:n], it.value, res.value)
    return out + (hist[:it.value],) if history else out


def ppr(g, seed: int, alpha: float = 0.15, max_iters: int = 100, tol: float = 0.0):
    """Seeded personalised PageRank, restart alpha, FP64; returns (x, iterations, last L1 change)."""
    n, rp, col = _csr(g)
    x = np.zeros(max(n, 1), dtype=np.float64)
    it = ctypes.c_uint32()
    res = ctypes.c_double()
    rc = _load().orc_ppr(n, _ptr(rp), _ptr(col), seed, alpha, max_iters, tol, _ptr(x), ctypes.byref(it),
                         ctypes.byref(res))
    assert rc == 0
    return x[:n], it.value, res.value


def nibble(g, seed: int, eps: float = 1e-9, max_iters: int = 1000):
    """Parallel Nibble (Alg. 4) in FP64: returns (PR, iterations, frontier sizes entering each iteration).
    Sinks are never kept on the frontier (the reading of PR >= eps * deg at deg 0)."""
    n, rp, col = _csr(g)
    pr = np.zeros(max(n, 1), dtype=np.float64)
    fr = np.zeros(max(max_iters, 1), dtype=np.uint64)
    it = ctypes.c_uint32()
    rc = _load().orc_nibble(n, _ptr(rp), _ptr(col), seed, eps, max_iters, _ptr(pr), ctypes.byref(it), _ptr(fr))
    assert rc == 0
    return pr[:n], it.value, fr[: it.value].copy()


def bfs(g, root: int):
    """Queue BFS; returns (level, parent) as uint32 with 0xFFFFFFFF for unreached (parent = min-ID candidate)."""
    n, rp, col = _csr(g)
    level = np.zeros(n, dtype=np.uint32)
    parent = np.zeros(n, dtype=np.uint32)
    assert _load().orc_bfs(n, _ptr(rp), _ptr(col), root, _ptr(level), _ptr(parent)) == 0
    return level, parent


def msbfs(g, sources):
    """BFS levels from each of several sources (the multi-source form of Alg. 5): row j is the hop
    distance from sources[j] over out-edges, 0xFFFFFFFF for unreached.  By definition every row is the
    single-source BFS of its source, so this is that BFS run once per source."""
    n = g.num_vertices
    src = [int(s) for s in sources]
    out = np.zeros((len(src), n), dtype=np.uint32)
    for j, s in enumerate(src):
        out[j] = bfs(g, s)[0]
    return out


def cc(g):
    """Union-find components (directions ignored); label = min vertex ID of the component."""
    n, rp, col = _csr(g)
    label = np.zeros(n, dtype=np.uint32)
    assert _load().orc_cc(n, _ptr(rp), _ptr(col), _ptr(label)) == 0
    return label


def sssp(g, root: int):
    """Dijkstra over non-negative int32 weights; uint64 distances, 2^64-1 for unreachable."""
    n, rp, col = _csr(g)
    assert g.weights is not None
    w = np.ascontiguousarray(g.weights, dtype=np.int32)
    if w.size == 0:
        w = np.zeros(1, dtype=np.int32)
    dist = np.zeros(n, dtype=np.uint64)
    assert _load().orc_sssp(n, _ptr(rp), _ptr(col), _ptr(w), root, _ptr(dist)) == 0
    return dist


def mode_decide(k: int, Ep: int, npng: int, Va: int, Ea: int, num: int = 2, den: int = 1) -> int:
    """Eq. (mode): 2 = PC, 1 = SC, 0 = not scattered (no active vertex or no out-edge)."""
    return _load().orc_mode_decide(k, Ep, npng, Va, Ea, num, den)


def mode_bytes(mode: int, k: int, Ep: int, npng: int, Va: int, Ea: int) -> float:
    """Traffic of Sec. 3.2 for the given mode with s_i = s_v = 4 bytes."""
    return _load().orc_mode_bytes(mode, k, Ep, npng, Va, Ea)


def partition_stats(g, P: int):
    """Per partition: E^p (out-edges) and n_png^p = r^p E^p (sum of out-partition-degrees)."""
    n, rp, col = _csr(g)
    k = (n + P - 1) // P
    Ep = np.zeros(k, dtype=np.uint64)
    npng = np.zeros(k, dtype=np.uint64)
    assert _load().orc_partition_stats(n, _ptr(rp), _ptr(col), P, _ptr(Ep), _ptr(npng)) == 0
    return Ep, npng


@dataclass
class GpopResult:
    values: np.ndarray          # float64 x (PageRank/PPR) or uint64 val (BFS parent / SSSP dist / CC label)
    level: np.ndarray | None    # BFS levels
    iterations: int
    residual: float
    modes: np.ndarray           # [iterations, k] uint8: 0 none, 1 SC, 2 PC
    frontier_vertices: np.ndarray
    frontier_edges: np.ndarray
    model_bytes: np.ndarray


def gpop(g, P: int, algo: str, source: int = 0, damping: float = 0.85, max_iters: int = 1000,
         tol: float = 0.0, policy: str = "analytic", bw_ratio=(2, 1)) -> GpopResult:
    """Serial GPOP engine (Alg. 2 with Alg. 3 and Eq. (mode)); for PPR pass damping = 1 - alpha."""
    n, rp, col = _csr(g)
    a = ALGOS[algo]
    w = None
    if algo == "sssp":
        w = np.ascontiguousarray(g.weights, dtype=np.int32)
        if w.size == 0:
            w = np.zeros(1, dtype=np.int32)
    k = (n + P - 1) // P
    x = np.zeros(n, dtype=np.float64) if algo in ("pagerank", "ppr") else None
    val = np.zeros(n, dtype=np.uint64) if x is None else None
    level = np.zeros(n, dtype=np.uint32) if algo == "bfs" else None
    cap = max(max_iters, 1)
    modes = np.zeros(cap * k, dtype=np.uint8)
    tva = np.zeros(cap, dtype=np.uint64)
    tea = np.zeros(cap, dtype=np.uint64)
    tby = np.zeros(cap, dtype=np.float64)
    it = ctypes.c_uint32()
    res = ctypes.c_double()
    rc = _load().orc_gpop(n, _ptr(rp), _ptr(col), _ptr(w), P, a, source, damping, max_iters, tol,
                          POLICIES[policy], bw_ratio[0], bw_ratio[1], _ptr(x), _ptr(val), _ptr(level),
                          _ptr(modes), _ptr(tva), _ptr(tea), _ptr(tby), ctypes.byref(it), ctypes.byref(res))
    assert rc == 0, rc
    t = it.value
    return GpopResult(x if x is not None else val, level, t, res.value, modes[: t * k].reshape(t, k),
                      tva[:t], tea[:t], tby[:t])
