"""GB300 partition-centric scatter/gather (GPOP, arXiv 1806.08092) behind a C ABI.

Python binding over libgpop.so: it only marshals arguments.  Every step of
pre-processing and of each iteration runs in the library's CUDA kernels;
PyTorch supplies device memory for outputs and the current CUDA stream.

    import paper_1806_08092_gb300 as gp
    g = gp.Graph.from_csr(row_ptr, col, weights=None, partition_size=16384)
    res = g.run("pagerank", max_iters=10)          # res.values: torch tensor on cuda
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from ._build import build as _build_lib
from ._lib import ALGOS, MODES, GpopError, LOG_RECORD_FLOATS, SELECTOR_PARAMS, SELECTOR_WEIGHTS  # noqa: F401
MSBFS_WIDTH = 32  # sources per gpop_run_msbfs engine pass (bits of a 32-bit message)

__all__ = ["build", "Graph", "RunResult", "GpopError", "selector_set", "selector_get", "selector_train",
           "selector_grad"]


def build(force: bool = False) -> str:
    """Compiles libgpop.so for sm_103a in place and loads it."""
    path = _build_lib(force=force)
    _lib.load(path)
    return path


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _as_buffer(a, dtype_np, name):
    """Returns (pointer, is_device, keepalive) for a numpy array or a torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.uint64: torch.uint64, np.uint32: torch.uint32, np.int32: torch.int32}[dtype_np]
            if a.dtype != tdt:
                a = a.to(tdt)
            a = a.contiguous()
            return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype_np)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


@dataclass
class RunResult:
    values: object                   # torch tensor (float32 PageRank/PPR, uint32 level/dist/label)
    parent: object | None            # BFS parents
    stats: dict
    modes: np.ndarray | None = None  # [iterations, k] uint8 (0 none, 1 SC, 2 PC) when traced
    frontier: np.ndarray | None = None  # [iterations, 2] (V_a, E_a) when traced
    log: np.ndarray | None = None    # LOG_BOTH records [n, 13]
    extra: dict = field(default_factory=dict)


class Graph:
    """A partitioned graph living on the GPU (owns a gpop_graph handle)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        self._info = None

    @classmethod
    def from_csr(cls, row_ptr, col, weights=None, partition_size: int = 0, stream=None) -> "Graph":
        lib = _lib.load()
        rp, rp_dev, rp_keep = _as_buffer(row_ptr, np.uint64, "row_ptr")
        cl, cl_dev, cl_keep = _as_buffer(col, np.uint32, "col")
        n = int(rp_keep.shape[0]) - 1
        m = int(cl_keep.shape[0])
        w = ctypes.c_void_p(None)
        w_keep = None
        if weights is not None:
            w, w_dev, w_keep = _as_buffer(weights, np.int32, "weights")
            if w_dev != rp_dev:
                raise ValueError("weights must live where row_ptr/col live")
        if rp_dev != cl_dev:
            raise ValueError("row_ptr and col must both be host or both be device memory")
        h = ctypes.c_void_p()
        _lib.check(lib.gpop_graph_build(n, m, rp, cl, w, partition_size, rp_dev, _stream_handle(stream),
                                        ctypes.byref(h)))
        del rp_keep, cl_keep, w_keep
        return cls(h)

    @classmethod
    def from_many(cls, graphs, partition_size: int = 0, stream=None) -> "Graph":
        """Builds several graphs as one, their disjoint union (gpop_graph_build_union).  graphs: a list of
        (row_ptr, col) or (row_ptr, col, weights) host arrays, local vertex IDs per graph."""
        lib = _lib.load()
        ng = len(graphs)
        keep = []
        nv = np.zeros(ng, dtype=np.uint32)
        ne = np.zeros(ng, dtype=np.uint64)
        rps = (ctypes.c_void_p * ng)()
        cols = (ctypes.c_void_p * ng)()
        weighted = ng > 0 and len(graphs[0]) > 2 and graphs[0][2] is not None
        ws = (ctypes.c_void_p * ng)() if weighted else None
        for i, gr in enumerate(graphs):
            rp = np.ascontiguousarray(gr[0], dtype=np.uint64)
            cl = np.ascontiguousarray(gr[1], dtype=np.uint32)
            nv[i], ne[i] = rp.shape[0] - 1, cl.shape[0]
            rps[i], cols[i] = rp.ctypes.data, cl.ctypes.data if cl.size else None
            keep += [rp, cl]
            if weighted:
                w = np.ascontiguousarray(gr[2], dtype=np.int32)
                ws[i] = w.ctypes.data if w.size else None
                keep.append(w)
        h = ctypes.c_void_p()
        _lib.check(lib.gpop_graph_build_union(ng, ctypes.c_void_p(nv.ctypes.data), ctypes.c_void_p(ne.ctypes.data),
                                              rps, cols, ws, partition_size, _stream_handle(stream), ctypes.byref(h)))
        del keep
        return cls(h)

    def union_offsets(self) -> np.ndarray:
        """First vertex of every graph of a union (and V at the end); empty for a graph not built as one."""
        lib = _lib.load()
        n = ctypes.c_uint32(0)
        _lib.check(lib.gpop_graph_union_offsets(self._h, None, ctypes.byref(n)))
        off = np.zeros(n.value + 1, dtype=np.uint32)
        if n.value:
            _lib.check(lib.gpop_graph_union_offsets(self._h, ctypes.c_void_p(off.ctypes.data), ctypes.byref(n)))
        return off if n.value else np.zeros(0, dtype=np.uint32)

    def run_bfs_union(self, sources, max_iters: int = 1000, mode: str = "analytic", bw_ratio=(2, 1),
                      device_out: bool = True, stream=None, profile: bool = False) -> RunResult:
        """BFS of every graph of a union from its own (local) source (gpop_run_bfs_union); values holds the
        union's V levels, graph i's at union_offsets()[i] onwards (0xFFFFFFFF = unreached)."""
        torch = _torch()
        lib = _lib.load()
        n = self.info()["num_vertices"]
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).astype(np.uint32))
        o = _lib.RunOpts()
        lib.gpop_run_opts_default(ctypes.byref(o))
        o.algo = ALGOS["bfs"]
        o.max_iters = max_iters
        o.mode = MODES[mode]
        o.bw_ratio_num, o.bw_ratio_den = bw_ratio
        o.cuda_stream = _stream_handle(stream)
        o.profile_kernels = int(profile)
        out = torch.empty(n, dtype=torch.uint32, device="cuda") if device_out else np.empty(n, dtype=np.uint32)
        pv = out.data_ptr() if device_out else out.ctypes.data
        st = _lib.RunStats()
        _lib.check(lib.gpop_run_bfs_union(self._h, ctypes.byref(o), ctypes.c_void_p(src.ctypes.data),
                                          ctypes.c_void_p(pv), int(device_out), ctypes.byref(st)))
        return RunResult(out, None, st.as_dict(), None, None, None)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.load().gpop_graph_destroy(h)
            except Exception:
                pass
            self._h = None

    def close(self):
        self.__del__()

    def info(self) -> dict:
        info = _lib.GraphInfo()
        _lib.check(_lib.load().gpop_graph_get_info(self._h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def partition_stats(self):
        k = self.info()["num_partitions"]
        ep = np.zeros(k, dtype=np.uint64)
        npng = np.zeros(k, dtype=np.uint64)
        _lib.check(_lib.load().gpop_graph_partition_stats(self._h, ctypes.c_void_p(ep.ctypes.data),
                                                          ctypes.c_void_p(npng.ctypes.data)))
        return ep, npng

    def run(self, algo: str, source: int = 0, damping: float = 0.85, max_iters: int = 1000, tol: float = 0.0,
            mode: str = "analytic", bw_ratio=(2, 1), device_out: bool = True, trace: bool = False,
            log_capacity: int = 0, stream=None, out=None, out_parent=None, profile: bool = False,
            msg_bf16: bool = False, epsilon: float = 1e-9, resume: bool = False, isg_waves: int = 0) -> RunResult:
        """Runs one application; outputs are torch tensors on cuda (device_out) or host numpy arrays.
        msg_bf16: PageRank / PPR messages travel through the bins as BF16 (gathered in FP32).
        epsilon: Nibble's threshold (a vertex stays on while PR >= epsilon * out-degree).
        resume: continue the state this graph holds (its last run of `algo`, or state_import) for up to
        max_iters more iterations, with the results of one uninterrupted run.
        isg_waves: CC and SSSP only, interleaved scatter-gather with this many waves (0: off)."""
        torch = _torch()
        lib = _lib.load()
        info = self.info()
        n, k = info["num_vertices"], info["num_partitions"]
        o = _lib.RunOpts()
        lib.gpop_run_opts_default(ctypes.byref(o))
        o.algo = ALGOS[algo]
        o.source = source
        o.damping = damping
        o.max_iters = max_iters
        o.tol_l1 = tol
        o.mode = MODES[mode]
        o.bw_ratio_num, o.bw_ratio_den = bw_ratio
        o.cuda_stream = _stream_handle(stream)
        o.profile_kernels = int(profile)
        o.msg_bf16 = int(msg_bf16)
        o.epsilon = epsilon
        o.resume = int(resume)
        o.isg_waves = int(isg_waves)
        modes = frontier = log = None
        if trace:
            modes = np.zeros(max(max_iters, 1) * k, dtype=np.uint8)
            frontier = np.zeros(max(max_iters, 1) * 2, dtype=np.uint64)
            o.trace_modes = ctypes.c_void_p(modes.ctypes.data)
            o.trace_frontier = ctypes.c_void_p(frontier.ctypes.data)
        if log_capacity:
            log = np.zeros(log_capacity * LOG_RECORD_FLOATS, dtype=np.float32)
            o.log_buffer = ctypes.c_void_p(log.ctypes.data)
            o.log_capacity = log_capacity
        fdt = algo in ("pagerank", "ppr", "nibble")
        if device_out:
            if out is None:
                out = torch.empty(n, dtype=torch.float32 if fdt else torch.uint32, device="cuda")
            if algo == "bfs" and out_parent is None:
                out_parent = torch.empty(n, dtype=torch.uint32, device="cuda")
            pv, pp = out.data_ptr(), (out_parent.data_ptr() if out_parent is not None else None)
        else:
            if out is None:
                out = np.empty(n, dtype=np.float32 if fdt else np.uint32)
            if algo == "bfs" and out_parent is None:
                out_parent = np.empty(n, dtype=np.uint32)
            pv = out.ctypes.data
            pp = out_parent.ctypes.data if out_parent is not None else None
        st = _lib.RunStats()
        _lib.check(lib.gpop_run(self._h, ctypes.byref(o), ctypes.c_void_p(pv), ctypes.c_void_p(pp),
                                int(device_out), ctypes.byref(st)))
        stats = st.as_dict()
        it = stats["iterations"]
        if trace:
            modes = modes[: it * k].reshape(it, k)
            frontier = frontier[: it * 2].reshape(it, 2)
        if log is not None:
            log = log[: stats["log_records"] * LOG_RECORD_FLOATS].reshape(-1, LOG_RECORD_FLOATS)
        return RunResult(out, out_parent if algo == "bfs" else None, stats, modes, frontier, log)

    def state_export(self) -> np.ndarray:
        """Checkpoint of the last successful run on this graph (gpop_state_export), as host bytes."""
        lib = _lib.load()
        size = ctypes.c_uint64(0)
        _lib.check(lib.gpop_state_export(self._h, None, 0, ctypes.byref(size)))
        buf = np.zeros(size.value, dtype=np.uint8)
        _lib.check(lib.gpop_state_export(self._h, ctypes.c_void_p(buf.ctypes.data), size.value, ctypes.byref(size)))
        return buf

    def state_import(self, buf) -> None:
        """Loads a checkpoint written by state_export of the same graph (same edges, weights and partition size)."""
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        _lib.check(_lib.load().gpop_state_import(self._h, ctypes.c_void_p(b.ctypes.data), b.size))

    def run_msbfs(self, sources, max_iters: int = 1000, mode: str = "analytic", bw_ratio=(2, 1),
                  device_out: bool = True, trace: bool = False, stream=None, out=None,
                  profile: bool = False) -> RunResult:
        """BFS levels from every source (gpop_run_msbfs: up to 32 sources per engine pass); values is a
        (len(sources), V) uint32 array, row j the levels from sources[j] (0xFFFFFFFF = unreached).  With
        trace (at most MSBFS_WIDTH sources, one pass), the per-iteration modes and union frontier sizes."""
        torch = _torch()
        lib = _lib.load()
        info = self.info()
        n, k = info["num_vertices"], info["num_partitions"]
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).astype(np.uint32))
        ns = src.shape[0]
        o = _lib.RunOpts()
        lib.gpop_run_opts_default(ctypes.byref(o))
        o.algo = ALGOS["bfs"]
        o.max_iters = max_iters
        o.mode = MODES[mode]
        o.bw_ratio_num, o.bw_ratio_den = bw_ratio
        o.cuda_stream = _stream_handle(stream)
        o.profile_kernels = int(profile)
        modes = frontier = None
        if trace:
            if ns > MSBFS_WIDTH:
                raise ValueError(f"trace covers one pass: at most {MSBFS_WIDTH} sources")
            modes = np.zeros(max(max_iters, 1) * k, dtype=np.uint8)
            frontier = np.zeros(max(max_iters, 1) * 2, dtype=np.uint64)
            o.trace_modes = ctypes.c_void_p(modes.ctypes.data)
            o.trace_frontier = ctypes.c_void_p(frontier.ctypes.data)
        if out is None:
            out = (torch.empty((ns, n), dtype=torch.uint32, device="cuda") if device_out
                   else np.empty((ns, n), dtype=np.uint32))
        pv = out.data_ptr() if device_out else out.ctypes.data
        st = _lib.RunStats()
        _lib.check(lib.gpop_run_msbfs(self._h, ctypes.byref(o), ctypes.c_void_p(src.ctypes.data if ns else None),
                                      ns, ctypes.c_void_p(pv if ns else None), int(device_out), ctypes.byref(st)))
        stats = st.as_dict()
        if trace:
            it = stats["iterations"]
            modes = modes[: it * k].reshape(it, k)
            frontier = frontier[: it * 2].reshape(it, 2)
        return RunResult(out, None, stats, modes, frontier, None)

    def run_ppr_batch(self, seeds, damping: float = 0.85, max_iters: int = 1000, tol: float = 0.0,
                      device_out: bool = True, stream=None, out=None, profile: bool = False) -> RunResult:
        """Seeded personalized PageRank for every seed (gpop_run_ppr_batch: up to 32 seeds per pass, one FP32
        value per seed in every message); values is a (len(seeds), V) float32 array, row j the vector of
        seeds[j].  The graph's partition size must be at most 1024."""
        torch = _torch()
        lib = _lib.load()
        n = self.info()["num_vertices"]
        sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.int64).astype(np.uint32))
        ns = sd.shape[0]
        o = _lib.RunOpts()
        lib.gpop_run_opts_default(ctypes.byref(o))
        o.algo = ALGOS["ppr"]
        o.damping = damping
        o.max_iters = max_iters
        o.tol_l1 = tol
        o.cuda_stream = _stream_handle(stream)
        o.profile_kernels = int(profile)
        if out is None:
            out = (torch.empty((ns, n), dtype=torch.float32, device="cuda") if device_out
                   else np.empty((ns, n), dtype=np.float32))
        pv = out.data_ptr() if device_out else out.ctypes.data
        st = _lib.RunStats()
        _lib.check(lib.gpop_run_ppr_batch(self._h, ctypes.byref(o), ctypes.c_void_p(sd.ctypes.data if ns else None),
                                          ns, ctypes.c_void_p(pv if ns else None), int(device_out), ctypes.byref(st)))
        return RunResult(out, None, st.as_dict(), None, None, None)


def probe_bounded_wait(tries: int) -> bool:
    """Runs the engine's bounded mbarrier wait against a phase nothing completes (gpop_probe_bounded_wait);
    True when the wait gave up after `tries` polls and raised the error word."""
    gave = ctypes.c_uint32(0)
    _lib.check(_lib.load().gpop_probe_bounded_wait(tries, ctypes.byref(gave)))
    return bool(gave.value)


def selector_set(params) -> None:
    """Installs learned-selector parameters (GPOP_SELECTOR_PARAMS floats) or removes them (None)."""
    lib = _lib.load()
    if params is None:
        _lib.check(lib.gpop_selector_set(None))
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.shape == (SELECTOR_PARAMS,)
    _lib.check(lib.gpop_selector_set(ctypes.c_void_p(p.ctypes.data)))


def selector_get():
    p = np.zeros(SELECTOR_PARAMS, dtype=np.float32)
    _lib.check(_lib.load().gpop_selector_get(ctypes.c_void_p(p.ctypes.data)))
    return p


def selector_train(features, targets, epochs: int = 2000, lr: float = 3e-3, seed: int = 1, stream=None):
    """Trains the MLP selector on the GPU; returns (params, final MSE)."""
    f = np.ascontiguousarray(features, dtype=np.float32)
    y = np.ascontiguousarray(targets, dtype=np.float32)
    assert f.ndim == 2 and f.shape[1] == 8 and y.shape == (f.shape[0],)
    p = np.zeros(SELECTOR_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _lib.check(_lib.load().gpop_selector_train(ctypes.c_void_p(f.ctypes.data), ctypes.c_void_p(y.ctypes.data),
                                               f.shape[0], epochs, lr, seed, _stream_handle(stream),
                                               ctypes.c_void_p(p.ctypes.data), ctypes.byref(loss)))
    return p, float(loss.value)


def selector_grad(weights, x, y, stream=None):
    """GPU forward + MSE parameter gradient on standardised inputs; returns (pred, grad, loss)."""
    w = np.ascontiguousarray(weights, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    yy = np.ascontiguousarray(y, dtype=np.float32)
    assert w.shape == (SELECTOR_WEIGHTS,)
    pred = np.zeros(yy.shape[0], dtype=np.float32)
    grad = np.zeros(SELECTOR_WEIGHTS, dtype=np.float32)
    loss = ctypes.c_float()
    _lib.check(_lib.load().gpop_selector_grad(ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(xx.ctypes.data),
                                              ctypes.c_void_p(yy.ctypes.data), yy.shape[0], _stream_handle(stream),
                                              ctypes.c_void_p(pred.ctypes.data), ctypes.c_void_p(grad.ctypes.data),
                                              ctypes.byref(loss)))
    return pred, grad, float(loss.value)
