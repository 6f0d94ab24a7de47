"""ctypes view of the C ABI in include/gpop.h (argument marshalling only).

Loading fails loudly when libgpop.so has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpop.so")

GPOP_OK = 0
STATUS_NAMES = {0: "GPOP_OK", 1: "GPOP_ERR_INVALID_ARG", 2: "GPOP_ERR_OOM", 3: "GPOP_ERR_CUDA",
                4: "GPOP_ERR_DEVICE_CHECK", 5: "GPOP_ERR_TIMEOUT", 6: "GPOP_ERR_NOT_CONVERGED",
                7: "GPOP_ERR_NO_SELECTOR"}

ALGOS = {"pagerank": 0, "bfs": 1, "cc": 2, "sssp": 3, "ppr": 4, "nibble": 5}
MODES = {"analytic": 0, "learned": 1, "force_sc": 2, "force_pc": 3, "log_both": 4}

SELECTOR_FEATURES = 8
SELECTOR_WEIGHTS = 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1
SELECTOR_PARAMS = SELECTOR_WEIGHTS + 4 * 8
LOG_RECORD_FLOATS = 13


class GraphInfo(ctypes.Structure):
    _fields_ = [("num_vertices", ctypes.c_uint32), ("partition_size", ctypes.c_uint32),
                ("num_partitions", ctypes.c_uint32), ("weighted", ctypes.c_uint32),
                ("num_edges", ctypes.c_uint64), ("num_bins", ctypes.c_uint64), ("num_png", ctypes.c_uint64),
                ("num_png_padded", ctypes.c_uint64), ("num_gather_tasks", ctypes.c_uint32),
                ("num_scatter_tasks", ctypes.c_uint32), ("max_row_bins", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64),
                ("num_pc_blocks", ctypes.c_uint64), ("num_pc_tasks", ctypes.c_uint32),
                ("num_pc_partials", ctypes.c_uint32)]


class RunOpts(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("source", ctypes.c_uint32), ("damping", ctypes.c_double),
                ("max_iters", ctypes.c_uint32), ("tol_l1", ctypes.c_double), ("mode", ctypes.c_int32),
                ("bw_ratio_num", ctypes.c_uint32), ("bw_ratio_den", ctypes.c_uint32), ("msg_bf16", ctypes.c_int32),
                ("profile_kernels", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p), ("trace_modes", ctypes.c_void_p),
                ("trace_frontier", ctypes.c_void_p), ("log_buffer", ctypes.c_void_p),
                ("log_capacity", ctypes.c_uint64), ("epsilon", ctypes.c_double), ("resume", ctypes.c_int32),
                ("isg_waves", ctypes.c_uint32)]


class RunStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint32), ("converged", ctypes.c_int32), ("residual", ctypes.c_double),
                ("edges_scattered", ctypes.c_uint64), ("vertices_scattered", ctypes.c_uint64),
                ("pc_partition_steps", ctypes.c_uint64), ("sc_partition_steps", ctypes.c_uint64),
                ("model_bytes", ctypes.c_double), ("device_ms", ctypes.c_double), ("log_records", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_double * 6), ("kernel_launches", ctypes.c_uint64 * 6),
                ("sc_vertices_scattered", ctypes.c_uint64), ("sc_edges_scattered", ctypes.c_uint64),
                ("gathered_vertices", ctypes.c_uint64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["kernel_ms"] = list(self.kernel_ms)
        d["kernel_launches"] = list(self.kernel_launches)
        return d


# every symbol include/gpop.h declares, with (restype, argtypes)
_vp, _u32, _u64, _i32, _f32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_float
SIGNATURES = {
    "gpop_graph_build": (ctypes.c_int, [_u32, _u64, _vp, _vp, _vp, _u32, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "gpop_graph_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(GraphInfo)]),
    "gpop_graph_partition_stats": (ctypes.c_int, [_vp, _vp, _vp]),
    "gpop_graph_destroy": (None, [_vp]),
    "gpop_run_opts_default": (None, [ctypes.POINTER(RunOpts)]),
    "gpop_run": (ctypes.c_int, [_vp, ctypes.POINTER(RunOpts), _vp, _vp, ctypes.c_int, ctypes.POINTER(RunStats)]),
    "gpop_run_msbfs": (ctypes.c_int, [_vp, ctypes.POINTER(RunOpts), _vp, ctypes.c_uint32, _vp, ctypes.c_int,
                                      ctypes.POINTER(RunStats)]),
    "gpop_run_ppr_batch": (ctypes.c_int, [_vp, ctypes.POINTER(RunOpts), _vp, ctypes.c_uint32, _vp, ctypes.c_int,
                                          ctypes.POINTER(RunStats)]),
    "gpop_graph_build_union": (ctypes.c_int, [_u32, _vp, _vp, _vp, _vp, _vp, _u32, _vp, ctypes.POINTER(_vp)]),
    "gpop_graph_union_offsets": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_u32)]),
    "gpop_run_bfs_union": (ctypes.c_int, [_vp, ctypes.POINTER(RunOpts), _vp, _vp, ctypes.c_int,
                                          ctypes.POINTER(RunStats)]),
    "gpop_probe_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "gpop_state_export": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "gpop_state_import": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64]),
    "gpop_selector_set": (ctypes.c_int, [_vp]),
    "gpop_selector_get": (ctypes.c_int, [_vp]),
    "gpop_selector_train": (ctypes.c_int, [_vp, _vp, _u32, _u32, _f32, _u64, _vp, _vp, _vp]),
    "gpop_selector_grad": (ctypes.c_int, [_vp, _vp, _vp, _u32, _vp, _vp, _vp, _vp]),
    "gpop_selector_grad_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _u32, _vp, _vp, _vp, _vp]),
    "gpop_last_error": (ctypes.c_char_p, []),
}

_lib = None


class GpopError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Loads libgpop.so; raises if it is missing (build it with paper_1806_08092_gb300.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_1806_08092_gb300.build() (needs nvcc) first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int):
    if status != GPOP_OK:
        raise GpopError(status, load().gpop_last_error().decode())
