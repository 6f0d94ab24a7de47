"""The C-ABI library builds, loads, and exports every symbol include/gpop.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1806_08092_gb300 as gp
from paper_1806_08092_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpop.h")


@pytest.fixture(scope="module")
def lib():
    gp.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpop_[a-z_]+)\s*\(", text)))


def test_header_declares_expected_api():
    names = declared_functions()
    for n in ("gpop_graph_build", "gpop_run", "gpop_graph_destroy", "gpop_last_error", "gpop_selector_train"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(gpop_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_struct_layouts_match_the_header(tmp_path):
    # compile a probe against the header with the host C compiler and compare layouts with ctypes
    src = tmp_path / "probe.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "gpop.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(gpop_graph_info), sizeof(gpop_run_opts), sizeof(gpop_run_stats),
         offsetof(gpop_run_opts, cuda_stream), offsetof(gpop_run_opts, log_capacity),
         offsetof(gpop_run_opts, epsilon), offsetof(gpop_run_opts, resume));
  printf("%d %d %d\n", GPOP_SELECTOR_WEIGHTS, GPOP_SELECTOR_PARAMS, GPOP_LOG_RECORD_FLOATS);
  return 0; }
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    a = [int(x) for x in lines[0].split()]
    assert a == [ctypes.sizeof(_lib.GraphInfo), ctypes.sizeof(_lib.RunOpts), ctypes.sizeof(_lib.RunStats),
                 _lib.RunOpts.cuda_stream.offset, _lib.RunOpts.log_capacity.offset, _lib.RunOpts.epsilon.offset,
                 _lib.RunOpts.resume.offset]
    b = [int(x) for x in lines[1].split()]
    assert b == [_lib.SELECTOR_WEIGHTS, _lib.SELECTOR_PARAMS, _lib.LOG_RECORD_FLOATS]


def test_opts_default_is_host_only(lib):
    o = _lib.RunOpts()
    lib.gpop_run_opts_default(ctypes.byref(o))
    assert (o.algo, o.damping, o.max_iters, o.mode, o.bw_ratio_num, o.bw_ratio_den) == (0, 0.85, 1000, 0, 2, 1)
    assert o.epsilon == 1e-9
    assert lib.gpop_last_error() is not None


def test_invalid_arguments_are_rejected_on_the_host(lib):
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    rp = np.array([0, 1], dtype=np.uint64)
    col = np.array([0], dtype=np.uint32)
    st = lib.gpop_graph_build(1, 1, ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(col.ctypes.data), None, 48, 0,
                              None, ctypes.byref(h))
    assert st == 1 and b"power of two" in lib.gpop_last_error()
    st = lib.gpop_graph_build(0, 0, ctypes.c_void_p(rp.ctypes.data), None, None, 0, 0, None, ctypes.byref(h))
    assert st == 1
    assert lib.gpop_run(None, None, None, None, 0, None) == 1


def test_union_build_arguments_are_checked_on_the_host(lib):
    # the union's CSR is assembled and checked on the host before any CUDA call
    h = ctypes.c_void_p()
    nv = np.array([3, 2], dtype=np.uint32)
    ne = np.array([2, 1], dtype=np.uint64)
    rp0 = np.array([0, 1, 2, 2], dtype=np.uint64)
    rp1 = np.array([0, 1, 1], dtype=np.uint64)
    c0 = np.array([1, 2], dtype=np.uint32)
    c1_bad = np.array([2], dtype=np.uint32)  # graph 1 has 2 vertices: destination 2 is outside it
    rps = (ctypes.c_void_p * 2)(rp0.ctypes.data, rp1.ctypes.data)
    cols = (ctypes.c_void_p * 2)(c0.ctypes.data, c1_bad.ctypes.data)
    st = lib.gpop_graph_build_union(2, ctypes.c_void_p(nv.ctypes.data), ctypes.c_void_p(ne.ctypes.data), rps, cols,
                                    None, 32, None, ctypes.byref(h))
    assert st == 1 and b"outside its graph" in lib.gpop_last_error()
    assert lib.gpop_graph_build_union(0, None, None, None, None, None, 32, None, ctypes.byref(h)) == 1
    rp1_short = np.array([0, 0, 0], dtype=np.uint64)  # row_ptr ends at 0 but the graph has one edge
    rps2 = (ctypes.c_void_p * 2)(rp0.ctypes.data, rp1_short.ctypes.data)
    st = lib.gpop_graph_build_union(2, ctypes.c_void_p(nv.ctypes.data), ctypes.c_void_p(ne.ctypes.data), rps2, cols,
                                    None, 32, None, ctypes.byref(h))
    assert st == 1 and b"row_ptr" in lib.gpop_last_error()
    n = ctypes.c_uint32(7)
    assert lib.gpop_graph_union_offsets(None, None, ctypes.byref(n)) == 1
    assert lib.gpop_run_bfs_union(None, None, None, None, 0, None) == 1


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load(str(tmp_path / "nope.so"))
