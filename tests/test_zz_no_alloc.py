"""gpop_selector_grad_noalloc: the allocation-free variant of the selector gradient, for callers that
cannot allocate device memory (inside CUDA-graph capture, under another framework's allocator, or in
loops where an allocation would synchronise the device).  Its outputs must match gpop_selector_grad's,
within the tolerance the selector tests use, on consecutive calls that share its fixed scratch array.

This file is collected last on purpose, so a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1806_08092_gb300 as gp
    from paper_1806_08092_gb300 import _lib
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gp.build()
    return gp, _lib.load()


def problem(n, seed):
    rng = np.random.default_rng(seed)
    from oracle import mlp
    w = rng.normal(0, 0.4, mlp.NW).astype(np.float32)
    X = rng.normal(0, 1, (n, 8)).astype(np.float32)
    Y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - X[:, 7]).astype(np.float32)
    return w, X, Y


def call_noalloc(lib, w, X, Y):
    n = Y.shape[0]
    dw = torch.from_numpy(w).cuda()
    dx = torch.from_numpy(X).cuda()
    dy = torch.from_numpy(Y).cuda()
    dpred = torch.empty(n, dtype=torch.float32, device="cuda")
    dgrad = torch.empty(w.shape[0], dtype=torch.float32, device="cuda")
    dloss = torch.empty(1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.gpop_selector_grad_noalloc(ctypes.c_void_p(dw.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
                                        ctypes.c_void_p(dy.data_ptr()), n, ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.c_void_p(dpred.data_ptr()), ctypes.c_void_p(dgrad.data_ptr()),
                                        ctypes.c_void_p(dloss.data_ptr()))
    assert st == 0, lib.gpop_last_error()
    stream.synchronize()
    return dpred.cpu().numpy(), dgrad.cpu().numpy(), float(dloss.item())


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(lib):
    gp, raw = lib
    from oracle import mlp
    # calls in a row share the scratch array: the largest accepted size (16384 samples fills every
    # scratch block and the loss slot) and one below it, then smaller calls, so stale partials of a
    # larger call must not leak into a smaller one's result
    for n, seed in ((16384, 4), (16383, 5), (5000, 1), (777, 2), (64, 3)):
        w, X, Y = problem(n, seed)
        pred, grad, loss = call_noalloc(raw, w, X, Y)
        ref_pred, ref_grad, ref_loss = gp.selector_grad(w, X, Y)
        assert np.max(np.abs(pred - ref_pred)) <= 1e-4 * max(1.0, float(np.max(np.abs(ref_pred))))
        assert np.max(np.abs(grad - ref_grad)) <= 1e-4 * float(np.max(np.abs(ref_grad)))
        assert loss == pytest.approx(ref_loss, rel=1e-4)
        # and directly against the FP64 reference of the network (oracle/mlp.py), same tolerance
        w64, X64, Y64 = w.astype(np.float64), X.astype(np.float64), Y.astype(np.float64)
        o_pred, o_grad = mlp.forward(w64, X64), mlp.grad(w64, X64, Y64)
        assert np.max(np.abs(pred - o_pred)) <= 1e-4 * max(1.0, float(np.max(np.abs(o_pred))))
        assert np.max(np.abs(grad - o_grad)) <= 1e-4 * float(np.max(np.abs(o_grad)))
        assert loss == pytest.approx(mlp.loss(w64, X64, Y64), rel=1e-4)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    _, raw = lib
    d = torch.zeros(16, dtype=torch.float32, device="cuda")
    ptr = ctypes.c_void_p(d.data_ptr())
    assert raw.gpop_selector_grad_noalloc(ptr, ptr, ptr, 16385, None, None, ptr, None) == 1
    assert b"16384" in raw.gpop_last_error()
    assert raw.gpop_selector_grad_noalloc(ptr, ptr, ptr, 0, None, None, ptr, None) == 1
