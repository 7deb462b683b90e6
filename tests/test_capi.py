"""The C-ABI library loads and exports every symbol include/grid.h declares
(no compute calls, no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grid_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_06976_gb300 import build_ext as build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_calls():
    names = _declared()
    for fn in ("grid_create", "grid_rnea", "grid_minv", "grid_fd", "grid_grad_fd"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_validation_without_gpu(lib):
    """grid_create rejects bad topologies on the host before touching a device."""
    lib.grid_create.restype = ctypes.c_int
    lib.grid_last_error.restype = ctypes.c_char_p
    import numpy as np
    parent = np.array([-1, 1], dtype=np.int32)          # parent[1] = 1 violates parent[i] < i
    axis = np.array([[0, 0, 1], [0, 1, 0]], dtype=np.float64)
    xt = np.zeros((2, 12))
    xt[:, 0] = xt[:, 4] = xt[:, 8] = 1
    inert = np.zeros((2, 10))
    inert[:, 0] = 1
    g = np.array([0, 0, -9.81])
    h = ctypes.c_void_p()
    P = ctypes.c_void_p
    st = lib.grid_create(2, parent.ctypes.data_as(P), axis.ctypes.data_as(P), xt.ctypes.data_as(P),
                         inert.ctypes.data_as(P), g.ctypes.data_as(P), 0, ctypes.byref(h))
    assert st == 2 and b"parent[1]" in lib.grid_last_error()
    parent = np.array([-1, 0], dtype=np.int32)
    inert[1, 0] = -1.0
    st = lib.grid_create(2, parent.ctypes.data_as(P), axis.ctypes.data_as(P), xt.ctypes.data_as(P),
                         inert.ctypes.data_as(P), g.ctypes.data_as(P), 0, ctypes.byref(h))
    assert st == 7
    st = lib.grid_create(40, parent.ctypes.data_as(P), axis.ctypes.data_as(P), xt.ctypes.data_as(P),
                         inert.ctypes.data_as(P), g.ctypes.data_as(P), 0, ctypes.byref(h))
    assert st == 2


def test_host_buffer_call_checks_arguments_without_gpu(lib):
    """grid_grad_fd_host and the host_chunk option refuse a null model on the
    host, before any CUDA call."""
    P = ctypes.c_void_p
    for name in ("grid_grad_fd_host", "grid_grad_fd_host_f64"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = [P, ctypes.c_int, P, P, P, P, P, P]
        assert fn(None, 4, None, None, None, None, None, None) == 1
    lib.grid_set_option.restype = ctypes.c_int
    lib.grid_set_option.argtypes = [P, ctypes.c_char_p, ctypes.c_int]
    assert lib.grid_set_option(None, b"host_chunk", 1024) == 1


def test_peak_loop_rejects_bad_arguments_without_gpu(lib):
    """grid_peak_loop checks its arguments on the host before any launch."""
    lib.grid_peak_loop.restype = ctypes.c_int
    lib.grid_peak_loop.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    fl = ctypes.c_double()
    for kind, blocks, threads, iters in ((3, 1, 32, 1), (0, 0, 32, 1), (0, 1, 33, 1), (0, 1, 2048, 1), (0, 1, 32, 0)):
        assert lib.grid_peak_loop(kind, blocks, threads, iters, ctypes.c_void_p(16), ctypes.byref(fl), None) == 1
