"""ctypes binding of the C-ABI in include/grid.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build_ext as _build

_lock = threading.Lock()
_lib = None

GRID_OK = 0
STATUS = {0: "GRID_OK", 1: "GRID_E_ARG", 2: "GRID_E_TOPOLOGY", 3: "GRID_E_ALIGN", 4: "GRID_E_CUDA",
          5: "GRID_E_NOMEM", 6: "GRID_E_TIMEOUT", 7: "GRID_E_NUMERIC"}
GRID_FP32, GRID_MIXED, GRID_FP64 = 0, 1, 2

_I = ctypes.c_int
_P = ctypes.c_void_p

# name -> argument types (every function returns grid_status)
SIGNATURES = {
    "grid_create": [_I, _P, _P, _P, _P, _P, _I, ctypes.POINTER(_P)],
    "grid_create_ex": [_I, _P, _P, _P, _P, _P, _P, _I, ctypes.POINTER(_P)],
    "grid_destroy": [_P],
    "grid_set_option": [_P, ctypes.c_char_p, _I],
    "grid_rnea": [_P, _I, _P, _P, _P, _P, _P],
    "grid_minv": [_P, _I, _P, _P, _P],
    "grid_fd": [_P, _I, _P, _P, _P, _P, _P],
    "grid_grad_fd": [_P, _I, _P, _P, _P, _P, _P, _P],
    "grid_rnea_f64": [_P, _I, _P, _P, _P, _P, _P],
    "grid_minv_f64": [_P, _I, _P, _P, _P],
    "grid_fd_f64": [_P, _I, _P, _P, _P, _P, _P],
    "grid_grad_fd_f64": [_P, _I, _P, _P, _P, _P, _P, _P],
    "grid_fd_vjp": [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P],
    "grid_grad_rnea": [_P, _I, _P, _P, _P, _P, _P],
    "grid_grad_rnea_f64": [_P, _I, _P, _P, _P, _P, _P],
    "grid_fd_vjp_f64": [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P],
    "grid_grad_fd_ex": [_P, _I, _P, _P, _P, _P, _P, _P, _P],
    "grid_grad_fd_ex_f64": [_P, _I, _P, _P, _P, _P, _P, _P, _P],
    "grid_grad_fd_host": [_P, _I, _P, _P, _P, _P, _P, _P],
    "grid_grad_fd_host_f64": [_P, _I, _P, _P, _P, _P, _P, _P],
    "grid_rollout": [_P, _I, _I, ctypes.c_float] + [_P] * 7 + [ctypes.c_float] + [_P] * 4,
    "grid_rollout_f64": [_P, _I, _I, ctypes.c_double] + [_P] * 7 + [ctypes.c_double] + [_P] * 4,
    "grid_riccati": [_P, _I, _I, ctypes.c_float] + [_P] * 10 + [ctypes.c_float] + [_P] * 4,
    "grid_riccati_f64": [_P, _I, _I, ctypes.c_double] + [_P] * 10 + [ctypes.c_double] + [_P] * 4,
    "grid_server_create": [_P, _I, _I, ctypes.c_size_t, ctypes.POINTER(_P)],
    "grid_server_set_idle_timeout": [_P, ctypes.c_double],
    "grid_server_start": [_P, _P],
    "grid_server_submit": [_P, _I, _I, _P, _P, _P, ctypes.POINTER(ctypes.c_longlong)],
    "grid_server_result": [_P, ctypes.c_longlong, _P, _I],
    "grid_server_stop": [_P],
    "grid_server_destroy": [_P],
    "grid_server_bench": [_P, ctypes.c_double, ctypes.c_double, ctypes.c_ulonglong, _P, _I, _P, _I, _P],
    "grid_peak_loop": [_I, _I, _I, _I, _P, ctypes.POINTER(ctypes.c_double), _P],
}


class GridError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA extension. Raises if it has not been built; the library
    has no CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(
                    f"CUDA extension not built ({path} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _I
        lib.grid_last_error.argtypes = []
        lib.grid_last_error.restype = ctypes.c_char_p
        lib.grid_model_dof.argtypes = [_P]
        lib.grid_model_dof.restype = _I
        lib.grid_server_kernel_status.argtypes = [_P]
        lib.grid_server_kernel_status.restype = _I
        _lib = lib
        return lib


def check(fn: str, status: int):
    if status != GRID_OK:
        msg = load().grid_last_error().decode(errors="replace")
        raise GridError(fn, status, msg)


def call(fn: str, *args):
    check(fn, getattr(load(), fn)(*args))
