"""FP64 CPU oracle for the dynamics path (RNEA, M, M^-1, FD, dRNEA, dFD).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The product path never
imports this package. The oracle shares no code with the CUDA path; both read
the raw model arrays produced by ``grid_inputs``.

The arithmetic lives in ``grid_oracle.cpp`` (plain C++, dense 6x6 spatial
algebra, FP64); this module compiles it with g++ on first use and marshals
numpy arrays through ctypes.

Pins (in tests/test_oracle_pins.py) tie every function to something other than
itself: the closed-form single pendulum and acrobot, a Lagrangian (energy /
Jacobian) formulation of M, G and C written independently with homogeneous
transforms, invariants (M = M^T > 0, M M^-1 = I, RNEA(FD) = tau, qd-linearity and
Euler homogeneity of dID/dqd), complex-step and central finite differences, and
sibling-permutation equivariance. Prismatic and fixed joints (in
tests/test_oracle_joint_types.py) are pinned by the closed-form slider and
cart-pole, the Lagrangian formulation on random trees of mixed joint types,
complex-step derivatives, and fixed bodies lumped into their parents by hand.
No function is left unpinned.

Joint arrays (q, qd, qdd, tau and the rows and columns of M, M^-1 and the
Jacobians) hold the moving joints only (``robot.nd`` of them), in body order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grid_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgrid_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_I = ctypes.c_int
_D = ctypes.c_double
_P = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            model = [_I, _P, _P, _P, _P, _P, _P]
            sig = {
                "oracle_rnea": model + [_I, _P, _P, _P, _P, _I],
                "oracle_mass_matrix": model + [_I, _P, _P, _I],
                "oracle_minv": model + [_I, _P, _P, _I],
                "oracle_fd": model + [_I, _P, _P, _P, _P, _I],
                "oracle_grad_rnea": model + [_I, _P, _P, _P, _P, _P, _I],
                "oracle_grad_fd": model + [_I, _P, _P, _P, _P, _P, _I],
                "oracle_fd_complex_step": model + [_I, _P, _P, _P, _D, _P, _I],
                "oracle_rnea_complex_step": model + [_I, _P, _P, _P, _D, _P, _P, _I],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = _I
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _f64(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _model_args(robot):
    parent, axis, xtree, inertia, gravity = robot.arrays()
    keep = (parent, robot.jtypes(), axis, xtree, inertia, gravity)
    return keep, [robot.n] + [_ptr(a) for a in keep]


def _check(code, what):
    if code == 1:
        raise OracleError(f"{what}: invalid model (parent[i] must satisfy -1 <= parent[i] < i, "
                          "joint types 0..2, at least one moving joint)")
    if code == 2:
        raise OracleError(f"{what}: mass matrix not positive definite")
    if code != 0:
        raise OracleError(f"{what}: status {code}")


def _states(robot, *xs):
    n = robot.nd
    out = [_f64(x).reshape(-1, n) for x in xs]
    N = out[0].shape[0]
    for x in out:
        if x.shape != (N, n):
            raise ValueError("state arrays must share shape [N, n]")
    return N, out


def rnea(robot, q, qd, qdd, nthreads=1):
    """tau = ID(q, qd, qdd) per knot point, [N, n]."""
    N, (q, qd, qdd) = _states(robot, q, qd, qdd)
    tau = np.empty_like(q)
    keep, margs = _model_args(robot)
    _check(_load().oracle_rnea(*margs, N, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(tau), nthreads), "rnea")
    return tau


def mass_matrix(robot, q, nthreads=1):
    """M(q) by CRBA, [N, n, n]."""
    N, (q,) = _states(robot, q)
    M = np.empty((N, robot.nd, robot.nd))
    keep, margs = _model_args(robot)
    _check(_load().oracle_mass_matrix(*margs, N, _ptr(q), _ptr(M), nthreads), "mass_matrix")
    return M


def minv(robot, q, nthreads=1):
    """M(q)^-1 by CRBA + Cholesky, full symmetric [N, n, n]."""
    N, (q,) = _states(robot, q)
    Mi = np.empty((N, robot.nd, robot.nd))
    keep, margs = _model_args(robot)
    _check(_load().oracle_minv(*margs, N, _ptr(q), _ptr(Mi), nthreads), "minv")
    return Mi


def fd(robot, q, qd, tau, nthreads=1):
    """qdd = M^-1 (tau - RNEA(q, qd, 0)), [N, n]."""
    N, (q, qd, tau) = _states(robot, q, qd, tau)
    qdd = np.empty_like(q)
    keep, margs = _model_args(robot)
    _check(_load().oracle_fd(*margs, N, _ptr(q), _ptr(qd), _ptr(tau), _ptr(qdd), nthreads), "fd")
    return qdd


def grad_rnea(robot, q, qd, qdd, nthreads=1):
    """(dtau/dq, dtau/dqd), each [N, n, n] (row = tau_i, column = joint j)."""
    N, (q, qd, qdd) = _states(robot, q, qd, qdd)
    dq = np.empty((N, robot.nd, robot.nd))
    dqd = np.empty_like(dq)
    keep, margs = _model_args(robot)
    _check(_load().oracle_grad_rnea(*margs, N, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(dq), _ptr(dqd),
                                    nthreads), "grad_rnea")
    return dq, dqd


def grad_fd(robot, q, qd, tau, nthreads=1, with_qdd=False):
    """J = [dqdd/dq | dqdd/dqd], [N, n, 2n]; optionally also qdd [N, n]."""
    N, (q, qd, tau) = _states(robot, q, qd, tau)
    J = np.empty((N, robot.nd, 2 * robot.nd))
    qdd = np.empty_like(q)
    keep, margs = _model_args(robot)
    _check(_load().oracle_grad_fd(*margs, N, _ptr(q), _ptr(qd), _ptr(tau), _ptr(J), _ptr(qdd),
                                  nthreads), "grad_fd")
    return (J, qdd) if with_qdd else J


def fd_complex_step(robot, q, qd, tau, h=1e-30, nthreads=1):
    """[dFD/dq | dFD/dqd] by complex-step differentiation, [N, n, 2n]."""
    N, (q, qd, tau) = _states(robot, q, qd, tau)
    J = np.empty((N, robot.nd, 2 * robot.nd))
    keep, margs = _model_args(robot)
    _check(_load().oracle_fd_complex_step(*margs, N, _ptr(q), _ptr(qd), _ptr(tau), h, _ptr(J),
                                          nthreads), "fd_complex_step")
    return J


def rnea_complex_step(robot, q, qd, qdd, h=1e-30, nthreads=1):
    """(dID/dq, dID/dqd) by complex-step differentiation, each [N, n, n]."""
    N, (q, qd, qdd) = _states(robot, q, qd, qdd)
    dq = np.empty((N, robot.nd, robot.nd))
    dqd = np.empty_like(dq)
    keep, margs = _model_args(robot)
    _check(_load().oracle_rnea_complex_step(*margs, N, _ptr(q), _ptr(qd), _ptr(qdd), h, _ptr(dq),
                                            _ptr(dqd), nthreads), "rnea_complex_step")
    return dq, dqd


def fd_vjp(robot, q, qd, tau, gbar, nthreads=1):
    """Vector-Jacobian product through FD for upstream gbar = dL/dqdd:
    (dL/dq, dL/dqd, dL/dtau) = (J_q^T gbar, J_qd^T gbar, M^-1 gbar) with J from
    grad_fd (dqdd/dtau = M^-1, symmetric)."""
    J = grad_fd(robot, q, qd, tau, nthreads)
    Mi = minv(robot, q, nthreads)
    g = _f64(gbar).reshape(-1, robot.nd)
    n = robot.nd
    dq = np.einsum("kij,ki->kj", J[:, :, :n], g)
    dqd = np.einsum("kij,ki->kj", J[:, :, n:], g)
    dtau = np.einsum("kij,ki->kj", Mi, g)
    return dq, dqd, dtau
