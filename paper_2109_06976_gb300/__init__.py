"""GB300-native batched rigid-body dynamics with analytical gradients.

Thin PyTorch-facing layer over the C-ABI of ``include/grid.h``: it only checks
shapes, allocates outputs with torch and passes device pointers and the current
CUDA stream. Every step of the computation runs in the CUDA kernels of
``csrc/``; there is no CPU fallback.

The operations follow Sec. IV-B of the GRiD paper (arXiv 2109.06976):
RNEA inverse dynamics, the direct inverse of the mass matrix, forward dynamics
qdd = M^-1 (tau - RNEA(q, qd, 0)) and the analytical gradient of forward
dynamics [dqdd/dq | dqdd/dqd] = -M^-1 [dID/dq | dID/dqd].
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import GRID_FP32, GRID_FP64, GRID_MIXED, GridError  # noqa: F401

__all__ = ["Model", "Server", "ForwardDynamics", "forward_dynamics", "GridError", "GRID_FP32",
           "GRID_MIXED", "GRID_FP64", "build"]

_PREC = {"fp32": GRID_FP32, "mixed": GRID_MIXED}


def build(verbose: bool = False) -> str:
    from . import build_ext as _b
    return _b.build(verbose=verbose)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


class Model:
    """A robot model resident on the current CUDA device.

    Per body: parent [nb] (int, -1 = fixed base, parent[i] < i), axis [nb, 3]
    unit joint axes, xtree [nb, 12] (E row-major then r), inertia [nb, 10] (m,
    COM, Ic about the COM: xx yy zz xy xz yz), optional jtype [nb] (0 revolute,
    1 prismatic, 2 fixed; None = all revolute); gravity [3]. Fixed bodies are
    merged into their parents, so every state array has ``n`` = the number of
    moving joints per knot point. See include/grid.h.
    """

    def __init__(self, parent, axis, xtree, inertia, gravity=(0.0, 0.0, -9.81), precision="fp32",
                 jtype=None):
        lib = _native.load()
        self._keep = (_np(parent, np.int32), None if jtype is None else _np(jtype, np.int32),
                      _np(axis, np.float64), _np(xtree, np.float64), _np(inertia, np.float64),
                      _np(gravity, np.float64))
        nb = int(self._keep[0].shape[0])
        h = ctypes.c_void_p()
        _native.check("grid_create_ex", lib.grid_create_ex(
            nb, *[None if a is None else a.ctypes.data_as(ctypes.c_void_p) for a in self._keep],
            _PREC[precision], ctypes.byref(h)))
        self._h = h
        self.n = int(lib.grid_model_dof(h))
        self.device = torch.cuda.current_device()

    @classmethod
    def from_robot(cls, robot, precision="fp32"):
        return cls(robot.parent, robot.axis, robot.xtree, robot.inertia, robot.gravity, precision,
                   jtype=robot.jtype)

    @property
    def handle(self):
        return self._h

    def set_option(self, key: str, value: int):
        _native.call("grid_set_option", self._h, key.encode(), int(value))

    def set_precision(self, precision: str):
        self.set_option("precision", _PREC[precision])

    def close(self):
        if getattr(self, "_h", None):
            _native.load().grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _state(self, *ts):
        out = []
        N = None
        dtype = None
        for t in ts:
            if t is None:
                out.append(None)
                continue
            if not (isinstance(t, torch.Tensor) and (t.is_cuda or t.is_pinned())):
                raise TypeError("states must be CUDA tensors or pinned host tensors (zero copy)")
            if t.shape[-1] != self.n:
                raise ValueError(f"last dimension must be n = {self.n}")
            t2 = t.reshape(-1, self.n).contiguous()
            if N is None:
                N, dtype = t2.shape[0], t2.dtype
            elif t2.shape[0] != N or t2.dtype != dtype:
                raise ValueError("state tensors must share batch size and dtype")
            out.append(t2)
        if dtype not in (torch.float32, torch.float64):
            raise TypeError("states must be float32 or float64")
        return N, dtype, out

    @staticmethod
    def _empty(shape, dtype, like):
        """Output buffer next to the inputs: device memory, or pinned host memory
        when the inputs are pinned host tensors (the kernel then reads and writes
        host memory directly over the CPU-GPU link)."""
        if like.is_cuda:
            return torch.empty(shape, dtype=dtype, device=like.device)
        return torch.empty(shape, dtype=dtype).pin_memory()

    @staticmethod
    def _fn(name, dtype):
        return name + ("_f64" if dtype == torch.float64 else "")

    @staticmethod
    def _stream():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    # ------------------------------------------------------------ operations
    def rnea(self, q, qd, qdd=None, out=None):
        """tau = ID(q, qd, qdd), [N, n]."""
        N, dt, (q, qd, qdd) = self._state(q, qd, qdd)
        tau = out if out is not None else self._empty((N, self.n), dt, q)
        _native.call(self._fn("grid_rnea", dt), self._h, N, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(tau),
                     self._stream())
        return tau

    def minv(self, q, out=None):
        """M(q)^-1, [N, n, n] (full symmetric)."""
        N, dt, (q,) = self._state(q)
        Mi = out if out is not None else self._empty((N, self.n, self.n), dt, q)
        _native.call(self._fn("grid_minv", dt), self._h, N, _ptr(q), _ptr(Mi), self._stream())
        return Mi

    def fd(self, q, qd, tau, out=None):
        """qdd = M^-1 (tau - RNEA(q, qd, 0)), [N, n]."""
        N, dt, (q, qd, tau) = self._state(q, qd, tau)
        qdd = out if out is not None else self._empty((N, self.n), dt, q)
        _native.call(self._fn("grid_fd", dt), self._h, N, _ptr(q), _ptr(qd), _ptr(tau), _ptr(qdd),
                     self._stream())
        return qdd

    def grad_rnea(self, q, qd, qdd=None, out=None):
        """[dID/dq | dID/dqd] at (q, qd, qdd), [N, n, 2n]."""
        N, dt, (q, qd, qdd) = self._state(q, qd, qdd)
        D = out if out is not None else self._empty((N, self.n, 2 * self.n), dt, q)
        _native.call(self._fn("grid_grad_rnea", dt), self._h, N, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(D),
                     self._stream())
        return D

    def grad_fd(self, q, qd, tau, out=None, qdd_out=None, return_qdd=False):
        """J = [dqdd/dq | dqdd/dqd], [N, n, 2n]; optionally also qdd [N, n]."""
        N, dt, (q, qd, tau) = self._state(q, qd, tau)
        J = out if out is not None else self._empty((N, self.n, 2 * self.n), dt, q)
        if return_qdd and qdd_out is None:
            qdd_out = self._empty((N, self.n), dt, q)
        _native.call(self._fn("grid_grad_fd", dt), self._h, N, _ptr(q), _ptr(qd), _ptr(tau), _ptr(J),
                     _ptr(qdd_out), self._stream())
        return (J, qdd_out) if return_qdd else J

    def grad_fd_host(self, q, qd, tau, out=None, qdd_out=None, return_qdd=False, sync=True):
        """grad_fd for states in host memory (grid_grad_fd_host): CPU tensors,
        page-locked for overlapped copies. The library moves the batch through
        device staging in chunks, overlapping the copies in, the kernel and the
        copies out. Outputs are CPU tensors (pinned when allocated here). With
        sync=True the call waits for the current stream, so the results are
        ready on return; with sync=False they are ready once the stream reaches
        this point, and the inputs must stay untouched until then."""
        ts = [q, qd, tau]
        N = dtype = None
        flat = []
        for t in ts:
            if not isinstance(t, torch.Tensor) or t.is_cuda:
                raise TypeError("grad_fd_host takes CPU tensors")
            if t.shape[-1] != self.n:
                raise ValueError(f"last dimension must be n = {self.n}")
            t2 = t.reshape(-1, self.n)
            if not t2.is_contiguous():
                raise ValueError("state tensors must be contiguous")
            if N is None:
                N, dtype = t2.shape[0], t2.dtype
            elif t2.shape[0] != N or t2.dtype != dtype:
                raise ValueError("state tensors must share batch size and dtype")
            flat.append(t2)
        if dtype not in (torch.float32, torch.float64):
            raise TypeError("states must be float32 or float64")
        J = out if out is not None else torch.empty((N, self.n, 2 * self.n), dtype=dtype).pin_memory()
        if return_qdd and qdd_out is None:
            qdd_out = torch.empty((N, self.n), dtype=dtype).pin_memory()
        for t in (J, qdd_out):
            if t is not None and (t.is_cuda or not t.is_contiguous() or t.dtype != dtype):
                raise ValueError("outputs must be contiguous CPU tensors of the states' dtype")
        _native.call(self._fn("grid_grad_fd_host", dtype), self._h, N, *(_ptr(t) for t in flat), _ptr(J),
                     _ptr(qdd_out), self._stream())
        if sync:
            torch.cuda.current_stream().synchronize()
        return (J, qdd_out) if return_qdd else J

    def grad_fd_minv(self, q, qd, tau, out=None, minv_out=None):
        """(J, M^-1): the gradient of FD [N, n, 2n] and M^-1 = dqdd/dtau [N, n, n]
        from one kernel (grid_grad_fd_ex)."""
        N, dt, (q, qd, tau) = self._state(q, qd, tau)
        J = out if out is not None else self._empty((N, self.n, 2 * self.n), dt, q)
        Mi = minv_out if minv_out is not None else self._empty((N, self.n, self.n), dt, q)
        _native.call(self._fn("grid_grad_fd_ex", dt), self._h, N, _ptr(q), _ptr(qd), _ptr(tau), _ptr(J), None,
                     _ptr(Mi), self._stream())
        return J, Mi

    # ------------------------------------------------------------ trajectories
    def _traj(self, *ts):
        """Trajectory tensors [B, H+1, n], contiguous, one dtype and device."""
        B, K1 = ts[0].shape[0], ts[0].shape[1]
        for t in ts:
            if t is None:
                continue
            if t.shape != (B, K1, self.n) or t.dtype != ts[0].dtype or not t.is_contiguous():
                raise ValueError(f"trajectory tensors must be contiguous [B, H+1, n={self.n}] of one dtype")
        return B, K1 - 1, ts[0].dtype

    def rollout(self, q0, qd0, U, dt, policy=None, out=None):
        """Semi-implicit Euler rollout through FD (grid_rollout). q0, qd0 [B, n];
        U [B, H+1, n] (entry H unused). policy = (K, kff, Qnom, QDnom, alpha) from
        riccati() and the nominal trajectory, or None. Returns Q, QD and the
        applied controls, each [B, H+1, n]."""
        B, H, dtp = self._traj(U)
        Q, QD, Ua = out if out is not None else tuple(torch.empty_like(U) for _ in range(3))
        K = kff = Qn = QDn = None
        alpha = 1.0
        if policy is not None:
            K, kff, Qn, QDn, alpha = policy
        _native.call(self._fn("grid_rollout", dtp), self._h, B, H, float(dt), _ptr(q0.contiguous()),
                     _ptr(qd0.contiguous()), _ptr(U), _ptr(K), _ptr(kff), _ptr(Qn), _ptr(QDn), float(alpha),
                     _ptr(Q), _ptr(QD), _ptr(Ua), self._stream())
        return Q, QD, Ua

    def riccati(self, Q, QD, U, J, Minv, Qref, QDref, wq, wr, wf, dt, mu=0.0):
        """iLQR backward pass about the nominal trajectory (grid_riccati). J, Minv
        from grad_fd_minv at the nominal knot points ([B (H+1), n, 2n] and
        [B (H+1), n, n]); weights wq, wf [2n], wr [n] on the device. Returns
        K [B, H+1, n, 2n], kff [B, H+1, n] and dV [B, 2]."""
        B, H, dtp = self._traj(Q, QD, U, Qref, QDref)
        n = self.n
        K = torch.empty((B, H + 1, n, 2 * n), dtype=dtp, device=Q.device)
        kff = torch.empty((B, H + 1, n), dtype=dtp, device=Q.device)
        dV = torch.empty((B, 2), dtype=dtp, device=Q.device)
        _native.call(self._fn("grid_riccati", dtp), self._h, B, H, float(dt), _ptr(Q), _ptr(QD), _ptr(U),
                     _ptr(J.contiguous()), _ptr(Minv.contiguous()), _ptr(Qref), _ptr(QDref), _ptr(wq), _ptr(wr),
                     _ptr(wf), float(mu), _ptr(K), _ptr(kff), _ptr(dV), self._stream())
        return K, kff, dV

    def ilqr_iteration(self, q0, qd0, U, Qref, QDref, wq, wr, wf, dt, mu=0.0, alpha=1.0):
        """One iLQR iteration on the device with no host transfer: rollout of the
        nominal controls, the gradient of FD and M^-1 at every knot point, the
        backward pass, and the forward pass under the new policy. Returns the new
        (Q, QD, U) [B, H+1, n] and dV [B, 2] of the step taken."""
        Q, QD, _ = self.rollout(q0, qd0, U, dt)
        J, Mi = self.grad_fd_minv(Q, QD, U)
        K, kff, dV = self.riccati(Q, QD, U, J, Mi, Qref, QDref, wq, wr, wf, dt, mu)
        Qn, QDn, Un = self.rollout(q0, qd0, U, dt, policy=(K, kff, Q, QD, alpha))
        return Qn, QDn, Un, dV

    def fd_vjp(self, q, qd, tau, gbar, out=None):
        """Vector-Jacobian product through FD for gbar = dL/dqdd:
        returns (dL/dq, dL/dqd, dL/dtau), each [N, n]. Forward intermediates are
        recomputed from (q, qd, tau); no Jacobian is formed."""
        N, dt, (q, qd, tau, gbar) = self._state(q, qd, tau, gbar)
        if out is None:
            out = tuple(self._empty((N, self.n), dt, q) for _ in range(3))
        dq, dqd, dtau = out
        _native.call(self._fn("grid_fd_vjp", dt), self._h, N, _ptr(q), _ptr(qd), _ptr(tau), _ptr(gbar),
                     _ptr(dq), _ptr(dqd), _ptr(dtau), self._stream())
        return dq, dqd, dtau


class ForwardDynamics(torch.autograd.Function):
    """qdd = FD(q, qd, tau) as a differentiable op. Forward: the FD kernel.
    Backward: the vector-Jacobian-product kernel (reverse-mode RNEA sweep),
    recomputing the forward intermediates; only q, qd, tau are saved."""

    @staticmethod
    def forward(ctx, model, q, qd, tau):
        ctx.model = model
        ctx.save_for_backward(q, qd, tau)
        return model.fd(q, qd, tau).view(q.shape)

    @staticmethod
    def backward(ctx, gbar):
        q, qd, tau = ctx.saved_tensors
        dq, dqd, dtau = ctx.model.fd_vjp(q, qd, tau, gbar.contiguous())
        return None, dq.view(q.shape), dqd.view(qd.shape), dtau.view(tau.shape)


def forward_dynamics(model, q, qd, tau):
    """Differentiable forward dynamics qdd = M^-1 (tau - RNEA(q, qd, 0))."""
    return ForwardDynamics.apply(model, q, qd, tau)


class Server:
    """Persistent-kernel server for gradient-of-FD requests of mixed robots and
    horizons (continuous batching; see include/grid.h). Host-side arrays are
    numpy float32 [H, n]."""

    def __init__(self, models, ring_slots=256, arena_bytes=256 << 20, idle_timeout=2.0):
        lib = _native.load()
        self.models = list(models)
        arr = (ctypes.c_void_p * len(self.models))(*[m.handle.value for m in self.models])
        h = ctypes.c_void_p()
        _native.check("grid_server_create", lib.grid_server_create(arr, len(self.models), ring_slots,
                                                                   arena_bytes, ctypes.byref(h)))
        self._h = h
        _native.call("grid_server_set_idle_timeout", h, float(idle_timeout))
        self._stream = None

    def start(self, stream=None):
        """Launch the persistent kernel (on its own non-blocking stream unless
        one is given)."""
        self._stream = stream
        _native.call("grid_server_start", self._h,
                     None if stream is None else ctypes.c_void_p(stream.cuda_stream))

    def submit(self, model_index, q, qd, tau):
        """Returns a request id, or None if no slot / arena space is free now."""
        arrs = [np.ascontiguousarray(x, dtype=np.float32) for x in (q, qd, tau)]
        H = arrs[0].shape[0]
        rid = ctypes.c_longlong()
        st = _native.load().grid_server_submit(self._h, model_index, H,
                                               *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                               ctypes.byref(rid))
        if st == 5:           # GRID_E_NOMEM: not admitted now
            return None
        _native.check("grid_server_submit", st)
        return rid.value

    def result(self, rid, H, n, wait_us=1_000_000):
        """Jacobians [H, n, 2n] (numpy), or None if not done within wait_us."""
        J = np.empty((H, n, 2 * n), dtype=np.float32)
        st = _native.load().grid_server_result(self._h, rid, J.ctypes.data_as(ctypes.c_void_p), int(wait_us))
        if st == 6:
            return None
        _native.check("grid_server_result", st)
        return J

    def kernel_status(self):
        return _native.load().grid_server_kernel_status(self._h)

    def stop(self):
        """Stop the persistent kernel; returns its status code (0 = ok)."""
        return _native.load().grid_server_stop(self._h)

    def bench(self, rate_hz, seconds, seed, horizons, pools):
        """Open-loop Poisson benchmark (native producer/consumer threads).
        pools[m]: float32 [3, K, n_m] (q, qd, tau). Returns a dict of stats."""
        K = pools[0].shape[1]
        keep = [np.ascontiguousarray(p, dtype=np.float32) for p in pools]
        ptrs = (ctypes.c_void_p * len(keep))(*[p.ctypes.data for p in keep])
        hz = (ctypes.c_int * len(horizons))(*horizons)
        stats = (ctypes.c_double * 9)()
        st = _native.load().grid_server_bench(self._h, float(rate_hz), float(seconds), int(seed), hz,
                                              len(horizons), ptrs, K, stats)
        keys = ["completed", "knot_points", "wall_s", "p50_ms", "p99_ms", "p50_ms_h128", "p99_ms_h128",
                "max_ms", "refused"]
        out = dict(zip(keys, list(stats)))
        out["status"] = st
        return out

    def close(self):
        if getattr(self, "_h", None):
            _native.load().grid_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
