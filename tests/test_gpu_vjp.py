"""GPU parity of the vector-Jacobian product through FD and of the autograd
Function built on it (the differentiation workload: the 12-DoF tree, 4096
rollouts x 64 steps in one batch, FP32, upstream gradients N(0, 1))."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import vec_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


def _robot(key):
    return gi.robot(key) if isinstance(key, str) else gi.random_tree(*key)


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dtype, device="cuda")


@pytest.mark.parametrize("key", ["chain7", "tree12", "tree30", (6, 4), (9, 8), (20, 3)], ids=str)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=str)
def test_vjp_matches_oracle(grid, key, dtype):
    r = _robot(key)
    m = grid.Model.from_robot(r)
    N = 37
    npdt = np.float32 if dtype == torch.float32 else np.float64
    q, qd, tau = (x.astype(npdt) for x in gi.states(r.n, N, 21))
    gb = gi.upstream(r.n, N, 21).astype(npdt)
    dq, dqd, dtau = m.fd_vjp(*(_dev(x, dtype) for x in (q, qd, tau, gb)))
    ref = oracle.fd_vjp(r, *(x.astype(np.float64) for x in (q, qd, tau, gb)))
    tol = 1e-4 if dtype == torch.float32 else 1e-10
    for got, want, name in zip((dq, dqd, dtau), ref, ("dq", "dqd", "dtau")):
        e = vec_rel_err(got.cpu().numpy(), want)
        assert e <= tol, (name, e)


def test_differentiation_workload(grid):
    """12-DoF tree, 4096 rollouts x 64 steps = 262,144 FD evaluations in one
    batch (FP32); the VJP is checked on 256 seeded samples against the
    Jacobian-transpose product and against FP64 central differences
    (h = 1e-6) of L = gbar . FD."""
    r = gi.tree12()
    m = grid.Model.from_robot(r)
    N = 4096 * 64
    q, qd, tau = (x.astype(np.float32) for x in gi.states(12, N, gi.workload_seed(4, 64)))
    gb = gi.upstream(12, N, gi.workload_seed(4, 64)).astype(np.float32)
    dq, dqd, dtau = m.fd_vjp(*(_dev(x, torch.float32) for x in (q, qd, tau, gb)))
    torch.cuda.synchronize()
    assert all(torch.isfinite(t).all() for t in (dq, dqd, dtau))
    idx = np.sort(gi.Stream(17).u64(256) % np.uint64(N)).astype(np.int64)
    q64, qd64, tau64, gb64 = (x[idx].astype(np.float64) for x in (q, qd, tau, gb))
    got = [t[torch.from_numpy(idx).cuda()].cpu().numpy() for t in (dq, dqd, dtau)]
    ref = oracle.fd_vjp(r, q64, qd64, tau64, gb64, nthreads=8)
    for g_, w_ in zip(got, ref):
        assert vec_rel_err(g_, w_) <= 1e-4
    # central differences of L = gbar . FD in FP64 (first 32 samples)
    h = 1e-6
    k = 32
    base = [q64[:k], qd64[:k], tau64[:k]]
    for u in range(3):
        fdiff = np.zeros((k, 12))
        for j in range(12):
            ap = [b.copy() for b in base]
            am = [b.copy() for b in base]
            ap[u][:, j] += h
            am[u][:, j] -= h
            fdiff[:, j] = ((oracle.fd(r, *ap) - oracle.fd(r, *am)) * gb64[:k]).sum(1) / (2 * h)
        assert vec_rel_err(got[u][:k], fdiff) <= 1e-4


def test_autograd_gradcheck_fp64(grid):
    """torch.autograd.gradcheck: the VJP kernel against finite differences of
    the FD kernel itself, in FP64."""
    for key in ("tree12", (6, 4)):
        r = _robot(key)
        m = grid.Model.from_robot(r)
        q, qd, tau = (_dev(x, torch.float64).requires_grad_() for x in gi.states(r.n, 3, 5))
        assert torch.autograd.gradcheck(lambda a, b, c: grid.forward_dynamics(m, a, b, c),
                                        (q, qd, tau), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_autograd_through_rollout(grid):
    """Gradients flow through a semi-implicit Euler rollout (dt = 0.01) built on
    the Function; checked against FP64 oracle finite differences of the same
    rollout."""
    r = gi.tree12()
    m = grid.Model.from_robot(r)
    B, H, dt = 4, 8, 0.01
    q0, qd0, _ = gi.states(12, B, 9)
    taus = gi.states(12, B * H, 10)[2].reshape(H, B, 12) * 0.2

    def rollout_torch(tau_seq):
        q = _dev(q0, torch.float64)
        qd = _dev(qd0, torch.float64)
        for t in range(H):
            qdd = grid.forward_dynamics(m, q, qd, tau_seq[t])
            qd = qd + dt * qdd
            q = q + dt * qd
        return (q ** 2).sum() + (qd ** 2).sum()

    tau_t = _dev(taus, torch.float64).requires_grad_()
    loss = rollout_torch(tau_t)
    loss.backward()
    g = tau_t.grad.cpu().numpy()

    def rollout_np(tau_seq):
        q, qd = q0.copy(), qd0.copy()
        for t in range(H):
            qd = qd + dt * oracle.fd(r, q, qd, tau_seq[t])
            q = q + dt * qd
        return (q ** 2).sum() + (qd ** 2).sum()

    h = 1e-6
    for (t, b, j) in [(0, 0, 0), (3, 1, 5), (7, 3, 11), (5, 2, 7)]:
        tp, tm = taus.copy(), taus.copy()
        tp[t, b, j] += h
        tm[t, b, j] -= h
        ref = (rollout_np(tp) - rollout_np(tm)) / (2 * h)
        assert abs(g[t, b, j] - ref) <= 1e-6 * max(1.0, abs(ref)), (t, b, j, g[t, b, j], ref)
