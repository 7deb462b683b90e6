"""GPU parity of the trajectory-optimisation step (rollout through FD, M^-1
from the gradient kernel, iLQR backward pass, policy rollout) against the
oracle's plain numpy forms (oracle/traj.py), FP64 and FP32, and one device
iteration reducing the tracking cost as predicted."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from oracle import traj
from tests.metrics import col_err_split

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = 0.01


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


def _problem(robot, B, H, seed):
    n = robot.nd
    s = gi.Stream(seed)
    q0, qd0, _ = gi.states(n, B, seed)
    U = 3.0 * s.normal((B, H + 1, n))
    U[:, H] = 0.0
    Qref = np.broadcast_to(0.5 * s.normal((B, 1, n)), (B, H + 1, n)).copy()
    QDref = np.zeros((B, H + 1, n))
    wq = np.concatenate([np.full(n, 10.0), np.full(n, 0.1)])
    wr = np.full(n, 1e-3)
    wf = 10.0 * wq
    return q0, qd0, U, Qref, QDref, wq, wr, wf


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("robot", [gi.chain7(), gi.tree12(), gi.cartpole(), gi.random_mixed(9, 5)],
                         ids=lambda r: r.name)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_rollout_and_minv_match_oracle(grid, robot, dtype):
    n, B, H = robot.nd, 13, 24
    q0, qd0, U, *_ = _problem(robot, B, H, 3)
    npdt = np.float64 if dtype == torch.float64 else np.float32
    q0, qd0, U = (x.astype(npdt).astype(np.float64) for x in (q0, qd0, U))
    m = grid.Model.from_robot(robot)
    Q, QD, Ua = m.rollout(_dev(q0, dtype), _dev(qd0, dtype), _dev(U, dtype), DT)
    qo, qdo, uo = traj.rollout(robot, DT, q0, qd0, U[:, :H])
    tol = 1e-9 if dtype == torch.float64 else 2e-3
    scale = max(np.abs(qo).max(), np.abs(qdo).max())
    assert np.abs(Q.cpu().numpy() - qo).max() <= tol * scale
    assert np.abs(QD.cpu().numpy() - qdo).max() <= tol * scale
    np.testing.assert_array_equal(Ua.cpu().numpy()[:, :H], U[:, :H].astype(npdt))
    # the gradient kernel's M^-1 output at the rolled-out knot points
    J, Mi = m.grad_fd_minv(Q, QD, _dev(U, dtype))
    qf, qdf, uf = (x.cpu().numpy().reshape(-1, n).astype(np.float64) for x in (Q, QD, _dev(U, dtype)))
    # FP32 bars as in the joint-type tests: small columns next to prismatic
    # (metre) columns take a 1e-3 floor, rounding-level columns an absolute bound
    if dtype == torch.float64:
        tol2, floor = (1e-10, 1e-12), 1e-6
    else:
        tol2 = (1e-3, 1e-5) if robot.name.startswith("mixed") else (1e-4, 1e-5)
        floor = 1e-3 if np.any(robot.jtypes() == gi.PRISMATIC) else 1e-4
    for got, ref in ((Mi, oracle.minv(robot, qf)), (J, oracle.grad_fd(robot, qf, qdf, uf))):
        e_nz, e_z = col_err_split(got.cpu().numpy(), ref, floor=floor)
        assert e_nz <= tol2[0] and e_z <= tol2[1], (e_nz, e_z)


@pytest.mark.parametrize("robot", [gi.chain7(), gi.tree12(), gi.cartpole()], ids=lambda r: r.name)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_riccati_matches_oracle(grid, robot, dtype):
    """The backward pass on the same nominal trajectory and derivatives: the
    oracle's numpy recursion fed the device's J and M^-1 (so that this test
    isolates the Riccati kernel), and in FP64 also the oracle's own."""
    n, B, H = robot.nd, 9, 20
    q0, qd0, U, Qref, QDref, wq, wr, wf = _problem(robot, B, H, 5)
    m = grid.Model.from_robot(robot)
    d = lambda x: _dev(x, dtype)
    Q, QD, _ = m.rollout(d(q0), d(qd0), d(U), DT)
    J, Mi = m.grad_fd_minv(Q, QD, d(U))
    mu = 1e-6
    K, kff, dV = m.riccati(Q, QD, d(U), J, Mi, d(Qref), d(QDref), d(wq), d(wr), d(wf), DT, mu)
    Qh, QDh, Jh, Mih = (x.cpu().numpy().astype(np.float64) for x in (Q, QD, J, Mi))
    Jh = Jh.reshape(B, H + 1, n, 2 * n)
    Mih = Mih.reshape(B, H + 1, n, n)
    I = np.eye(n)
    A = np.zeros((B, H, 2 * n, 2 * n))
    A[:, :, n:, :n] = DT * Jh[:, :H, :, :n]
    A[:, :, n:, n:] = I + DT * Jh[:, :H, :, n:]
    A[:, :, :n] = np.concatenate([I, np.zeros((n, n))], axis=1) + DT * A[:, :, n:]
    Bm = np.concatenate([DT * DT * Mih[:, :H], DT * Mih[:, :H]], axis=2)
    Uh = U.astype(Qh.dtype)
    Ko, ko, dVo = traj.riccati(A, Bm, Qh, QDh, Uh[:, :H], Qref, QDref, wq, wr, wf, mu)
    tol = 1e-9 if dtype == torch.float64 else 5e-3
    Kd, kd = K.cpu().numpy(), kff.cpu().numpy()
    assert np.abs(Kd[:, :H] - Ko).max() <= tol * np.abs(Ko).max()
    assert np.abs(kd[:, :H] - ko).max() <= tol * np.abs(ko).max()
    assert np.abs(dV.cpu().numpy() - dVo).max() <= tol * np.abs(dVo).max()
    assert np.all(Kd[:, H] == 0) and np.all(kd[:, H] == 0)
    if dtype == torch.float64:
        # the whole chain on the oracle: rollout, step Jacobians, backward pass
        qo, qdo, _ = traj.rollout(robot, DT, q0, qd0, U[:, :H])
        Ao, Bo = traj.step_jacobians(robot, DT, qo[:, :H].reshape(-1, n), qdo[:, :H].reshape(-1, n),
                                     U[:, :H].reshape(-1, n))
        Ko2, ko2, dVo2 = traj.riccati(Ao.reshape(B, H, 2 * n, 2 * n), Bo.reshape(B, H, 2 * n, n), qo, qdo,
                                      U[:, :H], Qref, QDref, wq, wr, wf, mu)
        assert np.abs(Kd[:, :H] - Ko2).max() <= 1e-8 * np.abs(Ko2).max()
        assert np.abs(dV.cpu().numpy() - dVo2).max() <= 1e-8 * np.abs(dVo2).max()


def test_policy_rollout_matches_oracle(grid):
    robot, B, H = gi.chain7(), 7, 16
    n = robot.nd
    q0, qd0, U, Qref, QDref, wq, wr, wf = _problem(robot, B, H, 8)
    m = grid.Model.from_robot(robot)
    d = lambda x: _dev(x, torch.float64)
    Q, QD, _ = m.rollout(d(q0), d(qd0), d(U), DT)
    J, Mi = m.grad_fd_minv(Q, QD, d(U))
    K, kff, dV = m.riccati(Q, QD, d(U), J, Mi, d(Qref), d(QDref), d(wq), d(wr), d(wf), DT, 1e-6)
    for alpha in (1.0, 0.3):
        Qn, QDn, Un = m.rollout(d(q0), d(qd0), d(U), DT, policy=(K, kff, Q, QD, alpha))
        qo, qdo, uo = traj.rollout(robot, DT, q0, qd0, U[:, :H], K.cpu().numpy()[:, :H], kff.cpu().numpy()[:, :H],
                                   Q.cpu().numpy(), QD.cpu().numpy(), alpha)
        assert np.abs(Qn.cpu().numpy() - qo).max() <= 1e-9 * np.abs(qo).max()
        assert np.abs(Un.cpu().numpy()[:, :H] - uo).max() <= 1e-9 * np.abs(uo).max()


def test_ilqr_iteration_reduces_cost_as_predicted(grid):
    """One device iteration (rollout, derivatives, backward pass, policy rollout)
    on the 7-DoF chain: with a small step the actual cost change matches the
    predicted alpha dV[0] + alpha^2 dV[1] to first order, and a backtracking line
    search over alpha lowers the cost of every trajectory."""
    robot, B, H = gi.chain7(), 16, 32
    q0, qd0, U, Qref, QDref, wq, wr, wf = _problem(robot, B, H, 12)
    U *= 0.1
    m = grid.Model.from_robot(robot)
    d = lambda x: _dev(x, torch.float64)

    def cost(Q, QD, Uu):
        return traj.cost(Q.cpu().numpy(), QD.cpu().numpy(), Uu.cpu().numpy()[:, :H], Qref, QDref, wq, wr, wf)

    Q, QD, _ = m.rollout(d(q0), d(qd0), d(U), DT)
    c0 = cost(Q, QD, d(U))
    alpha = 1e-3
    Qn, QDn, Un, dV = m.ilqr_iteration(d(q0), d(qd0), d(U), d(Qref), d(QDref), d(wq), d(wr), d(wf), DT, 1e-6,
                                       alpha)
    dV = dV.cpu().numpy()
    pred = alpha * dV[:, 0] + alpha ** 2 * dV[:, 1]
    assert np.all(pred < 0)
    np.testing.assert_allclose(cost(Qn, QDn, Un) - c0, pred, rtol=2e-2)
    best = np.full(B, np.inf)
    for a in (1.0, 0.5, 0.25, 0.125):                # backtracking line search
        Qn, QDn, Un, _ = m.ilqr_iteration(d(q0), d(qd0), d(U), d(Qref), d(QDref), d(wq), d(wr), d(wf), DT, 1e-6, a)
        best = np.fmin(best, cost(Qn, QDn, Un))         # a diverged full step is NaN
    assert np.all(best < c0)


def test_riccati_limits(grid):
    m = grid.Model.from_robot(gi.tree30())
    n = 30
    z = torch.zeros((1, 3, n), device="cuda")
    w = torch.ones(2 * n, device="cuda")
    with pytest.raises(grid.GridError) as ei:
        m.riccati(z, z, z, torch.zeros((3, n, 2 * n), device="cuda"), torch.zeros((3, n, n), device="cuda"),
                  z, z, w, w[:n], w, DT)
    assert ei.value.status == 1
