"""Pins of the oracle's trajectory-optimisation step (oracle/traj.py): closed-form
rollout, step Jacobians against central differences, the Riccati recursion
against scipy's discrete algebraic Riccati equation, and one iteration on a
linear system against the optimum of the dense equality-constrained QP."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from oracle import traj

scipy_linalg = pytest.importorskip("scipy.linalg")


def test_slider_rollout_closed_form():
    """q'' = u/m - g along a vertical slider: qd_k = qd_0 + k dt a and
    q_k = q_0 + dt (k qd_0 + dt a k (k + 1) / 2) for the semi-implicit step."""
    m, dt, H = 1.7, 0.01, 25
    r = gi.slider(m=m, axis=(0.0, 0.0, 1.0))
    q0 = np.array([[0.3], [-0.2]])
    qd0 = np.array([[0.1], [0.5]])
    u = np.array([2.0, 30.0])
    U = np.repeat(u[:, None, None], H, axis=1)
    q, qd, ua = traj.rollout(r, dt, q0, qd0, U)
    a = u / m - 9.81
    k = np.arange(H + 1)
    np.testing.assert_allclose(qd[:, :, 0], qd0 + k[None] * dt * a[:, None], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(q[:, :, 0], q0 + dt * (k[None] * qd0 + dt * a[:, None] * k * (k + 1) / 2),
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(ua, U)


@pytest.mark.parametrize("robot", [gi.chain7(), gi.random_mixed(7, 4), gi.tree12()], ids=lambda r: r.name)
def test_step_jacobians_match_central_differences(robot):
    n, dt, h = robot.nd, 0.01, 1e-6
    q, qd, u = gi.states(n, 3, 81)

    def step(q, qd, u):
        qdd = oracle.fd(robot, q, qd, u)
        qd1 = qd + dt * qdd
        return np.concatenate([q + dt * qd1, qd1], axis=1)

    A, Bm = traj.step_jacobians(robot, dt, q, qd, u)
    for j in range(2 * n):
        e = np.zeros((3, n))
        e[:, j % n] = h
        if j < n:
            col = (step(q + e, qd, u) - step(q - e, qd, u)) / (2 * h)
        else:
            col = (step(q, qd + e, u) - step(q, qd - e, u)) / (2 * h)
        np.testing.assert_allclose(A[:, :, j], col, rtol=1e-6, atol=1e-8)
    for j in range(n):
        e = np.zeros((3, n))
        e[:, j] = h
        col = (step(q, qd, u + e) - step(q, qd, u - e)) / (2 * h)
        np.testing.assert_allclose(Bm[:, :, j], col, rtol=1e-6, atol=1e-9)


def _random_lti(m, seed):
    s = gi.Stream(seed)
    A = np.eye(2 * m) + 0.05 * s.normal((2 * m, 2 * m))
    Bm = 0.1 * s.normal((2 * m, m))
    return A, Bm


def test_riccati_converges_to_dare_gain():
    """Time-invariant A, B and a long horizon: the first gain of the recursion
    equals the infinite-horizon LQR gain -(R + B^T P B)^-1 B^T P A with P from
    scipy's DARE solver."""
    m, H = 3, 400
    A, Bm = _random_lti(m, 5)
    wq = np.linspace(1.0, 2.0, 2 * m)
    wr = np.linspace(0.1, 0.3, m)
    wf = wq.copy()
    z = np.zeros((1, H + 1, m))
    K, kff, dV = traj.riccati(np.broadcast_to(A, (1, H, 2 * m, 2 * m)), np.broadcast_to(Bm, (1, H, 2 * m, m)),
                              z, z, np.zeros((1, H, m)), z, z, wq, wr, wf)
    P = scipy_linalg.solve_discrete_are(A, Bm, np.diag(wq), np.diag(wr))
    Kdare = -np.linalg.solve(np.diag(wr) + Bm.T @ P @ Bm, Bm.T @ P @ A)
    np.testing.assert_allclose(K[0, 0], Kdare, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(kff, 0.0, atol=1e-14)             # at the reference with zero controls


def test_one_iteration_solves_linear_quadratic_problem():
    """Linear time-varying dynamics with offsets, x_{k+1} = A_k x_k + B_k u_k + c_k:
    one backward pass plus a forward pass with alpha = 1 lands on the optimum of
    the QP (here solved densely by eliminating the states), and the predicted
    change dV[0] + dV[1] is the actual change of the cost."""
    m, H, Bn = 2, 12, 2
    s = gi.Stream(9)
    A = np.stack([np.stack([_random_lti(m, 100 + 20 * b + k)[0] for k in range(H)]) for b in range(Bn)])
    Bm = np.stack([np.stack([_random_lti(m, 100 + 20 * b + k)[1] for k in range(H)]) for b in range(Bn)])
    c = 0.05 * s.normal((Bn, H, 2 * m))
    x0 = s.normal((Bn, 2 * m))
    U = 0.3 * s.normal((Bn, H, m))
    ref = 0.5 * s.normal((Bn, H + 1, 2 * m))
    wq = np.linspace(1.0, 3.0, 2 * m)
    wr = np.linspace(0.2, 0.5, m)
    wf = 2.0 * wq

    def run(U, K=None, kff=None, X=None):
        Xn = np.zeros((Bn, H + 1, 2 * m))
        Un = np.zeros_like(U)
        Xn[:, 0] = x0
        for k in range(H):
            u = U[:, k] if K is None else U[:, k] + kff[:, k] + np.einsum("bij,bj->bi", K[:, k], Xn[:, k] - X[:, k])
            Un[:, k] = u
            Xn[:, k + 1] = np.einsum("bij,bj->bi", A[:, k], Xn[:, k]) + np.einsum("bij,bj->bi", Bm[:, k], u) + c[:, k]
        return Xn, Un

    def total(X, U):
        return traj.cost(X[:, :, :m], X[:, :, m:], U, ref[:, :, :m], ref[:, :, m:], wq, wr, wf)

    X, _ = run(U)
    K, kff, dV = traj.riccati(A, Bm, X[:, :, :m], X[:, :, m:], U, ref[:, :, :m], ref[:, :, m:], wq, wr, wf)
    X1, U1 = run(U, K, kff, X)
    np.testing.assert_allclose(total(X1, U1) - total(X, U), dV.sum(axis=1), rtol=1e-9, atol=1e-10)
    # dense optimum: X = Phi U + psi, minimise over the stacked controls
    for b in range(Bn):
        Phi = np.zeros((H + 1, 2 * m, H * m))
        psi = np.zeros((H + 1, 2 * m))
        psi[0] = x0[b]
        for k in range(H):
            Phi[k + 1] = A[b, k] @ Phi[k]
            Phi[k + 1][:, k * m:(k + 1) * m] += Bm[b, k]
            psi[k + 1] = A[b, k] @ psi[k] + c[b, k]
        W = [np.diag(wq)] * H + [np.diag(wf)]
        Hm = np.kron(np.eye(H), np.diag(wr))
        g = np.zeros(H * m)
        for k in range(H + 1):
            Hm += Phi[k].T @ W[k] @ Phi[k]
            g += Phi[k].T @ W[k] @ (psi[k] - ref[b, k])
        Uopt = np.linalg.solve(Hm, -g).reshape(H, m)
        np.testing.assert_allclose(U1[b], Uopt, rtol=1e-9, atol=1e-10)


def test_policy_rollout_closed_loop_slider():
    """The policy branch of the rollout, u_k = U_k + alpha kff_k + K_k (x_k - xnom_k),
    on a vertical slider (q'' = u/m - g exactly). With U = m g + u0, K = [-kp, -kd]
    and constant kff and xnom = (qn, qdn), the closed loop is a damped oscillator
    about the fixed point q* = qn + (u0 + alpha kff + kd qdn) / kp, qd* = 0, and
    the semi-implicit step maps the offset e = x - x* by the constant matrix
        A_cl = [[1 - dt^2 kp/m, dt (1 - dt kd/m)], [-dt kp/m, 1 - dt kd/m]],
    so e_k = A_cl^k e_0 (matrix powers, no recursion). A flipped sign of K dx,
    alpha applied to K instead of kff, or alpha left out moves the fixed point or
    the decay and fails this pin."""
    m, dt, H, alpha = 1.7, 0.01, 60, 0.37
    r = gi.slider(m=m, axis=(0.0, 0.0, 1.0))
    g = 9.81
    kp = np.array([40.0, 15.0])
    kd = np.array([6.0, 2.5])
    u0 = np.array([0.8, -1.1])
    kffv = np.array([2.0, -3.0])
    qn = np.array([0.25, -0.4])
    qdn = np.array([0.3, -0.2])
    q0 = np.array([[0.5], [0.1]])
    qd0 = np.array([[-0.2], [0.4]])
    Bn = 2
    U = np.repeat((m * g + u0)[:, None, None], H, axis=1)
    K = np.zeros((Bn, H, 1, 2))
    K[:, :, 0, 0] = -kp[:, None]
    K[:, :, 0, 1] = -kd[:, None]
    kff = np.repeat(kffv[:, None, None], H, axis=1)
    Qnom = np.repeat(qn[:, None, None], H + 1, axis=1)
    QDnom = np.repeat(qdn[:, None, None], H + 1, axis=1)
    q, qd, ua = traj.rollout(r, dt, q0, qd0, U, K=K, kff=kff, Qnom=Qnom, QDnom=QDnom, alpha=alpha)
    for b in range(Bn):
        qs = qn[b] + (u0[b] + alpha * kffv[b] + kd[b] * qdn[b]) / kp[b]
        Acl = np.array([[1 - dt * dt * kp[b] / m, dt * (1 - dt * kd[b] / m)],
                        [-dt * kp[b] / m, 1 - dt * kd[b] / m]])
        e0 = np.array([q0[b, 0] - qs, qd0[b, 0]])
        for k in range(H + 1):
            e = np.linalg.matrix_power(Acl, k) @ e0
            np.testing.assert_allclose(q[b, k, 0], qs + e[0], rtol=1e-11, atol=1e-11)
            np.testing.assert_allclose(qd[b, k, 0], e[1], rtol=1e-11, atol=1e-11)
            if k < H:    # the applied control holds the slider's acceleration: m (q'' + g)
                qdd = (-kp[b] * e[0] - kd[b] * e[1]) / m
                np.testing.assert_allclose(ua[b, k, 0], m * (qdd + g), rtol=1e-11, atol=1e-10)
