"""Pins for the FP64 oracle: every oracle function is tied to something other
than itself (closed forms, an independent Lagrangian formulation, invariants of
Eq. (1), complex-step and central finite differences, permutation symmetry).
CPU only."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests import lagrange

G = gi.G_STD


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("m,l", [(2.0, 0.5), (0.7, 1.3)])
def test_single_pendulum_closed_form(m, l):
    """tau = m g l cos q + m l^2 qdd (Eq. (1) for one revolute joint)."""
    r = gi.pendulum(m, l)
    s = gi.Stream(7)
    q = s.uniform(-np.pi, np.pi, (16, 1))
    qd = s.uniform(-2, 2, (16, 1))
    qdd = s.uniform(-3, 3, (16, 1))
    tau = s.uniform(-5, 5, (16, 1))
    np.testing.assert_allclose(oracle.rnea(r, q, qd, qdd), m * G * l * np.cos(q) + m * l * l * qdd,
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.mass_matrix(r, q)[:, 0, 0], m * l * l, rtol=1e-14)
    np.testing.assert_allclose(oracle.minv(r, q)[:, 0, 0], 1.0 / (m * l * l), rtol=1e-14)
    qdd_fd = oracle.fd(r, q, qd, tau)
    np.testing.assert_allclose(qdd_fd, (tau - m * G * l * np.cos(q)) / (m * l * l), rtol=0, atol=1e-12)
    dq, dqd = oracle.grad_rnea(r, q, qd, qdd)
    np.testing.assert_allclose(dq[:, 0, 0], -m * G * l * np.sin(q[:, 0]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(dqd[:, 0, 0], 0.0, atol=1e-14)
    J = oracle.grad_fd(r, q, qd, tau)
    np.testing.assert_allclose(J[:, 0, 0], (G / l) * np.sin(q[:, 0]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(J[:, 0, 1], 0.0, atol=1e-14)


def test_acrobot_closed_form():
    """Two-link planar arm: textbook M, Coriolis and gravity terms."""
    m1, m2, l1, lc1, lc2, i1, i2 = 1.5, 1.0, 0.6, 0.3, 0.2, 0.02, 0.01
    r = gi.double_pendulum(m1, m2, l1, 0.4, lc1, lc2, i1, i2)
    s = gi.Stream(11)
    for _ in range(8):
        q1, q2 = s.uniform(-np.pi, np.pi, 2)
        qd1, qd2 = s.uniform(-2, 2, 2)
        qdd = s.uniform(-3, 3, 2)
        c2 = np.cos(q2)
        M = np.array([[i1 + i2 + m1 * lc1 ** 2 + m2 * (l1 ** 2 + lc2 ** 2 + 2 * l1 * lc2 * c2),
                       i2 + m2 * (lc2 ** 2 + l1 * lc2 * c2)],
                      [i2 + m2 * (lc2 ** 2 + l1 * lc2 * c2), i2 + m2 * lc2 ** 2]])
        h = m2 * l1 * lc2 * np.sin(q2)
        cor = np.array([-h * (2 * qd1 * qd2 + qd2 ** 2), h * qd1 ** 2])
        grav = G * np.array([(m1 * lc1 + m2 * l1) * np.cos(q1) + m2 * lc2 * np.cos(q1 + q2),
                             m2 * lc2 * np.cos(q1 + q2)])
        q = np.array([[q1, q2]])
        qd = np.array([[qd1, qd2]])
        np.testing.assert_allclose(oracle.mass_matrix(r, q)[0], M, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(oracle.rnea(r, q, qd, qdd[None])[0], M @ qdd + cor + grav,
                                   rtol=1e-12, atol=1e-12)


# ------------------------------------------- independent Lagrangian formulation

LAGRANGE_ROBOTS = [gi.random_tree(n, s) for n, s in [(1, 0), (2, 1), (3, 2), (4, 3), (6, 4)]] + [
    gi.random_tree(5, 5, general=False), gi.chain7(), gi.tree12()]


@pytest.mark.parametrize("robot", LAGRANGE_ROBOTS, ids=lambda r: r.name)
def test_mass_matrix_and_gravity_match_jacobian_form(robot):
    q, qd, tau = gi.states(robot.n, 3, 99)
    M = oracle.mass_matrix(robot, q)
    Z = np.zeros_like(q)
    Gq = oracle.rnea(robot, q, Z, Z)
    for k in range(q.shape[0]):
        np.testing.assert_allclose(M[k], lagrange.mass_matrix(robot, q[k]), rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(Gq[k], lagrange.gravity_torque(robot, q[k]), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("robot", LAGRANGE_ROBOTS[:6], ids=lambda r: r.name)
def test_rnea_matches_lagrangian_inverse_dynamics(robot):
    q, qd, qdd = gi.states(robot.n, 3, 123)
    tau = oracle.rnea(robot, q, qd, qdd)
    for k in range(q.shape[0]):
        ref = lagrange.inverse_dynamics(robot, q[k], qd[k], qdd[k])
        np.testing.assert_allclose(tau[k], ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


# ---------------------------------------------------------------- invariants

ALL_ROBOTS = [gi.chain7(), gi.tree12(), gi.tree30(), gi.random_tree(6, 7), gi.random_tree(9, 8)]


@pytest.mark.parametrize("robot", ALL_ROBOTS, ids=lambda r: r.name)
def test_mass_matrix_invariants(robot):
    q, qd, tau = gi.states(robot.n, 6, 5)
    M = oracle.mass_matrix(robot, q)
    Mi = oracle.minv(robot, q)
    for k in range(q.shape[0]):
        np.testing.assert_allclose(M[k], M[k].T, rtol=0, atol=1e-14 * np.abs(M[k]).max())
        assert np.linalg.eigvalsh(M[k]).min() > 0
        np.testing.assert_allclose(M[k] @ Mi[k], np.eye(robot.n), atol=1e-10)
        np.testing.assert_allclose(Mi[k], Mi[k].T, rtol=0, atol=1e-12 * np.abs(Mi[k]).max())
    # CRBA columns equal RNEA(q, 0, e_j) - RNEA(q, 0, 0)
    Z = np.zeros_like(q)
    base = oracle.rnea(robot, q, Z, Z)
    for j in range(robot.n):
        e = np.zeros_like(q)
        e[:, j] = 1.0
        np.testing.assert_allclose(oracle.rnea(robot, q, Z, e) - base, M[:, :, j], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("robot", ALL_ROBOTS, ids=lambda r: r.name)
def test_fd_inverts_rnea(robot):
    q, qd, tau = gi.states(robot.n, 6, 6)
    qdd = oracle.fd(robot, q, qd, tau)
    np.testing.assert_allclose(oracle.rnea(robot, q, qd, qdd), tau, rtol=0, atol=1e-10)


@pytest.mark.parametrize("robot", ALL_ROBOTS, ids=lambda r: r.name)
def test_grad_rnea_qd_structure(robot):
    q, qd, qdd = gi.states(robot.n, 4, 8)
    Z = np.zeros_like(qd)
    _, dqd0 = oracle.grad_rnea(robot, q, Z, qdd)
    np.testing.assert_allclose(dqd0, 0.0, atol=1e-13)                    # zero at qd = 0
    _, dqd1 = oracle.grad_rnea(robot, q, qd, qdd)
    _, dqd2 = oracle.grad_rnea(robot, q, 2 * qd, qdd)
    np.testing.assert_allclose(dqd2, 2 * dqd1, rtol=1e-11, atol=1e-12)    # linear in qd
    lhs = np.einsum("kij,kj->ki", dqd1, qd)                               # Euler homogeneity
    rhs = 2 * (oracle.rnea(robot, q, qd, qdd) - oracle.rnea(robot, q, Z, qdd))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-11)


def test_zero_column_for_vertical_base_axis():
    """Chain joint 1 rotates about gravity at the fixed base: the dynamics are
    invariant to it, so column dqdd/dq_1 vanishes."""
    r = gi.chain7()
    assert np.allclose(r.axis[0], [0, 0, 1]) and r.parent[0] == -1
    q, qd, tau = gi.states(7, 8, 1016)
    J = oracle.grad_fd(r, q, qd, tau)
    np.testing.assert_allclose(J[:, :, 0], 0.0, atol=1e-12)
    assert np.abs(J[:, :, 1:]).max() > 1.0


def test_tree12_block_structure():
    """Legs attached to the fixed base do not interact: M, M^-1 and J are block
    diagonal by leg."""
    r = gi.tree12()
    q, qd, tau = gi.states(12, 4, 2032)
    J = oracle.grad_fd(r, q, qd, tau)
    Mi = oracle.minv(r, q)
    for a in range(4):
        for b in range(4):
            if a == b:
                continue
            ra, rb = slice(3 * a, 3 * a + 3), slice(3 * b, 3 * b + 3)
            np.testing.assert_allclose(Mi[:, ra, rb], 0.0, atol=1e-13)
            np.testing.assert_allclose(J[:, ra, rb], 0.0, atol=1e-12)
            np.testing.assert_allclose(J[:, ra, 12 + 3 * b:12 + 3 * b + 3], 0.0, atol=1e-12)


# -------------------------------------------------------- derivative pins

DERIV_ROBOTS = ALL_ROBOTS + [gi.random_tree(n, 20 + n) for n in (1, 2, 3, 4)] + [gi.pendulum()]


@pytest.mark.parametrize("robot", DERIV_ROBOTS, ids=lambda r: r.name)
def test_grad_rnea_matches_complex_step(robot):
    q, qd, qdd = gi.states(robot.n, 3, 31)
    dq, dqd = oracle.grad_rnea(robot, q, qd, qdd)
    cq, cqd = oracle.rnea_complex_step(robot, q, qd, qdd)
    scale = max(np.abs(cq).max(), np.abs(cqd).max())
    np.testing.assert_allclose(dq, cq, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(dqd, cqd, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("robot", DERIV_ROBOTS, ids=lambda r: r.name)
def test_grad_fd_matches_complex_step(robot):
    q, qd, tau = gi.states(robot.n, 3, 37)
    J = oracle.grad_fd(robot, q, qd, tau)
    Jc = oracle.fd_complex_step(robot, q, qd, tau)
    np.testing.assert_allclose(J, Jc, rtol=0, atol=1e-11 * np.abs(Jc).max())


@pytest.mark.parametrize("robot", [gi.random_tree(n, 40 + n) for n in (1, 2, 3, 4)] + [gi.chain7()],
                         ids=lambda r: r.name)
def test_grad_fd_matches_central_differences(robot):
    """Central differences of FD in FP64, h = 1e-6: agreement to 1e-6 relative."""
    n = robot.n
    q, qd, tau = gi.states(n, 2, 41)
    J = oracle.grad_fd(robot, q, qd, tau)
    h = 1e-6
    for u, x in enumerate((q, qd)):
        for j in range(n):
            e = np.zeros_like(x)
            e[:, j] = h
            args_p = [q, qd, tau]
            args_m = [q, qd, tau]
            args_p[u] = x + e
            args_m[u] = x - e
            col = (oracle.fd(robot, *args_p) - oracle.fd(robot, *args_m)) / (2 * h)
            np.testing.assert_allclose(J[:, :, u * n + j], col, rtol=0,
                                       atol=1e-6 * max(1.0, np.abs(J).max()))


def test_sibling_permutation_equivariance():
    """Renumbering the legs of the 12-DoF tree permutes every output and
    changes nothing else."""
    r = gi.tree12()
    perm = np.array([6, 7, 8, 0, 1, 2, 9, 10, 11, 3, 4, 5])
    rp = r.permuted(perm)
    q, qd, tau = gi.states(12, 3, 77)
    J = oracle.grad_fd(r, q, qd, tau)
    Jp = oracle.grad_fd(rp, q[:, perm], qd[:, perm], tau[:, perm])
    cols = np.concatenate([perm, 12 + perm])
    np.testing.assert_allclose(Jp, J[:, perm][:, :, cols], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.minv(rp, q[:, perm]), oracle.minv(r, q)[:, perm][:, :, perm],
                               rtol=1e-12, atol=1e-14)


def test_fd_vjp_matches_finite_differences_of_loss():
    r = gi.tree12()
    q, qd, tau = gi.states(12, 2, 4)
    gbar = gi.upstream(12, 2, 4)
    dq, dqd, dtau = oracle.fd_vjp(r, q, qd, tau, gbar)
    h = 1e-6
    for u, (x, g) in enumerate(((q, dq), (qd, dqd), (tau, dtau))):
        for j in range(12):
            e = np.zeros_like(x)
            e[:, j] = h
            a_p = [q, qd, tau]
            a_m = [q, qd, tau]
            a_p[u] = x + e
            a_m[u] = x - e
            fdiff = ((oracle.fd(r, *a_p) - oracle.fd(r, *a_m)) * gbar).sum(1) / (2 * h)
            np.testing.assert_allclose(g[:, j], fdiff, rtol=1e-6, atol=1e-6)


def test_invalid_model_rejected():
    r = gi.chain7()
    bad = gi.Robot("bad", np.array([-1, 1, 1, 2, 3, 4, 5], dtype=np.int32), r.axis, r.xtree,
                   r.inertia, r.gravity)
    q, qd, tau = gi.states(7, 1, 1)
    with pytest.raises(oracle.OracleError):
        oracle.fd(bad, q, qd, tau)
