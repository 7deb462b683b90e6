"""Pins of the FP64 oracle for prismatic and fixed joints (Sec. IV-B names
revolute, prismatic and fixed among the supported joints): closed forms of a
slider and a cart-pole, the independent Lagrangian formulation on random trees
of mixed joint types, complex-step derivatives, invariants, and fixed joints
against the same robot with every fixed body lumped into its parent by hand."""
import dataclasses

import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests import lagrange

G = 9.81
MIXED = [gi.random_mixed(n, s) for n, s in [(2, 1), (3, 2), (5, 3), (7, 4), (9, 5), (12, 6)]]


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("axis,gz", [((0.0, 0.0, 1.0), 1.0), ((1.0, 0.0, 0.0), 0.0),
                                     ((0.6, 0.0, 0.8), 0.8)])
def test_slider_closed_form(axis, gz):
    """A body translating along a fixed unit axis a: M = m, the gravity term is
    -m g.a (with g = (0, 0, -9.81)), and nothing depends on q or qd:
    tau = m qdd + m 9.81 a_z."""
    m = 1.7
    r = gi.slider(m=m, axis=axis)
    q, qd, qdd = gi.states(1, 5, 3)
    tau = oracle.rnea(r, q, qd, qdd)
    np.testing.assert_allclose(tau[:, 0], m * qdd[:, 0] + m * G * gz, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.mass_matrix(r, q)[:, 0, 0], m, rtol=1e-14)
    np.testing.assert_allclose(oracle.minv(r, q)[:, 0, 0], 1.0 / m, rtol=1e-14)
    np.testing.assert_allclose(oracle.fd(r, q, qd, tau)[:, 0], qdd[:, 0], rtol=1e-12, atol=1e-12)
    dq, dqd = oracle.grad_rnea(r, q, qd, qdd)
    np.testing.assert_allclose(dq, 0.0, atol=1e-13)
    np.testing.assert_allclose(dqd, 0.0, atol=1e-13)
    np.testing.assert_allclose(oracle.grad_fd(r, q, qd, tau), 0.0, atol=1e-13)


def test_cartpole_closed_form():
    """Cart x on a prismatic joint, pole angle t about y carrying a point mass
    mp at distance l. With L = KE - PE:
      M = [[mc + mp, mp l cos t], [mp l cos t, mp l^2]]
      tau_x = (mc + mp) x'' + mp l cos t t'' - mp l sin t t'^2
      tau_t = mp l cos t x'' + mp l^2 t'' - mp g l sin t."""
    mc, mp, l = 1.3, 0.4, 0.6
    r = gi.cartpole(mc, mp, l)
    q, qd, qdd = gi.states(2, 7, 17)
    t, td = q[:, 1], qd[:, 1]
    xdd, tdd = qdd[:, 0], qdd[:, 1]
    M = oracle.mass_matrix(r, q)
    np.testing.assert_allclose(M[:, 0, 0], mc + mp, rtol=1e-14)
    np.testing.assert_allclose(M[:, 0, 1], mp * l * np.cos(t), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(M[:, 1, 0], mp * l * np.cos(t), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(M[:, 1, 1], mp * l * l, rtol=1e-14)
    tau = oracle.rnea(r, q, qd, qdd)
    np.testing.assert_allclose(tau[:, 0], (mc + mp) * xdd + mp * l * np.cos(t) * tdd
                               - mp * l * np.sin(t) * td ** 2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(tau[:, 1], mp * l * np.cos(t) * xdd + mp * l * l * tdd
                               - mp * G * l * np.sin(t), rtol=1e-12, atol=1e-12)
    # derivatives of the closed form
    dq, dqd = oracle.grad_rnea(r, q, qd, qdd)
    np.testing.assert_allclose(dq[:, :, 0], 0.0, atol=1e-13)                  # nothing depends on x
    np.testing.assert_allclose(dq[:, 0, 1], -mp * l * np.sin(t) * tdd - mp * l * np.cos(t) * td ** 2,
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dq[:, 1, 1], -mp * l * np.sin(t) * xdd - mp * G * l * np.cos(t),
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dqd[:, 0, 1], -2 * mp * l * np.sin(t) * td, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dqd[:, 1, :], 0.0, atol=1e-13)
    np.testing.assert_allclose(dqd[:, 0, 0], 0.0, atol=1e-13)


# ------------------------------------------- independent Lagrangian formulation

@pytest.mark.parametrize("robot", MIXED + [gi.chain7_tool()], ids=lambda r: r.name)
def test_mixed_joints_match_lagrangian(robot):
    q, qd, qdd = gi.states(robot.nd, 3, 57)
    M = oracle.mass_matrix(robot, q)
    Z = np.zeros_like(q)
    Gq = oracle.rnea(robot, q, Z, Z)
    tau = oracle.rnea(robot, q, qd, qdd)
    for k in range(q.shape[0]):
        np.testing.assert_allclose(M[k], lagrange.mass_matrix(robot, q[k]), rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(Gq[k], lagrange.gravity_torque(robot, q[k]), rtol=1e-11, atol=1e-12)
        ref = lagrange.inverse_dynamics(robot, q[k], qd[k], qdd[k])
        np.testing.assert_allclose(tau[k], ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


# ---------------------------------------------------------------- invariants and derivatives

@pytest.mark.parametrize("robot", MIXED + [gi.chain7_tool(), gi.cartpole()], ids=lambda r: r.name)
def test_mixed_joints_invariants_and_derivatives(robot):
    nd = robot.nd
    q, qd, tau = gi.states(nd, 4, 61)
    M = oracle.mass_matrix(robot, q)
    Mi = oracle.minv(robot, q)
    for k in range(q.shape[0]):
        assert np.linalg.eigvalsh(M[k]).min() > 0
        np.testing.assert_allclose(M[k] @ Mi[k], np.eye(nd), atol=1e-10)
    qdd = oracle.fd(robot, q, qd, tau)
    np.testing.assert_allclose(oracle.rnea(robot, q, qd, qdd), tau, rtol=0, atol=1e-10)
    dq, dqd = oracle.grad_rnea(robot, q, qd, qdd)
    cq, cqd = oracle.rnea_complex_step(robot, q, qd, qdd)
    scale = max(np.abs(cq).max(), np.abs(cqd).max())
    np.testing.assert_allclose(dq, cq, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(dqd, cqd, rtol=0, atol=1e-12 * scale)
    J = oracle.grad_fd(robot, q, qd, tau)
    Jc = oracle.fd_complex_step(robot, q, qd, tau)
    np.testing.assert_allclose(J, Jc, rtol=0, atol=1e-11 * np.abs(Jc).max())


# ---------------------------------------------------------------- fixed joints by lumping

def _lump_fixed(robot):
    """The same robot with every fixed body merged into its parent (numpy,
    rigid-body composition written out here): the fixed body's mass, COM and
    rotational inertia join the parent's by the parallel-axis theorem, its
    children hang from the parent with composed fixed transforms, and a fixed
    body on the base is dropped with its inertia."""
    par = [int(p) for p in robot.parent]
    jt = list(robot.jtypes())
    axis = [np.array(a) for a in robot.axis]
    E = [robot.xtree[i, :9].reshape(3, 3).copy() for i in range(robot.n)]
    r = [robot.xtree[i, 9:].copy() for i in range(robot.n)]
    ine = [robot.inertia[i].copy() for i in range(robot.n)]
    alive = [True] * robot.n

    def Ic(p):
        Ixx, Iyy, Izz, Ixy, Ixz, Iyz = p[4:]
        return np.array([[Ixx, Ixy, Ixz], [Ixy, Iyy, Iyz], [Ixz, Iyz, Izz]])

    for f in range(robot.n):
        if jt[f] != gi.FIXED:
            continue
        alive[f] = False
        p = par[f]
        if p >= 0:
            # f's COM and inertia in p's frame: x_p = r_f + E_f^T x_f
            c_f = r[f] + E[f].T @ ine[f][1:4]
            I_f = E[f].T @ Ic(ine[f]) @ E[f]
            m1, c1, I1 = ine[p][0], ine[p][1:4], Ic(ine[p])
            m2 = ine[f][0]
            m = m1 + m2
            c = (m1 * c1 + m2 * c_f) / m
            Inew = np.zeros((3, 3))
            for mi, ci, Ii in ((m1, c1, I1), (m2, c_f, I_f)):
                d = ci - c
                Inew += Ii + mi * (d @ d * np.eye(3) - np.outer(d, d))
            ine[p] = np.array([m, *c, Inew[0, 0], Inew[1, 1], Inew[2, 2], Inew[0, 1], Inew[0, 2], Inew[1, 2]])
        for ch in range(f + 1, robot.n):
            if par[ch] == f:
                # X_T,ch X_T,f: E = E_ch E_f, r = r_f + E_f^T r_ch
                r[ch] = r[f] + E[f].T @ r[ch]
                E[ch] = E[ch] @ E[f]
                par[ch] = p
    keep = [i for i in range(robot.n) if alive[i]]
    new = {old: k for k, old in enumerate(keep)}
    parent = np.array([-1 if par[i] < 0 else new[par[i]] for i in keep], dtype=np.int32)
    return gi.Robot(robot.name + "-lumped", parent, np.array([axis[i] for i in keep]),
                    np.array([np.concatenate([E[i].reshape(9), r[i]]) for i in keep]),
                    np.array([ine[i] for i in keep]), robot.gravity.copy(),
                    np.array([jt[i] for i in keep], dtype=np.int32))


@pytest.mark.parametrize("robot", MIXED + [gi.chain7_tool()], ids=lambda r: r.name)
def test_fixed_joints_equal_lumped_robot(robot):
    lumped = _lump_fixed(robot)
    assert lumped.n == robot.nd
    q, qd, tau = gi.states(robot.nd, 4, 71)
    for fn in (oracle.minv, oracle.mass_matrix):
        a, b = fn(robot, q), fn(lumped, q)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())
    for fn in (oracle.rnea, oracle.fd, oracle.grad_fd):
        a, b = fn(robot, q, qd, tau), fn(lumped, q, qd, tau)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-11 * np.abs(b).max())


def test_prismatic_reading_fails_when_swapped():
    """Planted mistake in the robot instead of the oracle: treating the
    cart-pole's prismatic joint as revolute must change the dynamics (so the
    closed-form pins above are sensitive to the joint type)."""
    r = gi.cartpole()
    wrong = dataclasses.replace(r, jtype=np.array([gi.REVOLUTE, gi.REVOLUTE], dtype=np.int32))
    q, qd, qdd = gi.states(2, 3, 5)
    assert np.abs(oracle.rnea(r, q, qd, qdd) - oracle.rnea(wrong, q, qd, qdd)).max() > 1e-2
