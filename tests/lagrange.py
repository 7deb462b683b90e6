"""Independent Lagrangian dynamics for pinning the oracle (tests only).

Written with world-frame homogeneous kinematics and geometric Jacobians
(textbook manipulator dynamics), sharing nothing with the spatial-algebra
oracle: no Plucker transforms, no cross-product operators, no recursions.

  R_i = R_parent E_T,i^T Rot(a_i, q_i),   p_i = p_parent + R_parent r_i
  x_i = p_i + R_i c_i                     (COM of link i)
  Jv_i[:, j] = z_j x (x_i - p_j),  Jw_i[:, j] = z_j  for j on the path to i
  M = sum_i m_i Jv_i^T Jv_i + Jw_i^T R_i Ic_i R_i^T Jw_i
  G = -sum_i m_i Jv_i^T g
  C(q, qd) qd = Mdot qd - 1/2 d/dq (qd^T M qd)   (central differences in q)
  tau = M qdd + C qd + G                  (Eq. (1) with B = I, F = 0)
"""
import numpy as np


def _rot(a, q):
    a = np.asarray(a, dtype=float)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(q) * K + (1 - np.cos(q)) * K @ K


def kinematics(robot, q):
    n = robot.n
    R = [None] * n
    p = [None] * n
    for i in range(n):
        par = robot.parent[i]
        Rp = np.eye(3) if par < 0 else R[par]
        pp = np.zeros(3) if par < 0 else p[par]
        E = robot.xtree[i, :9].reshape(3, 3)
        r = robot.xtree[i, 9:]
        p[i] = pp + Rp @ r
        R[i] = Rp @ E.T @ _rot(robot.axis[i], q[i])
    return R, p


def _path(robot, i):
    out = []
    while i >= 0:
        out.append(i)
        i = robot.parent[i]
    return out


def mass_matrix(robot, q):
    n = robot.n
    R, p = kinematics(robot, q)
    M = np.zeros((n, n))
    for i in range(n):
        m = robot.inertia[i, 0]
        c = robot.inertia[i, 1:4]
        Ixx, Iyy, Izz, Ixy, Ixz, Iyz = robot.inertia[i, 4:]
        Ic = np.array([[Ixx, Ixy, Ixz], [Ixy, Iyy, Iyz], [Ixz, Iyz, Izz]])
        x = p[i] + R[i] @ c
        Jv = np.zeros((3, n))
        Jw = np.zeros((3, n))
        for j in _path(robot, i):
            z = R[j] @ robot.axis[j]
            Jv[:, j] = np.cross(z, x - p[j])
            Jw[:, j] = z
        M += m * Jv.T @ Jv + Jw.T @ (R[i] @ Ic @ R[i].T) @ Jw
    return M


def gravity_torque(robot, q):
    n = robot.n
    R, p = kinematics(robot, q)
    G = np.zeros(n)
    g = robot.gravity
    for i in range(n):
        m = robot.inertia[i, 0]
        x = p[i] + R[i] @ robot.inertia[i, 1:4]
        for j in _path(robot, i):
            z = R[j] @ robot.axis[j]
            G[j] -= m * np.cross(z, x - p[j]) @ g
    return G


def inverse_dynamics(robot, q, qd, qdd, h=1e-6):
    n = robot.n
    M = mass_matrix(robot, q)
    dM = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        dM.append((mass_matrix(robot, q + e) - mass_matrix(robot, q - e)) / (2 * h))
    Mdot = sum(dM[k] * qd[k] for k in range(n))
    grad_ke = np.array([0.5 * qd @ dM[k] @ qd for k in range(n)])
    return M @ qdd + Mdot @ qd - grad_ke + gravity_torque(robot, q)
