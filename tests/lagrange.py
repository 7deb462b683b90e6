"""Independent Lagrangian dynamics for pinning the oracle (tests only).

Written with world-frame homogeneous kinematics and geometric Jacobians
(textbook manipulator dynamics), sharing nothing with the spatial-algebra
oracle: no Plucker transforms, no cross-product operators, no recursions.

  revolute:  R_i = R_parent E_T,i^T Rot(a_i, q_i),  p_i = p_parent + R_parent r_i
  prismatic: R_i = R_parent E_T,i^T,  p_i = p_parent + R_parent r_i + R_i a_i q_i
  fixed:     R_i = R_parent E_T,i^T,  p_i = p_parent + R_parent r_i   (no joint variable)
  x_i = p_i + R_i c_i                     (COM of link i)
  for the moving joint j of a body on the path to i, with z_j = R_j a_j:
    revolute  Jv_i[:, j] = z_j x (x_i - p_j),  Jw_i[:, j] = z_j
    prismatic Jv_i[:, j] = z_j,                Jw_i[:, j] = 0
  M = sum_i m_i Jv_i^T Jv_i + Jw_i^T R_i Ic_i R_i^T Jw_i
  G = -sum_i m_i Jv_i^T g
  C(q, qd) qd = Mdot qd - 1/2 d/dq (qd^T M qd)   (central differences in q)
  tau = M qdd + C qd + G                  (Eq. (1) with B = I, F = 0)
"""
import numpy as np

REVOLUTE, PRISMATIC, FIXED = 0, 1, 2


def _jt(robot):
    return np.zeros(robot.n, dtype=int) if robot.jtype is None else np.asarray(robot.jtype)


def _dofs(robot):
    """body -> joint-variable index (-1 for a fixed joint)."""
    jt = _jt(robot)
    out, d = [], 0
    for i in range(robot.n):
        out.append(-1 if jt[i] == FIXED else d)
        d += jt[i] != FIXED
    return out


def _rot(a, q):
    a = np.asarray(a, dtype=float)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(q) * K + (1 - np.cos(q)) * K @ K


def kinematics(robot, q):
    n = robot.n
    jt, dof = _jt(robot), _dofs(robot)
    R = [None] * n
    p = [None] * n
    for i in range(n):
        par = robot.parent[i]
        Rp = np.eye(3) if par < 0 else R[par]
        pp = np.zeros(3) if par < 0 else p[par]
        E = robot.xtree[i, :9].reshape(3, 3)
        r = robot.xtree[i, 9:]
        p[i] = pp + Rp @ r
        R[i] = Rp @ E.T
        if jt[i] == REVOLUTE:
            R[i] = R[i] @ _rot(robot.axis[i], q[dof[i]])
        elif jt[i] == PRISMATIC:
            p[i] = p[i] + R[i] @ (np.asarray(robot.axis[i]) * q[dof[i]])
    return R, p


def _jacobians(robot, R, p, i, x):
    """Linear and angular Jacobians of the point x on body i, [3, nd] each."""
    jt, dof = _jt(robot), _dofs(robot)
    Jv = np.zeros((3, robot.nd))
    Jw = np.zeros((3, robot.nd))
    for j in _path(robot, i):
        if jt[j] == FIXED:
            continue
        z = R[j] @ robot.axis[j]
        if jt[j] == REVOLUTE:
            Jv[:, dof[j]] = np.cross(z, x - p[j])
            Jw[:, dof[j]] = z
        else:
            Jv[:, dof[j]] = z
    return Jv, Jw


def _path(robot, i):
    out = []
    while i >= 0:
        out.append(i)
        i = robot.parent[i]
    return out


def mass_matrix(robot, q):
    nd = robot.nd
    R, p = kinematics(robot, q)
    M = np.zeros((nd, nd))
    for i in range(robot.n):
        m = robot.inertia[i, 0]
        c = robot.inertia[i, 1:4]
        Ixx, Iyy, Izz, Ixy, Ixz, Iyz = robot.inertia[i, 4:]
        Ic = np.array([[Ixx, Ixy, Ixz], [Ixy, Iyy, Iyz], [Ixz, Iyz, Izz]])
        x = p[i] + R[i] @ c
        Jv, Jw = _jacobians(robot, R, p, i, x)
        M += m * Jv.T @ Jv + Jw.T @ (R[i] @ Ic @ R[i].T) @ Jw
    return M


def gravity_torque(robot, q):
    R, p = kinematics(robot, q)
    G = np.zeros(robot.nd)
    g = robot.gravity
    for i in range(robot.n):
        m = robot.inertia[i, 0]
        x = p[i] + R[i] @ robot.inertia[i, 1:4]
        Jv, _ = _jacobians(robot, R, p, i, x)
        G -= m * Jv.T @ g
    return G


def inverse_dynamics(robot, q, qd, qdd, h=1e-6):
    n = robot.nd
    M = mass_matrix(robot, q)
    dM = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        dM.append((mass_matrix(robot, q + e) - mass_matrix(robot, q - e)) / (2 * h))
    Mdot = sum(dM[k] * qd[k] for k in range(n))
    grad_ke = np.array([0.5 * qd @ dM[k] @ qd for k in range(n)])
    return M @ qdd + Mdot @ qd - grad_ke + gravity_torque(robot, q)
