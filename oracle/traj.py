"""Trajectory-optimisation step on the FP64 oracle: rollout, linearisation and
the iLQR (DDP without second-order dynamics terms) backward pass.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests are the only
callers. Plain numpy loops over knot points, written from the textbook forms:

Dynamics (a semi-implicit Euler step through forward dynamics, Sec. IV-B):
    qdd_k = FD(q_k, qd_k, u_k)
    qd_{k+1} = qd_k + dt qdd_k,   q_{k+1} = q_k + dt qd_{k+1}
so with Jq = dqdd/dq, Jv = dqdd/dqd and dqdd/du = M^-1 (Sec. IV-B items 3, 5),
the step's Jacobians w.r.t. x = (q, qd) and u are
    A = [[1 + dt^2 Jq, dt (1 + dt Jv)], [dt Jq, 1 + dt Jv]],   B = [[dt^2 M^-1], [dt M^-1]].

Cost: sum_k 1/2 (x_k - r_k)^T W_q (x_k - r_k) + 1/2 u_k^T W_r u_k over k < H, plus
1/2 (x_H - r_H)^T W_f (x_H - r_H); diagonal weights.

Backward pass (Li and Todorov 2004; Tassa, Erez and Todorov 2012), k = H-1 .. 0:
    Q_x = l_x + A^T V_x,   Q_u = l_u + B^T V_x
    Q_xx = l_xx + A^T V_xx A,   Q_uu = l_uu + B^T V_xx B + mu 1,   Q_ux = B^T V_xx A
    K = -Q_uu^-1 Q_ux,   k = -Q_uu^-1 Q_u
    V_x = Q_x + K^T Q_uu k + K^T Q_u + Q_ux^T k
    V_xx = Q_xx + K^T Q_uu K + K^T Q_ux + Q_ux^T K   (then symmetrised)
    dV += (k^T Q_u, 1/2 k^T Q_uu k)
starting from V_x = W_f (x_H - r_H), V_xx = W_f.

Pins (tests/test_oracle_traj.py): the rollout of a slider under constant force
against its closed form; the rollout under a feedback policy on the same slider
against the closed-loop fixed point and powers of the closed-loop matrix; A and
B against central differences of the step;
the Riccati gains of a linear time-invariant system against the discrete
algebraic Riccati equation solved by scipy; one iteration on a linear system
reaching the optimum of the equality-constrained QP solved by a dense KKT
system, with the predicted reduction dV equal to the actual one.
"""
from __future__ import annotations

import numpy as np

from . import fd, grad_fd, minv


def rollout(robot, dt, q0, qd0, U, K=None, kff=None, Qnom=None, QDnom=None, alpha=1.0):
    """q, qd [B, H+1, n] and the applied controls [B, H, n]. With a policy
    (K [B, H, n, 2n], kff [B, H, n] and the nominal states), the control at step k
    is u_k = U_k + alpha kff_k + K_k (x_k - xnom_k)."""
    q0 = np.asarray(q0, np.float64)
    Bn, n = q0.shape
    H = np.asarray(U).shape[1]
    q = np.zeros((Bn, H + 1, n))
    qd = np.zeros((Bn, H + 1, n))
    ua = np.zeros((Bn, H, n))
    q[:, 0], qd[:, 0] = q0, qd0
    for k in range(H):
        u = np.asarray(U[:, k], np.float64).copy()
        if K is not None:
            dx = np.concatenate([q[:, k] - Qnom[:, k], qd[:, k] - QDnom[:, k]], axis=1)
            u = u + alpha * kff[:, k] + np.einsum("bij,bj->bi", K[:, k], dx)
        ua[:, k] = u
        qdd = fd(robot, q[:, k], qd[:, k], u)
        qd[:, k + 1] = qd[:, k] + dt * qdd
        q[:, k + 1] = q[:, k] + dt * qd[:, k + 1]
    return q, qd, ua


def step_jacobians(robot, dt, q, qd, u):
    """A [N, 2n, 2n] and B [N, 2n, n] of the semi-implicit Euler step at each
    knot point (q, qd, u [N, n])."""
    n = q.shape[1]
    J = grad_fd(robot, q, qd, u)
    Mi = minv(robot, q)
    Jq, Jv = J[:, :, :n], J[:, :, n:]
    I = np.eye(n)[None]
    A = np.zeros((q.shape[0], 2 * n, 2 * n))
    A[:, n:, :n] = dt * Jq
    A[:, n:, n:] = I + dt * Jv
    A[:, :n, :n] = I + dt * A[:, n:, :n]
    A[:, :n, n:] = dt * A[:, n:, n:]
    Bm = np.zeros((q.shape[0], 2 * n, n))
    Bm[:, n:] = dt * Mi
    Bm[:, :n] = dt * Bm[:, n:]
    return A, Bm


def cost(q, qd, u, qref, qdref, wq, wr, wf):
    """Total tracking cost per trajectory [B]."""
    x = np.concatenate([q, qd], axis=2)
    r = np.concatenate([qref, qdref], axis=2)
    e = x - r
    run = 0.5 * np.einsum("bki,i,bki->b", e[:, :-1], wq, e[:, :-1]) + 0.5 * np.einsum("bki,i,bki->b", u, wr, u)
    return run + 0.5 * np.einsum("bi,i,bi->b", e[:, -1], wf, e[:, -1])


def riccati(A, Bm, q, qd, u, qref, qdref, wq, wr, wf, mu=0.0):
    """Backward pass. A [B, H, 2n, 2n], Bm [B, H, 2n, n], states [B, H+1, n],
    controls [B, H, n], references [B, H+1, n]. Returns K [B, H, n, 2n],
    kff [B, H, n], dV [B, 2]."""
    Bn, H, n2, n = Bm.shape
    x = np.concatenate([q, qd], axis=2)
    r = np.concatenate([qref, qdref], axis=2)
    Wq, Wr, Wf = np.diag(wq), np.diag(wr), np.diag(wf)
    K = np.zeros((Bn, H, n, n2))
    kff = np.zeros((Bn, H, n))
    dV = np.zeros((Bn, 2))
    for b in range(Bn):
        Vx = Wf @ (x[b, H] - r[b, H])
        Vxx = Wf.copy()
        for k in range(H - 1, -1, -1):
            a, bm = A[b, k], Bm[b, k]
            lx = Wq @ (x[b, k] - r[b, k])
            lu = Wr @ u[b, k]
            Qx = lx + a.T @ Vx
            Qu = lu + bm.T @ Vx
            Qxx = Wq + a.T @ Vxx @ a
            Quu = Wr + bm.T @ Vxx @ bm + mu * np.eye(n)
            Qux = bm.T @ Vxx @ a
            Kk = -np.linalg.solve(Quu, Qux)
            kk = -np.linalg.solve(Quu, Qu)
            Vx = Qx + Kk.T @ Quu @ kk + Kk.T @ Qu + Qux.T @ kk
            Vxx = Qxx + Kk.T @ Quu @ Kk + Kk.T @ Qux + Qux.T @ Kk
            Vxx = 0.5 * (Vxx + Vxx.T)
            K[b, k], kff[b, k] = Kk, kk
            dV[b] += (kk @ Qu, 0.5 * kk @ Quu @ kk)
    return K, kff, dV
