"""Operation count of one gradient-of-forward-dynamics evaluation, by execution.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests are the only
callers (they also check the flop table that the benchmark divides by against
this count). Nothing here is shared with the CUDA path.

The method's own steps for one knot point are executed once in compact form on
a counting scalar, in the order of Sec. IV-B:
  a2 joint transforms X_i = X_J(q_i) X_T,i held as (E, r) (Sec. III-B),
  a3 RNEA(q, qd, 0): forward v, a, f and backward c_i = S_i^T F_i,
  a4 M^-1 directly by the articulated-inertia recursion (Carpentier 2018; the
     paper cites it in Sec. IV-B), backward sweep then forward sweep,
  a5 qdd = M^-1 (tau - c),
  a6 RNEA at qdd as a linear update of the accelerations and forces,
  a7 dRNEA forward pass of Alg. 1 for every column (u, j), over subtree(j),
  a8 its backward pass over subtree(j) and the ancestors of j, with the
     accumulated-force term X^T (S_j x* F_j) for u = q (the readings c3-c5),
  a9 J = -M^-1 [dc/dq | dc/dqd], restricted to the blocks of the base branches.
The values are real results: tests check them against the oracle's dense FP64
route (CRBA + Cholesky, Alg. 1 with dense 6x6 algebra), so every counted
operation belongs to a correct evaluation of the method.

Counting rules:
  * every multiply, add, subtract and divide between values that depend on the
    knot point's state counts 1 (an FMA counts 2); sin and cos count 1 each;
    a change of sign counts 0;
  * arithmetic among model constants only (inertias, axes, fixed transforms,
    gravity) counts 0: it is done once when the model is created;
  * structural zeros count 0: the linear half of a revolute S_i = [a_i; 0], the
    base's zero velocity and the zero derivatives of bodies outside the column's
    subtree or above its joint, and E_J E_T when E_T is the identity;
  * the joint axes are general unit vectors: products with an axis component
    count even where that component is zero.
Revolute joints only (the workload robots).
"""
from __future__ import annotations

import math

import numpy as np


class Counter:
    def __init__(self):
        self.n = 0


class Num:
    """A value that depends on the knot point's state; arithmetic on it counts."""
    __slots__ = ("v",)

    def __init__(self, v):
        self.v = float(v)


# Scalars are Num (state-dependent, counted), float (model constant) or None
# (structural zero). Vectors and matrices are Python lists of scalars.
_C = Counter()


def _val(a):
    return 0.0 if a is None else (a.v if isinstance(a, Num) else float(a))


def _res(a, b, v):
    if isinstance(a, Num) or isinstance(b, Num):
        _C.n += 1
        return Num(v)
    return float(v)


def add(a, b):
    if a is None:
        return b
    if b is None:
        return a
    return _res(a, b, _val(a) + _val(b))


def sub(a, b):
    if b is None:
        return a
    if a is None:
        return neg(b)
    return _res(a, b, _val(a) - _val(b))


def mul(a, b):
    if a is None or b is None:
        return None
    return _res(a, b, _val(a) * _val(b))


def div(a, b):
    if a is None:
        return None
    return _res(a, b, _val(a) / _val(b))


def neg(a):
    if a is None:
        return None
    return Num(-a.v) if isinstance(a, Num) else -float(a)


def fsin(a):
    _C.n += 1
    return Num(math.sin(_val(a)))


def fcos(a):
    _C.n += 1
    return Num(math.cos(_val(a)))


def dot(a, b):
    s = None
    for x, y in zip(a, b):
        s = add(s, mul(x, y))
    return s


def vadd(a, b):
    return [add(x, y) for x, y in zip(a, b)]


def vsub(a, b):
    return [sub(x, y) for x, y in zip(a, b)]


def vscale(a, s):
    return [mul(x, s) for x in a]


def is_zero(a):
    return all(x is None for x in a)


Z6 = [None] * 6


# ---------------------------------------------------------------- spatial algebra, compact forms
def cross3(a, b):
    return [sub(mul(a[1], b[2]), mul(a[2], b[1])),
            sub(mul(a[2], b[0]), mul(a[0], b[2])),
            sub(mul(a[0], b[1]), mul(a[1], b[0]))]


def mat3_vec(E, w):          # E w, E row-major 3x3
    return [dot(E[3 * i:3 * i + 3], w) for i in range(3)]


def mat3t_vec(E, w):         # E^T w
    return [dot([E[i], E[3 + i], E[6 + i]], w) for i in range(3)]


def x_mul(E, r, m):
    """X m = [E w; E (v - r x w)] for X = [E 0; -E r~ E], m = [w; v]."""
    w, v = m[:3], m[3:]
    return mat3_vec(E, w) + mat3_vec(E, vsub(v, cross3(r, w)))


def xt_mul(E, r, f):
    """X^T f = [E^T n + r x (E^T f); E^T f] for f = [n; f]."""
    g = mat3t_vec(E, f[3:])
    return vadd(mat3t_vec(E, f[:3]), cross3(r, g)) + g


def i_mul(I, m):
    """I m for I = (mass, h = mass c, Ibar about the body origin): [Ibar w + h x v; mass v - h x w]."""
    mass, h, Ib = I
    w, v = m[:3], m[3:]
    return vadd(mat3_vec(Ib, w), cross3(h, v)) + vsub(vscale(v, mass), cross3(h, w))


def crm(a, b):
    """a x b (motion cross product, Eq. (2))."""
    return cross3(a[:3], b[:3]) + vadd(cross3(a[:3], b[3:]), cross3(a[3:], b[:3]))


def crf(a, f):
    """a x* f (force cross product, Eq. (2))."""
    return vadd(cross3(a[:3], f[:3]), cross3(a[3:], f[3:])) + cross3(a[:3], f[3:])


def s_vec(ax):               # S = [a; 0] (revolute)
    return [float(x) for x in ax] + [None, None, None]


def st_f(ax, f):             # S^T f
    return dot([float(x) for x in ax], f[:3])


def mat6_s(A, ax):           # A S = A[:, :3] a
    return [dot(A[r][:3], [float(x) for x in ax]) for r in range(6)]


# ---------------------------------------------------------------- the method
def _model(robot):
    parent, axis, xtree, inertia, gravity = robot.arrays()
    if robot.jtype is not None and np.any(robot.jtypes() != 0):
        raise ValueError("the operation count covers revolute joints only")
    n = robot.n
    inert, I6 = [], []
    for i in range(n):
        m, c, (xx, yy, zz, xy, xz, yz) = inertia[i, 0], inertia[i, 1:4], inertia[i, 4:10]
        Ic = np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])
        Ib = Ic + m * (np.dot(c, c) * np.eye(3) - np.outer(c, c))      # about the body origin
        h = m * c
        inert.append((float(m), [float(x) for x in h], [float(x) for x in Ib.ravel()]))
        ht = np.array([[0, -h[2], h[1]], [h[2], 0, -h[0]], [-h[1], h[0], 0]])
        full = np.block([[Ib, ht], [ht.T, m * np.eye(3)]])
        # structural zeros of [Ibar h~; h~^T mass 1]: the diagonals of h~ and the
        # off-diagonal entries of mass 1 (whatever the values of c)
        zero = lambda r, s: (r < 3) != (s < 3) and r % 3 == s % 3 or (r >= 3 and s >= 3 and r != s)
        I6.append([[None if zero(r, s) else float(full[r, s]) for s in range(6)] for r in range(6)])
    a0 = [None, None, None] + [-float(g) for g in gravity]     # a general direction: zeros count
    return parent.tolist(), axis, xtree, inert, I6, a0


def _topology(parent):
    n = len(parent)
    children = [[] for _ in range(n)]
    for i, p in enumerate(parent):
        if p >= 0:
            children[p].append(i)
    subt = [[i] for i in range(n)]
    for i in reversed(range(n)):
        for c in children[i]:
            subt[i] += subt[c]
    for i in range(n):
        subt[i].sort()
    anc = [[] for _ in range(n)]
    for i in range(n):
        p = parent[i]
        while p >= 0:
            anc[i].append(p)
            p = parent[p]
    root = [i if parent[i] < 0 else None for i in range(n)]
    for i in range(n):
        if parent[i] >= 0:
            root[i] = root[parent[i]]
    comp = [sorted(k for k in range(n) if root[k] == root[i]) for i in range(n)]
    return children, subt, anc, comp


def grad_fd_counted(robot, q, qd, tau):
    """Runs the method for one knot point on the counting scalar.
    Returns (counts by step, J [n, 2n], qdd [n], Minv [n, n]) with the values
    as FP64 numpy arrays."""
    parent, axis, xtree, inert, I6, a0 = _model(robot)
    n = len(parent)
    children, subt, anc, comp = _topology(parent)
    q = [Num(x) for x in q]
    qd = [Num(x) for x in qd]
    tau = [Num(x) for x in tau]
    counts = {}

    def mark(name, start):
        counts[name] = _C.n - start
        return _C.n

    t0 = _C.n = 0
    # a2: joint transforms, E_J = R(a, q)^T = cos q 1 + (1 - cos q) a a^T - sin q a~
    E, r = [], []
    for i in range(n):
        a = [float(x) for x in axis[i]]
        s, co = fsin(q[i]), fcos(q[i])
        omc = sub(1.0, co)
        EJ = [None] * 9
        for u in range(3):
            for v in range(3):
                e = mul(mul(omc, a[u]), a[v])
                e = add(co, e) if u == v else e
                # - sin q a~ : a~ = [[0, -a2, a1], [a2, 0, -a0], [-a1, a0, 0]]
                if u != v:
                    k = 3 - u - v
                    sign = 1.0 if (u, v) in ((0, 1), (1, 2), (2, 0)) else -1.0
                    e = add(e, mul(s, sign * a[k]))
                EJ[3 * u + v] = e
        ET = xtree[i, :9]
        if np.array_equal(ET, np.eye(3).ravel()):
            Ei = EJ
        else:
            Ei = [dot(EJ[3 * u:3 * u + 3], [float(ET[v]), float(ET[3 + v]), float(ET[6 + v])])
                  for u in range(3) for v in range(3)]
        E.append(Ei)
        r.append([float(x) for x in xtree[i, 9:12]])
    t0 = mark("transforms", t0)

    # a3: RNEA(q, qd, 0)
    v, a, f, Xa, Xv = [None] * n, [None] * n, [None] * n, [None] * n, [None] * n
    vJ, gam = [None] * n, [None] * n
    for i in range(n):
        p = parent[i]
        vJ[i] = vscale(s_vec(axis[i]), qd[i])
        Xv[i] = Z6 if p < 0 else x_mul(E[i], r[i], v[p])
        v[i] = vadd(Xv[i], vJ[i])
        Xa[i] = x_mul(E[i], r[i], a0 if p < 0 else a[p])
        a[i] = vadd(Xa[i], crm(v[i], vJ[i]))
        gam[i] = i_mul(inert[i], v[i])
        f[i] = vadd(i_mul(inert[i], a[i]), crf(v[i], gam[i]))
    F = [list(x) for x in f]
    c = [None] * n
    for i in reversed(range(n)):
        c[i] = st_f(axis[i], F[i])
        if parent[i] >= 0:
            F[parent[i]] = vadd(F[parent[i]], xt_mul(E[i], r[i], F[i]))
    t0 = mark("rnea_bias", t0)

    # a4: M^-1 by the articulated-inertia recursion.
    # Backward: I^A_i = I_i + sum_children X_c^T (I^A_c - U_c D_c^-1 U_c^T) X_c,
    # U_i = I^A_i S_i, D_i = S_i^T U_i, Minv[i][i] = D_i^-1,
    # Minv[i][k] = -D_i^-1 S_i^T Fc[k] (k in subtree(i), k != i),
    # Fc[k] <- X_i^T (Fc[k] + U_i Minv[i][k]) for k in subtree(i).
    Mi = [[None] * n for _ in range(n)]
    IA = [[row[:] for row in I6[i]] for i in range(n)]
    Fc = [Z6] * n
    U, Dinv = [None] * n, [None] * n
    for i in reversed(range(n)):
        S_ax = axis[i]
        U[i] = mat6_s(IA[i], S_ax)
        D = st_f(S_ax, U[i])
        Dinv[i] = div(1.0, D)
        Mi[i][i] = Dinv[i]
        for k in subt[i]:
            if k != i:
                Mi[i][k] = neg(mul(Dinv[i], st_f(S_ax, Fc[k])))
        for k in subt[i]:
            Fc[k] = vadd(Fc[k], vscale(U[i], Mi[i][k]))
        p = parent[i]
        if p >= 0:
            for k in subt[i]:
                Fc[k] = xt_mul(E[i], r[i], Fc[k])
            w = vscale(U[i], Dinv[i])
            A = [[sub(IA[i][u][s], mul(w[u], U[i][s])) if s >= u else None for s in range(6)] for u in range(6)]
            for u in range(6):
                for s in range(u):
                    A[u][s] = A[s][u]
            # X^T A X: B = X^T A column by column, then X^T B^T (A and the result symmetric)
            B = [xt_mul(E[i], r[i], [A[u][s] for u in range(6)]) for s in range(6)]   # column s of X^T A
            for s in range(6):
                col = xt_mul(E[i], r[i], [B[u][s] for u in range(6)])             # column s of X^T A X
                for u in range(6):
                    IA[p][u][s] = add(IA[p][u][s], col[u])
    # Forward: for k >= i in i's base branch, t = X_i P_parent[k],
    # Minv[i][k] -= D_i^-1 U_i^T t, P_i[k] = S_i Minv[i][k] + t.
    P = [[None] * n for _ in range(n)]
    for i in range(n):
        p = parent[i]
        S = s_vec(axis[i])
        for k in comp[i]:
            if k < i:
                continue
            t = Z6 if p < 0 or P[p][k] is None else x_mul(E[i], r[i], P[p][k])
            if not is_zero(t):
                Mi[i][k] = sub(Mi[i][k], mul(Dinv[i], dot(U[i], t)))
            P[i][k] = vadd(vscale(S, Mi[i][k]), t)
    for i in range(n):
        for k in comp[i]:
            if k < i:
                Mi[i][k] = Mi[k][i]
    t0 = mark("minv", t0)

    # a5: qdd = M^-1 (tau - c)
    rhs = [sub(tau[i], c[i]) for i in range(n)]
    qdd = [dot([Mi[i][k] for k in comp[i]], [rhs[k] for k in comp[i]]) for i in range(n)]
    t0 = mark("fd", t0)

    # a6: RNEA at qdd: da_i = X_i da_p + S_i qdd_i, a_i += da_i, f_i += I_i da_i;
    # X_i a_p at qdd for the case term; accumulated forces F_i
    da = [None] * n
    for i in range(n):
        p = parent[i]
        Xda = Z6 if p < 0 else x_mul(E[i], r[i], da[p])
        da[i] = vadd(Xda, vscale(s_vec(axis[i]), qdd[i]))
        Xa[i] = vadd(Xa[i], Xda)
        a[i] = vadd(a[i], da[i])
        f[i] = vadd(f[i], i_mul(inert[i], da[i]))
    F = [list(x) for x in f]
    for i in reversed(range(n)):
        if parent[i] >= 0:
            F[parent[i]] = vadd(F[parent[i]], xt_mul(E[i], r[i], F[i]))
    t0 = mark("rnea_qdd", t0)

    # a7, a8: dRNEA, one column (u, j) at a time
    dc = [[None] * (2 * n) for _ in range(n)]
    for uq in (True, False):
        for j in range(n):
            S_j = s_vec(axis[j])
            dv, dA, df = {}, {}, {}
            for k in subt[j]:
                p = parent[k]
                dvp = dv.get(p, Z6)
                dap = dA.get(p, Z6)
                dvk = Z6 if is_zero(dvp) else x_mul(E[k], r[k], dvp)
                dak = Z6 if is_zero(dap) else x_mul(E[k], r[k], dap)
                if k == j:
                    if uq:
                        dvk = vadd(dvk, crm(Xv[k], S_j))
                        dak = vadd(dak, crm(Xa[k], S_j))
                    else:
                        dvk = vadd(dvk, S_j)
                        dak = vadd(dak, crm(v[k], S_j))
                dak = vadd(dak, crm(dvk, vJ[k]))
                dv[k], dA[k] = dvk, dak
                df[k] = vadd(vadd(i_mul(inert[k], dak), crf(dvk, gam[k])), crf(v[k], i_mul(inert[k], dvk)))
            # backward over subtree(j) and the ancestors of j, leaves to root; for
            # u = q the parent of j also receives X_j^T (S_j x* F_j)
            dF = {k: df[k] for k in subt[j]}
            if uq and parent[j] >= 0:
                dF[j] = vadd(dF[j], crf(S_j, F[j]))
            for k in reversed(sorted(list(subt[j]) + anc[j])):
                col = (0 if uq else n) + j
                dc[k][col] = st_f(axis[k], dF[k])
                p = parent[k]
                if p >= 0:
                    dF[p] = vadd(dF.get(p, Z6), xt_mul(E[k], r[k], dF[k]))
    t0 = mark("grad_rnea", t0)

    # a9: J = -M^-1 dc on the blocks of the base branches
    J = [[None] * (2 * n) for _ in range(n)]
    for i in range(n):
        for col in range(2 * n):
            j = col % n
            if comp[j] is comp[i] or comp[j] == comp[i]:
                J[i][col] = neg(dot([Mi[i][k] for k in comp[i]], [dc[k][col] for k in comp[i]]))
    mark("product", t0)
    counts["total"] = sum(counts.values())

    def arr(x):
        return np.array([[_val(e) for e in row] for row in x]) if isinstance(x[0], list) else \
            np.array([_val(e) for e in x])
    return counts, arr(J), arr(qdd), arr(Mi)


def grad_fd_flops_per_knot(robot, seed=12345):
    """Total counted operations of one knot point (the count does not depend on
    the state's values)."""
    rng = np.random.default_rng(seed)
    n = robot.n
    q, qd, tau = rng.uniform(-np.pi, np.pi, n), rng.uniform(-1, 1, n), rng.uniform(-5, 5, n)
    return grad_fd_counted(robot, q, qd, tau)[0]["total"]
