"""Pins of the operation count (oracle/opcount.py) that the benchmark's roofline
divides by: primitive costs and the whole method for one and two bodies counted
by hand, the counted route's values against the oracle's dense FP64 route, and
the benchmark's flop table against the count."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from oracle import opcount as oc


def _nums(k, seed):
    rng = np.random.default_rng(seed)
    return [oc.Num(x) for x in rng.normal(size=k)]


def _count(fn, *args):
    c0 = oc._C.n
    fn(*args)
    return oc._C.n - c0


def test_primitive_costs():
    """Compact forms with state-dependent operands everywhere:
    X m = [E w; E (v - r x w)]: 15 + (9 + 3) + 15 = 42; X^T f likewise 15 + 15 + 9 + 3;
    I m = [Ibar w + h x v; m v - h x w]: (15 + 9 + 3) + (3 + 9 + 3) = 42;
    a x b and a x* f: three 3-vector cross products (9 each) and one 3-add = 30;
    S^T f = a . n: 3 + 2."""
    E, r, m = _nums(9, 1), _nums(3, 2), _nums(6, 3)
    inert = (1.3, [0.1, -0.2, 0.05], [0.3, 0.01, 0.02, 0.01, 0.4, 0.03, 0.02, 0.03, 0.5])
    ax = [0.0, 0.6, 0.8]
    assert _count(oc.x_mul, E, r, m) == 42
    assert _count(oc.xt_mul, E, r, m) == 42
    assert _count(oc.i_mul, inert, m) == 42
    assert _count(oc.crm, m, _nums(6, 4)) == 30
    assert _count(oc.crf, m, _nums(6, 5)) == 30
    assert _count(oc.st_f, ax, m) == 5
    # structural zeros: X applied to a revolute S q (= [a q; 0]) skips v - r x w's v
    # and leaves 15 + 9 + 15; a cross product with S q's zero half costs 18
    sq = _nums(3, 6) + [None] * 3
    assert _count(oc.x_mul, E, r, sq) == 39
    assert _count(oc.crm, m, sq) == 18
    # model constants alone cost nothing (done once at model creation)
    assert _count(oc.x_mul, [0.5] * 9, [0.1] * 3, [0.2] * 6) == 0


def _prefix(n):
    """A chain of the first n bodies of a random tree: general unit axes, E_T = 1."""
    r = gi.random_tree(7, 31)
    xt = np.concatenate([np.tile(np.eye(3).ravel(), (n, 1)), r.xtree[:n, 9:]], axis=1)
    return gi.Robot(f"first{n}", np.arange(-1, n - 1, dtype=np.int32), r.axis[:n].copy(), xt,
                    r.inertia[:n].copy(), r.gravity.copy())


def test_count_one_body_by_hand():
    """One revolute joint on the fixed base, E_T = 1.
    transforms 36: sin, cos (2); 1 - cos (1); E_J's diagonal (1-c) a_u a_u + c: 3 x 3;
      off-diagonal (1-c) a_u a_v +- s a_k: 6 x 4.
    RNEA(q, qd, 0) 122: S qd 3; X a_0 with a_0 = [0; -g] 15; v x S qd = [w x w'; 0] 9;
      gamma = I v with v = [w; 0] 15 + 9; f = I a 42 + v x* gamma 18 + 6; c = S^T f 5.
    M^-1 0: M = S^T I S is a model constant.
    FD 2: tau - c, one product.
    RNEA at qdd 36: S qdd 3; a += 3; f += I (S qdd) 24 + 6.
    dRNEA 124: column q: da = (X a_0) x S = [0; 9 ops] 9, df = I da (da = [0; v]) 12,
      dc = 5; column qd: da = v x S 9, + S x S qd 9 + 3, df = I da 24 + S x* gamma 18 +
      v x* (I S) 18 + 6 + 6, dc = 5.
    product 2: one product per column."""
    cnt = oc.grad_fd_counted(_prefix(1), [0.4], [0.3], [-1.2])[0]
    assert cnt == {"transforms": 36, "rnea_bias": 122, "minv": 0, "fd": 2, "rnea_qdd": 36,
                   "grad_rnea": 124, "product": 2, "total": 322}


def test_count_two_bodies_by_hand():
    """Chain of two revolute joints (bodies 0 and 1), E_T = 1.
    transforms 72 (2 x 36).
    RNEA(q, qd, 0) 406: body 0 as for one body, 117 before its S^T f; body 1: S qd 3,
      X v_0 (v_0 = [w; 0]) 39, + S qd 3, X a_0 42, v x S qd 18 + 6, gamma 42,
      f = I a 42 + v x* gamma 30 + 6 (231); backward S^T F 5 + 5 and X^T F 42 + 6.
    M^-1 694: body 1 (a leaf: U, D, D^-1 and the downdate are model constants):
      X^T of its F column 42, congruence X^T A X as 12 X^T products 504, added to
      the 24 non-structural entries of I_0 (570); body 0: U = I^A S 30, D 5,
      D^-1 1, Minv[0][1] 5 + 1, F columns 6 + 12 (60); forward: P_0 = S Minv[0][k]
      3 + 3; body 1: X P_0 39, U . t 11, times D^-1 and subtract 2, P_1 3 + 3 (58).
    FD 8: 2 subtractions, 2 x (2 products + 1 add).
    RNEA at qdd 189: body 0 36; body 1: X da_0 39, + S qdd 3 + 3, X a_p update 6,
      a += 6, f += I da 42 + 6; X^T F 42 + 6.
    dRNEA 982: column (q, 0): body 0 9 + 12, body 1 X da 15 + I da 12, backward
      5 + (42 + 6) + 5 (106); column (q, 1): (X v) x S 18, (X a) x S 18,
      dv x S qd 18 + 6, df 42 + 30 + (42 + 30) + 12, S x* F 18 + 6, backward
      5 + 42 + 5 (292); column (qd, 0): body 0 9 + 12 + 72, body 1 X S 30, X da 39,
      24, 156, backward 5 + 48 + 5 (400); column (qd, 1): v x S 18, S x S qd 9 + 3,
      df 42 + 18 + 30 + 12, backward 5 + 42 + 5 (184).
    product 24: 2 rows x 4 columns x (2 products + 1 add)."""
    cnt = oc.grad_fd_counted(_prefix(2), [0.4, -0.7], [0.3, 0.5], [-1.2, 2.0])[0]
    assert cnt == {"transforms": 72, "rnea_bias": 406, "minv": 694, "fd": 8, "rnea_qdd": 189,
                   "grad_rnea": 982, "product": 24, "total": 2375}


@pytest.mark.parametrize("robot", [gi.chain7(), gi.tree12(), gi.tree30(), gi.random_tree(9, 4),
                                   gi.random_tree(12, 8, max_children=2)], ids=lambda r: r.name)
def test_counted_route_matches_oracle(robot):
    """The counted evaluation is a correct one: its J, qdd and M^-1 equal the
    oracle's (CRBA + Cholesky and dense 6x6 algebra) to FP64 rounding."""
    q, qd, tau = gi.states(robot.n, 2, 77)
    Jr, qddr = oracle.grad_fd(robot, q, qd, tau, with_qdd=True)
    Mr = oracle.minv(robot, q)
    for k in range(2):
        _, J, qdd, Mi = oc.grad_fd_counted(robot, q[k], qd[k], tau[k])
        np.testing.assert_allclose(J, Jr[k], rtol=0, atol=1e-11 * np.abs(Jr[k]).max())
        np.testing.assert_allclose(qdd, qddr[k], rtol=0, atol=1e-11 * np.abs(qddr[k]).max())
        np.testing.assert_allclose(Mi, Mr[k], rtol=0, atol=1e-11 * np.abs(Mr[k]).max())


def test_count_does_not_depend_on_the_state():
    r = gi.tree12()
    q, qd, tau = gi.states(12, 2, 5)
    c0 = oc.grad_fd_counted(r, q[0], qd[0], tau[0])[0]
    c1 = oc.grad_fd_counted(r, q[1], qd[1], tau[1])[0]
    assert c0 == c1


def test_bench_flop_table_is_the_count():
    import bench
    for name, flops in bench.FLOPS_PER_KNOT.items():
        assert flops == oc.grad_fd_flops_per_knot(gi.robot(name)), name
