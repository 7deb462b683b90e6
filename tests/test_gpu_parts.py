"""Robots whose base components differ (the 30-DoF tree: torso with two arms,
and two legs) run the gradient of FD per component, the parts at the same time
on streams of their own. Checked against the FP64 oracle, against the kernel that runs the
whole robot, for every output entry (outputs pre-filled with NaN), and bit for
bit against the same components built as robots of their own."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import FLOOR32, FLOOR64, col_rel_err, col_rel_err_knots, fp32_bar, vec_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_PARTS = 401            # batch sizes above and below two knot points per SM
N_SMALL = 37


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


def _sub(r, idx):
    idx = list(idx)
    pos = {b: i for i, b in enumerate(idx)}
    par = np.array([pos.get(int(p), -1) for p in r.parent[idx]], dtype=np.int32)
    return gi.Robot(f"{r.name}[{idx[0]}:{idx[-1]}]", par, r.axis[idx].copy(), r.xtree[idx].copy(),
                    r.inertia[idx].copy(), r.gravity.copy())


def _interleaved_tree30():
    """The 30-DoF tree with its components interleaved in the caller's numbering
    (parents still before children): the parts gather and scatter by joint."""
    r = gi.tree30()
    arms_torso, leg1, leg2 = list(range(20)), list(range(20, 25)), list(range(25, 30))
    perm = []
    while arms_torso or leg1 or leg2:
        for lst in (arms_torso, leg1, arms_torso, leg2):
            if lst:
                perm.append(lst.pop(0))
    return r.permuted(perm)


ROBOTS = {"tree30": gi.tree30, "tree30-interleaved": _interleaved_tree30,
          "rand13": lambda: gi.random_tree(13, 21), "rand20": lambda: gi.random_tree(20, 3),
          "rand9": lambda: gi.random_tree(9, 8)}


def _inputs(n, N, seed, dt):
    q, qd, tau = gi.states(n, N, seed)
    npdt = np.float32 if dt == torch.float32 else np.float64
    dev = [torch.from_numpy(x.astype(npdt)).cuda() for x in (q, qd, tau)]
    return dev, [x.astype(npdt).astype(np.float64) for x in (q, qd, tau)]


@pytest.mark.parametrize("name", list(ROBOTS))
@pytest.mark.parametrize("prec", ["fp32", "mixed", "fp64"])
@pytest.mark.parametrize("N", [N_PARTS, N_SMALL])
def test_parts_match_oracle_and_whole_robot(grid, name, prec, N):
    r = ROBOTS[name]()
    roots = int(np.sum(r.parent < 0))
    assert roots >= 2, "the robot has several base components"
    n = r.n
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = grid.Model.from_robot(r, precision="mixed" if prec == "mixed" else "fp32")
    whole = grid.Model.from_robot(r, precision="mixed" if prec == "mixed" else "fp32")
    whole.set_option("specialize", 0)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 4100 + n, dt)
    J = torch.full((N, n, 2 * n), float("nan"), device="cuda", dtype=dt)
    Mi = torch.full((N, n, n), float("nan"), device="cuda", dtype=dt)
    m.grad_fd_minv(q, qd, tau, out=J, minv_out=Mi)
    qdd = torch.full((N, n), float("nan"), device="cuda", dtype=dt)
    J2 = m.grad_fd(q, qd, tau, qdd_out=qdd)
    Jw, qddw = whole.grad_fd(q, qd, tau, return_qdd=True)
    torch.cuda.synchronize()
    J, Mi, qdd, J2, Jw, qddw = (x.cpu().numpy() for x in (J, Mi, qdd, J2, Jw, qddw))
    assert np.isfinite(J).all() and np.isfinite(Mi).all() and np.isfinite(qdd).all()
    np.testing.assert_array_equal(J, J2)
    ref_J, ref_qdd = oracle.grad_fd(r, q64, qd64, tau64, nthreads=8, with_qdd=True)
    ref_Mi = oracle.minv(r, q64, nthreads=8)
    # entries coupling two base components are exactly zero
    root = np.array([i if p < 0 else -1 for i, p in enumerate(r.parent)])
    for i in range(n):
        if root[i] < 0:
            root[i] = root[r.parent[i]]
    cross = root[:, None] != root[None, :]
    assert np.all(Mi[:, cross] == 0) and np.all(J[:, :, :n][:, cross] == 0) and np.all(J[:, :, n:][:, cross] == 0)
    if prec == "fp64":
        assert col_rel_err(J, ref_J, FLOOR64) <= 1e-10
        assert col_rel_err(Mi, ref_Mi, FLOOR64) <= 1e-10
        assert vec_rel_err(qdd, ref_qdd) <= 1e-10
        assert col_rel_err(J, Jw, FLOOR64) <= 1e-10
    else:
        bar = fp32_bar(ref_Mi) if name.startswith("rand") else 1e-4
        assert np.all(col_rel_err_knots(J, ref_J, FLOOR32) <= bar)
        assert col_rel_err(Mi, ref_Mi, FLOOR32) <= 1e-4
        assert vec_rel_err(qdd, ref_qdd) <= 1e-4
        assert np.all(col_rel_err_knots(J, Jw, FLOOR32) <= 2 * np.maximum(bar, 1e-4))
        assert vec_rel_err(qdd, qddw) <= 1e-4


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("N", [N_PARTS, 1])
def test_parts_are_the_components_run_alone(grid, dt, N):
    """The 30-DoF tree's rows are, bit for bit, those of its torso-and-arms
    component and of each leg built as robots of their own (the same kernels on
    the same models), with exact zeros between components."""
    r = gi.tree30()
    m = grid.Model.from_robot(r)
    (q, qd, tau), _ = _inputs(30, N, 77, dt)
    J, qdd = m.grad_fd(q, qd, tau, return_qdd=True)
    J, qdd = J.cpu().numpy(), qdd.cpu().numpy()
    for idx in (range(0, 20), range(20, 25), range(25, 30)):
        idx = list(idx)
        sub = grid.Model.from_robot(_sub(r, idx))
        sel = torch.tensor(idx, device="cuda")
        Js, qdds = sub.grad_fd(q[:, sel].contiguous(), qd[:, sel].contiguous(), tau[:, sel].contiguous(),
                               return_qdd=True)
        Js, qdds = Js.cpu().numpy(), qdds.cpu().numpy()
        k = len(idx)
        np.testing.assert_array_equal(J[:, idx][:, :, idx], Js[:, :, :k])
        np.testing.assert_array_equal(J[:, idx][:, :, [30 + i for i in idx]], Js[:, :, k:])
        np.testing.assert_array_equal(qdd[:, idx], qdds)
        sub.close()
