"""GPU parity for prismatic and fixed joints: every entry point through the
C-ABI against the FP64 oracle (which treats fixed joints natively, while the
library merges them into their parents at creation), FP32 and FP64."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import FLOOR32, col_err_split, col_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOTS = [gi.slider(), gi.cartpole(), gi.chain7_tool()] + \
    [gi.random_mixed(n, s) for n, s in [(2, 1), (3, 2), (5, 3), (7, 4), (9, 5), (12, 6), (20, 7), (38, 8)]]


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


@pytest.mark.parametrize("robot", ROBOTS, ids=lambda r: r.name)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_joint_types_match_oracle(grid, robot, dtype):
    nd = robot.nd
    m = grid.Model.from_robot(robot)
    assert m.n == nd
    N = 45
    npdt = np.float32 if dtype == torch.float32 else np.float64
    q, qd, tau = (x.astype(npdt) for x in gi.states(nd, N, 19))
    gbar = gi.upstream(nd, N, 19).astype(npdt)
    q64, qd64, tau64, g64 = (x.astype(np.float64) for x in (q, qd, tau, gbar))
    dq_, dqd_, dtau_, dg_ = (torch.from_numpy(x).cuda() for x in (q, qd, tau, gbar))
    # Bars on (e over non-zero columns, e over structurally zero columns). FP64:
    # 1e-10 / 1e-12. FP32: 1e-4 / 1e-5 on the constructed robots; the random
    # mixed trees put prismatic (metres) and revolute (radians) columns side by
    # side and their mass matrices reach condition numbers ~1e3, so FP32 rounding
    # (~1e-7 of the largest column, times the conditioning) is held to 1e-3,
    # and a column counts as small below 1e-3 of the largest when a joint is
    # prismatic (different units) instead of 1e-4.
    if dtype == torch.float64:
        tol, floor = (1e-10, 1e-12), 1e-6
    else:
        tol = (1e-3, 1e-5) if robot.name.startswith("mixed") else (1e-4, 1e-5)
        floor = 1e-3 if np.any(robot.jtypes() == gi.PRISMATIC) else FLOOR32

    def ok(x, y, vec=False):
        x, y = np.asarray(x), np.asarray(y)
        if vec:
            x, y = x[:, :, None], y[:, :, None]
        e_nz, e_z = col_err_split(x, y, floor=floor)
        return e_nz <= tol[0] and e_z <= tol[1]

    assert ok(m.rnea(dq_, dqd_, dtau_).cpu().numpy(), oracle.rnea(robot, q64, qd64, tau64), vec=True)
    assert ok(m.minv(dq_).cpu().numpy(), oracle.minv(robot, q64))
    assert ok(m.fd(dq_, dqd_, dtau_).cpu().numpy(), oracle.fd(robot, q64, qd64, tau64), vec=True)
    J, qdd = m.grad_fd(dq_, dqd_, dtau_, return_qdd=True)
    Jo, qddo = oracle.grad_fd(robot, q64, qd64, tau64, with_qdd=True)
    assert ok(J.cpu().numpy(), Jo)
    assert ok(qdd.cpu().numpy(), qddo, vec=True)
    dq, dqd = oracle.grad_rnea(robot, q64, qd64, tau64)
    assert ok(m.grad_rnea(dq_, dqd_, dtau_).cpu().numpy(), np.concatenate([dq, dqd], axis=2))
    # the three VJP outputs as the columns of one [N, nd, 3] block
    got = np.stack([x.cpu().numpy() for x in m.fd_vjp(dq_, dqd_, dtau_, dg_)], axis=2)
    ref = np.stack(oracle.fd_vjp(robot, q64, qd64, tau64, g64), axis=2)
    assert ok(got, ref)


def test_chain_with_fixed_bodies_uses_chain_kernel_result(grid):
    """A 7-DoF chain with fixed sensor and tool bodies reduces to a serial
    chain; the chain-compiled and run-time-topology kernels agree and match
    the oracle."""
    r = gi.chain7_tool()
    spec = grid.Model.from_robot(r)
    gen = grid.Model.from_robot(r)
    gen.set_option("specialize", 0)
    q, qd, tau = (x.astype(np.float32) for x in gi.states(7, 300, 23))
    d = [torch.from_numpy(x).cuda() for x in (q, qd, tau)]
    Js = spec.grad_fd(*d).cpu().numpy()
    Jg = gen.grad_fd(*d).cpu().numpy()
    ref = oracle.grad_fd(r, *(x.astype(np.float64) for x in (q, qd, tau)))
    assert col_rel_err(Js, ref) <= 1e-4
    assert col_rel_err(Jg, ref) <= 1e-4
    assert col_rel_err(Js, Jg) <= 1e-4


def test_joint_type_errors(grid):
    r = gi.cartpole()
    with pytest.raises(grid.GridError) as ei:
        grid.Model(r.parent, r.axis, r.xtree, r.inertia, jtype=[1, 3])
    assert ei.value.status == 1
    with pytest.raises(grid.GridError) as ei:
        grid.Model(r.parent, r.axis, r.xtree, r.inertia, jtype=[2, 2])
    assert ei.value.status == 2
