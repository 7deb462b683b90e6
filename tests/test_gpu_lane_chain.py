"""GPU parity of the one-lane-per-knot-point kernel for serial chains (the
throughput form that large batches of chains of 2 .. 8 revolute bodies take by
default): against the FP64 oracle and against the 8-lane chain kernel, on
ragged batches that span several warps, with M^-1 and qdd written beside J."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import FLOOR32, col_rel_err, col_rel_err_knots, fp32_bar, vec_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


def _inputs(n, N, seed):
    q, qd, tau = (x.astype(np.float32) for x in gi.states(n, N, seed))
    return [torch.from_numpy(x).cuda() for x in (q, qd, tau)], [x.astype(np.float64) for x in (q, qd, tau)]


CHAINS = [(n, s, g) for n in range(2, 9) for s, g in ((1, True), (2, False))]


@pytest.mark.parametrize("n,seed,general", CHAINS, ids=lambda x: str(x))
@pytest.mark.parametrize("N", [1, 77, 1000])
def test_lane_chain_matches_oracle(grid, n, seed, general, N):
    """lanes = 1 forced on random chains (general axes and rotated fixed
    transforms when `general`): J, qdd and M^-1 against the oracle, per knot
    point within the FP32 bar (the larger of 1e-4 and n kappa(M) u)."""
    r = gi.random_tree(n, seed, general=general, max_children=1)
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 31 + N)
    J, qdd = m.grad_fd(q, qd, tau, return_qdd=True)
    J2, Mi = m.grad_fd_minv(q, qd, tau)
    J, qdd, J2, Mi = (x.cpu().numpy() for x in (J, qdd, J2, Mi))
    ref = oracle.grad_fd(r, q64, qd64, tau64)
    mref = oracle.minv(r, q64)
    bar = fp32_bar(mref)
    assert np.all(col_rel_err_knots(J, ref, floor=FLOOR32) <= bar)
    assert vec_rel_err(qdd, oracle.fd(r, q64, qd64, tau64)) <= TOL32
    np.testing.assert_array_equal(J, J2)                        # same kernel, same arithmetic
    assert col_rel_err(Mi, mref, FLOOR32) <= TOL32
    np.testing.assert_array_equal(Mi, np.swapaxes(Mi, 1, 2))    # exactly symmetric
    m.close()


@pytest.mark.parametrize("n", [2, 5, 7, 8])
def test_lane_chain_agrees_with_8_lane_kernel(grid, n):
    """The default dispatch (lanes 0) of a batch above the switch-over size takes
    the one-lane kernel; it agrees with the 8-lane chain kernel on the same
    knot points within the FP32 bar of both against the oracle, checked on
    sampled knot points."""
    r = gi.random_tree(n, 4, general=True, max_children=1)
    one = grid.Model.from_robot(r)
    eight = grid.Model.from_robot(r)
    eight.set_option("lanes", 8)
    N = 32768 + 4093                                   # above the switch-over, ragged last warp
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 5)
    J1 = one.grad_fd(q, qd, tau).cpu().numpy()
    J8 = eight.grad_fd(q, qd, tau).cpu().numpy()
    idx = np.sort(gi.Stream(9).u64(200) % np.uint64(N)).astype(np.int64)
    idx = np.unique(np.concatenate([idx, [0, N - 1]]))
    ref = oracle.grad_fd(r, q64[idx], qd64[idx], tau64[idx])
    bar = fp32_bar(oracle.minv(r, q64[idx]))
    assert np.all(col_rel_err_knots(J1[idx], ref, floor=FLOOR32) <= bar)
    assert np.all(col_rel_err_knots(J8[idx], ref, floor=FLOOR32) <= bar)
    assert np.all(col_rel_err_knots(J1, J8, floor=FLOOR32) <= 2 * fp32_bar(oracle.minv(r, q64[:4096])).max())
    one.close()
    eight.close()


def test_lane_chain_writes_every_entry(grid):
    """Outputs pre-filled with NaN: J, M^-1 and qdd of every knot point of a
    ragged batch are written, and nothing past the batch is touched."""
    r = gi.chain7()
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)
    N = 32 * 5 + 13
    (q, qd, tau), (q64, qd64, tau64) = _inputs(7, N, 3)
    J = torch.full((N + 1, 7, 14), float("nan"), device="cuda")
    Mi = torch.full((N + 1, 7, 7), float("nan"), device="cuda")
    m.grad_fd_minv(q, qd, tau, out=J[:N], minv_out=Mi[:N])
    qdd = torch.full((N + 1, 7), float("nan"), device="cuda")
    m.grad_fd(q, qd, tau, qdd_out=qdd[:N])
    Jh, Mh, qh = J.cpu().numpy(), Mi.cpu().numpy(), qdd.cpu().numpy()
    assert np.isfinite(Jh[:N]).all() and np.isfinite(Mh[:N]).all() and np.isfinite(qh[:N]).all()
    assert np.isnan(Jh[N]).all() and np.isnan(Mh[N]).all() and np.isnan(qh[N]).all()
    assert col_rel_err(Jh[:N], oracle.grad_fd(r, q64, qd64, tau64), FLOOR32) <= TOL32
    assert col_rel_err(Mh[:N], oracle.minv(r, q64), FLOOR32) <= TOL32
    m.close()


def test_lane_chain_workload_chain7_and_repeatable(grid):
    """The 7-DoF workload chain through the default dispatch at the benchmark's
    trajectory length (2048 trajectories x 128 knot points): sampled knot points
    against the oracle, and two calls bit-identical."""
    r = gi.chain7()
    m = grid.Model.from_robot(r)
    N = 2048 * 128
    (q, qd, tau), (q64, qd64, tau64) = _inputs(7, N, gi.workload_seed(2, 128))
    J = m.grad_fd(q, qd, tau)
    J2 = m.grad_fd(q, qd, tau)
    torch.cuda.synchronize()
    assert torch.equal(J, J2)
    idx = np.sort(gi.Stream(11).u64(256) % np.uint64(N)).astype(np.int64)
    ref = oracle.grad_fd(r, q64[idx], qd64[idx], tau64[idx], nthreads=8)
    assert col_rel_err(J[torch.from_numpy(idx).cuda()].cpu().numpy(), ref, FLOOR32) <= TOL32
    m.close()


def test_lane_option_checks(grid):
    """lanes = 1 applies to chains in FP32 only: FP64 and other robots keep
    their kernels, and an unknown lane count is refused."""
    r = gi.tree12()
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)                          # not a chain: the tree's own kernel
    (q, qd, tau), (q64, qd64, tau64) = _inputs(12, 40, 2)
    J = m.grad_fd(q, qd, tau).cpu().numpy()
    assert col_rel_err(J, oracle.grad_fd(r, q64, qd64, tau64), FLOOR32) <= TOL32
    with pytest.raises(grid.GridError):
        m.set_option("lanes", 2)
    m.close()
    c = grid.Model.from_robot(gi.chain7())
    c.set_option("lanes", 1)
    q, qd, tau = (torch.from_numpy(x).cuda() for x in gi.states(7, 50, 4))   # FP64: 8-lane FP64 kernel
    J = c.grad_fd(q, qd, tau).cpu().numpy()
    q64, qd64, tau64 = gi.states(7, 50, 4)
    assert col_rel_err(J, oracle.grad_fd(gi.chain7(), q64, qd64, tau64)) <= 1e-10
    c.close()


def _interleaved_tree30():
    """The 30-DoF tree with its components interleaved in the caller's numbering
    (parents still before children): its leg parts sit at scattered joints."""
    r = gi.tree30()
    arms_torso, leg1, leg2 = list(range(20)), list(range(20, 25)), list(range(25, 30))
    perm = []
    while arms_torso or leg1 or leg2:
        for lst in (arms_torso, leg1, arms_torso, leg2):
            if lst:
                perm.append(lst.pop(0))
    return r.permuted(perm)


PLACED = {"tree12": gi.tree12, "tree30": gi.tree30, "tree30-interleaved": _interleaved_tree30,
          "rand13": lambda: gi.random_tree(13, 21), "rand9": lambda: gi.random_tree(9, 8)}


@pytest.mark.parametrize("key", list(PLACED))
@pytest.mark.parametrize("N", [1, 77])
def test_lane_chain_placed_components(grid, key, N):
    """Chains that are components of a larger robot (the quadruped's legs, the
    humanoid's legs, chain components of random trees) with lanes = 1: each leg
    writes its rows of J and M^-1 (its blocks and exact zeros beside them) and
    its entries of qdd, at its caller joints. Outputs pre-filled with NaN; J, M^-1
    and qdd against the oracle."""
    r = PLACED[key]()
    n = r.n
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 41 + N)
    J = torch.full((N, n, 2 * n), float("nan"), device="cuda")
    Mi = torch.full((N, n, n), float("nan"), device="cuda")
    qdd = torch.full((N, n), float("nan"), device="cuda")
    m.grad_fd_minv(q, qd, tau, out=J, minv_out=Mi)
    J2, _ = m.grad_fd(q, qd, tau, qdd_out=qdd, return_qdd=True)
    Jh, Mh, qh, J2h = (x.cpu().numpy() for x in (J, Mi, qdd, J2))
    assert np.isfinite(Jh).all() and np.isfinite(Mh).all() and np.isfinite(qh).all()
    np.testing.assert_array_equal(Jh, J2h)
    ref, mref = oracle.grad_fd(r, q64, qd64, tau64), oracle.minv(r, q64)
    if key.startswith("rand"):
        bar = fp32_bar(mref)
        assert np.all(col_rel_err_knots(Jh, ref, floor=FLOOR32) <= bar)
    else:
        assert col_rel_err(Jh, ref, FLOOR32) <= TOL32
    assert col_rel_err(Mh, mref, FLOOR32) <= TOL32
    assert vec_rel_err(qh, oracle.fd(r, q64, qd64, tau64)) <= TOL32
    if key == "tree12":                                   # exact zeros between the legs
        for c in range(4):
            jmask = np.ones(24, bool)
            jmask[3 * c:3 * c + 3] = jmask[12 + 3 * c:12 + 3 * c + 3] = False
            mmask = np.ones(12, bool)
            mmask[3 * c:3 * c + 3] = False
            rows = slice(3 * c, 3 * c + 3)
            assert np.all(Jh[:, rows][:, :, jmask] == 0) and np.all(Mh[:, rows][:, :, mmask] == 0)
    m.close()


@pytest.mark.parametrize("key", ["tree12", "tree30", "rand13"])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_lane_chain_placed_outputs_off_16_bytes(grid, key, offset):
    """Placed legs write whole rows of J, M^-1 and the gradient of ID (their blocks
    and the zeros beside them) from blocks staged per warp: outputs that start
    1 .. 3 floats past a 16-byte boundary (NaN-filled around them) give the same
    values as aligned ones, and nothing outside is written."""
    r = PLACED[key]()
    n = r.n
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)
    N = 77
    (q, qd, tau), _ = _inputs(n, N, 71 + offset)

    def view(shape):
        size = int(np.prod(shape))
        buf = torch.full((size + 8,), float("nan"), device="cuda")
        return buf, buf[offset:offset + size].view(shape)

    bj, J = view((N, n, 2 * n))
    bm, Mi = view((N, n, n))
    bd, D = view((N, n, 2 * n))
    bi, M2 = view((N, n, n))
    m.grad_fd_minv(q, qd, tau, out=J, minv_out=Mi)
    m.grad_rnea(q, qd, tau, out=D)
    m.minv(q, out=M2)
    J0, Mi0 = m.grad_fd_minv(q, qd, tau)
    D0, M20 = m.grad_rnea(q, qd, tau), m.minv(q)
    torch.cuda.synchronize()
    for b, x, x0 in ((bj, J, J0), (bm, Mi, Mi0), (bd, D, D0), (bi, M2, M20)):
        assert torch.equal(x, x0)
        hb = b.cpu().numpy()
        assert np.isnan(hb[:offset]).all() and np.isnan(hb[offset + x.numel():]).all()
    m.close()


@pytest.mark.parametrize("key", ["tree12", "tree30"])
def test_lane_chain_placed_default_dispatch(grid, key):
    """Above the switch-over size the quadruped's legs and the humanoid's leg
    parts take the one-lane kernel by default; sampled knot points of a ragged
    batch against the oracle, and the result equal to the forced lanes = 1 run."""
    r = gi.robot(key)
    n = r.n
    m = grid.Model.from_robot(r)
    one = grid.Model.from_robot(r)
    one.set_option("lanes", 1)
    N = 32768 + 7
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 12)
    J = m.grad_fd(q, qd, tau)
    J1 = one.grad_fd(q, qd, tau)
    torch.cuda.synchronize()
    assert torch.equal(J, J1)
    idx = np.unique(np.concatenate([np.sort(gi.Stream(13).u64(128) % np.uint64(N)).astype(np.int64), [0, N - 1]]))
    ref = oracle.grad_fd(r, q64[idx], qd64[idx], tau64[idx], nthreads=8)
    assert col_rel_err(J[torch.from_numpy(idx).cuda()].cpu().numpy(), ref, FLOOR32) <= TOL32
    m.close()
    one.close()


@pytest.mark.parametrize("key", ["chain7", "tree12"])
def test_lane_chain_precision_report(grid, key, capsys):
    """The one-lane kernel (lanes = 1) on the 7-DoF chain and the 12-DoF tree's
    legs at N = 1024 against the FP64 oracle: the per-column metric with the
    tight floor (1e-6) and with the FP32 floor (1e-4), and the ratio of the
    1e-6-floor error to the derived per-column bound (tests/metrics.py:
    derived_col_bar). Printed for the record."""
    from tests.metrics import col_rel_err_cols, derived_col_bar
    r = gi.robot(key)
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)
    N = 1024
    (q, qd, tau), (q64, qd64, tau64) = _inputs(r.n, N, gi.workload_seed(3, N))
    ref_J, ref_qdd = oracle.grad_fd(r, q64, qd64, tau64, nthreads=8, with_qdd=True)
    ref_mi = oracle.minv(r, q64, nthreads=8)
    dq, dqd = oracle.grad_rnea(r, q64, qd64, ref_qdd, nthreads=8)
    J = m.grad_fd(q, qd, tau).cpu().numpy()
    e6 = col_rel_err_cols(J, ref_J, 1e-6)
    e4 = col_rel_err_cols(J, ref_J, FLOOR32)
    bar = derived_col_bar(ref_mi, np.concatenate([dq, dqd], axis=2), ref_J)
    line = (f"{key} one lane per knot point N={N}: max err floor 1e-6 {e6.max():.2e} "
            f"(p50 {np.median(e6.max(axis=1)):.2e}), floor 1e-4 {e4.max():.2e}; "
            f"err / derived bar max {(e6 / bar).max():.2f}")
    with capsys.disabled():
        print("\n" + line)
    assert e4.max() <= TOL32, line
    assert (e6 / bar).max() <= 1.0, line
    m.close()


FDV = [("chain7", None), ("tree12", None), ("rand-chain5", (5, 3)), ("rand-chain8", (8, 6))]


def _fdv_robot(key, spec):
    return gi.robot(key) if spec is None else gi.random_tree(spec[0], spec[1], general=True, max_children=1)


@pytest.mark.parametrize("key,spec", FDV, ids=[k for k, _ in FDV])
@pytest.mark.parametrize("N", [1, 77])
def test_lane_fd_and_vjp_match_oracle(grid, key, spec, N):
    """FD and the vector-Jacobian product through FD with one lane per knot point
    (lanes = 1) on chains and on the 12-DoF tree's legs: qdd against the oracle's
    FD, and (dL/dq, dL/dqd, dL/dtau) for upstream gradients N(0, 1) against the
    oracle's transpose products with the FD Jacobian and M^-1."""
    r = _fdv_robot(key, spec)
    n = r.n
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 51 + N)
    gb = gi.upstream(n, N, 51 + N).astype(np.float32)
    qdd = m.fd(q, qd, tau).cpu().numpy()
    assert vec_rel_err(qdd, oracle.fd(r, q64, qd64, tau64)) <= TOL32
    dq, dqd, dtau = (x.cpu().numpy() for x in m.fd_vjp(q, qd, tau, torch.from_numpy(gb).cuda()))
    rq, rqd, rtau = oracle.fd_vjp(r, q64, qd64, tau64, gb.astype(np.float64))
    tol = TOL32 if spec is None else float(fp32_bar(oracle.minv(r, q64)).max())
    for x, y, name in ((dq, rq, "dq"), (dqd, rqd, "dqd"), (dtau, rtau, "dtau")):
        assert vec_rel_err(x, y) <= tol, name
    m.close()


@pytest.mark.parametrize("key", ["chain7", "tree12"])
def test_lane_fd_and_vjp_default_dispatch(grid, key):
    """Above the switch-over size FD and the VJP of chains and of the 12-DoF tree's
    legs take the one-lane kernel by default: equal to the forced lanes = 1 run, and
    sampled knot points against the oracle."""
    r = gi.robot(key)
    n = r.n
    m = grid.Model.from_robot(r)
    one = grid.Model.from_robot(r)
    one.set_option("lanes", 1)
    N = 32768 + 11
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 23)
    gb = torch.from_numpy(gi.upstream(n, N, 23).astype(np.float32)).cuda()
    a = m.fd(q, qd, tau)
    b = one.fd(q, qd, tau)
    va = m.fd_vjp(q, qd, tau, gb)
    vb = one.fd_vjp(q, qd, tau, gb)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and all(torch.equal(x, y) for x, y in zip(va, vb))
    idx = np.unique(np.concatenate([np.sort(gi.Stream(29).u64(128) % np.uint64(N)).astype(np.int64), [0, N - 1]]))
    ti = torch.from_numpy(idx).cuda()
    assert vec_rel_err(a[ti].cpu().numpy(), oracle.fd(r, q64[idx], qd64[idx], tau64[idx])) <= TOL32
    ref = oracle.fd_vjp(r, q64[idx], qd64[idx], tau64[idx], gb[ti].cpu().numpy().astype(np.float64))
    for x, y in zip(va, ref):
        assert vec_rel_err(x[ti].cpu().numpy(), y) <= TOL32
    m.close()
    one.close()


@pytest.mark.parametrize("key,spec", FDV, ids=[k for k, _ in FDV])
@pytest.mark.parametrize("N", [1, 77])
def test_lane_rnea_minv_grad_id_match_oracle(grid, key, spec, N):
    """RNEA (with accelerations given and with zero), M^-1 and the gradient of ID
    with one lane per knot point (lanes = 1) on chains and on the 12-DoF tree's
    legs, outputs pre-filled with NaN: every entry written, against the oracle,
    M^-1 exactly symmetric."""
    r = _fdv_robot(key, spec)
    n = r.n
    m = grid.Model.from_robot(r)
    m.set_option("lanes", 1)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 61 + N)
    nan = lambda *shape: torch.full(shape, float("nan"), device="cuda")
    t1 = m.rnea(q, qd, tau, out=nan(N, n)).cpu().numpy()              # tau's values as accelerations
    t0 = m.rnea(q, qd, out=nan(N, n)).cpu().numpy()
    Mi = m.minv(q, out=nan(N, n, n)).cpu().numpy()
    D = m.grad_rnea(q, qd, tau, out=nan(N, n, 2 * n)).cpu().numpy()
    for x in (t1, t0, Mi, D):
        assert np.isfinite(x).all()
    assert vec_rel_err(t1, oracle.rnea(r, q64, qd64, tau64)) <= TOL32
    assert vec_rel_err(t0, oracle.rnea(r, q64, qd64, 0 * qd64)) <= TOL32
    mref = oracle.minv(r, q64)
    assert col_rel_err(Mi, mref, FLOOR32) <= (TOL32 if spec is None else float(fp32_bar(mref).max()))
    np.testing.assert_array_equal(Mi, np.swapaxes(Mi, 1, 2))
    rq, rqd = oracle.grad_rnea(r, q64, qd64, tau64)
    assert col_rel_err(D, np.concatenate([rq, rqd], axis=2), FLOOR32) <= TOL32
    if key == "tree12":                                   # exact zeros between the legs
        for c in range(4):
            jm = np.ones(24, bool)
            jm[3 * c:3 * c + 3] = jm[12 + 3 * c:12 + 3 * c + 3] = False
            mm = np.ones(12, bool)
            mm[3 * c:3 * c + 3] = False
            rows = slice(3 * c, 3 * c + 3)
            assert np.all(D[:, rows][:, :, jm] == 0) and np.all(Mi[:, rows][:, :, mm] == 0)
    m.close()


@pytest.mark.parametrize("key", ["chain7", "tree12"])
def test_lane_rnea_minv_grad_id_default_dispatch(grid, key):
    """Above the switch-over size RNEA, M^-1 and the gradient of ID of chains and
    of the 12-DoF tree's legs take the one-lane kernel by default: equal to the
    forced lanes = 1 run, and sampled knot points against the oracle."""
    r = gi.robot(key)
    n = r.n
    m = grid.Model.from_robot(r)
    one = grid.Model.from_robot(r)
    one.set_option("lanes", 1)
    N = 32768 + 5
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 27)
    outs = [(m.rnea(q, qd, tau), one.rnea(q, qd, tau)), (m.minv(q), one.minv(q)),
            (m.grad_rnea(q, qd, tau), one.grad_rnea(q, qd, tau))]
    torch.cuda.synchronize()
    for a, b in outs:
        assert torch.equal(a, b)
    idx = np.unique(np.concatenate([np.sort(gi.Stream(31).u64(96) % np.uint64(N)).astype(np.int64), [0, N - 1]]))
    ti = torch.from_numpy(idx).cuda()
    assert vec_rel_err(outs[0][0][ti].cpu().numpy(), oracle.rnea(r, q64[idx], qd64[idx], tau64[idx])) <= TOL32
    assert col_rel_err(outs[1][0][ti].cpu().numpy(), oracle.minv(r, q64[idx]), FLOOR32) <= TOL32
    rq, rqd = oracle.grad_rnea(r, q64[idx], qd64[idx], tau64[idx])
    assert col_rel_err(outs[2][0][ti].cpu().numpy(), np.concatenate([rq, rqd], axis=2), FLOOR32) <= TOL32
    m.close()
    one.close()
