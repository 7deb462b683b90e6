"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the
same seeded inputs. FP32 bar: 1e-4 per-column relative error (tests/metrics.py)
on the workload robots; FP64: 1e-10 on every robot."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import (FLOOR32, FLOOR64, col_rel_err, col_rel_err_cols, col_rel_err_knots, col_rel_err_stats,
                           derived_col_bar, fp32_bar, vec_rel_err)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOAD = ["chain7", "tree12", "tree30"]
RANDOM = [(3, 2), (6, 4), (9, 8), (13, 21), (1, 5), (20, 3), (32, 7)]
TOL32 = 1e-4
TOL64 = 1e-10


def _robot(key):
    if isinstance(key, str):
        return gi.robot(key)
    return gi.random_tree(*key)


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


_models = {}


def _model(grid, key, precision="fp32"):
    k = (str(key), precision)
    if k not in _models:
        _models[k] = grid.Model.from_robot(_robot(key), precision=precision)
    return _models[k]


def _inputs(n, N, seed, dtype):
    q, qd, tau = gi.states(n, N, seed)
    npdt = np.float32 if dtype == torch.float32 else np.float64
    q, qd, tau = (x.astype(npdt) for x in (q, qd, tau))
    dev = [torch.from_numpy(x).cuda() for x in (q, qd, tau)]
    host64 = [x.astype(np.float64) for x in (q, qd, tau)]
    return dev, host64


def _floor(key, dtype):
    return FLOOR64 if dtype == torch.float64 else FLOOR32


CASES = [(k, dt) for k in WORKLOAD for dt in (torch.float32, torch.float64)] + \
        [(k, torch.float64) for k in RANDOM] + [(k, torch.float32) for k in RANDOM]


@pytest.mark.parametrize("key,dtype", CASES, ids=lambda x: str(x))
@pytest.mark.parametrize("N", [1, 37])
def test_all_outputs_match_oracle(grid, key, dtype, N):
    r = _robot(key)
    m = _model(grid, key)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(r.n, N, 1000 + N, dtype)
    tol = TOL32 if dtype == torch.float32 else TOL64
    fl = _floor(key, dtype)
    # RNEA with qdd = tau values as accelerations, and with qdd = 0 (NULL)
    e = vec_rel_err(m.rnea(q, qd, tau).cpu().numpy(), oracle.rnea(r, q64, qd64, tau64), fl)
    assert e <= tol, f"rnea {e}"
    e = vec_rel_err(m.rnea(q, qd).cpu().numpy(), oracle.rnea(r, q64, qd64, 0 * qd64), fl)
    assert e <= tol, f"rnea(qdd=0) {e}"
    Mi = m.minv(q).cpu().numpy()
    e = col_rel_err(Mi, oracle.minv(r, q64), fl)
    assert e <= tol, f"minv {e}"
    np.testing.assert_array_equal(Mi, np.swapaxes(Mi, 1, 2))      # exactly symmetric output
    qdd_ref = oracle.fd(r, q64, qd64, tau64)
    e = vec_rel_err(m.fd(q, qd, tau).cpu().numpy(), qdd_ref, fl)
    assert e <= tol, f"fd {e}"
    dID = m.grad_rnea(q, qd, tau).cpu().numpy()             # tau values used as accelerations
    rq, rqd = oracle.grad_rnea(r, q64, qd64, tau64)
    e = col_rel_err(dID, np.concatenate([rq, rqd], axis=2), fl)
    assert e <= tol, f"grad_rnea {e}"
    J, qdd = m.grad_fd(q, qd, tau, return_qdd=True)
    e = col_rel_err(J.cpu().numpy(), oracle.grad_fd(r, q64, qd64, tau64), fl)
    assert e <= tol, f"grad_fd {e}"
    e = vec_rel_err(qdd.cpu().numpy(), qdd_ref, fl)
    assert e <= tol, f"grad_fd qdd {e}"


@pytest.mark.parametrize("key", WORKLOAD)
@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_lane_counts_agree(grid, key, lanes):
    """Every cooperative mapping gives the oracle's result (ragged N spanning
    several tiles)."""
    r = _robot(key)
    m = grid.Model.from_robot(r)
    m.set_option("lanes", lanes)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(r.n, 29, 7, torch.float64)
    try:
        J = m.grad_fd(q, qd, tau).cpu().numpy()
    except grid.GridError as e:
        # a mapping whose per-warp workspace exceeds shared memory is refused
        assert e.status == 1 and "shared memory" in str(e), e
    else:
        assert col_rel_err(J, oracle.grad_fd(r, q64, qd64, tau64)) <= TOL64
    (q, qd, tau), (q64, qd64, tau64) = _inputs(r.n, 29, 7, torch.float32)
    J = m.grad_fd(q, qd, tau).cpu().numpy()
    assert col_rel_err(J, oracle.grad_fd(r, q64, qd64, tau64)) <= TOL32


CHAINS = [(n, s, g) for n in range(2, 10) for s, g in ((1, True), (2, False))]


@pytest.mark.parametrize("n,seed,general", CHAINS, ids=lambda x: str(x))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_chain_specialised_kernel(grid, n, seed, general, dtype):
    """Serial chains (parent[i] = i - 1): the kernel compiled for the chain's
    length against the oracle and against the run-time-topology kernel, on a
    ragged batch; n = 9 has no specialised kernel and takes the general one."""
    r = gi.random_tree(n, seed, general=general, max_children=1)
    assert all(int(r.parent[i]) == i - 1 for i in range(n))
    spec = grid.Model.from_robot(r)
    gen = grid.Model.from_robot(r)
    gen.set_option("specialize", 0)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, 77, 11, dtype)
    Js, qdds = spec.grad_fd(q, qd, tau, return_qdd=True)
    Jg, qddg = gen.grad_fd(q, qd, tau, return_qdd=True)
    Js, qdds, Jg, qddg = (x.cpu().numpy() for x in (Js, qdds, Jg, qddg))
    ref = oracle.grad_fd(r, q64, qd64, tau64)
    tol, fl = (TOL32, 1e-4) if dtype == torch.float32 else (TOL64, 1e-6)
    # FP32: random inertias, so the per-knot bound n kappa(M) u where it exceeds 1e-4
    bar = fp32_bar(oracle.minv(r, q64)) if dtype == torch.float32 else tol
    assert np.all(col_rel_err_knots(Js, ref, floor=fl) <= bar)
    assert vec_rel_err(qdds, oracle.fd(r, q64, qd64, tau64)) <= tol
    # both kernels meet the bar; they differ only in rounding order
    assert np.all(col_rel_err_knots(Jg, ref, floor=fl) <= bar)
    assert np.all(col_rel_err_knots(Js, Jg, floor=fl) <= 2 * bar)
    assert vec_rel_err(qdds, qddg) <= tol


def _forest(K, L, seed):
    import dataclasses
    base = gi.random_tree(K * L, seed, general=True, max_children=1)
    par = np.array([-1 if i % L == 0 else i - 1 for i in range(K * L)], dtype=np.int32)
    return dataclasses.replace(base, name=f"forest{K}x{L}", parent=par)


@pytest.mark.parametrize("shape", [None, (4, 3), (2, 6), (4, 4), (3, 2)], ids=lambda x: str(x))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("N", [37, 400])
def test_forest_specialised_kernel(grid, shape, dtype, N):
    """K equal chains on the base (the 12-DoF tree is 4 x 3): the kernel compiled
    for the forest's shape (32 lanes per knot point for the small batch, 8 for
    the large one) against the oracle and the run-time-topology kernel ((3, 2)
    has no compiled shape and takes the general kernel)."""
    r = gi.tree12() if shape is None else _forest(*shape, 3)
    n = r.n
    spec = grid.Model.from_robot(r)
    gen = grid.Model.from_robot(r)
    gen.set_option("specialize", 0)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(n, N, 13, dtype)
    Js = spec.grad_fd(q, qd, tau).cpu().numpy()
    Jg = gen.grad_fd(q, qd, tau).cpu().numpy()
    ref = oracle.grad_fd(r, q64, qd64, tau64)
    fl = FLOOR32 if dtype == torch.float32 else FLOOR64
    tol = TOL32 if dtype == torch.float32 else TOL64
    if shape is not None and dtype == torch.float32:   # random inertias: per-knot bar
        tol = fp32_bar(oracle.minv(r, q64))
    assert np.all(col_rel_err_knots(Js, ref, floor=fl) <= tol)
    assert np.all(col_rel_err_knots(Jg, ref, floor=fl) <= tol)


@pytest.mark.parametrize("N", [1, 203])
def test_forest_branches_write_whole_outputs(grid, N):
    """A forest on the fixed base runs as independent chains (one lane group per
    chain and knot point): J and M^-1 get every entry written, the chains'
    diagonal blocks and exact zeros elsewhere (outputs pre-filled with NaN)."""
    r = gi.tree12()
    m = grid.Model.from_robot(r)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(12, N, 17, torch.float32)
    J = torch.full((N, 12, 24), float("nan"), device="cuda")
    Mi = torch.full((N, 12, 12), float("nan"), device="cuda")
    m.grad_fd_minv(q, qd, tau, out=J, minv_out=Mi)
    Jh, Mh = J.cpu().numpy(), Mi.cpu().numpy()
    assert np.isfinite(Jh).all() and np.isfinite(Mh).all()
    for c in range(4):
        rows = slice(3 * c, 3 * c + 3)
        jmask = np.ones(24, bool)
        jmask[3 * c:3 * c + 3] = jmask[12 + 3 * c:12 + 3 * c + 3] = False
        mmask = np.ones(12, bool)
        mmask[3 * c:3 * c + 3] = False
        assert np.all(Jh[:, rows][:, :, jmask] == 0) and np.all(Mh[:, rows][:, :, mmask] == 0)
    assert col_rel_err(Jh, oracle.grad_fd(r, q64, qd64, tau64), FLOOR32) <= TOL32
    assert col_rel_err(Mh, oracle.minv(r, q64), FLOOR32) <= TOL32
    m.close()


@pytest.mark.parametrize("key", WORKLOAD)
def test_grad_fd_workload_sizes(grid, key):
    """The workload batch sizes (N = 16 .. 1024) in one call each."""
    r = _robot(key)
    m = _model(grid, key)
    for N in (16, 128, 512) if key != "tree30" else (128, 1024):
        (q, qd, tau), (q64, qd64, tau64) = _inputs(r.n, N, gi.workload_seed(2, N), torch.float32)
        J = m.grad_fd(q, qd, tau).cpu().numpy()
        mx, p50 = col_rel_err_stats(J, oracle.grad_fd(r, q64, qd64, tau64, nthreads=8), FLOOR32)
        assert mx <= TOL32, (N, mx, p50)


def test_grad_fd_bench_size_sampled(grid):
    """The benchmark's launch (7-DoF chain, 4096 trajectories x 128 knot points
    in one call) checked on 256 sampled knot points."""
    r = gi.chain7()
    m = _model(grid, "chain7")
    N = 4096 * 128
    (q, qd, tau), (q64, qd64, tau64) = _inputs(7, N, gi.workload_seed(2, 128), torch.float32)
    J = m.grad_fd(q, qd, tau)
    torch.cuda.synchronize()
    idx = np.sort(gi.Stream(5).u64(256) % np.uint64(N)).astype(np.int64)
    Js = J[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.grad_fd(r, q64[idx], qd64[idx], tau64[idx], nthreads=8)
    assert col_rel_err(Js, ref, FLOOR32) <= TOL32
    assert torch.isfinite(J).all()


def test_mixed_precision_tree30(grid):
    """FP64 pivots in the M^-1 recursion: parity holds and the error is
    reported next to the all-FP32 form."""
    r = gi.tree30()
    m32 = _model(grid, "tree30")
    mm = _model(grid, "tree30", "mixed")
    (q, qd, tau), (q64, qd64, tau64) = _inputs(30, 128, gi.workload_seed(3, 128), torch.float32)
    ref = oracle.grad_fd(r, q64, qd64, tau64, nthreads=8)
    e32 = col_rel_err(m32.grad_fd(q, qd, tau).cpu().numpy(), ref, FLOOR32)
    emx = col_rel_err(mm.grad_fd(q, qd, tau).cpu().numpy(), ref, FLOOR32)
    assert e32 <= TOL32 and emx <= TOL32, (e32, emx)


def test_empty_batch_and_errors(grid):
    r = gi.chain7()
    m = _model(grid, "chain7")
    z = torch.empty((0, 7), device="cuda")
    assert m.grad_fd(z, z, z).shape == (0, 7, 14)
    q = torch.zeros((4, 7), device="cuda")
    with pytest.raises(grid.GridError):
        grid._native.call("grid_fd", m.handle, 4, None, None, None, None, None)
    buf = torch.zeros(64, device="cuda")
    import ctypes
    mis = ctypes.c_void_p(buf.data_ptr() + 2)
    with pytest.raises(grid.GridError) as ei:
        grid._native.call("grid_fd", m.handle, 1, mis, mis, mis, mis, None)
    assert ei.value.status == 3
    with pytest.raises(grid.GridError):
        grid.Model([-1, 1], np.eye(3)[:2], r.xtree[:2], r.inertia[:2])
    bad_axis = r.axis.copy()
    bad_axis[0] *= 2
    with pytest.raises(grid.GridError):
        grid.Model(r.parent, bad_axis, r.xtree, r.inertia)
    del q


def test_permuted_numbering(grid):
    """A robot given in non-depth-first order (legs interleaved) is renumbered
    internally; results come back in the caller's order."""
    r = gi.tree12()
    perm = np.array([0, 3, 6, 9, 1, 4, 7, 10, 2, 5, 8, 11])   # breadth-first order
    rp = r.permuted(perm)
    m = grid.Model.from_robot(rp)
    (q, qd, tau), (q64, qd64, tau64) = _inputs(12, 9, 11, torch.float64)
    J = m.grad_fd(q, qd, tau).cpu().numpy()
    assert col_rel_err(J, oracle.grad_fd(rp, q64, qd64, tau64)) <= TOL64
    Mi = m.minv(q).cpu().numpy()
    assert col_rel_err(Mi, oracle.minv(rp, q64)) <= TOL64


def test_repeatable(grid):
    r = gi.tree12()
    m = _model(grid, "tree12")
    (q, qd, tau), _ = _inputs(12, 300, 3, torch.float32)
    a = m.grad_fd(q, qd, tau)
    b = m.grad_fd(q, qd, tau)
    assert torch.equal(a, b)


def test_precision_report_tree30(grid, capsys):
    """Per-output error of the FP32 and mixed (FP64 pivots) forms against the
    FP64 oracle on the 30-DoF tree at N = 128 and 1024 (max and median over
    knot points of the per-knot worst column). Printed for the record."""
    r = gi.tree30()
    lines = []
    for prec in ("fp32", "mixed"):
        m = _model(grid, "tree30", prec)
        for N in (128, 1024):
            (q, qd, tau), (q64, qd64, tau64) = _inputs(30, N, gi.workload_seed(3, N), torch.float32)
            ref_tau = oracle.rnea(r, q64, qd64, tau64, nthreads=8)
            ref_mi = oracle.minv(r, q64, nthreads=8)
            ref_J, ref_qdd = oracle.grad_fd(r, q64, qd64, tau64, nthreads=8, with_qdd=True)
            J, qdd = m.grad_fd(q, qd, tau, return_qdd=True)
            outs = {
                "rnea": (m.rnea(q, qd, tau).cpu().numpy()[:, :, None], ref_tau[:, :, None]),
                "minv": (m.minv(q).cpu().numpy(), ref_mi),
                "fd": (m.fd(q, qd, tau).cpu().numpy()[:, :, None], ref_qdd[:, :, None]),
                "grad_fd": (J.cpu().numpy(), ref_J),
            }
            for name, (x, y) in outs.items():
                mx, p50 = col_rel_err_stats(x, y, FLOOR32)
                lines.append(f"tree30 {prec:5s} N={N:4d} {name:8s} max {mx:.2e} p50 {p50:.2e}")
                assert mx <= TOL32, lines[-1]
    with capsys.disabled():
        print("\n" + "\n".join(lines))


def test_zero_copy_host_buffers(grid):
    """Pinned host buffers passed straight to the kernels (read and written over
    the CPU-GPU link) give the same results as device buffers."""
    r = gi.chain7()
    m = _model(grid, "chain7")
    (q, qd, tau), _ = _inputs(7, 301, 19, torch.float32)
    J_dev, qdd_dev = m.grad_fd(q, qd, tau, return_qdd=True)
    hq, hqd, htau = (t.cpu().pin_memory() for t in (q, qd, tau))
    J_host, qdd_host = m.grad_fd(hq, hqd, htau, return_qdd=True)
    torch.cuda.synchronize()
    assert not J_host.is_cuda and J_host.is_pinned()
    assert torch.equal(J_host, J_dev.cpu()) and torch.equal(qdd_host, qdd_dev.cpu())
    gb = torch.from_numpy(gi.upstream(7, 301, 19).astype(np.float32))
    dv = m.fd_vjp(q, qd, tau, gb.cuda())
    hv = m.fd_vjp(hq, hqd, htau, gb.pin_memory())
    torch.cuda.synchronize()
    for a, b in zip(dv, hv):
        assert torch.equal(a.cpu(), b)


@pytest.mark.parametrize("key,prec", [("chain7", "fp32"), ("tree12", "fp32"), ("tree30", "fp32"),
                                      ("tree30", "mixed")])
def test_precision_report_workload(grid, key, prec, capsys):
    """FP32 gradient of FD of each workload robot at N = 1024 against the FP64
    oracle, measured three ways: the per-column metric with the tight floor
    (1e-6) and with the FP32 floor (1e-4), and the ratio of the 1e-6-floor error
    to the derived per-column bound max(1e-4, n kappa_2(M) u alpha_j)
    (tests/metrics.py: derived_col_bar). Printed for the record."""
    r = _robot(key)
    m = _model(grid, key, prec)
    N = 1024
    (q, qd, tau), (q64, qd64, tau64) = _inputs(r.n, N, gi.workload_seed(3, N), torch.float32)
    ref_J, ref_qdd = oracle.grad_fd(r, q64, qd64, tau64, nthreads=8, with_qdd=True)
    ref_mi = oracle.minv(r, q64, nthreads=8)
    dq, dqd = oracle.grad_rnea(r, q64, qd64, ref_qdd, nthreads=8)
    J = m.grad_fd(q, qd, tau).cpu().numpy()
    e6 = col_rel_err_cols(J, ref_J, 1e-6)
    e4 = col_rel_err_cols(J, ref_J, FLOOR32)
    bar = derived_col_bar(ref_mi, np.concatenate([dq, dqd], axis=2), ref_J)
    nku = r.n * np.linalg.cond(ref_mi) * 2.0 ** -24
    line = (f"{key} {prec:5s} N={N}: max err floor 1e-6 {e6.max():.2e} (p50 {np.median(e6.max(axis=1)):.2e}), "
            f"floor 1e-4 {e4.max():.2e}; n kappa u max {nku.max():.2e}; "
            f"err / derived bar max {(e6 / bar).max():.2f}; columns above 1e-4 (floor 1e-6): "
            f"{int((e6 > 1e-4).sum())} of {e6.size}")
    with capsys.disabled():
        print("\n" + line)
    assert e4.max() <= TOL32, line
    # with the tight 1e-6 floor, every column meets the derived per-column bound
    assert (e6 / bar).max() <= 1.0, line
