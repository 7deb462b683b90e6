"""Run-time specialisation (grid_set_option "specialize" = 2): the gradient
kernel compiled by NVRTC for a robot's own topology, against the oracle and
against the run-time-topology kernel, FP32 and FP64, on trees without a
precompiled shape and at both lane mappings."""
import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import FLOOR32, FLOOR64, col_rel_err_knots, fp32_bar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


@pytest.mark.parametrize("key", ["tree30", (9, 8), (13, 21)], ids=str)
@pytest.mark.parametrize("N", [29, 700])
def test_runtime_specialised_kernel(grid, key, N):
    r = gi.robot(key) if isinstance(key, str) else gi.random_tree(*key)
    spec = grid.Model.from_robot(r)
    spec.set_option("specialize", 2)
    gen = grid.Model.from_robot(r)
    gen.set_option("specialize", 0)
    for dt, tol in ((torch.float32, 1e-4), (torch.float64, 1e-10)):
        npdt = np.float32 if dt == torch.float32 else np.float64
        q, qd, tau = (x.astype(npdt) for x in gi.states(r.n, N, 31))
        d = [torch.from_numpy(x).cuda() for x in (q, qd, tau)]
        Js, qdds = spec.grad_fd(*d, return_qdd=True)
        Jg = gen.grad_fd(*d)
        ref, qddo = oracle.grad_fd(r, *(x.astype(np.float64) for x in (q, qd, tau)), nthreads=8, with_qdd=True)
        f = FLOOR32 if dt == torch.float32 else FLOOR64
        bar = tol
        if dt == torch.float32 and not isinstance(key, str):   # random inertias: per-knot n kappa(M) u
            bar = fp32_bar(oracle.minv(r, q.astype(np.float64), nthreads=8), tol)
        assert np.all(col_rel_err_knots(Js.cpu().numpy(), ref, floor=f) <= bar)
        assert np.all(col_rel_err_knots(Jg.cpu().numpy(), ref, floor=f) <= bar)
        assert np.abs(qdds.cpu().numpy() - qddo).max() <= tol * max(1.0, np.abs(qddo).max()) * 10
