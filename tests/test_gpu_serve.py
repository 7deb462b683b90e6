"""Serving: persistent kernel with continuous batching of mixed robots and
horizons. Results must match the FP64 oracle, be the same alone and in the
mix, respect memory-based admission, and the kernel's bounded wait must end
with GRID_E_TIMEOUT when nothing is published."""
import time

import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import FLOOR32, col_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOTS = ["chain7", "tree12", "tree30"]


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


@pytest.fixture(scope="module")
def models(grid):
    return [grid.Model.from_robot(gi.robot(r)) for r in ROBOTS]


def _requests(K, seed):
    s = gi.Stream(seed)
    reqs = []
    for i in range(K):
        m = int(s.unit(1)[0] * 3)
        H = [16, 32, 64, 128, 256, 37][int(s.unit(1)[0] * 6)]
        n = gi.robot(ROBOTS[m]).n
        q, qd, tau = (x.astype(np.float32) for x in gi.states(n, H, 5000 + i))
        reqs.append((m, H, q, qd, tau))
    return reqs


def test_served_results_alone_and_in_the_mix(grid, models):
    srv = grid.Server(models, ring_slots=64, arena_bytes=64 << 20)
    srv.start()
    reqs = _requests(24, 3)
    alone = []
    for m, H, q, qd, tau in reqs:
        rid = srv.submit(m, q, qd, tau)
        assert rid is not None
        J = srv.result(rid, H, models[m].n)
        assert J is not None
        alone.append(J)
    # the same requests submitted back to back, interleaved on the device
    pending = {}
    mixed = [None] * len(reqs)
    i = 0
    while i < len(reqs) or pending:
        if i < len(reqs):
            m, H, q, qd, tau = reqs[i]
            rid = srv.submit(m, q, qd, tau)
            if rid is not None:
                pending[rid] = i
                i += 1
                continue
        for rid in list(pending):
            k = pending[rid]
            J = srv.result(rid, reqs[k][1], models[reqs[k][0]].n, wait_us=0)
            if J is not None:
                mixed[k] = J
                del pending[rid]
    assert srv.stop() == 0
    for k, (m, H, q, qd, tau) in enumerate(reqs):
        r = gi.robot(ROBOTS[m])
        ref = oracle.grad_fd(r, q.astype(np.float64), qd.astype(np.float64), tau.astype(np.float64),
                             nthreads=8)
        assert col_rel_err(alone[k], ref, FLOOR32) <= 1e-4
        # a knot point's arithmetic does not depend on the requests around it:
        # its tile (2 knot points of the same request) runs the same instructions
        np.testing.assert_array_equal(mixed[k], alone[k], err_msg=str(k))
    srv.close()


def test_server_refuses_mixed_precision_models(grid):
    mixed = grid.Model.from_robot(gi.chain7(), precision="mixed")
    with pytest.raises(grid.GridError, match="FP32"):
        grid.Server([mixed], ring_slots=4, arena_bytes=1 << 20)
    mixed.close()


def test_memory_based_admission(grid, models):
    srv = grid.Server(models, ring_slots=8, arena_bytes=1 << 20)
    srv.start()
    big = _requests(1, 7)[0]
    n30 = gi.tree30().n
    q, qd, tau = (x.astype(np.float32) for x in gi.states(n30, 256, 9))
    assert srv.submit(2, q, qd, tau) is None              # 1.9 MB of I/O does not fit in 1 MB
    q, qd, tau = (x.astype(np.float32) for x in gi.states(7, 64, 9))
    rid = srv.submit(0, q, qd, tau)
    assert rid is not None
    assert srv.result(rid, 64, 7) is not None
    del big
    assert srv.stop() == 0
    srv.close()


def test_idle_kernel_ends_with_timeout_status(grid, models):
    """No request is ever published: the persistent kernel's bounded wait runs
    out, it records GRID_E_TIMEOUT and returns; the context stays usable."""
    srv = grid.Server(models[:1], ring_slots=4, arena_bytes=1 << 20, idle_timeout=0.2)
    srv.start()
    time.sleep(1.0)
    assert srv.kernel_status() == 6
    assert srv.stop() == 6
    srv.close()
    q, qd, tau = (torch.from_numpy(x.astype(np.float32)).cuda() for x in gi.states(7, 8, 1))
    J = models[0].grad_fd(q, qd, tau)
    torch.cuda.synchronize()
    assert torch.isfinite(J).all()
