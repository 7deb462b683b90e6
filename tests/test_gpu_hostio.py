"""grid_grad_fd_host: the gradient of FD on host buffers, pipelined through
device staging in chunks (copy in, kernel, copy out overlapped on three
streams). Checked against the device-buffer call on the same knot points (bit
for bit where the kernel configuration does not depend on the chunk's size)
and against the oracle, over ragged batches that reuse every staging slot
several times, with pinned and pageable buffers, both precisions, a growing
chunk size, a side stream and two threads sharing one model."""
import threading

import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import FLOOR32, col_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grid():
    import paper_2109_06976_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


def _host(robot, N, seed, dtype, pinned=True):
    npdt = np.float32 if dtype == torch.float32 else np.float64
    ts = [torch.from_numpy(x.astype(npdt)) for x in gi.states(robot.n, N, seed)]
    return [t.pin_memory() for t in ts] if pinned else ts


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_chain_matches_device_call_bit_for_bit(grid, dtype, pinned):
    r = gi.chain7()
    m = grid.Model.from_robot(r)
    m.set_option("host_chunk", 1000)            # 11 chunks: each staging slot reused 3 or 4 times
    N = 10007
    q, qd, tau = _host(r, N, 41, dtype, pinned)
    J, qdd = m.grad_fd_host(q, qd, tau, return_qdd=True)
    Jd, qddd = m.grad_fd(q.cuda(), qd.cuda(), tau.cuda(), return_qdd=True)
    np.testing.assert_array_equal(J.numpy(), Jd.cpu().numpy())
    np.testing.assert_array_equal(qdd.numpy(), qddd.cpu().numpy())
    idx = np.array([0, 999, 1000, 5003, N - 1])
    x = [t.numpy()[idx].astype(np.float64) for t in (q, qd, tau)]
    tol, fl = (1e-4, FLOOR32) if dtype == torch.float32 else (1e-10, 1e-6)
    assert col_rel_err(J.numpy()[idx], oracle.grad_fd(r, *x), fl) <= tol
    m.close()


def test_tree_and_default_chunk(grid):
    """The 12-DoF tree: the last chunk (7 knot points) runs at another lane
    count than the others, so it is checked against the oracle; with the
    default chunk size the whole batch is one chunk."""
    r = gi.tree12()
    m = grid.Model.from_robot(r)
    N = 5007
    q, qd, tau = _host(r, N, 43, torch.float32)
    ref = oracle.grad_fd(r, *(t.numpy().astype(np.float64) for t in (q, qd, tau)), nthreads=8)
    m.set_option("host_chunk", 500)
    J = m.grad_fd_host(q, qd, tau)
    assert col_rel_err(J.numpy(), ref, FLOOR32) <= 1e-4
    m.set_option("host_chunk", 0)
    J0 = m.grad_fd_host(q, qd, tau)
    np.testing.assert_array_equal(J0.numpy(), m.grad_fd(q.cuda(), qd.cuda(), tau.cuda()).cpu().numpy())
    m.close()


def test_staging_grows_and_small_batches(grid):
    r = gi.chain7()
    m = grid.Model.from_robot(r)
    q, qd, tau = _host(r, 3000, 47, torch.float32)
    want = m.grad_fd(q.cuda(), qd.cuda(), tau.cuda()).cpu().numpy()
    for chunk in (64, 700, 3000, 128):            # slots replaced when a call needs larger chunks
        m.set_option("host_chunk", chunk)
        np.testing.assert_array_equal(m.grad_fd_host(q, qd, tau).numpy(), want)
    one = m.grad_fd_host(q[:1], qd[:1], tau[:1])
    np.testing.assert_array_equal(one.numpy(), want[:1])
    empty = m.grad_fd_host(q[:0], qd[:0], tau[:0])
    assert empty.shape == (0, 7, 14)
    with pytest.raises(TypeError):
        m.grad_fd_host(q.cuda(), qd.cuda(), tau.cuda())
    m.close()


def test_side_stream_without_host_sync(grid):
    r = gi.chain7()
    m = grid.Model.from_robot(r)
    m.set_option("host_chunk", 512)
    q, qd, tau = _host(r, 4099, 53, torch.float32)
    want = m.grad_fd(q.cuda(), qd.cuda(), tau.cuda()).cpu().numpy()
    J = torch.full((4099, 7, 14), float("nan")).pin_memory()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(2_000_000)              # earlier work on the stream: the pipeline waits for it
        m.grad_fd_host(q, qd, tau, out=J, sync=False)
    s.synchronize()
    np.testing.assert_array_equal(J.numpy(), want)
    m.close()


def test_two_threads_share_a_model(grid):
    r = gi.chain7()
    m = grid.Model.from_robot(r)
    m.set_option("host_chunk", 777)
    batches = [_host(r, 3001 + 13 * i, 60 + i, torch.float32) for i in range(2)]
    wants = [m.grad_fd(*(t.cuda() for t in b)).cpu().numpy() for b in batches]
    got = [None, None]
    errors = []

    def work(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(3):
                    got[i] = m.grad_fd_host(*batches[i]).numpy().copy()
        except Exception as e:                    # surfaced in the main thread
            errors.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for i in range(2):
        np.testing.assert_array_equal(got[i], wants[i])
    m.close()
