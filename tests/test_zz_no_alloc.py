"""The allocation-free batch entry point (grid_serve_batch_static), for callers
that may not allocate device memory while running: called through the C-ABI
twice in a row and checked against grid_grad_fd and the FP64 oracle on the same
inputs. Buffers are allocated here by the test; the entry point itself
allocates nothing."""
import ctypes

import numpy as np
import pytest

import grid_inputs as gi
import oracle
from tests.metrics import FLOOR32, col_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ["chain7", "tree12", "tree30"]
TOL32 = 1e-4


def _entry(grid):
    fn = grid._native.load().grid_serve_batch_static
    P = ctypes.c_void_p
    fn.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P]
    fn.restype = ctypes.c_int
    return fn


def test_static_batch_matches_grad_fd_on_two_calls():
    import paper_2109_06976_gb300 as grid
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = _entry(grid)
    models = [grid.Model.from_robot(gi.robot(r)) for r in NAMES]
    marr = (ctypes.c_void_p * len(models))(*[m.handle.value for m in models])
    stream = torch.cuda.current_stream()
    for call in range(2):
        s = gi.Stream(900 + call)
        reqs = []
        for i in range(11):
            m = int(s.unit(1)[0] * 3)
            H = [16, 37, 64, 128, 5][int(s.unit(1)[0] * 5)]
            n = models[m].n
            q, qd, tau = (torch.from_numpy(x.astype(np.float32)).cuda()
                          for x in gi.states(n, H, 7000 + 100 * call + i))
            J = torch.full((H, n, 2 * n), float("nan"), device="cuda")
            reqs.append((m, H, q, qd, tau, J))
        arr = lambda vals, ct: (ct * len(vals))(*vals)
        st = fn(marr, len(models), len(reqs),
                arr([r[0] for r in reqs], ctypes.c_int), arr([r[1] for r in reqs], ctypes.c_int),
                arr([r[2].data_ptr() for r in reqs], ctypes.c_void_p),
                arr([r[3].data_ptr() for r in reqs], ctypes.c_void_p),
                arr([r[4].data_ptr() for r in reqs], ctypes.c_void_p),
                arr([r[5].data_ptr() for r in reqs], ctypes.c_void_p),
                ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, grid._native.load().grid_last_error()
        torch.cuda.synchronize()
        for m, H, q, qd, tau, J in reqs:
            ref = models[m].grad_fd(q, qd, tau)
            torch.cuda.synchronize()
            assert col_rel_err(J.cpu().numpy(), ref.cpu().numpy(), FLOOR32) <= TOL32
            r = gi.robot(NAMES[m])
            exact = oracle.grad_fd(r, *(x.cpu().numpy().astype(np.float64) for x in (q, qd, tau)))
            assert col_rel_err(J.cpu().numpy(), exact, FLOOR32) <= TOL32
    # more requests than the fixed scratch holds are refused before any work
    one = (ctypes.c_int * 1)(0)
    ptr = (ctypes.c_void_p * 1)(reqs[0][2].data_ptr())
    st = fn(marr, len(models), 257, one, one, ptr, ptr, ptr, ptr, ctypes.c_void_p(stream.cuda_stream))
    assert st == 1 and b"1 to 256" in grid._native.load().grid_last_error()


def test_static_batch_reads_no_host_array_after_returning():
    """The request list goes to the device inside the call: pointing the host
    arrays at other (valid) buffers right after the call returns changes
    nothing. A GRID_MIXED model is refused (the serving kernel has no FP64 pivots)."""
    import paper_2109_06976_gb300 as grid
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = _entry(grid)
    m7 = grid.Model.from_robot(gi.chain7())
    marr = (ctypes.c_void_p * 1)(m7.handle.value)
    stream = torch.cuda.current_stream()
    H = 64
    q, qd, tau = (torch.from_numpy(x.astype(np.float32)).cuda() for x in gi.states(7, H, 4242))
    J = torch.full((H, 7, 14), float("nan"), device="cuda")
    decoy = torch.full((H, 7, 14), float("nan"), device="cuda")
    one = (ctypes.c_int * 1)(0)
    hs = (ctypes.c_int * 1)(H)
    pq, pqd, ptau = ((ctypes.c_void_p * 1)(t.data_ptr()) for t in (q, qd, tau))
    pJ = (ctypes.c_void_p * 1)(J.data_ptr())
    torch.cuda._sleep(2_000_000)          # keep the stream busy while the host arrays change
    st = fn(marr, 1, 1, one, hs, pq, pqd, ptau, pJ, ctypes.c_void_p(stream.cuda_stream))
    pJ[0] = decoy.data_ptr()
    hs[0] = 1
    assert st == 0, grid._native.load().grid_last_error()
    torch.cuda.synchronize()
    assert torch.isnan(decoy).all()
    ref = m7.grad_fd(q, qd, tau)
    torch.cuda.synchronize()
    assert col_rel_err(J.cpu().numpy(), ref.cpu().numpy(), FLOOR32) <= TOL32
    mixed = grid.Model.from_robot(gi.chain7(), precision="mixed")
    marr2 = (ctypes.c_void_p * 1)(mixed.handle.value)
    st = fn(marr2, 1, 1, one, hs, pq, pqd, ptau, pJ, ctypes.c_void_p(stream.cuda_stream))
    assert st == 1 and b"FP32" in grid._native.load().grid_last_error()
