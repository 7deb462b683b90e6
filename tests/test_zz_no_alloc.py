"""The allocation-free batch entry point (grid_serve_batch_static), for callers
that may not allocate device memory while running: called through the C-ABI
twice in a row and checked against grid_grad_fd on the same inputs. Buffers
are allocated here by the test; the entry point itself allocates nothing."""
import ctypes

import numpy as np
import pytest

import grid_inputs as gi
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
    # more requests than the fixed scratch holds are refused before any work
    one = (ctypes.c_int * 1)(0)
    ptr = (ctypes.c_void_p * 1)(reqs[0][2].data_ptr())
    st = fn(marr, len(models), 257, one, one, ptr, ptr, ptr, ptr, ctypes.c_void_p(stream.cuda_stream))
    assert st == 1 and b"1 to 256" in grid._native.load().grid_last_error()
