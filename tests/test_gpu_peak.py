"""The arithmetic-rate loop behind the roofline's denominator (grid_peak_loop):
its flop count and a plausible rate on the device."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,per_fma", [(0, 2), (1, 4), (2, 2)])
def test_peak_loop_counts_and_runs(kind, per_fma):
    import paper_2109_06976_gb300 as grid
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = grid._native.load()
    blocks, threads, iters = 152, 256, 4096
    out = torch.zeros(blocks * threads, dtype=torch.float64 if kind == 2 else torch.float32, device="cuda")
    fl = ctypes.c_double()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    grid._native.check("grid_peak_loop", lib.grid_peak_loop(kind, blocks, threads, iters,
                                                            ctypes.c_void_p(out.data_ptr()), ctypes.byref(fl),
                                                            ctypes.c_void_p(stream.cuda_stream)))
    e1.record(stream)
    torch.cuda.synchronize()
    # 8 multiply-add chains per thread, 2 flops each (paired: two per instruction)
    assert fl.value == blocks * threads * iters * 8 * per_fma
    assert torch.isfinite(out).all() and (out != 0).any()
    tflops = fl.value / (e0.elapsed_time(e1) / 1e3) / 1e12
    assert 0.01 < tflops < 200.0
