"""The parity metrics (tests/metrics.py) on hand-made cases: the per-knot form
agrees with the scalar one, and the FP32 bar n kappa(M) u bounds the error of an
FP32 solve through a computed inverse on random SPD matrices at conditions of
1e1 to 1e4."""
import numpy as np

from tests.metrics import U32, col_rel_err, col_rel_err_knots, fp32_bar


def test_per_knot_metric_matches_scalar():
    rng = np.random.default_rng(1)
    y = rng.normal(size=(9, 5, 10))
    y[:, :, 3] *= 1e-9                              # a column below the floor
    x = y + 1e-6 * rng.normal(size=y.shape)
    e = col_rel_err_knots(x, y, floor=1e-4)
    assert e.shape == (9,)
    assert e.max() == col_rel_err(x, y, floor=1e-4)
    # the knot with the planted error is the one that reads it
    x[4, 2, 7] += 1.0
    e2 = col_rel_err_knots(x, y, floor=1e-4)
    assert np.argmax(e2) == 4 and np.allclose(np.delete(e2, 4), np.delete(e, 4))


def test_fp32_bar_values():
    d = np.array([[1.0, 0.0], [0.0, 1e-5]])          # kappa = 1e5, n = 2
    assert np.isclose(fp32_bar(d[None])[0], 2 * 1e5 * U32)
    assert fp32_bar(np.eye(3)[None])[0] == 1e-4      # well conditioned: the flat bar


def test_fp32_bar_bounds_an_fp32_solve():
    rng = np.random.default_rng(7)
    worst = 0.0
    for n in (4, 7, 12, 30):
        for logk in (1, 2, 3, 4):
            Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
            M = (Q * np.logspace(0, -logk, n)) @ Q.T
            Mi = np.linalg.inv(M)
            Mi32 = np.linalg.inv(M.astype(np.float32))
            for _ in range(8):
                b = rng.normal(size=n)
                x = Mi @ b
                x32 = Mi32 @ b.astype(np.float32)
                err = np.abs(x32 - x).max() / np.linalg.norm(x)
                bound = n * np.linalg.cond(Mi) * U32
                worst = max(worst, err / bound)
    assert worst <= 1.0, worst
