"""Error metric of the parity tests.

Per knot point and output column j (a vector output counts as one column):
    e_j = max_i |x_ij - y_ij| / max(||y_:j||_2, floor * max_k ||y_:k||_2, 1e-30)
with y the FP64 oracle. FP64 is held to e <= 1e-10 with floor = 1e-6 (FLOOR64).
FP32 is held to e <= 1e-4 with floor = 1e-4 (FLOOR32): an FP32 result resolves
a column only to about u = 6e-8 of the largest column, so a relative bar on a
column far below that scale measures the order of the roundings, not the
method. With the floor, a column below 1e-4 of the largest is held to an
absolute 1e-8 of the largest column. (The 12-DoF tree has 0.1 % of its columns
below 1e-4 of the largest; on one of them, at 1.3e-5, the error moved across
1e-4 with the summation order of the spatial products alone.)
"""
import numpy as np

FLOOR32 = 1e-4
FLOOR64 = 1e-6


def col_rel_err(x, y, floor=1e-6):
    """Largest per-column relative error over all knot points. x, y: [N, rows, cols]."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    assert x.shape == y.shape, (x.shape, y.shape)
    nrm = np.linalg.norm(y, axis=-2)                                  # [N, cols]
    den = np.maximum(nrm, floor * nrm.max(axis=-1, keepdims=True))
    den = np.maximum(den, 1e-30)
    return float((np.abs(x - y).max(axis=-2) / den).max()) if x.size else 0.0


def col_rel_err_knots(x, y, floor=1e-6):
    """The metric above per knot point: [N], the largest column error of each."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    assert x.shape == y.shape, (x.shape, y.shape)
    nrm = np.linalg.norm(y, axis=-2)
    den = np.maximum(np.maximum(nrm, floor * nrm.max(axis=-1, keepdims=True)), 1e-30)
    return (np.abs(x - y).max(axis=-2) / den).max(axis=-1)


U32 = 2.0 ** -24     # unit roundoff of FP32


def fp32_bar(minv, tol=1e-4):
    """Per-knot FP32 bar for random test trees: the larger of `tol` and
    n kappa_2(M) u, the first-order forward-error bound of a solve with a
    computed inverse (u = 2^-24). The columns -M^-1 dID/dq_j of such a tree can be
    small against ||M^-1|| ||dID/dq_j||; then any rounding order leaves an error
    of that size. Example: a 12-DoF random forest at kappa = 380 measured
    2e-5 to 2e-4 on one column, depending on the evaluation order alone.
    minv: [N, n, n] from the oracle."""
    minv = np.asarray(minv, dtype=np.float64)
    return np.maximum(tol, minv.shape[-1] * np.linalg.cond(minv) * U32)


def col_rel_err_stats(x, y, floor=1e-6):
    """(max, p50) over knot points of the per-knot max column error."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    nrm = np.linalg.norm(y, axis=-2)
    den = np.maximum(np.maximum(nrm, floor * nrm.max(axis=-1, keepdims=True)), 1e-30)
    per_knot = (np.abs(x - y).max(axis=-2) / den).max(axis=-1)
    return float(per_knot.max()), float(np.median(per_knot))


def vec_rel_err(x, y, floor=1e-6):
    """Vector outputs [N, n] as one column each."""
    return col_rel_err(np.asarray(x)[:, :, None], np.asarray(y)[:, :, None], floor)


def col_err_split(x, y, zero=1e-12, floor=1e-6):
    """Errors for outputs with structurally zero columns (their oracle norm is at
    rounding level, e.g. d/dq of a prismatic base joint, or a column that is zero
    by cancellation of O(1) terms, where FP32 leaves noise of ~1e-7 of the
    largest column). Per knot point, with m = the largest column norm:
      e_nz = the metric above (with `floor`) over columns with norm > zero * m,
      e_z  = max |x - y| / m over the structurally zero columns.
    Returns (max e_nz, max e_z) over knot points."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    assert x.shape == y.shape, (x.shape, y.shape)
    if x.size == 0:
        return 0.0, 0.0
    nrm = np.linalg.norm(y, axis=-2)                                   # [N, cols]
    m = np.maximum(nrm.max(axis=-1, keepdims=True), 1e-30)
    diff = np.abs(x - y).max(axis=-2)
    zmask = nrm <= zero * m
    e_nz = np.where(zmask, 0.0, diff / np.maximum(nrm, floor * m))
    e_z = np.where(zmask, diff / m, 0.0)
    return float(e_nz.max()), float(e_z.max())


def derived_col_bar(minv, dc, J, tol=1e-4):
    """Per knot point and column j, the FP32 bar max(tol, n kappa_2(M) u alpha_j) with
    alpha_j = ||M^-1||_2 ||dc_:j||_2 / ||J_:j||_2: the first-order error of
    J_:j = -M^-1 dc_:j computed through a computed inverse is about
    n kappa_2(M) u ||M^-1|| ||dc_:j||, so a column made small by cancellation in the
    product (alpha_j >> 1) carries that much more error relative to its own norm.
    minv [N, n, n], dc [N, n, 2n] (dID/dq | dID/dqd at qdd) and J [N, n, 2n] from the
    oracle. Returns [N, 2n]."""
    minv = np.asarray(minv, dtype=np.float64)
    dc = np.asarray(dc, dtype=np.float64)
    J = np.asarray(J, dtype=np.float64)
    n = minv.shape[-1]
    nrm_mi = np.linalg.norm(minv, ord=2, axis=(-2, -1))               # [N]
    kappa = np.linalg.cond(minv)                                      # [N]
    alpha = nrm_mi[:, None] * np.linalg.norm(dc, axis=-2) / np.maximum(np.linalg.norm(J, axis=-2), 1e-300)
    return np.maximum(tol, n * kappa[:, None] * U32 * alpha)


def col_rel_err_cols(x, y, floor=1e-6):
    """The per-column metric itself, [N, cols]."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    nrm = np.linalg.norm(y, axis=-2)
    den = np.maximum(np.maximum(nrm, floor * nrm.max(axis=-1, keepdims=True)), 1e-30)
    return np.abs(x - y).max(axis=-2) / den
