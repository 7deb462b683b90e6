"""Algorithmic operation count of one gradient-of-forward-dynamics evaluation.

Counts the floating-point operations of the method's own steps, independent of
how a kernel schedules them: RNEA(q, qd, 0) (Sec. IV-B), the direct M^-1
articulated-inertia recursion (Sec. IV-B, Carpentier 2018), qdd = M^-1 (tau - c),
RNEA at qdd, the analytical RNEA derivatives (Alg. 1 forward pass over
subtree(j) for every column, backward pass over subtree(j) and the ancestors of
j) and the product -M^-1 dID restricted to the base-branch blocks.

Rules: every multiply and every add counts 1 (an FMA counts 2); sin and cos
count 1 each; a division counts 1. Spatial transforms use the compact (E, r)
form and inertias the compact (m, h, Ibar) form; revolute joints with a general
unit axis. Primitive costs (flops):
  X m, X^T f, I m                  42 each
  m x (a s) (S qd-type products)   21
  a x b, a x* f (general)          30
  S^T f                            5
"""
from __future__ import annotations

XM = 42          # X m / X^T f / I m
CRM_S = 21       # v x (S qd) with S qd = [a qd; 0]
CR = 30          # general motion or force cross product
ST = 5           # S^T f
ADD6 = 6


def _topology(parent):
    n = len(parent)
    depth, sub = [0] * n, [1] * n
    for i in range(n):
        depth[i] = 0 if parent[i] < 0 else depth[parent[i]] + 1
    for i in reversed(range(n)):
        if parent[i] >= 0:
            sub[parent[i]] += sub[i]
    comp = [0] * n
    for i in range(n):
        comp[i] = i if parent[i] < 0 else comp[parent[i]]
    comp_size = {c: sub[c] for c in set(comp)}
    return depth, sub, comp, comp_size


def grad_fd_flops(parent) -> dict:
    """Per-knot-point flop counts by step, and the total."""
    parent = [int(p) for p in parent]
    n = len(parent)
    depth, sub, comp, comp_size = _topology(parent)
    has_p = [p >= 0 for p in parent]
    out = {}
    # RNEA(q, qd, 0): forward v (X v + S qd), a (X a + v x S qd), f (I a + v x* I v)
    fwd = (XM + 6) + (XM + CRM_S + ADD6) + (XM + XM + CR + ADD6)
    bwd_body = lambda i: ST + (XM + ADD6 if has_p[i] else 0)
    out["rnea_bias"] = n * fwd + sum(bwd_body(i) for i in range(n))
    # direct M^-1, backward: U (6 x S^T), D, 1/D, row of subtree, F columns,
    # downdate (21 entries x 3) and congruence (12 transforms) + accumulate (36)
    mb = 0
    for i in range(n):
        mb += 6 * ST + ST + 1 + 6 * (sub[i] - 1)
        if has_p[i]:
            mb += sub[i] * (12 + XM) + 21 * 3 + 12 * XM + 36
    # forward: per (i, k >= i in the branch): X P, U.t, scale, subtract, P = S m + t
    mf = 0
    for i in range(n):
        cols = comp_size[comp[i]] - (i - comp[i])
        mf += cols * ((XM + 11 + 2 + 6) if has_p[i] else 6)
    out["minv"] = mb + mf
    out["fd"] = sum(1 + 2 * comp_size[comp[i]] for i in range(n))
    # RNEA at qdd: da = X da_p + S qdd, f += I da; backward sweep again
    out["rnea_qdd"] = n * (XM + 6 + XM + ADD6) + sum(bwd_body(i) for i in range(n))
    # dRNEA: forward over subtree(j) per column, backward over subtree(j) + ancestors
    col_fwd = (XM) + (XM + CRM_S + ADD6) + (XM + CR + XM + CR + 2 * ADD6)
    root_extra = {0: CRM_S + 3 + ADD6, 1: 3 + CRM_S + ADD6}      # case terms (u = q / qd)
    g = 0
    for u in (0, 1):
        for j in range(n):
            g += sub[j] * col_fwd + root_extra[u] + (XM if u == 0 else 0)   # (X a_p) x S needs X a_p
            touched = sub[j] + depth[j]          # subtree(j) and the ancestors of j
            g += touched * ST + (touched - 1) * (XM + ADD6)  # dc_i = S^T dF_i; push to parent
            if u == 0 and has_p[j]:
                g += 12 + XM + ADD6              # X^T (S x* F_j)
    out["grad_rnea"] = g
    out["product"] = sum((2 * comp_size[comp[i]]) * (2 * comp_size[comp[i]]) for i in range(n))
    out["total"] = sum(out.values())
    return out


def grad_fd_flops_per_knot(parent) -> int:
    return int(grad_fd_flops(parent)["total"])
