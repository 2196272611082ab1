"""Collapsed-coordinate Gauss rules on the tetrahedron (test infrastructure).

The paper's WADG baseline uses quadrature exact to degree 2N+1 (Sec. 3.3) and
switches to a collapsed-coordinate rule for N > 7. The Xiao-Gimbutas tables are
not available here, so the oracle uses the collapsed (Duffy) rule for every
degree: Gauss-Legendre in each of (u, v, w) in [0, 1]^3, mapped by

    lambda1 = u, lambda2 = v (1-u), lambda3 = w (1-u)(1-v),
    lambda0 = 1 - lambda1 - lambda2 - lambda3,

with Jacobian (1-u)^2 (1-v). Weights are normalised to sum to 1, so
sum_q w_q f(lambda_q) approximates (1/|T|) int_T f.
"""
from __future__ import annotations

import numpy as np

__all__ = ["tet_rule", "tri_rule"]


def _gauss01(q: int):
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def tet_rule(degree: int):
    """Barycentric points (Q, 4) and normalised weights (Q,), exact to ``degree``."""
    q = degree // 2 + 2
    x, w = _gauss01(q)
    u, v, s = np.meshgrid(x, x, x, indexing="ij")
    wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
    l1 = u
    l2 = v * (1.0 - u)
    l3 = s * (1.0 - u) * (1.0 - v)
    l0 = 1.0 - l1 - l2 - l3
    wt = 6.0 * wu * wv * ws * (1.0 - u) ** 2 * (1.0 - v)
    lam = np.stack([l0, l1, l2, l3], axis=-1).reshape(-1, 4)
    return lam, wt.ravel()


def tri_rule(degree: int):
    """Barycentric points (Q, 3) and normalised weights on a triangle."""
    q = degree // 2 + 2
    x, w = _gauss01(q)
    u, v = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    l1 = u
    l2 = v * (1.0 - u)
    l0 = 1.0 - l1 - l2
    wt = 2.0 * wu * wv * (1.0 - u)
    lam = np.stack([l0, l1, l2], axis=-1).reshape(-1, 3)
    return lam, wt.ravel()
