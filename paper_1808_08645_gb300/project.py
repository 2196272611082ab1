"""L2 projection of fields onto per-element Bernstein polynomials (tools layer).

The paper prepares c^2 in preprocessing: it is approximated per element by
its L2 projection onto P^M (Sec. 5 and the convergence study of Sec. 6.1),
and the initial condition is projected onto P^N. These helpers do that on
the host, in FP64 with numpy/scipy; they are not part of the GPU hot path.

    coeffs[k] = M^{-1} int_{D^k} f B_alpha / |D^k|

with M the mass matrix of the unit-volume reference element, evaluated by a
collapsed-coordinate Gauss-Jacobi rule (exact for degree 2q - 1 in each
collapsed direction), in element chunks. ``project_c2`` also checks that
every Bernstein coefficient is positive, which makes c^2_M > 0 on the element
(convex hull property; the solver rejects anything else with
BBW_ERR_NONPOS_C2).
"""
from __future__ import annotations

from math import factorial

import numpy as np
from scipy.special import roots_jacobi

__all__ = ["tet_rule", "lattice", "bernstein_values", "reference_mass", "l2_project", "project_c2",
           "NonPositiveC2"]


class NonPositiveC2(ValueError):
    """A projected c^2 has a Bernstein coefficient <= 0."""


def tet_rule(q: int):
    """(lam [P, 4], w [P]) with sum(w) = 1: the Stroud conical product rule on
    the simplex with q points per direction (Gauss-Jacobi weights (2,0),
    (1,0), (0,0) in the collapsed coordinates)."""
    a, wa = roots_jacobi(q, 2.0, 0.0)
    b, wb = roots_jacobi(q, 1.0, 0.0)
    c, wc = roots_jacobi(q, 0.0, 0.0)
    a, b, c = (a + 1) / 2, (b + 1) / 2, (c + 1) / 2
    wa, wb, wc = wa / 8, wb / 4, wc / 2
    A, B, Cc = np.meshgrid(a, b, c, indexing="ij")
    W = (wa[:, None, None] * wb[None, :, None] * wc[None, None, :])
    l3 = A
    l2 = (1 - A) * B
    l1 = (1 - A) * (1 - B) * Cc
    l0 = 1 - l1 - l2 - l3
    lam = np.stack([l0, l1, l2, l3], -1).reshape(-1, 4)
    w = W.reshape(-1) * 6.0  # the collapsed Jacobian integrates to 1/6 on the unit tetrahedron
    return lam, w


def lattice(n: int) -> np.ndarray:
    """Multi-indices (alpha_0..alpha_3) of degree n in the library order."""
    out = []
    for l in range(n + 1):
        for k in range(n - l + 1):
            for j in range(n - l - k + 1):
                out.append((n - j - k - l, j, k, l))
    return np.array(out, dtype=np.int64)


def bernstein_values(n: int, lam: np.ndarray) -> np.ndarray:
    """[P, N_p] values B^n_alpha(lam) = n!/alpha! lam^alpha."""
    A = lattice(n)
    coef = np.array([factorial(n) / np.prod([factorial(int(x)) for x in a]) for a in A])
    return coef[None, :] * np.prod(lam[:, None, :] ** A[None, :, :], axis=2)


def reference_mass(n: int) -> np.ndarray:
    """Mass matrix of the degree-n Bernstein basis on the unit-volume simplex
    (Dirichlet moments: int lambda^g = 3! g! / (|g| + 3)!)."""
    A = lattice(n)
    f = [factorial(i) for i in range(2 * n + 4)]
    coef = np.array([f[n] / np.prod([f[int(x)] for x in a]) for a in A])
    S = A[:, None, :] + A[None, :, :]
    mom = 6.0 / f[2 * n + 3] * np.prod(np.vectorize(lambda x: f[x])(S), axis=2)
    return coef[:, None] * coef[None, :] * mom


def l2_project(vxyz, etov, n: int, field, q: int | None = None, chunk: int = 8192) -> np.ndarray:
    """[K, N_p] Bernstein coefficients of the per-element L2 projection of
    field(x [P, 3]) -> [P] onto P^n (degree-n Bernstein basis, library order)."""
    vxyz = np.asarray(vxyz, dtype=np.float64)
    etov = np.asarray(etov, dtype=np.int64)
    q = q or n + 3
    lam, w = tet_rule(q)
    Bv = bernstein_values(n, lam)                # [P, Np]
    WB = w[:, None] * Bv                          # quadrature times basis
    L = np.linalg.cholesky(reference_mass(n))
    out = np.empty((len(etov), Bv.shape[1]))
    for k0 in range(0, len(etov), chunk):
        X = vxyz[etov[k0:k0 + chunk]]             # [k, 4, 3]
        pts = np.einsum("pa,kai->kpi", lam, X)    # [k, P, 3]
        F = np.asarray(field(pts.reshape(-1, 3)), dtype=np.float64).reshape(len(X), -1)
        rhs = F @ WB                              # [k, Np] = int f B / |D|
        y = np.linalg.solve(L, rhs.T)
        out[k0:k0 + chunk] = np.linalg.solve(L.T, y).T
    return out


def project_c2(vxyz, etov, M: int, field, q: int | None = None) -> np.ndarray:
    """The L2 projection of c^2 onto P^M per element, [K, M_p]; raises
    NonPositiveC2 if any Bernstein coefficient is <= 0 (the solver would reject
    it with BBW_ERR_NONPOS_C2)."""
    c2 = l2_project(vxyz, etov, M, field, q=q or M + 4)
    bad = ~(c2 > 0)
    if bad.any():
        k = int(np.argwhere(bad.any(axis=1))[0, 0])
        raise NonPositiveC2(f"{int(bad.sum())} projected c^2 coefficients <= 0 (first in element {k})")
    return c2
