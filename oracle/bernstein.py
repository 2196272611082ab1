"""Bernstein-Bezier algebra on the reference tetrahedron, by plain definitions.

Test infrastructure (see the package docstring): only tests, smoke() and the
bench's CPU-baseline leg may use this module.

Everything is FP64 and dense. Matrices are built from the moment integral of
a barycentric monomial over a d-simplex, normalised by the simplex measure,

    (1/|T|) * int_T lambda^gamma = d! * prod(gamma_i!) / (|gamma| + d)!,

and operators are obtained by dense LU solves against the Bernstein mass
matrix. None of the sparse stencils or telescoped forms of Sec. 5 are used to
*build* anything here; they are only fitted (``projection_coeffs``,
``mass_inverse_coeffs``) so that Table 1 and Table 2 can pin this module.

Conventions (readings of the paper, each listed in the design notes):
  * barycentric coordinates and basis B^N_alpha = C^N_alpha lambda^alpha
    (Sec. 2);
  * multi-index order: for l in 0..N, k in 0..N-l, j in 0..N-l-k:
    alpha = (N-j-k-l, j, k, l)  (the paper leaves the order open);
  * face f of the tetrahedron is {lambda_f = 0}; its nodes are the alpha with
    alpha_f = 0, and a face multi-index lists the remaining three entries in
    increasing vertex order;
  * every mass matrix is normalised by the measure of its simplex, so the
    physical matrices are |T| * M and |f| * M_f (Sec. 3.1).
"""
from __future__ import annotations

from functools import lru_cache
from math import comb, factorial

import numpy as np

__all__ = [
    "np_count", "multi_indices", "face_multi_indices", "index_of",
    "multinomial", "moment", "mass", "mixed_mass", "face_mass",
    "weighted_mass_terms", "elevation", "elevation_chain", "derivative",
    "lift", "projection", "projection_coeffs", "mass_inverse_coeffs",
    "evaluate", "product", "condition_number",
]


def np_count(n: int, d: int = 3) -> int:
    """Dimension of P^n on a d-simplex: C(n+d, d) (N_p in Sec. 2)."""
    return comb(n + d, d) if n >= 0 else 0


@lru_cache(maxsize=None)
def multi_indices(n: int) -> tuple:
    """All alpha with |alpha| = n on the tetrahedron, in the library order."""
    out = []
    for l in range(n + 1):
        for k in range(n - l + 1):
            for j in range(n - l - k + 1):
                out.append((n - j - k - l, j, k, l))
    return tuple(out)


@lru_cache(maxsize=None)
def face_multi_indices(n: int) -> tuple:
    """All (b0, b1, b2) with sum n on a triangle: b2 outer, b1 inner."""
    out = []
    for b2 in range(n + 1):
        for b1 in range(n - b2 + 1):
            out.append((n - b1 - b2, b1, b2))
    return tuple(out)


@lru_cache(maxsize=None)
def _index_map(n: int) -> dict:
    return {a: i for i, a in enumerate(multi_indices(n))}


def index_of(alpha) -> int:
    """Position of a multi-index in ``multi_indices(|alpha|)`` (dict lookup)."""
    alpha = tuple(int(x) for x in alpha)
    return _index_map(sum(alpha))[alpha]


def multinomial(alpha) -> int:
    """C^N_alpha = N! / prod(alpha_i!) (Sec. 2)."""
    r = factorial(sum(alpha))
    for a in alpha:
        r //= factorial(a)
    return r


def moment(gamma, d: int = 3) -> float:
    """Normalised integral of lambda^gamma over a d-simplex (Dirichlet)."""
    num = factorial(d)
    for g in gamma:
        num *= factorial(g)
    return num / factorial(sum(gamma) + d)


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


@lru_cache(maxsize=None)
def mixed_mass(n: int, m: int) -> np.ndarray:
    """(1/|T|) int_T B^n_alpha B^m_beta, rows alpha (deg n), cols beta (deg m)."""
    A, B = multi_indices(n), multi_indices(m)
    out = np.empty((len(A), len(B)))
    for i, a in enumerate(A):
        ca = multinomial(a)
        for j, b in enumerate(B):
            out[i, j] = ca * multinomial(b) * moment(_add(a, b))
    out.setflags(write=False)
    return out


def mass(n: int) -> np.ndarray:
    """Normalised Bernstein mass matrix M (Sec. 3.1)."""
    return mixed_mass(n, n)


@lru_cache(maxsize=None)
def face_mass(n: int, f: int) -> np.ndarray:
    """Normalised face mass matrix M_f of face f = {lambda_f = 0} (Sec. 3.1).

    A degree-n Bernstein function restricted to face f vanishes unless
    alpha_f = 0; then it is the 2D Bernstein function on the face's three
    vertices with the remaining entries of alpha.
    """
    A = multi_indices(n)
    out = np.zeros((len(A), len(A)))
    for i, a in enumerate(A):
        if a[f]:
            continue
        for j, b in enumerate(A):
            if b[f]:
                continue
            g = tuple(x + y for t, (x, y) in enumerate(zip(a, b)) if t != f)
            out[i, j] = multinomial(a) * multinomial(b) * moment(g, d=2)
    out.setflags(write=False)
    return out


@lru_cache(maxsize=None)
def weighted_mass_terms(n: int, m: int) -> np.ndarray:
    """T[beta, alpha, gamma] = (1/|T|) int B^n_alpha B^m_beta B^n_gamma.

    For a weight w = sum_beta w_beta B^m_beta the weighted mass matrix
    M_w of Sec. 3.1 is sum_beta w_beta T[beta] (exactly, no quadrature).
    """
    A, B = multi_indices(n), multi_indices(m)
    out = np.empty((len(B), len(A), len(A)))
    for q, b in enumerate(B):
        cb = multinomial(b)
        for i, a in enumerate(A):
            ca = multinomial(a)
            ab = _add(a, b)
            for j, g in enumerate(A):
                out[q, i, j] = ca * cb * multinomial(g) * moment(_add(ab, g))
    out.setflags(write=False)
    return out


def _solve_mass(n: int, rhs: np.ndarray) -> np.ndarray:
    return np.linalg.solve(mass(n), rhs)


@lru_cache(maxsize=None)
def elevation(n: int) -> np.ndarray:
    """E^n_{n-1}: coefficient map P^{n-1} -> P^n (Sec. 5.2).

    Built as the L2 projection of each degree-(n-1) basis function onto P^n,
    which is exact because P^{n-1} is contained in P^n; the sparse identity of
    Eq. (12) is *not* used here (it is a test of this matrix).
    """
    out = _solve_mass(n, mixed_mass(n, n - 1))
    out.setflags(write=False)
    return out


def elevation_chain(n: int, i: int) -> np.ndarray:
    """E^n_{n-i} = E^n_{n-1} E^{n-1}_{n-2} ... E^{n-i+1}_{n-i} (Eq. 13)."""
    out = np.eye(np_count(n))
    for k in range(i):
        out = out @ elevation(n - k)
    return out


@lru_cache(maxsize=None)
def derivative(n: int) -> np.ndarray:
    """Barycentric derivative matrices D^m = M^{-1} S_m, m = 0..3 (Sec. 4).

    (S_m)_{alpha,beta} = (1/|T|) int B^n_alpha dB^n_beta/dlambda_m with
    dB^n_beta/dlambda_m = n B^{n-1}_{beta - e_m} (differentiating
    lambda^beta). The physical derivative of p is sum_m (dlambda_m/dx_i) D^m p.
    """
    A = multi_indices(n)
    S = np.zeros((4, len(A), len(A)))
    for m in range(4):
        for j, b in enumerate(A):
            if b[m] == 0:
                continue
            bm = list(b)
            bm[m] -= 1
            bm = tuple(bm)
            cb = n * multinomial(bm)
            for i, a in enumerate(A):
                S[m, i, j] = multinomial(a) * cb * moment(_add(a, bm))
    out = np.stack([_solve_mass(n, S[m]) for m in range(4)])
    out.setflags(write=False)
    return out


@lru_cache(maxsize=None)
def lift(n: int) -> np.ndarray:
    """Reference lift matrices L^f = M^{-1} M_f, f = 0..3 (Eq. 4).

    Columns of face nodes only are meaningful; the result is returned as a
    full N_p x N_p matrix per face with zero columns off the face.
    """
    out = np.stack([_solve_mass(n, face_mass(n, f)) for f in range(4)])
    out.setflags(write=False)
    return out


@lru_cache(maxsize=None)
def projection(n: int, m: int) -> np.ndarray:
    """L2 projection P^{n+m}_n = M_n^{-1} M_{n,n+m} (Sec. 5.3), dense."""
    out = _solve_mass(n, mixed_mass(n, n + m))
    out.setflags(write=False)
    return out


def projection_coeffs(n: int, m: int):
    """c_j of Theorem 5.3, by least squares against the dense projection.

    Returns (c, relative residual). The paper obtains c_j by "solving a linear
    system"; here the overdetermined system  sum_j c_j E^n_{n-j} (E^n_{n-j})^T
    (E^{n+m}_n)^T = P^{n+m}_n  is solved in the least-squares sense.
    """
    red = elevation_chain(n + m, m).T
    cols = []
    for j in range(n + 1):
        E = elevation_chain(n, j)
        cols.append((E @ E.T @ red).ravel())
    A = np.stack(cols, axis=1)
    P = projection(n, m).ravel()
    c, *_ = np.linalg.lstsq(A, P, rcond=None)
    res = np.linalg.norm(A @ c - P) / np.linalg.norm(P)
    return c, res


def mass_inverse_coeffs(n: int):
    """c_j of Theorem 5.5 (M^{-1} = sum_j c_j E^n_{n-j} (E^n_{n-j})^T).

    Least squares against the dense inverse of the *unnormalised* mass
    matrix of the reference element of Sec. 2 (r,s,t >= -1, volume 4/3),
    which is the normalisation Table 2 uses.
    """
    Minv = np.linalg.inv(mass(n) * (4.0 / 3.0))
    cols = []
    for j in range(n + 1):
        E = elevation_chain(n, j)
        cols.append((E @ E.T).ravel())
    A = np.stack(cols, axis=1)
    c, *_ = np.linalg.lstsq(A, Minv.ravel(), rcond=None)
    res = np.linalg.norm(A @ c - Minv.ravel()) / np.linalg.norm(Minv)
    return c, res


def condition_number(c) -> float:
    """sum_j |c_j| (Eq. 18)."""
    return float(np.sum(np.abs(c)))


def evaluate(coeffs: np.ndarray, n: int, lam: np.ndarray) -> np.ndarray:
    """Evaluate sum_alpha coeffs[..., alpha] B^n_alpha at barycentric points.

    ``lam`` has shape (P, 4); returns shape coeffs.shape[:-1] + (P,).
    """
    A = multi_indices(n)
    lam = np.asarray(lam, dtype=np.float64)
    basis = np.empty((len(A), lam.shape[0]))
    for i, a in enumerate(A):
        basis[i] = multinomial(a) * np.prod(lam ** np.array(a), axis=1)
    return np.asarray(coeffs) @ basis


def product(a: np.ndarray, n: int, b: np.ndarray, m: int) -> np.ndarray:
    """Coefficients in P^{n+m} of f*g, by L2 projection of the exact product.

    f = sum a_alpha B^n_alpha, g = sum b_beta B^m_beta. The product lies in
    P^{n+m}, so projecting it is exact: h = M_{n+m}^{-1} (int B^{n+m}_gamma f g).
    """
    G, A, B = multi_indices(n + m), multi_indices(n), multi_indices(m)
    rhs = np.zeros(len(G))
    for gi, g in enumerate(G):
        cg = multinomial(g)
        s = 0.0
        for ai, al in enumerate(A):
            if a[ai] == 0.0:
                continue
            ca = multinomial(al) * a[ai]
            ga = _add(g, al)
            for bi, be in enumerate(B):
                s += ca * multinomial(be) * b[bi] * moment(_add(ga, be))
        rhs[gi] = cg * s
    return _solve_mass(n + m, rhs)
