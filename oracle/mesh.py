"""Mesh connectivity, affine geometry and face-node matching (test infrastructure).

Plain, brute-force versions of what the solver needs from a tetrahedral mesh:

* neighbours by matching the sorted global-vertex triple of every face
  (Sec. 3.1: D^k non-overlapping, conforming);
* per-element barycentric gradients, volume, face areas and outward normals
  from the vertex coordinates (the affine map of Sec. 2);
* face-node matching by *coordinate equality* of Bernstein domain points
  x_alpha = sum_i alpha_i v_i / N (Sec. 4: jumps of Bernstein traces are
  differences of face coefficients under a node-to-node map).
"""
from __future__ import annotations

import numpy as np

from .bernstein import multi_indices

__all__ = ["FACE_VERTS", "connectivity", "geometry", "domain_points",
           "face_node_map", "locate_point"]

#: local vertices of face f = {lambda_f = 0}, in increasing order
FACE_VERTS = tuple(tuple(v for v in range(4) if v != f) for f in range(4))


def connectivity(etov: np.ndarray):
    """Return (etoe, etof): neighbour element and its local face, -1 on walls.

    Faces are keyed by their sorted global vertex ids; a key seen twice is an
    interior face, once a wall, more than twice a non-manifold mesh (error).
    """
    etov = np.asarray(etov, dtype=np.int64)
    K = etov.shape[0]
    seen: dict = {}
    for e in range(K):
        for f in range(4):
            key = tuple(sorted(int(etov[e, v]) for v in FACE_VERTS[f]))
            seen.setdefault(key, []).append((e, f))
    etoe = -np.ones((K, 4), dtype=np.int64)
    etof = -np.ones((K, 4), dtype=np.int64)
    for key, owners in seen.items():
        if len(owners) > 2:
            raise ValueError(f"non-manifold face {key}")
        if len(owners) == 2:
            (e1, f1), (e2, f2) = owners
            etoe[e1, f1], etof[e1, f1] = e2, f2
            etoe[e2, f2], etof[e2, f2] = e1, f1
    return etoe, etof


def geometry(vxyz: np.ndarray, etov: np.ndarray):
    """Affine geometry per element.

    Returns a dict with
      vol   (K,)       signed volume (positive for a valid orientation)
      grad  (K, 4, 3)  d lambda_m / d x_i
      area  (K, 4)     face areas
      normal(K, 4, 3)  outward unit normals
    """
    X = np.asarray(vxyz, dtype=np.float64)[np.asarray(etov)]  # (K, 4, 3)
    K = X.shape[0]
    A = np.ones((K, 4, 4))
    A[:, 1:, :] = np.transpose(X, (0, 2, 1))  # columns are [1, x, y, z] of vertices
    # lambda = A^{-1} [1, x, y, z]^T, so d lambda_m / d x_i = (A^{-1})[m, 1+i]
    Ainv = np.linalg.inv(A)
    grad = Ainv[:, :, 1:]
    vol = np.linalg.det(A) / 6.0
    area = np.empty((K, 4))
    normal = np.empty((K, 4, 3))
    for f in range(4):
        a, b, c = (X[:, v] for v in FACE_VERTS[f])
        cr = np.cross(b - a, c - a)
        nrm = np.linalg.norm(cr, axis=1)
        area[:, f] = 0.5 * nrm
        n = cr / nrm[:, None]
        # outward: pointing away from the opposite vertex f
        s = np.sign(np.einsum("ki,ki->k", n, a - X[:, f]))
        normal[:, f] = n * s[:, None]
    return {"vol": vol, "grad": grad, "area": area, "normal": normal}


def domain_points(vxyz: np.ndarray, etov: np.ndarray, n: int) -> np.ndarray:
    """Physical Bernstein domain points, shape (K, N_p, 3)."""
    X = np.asarray(vxyz, dtype=np.float64)[np.asarray(etov)]
    A = np.array(multi_indices(n), dtype=np.float64) / max(n, 1)
    return np.einsum("pa,kai->kpi", A, X)


def face_node_map(vxyz, etov, etoe, etof, n: int) -> np.ndarray:
    """Neighbour coefficient index for every face node, by coordinate matching.

    Returns ``nmap`` of shape (K, 4, N_p): for a face node alpha (alpha_f = 0)
    of element e, ``nmap[e, f, i]`` is the flat index nb * N_p + i' of the
    neighbour coefficient at the same physical domain point; entries off the
    face and on walls are -1.
    """
    K = len(etov)
    A = multi_indices(n)
    Np = len(A)
    pts = domain_points(vxyz, etov, n)
    scale = np.abs(np.asarray(vxyz)).max() + 1.0
    nmap = -np.ones((K, 4, Np), dtype=np.int64)
    for e in range(K):
        for f in range(4):
            nb = etoe[e, f]
            if nb < 0:
                continue
            fb = etof[e, f]
            mine = [i for i, a in enumerate(A) if a[f] == 0]
            theirs = [i for i, a in enumerate(A) if a[fb] == 0]
            for i in mine:
                d = np.linalg.norm(pts[nb, theirs] - pts[e, i], axis=1)
                j = int(np.argmin(d))
                if d[j] > 1e-10 * scale:
                    raise ValueError("face nodes do not match")
                nmap[e, f, i] = nb * Np + theirs[j]
    return nmap


def locate_point(vxyz, etov, x, tol: float = 1e-12):
    """Lowest element id whose closure contains x, and x's barycentrics there."""
    geo = geometry(vxyz, etov)
    X = np.asarray(vxyz, dtype=np.float64)[np.asarray(etov)]
    x = np.asarray(x, dtype=np.float64)
    for e in range(len(etov)):
        # lambda is affine with lambda(v_0) = e_0 and gradient grad
        lam = geo["grad"][e] @ (x - X[e, 0]) + np.array([1.0, 0.0, 0.0, 0.0])
        if np.all(lam >= -tol):
            return e, lam
    raise ValueError("point outside the mesh")
