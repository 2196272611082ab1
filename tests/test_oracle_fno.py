"""Pins of the FP64 reference network (oracle/fno.py): the DCT basis is
orthonormal, its hand-written backward equals central differences of its
forward, and a mode-free layer reduces to the pointwise network."""
import numpy as np
import pytest

from oracle import fno

CFG = dict(grid=6, width=3, modes=(2, 3, 2), layers=2, cin=4, hidden=5, nt=4, rx=[0, 3], ry=[1, 2], rz=[4, 1])


def test_cosine_basis_is_orthonormal():
    for n, m in ((64, 6), (7, 7)):
        P = fno.cosine_basis(n, m)
        assert np.allclose(P.T @ P, np.eye(m), atol=1e-13)
    # the full basis diagonalises nothing special but is a complete orthogonal transform
    P = fno.cosine_basis(8, 8)
    assert np.allclose(P @ P.T, np.eye(8), atol=1e-13)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    p = fno.init_params(CFG, seed=1)
    x = rng.standard_normal((2, 6, 6, 6, 4))
    dy = rng.standard_normal((2, 2, 4))
    y, cache = fno.forward(p, CFG, x)
    g = fno.backward(p, CFG, cache, dy)
    eps = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            yp, _ = fno.forward(p, CFG, x)
            flat[idx] = old - eps
            ym, _ = fno.forward(p, CFG, x)
            flat[idx] = old
            fd = np.sum(dy * (yp - ym)) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)


def test_zero_spectral_weights_give_the_pointwise_network():
    rng = np.random.default_rng(2)
    p = fno.init_params(CFG, seed=3)
    for l in range(CFG["layers"]):
        p[f"W{l}_sp"][:] = 0.0
    x = rng.standard_normal((1, 6, 6, 6, 4))
    y, _ = fno.forward(p, CFG, x)
    u = x @ p["W0"] + p["b0"]
    for l in range(CFG["layers"]):
        v = u @ p[f"W{l}_pw"] + p[f"b{l}_pw"]
        u = 0.5 * v * (1 + np.vectorize(__import__("math").erf)(v / np.sqrt(2)))
    # receiver r: the mean over its 2 x 2 x 2 block, written as a block average
    r = np.stack([u[:, x0:x0 + 2, y0:y0 + 2, z0:z0 + 2].mean(axis=(1, 2, 3))
                  for x0, y0, z0 in zip(CFG["rx"], CFG["ry"], CFG["rz"])], axis=1)
    hp = r @ p["W1"] + p["b1"]
    h = 0.5 * hp * (1 + np.vectorize(__import__("math").erf)(hp / np.sqrt(2)))
    assert np.allclose(y, h @ p["W2"] + p["b2"], atol=1e-13)
