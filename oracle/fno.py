"""FP64 reference of the neural-operator surrogate (test infrastructure).

TEST INFRASTRUCTURE: only tests/ and bench.py's CPU-baseline arm may import
this module. It shares no code with the GPU path.

The network (a Fourier-type neural operator on a G^3 grid, in a truncated
cosine basis):

    u_0     = x W_0 + b_0                                   (lift, per grid point)
    pre_l   = u_l W_l + b_l + K_l(u_l),  u_{l+1} = gelu(pre_l),   l < L
    K_l(u)  = Phi ( [Phi^T u]_modes  W_l,mode )            (spectral convolution)
    r       = mean of u_L over the 2 x 2 x 2 grid points of each receiver
    traces  = gelu(r W_1 + b_1) W_2 + b_2

with Phi the orthonormal DCT-II basis truncated to m_x x m_y x m_z modes
(one C x C weight matrix per mode) and gelu(x) = x (1 + erf(x / sqrt 2)) / 2.
Everything is written with plain einsums over named axes; ``backward`` is the
chain rule written out by hand, pinned against central differences of
``forward`` in the tests.
"""
from __future__ import annotations

from math import sqrt

import numpy as np
from scipy.special import erf

__all__ = ["cosine_basis", "init_params", "forward", "backward"]


def cosine_basis(n: int, m: int) -> np.ndarray:
    """[n, m] orthonormal DCT-II vectors phi_k(i) = c_k cos(pi k (i + 1/2) / n)."""
    i = np.arange(n)[:, None] + 0.5
    k = np.arange(m)[None, :]
    phi = np.cos(np.pi * k * i / n) * sqrt(2.0 / n)
    phi[:, 0] = sqrt(1.0 / n)
    return phi


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / sqrt(2.0)))


def _gelu_grad(x):
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * np.exp(-0.5 * x * x) / sqrt(2.0 * np.pi)


def init_params(cfg: dict, seed: int = 0) -> dict:
    """Random parameters of the shapes the network uses (FP64)."""
    rng = np.random.default_rng(seed)
    C, cin, H, T, L = cfg["width"], cfg["cin"], cfg["hidden"], cfg["nt"], cfg["layers"]
    nm = int(np.prod(cfg["modes"]))
    p = {"W0": rng.uniform(-1, 1, (cin, C)) / sqrt(cin), "b0": rng.uniform(-0.1, 0.1, C)}
    for l in range(L):
        p[f"W{l}_pw"] = rng.uniform(-1, 1, (C, C)) / sqrt(C)
        p[f"b{l}_pw"] = rng.uniform(-0.1, 0.1, C)
        p[f"W{l}_sp"] = rng.uniform(-1, 1, (nm, C, C)) / C
    p["W1"] = rng.uniform(-1, 1, (C, H)) / sqrt(C)
    p["b1"] = rng.uniform(-0.1, 0.1, H)
    p["W2"] = rng.uniform(-1, 1, (H, T)) / sqrt(H)
    p["b2"] = rng.uniform(-0.1, 0.1, T)
    return p


def _bases(cfg):
    G = cfg["grid"]
    mx, my, mz = cfg["modes"]
    return cosine_basis(G, mx), cosine_basis(G, my), cosine_basis(G, mz)


def forward(p: dict, cfg: dict, x: np.ndarray):
    """traces [B, R, T] for inputs x [B, G, G, G, cin]; returns (traces, cache)."""
    Px, Py, Pz = _bases(cfg)
    mx, my, mz = cfg["modes"]
    C = cfg["width"]
    rx, ry, rz = np.asarray(cfg["rx"]), np.asarray(cfg["ry"]), np.asarray(cfg["rz"])
    u = x @ p["W0"] + p["b0"]
    us, pres, ss = [u], [], []
    for l in range(cfg["layers"]):
        s = np.einsum("bxyzc,xi,yj,zk->bijkc", u, Px, Py, Pz)
        W = p[f"W{l}_sp"].reshape(mx, my, mz, C, C)
        t = np.einsum("bijkc,ijkcd->bijkd", s, W)
        spec = np.einsum("bijkd,xi,yj,zk->bxyzd", t, Px, Py, Pz)
        pre = u @ p[f"W{l}_pw"] + p[f"b{l}_pw"] + spec
        u = _gelu(pre)
        us.append(u)
        pres.append(pre)
        ss.append(s)
    r = 0.0
    for dx_ in (0, 1):
        for dy_ in (0, 1):
            for dz_ in (0, 1):
                r = r + u[:, rx + dx_, ry + dy_, rz + dz_] / 8.0
    hpre = r @ p["W1"] + p["b1"]
    h = _gelu(hpre)
    y = h @ p["W2"] + p["b2"]
    return y, dict(us=us, pres=pres, ss=ss, r=r, hpre=hpre, h=h, x=x)


def backward(p: dict, cfg: dict, cache: dict, dy: np.ndarray) -> dict:
    """Gradients of sum(dy * traces) with respect to every parameter."""
    Px, Py, Pz = _bases(cfg)
    mx, my, mz = cfg["modes"]
    C = cfg["width"]
    rx, ry, rz = np.asarray(cfg["rx"]), np.asarray(cfg["ry"]), np.asarray(cfg["rz"])
    g = {}
    h, hpre, r = cache["h"], cache["hpre"], cache["r"]
    g["W2"] = np.einsum("brh,brt->ht", h, dy)
    g["b2"] = dy.sum(axis=(0, 1))
    dh = dy @ p["W2"].T * _gelu_grad(hpre)
    g["W1"] = np.einsum("brc,brh->ch", r, dh)
    g["b1"] = dh.sum(axis=(0, 1))
    dr = dh @ p["W1"].T
    du = np.zeros_like(cache["us"][-1])
    for dx_ in (0, 1):
        for dy_ in (0, 1):
            for dz_ in (0, 1):
                np.add.at(du, (slice(None), rx + dx_, ry + dy_, rz + dz_), dr / 8.0)
    for l in reversed(range(cfg["layers"])):
        u, pre, s = cache["us"][l], cache["pres"][l], cache["ss"][l]
        dpre = du * _gelu_grad(pre)
        g[f"W{l}_pw"] = np.einsum("bxyzc,bxyzd->cd", u, dpre)
        g[f"b{l}_pw"] = dpre.sum(axis=(0, 1, 2, 3))
        dt = np.einsum("bxyzd,xi,yj,zk->bijkd", dpre, Px, Py, Pz)
        W = p[f"W{l}_sp"].reshape(mx, my, mz, C, C)
        g[f"W{l}_sp"] = np.einsum("bijkc,bijkd->ijkcd", s, dt).reshape(-1, C, C)
        ds = np.einsum("bijkd,ijkcd->bijkc", dt, W)
        du = dpre @ p[f"W{l}_pw"].T + np.einsum("bijkc,xi,yj,zk->bxyzc", ds, Px, Py, Pz)
    g["W0"] = np.einsum("bxyzi,bxyzc->ic", cache["x"], du)
    g["b0"] = du.sum(axis=(0, 1, 2, 3))
    return g
