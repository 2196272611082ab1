"""Pins of the elastic oracle (oracle/elastic.py) against what the paper and
the mathematics fix, each independent of the oracle's own formulas:

* mu = 0, rho = 1, sigma = -p I: the velocity-stress system is the acoustic
  one with c^2 = lambda (Sec. 2.2 reduces to Eq. 1), so the elastic operator
  must equal the (separately pinned) acoustic oracle;
* a global polynomial state of degree <= N whose traction vanishes on the
  walls has no jumps anywhere, so the right-hand side must be the exact
  rho^{-1} div sigma and Hooke's law applied to the strain rate (written here
  from the textbook definitions, not from the A_i matrices);
* the assembled operator is skew in the weight-adjusted energy inner product
  for tau = 0 and dissipative for tau > 0 (energy stability, Sec. 2.2);
* the matrix-weighted update equals a quadrature L2 projection of C(x) r(x)
  with C(x) assembled pointwise from Hooke's law (Eq. 7 with a matrix weight);
* with central fluxes the operator is rotation covariant (v -> R v,
  sigma -> R sigma R^T, the stress rotated as a tensor, not through A_i).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.acoustic import AcousticOracle
from oracle.elastic import ElasticOracle
from oracle.mesh import domain_points
from oracle.quadrature import tet_rule
from paper_1808_08645_gb300 import inputs


def _rand_bary(rng, P):
    x = rng.exponential(size=(P, 4))
    return x / x.sum(1, keepdims=True)


def hooke(lam, mu, strain):
    """Isotropic stress from the engineering strain vector
    (e_xx, e_yy, e_zz, g_yz, g_xz, g_xy): sigma = lam tr(e) I + 2 mu e, with
    shear stress mu * g (textbook linear elasticity)."""
    tr = strain[0] + strain[1] + strain[2]
    return np.stack([lam * tr + 2 * mu * strain[0], lam * tr + 2 * mu * strain[1],
                     lam * tr + 2 * mu * strain[2], mu * strain[3], mu * strain[4], mu * strain[5]])


def test_mu_zero_reduces_to_the_acoustic_operator():
    vxyz, etov = inputs.cube_mesh(1, jitter=0.1, shuffle=True, seed=2)
    K = len(etov)
    N, M = 3, 1
    rng = np.random.default_rng(0)
    c2 = rng.uniform(0.5, 2.0, (K, bb.np_count(M)))
    tau = 0.7
    ac = AcousticOracle(vxyz, etov, N, M, c2, tau_p=tau, tau_u=0.0)
    el = ElasticOracle(vxyz, etov, N, M, np.ones_like(c2), c2, np.zeros_like(c2), tau_v=0.0, tau_s=tau)
    qa = rng.standard_normal((4, K, ac.Np))
    qe = np.zeros((9, K, el.Np))
    qe[:3] = qa[1:4]
    qe[3:6] = -qa[0]
    ra, re = ac.rhs(qa), el.rhs(qe)
    scale = np.abs(ra).max()
    assert np.abs(re[:3] - ra[1:4]).max() <= 1e-12 * scale
    for a in range(3):
        assert np.abs(re[3 + a] + ra[0]).max() <= 1e-12 * scale
    assert np.abs(re[6:]).max() <= 1e-12 * scale


def _poly_state():
    """v of degree <= 4, sigma of degree <= 4 with zero traction on the unit
    cube walls (sigma_xx vanishes on x = 0, 1, sigma_xy on x and y walls, ...).
    Returns value and derivative functions of x (P, 3)."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    bx, by, bz = x * (1 - x), y * (1 - y), z * (1 - z)
    v = [1 + 2 * x - y + x * y * z + 0.5 * z ** 3,
         0.3 - x ** 2 + y * z - 0.2 * x * y ** 2,
         -0.7 + 0.4 * x * z + y ** 2 * z - x ** 4]
    s = [bx * (1 + 0.5 * y - 0.3 * z), by * (0.8 - x + 0.2 * z), bz * (1.2 + 0.4 * x * y),
         by * bz * 1.5, bx * bz * (-0.9), bx * by * 0.6]
    X = (x, y, z)
    fv = [sp.lambdify(X, e, "numpy") for e in v + s]
    dv = [[sp.lambdify(X, sp.diff(e, c), "numpy") for c in X] for e in v]
    ds = [[sp.lambdify(X, sp.diff(e, c), "numpy") for c in X] for e in s]

    def ev(fs, P):
        return np.stack([np.broadcast_to(np.asarray(f(P[:, 0], P[:, 1], P[:, 2]), float), (len(P),))
                         for f in fs])

    return ev, fv, dv, ds


def test_polynomial_state_is_differentiated_exactly():
    ev, fv, dv, ds = _poly_state()
    vxyz, etov = inputs.cube_mesh(2, jitter=0.12, shuffle=True, seed=9)
    K = len(etov)
    N, M = 4, 2
    Mp = bb.np_count(M)
    rho_inv, lam, mu = 0.8, 1.7, 0.6
    el = ElasticOracle(vxyz, etov, N, M, np.full((K, Mp), rho_inv), np.full((K, Mp), lam),
                       np.full((K, Mp), mu), tau_v=1.0, tau_s=1.0)
    # Bernstein coefficients by interpolation at the domain points (exact for degree <= N)
    nodes = np.array(bb.multi_indices(N), float) / N
    Vn = bb.evaluate(np.eye(el.Np), N, nodes).T
    pts = domain_points(vxyz, etov, N)
    q = np.empty((9, K, el.Np))
    for k in range(K):
        q[:, k] = np.linalg.solve(Vn, ev(fv, pts[k]).T).T
    r = el.rhs(q)
    rng = np.random.default_rng(1)
    X = np.asarray(vxyz)[np.asarray(etov)]
    for k in range(0, K, 5):
        lamq = _rand_bary(rng, 7)
        P = lamq @ X[k]
        got = np.stack([bb.evaluate(r[c, k], N, lamq) for c in range(9)])
        gs = [ev(d, P) for d in ds]          # gs[a][i] = d sigma_a / dx_i
        gv = [ev(d, P) for d in dv]          # gv[c][i] = d v_c / dx_i
        div = np.stack([gs[0][0] + gs[5][1] + gs[4][2],
                        gs[5][0] + gs[1][1] + gs[3][2],
                        gs[4][0] + gs[3][1] + gs[2][2]])
        strain = np.stack([gv[0][0], gv[1][1], gv[2][2], gv[1][2] + gv[2][1],
                           gv[0][2] + gv[2][0], gv[0][1] + gv[1][0]])
        want = np.concatenate([rho_inv * div, hooke(lam, mu, strain)])
        assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


def _assemble(orc):
    n = 9 * orc.K * orc.Np
    A = np.empty((n, n))
    for c in range(n):
        q = np.zeros(n)
        q[c] = 1.0
        A[:, c] = orc.rhs(q.reshape(9, orc.K, orc.Np)).ravel()
    return A


def _energy_matrix(orc):
    Hv, Hs, Np = orc.energy_matrix_blocks()
    K = orc.K
    n = 9 * K * Np
    H = np.zeros((n, n))
    idx = lambda fld, k: np.arange((fld * K + k) * Np, (fld * K + k + 1) * Np)
    for k in range(K):
        for c in range(3):
            ii = idx(c, k)
            H[np.ix_(ii, ii)] = Hv[k]
        ii = np.concatenate([idx(3 + a, k) for a in range(6)])
        H[np.ix_(ii, ii)] = Hs[k]
    return H


@pytest.mark.parametrize("tau", [0.0, 1.0])
def test_assembled_operator_energy_stability(tau):
    """H A + A^T H = 0 for tau = 0 (central fluxes), <= 0 for tau > 0."""
    vxyz, etov = inputs.cube_mesh(1, jitter=0.1, shuffle=True, seed=5)
    K = len(etov)
    N, M = 2, 1
    rng = np.random.default_rng(3)
    Mp = bb.np_count(M)
    orc = ElasticOracle(vxyz, etov, N, M, rng.uniform(0.5, 1.5, (K, Mp)), rng.uniform(0.5, 2.0, (K, Mp)),
                        rng.uniform(0.3, 1.0, (K, Mp)), tau_v=tau, tau_s=tau)
    A = _assemble(orc)
    H = _energy_matrix(orc)
    S = H @ A + A.T @ H
    scale = np.abs(H @ A).max()
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    if tau == 0.0:
        assert np.abs(S).max() < 1e-10 * scale
    else:
        assert ev.max() < 1e-10 * scale and ev.min() < -1e-3 * scale


def test_matrix_weighted_update_matches_quadrature():
    """(I x M^{-1}) M_C r = L2 projection of C(x) r(x), C(x) from Hooke's law
    with lambda(x), mu(x) of degree M; velocity rows with rho^{-1}(x)."""
    vxyz, etov = inputs.cube_mesh(1, jitter=0.0, shuffle=False, seed=0)
    N, M = 3, 2
    K = len(etov)
    Mp, Np = bb.np_count(M), bb.np_count(N)
    rng = np.random.default_rng(7)
    ri, la, mu = (rng.uniform(0.4, 2.0, (K, Mp)) for _ in range(3))
    orc = ElasticOracle(vxyz, etov, N, M, ri, la, mu)
    r = rng.standard_normal((9, K, Np))
    got = orc.wadg(r)
    lq, w = tet_rule(2 * N + M)
    Vq = bb.evaluate(np.eye(Np), N, lq).T                      # (Q, Np)
    Pq = np.linalg.solve(bb.mass(N), Vq.T * w)                  # (Np, Q)
    for k in range(K):
        rq = r[:, k] @ Vq.T                                     # (9, Q)
        want_v = Pq @ (bb.evaluate(ri[k], M, lq) * rq[:3]).T
        want_s = Pq @ hooke(bb.evaluate(la[k], M, lq), bb.evaluate(mu[k], M, lq), rq[3:]).T
        assert np.allclose(got[:3, k], want_v.T, atol=1e-11)
        assert np.allclose(got[3:, k], want_s.T, atol=1e-11)


def test_energy_decays_over_steps_with_penalty():
    vxyz, etov = inputs.cube_mesh(1, jitter=0.1, shuffle=True, seed=6)
    K = len(etov)
    N, M = 2, 1
    Mp = bb.np_count(M)
    rng = np.random.default_rng(11)
    orc = ElasticOracle(vxyz, etov, N, M, np.full((K, Mp), 1.0), rng.uniform(0.5, 2.0, (K, Mp)),
                        rng.uniform(0.3, 1.0, (K, Mp)))
    q = rng.standard_normal((9, K, orc.Np))
    e = [orc.energy(q)]
    res = np.zeros_like(q)
    for _ in range(4):
        q, res = orc.step(q, res, 2e-3)
        e.append(orc.energy(q))
    assert all(b < a for a, b in zip(e, e[1:]))


def _voigt_to_tensor(s):
    """(xx, yy, zz, yz, xz, xy) -> symmetric 3x3 tensor, leading axes kept."""
    T = np.empty(s.shape[1:] + (3, 3))
    T[..., 0, 0], T[..., 1, 1], T[..., 2, 2] = s[0], s[1], s[2]
    T[..., 1, 2] = T[..., 2, 1] = s[3]
    T[..., 0, 2] = T[..., 2, 0] = s[4]
    T[..., 0, 1] = T[..., 1, 0] = s[5]
    return T


def _tensor_to_voigt(T):
    return np.stack([T[..., 0, 0], T[..., 1, 1], T[..., 2, 2], T[..., 1, 2], T[..., 0, 2], T[..., 0, 1]])


def test_central_flux_operator_is_rotation_covariant():
    """Isotropic media, tau = 0: rotating the mesh by R and the fields by
    v -> R v, sigma -> R sigma R^T rotates the right-hand side the same way
    (the velocity-stress system is frame-indifferent; the rotation acts on
    the stress tensor, written here without the A_i matrices). Bernstein
    coefficients rotate like values because the rotation is linear and the
    elements keep their vertex order."""
    vxyz, etov = inputs.cube_mesh(1, jitter=0.1, shuffle=True, seed=12)
    K = len(etov)
    N, M = 3, 1
    Mp = bb.np_count(M)
    rng = np.random.default_rng(21)
    media = (rng.uniform(0.5, 1.5, (K, Mp)), rng.uniform(0.5, 2.0, (K, Mp)), rng.uniform(0.3, 1.0, (K, Mp)))
    A = rng.standard_normal((3, 3))
    R, _ = np.linalg.qr(A)
    if np.linalg.det(R) < 0:
        R[:, 0] = -R[:, 0]
    q = rng.standard_normal((9, K, bb.np_count(N)))
    r = ElasticOracle(vxyz, etov, N, M, *media, tau_v=0.0, tau_s=0.0).rhs(q)
    qr = np.empty_like(q)
    qr[:3] = np.einsum("ij,jkn->ikn", R, q[:3])
    qr[3:] = _tensor_to_voigt(R @ _voigt_to_tensor(q[3:]) @ R.T)
    rr = ElasticOracle(np.asarray(vxyz) @ R.T, etov, N, M, *media, tau_v=0.0, tau_s=0.0).rhs(qr)
    want = np.empty_like(r)
    want[:3] = np.einsum("ij,jkn->ikn", R, r[:3])
    want[3:] = _tensor_to_voigt(R @ _voigt_to_tensor(r[3:]) @ R.T)
    assert np.abs(rr - want).max() <= 1e-11 * np.abs(r).max()
