"""Pins of the oracle's receiver-misfit gradient (oracle/adjoint.py) against
finite differences of the oracle's own forward run, and of the operator
identity L(tau)^T = -M_w L(-tau) M_w^{-1} that the GPU adjoint is built on
(M_w the weight-adjusted mass of Eq. (4); the identity is the energy
structure of the penalty-flux DG operator: skew central part, symmetric
penalty part linear in tau)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import bernstein as bb
from oracle.acoustic import AcousticOracle
from paper_1808_08645_gb300 import inputs

N, M = 2, 1
XR = np.array([[0.3, 0.4, 0.9], [0.7, 0.2, 0.5], [0.5, 0.5, 0.0]])


def _case(seed=0, source=True):
    vxyz, etov = inputs.cube_mesh(1, jitter=0.1, shuffle=True, seed=3 + seed)
    K = len(etov)
    rng = np.random.default_rng(seed)
    c2 = rng.uniform(0.5, 2.0, (K, bb.np_count(M)))
    q0 = rng.standard_normal((4, K, bb.np_count(N))) * 0.1
    return vxyz, etov, c2, q0, rng, source


def _oracle(vxyz, etov, c2, source, tau=1.0):
    o = AcousticOracle(vxyz, etov, N, M, c2, tau_p=tau, tau_u=tau)
    if source:
        o.set_point_source(np.array([0.5, 0.5, 0.5]), np.random.default_rng(5).uniform(-1.0, 1.0, 40))
    return o


def _traces(vxyz, etov, c2, q0, source, dt=0.01, nsteps=3):
    o = _oracle(vxyz, etov, c2, source)
    return adj.record(o, q0, dt, nsteps, adj.receiver_matrix(o, XR))[0]


@pytest.mark.parametrize("source", [True, False])
def test_c2_gradient_matches_central_differences(source):
    vxyz, etov, c2, q0, rng, src = _case(1, source)
    o = _oracle(vxyz, etov, c2, src)
    R = adj.receiver_matrix(o, XR)
    tr, _ = adj.record(o, q0, 0.01, 3, R)
    g = rng.standard_normal(tr.shape)
    gc, _ = adj.misfit_gradient(o, q0, 0.01, 3, R, g)
    d = rng.standard_normal(c2.shape)
    eps = 1e-5
    fd = (np.sum(g * _traces(vxyz, etov, c2 + eps * d, q0, src))
          - np.sum(g * _traces(vxyz, etov, c2 - eps * d, q0, src))) / (2 * eps)
    assert abs(fd - np.sum(gc * d)) <= 1e-7 * abs(fd)


def test_initial_state_gradient_matches_central_differences():
    vxyz, etov, c2, q0, rng, src = _case(2)
    o = _oracle(vxyz, etov, c2, src)
    R = adj.receiver_matrix(o, XR)
    tr, _ = adj.record(o, q0, 0.01, 3, R)
    g = rng.standard_normal(tr.shape)
    _, gq = adj.misfit_gradient(o, q0, 0.01, 3, R, g)
    d = rng.standard_normal(q0.shape)
    eps = 1e-5
    fd = (np.sum(g * _traces(vxyz, etov, c2, q0 + eps * d, src))
          - np.sum(g * _traces(vxyz, etov, c2, q0 - eps * d, src))) / (2 * eps)
    assert abs(fd - np.sum(gq * d)) <= 1e-9 * abs(fd)


def test_receivers_sample_the_pressure_polynomial():
    """R q equals the pressure polynomial evaluated at the receiver points."""
    vxyz, etov, c2, q0, rng, src = _case(3)
    o = _oracle(vxyz, etov, c2, False)
    R = adj.receiver_matrix(o, XR)
    from oracle.mesh import locate_point
    for r, x in enumerate(XR):
        e, lam = locate_point(o.vxyz, o.etov, x)
        want = bb.evaluate(q0[0, e], N, lam[None, :])[0]
        assert abs(R[r] @ q0.ravel() - want) <= 1e-13 * max(1.0, abs(want))


def test_operator_transpose_identity():
    """L(tau)^T = -M_w L(-tau) M_w^{-1}, and M_w L + L^T M_w <= 0."""
    vxyz, etov, c2, _, _, _ = _case(4)
    o, om = _oracle(vxyz, etov, c2, False, 1.0), _oracle(vxyz, etov, c2, False, -1.0)
    L, Lm = adj._stage_matrix(o), adj._stage_matrix(om)
    K, Np = o.K, o.Np
    vol = o.geo["vol"]
    Mc2 = np.einsum("kb,bij->kij", c2, o.T)
    Mw = np.zeros_like(L)
    for k in range(K):
        for f in range(4):
            sl = slice((f * K + k) * Np, (f * K + k + 1) * Np)
            Mw[sl, sl] = vol[k] * (o.Mhat @ np.linalg.solve(Mc2[k], o.Mhat) if f == 0 else o.Mhat)
    assert np.linalg.norm(L.T + Mw @ Lm @ np.linalg.inv(Mw)) <= 1e-12 * np.linalg.norm(L)
    S = Mw @ L + L.T @ Mw
    assert np.max(np.linalg.eigvalsh(0.5 * (S + S.T))) <= 1e-12 * np.linalg.norm(S)
