"""Receivers and the gradient of a receiver misfit with respect to the c^2
coefficients, by plain definitions (FP64, dense, small meshes only).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline arm may import this module. It shares no code with the GPU path.

The paper has no adjoint; what is differentiated is the discrete LSRK time
stepping of the semi-discrete system dq/dt = L(c2) q + s(t) that
``AcousticOracle`` integrates (Eq. (2) fluxes, weight-adjusted update of
Eq. (4), five-stage LSRK of Sec. 6.3.1). The gradient is the reverse sweep of
that linear recursion with the dense transpose of the stage matrix, built
column by column from the oracle's own right-hand side; the c^2 derivative
uses that the pressure rows depend on c^2 only through the weight-adjusted
update, which is linear in c^2: d(M^{-1} M_{c2} v)/d c2_beta = M^{-1} T_beta v
(T_beta: the mass matrix weighted by the degree-M Bernstein basis function beta).
Receivers sample the pressure after every step by point evaluation.
"""
from __future__ import annotations

import numpy as np

from . import bernstein as bb
from .acoustic import LSRK_A, LSRK_B, AcousticOracle
from .mesh import locate_point

__all__ = ["receiver_matrix", "record", "misfit_gradient"]


def receiver_matrix(orc: AcousticOracle, xyz) -> np.ndarray:
    """R [nrec, 4 K Np] with R q = pressure at the receivers (point evaluation
    on the containing element, lowest index on shared faces)."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    R = np.zeros((len(xyz), 4 * orc.K * orc.Np))
    for r, x in enumerate(xyz):
        e, lam = locate_point(orc.vxyz, orc.etov, x)
        B = bb.evaluate(np.eye(orc.Np), orc.N, lam[None, :])[:, 0]
        R[r, e * orc.Np:(e + 1) * orc.Np] = B  # field 0 (p), element e
    return R


def record(orc: AcousticOracle, q0, dt: float, nsteps: int, R: np.ndarray, step0: int = 0):
    """Traces [nsteps, nrec] after every step, and the stage inputs of every
    step (list of 5 arrays per step) for the reverse sweep."""
    q = np.asarray(q0, dtype=np.float64).copy()
    res = np.zeros_like(q)
    traces, stages = [], []
    for n in range(nsteps):
        ins = []
        for s in range(5):
            ins.append(q.copy())
            q, res = orc.stage(q, res, s, dt, step0 + n)
        stages.append(ins)
        traces.append(R @ q.ravel())
    return np.array(traces), stages


def _stage_matrix(orc: AcousticOracle) -> np.ndarray:
    """L with rhs(q, k) = L q + rhs(0, k): the linear part, column by column."""
    n = 4 * orc.K * orc.Np
    src = orc.source
    orc.source = None
    L = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = orc.rhs(e.reshape(4, orc.K, orc.Np)).ravel()
    orc.source = src
    return L


def misfit_gradient(orc: AcousticOracle, q0, dt: float, nsteps: int, R: np.ndarray, trace_grad,
                    step0: int = 0):
    """(grad_c2 [K, Mp], grad_q0 [4, K, Np]) of J = sum(trace_grad * traces)."""
    g = np.asarray(trace_grad, dtype=np.float64).reshape(nsteps, -1)
    _, stages = record(orc, q0, dt, nsteps, R, step0)
    L = _stage_matrix(orc)
    K, Np, Mp = orc.K, orc.Np, bb.np_count(orc.M)
    Minv = np.linalg.inv(orc.Mhat)
    qb = np.zeros(4 * K * Np)
    rb = np.zeros_like(qb)
    gc = np.zeros((K, Mp))
    for n in range(nsteps - 1, -1, -1):
        qb += R.T @ g[n]
        for s in range(4, -1, -1):
            rt = rb + float(LSRK_B[s]) * qb
            qb = qb + dt * (L.T @ rt)
            _, v = orc.spatial(stages[n][s], 5 * (step0 + n) + s)
            rp = rt.reshape(4, K, Np)[0]
            for k in range(K):
                for b in range(Mp):
                    gc[k, b] += dt * rp[k] @ (Minv @ (orc.T[b] @ v[k]))
            rb = float(LSRK_A[s]) * rt
    return gc, qb.reshape(4, K, Np)
