"""Semi-discrete acoustic WADG operator and LSRK stage, FP64 (test infrastructure).

The right-hand side follows the strong DG form of Eq. (2) with penalty fluxes
(Sec. 3.1), lifted by L^f = M^{-1} M_f, and the weight-adjusted mass of Eq. (4):

    dU_i/dt = -d_i p + sum_f (A_f/V) n_i L^f (1/2)(tau_u [[u]].n - [[p]])
    dp/dt   = M^{-1} M_{c2} ( -div u + sum_f (A_f/V) L^f (1/2)(tau_p [[p]] - n.[[u]])
                               + source )

Readings of the paper used here (listed in the design notes):
  * the weight is c^2 (Eq. 4 has M^{-1} M_{c^2}); M_{c^2} is the exact
    weighted mass matrix of the degree-M Bernstein polynomial c^2_M;
  * the signs of the volume and flux terms are those of Eq. (2) (the leading
    minus sign of Eq. (4) applies to the volume term only);
  * walls are p = 0 mirrors: p+ = -p, u+ = u;
  * the time integrator is the 5-stage, 2N-storage RK4 of Carpenter and
    Kennedy (cited in Sec. 6.3.1); its stage times are derived from a, b.

Everything is dense: D^m = M^{-1} S_m, L^f = M^{-1} M_f and
M^{-1} M_{c^2} = M^{-1} sum_beta c2_beta T_beta, with no sparse stencil and no
telescoped projection.
"""
from __future__ import annotations

from fractions import Fraction
from math import ceil, exp, pi

import numpy as np

from . import bernstein as bb
from .mesh import connectivity, face_node_map, geometry, locate_point

__all__ = ["LSRK_A", "LSRK_B", "lsrk_stage_times", "stability_polynomial",
           "AcousticOracle", "ricker", "cfl_dt"]

# Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage RK.
LSRK_A = (
    Fraction(0),
    Fraction(-567301805773, 1357537059087),
    Fraction(-2404267990393, 2016746695238),
    Fraction(-3550918686646, 2091501179385),
    Fraction(-1275806237668, 842570457699),
)
LSRK_B = (
    Fraction(1432997174477, 9575080441755),
    Fraction(5161836677717, 13612068292357),
    Fraction(1720146321549, 2090206949498),
    Fraction(3134564353537, 4481467310338),
    Fraction(2277821191437, 14882151754819),
)


def _butcher():
    """Equivalent Butcher matrix and weights of the 2N-storage scheme.

    With dq_s = a_s dq_{s-1} + h F_s and q_s = q_{s-1} + b_s dq_s, stage s
    (0-based) sees q_{s-1} = q_0 + h sum_{m<s} A[s][m] F_m where
    A[s][m] = sum_{i=m}^{s-1} b_i prod_{r=m+1}^{i} a_r.
    """
    S = len(LSRK_A)
    A = [[Fraction(0)] * S for _ in range(S + 1)]
    for s in range(1, S + 1):
        for m in range(s):
            acc = Fraction(0)
            for i in range(m, s):
                prod = Fraction(1)
                for r in range(m + 1, i + 1):
                    prod *= LSRK_A[r]
                acc += LSRK_B[i] * prod
            A[s][m] = acc
    return A


def lsrk_stage_times():
    """c_s = sum_m A[s][m] (row sums of the Butcher matrix), exact rationals."""
    A = _butcher()
    return tuple(sum(A[s][:s], Fraction(0)) for s in range(len(LSRK_A)))


def stability_polynomial():
    """Coefficients of R(z) for y' = z y over one step, exact rationals."""
    S = len(LSRK_A)
    # track q and dq as polynomials in z (lists of Fractions)
    q = [Fraction(1)]
    dq = [Fraction(0)]

    def add(x, y):
        n = max(len(x), len(y))
        return [(x[i] if i < len(x) else 0) + (y[i] if i < len(y) else 0) for i in range(n)]

    for s in range(S):
        zq = [Fraction(0)] + q
        dq = add([LSRK_A[s] * c for c in dq], zq)
        q = add(q, [LSRK_B[s] * c for c in dq])
    return q


def ricker(t: float, f0: float, t0: float) -> float:
    """Ricker wavelet (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)."""
    a = (pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * exp(-a)


def cfl_dt(geo, c2: np.ndarray, n: int, cfl: float) -> float:
    """dt = CFL / (sqrt(max c2 coefficient) * (N+1)(N+3)/3 * max_f A_f/V)."""
    ratio = np.max(geo["area"] / geo["vol"][:, None])
    cn = (n + 1) * (n + 3) / 3.0
    return cfl / (np.sqrt(np.max(c2)) * cn * ratio)


class AcousticOracle:
    """Dense FP64 WADG solver on an affine tetrahedral mesh.

    State layout: q[field, element, coefficient] with fields (p, u, v, w).
    """

    def __init__(self, vxyz, etov, n: int, m: int, c2: np.ndarray,
                 tau_p: float = 1.0, tau_u: float = 1.0):
        self.vxyz = np.asarray(vxyz, dtype=np.float64)
        self.etov = np.asarray(etov, dtype=np.int64)
        self.N, self.M = n, m
        self.K = len(self.etov)
        self.Np = bb.np_count(n)
        self.c2 = np.asarray(c2, dtype=np.float64).reshape(self.K, bb.np_count(m))
        self.tau_p, self.tau_u = float(tau_p), float(tau_u)
        self.etoe, self.etof = connectivity(self.etov)
        self.geo = geometry(self.vxyz, self.etov)
        if np.any(self.geo["vol"] <= 0):
            raise ValueError("inverted element")
        self.nmap = face_node_map(self.vxyz, self.etov, self.etoe, self.etof, n)
        self.D = bb.derivative(n)
        self.L = bb.lift(n)
        self.Mhat = bb.mass(n)
        self.T = bb.weighted_mass_terms(n, m)
        A = bb.multi_indices(n)
        self.face_nodes = [np.array([i for i, a in enumerate(A) if a[f] == 0]) for f in range(4)]
        # sources: (elements, coefficient vectors [n, Np], amplitude samples);
        # sample 5 n + s drives stage s of step n, zero past the end
        self.source = None

    # -- sources -------------------------------------------------------------
    def set_point_source(self, x, amp):
        """Point source delta(x - x_s) a(t) added to the pressure equation,
        a(t) given by one sample per RK stage.

        Its degree-N coefficients on the containing element are
        M^{-1} B(x_s) / |T| (test against every basis function, strong form).
        """
        e, lam = locate_point(self.vxyz, self.etov, x)
        B = bb.evaluate(np.eye(self.Np), self.N, lam[None, :])[:, 0]
        vec = np.linalg.solve(self.Mhat, B) / self.geo["vol"][e]
        self.set_forcing([e], vec[None, :], amp)
        return e, vec

    def set_forcing(self, elems, coeffs, amp):
        """Forcing a(t) g(x) in the pressure equation: g given by degree-N
        Bernstein coefficients coeffs [n, Np] on elements elems, a(t) by one
        sample per RK stage."""
        elems = np.asarray(elems, dtype=np.int64).ravel()
        coeffs = np.asarray(coeffs, dtype=np.float64).reshape(len(elems), self.Np)
        self.source = (elems, coeffs, np.asarray(amp, dtype=np.float64).ravel())

    def source_amplitude(self, k) -> float:
        """Amplitude sample k (None or past the end of the series: 0)."""
        if self.source is None or k is None or not 0 <= k < len(self.source[2]):
            return 0.0
        return float(self.source[2][k])

    # -- operator ------------------------------------------------------------
    def traces(self, q: np.ndarray, f: int):
        """Own and neighbour values of the four fields on face f's nodes."""
        idx = self.face_nodes[f]
        own = q[:, :, idx]                                   # (4, K, Nfp)
        nb = self.nmap[:, f, idx]                            # (K, Nfp)
        flat = q.reshape(4, -1)
        wall = nb < 0
        nbr = flat[:, np.where(wall, 0, nb)]                 # (4, K, Nfp)
        mirror = own.copy()
        mirror[0] = -own[0]                                  # p+ = -p, u+ = u
        nbr = np.where(wall[None], mirror, nbr)
        return own, nbr

    def rhs(self, q: np.ndarray, k=None) -> np.ndarray:
        """Semi-discrete right-hand side with the sources at amplitude sample k:
        velocity rows as they are, the pressure bracket through the
        weight-adjusted update (Eq. 4)."""
        out, bracket = self.spatial(q, k)
        out[0] = self.wadg(bracket)
        return out

    def spatial(self, q: np.ndarray, k=None):
        """(out, bracket): out[1:4] the velocity right-hand sides, bracket the
        pressure right-hand side before the weight-adjusted update (volume
        term, lifted penalty fluxes of Eq. (2) and the sources at amplitude
        sample k)."""
        q = np.asarray(q, dtype=np.float64)
        p, u = q[0], q[1:4]
        g = self.geo["grad"]                                 # (K, 4, 3)
        Dp = np.einsum("mab,kb->kma", self.D, p)
        gradp = np.einsum("kmi,kma->ika", g, Dp)             # (3, K, Np)
        Du = np.einsum("mab,ikb->ikma", self.D, u)
        divu = np.einsum("kmi,ikma->ka", g, Du)              # (K, Np)
        lift_p = np.zeros_like(p)
        lift_u = np.zeros_like(u)
        for f in range(4):
            own, nbr = self.traces(q, f)
            jp = nbr[0] - own[0]
            ju = nbr[1:4] - own[1:4]
            n = self.geo["normal"][:, f, :]                  # (K, 3)
            ndu = np.einsum("ki,ikj->kj", n, ju)
            Fp = np.zeros_like(p)
            Fu = np.zeros_like(p)
            Fp[:, self.face_nodes[f]] = 0.5 * (self.tau_p * jp - ndu)
            Fu[:, self.face_nodes[f]] = 0.5 * (self.tau_u * ndu - jp)
            sc = self.geo["area"][:, f] / self.geo["vol"]    # A_f / V
            LFp = np.einsum("ab,kb->ka", self.L[f], Fp) * sc[:, None]
            LFu = np.einsum("ab,kb->ka", self.L[f], Fu) * sc[:, None]
            lift_p += LFp
            lift_u += np.einsum("ki,ka->ika", n, LFu)
        out = np.empty_like(q)
        out[1:4] = -gradp + lift_u
        bracket = -divu + lift_p
        a = self.source_amplitude(k)
        if a != 0.0:
            bracket[self.source[0]] += a * self.source[1]
        out[0] = 0.0
        return out, bracket

    def wadg(self, r: np.ndarray) -> np.ndarray:
        """M^{-1} M_{c2} r per element (the weight-adjusted update, Eq. 4)."""
        Tr = np.einsum("bij,kj->kbi", self.T, r)             # (K, Mp, Np)
        Mr = np.einsum("kb,kbi->ki", self.c2, Tr)
        return np.linalg.solve(self.Mhat, Mr.T).T

    # -- time stepping -------------------------------------------------------
    def stage(self, q, res, s: int, dt: float, step: int = 0):
        """Stage s of RK step `step`: res = a_s res + dt rhs(q), q += b_s res,
        with the sources at amplitude sample 5 step + s (the stage time is
        t + c_s dt)."""
        r = self.rhs(q, 5 * int(step) + s)
        res = float(LSRK_A[s]) * res + dt * r
        q = q + float(LSRK_B[s]) * res
        return q, res

    def step(self, q, res, dt: float, step: int = 0):
        for s in range(5):
            q, res = self.stage(q, res, s, dt, step)
        return q, res

    def run(self, q, dt: float, nsteps: int, step0: int = 0):
        res = np.zeros_like(q)
        for i in range(nsteps):
            q, res = self.step(q, res, dt, step0 + i)
        return q, res

    def dt_for(self, T: float, cfl: float):
        """(dt, nsteps) with nsteps = ceil(T / dt_cfl), dt = T / nsteps."""
        dt = cfl_dt(self.geo, self.c2, self.N, cfl)
        nsteps = int(ceil(T / dt))
        return T / nsteps, nsteps

    # -- energy --------------------------------------------------------------
    def energy(self, q) -> float:
        """sum_k V_k (p^T M (M_{c2})^{-1} M p + sum_i u_i^T M u_i)."""
        q = np.asarray(q, dtype=np.float64)
        vol = self.geo["vol"]
        Mc2 = np.einsum("kb,bij->kij", self.c2, self.T)
        Mp = q[0] @ self.Mhat
        ep = np.einsum("ki,ki->k", Mp, np.linalg.solve(Mc2, Mp[..., None])[..., 0])
        eu = np.einsum("ika,ab,ikb->k", q[1:4], self.Mhat, q[1:4])
        return float(np.sum(vol * (ep + eu)))
