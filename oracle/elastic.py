"""Semi-discrete elastic WADG operator and LSRK stage, FP64 (test infrastructure).

Velocity-stress form of Sec. 2.2 (Eq. ewave): with v the velocity and sigma
the six unique stress entries in the order (xx, yy, zz, yz, xz, xy),

    rho dv/dt       = sum_i A_i^T d sigma / dx_i
    C^{-1} dsigma/dt = sum_i A_i dv / dx_i

A_i the 6x3 matrices printed in Sec. 2.2 and C the isotropic constitutive
matrix (2 mu + lambda on the normal diagonal, lambda off it, mu on the shear
diagonal). The DG form is the one displayed in Sec. 2.2, in strong form, with
penalty fluxes on every face ([[x]] = x+ - x, A_n = sum_i n_i A_i):

    F_v     = (1/2) A_n^T [[sigma]] + (tau_v / 2) A_n^T A_n [[v]]
    F_sigma = (1/2) A_n [[v]]       + (tau_s / 2) A_n A_n^T [[sigma]]

and the weight-adjusted update of Eq. (ewadg): the velocity right-hand side
goes through M^{-1} M_{rho^{-1}} per component, the stress right-hand side
through (I x M^{-1}) M_C, M_C the 6x6 block matrix of scalar weighted mass
matrices M_{C_ab}.

Readings of the paper used here (listed in the design notes):
  * the weights are rho^{-1}, lambda and mu, each a degree-M Bernstein
    polynomial per element (the same reading as c^2 in the acoustic case);
    M_{C_ab} is the exact weighted mass matrix of C_ab = L6[a, b] lambda +
    U6[a, b] mu;
  * walls are traction-free mirrors: sigma+ = -sigma, v+ = v, the elastic
    counterpart of the acoustic p = 0 wall;
  * the time integrator is the acoustic one (five-stage 2N-storage RK4).

Everything is dense: D^m = M^{-1} S_m, L^f = M^{-1} M_f and the weighted mass
matrices sum_beta w_beta T_beta; no sparse stencil, no telescoped projection.
"""
from __future__ import annotations

import numpy as np

from . import bernstein as bb
from .acoustic import LSRK_A, LSRK_B
from .mesh import connectivity, face_node_map, geometry

__all__ = ["A_MATRICES", "LAMBDA_PATTERN", "MU_PATTERN", "ElasticOracle", "a_normal"]

# A_1, A_2, A_3 of Sec. 2.2, rows in the stress order (xx, yy, zz, yz, xz, xy)
A_MATRICES = np.array([
    [[1, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 1], [0, 1, 0]],
    [[0, 0, 0], [0, 1, 0], [0, 0, 0], [0, 0, 1], [0, 0, 0], [1, 0, 0]],
    [[0, 0, 0], [0, 0, 0], [0, 0, 1], [0, 1, 0], [1, 0, 0], [0, 0, 0]],
], dtype=np.float64)

# isotropic C = lambda * LAMBDA_PATTERN + mu * MU_PATTERN (Sec. 2.2)
LAMBDA_PATTERN = np.zeros((6, 6))
LAMBDA_PATTERN[:3, :3] = 1.0
MU_PATTERN = np.diag([2.0, 2.0, 2.0, 1.0, 1.0, 1.0])


def a_normal(n: np.ndarray) -> np.ndarray:
    """A_n = sum_i n_i A_i for normals n of shape (..., 3): shape (..., 6, 3)."""
    return np.einsum("...i,iab->...ab", n, A_MATRICES)


class ElasticOracle:
    """Dense FP64 elastic WADG solver on an affine tetrahedral mesh.

    State layout: q[field, element, coefficient] with fields
    (v_x, v_y, v_z, s_xx, s_yy, s_zz, s_yz, s_xz, s_xy). The media rho_inv,
    lam and mu are [K, M_p] Bernstein coefficients of degree M.
    """

    NF = 9

    def __init__(self, vxyz, etov, n: int, m: int, rho_inv, lam, mu,
                 tau_v: float = 1.0, tau_s: float = 1.0):
        self.vxyz = np.asarray(vxyz, dtype=np.float64)
        self.etov = np.asarray(etov, dtype=np.int64)
        self.N, self.M = n, m
        self.K = len(self.etov)
        self.Np = bb.np_count(n)
        Mp = bb.np_count(m)
        self.rho_inv = np.asarray(rho_inv, dtype=np.float64).reshape(self.K, Mp)
        self.lam = np.asarray(lam, dtype=np.float64).reshape(self.K, Mp)
        self.mu = np.asarray(mu, dtype=np.float64).reshape(self.K, Mp)
        self.tau_v, self.tau_s = float(tau_v), float(tau_s)
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

    # -- operator ------------------------------------------------------------
    def traces(self, q: np.ndarray, f: int):
        """Own and neighbour values of the nine fields on face f's nodes; on
        walls the neighbour is the traction-free mirror (sigma+ = -sigma)."""
        idx = self.face_nodes[f]
        own = q[:, :, idx]
        nb = self.nmap[:, f, idx]
        flat = q.reshape(self.NF, -1)
        wall = nb < 0
        nbr = flat[:, np.where(wall, 0, nb)]
        mirror = own.copy()
        mirror[3:] = -own[3:]
        return own, np.where(wall[None], mirror, nbr)

    def gradients(self, x: np.ndarray) -> np.ndarray:
        """d x / d x_i for fields x of shape (F, K, Np): shape (3, F, K, Np)."""
        g = self.geo["grad"]                                   # (K, 4, 3)
        Dx = np.einsum("mab,fkb->fkma", self.D, x)
        return np.einsum("kmi,fkma->ifka", g, Dx)

    def spatial(self, q: np.ndarray) -> np.ndarray:
        """The bracket of Eq. (ewadg) for all nine fields: volume terms plus
        lifted fluxes, before the weight-adjusted update."""
        q = np.asarray(q, dtype=np.float64)
        v, s = q[:3], q[3:]
        ds = self.gradients(s)                                  # (3, 6, K, Np)
        dv = self.gradients(v)                                  # (3, 3, K, Np)
        out = np.empty_like(q)
        out[:3] = np.einsum("iab,iakn->bkn", A_MATRICES, ds)    # sum_i A_i^T ds/dx_i
        out[3:] = np.einsum("iab,ibkn->akn", A_MATRICES, dv)    # sum_i A_i dv/dx_i
        for f in range(4):
            own, nbr = self.traces(q, f)
            jv = nbr[:3] - own[:3]                               # (3, K, Nfp)
            js = nbr[3:] - own[3:]                               # (6, K, Nfp)
            An = a_normal(self.geo["normal"][:, f, :])           # (K, 6, 3)
            AnT_js = np.einsum("kab,akn->bkn", An, js)           # traction of [[sigma]]
            An_jv = np.einsum("kab,bkn->akn", An, jv)
            Fv = 0.5 * AnT_js + 0.5 * self.tau_v * np.einsum("kab,akn->bkn", An, An_jv)
            Fs = 0.5 * An_jv + 0.5 * self.tau_s * np.einsum("kab,bkn->akn", An, AnT_js)
            F = np.zeros_like(q)
            F[:3][:, :, self.face_nodes[f]] = Fv
            F[3:][:, :, self.face_nodes[f]] = Fs
            sc = self.geo["area"][:, f] / self.geo["vol"]        # A_f / V
            out += np.einsum("ab,fkb->fka", self.L[f], F) * sc[None, :, None]
        return out

    def weighted_mass(self, w: np.ndarray) -> np.ndarray:
        """M_w per element for degree-M weights w [K, M_p]: (K, Np, Np)."""
        return np.einsum("kb,bij->kij", w, self.T)

    def wadg(self, r: np.ndarray) -> np.ndarray:
        """Eq. (ewadg): M^{-1} M_{rho^{-1}} r_v per velocity component and
        (I x M^{-1}) M_C r_sigma for the stress, per element."""
        r = np.asarray(r, dtype=np.float64)
        out = np.empty_like(r)
        Mr = self.weighted_mass(self.rho_inv)
        Ml = self.weighted_mass(self.lam)
        Mm = self.weighted_mass(self.mu)
        # M^{-1} by an LU solve (backward stable), not an explicit inverse
        for c in range(3):
            out[c] = np.linalg.solve(self.Mhat, np.einsum("kjl,kl->jk", Mr, r[c])).T
        for a in range(6):
            acc = np.zeros_like(r[0])
            for b in range(6):
                if LAMBDA_PATTERN[a, b]:
                    acc += LAMBDA_PATTERN[a, b] * np.einsum("kjl,kl->kj", Ml, r[3 + b])
                if MU_PATTERN[a, b]:
                    acc += MU_PATTERN[a, b] * np.einsum("kjl,kl->kj", Mm, r[3 + b])
            out[3 + a] = np.linalg.solve(self.Mhat, acc.T).T
        return out

    def rhs(self, q: np.ndarray) -> np.ndarray:
        return self.wadg(self.spatial(q))

    # -- time stepping -------------------------------------------------------
    def stage(self, q, res, s: int, dt: float):
        """One LSRK stage: res = a_s res + dt rhs(q); q += b_s res."""
        res = float(LSRK_A[s]) * res + dt * self.rhs(q)
        q = q + float(LSRK_B[s]) * res
        return q, res

    def step(self, q, res, dt: float):
        for s in range(5):
            q, res = self.stage(q, res, s, dt)
        return q, res

    def run(self, q, dt: float, nsteps: int):
        res = np.zeros_like(q)
        for _ in range(nsteps):
            q, res = self.step(q, res, dt)
        return q, res

    # -- energy --------------------------------------------------------------
    def energy_matrix_blocks(self):
        """Per element the weight-adjusted mass matrices that the scheme
        conserves: V_k M (M_{rho^{-1}})^{-1} M for each velocity component
        and V_k (I x M) M_C^{-1} (I x M) for the stress (Sec. 2.2)."""
        vol = self.geo["vol"]
        Np = self.Np
        Mr = self.weighted_mass(self.rho_inv)
        Ml = self.weighted_mass(self.lam)
        Mm = self.weighted_mass(self.mu)
        Hv, Hs = [], []
        for k in range(self.K):
            Hv.append(vol[k] * self.Mhat @ np.linalg.solve(Mr[k], self.Mhat))
            MC = np.kron(LAMBDA_PATTERN, Ml[k]) + np.kron(MU_PATTERN, Mm[k])
            IM = np.kron(np.eye(6), self.Mhat)
            Hs.append(vol[k] * IM @ np.linalg.solve(MC, IM))
        return Hv, Hs, Np

    def energy(self, q) -> float:
        q = np.asarray(q, dtype=np.float64)
        Hv, Hs, Np = self.energy_matrix_blocks()
        e = 0.0
        for k in range(self.K):
            for c in range(3):
                e += q[c, k] @ Hv[k] @ q[c, k]
            sk = q[3:, k].reshape(-1)
            e += sk @ Hs[k] @ sk
        return float(e)
