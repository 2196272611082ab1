"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU. Each test ties an oracle function to something other than itself:
printed tables (Tables 1-2, Eq. 18), exact identities checked by point
evaluation (Eq. 12, the product of Sec. 5.1), quadrature (Sec. 3.3),
closed forms (the standing wave), energy stability of the assembled operator
(Eq. 2 with penalty fluxes) and the RK stability polynomial.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.acoustic import (AcousticOracle, LSRK_A, LSRK_B, lsrk_stage_times,
                             stability_polynomial)
from oracle.mesh import FACE_VERTS, connectivity, geometry
from oracle.quadrature import tet_rule, tri_rule
from paper_1808_08645_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                out.append(line.split())
    return out


def _rand_bary(rng, P):
    x = rng.exponential(size=(P, 4))
    return x / x.sum(1, keepdims=True)


# -- printed tables ----------------------------------------------------------

@pytest.mark.parametrize("row", _rows("table1_projection_coeffs.txt"), ids=lambda r: f"N{r[0]}M{r[1]}")
def test_table1_projection_coeffs(row):
    N, M = int(row[0]), int(row[1])
    want = np.array([float(x) for x in row[2:]])
    c, res = bb.projection_coeffs(N, M)
    assert res < 1e-10  # Theorem 5.3: the decomposition is exact
    assert np.allclose(c, want, atol=5.1e-5, rtol=0)


@pytest.mark.parametrize("row", _rows("table2_mass_inverse_coeffs.txt"), ids=lambda r: f"N{r[0]}")
def test_table2_mass_inverse_coeffs(row):
    N = int(row[0])
    want = np.array([float(x) for x in row[1:]])
    c, res = bb.mass_inverse_coeffs(N)
    assert res < 1e-9  # Theorem 5.5
    assert np.allclose(c, want, rtol=1e-9, atol=1e-7)


@pytest.mark.parametrize("row", _rows("condition_numbers.txt"), ids=lambda r: f"{r[0]}{r[2]}")
def test_condition_numbers(row):
    op, N, M, val, tol = row[0], int(row[1]), int(row[2]), float(row[3]), float(row[4])
    c = bb.mass_inverse_coeffs(N)[0] if op == "mass_inverse" else bb.projection_coeffs(N, M)[0]
    assert abs(bb.condition_number(c) - val) <= tol * val


def test_table1_mislabelled_row_is_n1():
    # The first row of Table 1 cannot be N=2 (three coefficients); N=2, M=1 is:
    c, _ = bb.projection_coeffs(2, 1)
    assert len(c) == 3 and not np.allclose(c[:2], [0.6667, -0.0667], atol=1e-3)


# -- quadrature and moments --------------------------------------------------

def test_moment_formula_against_quadrature():
    lam, w = tet_rule(12)
    for g in [(0, 0, 0, 0), (3, 1, 0, 2), (2, 2, 2, 2), (0, 5, 1, 0), (6, 0, 0, 6)]:
        q = np.sum(w * np.prod(lam ** np.array(g), axis=1))
        assert abs(q - bb.moment(g)) < 1e-14
    lam2, w2 = tri_rule(10)
    for g in [(0, 0, 0), (2, 3, 1), (5, 0, 5)]:
        q = np.sum(w2 * np.prod(lam2 ** np.array(g), axis=1))
        assert abs(q - bb.moment(g, d=2)) < 1e-14


@pytest.mark.parametrize("N", [1, 2, 4])
def test_mass_matrix_against_quadrature(N):
    lam, w = tet_rule(2 * N)
    V = bb.evaluate(np.eye(bb.np_count(N)), N, lam)     # (Np, Q)
    assert np.allclose((V * w) @ V.T, bb.mass(N), atol=1e-15)


# -- elevation (Eq. 12) -------------------------------------------------------

@pytest.mark.parametrize("N", [1, 3, 6])
def test_elevation_is_the_sparse_identity(N):
    E = bb.elevation(N)
    S = np.zeros_like(E)
    lo = bb.multi_indices(N - 1)
    for c, b in enumerate(lo):
        for j in range(4):
            g = list(b)
            g[j] += 1
            S[bb.index_of(g), c] = (b[j] + 1) / N
    assert np.allclose(E, S, atol=1e-11)
    assert np.all((np.abs(E) > 1e-11).sum(axis=0) == 4)


def test_elevation_preserves_values():
    rng = np.random.default_rng(1)
    lam = _rand_bary(rng, 20)
    a = rng.standard_normal(bb.np_count(4))
    assert np.allclose(bb.evaluate(a, 4, lam), bb.evaluate(bb.elevation(5) @ a, 5, lam), atol=1e-12)


# -- product (Sec. 5.1) -------------------------------------------------------

@pytest.mark.parametrize("N,M", [(2, 1), (3, 2), (4, 3)])
def test_product_pointwise(N, M):
    rng = np.random.default_rng(N * 10 + M)
    a = rng.standard_normal(bb.np_count(N))
    b = rng.standard_normal(bb.np_count(M))
    h = bb.product(a, N, b, M)
    lam = _rand_bary(rng, 25)
    assert np.allclose(bb.evaluate(h, N + M, lam),
                       bb.evaluate(a, N, lam) * bb.evaluate(b, M, lam), atol=1e-11)


def test_product_of_basis_functions():
    # B^N_alpha B^M_beta = C(alpha+beta, alpha) / C(N+M, N) B^{N+M}_{alpha+beta}
    N, M = 3, 2
    from math import comb
    for ai in [0, 5, 11]:
        for bi in [0, 4, 9]:
            a = np.eye(bb.np_count(N))[ai]
            b = np.eye(bb.np_count(M))[bi]
            al, be = bb.multi_indices(N)[ai], bb.multi_indices(M)[bi]
            g = tuple(x + y for x, y in zip(al, be))
            want = np.zeros(bb.np_count(N + M))
            c = 1
            for x, y in zip(g, al):
                c *= comb(x, y)
            want[bb.index_of(g)] = c / comb(N + M, N)
            assert np.allclose(bb.product(a, N, b, M), want, atol=1e-12)


# -- derivative ---------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 3, 5])
def test_derivative_complex_step(N):
    rng = np.random.default_rng(7 + N)
    V = rng.standard_normal((4, 3))
    A = np.ones((4, 4))
    A[1:, :] = V.T
    Ainv = np.linalg.inv(A)
    grad = Ainv[:, 1:]                                    # d lambda_m / d x_i
    a = rng.standard_normal(bb.np_count(N))
    D = bb.derivative(N)
    x0 = V.mean(0) + 0.1 * rng.standard_normal(3)
    h = 1e-30
    for i in range(3):
        coeff = sum(grad[m, i] * (D[m] @ a) for m in range(4))
        lam0 = Ainv @ np.concatenate([[1.0], x0])
        exact = bb.evaluate(coeff, N, lam0[None])[0]
        xc = x0.astype(complex)
        xc[i] += 1j * h
        lamc = Ainv @ np.concatenate([[1.0], xc])
        basis = np.array([bb.multinomial(al) * np.prod(lamc ** np.array(al)) for al in bb.multi_indices(N)])
        cs = (a @ basis).imag / h
        assert abs(exact - cs) < 1e-10 * max(1.0, abs(cs))


def test_derivative_sparsity():
    # each row of D^m has at most d+1 = 4 nonzeros (Sec. 4)
    for N in (2, 5):
        D = bb.derivative(N)
        assert np.max((np.abs(D) > 1e-9).sum(axis=2)) <= 4


# -- lift ---------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 3, 5])
def test_lift_defining_property(N):
    """int_T (L^f g) phi / |T| = int_f g phi / |f| for every phi in P^N."""
    rng = np.random.default_rng(N)
    lamT, wT = tet_rule(2 * N)
    lamF, wF = tri_rule(2 * N)
    Np = bb.np_count(N)
    L = bb.lift(N)
    for f in range(4):
        g = np.zeros(Np)
        nodes = [i for i, a in enumerate(bb.multi_indices(N)) if a[f] == 0]
        g[nodes] = rng.standard_normal(len(nodes))
        vol = bb.evaluate(np.eye(Np), N, lamT)                 # (Np, Q)
        lhs = (vol * wT) @ bb.evaluate(L[f] @ g, N, lamT)
        lam4 = np.zeros((len(wF), 4))
        lam4[:, list(FACE_VERTS[f])] = lamF
        fb = bb.evaluate(np.eye(Np), N, lam4)
        rhs = (fb * wF) @ bb.evaluate(g, N, lam4)
        assert np.allclose(lhs, rhs, atol=1e-12)


def test_lift_l0_sparsity():
    # L0 (the face block of the lift) has at most seven nonzeros per row (Sec. 4)
    for N in (3, 6):
        L = bb.lift(N)[0]
        nodes = [i for i, a in enumerate(bb.multi_indices(N)) if a[0] == 0]
        L0 = L[np.ix_(nodes, nodes)]
        assert np.max((np.abs(L0) > 1e-8 * np.abs(L0).max()).sum(axis=1)) == 7


# -- projection and WADG (Sec. 3.3, Sec. 5.3) --------------------------------

@pytest.mark.parametrize("N,M", [(2, 1), (4, 2), (3, 3)])
def test_projection_idempotent_and_orthogonal(N, M):
    P = bb.projection(N, M)
    assert np.allclose(P @ bb.elevation_chain(N + M, M), np.eye(bb.np_count(N)), atol=1e-10)
    rng = np.random.default_rng(3)
    h = rng.standard_normal(bb.np_count(N + M))
    lam, w = tet_rule(2 * (N + M))
    r = bb.evaluate(h, N + M, lam) - bb.evaluate(P @ h, N, lam)
    test = bb.evaluate(np.eye(bb.np_count(N)), N, lam)
    assert np.abs((test * w) @ r).max() < 1e-11


@pytest.mark.parametrize("N,M", [(2, 1), (3, 2), (4, 2)])
def test_wadg_matches_quadrature_wadg(N, M):
    """M^{-1} M_{c2} u equals P_q diag(c2(x_q)) V_q u (Eq. 7 with weight c^2)
    when c2 is a degree-M polynomial and the rule is exact to 2N+M."""
    rng = np.random.default_rng(N + 5 * M)
    c2 = rng.uniform(0.5, 2.0, bb.np_count(M))
    u = rng.standard_normal(bb.np_count(N))
    Mc2 = np.einsum("b,bij->ij", c2, bb.weighted_mass_terms(N, M))
    ours = np.linalg.solve(bb.mass(N), Mc2 @ u)
    lam, w = tet_rule(2 * N + M)
    Vq = bb.evaluate(np.eye(bb.np_count(N)), N, lam).T         # (Q, Np)
    Pq = np.linalg.solve(bb.mass(N), Vq.T * w)
    quad = Pq @ (bb.evaluate(c2, M, lam) * (Vq @ u))
    assert np.allclose(ours, quad, atol=1e-11)
    # and equals the projection of the product of Sec. 5.1
    assert np.allclose(ours, bb.projection(N, M) @ bb.product(u, N, c2, M), atol=1e-10)


# -- time integrator ----------------------------------------------------------

def test_lsrk_stability_polynomial():
    R = stability_polynomial()
    want = [1, 1, Fraction(1, 2), Fraction(1, 6), Fraction(1, 24), Fraction(1, 200)]
    assert len(R) == 6
    for r, w in zip(R, want):
        assert abs(float(r - w)) < 1e-12


def test_lsrk_stage_times():
    c = lsrk_stage_times()
    assert c[0] == 0 and c[1] == LSRK_B[0]
    assert all(0 < float(x) < 1 for x in c[1:])
    # the stage times quoted with the published scheme agree to ~1e-7
    quoted = [0.0, 0.1496590219993, 0.3704009573644, 0.6222557631345, 0.9582821306748]
    assert np.allclose([float(x) for x in c], quoted, atol=2e-7)


# -- mesh -----------------------------------------------------------------------

def test_cube_mesh_connectivity():
    vxyz, etov = inputs.cube_mesh(3, shuffle=True, seed=2)
    etoe, etof = connectivity(etov)
    K = len(etov)
    assert K == 162
    walls = (etoe < 0).sum()
    assert walls == 6 * 9 * 2                                # 2 triangles per boundary square
    for e in range(K):
        for f in range(4):
            nb = etoe[e, f]
            if nb >= 0:
                assert etoe[nb, etof[e, f]] == e and etof[nb, etof[e, f]] == f
    geo = geometry(vxyz, etov)
    assert np.all(geo["vol"] > 0) and abs(geo["vol"].sum() - 1.0) < 1e-12
    # outward normals: n_f = -grad lambda_f / |grad lambda_f| and A_f/V = 3 |grad lambda_f|
    gn = np.linalg.norm(geo["grad"], axis=2)
    assert np.allclose(geo["normal"], -geo["grad"] / gn[..., None], atol=1e-12)
    assert np.allclose(geo["area"] / geo["vol"][:, None], 3 * gn, rtol=1e-12)


# -- assembled semi-discrete operator (brute force on small meshes) ---------

def _energy_matrix(orc):
    """Block-diagonal H with E(q) = q^T H q (the oracle's energy)."""
    K, Np = orc.K, orc.Np
    H = np.zeros((4 * K * Np, 4 * K * Np))
    for e in range(K):
        Mc2 = np.einsum("b,bij->ij", orc.c2[e], orc.T)
        Hp = orc.Mhat @ np.linalg.solve(Mc2, orc.Mhat) * orc.geo["vol"][e]
        sl = slice(e * Np, (e + 1) * Np)
        H[sl, sl] = Hp
        for fld in range(1, 4):
            o = fld * K * Np
            H[o + e * Np:o + (e + 1) * Np, o + e * Np:o + (e + 1) * Np] = orc.Mhat * orc.geo["vol"][e]
    return H


def _assemble(orc):
    n = 4 * orc.K * orc.Np
    A = np.empty((n, n))
    for c in range(n):
        q = np.zeros(n)
        q[c] = 1.0
        A[:, c] = orc.rhs(q.reshape(4, orc.K, orc.Np)).ravel()
    return A


@pytest.mark.parametrize("tau", [0.0, 1.0])
def test_assembled_operator_energy_stability(tau):
    """Eq. (2) with penalty fluxes: H A + A^T H = 0 for tau = 0, <= 0 for tau > 0."""
    vxyz, etov = inputs.cube_mesh(1, jitter=0.0, shuffle=True, seed=4)
    rng = np.random.default_rng(0)
    N, M = 2, 1
    c2 = rng.uniform(0.7, 1.6, (len(etov), bb.np_count(M)))
    orc = AcousticOracle(vxyz, etov, N, M, c2, tau_p=tau, tau_u=tau)
    A = _assemble(orc)
    H = _energy_matrix(orc)
    S = H @ A + A.T @ H
    scale = np.abs(H @ A).max()
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    if tau == 0.0:
        assert np.abs(S).max() < 1e-10 * scale
    else:
        assert ev.max() < 1e-10 * scale and ev.min() < -1e-3 * scale


def test_constant_state_is_steady_without_walls_effect():
    # u constant, p = 0 has zero rhs in the interior and on mirror walls
    vxyz, etov = inputs.cube_mesh(2, shuffle=True, seed=1)
    K = len(etov)
    orc = AcousticOracle(vxyz, etov, 3, 1, np.ones((K, 4)))
    q = np.zeros((4, K, orc.Np))
    q[1] = 0.3
    q[2] = -1.1
    q[3] = 0.25
    assert np.abs(orc.rhs(q)).max() < 1e-11


@pytest.mark.slow
def test_standing_wave_converges():
    """c2 = 1, p = 0 walls: p = sin(pi x) sin(pi y) sin(pi z) cos(sqrt(3) pi t)."""
    from oracle.quadrature import tet_rule as rule
    errs = []
    for n in (2, 4):
        vxyz, etov = inputs.cube_mesh(n)
        K = len(etov)
        N = 3
        orc = AcousticOracle(vxyz, etov, N, 0, np.ones((K, 1)))
        lam, w = rule(2 * N + 4)
        X = np.asarray(vxyz)[etov]
        xq = np.einsum("qa,kai->kqi", lam, X)
        Vq = bb.evaluate(np.eye(orc.Np), N, lam)               # (Np, Q)
        Pq = np.linalg.solve(bb.mass(N), Vq * w)              # (Np, Q)

        def proj(f):
            return np.einsum("aq,kq->ka", Pq, f(xq))

        s = np.sin(np.pi * xq)
        c = np.cos(np.pi * xq)
        q0 = np.zeros((4, K, orc.Np))
        q0[0] = proj(lambda x: np.prod(np.sin(np.pi * x), axis=-1))
        T = 0.1
        dt, ns = orc.dt_for(T, 0.25)
        q, _ = orc.run(q0, dt, ns)
        w3 = np.sqrt(3) * np.pi
        pex = s[..., 0] * s[..., 1] * s[..., 2] * np.cos(w3 * T)
        uex = -np.pi * np.stack([c[..., 0] * s[..., 1] * s[..., 2],
                                 s[..., 0] * c[..., 1] * s[..., 2],
                                 s[..., 0] * s[..., 1] * c[..., 2]]) * np.sin(w3 * T) / w3
        ph = np.einsum("aq,ka->kq", Vq, q[0])
        uh = np.einsum("aq,ika->ikq", Vq, q[1:4])
        vol = orc.geo["vol"][:, None]
        err = np.sqrt(np.sum(vol * w * ((ph - pex) ** 2 + np.sum((uh - uex) ** 2, axis=0))))
        errs.append(err)
    rate = np.log2(errs[0] / errs[1])
    # rate -> N + 1 = 4; 3.6 is observed on 2^3 -> 4^3 hexes
    assert errs[1] < 1e-3 and rate > 3.3


# -- sources and energy -----------------------------------------------------------

def test_point_source_vector_reproduces_point_values():
    """M^{-1} B(x_s)/|T| tested against any phi in P^N integrates to phi(x_s)."""
    vxyz, etov = inputs.cube_mesh(1, jitter=0.0, shuffle=True, seed=6)
    N = 4
    orc = AcousticOracle(vxyz, etov, N, 0, np.ones((len(etov), 1)))
    xs = np.array([0.31, 0.62, 0.44])
    e, vec = orc.set_point_source(xs, [1.0])
    lam_s = geometry(vxyz, etov)["grad"][e] @ (xs - vxyz[etov[e, 0]]) + np.array([1.0, 0, 0, 0])
    assert np.all(lam_s >= -1e-12)
    lam, w = tet_rule(2 * N)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(orc.Np)
    integral = orc.geo["vol"][e] * np.sum(w * bb.evaluate(vec, N, lam) * bb.evaluate(phi, N, lam))
    assert abs(integral - bb.evaluate(phi, N, lam_s[None])[0]) < 1e-10


def test_ricker_closed_form():
    from oracle.acoustic import ricker
    f0, t0 = 10.0, 0.1
    assert ricker(t0, f0, t0) == 1.0
    tz = t0 + 1.0 / (np.pi * f0 * np.sqrt(2.0))   # zero crossing of (1 - 2a)
    assert abs(ricker(tz, f0, t0)) < 1e-15
    # one period of pi f0 away from the peak: a = 1, so r = (1 - 2) e^{-1}
    for tm in (t0 - 1.0 / (np.pi * f0), t0 + 1.0 / (np.pi * f0)):
        assert abs(ricker(tm, f0, t0) + np.exp(-1.0)) < 1e-15


def test_energy_conserved_without_penalty():
    """tau = 0: the semi-discrete energy is conserved; RK4 drifts by O(dt^4)."""
    vxyz, etov = inputs.cube_mesh(1, jitter=0.1, shuffle=True, seed=2)
    K = len(etov)
    rng = np.random.default_rng(1)
    orc = AcousticOracle(vxyz, etov, 2, 1, rng.uniform(0.7, 1.5, (K, 4)), tau_p=0.0, tau_u=0.0)
    q = rng.standard_normal((4, K, orc.Np))
    e0 = orc.energy(q)
    dt = 0.2 * orc.dt_for(1.0, 0.5)[0]
    q1, _ = orc.run(q, dt, 20)
    assert abs(orc.energy(q1) - e0) < 1e-6 * e0
    orc1 = AcousticOracle(vxyz, etov, 2, 1, orc.c2, tau_p=1.0, tau_u=1.0)
    q2, _ = orc1.run(q, dt, 20)
    assert orc1.energy(q2) < 0.99 * e0
