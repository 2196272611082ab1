"""Pins of the CFL time-step rule (oracle ``cfl_dt``) that do not restate it.

The paper gives no step-size rule (Sec. 6.3.1 only names the RK scheme), so
the library's rule dt = CFL / (sqrt(max c2) (N+1)(N+3)/3 max_{k,f} |f|/|D^k|)
is pinned three ways:

* geometry worked out by hand: a Kuhn tetrahedron of a hexahedron of side h
  has two right-angle faces of area h^2/2 and two faces of area h^2 sqrt(2)/2,
  and volume h^3/6, so max |f|/|D| = 3 sqrt(2) / h on an n^3-hex unit cube;
* linear stability: every eigenvalue z of the assembled semi-discrete
  operator (Eq. 2 with penalty fluxes and the weight-adjusted mass of Eq. 4)
  satisfies |R(dt z)| <= 1 for the RK stability polynomial R, while 8 dt is
  unstable (so the rule is not vacuous);
* energy: with tau = 1 the weight-adjusted energy does not grow over 200 CFL
  steps for every N = 1..9, and grows without bound at 8 dt.
"""
from math import sqrt

import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.acoustic import AcousticOracle, cfl_dt, stability_polynomial
from oracle.mesh import geometry
from paper_1808_08645_gb300 import inputs

_R = [float(c) for c in stability_polynomial()]


def _stab(z):
    return sum(c * z ** i for i, c in enumerate(_R))


def _assemble(orc):
    n = 4 * orc.K * orc.Np
    A = np.empty((n, n))
    for c in range(n):
        q = np.zeros(n)
        q[c] = 1.0
        A[:, c] = orc.rhs(q.reshape(4, orc.K, orc.Np)).ravel()
    return A


@pytest.mark.parametrize("hexes", [1, 2])
def test_face_to_volume_ratio_of_kuhn_cubes(hexes):
    vxyz, etov = inputs.cube_mesh(hexes)
    geo = geometry(vxyz, etov)
    h = 1.0 / hexes
    assert np.allclose(geo["vol"], h ** 3 / 6.0, rtol=0, atol=1e-15)
    areas = np.sort(geo["area"], axis=1)
    want = np.array([0.5, 0.5, sqrt(2) / 2, sqrt(2) / 2]) * h * h
    assert np.allclose(areas, want[None, :], rtol=0, atol=1e-15)
    ratio = np.max(geo["area"] / geo["vol"][:, None])
    assert abs(ratio - 3.0 * sqrt(2.0) * hexes) < 1e-12


@pytest.mark.parametrize("hexes,N,cfl", [(1, 1, 0.5), (2, 3, 0.5), (2, 9, 0.25)])
def test_cfl_dt_hand_values(hexes, N, cfl):
    vxyz, etov = inputs.cube_mesh(hexes)
    K = len(etov)
    geo = geometry(vxyz, etov)
    # c2 = 4 everywhere except one coefficient of one element (its maximum 9)
    c2 = np.full((K, 4), 4.0)
    c2[K // 2, 2] = 9.0
    cn = (N + 1) * (N + 3) / 3.0
    want = cfl / (3.0 * cn * 3.0 * sqrt(2.0) * hexes)
    assert abs(cfl_dt(geo, c2, N, cfl) - want) < 1e-15 * want
    # constant c2 = 4: sqrt gives 2
    c2[:] = 4.0
    want = cfl / (2.0 * cn * 3.0 * sqrt(2.0) * hexes)
    assert abs(cfl_dt(geo, c2, N, cfl) - want) < 1e-15 * want


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_cfl_dt_is_linearly_stable(N):
    vxyz, etov = inputs.cube_mesh(1, jitter=0.15, shuffle=True, seed=3)
    rng = np.random.default_rng(N)
    M = 2
    c2 = rng.uniform(0.5, 2.0, (len(etov), bb.np_count(M)))
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    ev = np.linalg.eigvals(_assemble(orc))
    assert ev.real.max() < 1e-9 * np.abs(ev).max()   # dissipative semi-discretisation
    dt = cfl_dt(orc.geo, orc.c2, N, 0.5)
    assert np.abs(_stab(dt * ev)).max() <= 1.0 + 1e-9
    assert np.abs(_stab(8.0 * dt * ev)).max() > 1.01


@pytest.mark.parametrize("N", list(range(1, 10)))
def test_energy_does_not_grow_at_cfl_dt(N):
    vxyz, etov = inputs.cube_mesh(1, jitter=0.15, shuffle=True, seed=5)
    K = len(etov)
    rng = np.random.default_rng(10 + N)
    M = 2
    c2 = rng.uniform(0.5, 2.0, (K, bb.np_count(M)))
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    q0 = rng.standard_normal((4, K, orc.Np))
    dt = cfl_dt(orc.geo, orc.c2, N, 0.5)
    e_prev = orc.energy(q0)
    q, res = q0, np.zeros_like(q0)
    for i in range(200):
        q, res = orc.step(q, res, dt, i * dt)
        if i % 20 == 19:
            e = orc.energy(q)
            assert e <= e_prev * (1 + 1e-12)
            e_prev = e
    # eight times the step: the energy explodes
    q, res = q0, np.zeros_like(q0)
    for i in range(60):
        q, res = orc.step(q, res, 8.0 * dt, i * dt)
    assert orc.energy(q) > 1e3 * orc.energy(q0)
