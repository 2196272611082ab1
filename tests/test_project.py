"""The L2 projection tools (tools layer, host only): exactness on polynomials,
orthogonality of the residual (checked with the oracle's own quadrature),
and the positivity check of projected c^2."""
import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.quadrature import tet_rule as oracle_tet_rule
from paper_1808_08645_gb300 import inputs
from paper_1808_08645_gb300 import project as pj


def _poly(deg, seed):
    rng = np.random.default_rng(seed)
    terms = [(i, j, k, rng.standard_normal()) for i in range(deg + 1) for j in range(deg + 1 - i)
             for k in range(deg + 1 - i - j)]

    def f(x):
        return sum(c * x[:, 0] ** i * x[:, 1] ** j * x[:, 2] ** k for i, j, k, c in terms)
    return f


def test_rule_integrates_monomials_exactly():
    lam, w = pj.tet_rule(4)  # exact to degree 7
    assert abs(w.sum() - 1.0) < 1e-14
    from math import factorial
    for g in [(7, 0, 0, 0), (2, 2, 2, 1), (0, 3, 1, 3), (1, 1, 1, 1)]:
        want = 6.0 * np.prod([factorial(x) for x in g]) / factorial(sum(g) + 3)
        assert abs(np.sum(w * np.prod(lam ** np.array(g), axis=1)) - want) < 1e-14 * max(want, 1e-3)


@pytest.mark.parametrize("n", [1, 3, 5])
def test_projection_reproduces_polynomials(n):
    vxyz, etov = inputs.cube_mesh(2, jitter=0.15, shuffle=True, seed=n)
    f = _poly(n, n)
    c = pj.l2_project(vxyz, etov, n, f)
    rng = np.random.default_rng(0)
    for e in range(0, len(etov), 7):
        lam = rng.dirichlet(np.ones(4), 5)
        x = lam @ vxyz[etov[e]]
        assert np.allclose(bb.evaluate(c[e], n, lam), f(x), atol=1e-11)


def test_projection_residual_is_orthogonal():
    """int (f - P f) B_alpha = 0 on every element, with a smooth non-polynomial
    f, checked by the oracle's quadrature (a different rule)."""
    n = 3
    vxyz, etov = inputs.cube_mesh(1, jitter=0.1, shuffle=True, seed=2)
    f = inputs.gaussian_pulse((0.4, 0.5, 0.6), 0.3)
    c = pj.l2_project(vxyz, etov, n, f, q=20)
    lam, w = oracle_tet_rule(24)
    for e in range(len(etov)):
        x = lam @ vxyz[etov[e]]
        Bv = bb.evaluate(np.eye(bb.np_count(n)), n, lam)  # [Np, P]
        r = f(x) - bb.evaluate(c[e], n, lam)
        assert np.abs(Bv @ (w * r)).max() < 1e-9


def test_project_c2_rejects_non_positive_coefficients():
    vxyz, etov = inputs.cube_mesh(2)
    c2 = pj.project_c2(vxyz, etov, 1, inputs.c2_config_small)
    assert (c2 > 0).all()
    with pytest.raises(pj.NonPositiveC2):
        pj.project_c2(vxyz, etov, 2, lambda x: np.where(x[:, 0] + 0.3 * x[:, 1] > 0.55, 1.0, 1e-3) - 0.2)
