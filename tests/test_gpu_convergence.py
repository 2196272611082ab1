"""Convergence of the GPU solver (FP64, through the C ABI) on the
heterogeneous manufactured solution of the paper's convergence study
(Sec. 6.1), on meshes too large for the oracle: 4^3, 8^3 and 16^3 hexes
(384 to 24,576 tets). Same problem as tests/test_oracle_convergence.py:
c^2 = 1 + sin sin sin / 2 L2-projected onto P^M (the tools layer), the
forcing (3 - 1/c^2) pi sin sin sin(x) sin(pi t) through bbw_set_forcing,
p = 0 walls, exact p = sin sin sin(x) cos(pi t).

Expected (the paper's observation): rate N + 1 for M >= 1; M = 0 limits the
rate to 2.
"""
import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.quadrature import tet_rule as rule
from paper_1808_08645_gb300 import binding as B
from paper_1808_08645_gb300 import inputs
from paper_1808_08645_gb300 import project

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_08645_gb300 import build
    build.build()


def _error(hexes: int, N: int, M: int, T: float = 0.2, cfl: float = 0.25) -> float:
    vxyz, etov = inputs.cube_mesh(hexes)
    K = len(etov)
    c2f = inputs.c2_config_small
    c2 = project.project_c2(vxyz, etov, M, c2f)
    g = project.l2_project(vxyz, etov, N, inputs.manufactured_forcing(c2f))
    sss = lambda x: np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])
    q0 = np.zeros((4, K, bb.np_count(N)))
    q0[0] = project.l2_project(vxyz, etov, N, sss)
    s = B.Solver(vxyz, etov, N, M, B.F64)
    s.set_c2(c2)
    s.set_state(q0)
    dt0 = s.cfl_dt(cfl)
    nsteps = int(np.ceil(T / dt0))
    dt = T / nsteps
    cs = B.lsrk_coeffs()[2]
    amp = [np.sin(np.pi * (k // 5 + cs[k % 5]) * dt) for k in range(5 * nsteps)]
    s.set_forcing(np.arange(K), g, amp)
    s.step(dt, nsteps)
    q, t = s.get_state()
    s.close()
    assert abs(t - T) < 1e-12
    # L2 error by quadrature (the oracle's rule, exact to degree 2N + 4 in the polynomial part)
    lam, w = rule(2 * N + 4)
    xq = np.einsum("qa,kai->kqi", lam, np.asarray(vxyz)[etov])
    Vq = bb.evaluate(np.eye(bb.np_count(N)), N, lam)
    sn, cn = np.sin(np.pi * xq), np.cos(np.pi * xq)
    pex = sn[..., 0] * sn[..., 1] * sn[..., 2] * np.cos(np.pi * T)
    uex = -np.stack([cn[..., 0] * sn[..., 1] * sn[..., 2], sn[..., 0] * cn[..., 1] * sn[..., 2],
                     sn[..., 0] * sn[..., 1] * cn[..., 2]]) * np.sin(np.pi * T)
    ph = np.einsum("aq,ka->kq", Vq, q[0])
    uh = np.einsum("aq,ika->ikq", Vq, q[1:4])
    vol = np.abs(np.linalg.det(np.asarray(vxyz)[etov][:, 1:] - np.asarray(vxyz)[etov][:, :1])) / 6.0
    return float(np.sqrt(np.sum(vol[:, None] * w * ((ph - pex) ** 2 + np.sum((uh - uex) ** 2, axis=0)))))


def test_rate_N_plus_1_for_linear_and_quadratic_c2():
    for N, M in ((3, 1), (3, 2), (2, 1)):
        e = [_error(h, N, M) for h in (4, 8, 16)]
        rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        print(f"N={N} M={M} errors {e} rates {rates}")
        assert rates[-1] > N + 1 - 0.35, (N, M, e, rates)


def test_piecewise_constant_c2_limits_the_rate_to_two():
    e = [_error(h, 3, 0) for h in (4, 8, 16)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    print(f"N=3 M=0 errors {e} rates {rates}")
    assert abs(rates[-1] - 2.0) < 0.3, (e, rates)
