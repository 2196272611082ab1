"""GPU parity of the elastic stage kernel (bbw_elastic_* through the C ABI)
against the FP64 elastic oracle: every degree in both precisions, media of
every degree, penalties, padded groups, the final time of a short run, the
full-size throughput mesh (sampled), the acoustic limit (mu = 0) against the
acoustic kernel, energy decay, device-resident state transfers, advance(),
and the error paths."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import bernstein as bb
from oracle.elastic import ElasticOracle
from paper_1808_08645_gb300 import binding as B
from paper_1808_08645_gb300 import inputs
from parity_util import TOL_FINAL, TOL_STAGE, rel_l2, rounded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_08645_gb300 import build
    build.build()
    torch.cuda.init()


def _case(hexes, N, M, prec, seed=0, jitter=0.15, shuffle=True):
    vxyz, etov = inputs.cube_mesh(hexes, jitter=jitter, shuffle=shuffle, seed=seed)
    rng = np.random.default_rng(seed + 1000 * N + 100 * M)
    K, Np, Mp = len(etov), bb.np_count(N), bb.np_count(M)
    media = (rounded(rng.uniform(0.5, 1.5, (K, Mp)), prec), rounded(rng.uniform(0.5, 2.0, (K, Mp)), prec),
             rounded(rng.uniform(0.3, 1.2, (K, Mp)), prec))
    q = rounded(rng.standard_normal((9, K, Np)), prec)
    res = rounded(rng.standard_normal((9, K, Np)), prec)
    return vxyz, etov, media, q, res


def _solver(vxyz, etov, N, M, prec, media, q, res, tau=(1.0, 1.0)):
    s = B.ElasticSolver(vxyz, etov, N, M, prec)
    s.set_media(*media)
    s.set_params(*tau)
    s.set_state(q, res)
    return s


def _oracle(vxyz, etov, N, M, media, tau=(1.0, 1.0)):
    return ElasticOracle(vxyz, etov, N, M, *media, tau_v=tau[0], tau_s=tau[1])


def _stage_check(vxyz, etov, N, M, prec, media, q, res, s, dt, tau=(1.0, 1.0)):
    g = _solver(vxyz, etov, N, M, prec, media, q, res, tau)
    g.stage(s, dt)
    qg, rg, _ = g.get_state(with_res=True)
    g.close()
    qo, ro = _oracle(vxyz, etov, N, M, media, tau).stage(q, res, s, dt)
    return rel_l2(rg, ro), rel_l2(qg, qo)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("N", range(1, 10))
def test_elastic_stage_parity_all_degrees(N, prec):
    M = 2
    vxyz, etov, media, q, res = _case(1, N, M, prec, seed=N)
    er, eq = _stage_check(vxyz, etov, N, M, prec, media, q, res, N % 5, 1e-3)
    assert er <= TOL_STAGE[prec] and eq <= TOL_STAGE[prec], (er, eq)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("M", [0, 1, 3])
def test_elastic_stage_parity_media_degrees(M, prec):
    N = 4
    vxyz, etov, media, q, res = _case(1, N, M, prec, seed=20 + M)
    er, eq = _stage_check(vxyz, etov, N, M, prec, media, q, res, 1, 2e-3)
    assert er <= TOL_STAGE[prec] and eq <= TOL_STAGE[prec], (er, eq)


@pytest.mark.parametrize("tau", [(0.0, 0.0), (0.5, 2.0)])
def test_elastic_stage_parity_penalties(tau):
    N, M, prec = 5, 1, 64
    vxyz, etov, media, q, res = _case(1, N, M, prec, seed=7)
    er, eq = _stage_check(vxyz, etov, N, M, prec, media, q, res, 2, 1e-3, tau)
    assert er <= TOL_STAGE[prec] and eq <= TOL_STAGE[prec], (er, eq)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("N", [1, 3, 5, 8])
def test_elastic_padded_groups(N, prec):
    """K = 1 and K = 5: the last group of V elements is padded."""
    M = 2
    vxyz, etov, media, q, res = _case(1, N, M, prec, seed=30 + N)
    for K in (1, 5):
        sub = etov[:K]
        verts, inv = np.unique(sub, return_inverse=True)
        ev, vx = inv.reshape(sub.shape), vxyz[verts]
        md = tuple(m[:K] for m in media)
        er, eq = _stage_check(vx, ev, N, M, prec, md, q[:, :K], res[:, :K], 3, 1e-3)
        assert er <= TOL_STAGE[prec] and eq <= TOL_STAGE[prec], (K, er, eq)


@pytest.mark.parametrize("prec", [32, 64])
def test_elastic_final_time_parity(prec):
    """2^3 x 6 tets, N = 3, M = 1, heterogeneous media, Gaussian pulse, 10
    steps at the CFL step."""
    N, M = 3, 1
    vxyz, etov = inputs.cube_mesh(2, jitter=0.1, shuffle=True, seed=3)
    media = tuple(rounded(x, prec) for x in inputs.elastic_media(vxyz, etov, M, seed=2))
    q0 = rounded(inputs.elastic_pulse(vxyz, etov, N, width=0.25), prec)
    g = _solver(vxyz, etov, N, M, prec, media, q0, None)
    dt = g.cfl_dt(0.5)
    g.step(dt, 10)
    qg, t = g.get_state()
    assert abs(t - 10 * dt) < 1e-12
    g.close()
    qo, _ = _oracle(vxyz, etov, N, M, media).run(q0, dt, 10)
    assert rel_l2(qg, qo) <= TOL_FINAL[prec]
    assert np.abs(qo).max() > 1e-3  # the pulse has not decayed away


def _patch(etoe, e):
    out = [int(e)]
    for nb in etoe[e]:
        if nb >= 0 and int(nb) not in out:
            out.append(int(nb))
    return out


@pytest.mark.parametrize("N", [1, 5, 9])
def test_elastic_full_size_sampled(N):
    """196,608 tets (the elastic throughput workload) in the bench's launch
    shape: one stage on the GPU, sampled elements checked against the oracle
    on the sub-mesh of the element and its face neighbours (an element's
    right-hand side depends on nothing else)."""
    cfg = inputs.ELASTIC_CONFIG
    M, prec = cfg["M"], 32
    vxyz, etov = inputs.cube_mesh(cfg["hexes"])
    K, Np = len(etov), bb.np_count(N)
    media = tuple(rounded(x, prec) for x in inputs.elastic_media(vxyz, etov, M, seed=cfg["seed"]))
    rng = np.random.default_rng(N)
    q = rounded(rng.standard_normal((9, K, Np)), prec)
    res = rounded(rng.standard_normal((9, K, Np)), prec)
    g = _solver(vxyz, etov, N, M, prec, media, q, res)
    g.stage(2, 1e-4)
    qg, rg, _ = g.get_state(with_res=True)
    g.close()
    etoe = B.mesh_analyze(vxyz, etov, N)["etoe"]
    sample = sorted(set([0, K - 1] + list(rng.choice(K, 16, replace=False))))
    got, want = [], []
    for e in sample:
        els = _patch(etoe, e)
        sub = np.asarray(etov)[els]
        verts, inv = np.unique(sub, return_inverse=True)
        orc = _oracle(np.asarray(vxyz)[verts], inv.reshape(sub.shape), N, M, tuple(m[els] for m in media))
        qo, ro = orc.stage(q[:, els], res[:, els], 2, 1e-4)
        got.append(rg[:, e])
        want.append(ro[:, 0])
    assert rel_l2(np.array(got), np.array(want)) <= TOL_STAGE[prec]


@pytest.mark.parametrize("prec", [32, 64])
def test_elastic_acoustic_limit_matches_the_acoustic_kernel(prec):
    """mu = 0, rho = 1, lambda = c^2, tau_v = 0, sigma = -p I: the elastic
    stage must reproduce the acoustic stage (tau_u = 0, tau_p = tau_s)."""
    N, M = 4, 1
    vxyz, etov = inputs.cube_mesh(2, jitter=0.1, shuffle=True, seed=8)
    K, Np, Mp = len(etov), bb.np_count(N), bb.np_count(M)
    rng = np.random.default_rng(5)
    c2 = rounded(rng.uniform(0.5, 2.0, (K, Mp)), prec)
    qa = rounded(rng.standard_normal((4, K, Np)), prec)
    ra = rounded(rng.standard_normal((4, K, Np)), prec)
    a = B.Solver(vxyz, etov, N, M, prec)
    a.set_c2(c2)
    a.set_params(0.8, 0.0)
    a.set_state(qa, ra)
    a.stage(3, 1e-3)
    qa1, ra1, _ = a.get_state(with_res=True)
    a.close()
    qe = np.zeros((9, K, Np))
    re = np.zeros((9, K, Np))
    qe[:3], re[:3] = qa[1:], ra[1:]
    qe[3:6], re[3:6] = -qa[0], -ra[0]
    e = _solver(vxyz, etov, N, M, prec, (np.ones_like(c2), c2, np.zeros_like(c2)), qe, re, tau=(0.0, 0.8))
    e.stage(3, 1e-3)
    qe1, re1, _ = e.get_state(with_res=True)
    e.close()
    tol = TOL_STAGE[prec]
    assert rel_l2(re1[:3], ra1[1:]) <= tol and rel_l2(qe1[:3], qa1[1:]) <= tol
    for k in range(3):
        assert rel_l2(-re1[3 + k], ra1[0]) <= tol and rel_l2(-qe1[3 + k], qa1[0]) <= tol
    assert np.abs(re1[6:]).max() <= tol * np.abs(ra1).max()


def test_elastic_energy_decays_on_the_gpu():
    """FP64, tau = 1: the weight-adjusted energy of the GPU states decreases
    step by step (energy stability, Sec. 2.2)."""
    N, M = 2, 1
    vxyz, etov, media, q, _ = _case(1, N, M, 64, seed=12)
    orc = _oracle(vxyz, etov, N, M, media)
    g = _solver(vxyz, etov, N, M, 64, media, q, None)
    e = [orc.energy(q)]
    for _ in range(4):
        g.step(2e-3, 1)
        e.append(orc.energy(g.get_state()[0]))
    g.close()
    assert all(b < a for a, b in zip(e, e[1:]))


def test_elastic_state_roundtrip_and_time():
    N, M = 6, 2
    vxyz, etov, media, q, res = _case(1, N, M, 64, seed=13)
    g = _solver(vxyz, etov, N, M, 64, media, q, res)
    q2, r2, t = g.get_state(with_res=True)
    assert np.array_equal(q2, q) and np.array_equal(r2, res) and t == 0.0
    g.step(1e-3, 2)
    t, n = g.time()
    assert abs(t - 2e-3) < 1e-15 and n == 10
    g.close()


def test_elastic_rejects_bad_media_and_reports_nonfinite():
    N, M = 2, 1
    vxyz, etov, media, q, res = _case(1, N, M, 32, seed=14)
    g = _solver(vxyz, etov, N, M, 32, media, q, res)
    bad = media[0].copy()
    bad[0, 0] = 0.0
    with pytest.raises(B.BBWError, match="BBW_ERR_NONPOS_C2"):
        g.set_media(bad, media[1], media[2])
    neg = media[2].copy()
    neg[1, 1] = -0.1
    with pytest.raises(B.BBWError, match="BBW_ERR_NONPOS_C2"):
        g.set_media(media[0], media[1], neg)
    with pytest.raises(B.BBWError, match="BBW_ERR_ARG"):
        g.stage(5, 1e-3)
    q2 = q.copy()
    q2[4, 3, 1] = np.inf
    g.set_state(q2)
    g.stage(0, 1e-3)
    with pytest.raises(B.BBWError, match="BBW_ERR_NONFINITE"):
        g.sync()
    g.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_elastic_device_state_roundtrip_and_advance(prec):
    """set_state_device / get_state_device with torch tensors of either
    dtype, then advance(): same result as the host path."""
    N, M = 4, 2
    vxyz, etov, media, q, res = _case(1, N, M, prec, seed=15)
    K, Np = len(etov), bb.np_count(N)
    g = _solver(vxyz, etov, N, M, prec, media, q, res)
    dev = torch.device("cuda")
    for dt_ in (B.F32, B.F64):
        tq = torch.tensor(q, dtype=torch.float32 if dt_ == B.F32 else torch.float64, device=dev)
        tr = torch.tensor(res, dtype=tq.dtype, device=dev)
        g.set_state_device(tq, tr, dtype=dt_, t=0.25)
        oq, orr = torch.empty_like(tq), torch.empty_like(tr)
        g.get_state_device(oq, orr, dtype=dt_)
        g.sync()
        want_q = q.astype(np.float32) if dt_ == B.F32 else q
        assert np.array_equal(oq.cpu().numpy(), want_q)
        assert g.time()[0] == 0.25
    g.set_state(q)
    dt, n = g.advance(0.01, 0.5)
    assert n >= 1 and abs(dt * n - 0.01) < 1e-15
    qa, t = g.get_state()
    g.set_state(q)
    g.step(dt, n)
    qb, _ = g.get_state()
    assert np.array_equal(qa, qb) and abs(t - 0.01) < 1e-12
    g.close()

