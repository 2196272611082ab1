"""GPU parity of the fused BBWADG stage against the FP64 oracle (needs a GB300).

Every test calls the CUDA path through the C ABI (binding.Solver /
binding.wadg_update) and compares element by element with the oracle on the
same seeded inputs: per stage relative L2 <= 1e-5 in FP32 (1e-11 in FP64),
final time <= 1e-4 (1e-10). Meshes span several CTA tiles with a ragged tail.
"""
import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.acoustic import AcousticOracle
from paper_1808_08645_gb300 import binding as B
from paper_1808_08645_gb300 import inputs
from paper_1808_08645_gb300 import project

from parity_util import (TOL_FINAL, TOL_STAGE, oracle_stage_on_patch, random_case,
                         rel_l2, rounded, stage_times)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_08645_gb300 import build
    build.build()
    torch.cuda.init()


def _solver(vxyz, etov, N, M, prec, c2, q, res, t=0.0):
    s = B.Solver(vxyz, etov, N, M, prec)
    s.set_c2(c2)
    s.set_state(q, res, t)
    return s


# -- the weight-adjusted update alone -----------------------------------------

@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("N", range(1, 10))
@pytest.mark.parametrize("M", [0, 1, 2, 3])
def test_wadg_update_parity(N, M, prec):
    """out = P^{N+M}_N(c2 * r) equals the oracle's M^{-1} M_{c2} r."""
    rng = np.random.default_rng(N * 7 + M)
    K = 37  # several tiles at every N, ragged tail
    Np, Mp = bb.np_count(N), bb.np_count(M)
    r = rounded(rng.standard_normal((K, Np)), prec)
    c2 = rounded(rng.uniform(0.5, 2.0, (K, Mp)), prec)
    T = bb.weighted_mass_terms(N, M)
    want = np.linalg.solve(bb.mass(N), np.einsum("kb,bij,kj->ki", c2, T, r).T).T
    dt = torch.float32 if prec == 32 else torch.float64
    dr = torch.tensor(r, dtype=dt, device="cuda")
    dc = torch.tensor(c2, dtype=dt, device="cuda")
    out = torch.full_like(dr, float("nan"))
    B.wadg_update(N, M, prec, K, dr, dc, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    assert rel_l2(got, want) <= TOL_STAGE[prec]


def test_wadg_update_empty_is_noop():
    B.wadg_update(3, 2, 32, 0, 0, 0, 0)


# -- one stage ------------------------------------------------------------------

@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("N", range(1, 10))
def test_stage_parity_all_degrees(N, prec):
    M = 2
    vxyz, etov, c2, q, res = random_case(3 if N <= 6 else 2, N, M, prec, seed=N)
    dt, t = 1e-3, 0.37
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    for s in (0, 3):
        solver = _solver(vxyz, etov, N, M, prec, c2, q, res, t)
        solver.stage(s, dt)
        qg, rg, _ = solver.get_state(with_res=True)
        qo, ro = orc.stage(q, res, s, dt)
        assert rel_l2(rg, ro) <= TOL_STAGE[prec], (s, rel_l2(rg, ro))
        assert rel_l2(qg, qo) <= TOL_STAGE[prec]
        solver.close()


@pytest.mark.parametrize("M", [0, 1, 3])
def test_stage_parity_other_weight_degrees(M):
    N, prec = 4, 32
    vxyz, etov, c2, q, res = random_case(2, N, M, prec, seed=11)
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    solver = _solver(vxyz, etov, N, M, prec, c2, q, res)
    solver.stage(2, 2e-3)
    qg, rg, _ = solver.get_state(with_res=True)
    qo, ro = orc.stage(q, res, 2, 2e-3)
    assert rel_l2(rg, ro) <= TOL_STAGE[prec]


@pytest.mark.parametrize("tau", [(0.0, 0.0), (0.5, 2.0)])
def test_stage_parity_penalties(tau):
    N, M, prec = 3, 2, 64
    vxyz, etov, c2, q, res = random_case(2, N, M, prec, seed=5)
    orc = AcousticOracle(vxyz, etov, N, M, c2, tau_p=tau[0], tau_u=tau[1])
    solver = _solver(vxyz, etov, N, M, prec, c2, q, res)
    solver.set_params(*tau)
    solver.stage(1, 1e-3)
    _, rg, _ = solver.get_state(with_res=True)
    _, ro = orc.stage(q, res, 1, 1e-3)
    assert rel_l2(rg, ro) <= TOL_STAGE[prec]


def test_stage_parity_single_element_and_unjittered_mesh():
    for hexes, jitter, shuffle in ((0, 0.0, False), (2, 0.0, False)):
        if hexes == 0:
            vxyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
            etov = np.array([[0, 1, 2, 3]])
            rng = np.random.default_rng(0)
            c2 = rounded(rng.uniform(0.5, 2, (1, 10)), 32)
            q = rounded(rng.standard_normal((4, 1, 20)), 32)
            res = rounded(rng.standard_normal((4, 1, 20)), 32)
        else:
            vxyz, etov, c2, q, res = random_case(hexes, 3, 2, 32, seed=3, jitter=jitter, shuffle=shuffle)
        orc = AcousticOracle(vxyz, etov, 3, 2, c2)
        solver = _solver(vxyz, etov, 3, 2, 32, c2, q, res)
        solver.stage(4, 1e-3)
        _, rg, _ = solver.get_state(with_res=True)
        _, ro = orc.stage(q, res, 4, 1e-3)
        assert rel_l2(rg, ro) <= TOL_STAGE[32]


def test_stage_parity_point_source():
    """A point source driven by arbitrary (random) amplitude samples, one per
    stage, over two steps; samples past the end of the series are zero."""
    N, M, prec = 4, 2, 32
    vxyz, etov, c2, q, res = random_case(2, N, M, prec, seed=8)
    q *= 1e-3  # make the source dominate its element
    xs = np.array([0.41, 0.52, 0.37])
    amp = np.random.default_rng(3).uniform(-2.0, 2.0, 7)  # ends inside the second step
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    e_or, _ = orc.set_point_source(xs, amp)
    solver = _solver(vxyz, etov, N, M, prec, c2, q, res, t=0.08)
    e_gpu = solver.set_point_source(xs, amp)
    assert e_gpu == e_or
    solver.step(2e-3, 3)
    qg, rg, tg = solver.get_state(with_res=True)
    qo, ro = q, res
    for n in range(3):
        qo, ro = orc.step(qo, ro, 2e-3, n)
    assert abs(tg - 0.086) < 1e-15
    assert rel_l2(rg[:, e_or], ro[:, e_or]) <= 1e-5
    assert rel_l2(qg, qo) <= 1e-5


@pytest.mark.parametrize("prec", [32, 64])
def test_manufactured_forcing_parity(prec):
    """The separable forcing of the convergence study (Sec. 6.1),
    f = (3 - 1/c^2) pi sin sin sin(x) sin(pi t), on every element through
    bbw_set_forcing with sin(pi t) sampled at the stage times; the run
    starting from the manufactured solution at t = 0 (p = sin sin sin,
    u = 0) matches the oracle driven by the same samples."""
    N, M, hexes = 3, 1, 2
    vxyz, etov = inputs.cube_mesh(hexes, jitter=0.1, shuffle=True, seed=6)
    K, Np = len(etov), bb.np_count(N)
    c2 = rounded(inputs.sample_at_domain_points(vxyz, etov, M, inputs.c2_config_small), prec)
    g = rounded(inputs.sample_at_domain_points(vxyz, etov, N,
                                               inputs.manufactured_forcing(inputs.c2_config_small)), prec)
    q0 = np.zeros((4, K, Np))
    q0[0] = inputs.sample_at_domain_points(
        vxyz, etov, N, lambda x: np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2]))
    q0 = rounded(q0, prec)
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    dt, nsteps = orc.dt_for(0.1, 0.5)
    amp = inputs.ricker_samples(0.0, 0.0, dt, nsteps, stage_times(), signal=lambda t: np.sin(np.pi * t))
    elems = np.arange(K)
    orc.set_forcing(elems, g, amp)
    solver = _solver(vxyz, etov, N, M, prec, c2, q0, None)
    solver.set_forcing(elems, g, amp)
    solver.step(dt, nsteps)
    qg, _ = solver.get_state()
    qo, _ = orc.run(q0, dt, nsteps)
    assert rel_l2(qg, qo) <= TOL_FINAL[prec]
    # the forcing changes the result (the test is not vacuous)
    orc.source = None
    qn, _ = orc.run(q0, dt, nsteps)
    assert rel_l2(qn, qo) > 1e-3


# -- whole runs -------------------------------------------------------------------

@pytest.mark.parametrize("prec", [32, 64])
def test_final_time_parity_small_config(prec):
    """4^3 x 6 = 384 tets, N=3, M=1, c2 = 1 + 0.5 sin sin sin, p = 0 walls,
    Gaussian pulse, CFL dt, T = 0.5."""
    cfg = inputs.PARITY_CONFIG
    N, M = cfg["N"], cfg["M"]
    vxyz, etov = inputs.cube_mesh(cfg["hexes"])
    # c^2 and the Gaussian L2-projected per element (the tools layer)
    c2 = rounded(project.project_c2(vxyz, etov, M, inputs.c2_config_small), prec)
    K, Np = len(etov), bb.np_count(N)
    q0 = np.zeros((4, K, Np))
    q0[0] = project.l2_project(vxyz, etov, N, inputs.gaussian_pulse())
    q0 = rounded(q0, prec)
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    dt, nsteps = orc.dt_for(cfg["T"], cfg["cfl"])
    solver = _solver(vxyz, etov, N, M, prec, c2, q0, None)
    dtg, ng = solver.advance(cfg["T"], cfg["cfl"])
    assert ng == nsteps and abs(dtg - dt) <= 1e-14 * dt
    qg, tg = solver.get_state()
    qo, _ = orc.run(q0, dt, nsteps)
    assert abs(tg - cfg["T"]) < 1e-12
    assert rel_l2(qg, qo) <= TOL_FINAL[prec]


def test_checkpoint_resume_is_bit_identical():
    N, M = 5, 2
    vxyz, etov, c2, q, _ = random_case(2, N, M, 32, seed=21)
    xs = np.array([0.5, 0.5, 0.5])
    amp = B.ricker_samples(1e-3, 5, f0=10.0, t0=0.002)
    a = _solver(vxyz, etov, N, M, 32, c2, q, None)
    a.set_point_source(xs, amp)
    a.step(1e-3, 5)
    qa, ra, ta = a.get_state(with_res=True)
    b = _solver(vxyz, etov, N, M, 32, c2, q, None)
    b.set_point_source(xs, amp)
    b.step(1e-3, 2)
    qb, rb, tb = b.get_state(with_res=True)
    c = _solver(vxyz, etov, N, M, 32, c2, qb, rb, tb)
    c.set_point_source(xs, amp[10:])  # samples count from the last set_state
    c.step(1e-3, 3)
    qc, rc, tc = c.get_state(with_res=True)
    assert np.array_equal(qa, qc) and np.array_equal(ra, rc) and ta == tc


def test_device_state_roundtrip_and_dtype_conversion():
    N, M = 3, 2
    vxyz, etov, c2, q, res = random_case(2, N, M, 32, seed=4)
    s = _solver(vxyz, etov, N, M, 32, c2, q, res)
    dq = torch.tensor(q, dtype=torch.float64, device="cuda")
    s.set_state_device(dq, None, dtype=64, t=0.0)
    out = torch.empty_like(dq, dtype=torch.float32)
    s.get_state_device(out, None, dtype=32)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.float64), q)
    s.stage(0, 1e-3)
    qg, rg, _ = s.get_state(with_res=True)
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    _, ro = orc.stage(q, np.zeros_like(q), 0, 1e-3)
    assert rel_l2(rg, ro) <= TOL_STAGE[32]


def test_nonfinite_state_is_reported_on_the_host():
    N, M = 2, 1
    vxyz, etov, c2, q, res = random_case(1, N, M, 32, seed=2)
    q[0, 0, 0] = np.nan
    s = _solver(vxyz, etov, N, M, 32, c2, q, res)
    s.stage(0, 1e-3)
    with pytest.raises(B.BBWError) as ei:
        s.sync()
    assert ei.value.status == -5
    s.sync()  # the flag is cleared once reported


def test_rejects_nonpositive_c2():
    vxyz, etov, c2, q, res = random_case(1, 2, 1, 32, seed=2)
    s = B.Solver(vxyz, etov, 2, 1, 32)
    c2[3, 1] = 0.0
    with pytest.raises(B.BBWError) as ei:
        s.set_c2(c2)
    assert ei.value.status == -3


# -- full size, sampled -------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 5, 9])
def test_full_size_sweep_mesh_sampled(N):
    """196,608 tets (the throughput workload) in the bench's launch shape:
    one stage on GPU, sampled elements checked against the oracle patch by patch."""
    cfg = inputs.SWEEP_CONFIG
    M, prec = cfg["M"], 32
    vxyz, etov = inputs.cube_mesh(cfg["hexes"])
    K, Np = len(etov), bb.np_count(N)
    field = inputs.c2_smooth_random(seed=0)
    c2 = rounded(inputs.sample_at_domain_points(vxyz, etov, M, field), prec)
    rng = np.random.default_rng(N)
    q = rounded(rng.standard_normal((4, K, Np)), prec)
    res = rounded(rng.standard_normal((4, K, Np)), prec)
    s = _solver(vxyz, etov, N, M, prec, c2, q, res, t=0.05)
    amp = inputs.ricker_samples(cfg["f0"], 1.0 / cfg["f0"], 1e-4, 1, stage_times(), t_start=0.05)
    src = s.set_point_source(np.array(cfg["source"]), amp)
    s.stage(2, 1e-4)
    qg, rg, _ = s.get_state(with_res=True)
    etoe = B.mesh_analyze(vxyz, etov, N)["etoe"]
    sample = sorted(set([0, K - 1, src] + list(rng.choice(K, 24, replace=False))))
    got, want = [], []
    for e in sample:
        qo, ro = oracle_stage_on_patch(vxyz, etov, etoe, e, N, M, c2, q, res, 2, 1e-4, 0,
                                       source=(np.array(cfg["source"]), amp) if e == src else None)
        got.append(rg[:, e])
        want.append(ro)
    assert rel_l2(np.array(got), np.array(want)) <= TOL_STAGE[prec]


# -- edge cases of the grouped layout -----------------------------------------------

@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("N", [1, 4, 7, 9])
def test_stage_parity_element_counts_not_multiple_of_group(N, prec):
    """K = 1 and K = 5: the last group of V elements is padded."""
    M = 2
    vxyz, etov, c2, q, res = random_case(1, N, M, prec, seed=30 + N)
    for K in (1, 5):
        sub = etov[:K]
        verts, inv = np.unique(sub, return_inverse=True)
        ev = inv.reshape(sub.shape)
        vx = vxyz[verts]
        orc = AcousticOracle(vx, ev, N, M, c2[:K])
        solver = _solver(vx, ev, N, M, prec, c2[:K], q[:, :K], res[:, :K])
        solver.stage(1, 1e-3)
        qg, rg, _ = solver.get_state(with_res=True)
        qo, ro = orc.stage(q[:, :K], res[:, :K], 1, 1e-3)
        assert rel_l2(rg, ro) <= TOL_STAGE[prec], (K, rel_l2(rg, ro))
        assert rel_l2(qg, qo) <= TOL_STAGE[prec]
        solver.close()


@pytest.mark.parametrize("N,M", [(9, 3), (9, 0), (8, 3), (2, 0)])
def test_stage_parity_extreme_shapes_fp64(N, M):
    vxyz, etov, c2, q, res = random_case(1, N, M, 64, seed=40 + N + M)
    orc = AcousticOracle(vxyz, etov, N, M, c2)
    solver = _solver(vxyz, etov, N, M, 64, c2, q, res)
    solver.stage(3, 5e-4)
    _, rg, _ = solver.get_state(with_res=True)
    _, ro = orc.stage(q, res, 3, 5e-4)
    assert rel_l2(rg, ro) <= TOL_STAGE[64]


@pytest.mark.parametrize("prec", [32, 64])
def test_host_state_roundtrip_through_grouped_layout(prec):
    for N, K in ((1, 7), (6, 9), (9, 3)):
        vxyz, etov, c2, q, res = random_case(2, N, 1, prec, seed=N)
        sub = etov[:K]
        verts, inv = np.unique(sub, return_inverse=True)
        s = _solver(vxyz[verts], inv.reshape(sub.shape), N, 1, prec, c2[:K], q[:, :K], res[:, :K], t=0.25)
        qg, rg, t = s.get_state(with_res=True)
        assert np.array_equal(qg, q[:, :K]) and np.array_equal(rg, res[:, :K]) and t == 0.25
        s.close()


def test_solver_face_node_map_matches_mesh_analysis():
    vxyz, etov, c2, q, res = random_case(2, 5, 2, 32, seed=12)
    s = _solver(vxyz, etov, 5, 2, 32, c2, q, res)
    ref = B.mesh_analyze(vxyz, etov, 5)
    assert np.array_equal(s.face_node_map(), ref["nmap"])
    etoe, etof, fperm = s.connectivity()
    assert np.array_equal(etoe, ref["etoe"]) and np.array_equal(fperm, ref["fperm"])


def test_wadg_update_single_element():
    rng = np.random.default_rng(3)
    for N, M in ((1, 2), (9, 2)):
        Np, Mp = bb.np_count(N), bb.np_count(M)
        r = rounded(rng.standard_normal((1, Np)), 32)
        c2 = rounded(rng.uniform(0.5, 2, (1, Mp)), 32)
        want = np.linalg.solve(bb.mass(N), np.einsum("kb,bij,kj->ki", c2, bb.weighted_mass_terms(N, M), r).T).T
        dr = torch.tensor(r, dtype=torch.float32, device="cuda")
        dc = torch.tensor(c2, dtype=torch.float32, device="cuda")
        out = torch.full_like(dr, float("nan"))
        B.wadg_update(N, M, 32, 1, dr, dc, out)
        torch.cuda.synchronize()
        assert rel_l2(out.double().cpu().numpy(), want) <= TOL_STAGE[32]


# -- the GPU solver against the closed-form solution ------------------------------

def test_gpu_standing_wave_converges():
    """c2 = 1, p = 0 walls: p = sin(pi x) sin(pi y) sin(pi z) cos(sqrt(3) pi t);
    the GPU solution converges at a rate near N + 1 = 4 (N = 3, FP64)."""
    from oracle.quadrature import tet_rule
    N, T = 3, 0.1
    errs = []
    for hexes in (2, 4):
        vxyz, etov = inputs.cube_mesh(hexes)
        K = len(etov)
        lam, w = tet_rule(2 * N + 4)
        X = np.asarray(vxyz)[etov]
        xq = np.einsum("qa,kai->kqi", lam, X)
        Vq = bb.evaluate(np.eye(bb.np_count(N)), N, lam)
        Pq = np.linalg.solve(bb.mass(N), Vq * w)
        s3 = np.sin(np.pi * xq)
        c3 = np.cos(np.pi * xq)
        q0 = np.zeros((4, K, bb.np_count(N)))
        q0[0] = np.einsum("aq,kq->ka", Pq, s3[..., 0] * s3[..., 1] * s3[..., 2])
        s = _solver(vxyz, etov, N, 0, 64, np.ones((K, 1)), q0, None)
        s.advance(T, 0.25)
        q, _ = s.get_state()
        w3 = np.sqrt(3) * np.pi
        pex = s3[..., 0] * s3[..., 1] * s3[..., 2] * np.cos(w3 * T)
        uex = -np.pi * np.stack([c3[..., 0] * s3[..., 1] * s3[..., 2], s3[..., 0] * c3[..., 1] * s3[..., 2],
                                 s3[..., 0] * s3[..., 1] * c3[..., 2]]) * np.sin(w3 * T) / w3
        ph = np.einsum("aq,ka->kq", Vq, q[0])
        uh = np.einsum("aq,ika->ikq", Vq, q[1:4])
        vol = B.mesh_analyze(vxyz, etov, N)["vol"][:, None]
        errs.append(np.sqrt(np.sum(vol * w * ((ph - pex) ** 2 + np.sum((uh - uex) ** 2, axis=0)))))
        s.close()
    assert errs[1] < 1e-3 and np.log2(errs[0] / errs[1]) > 3.3


def test_get_state_into_pinned_output_array():
    """bbw_get_state into a caller-given pinned float64 array equals the
    allocating call; a wrong shape or dtype is rejected before any copy."""
    N, M = 4, 2
    vxyz, etov, c2, q, _ = random_case(1, N, M, 32, seed=31)
    s = _solver(vxyz, etov, N, M, 32, c2, q, None)
    s.step(1e-3, 2)
    want, _ = s.get_state()
    out = torch.empty(q.size, dtype=torch.float64, pin_memory=True).numpy()
    got, _ = s.get_state(out=out)
    assert np.array_equal(got, want) and np.shares_memory(got, out)
    with pytest.raises(ValueError):
        s.get_state(out=np.empty(q.size, np.float32))
    s.close()


def test_projected_layer_jump_with_negative_coefficients_is_rejected():
    """The sweep's medium (smooth field with a planar jump) L2-projected onto
    P^2 of a coarse 2^3 x 6 mesh undershoots below zero next to the jump;
    bbw_set_c2 rejects it with BBW_ERR_NONPOS_C2 and keeps the previous c^2."""
    vxyz, etov = inputs.cube_mesh(2)
    c2 = project.l2_project(vxyz, etov, 2, inputs.c2_smooth_random(seed=0), q=6)
    assert (c2 <= 0).any()
    with pytest.raises(project.NonPositiveC2):
        project.project_c2(vxyz, etov, 2, inputs.c2_smooth_random(seed=0))
    s = B.Solver(vxyz, etov, 3, 2, B.F32)
    with pytest.raises(B.BBWError) as ei:
        s.set_c2(c2)
    assert ei.value.status == -3
    s.close()
