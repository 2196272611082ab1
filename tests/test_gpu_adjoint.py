"""GPU receiver-misfit gradient (bbw_set_receivers / bbw_record / bbw_adjoint)
against the FP64 oracle adjoint and against finite differences of the GPU
forward run; checkpoint spacing does not change the result."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import bernstein as bb
from oracle.acoustic import AcousticOracle
from paper_1808_08645_gb300 import binding as B
from paper_1808_08645_gb300 import inputs
from parity_util import rel_l2, rounded

pytestmark = pytest.mark.gpu

XR = np.array([[0.3, 0.4, 0.9], [0.7, 0.2, 0.5], [0.5, 0.5, 0.0], [0.15, 0.8, 0.6]])
SRC = np.array([0.5, 0.5, 0.5])
#: source amplitude samples (one per RK stage; past the end: zero)
AMP = np.random.default_rng(99).uniform(-1.0, 1.0, 40)


def _case(hexes, N, M, prec, seed=0, jitter=0.1):
    vxyz, etov = inputs.cube_mesh(hexes, jitter=jitter, shuffle=True, seed=seed)
    K = len(etov)
    rng = np.random.default_rng(seed + 7)
    c2 = rounded(rng.uniform(0.5, 2.0, (K, bb.np_count(M))), prec)
    q0 = rounded(rng.standard_normal((4, K, bb.np_count(N))) * 0.1, prec)
    return vxyz, etov, c2, q0, rng


def _gpu(vxyz, etov, N, M, prec, c2, q0, source=True):
    s = B.Solver(vxyz, etov, N, M, prec)
    s.set_c2(c2)
    s.set_state(q0)
    if source:
        s.set_point_source(SRC, AMP)
    s.set_receivers(XR)
    return s


@pytest.mark.parametrize("prec,tol", [(64, 1e-9), (32, 1e-4)])
@pytest.mark.parametrize("N,M", [(2, 1), (4, 2)])
def test_gradient_matches_oracle_adjoint(N, M, prec, tol):
    vxyz, etov, c2, q0, rng = _case(1, N, M, prec, seed=N)
    dt, nsteps = 0.01, 3
    s = _gpu(vxyz, etov, N, M, prec, c2, q0)
    tr = s.record(dt, nsteps, checkpoint_every=2)
    o = AcousticOracle(vxyz, etov, N, M, c2)
    o.set_point_source(SRC, AMP)
    R = adj.receiver_matrix(o, XR)
    tro, _ = adj.record(o, q0, dt, nsteps, R)
    assert rel_l2(tr, tro) <= (1e-11 if prec == 64 else 1e-4)
    g = rng.standard_normal(tr.shape)
    gc, gq = s.adjoint(g, want_q0=True)
    gco, gqo = adj.misfit_gradient(o, q0, dt, nsteps, R, g)
    assert rel_l2(gc, gco) <= tol
    assert rel_l2(gq, gqo) <= tol
    s.close()


def test_checkpoint_spacing_does_not_change_the_gradient():
    """Checkpoint spacings 1, 3, 7 and 0 (every stage's bracket kept, no
    recomputation; then a checkpointed run on the same solver, which must
    not reuse the kept brackets) give bitwise equal gradients."""
    N, M = 3, 2
    vxyz, etov, c2, q0, rng = _case(2, N, M, 32, seed=5)
    g = rng.standard_normal((7, len(XR)))
    out = []
    for every in (1, 3, 7, 0):
        s = _gpu(vxyz, etov, N, M, 32, c2, q0)
        s.record(2e-3, 7, checkpoint_every=every)
        out.append(s.adjoint(g, want_q0=True))
        if every == 0:
            s.set_state(q0)
            s.record(2e-3, 7, checkpoint_every=2)
            out.append(s.adjoint(g, want_q0=True))
        s.close()
    for gc, gq in out[1:]:
        assert np.array_equal(gc, out[0][0]) and np.array_equal(gq, out[0][1])


def test_gradient_matches_gpu_finite_differences():
    """FP64 on a 2^3 x 6 mesh, N = 3, M = 2, 12 steps: directional derivative
    of the L2 misfit against central differences of GPU forward runs."""
    N, M = 3, 2
    vxyz, etov, c2, q0, rng = _case(2, N, M, 64, seed=11)
    dt, nsteps = 2e-3, 12
    data = rng.standard_normal((nsteps, len(XR))) * 1e-3

    def misfit(c2v):
        s = _gpu(vxyz, etov, N, M, 64, c2v, q0)
        tr = s.record(dt, nsteps, checkpoint_every=5)
        return 0.5 * np.sum((tr - data) ** 2), tr, s

    J0, tr, s = misfit(c2)
    gc, _ = s.adjoint(tr - data)
    s.close()
    d = rng.uniform(-1.0, 1.0, c2.shape) * 0.1
    eps = 1e-6
    fd = (misfit(c2 + eps * d)[0] - misfit(c2 - eps * d)[0]) / (2 * eps)
    assert abs(fd - np.sum(gc * d)) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("N,tol32", [(8, 5e-3), (9, 0.1)])
def test_high_degree_gradients(N, tol32):
    """N = 8 and 9, where the contraction's tables sit in shared memory (FP32,
    N = 8) or are read from global memory (N = 9, and FP64): the FP64
    directional derivative matches GPU central differences, and FP32 matches
    FP64 on the same rounded inputs to within its conditioning. The c^2
    gradient integrates the product of two Bernstein expansions whose
    coefficients grow with N far beyond the functions they represent (the
    lifted fluxes in the bracket, the dual variable), so FP32 agrees with
    FP64 to 1e-5 at N = 5, 1.4e-3 at N = 8 and 3.7e-2 at N = 9 (measured),
    while the state gradient stays within 2.3e-5."""
    M = 2
    vxyz, etov, c2, q0, rng = _case(1, N, M, 32, seed=N)
    dt, nsteps = 5e-4, 4
    data = rng.standard_normal((nsteps, len(XR))) * 1e-3

    def run(c2v, prec):
        s = _gpu(vxyz, etov, N, M, prec, c2v, q0)
        tr = s.record(dt, nsteps, checkpoint_every=2)
        return 0.5 * np.sum((tr - data) ** 2), tr, s

    _, tr, s = run(c2, 64)
    g64, _ = s.adjoint(tr - data)
    s.close()
    d = rng.uniform(-1.0, 1.0, c2.shape) * 0.1
    eps = 1e-6
    fd = (run(c2 + eps * d, 64)[0] - run(c2 - eps * d, 64)[0]) / (2 * eps)
    assert abs(fd - np.sum(g64 * d)) <= 1e-6 * abs(fd)
    _, tr32, s32 = run(c2, 32)
    g32, _ = s32.adjoint(tr32 - data)
    s32.close()
    assert rel_l2(g32, g64) <= tol32


def test_adjoint_needs_a_recorded_run():
    vxyz, etov, c2, q0, _ = _case(1, 2, 1, 32)
    s = _gpu(vxyz, etov, 2, 1, 32, c2, q0)
    with pytest.raises(B.BBWError, match="BBW_ERR_ARG"):
        s.adjoint(np.zeros((1, len(XR))))
    with pytest.raises(B.BBWError, match="BBW_ERR_ARG"):
        s.set_receivers(np.array([[3.0, 0.5, 0.5]]))
    s.close()


def test_autograd_function_gradcheck_and_backward():
    """torch.autograd.gradcheck (FP64 solver, double tensors) and
    loss.backward() against bbw_adjoint."""
    import torch

    from paper_1808_08645_gb300.autograd import receiver_traces

    N, M = 2, 1
    vxyz, etov, c2, q0, rng = _case(1, N, M, 64, seed=21)
    s = _gpu(vxyz, etov, N, M, 64, c2, q0)
    c2t = torch.tensor(c2, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda c: receiver_traces(s, c, q0, 0.01, 3, 2), (c2t,),
                                    eps=1e-6, atol=1e-8, rtol=1e-5)
    data = torch.tensor(rng.standard_normal((3, len(XR))) * 1e-2)
    loss = 0.5 * ((receiver_traces(s, c2t, q0, 0.01, 3, 2) - data) ** 2).sum()
    loss.backward()
    s.set_c2(c2)  # the same run again
    s.set_state(q0)
    tr = s.record(0.01, 3, 2)
    gc, _ = s.adjoint(tr - data.numpy())
    assert np.allclose(c2t.grad.numpy(), gc, rtol=1e-12, atol=1e-14)
    s.close()


def test_backward_of_an_earlier_forward_uses_its_own_run():
    """Two forwards on one solver, then the backward of the first: its gradient
    is the first run's (the autograd function records that run again)."""
    import torch

    from paper_1808_08645_gb300.autograd import receiver_traces

    N, M = 2, 1
    vxyz, etov, c2, q0, rng = _case(1, N, M, 64, seed=23)
    s = _gpu(vxyz, etov, N, M, 64, c2, q0)
    c2a = torch.tensor(c2, dtype=torch.float64, requires_grad=True)
    c2b = torch.tensor(c2 * 1.3, dtype=torch.float64, requires_grad=True)
    data = torch.tensor(rng.standard_normal((3, len(XR))) * 1e-2)
    la = 0.5 * ((receiver_traces(s, c2a, q0, 0.01, 3, 2) - data) ** 2).sum()
    lb = 0.5 * ((receiver_traces(s, c2b, q0, 0.01, 3, 2) - data) ** 2).sum()
    la.backward()
    lb.backward()
    for c2v, got in ((c2, c2a.grad), (c2 * 1.3, c2b.grad)):
        s.set_c2(c2v)
        s.set_state(q0)
        tr = s.record(0.01, 3, 2)
        gc, _ = s.adjoint(tr - data.numpy())
        assert np.allclose(got.numpy(), gc, rtol=1e-12, atol=1e-14)
    assert not np.allclose(c2a.grad.numpy(), c2b.grad.numpy())
    s.close()


def test_gradient_on_the_adjoint_workload_mesh():
    """The adjoint workload's mesh and degree (16^3 x 6 = 24,576 tets, N = 5,
    M = 2, 64 receivers on the top face) in FP64, over 20 steps: the adjoint's
    directional derivative of the L2 misfit matches central differences of
    GPU forward runs, and FP32 matches FP64."""
    cfg = inputs.ADJOINT_CONFIG
    N, M = cfg["N"], cfg["M"]
    vxyz, etov = inputs.cube_mesh(cfg["hexes"])
    K = len(etov)
    c2 = inputs.sample_at_domain_points(vxyz, etov, M, inputs.c2_smooth_random(seed=cfg["model_seed"]))
    rec = inputs.top_face_receivers()
    nsteps = 20
    rng = np.random.default_rng(3)

    # a pressure pulse just below the receivers, so that 20 steps already
    # give traces that depend on c^2 (plus the workload's point source)
    q0 = np.zeros((4, K, bb.np_count(N)))
    q0[0] = inputs.sample_at_domain_points(vxyz, etov, N, inputs.gaussian_pulse((0.5, 0.5, 0.9), 0.1))

    def solver(prec, c2v):
        s = B.Solver(vxyz, etov, N, M, prec)
        s.set_c2(c2v)
        s.set_state(q0)
        s.set_receivers(rec)
        return s

    s = solver(64, c2)
    dt = s.cfl_dt(cfg["cfl"])
    amp = B.ricker_samples(dt, nsteps, f0=40.0, t0=2 * dt)
    s.set_point_source(np.array(cfg["source"]), amp)
    tr = s.record(dt, nsteps, 5)
    data = tr * 0.9 + 1e-3 * rng.standard_normal(tr.shape) * np.abs(tr).max()
    gc, _ = s.adjoint(tr - data)
    s.close()

    def misfit(c2v):
        t = solver(64, c2v)
        t.set_point_source(np.array(cfg["source"]), amp)
        out = t.record(dt, nsteps, 5)
        t.close()
        return 0.5 * np.sum((out - data) ** 2)

    d = rng.uniform(-1.0, 1.0, c2.shape) * 0.1
    eps = 1e-5
    fd = (misfit(c2 + eps * d) - misfit(c2 - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(gc * d)) <= 1e-6 * abs(fd)
    s32 = solver(32, c2)
    s32.set_point_source(np.array(cfg["source"]), amp)
    tr32 = s32.record(dt, nsteps, 5)
    gc32, _ = s32.adjoint(tr32 - data)
    s32.close()
    assert rel_l2(gc32, gc) <= 1e-3
