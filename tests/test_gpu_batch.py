"""Batched instances (bbw_batch_*): every instance of a batch evolves exactly as
it does alone in a bbw_solver, with and without graph replay, and matches the
FP64 oracle.

The batch runs the single-mesh stage kernel over the disjoint union of the
instances of one degree, so per-instance results are compared bitwise against
solo solvers given the same inputs; one instance is also checked against the
oracle at the final-time tolerance.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.acoustic import AcousticOracle
from paper_1808_08645_gb300 import binding as B
from paper_1808_08645_gb300 import inputs
from parity_util import TOL_FINAL, rel_l2, rounded

pytestmark = pytest.mark.gpu

M = 2
# (hexes, jitter, degree, source point or None): two instances share N = 3 and
# N = 2, single-hex and multi-hex meshes, sources in some instances only
SPECS = [(2, 0.0, 3, (0.5, 0.5, 0.5)), (1, 0.1, 2, None), (3, 0.15, 5, (0.3, 0.6, 0.4)),
         (2, 0.1, 3, None), (2, 0.0, 2, (0.7, 0.2, 0.5)), (1, 0.0, 7, None)]


def _instances(prec, seed=0):
    out = []
    for j, (hexes, jit, N, xs) in enumerate(SPECS):
        vxyz, etov = inputs.cube_mesh(hexes, jitter=jit, shuffle=True, seed=seed + j)
        rng = np.random.default_rng(seed + 17 * j)
        K, Np, Mp = len(etov), bb.np_count(N), bb.np_count(M)
        c2 = rounded(rng.uniform(0.5, 2.0, (K, Mp)), prec)
        q = rounded(rng.standard_normal((4, K, Np)) * 1e-2, prec)
        # amplitude samples of uneven lengths (the batch pads them with zeros)
        amp = rng.uniform(-1.0, 1.0, 11 + 3 * j)
        out.append(dict(vxyz=vxyz, etov=etov, N=N, c2=c2, q=q, xs=xs, amp=amp))
    return out


def _batch(insts, prec):
    b = B.Batch([(d["vxyz"], d["etov"]) for d in insts], [d["N"] for d in insts], M, prec)
    for i, d in enumerate(insts):
        b.set_c2(i, d["c2"])
        b.set_state(i, d["q"])
        if d["xs"] is not None:
            b.set_point_source(i, np.array(d["xs"]), d["amp"])
    return b


def _solo(d, prec):
    s = B.Solver(d["vxyz"], d["etov"], d["N"], M, prec)
    s.set_c2(d["c2"])
    s.set_state(d["q"])
    if d["xs"] is not None:
        s.set_point_source(np.array(d["xs"]), d["amp"])
    return s


@pytest.mark.parametrize("prec", [32, 64])
def test_batch_matches_solo_solvers_bitwise(prec):
    insts = _instances(prec)
    dt, nsteps = 2e-3, 4
    b = _batch(insts, prec)
    n, nb, _ = b.info()
    assert n == len(insts) and nb == len({d["N"] for d in insts})
    b.step(dt, nsteps, graph=True)
    b.sync()
    t, steps = b.time()
    assert steps == nsteps and abs(t - nsteps * dt) < 1e-15
    for i, d in enumerate(insts):
        s = _solo(d, prec)
        s.step(dt, nsteps)
        qs, rs, _ = s.get_state(with_res=True)
        qb, rb = b.get_state(i, with_res=True)
        assert np.array_equal(qb, qs), (i, rel_l2(qb, qs))
        assert np.array_equal(rb, rs), (i, rel_l2(rb, rs))
        s.close()
    b.close()


def test_graph_replay_equals_direct_launches():
    insts = _instances(32, seed=5)
    a, c = _batch(insts, 32), _batch(insts, 32)
    a.step(1e-3, 3, graph=True)
    c.step(1e-3, 3, graph=False)
    for i in range(len(insts)):
        assert np.array_equal(a.get_state(i), c.get_state(i))
    # the cached graph of each parity is reused, and rebuilt when dt changes
    a.step(1e-3, 2, graph=True)
    a.step(5e-4, 1, graph=True)
    c.step(1e-3, 2, graph=False)
    c.step(5e-4, 1, graph=False)
    for i in range(len(insts)):
        assert np.array_equal(a.get_state(i), c.get_state(i))
    a.close()
    c.close()


def test_batch_instance_matches_oracle():
    """Instance 2 (N = 5, jittered 3^3 x 6 mesh, point source) against the
    FP64 oracle after 3 steps; the other instances share its launches."""
    prec = 32
    insts = _instances(prec, seed=9)
    b = _batch(insts, prec)
    dt, nsteps = 1e-3, 3
    b.step(dt, nsteps)
    d = insts[2]
    orc = AcousticOracle(d["vxyz"], d["etov"], d["N"], M, d["c2"])
    orc.set_point_source(np.array(d["xs"]), d["amp"])
    qo, _ = orc.run(d["q"], dt, nsteps)
    assert rel_l2(b.get_state(2), qo) <= TOL_FINAL[prec]
    b.close()


def test_member_layout_and_moving_a_source():
    insts = _instances(32, seed=3)
    b = _batch(insts, 32)
    firsts = {}
    for i, d in enumerate(insts):
        m = b.member(i)
        assert m["N"] == d["N"] and m["K"] == len(d["etov"]) and m["Np"] == bb.np_count(d["N"])
        firsts.setdefault(m["bucket"], []).append((m["first"], m["K"]))
    for ranges in firsts.values():  # instances of a bucket do not overlap
        ranges.sort()
        for (f0, k0), (f1, _) in zip(ranges, ranges[1:]):
            assert f1 >= f0 + k0
    # moving instance 0's source equals a solo solver with the moved source
    d = dict(insts[0], xs=(0.2, 0.3, 0.7))
    e = b.set_point_source(0, np.array(d["xs"]), d["amp"])
    s = _solo(d, 32)
    assert e == s.set_point_source(np.array(d["xs"]), d["amp"])
    b.step(2e-3, 2)
    s.step(2e-3, 2)
    assert np.array_equal(b.get_state(0), s.get_state()[0])
    b.close()
    s.close()


def test_batch_cfl_dt_is_the_smallest_instance_dt():
    insts = _instances(32, seed=4)
    b = _batch(insts, 32)
    want = min(_solo(d, 32).cfl_dt(0.5) for d in insts)
    assert abs(b.cfl_dt(0.5) - want) <= 1e-15 * want
    b.close()


def test_batch_argument_errors():
    insts = _instances(32)
    b = _batch(insts[:2], 32)
    with pytest.raises(B.BBWError, match="BBW_ERR_ARG"):
        b.member(2)
    with pytest.raises(B.BBWError, match="BBW_ERR_NONPOS_C2"):
        b.set_c2(0, -np.ones((len(insts[0]["etov"]), bb.np_count(M))))
    with pytest.raises(B.BBWError, match="BBW_ERR_ARG"):
        b.set_point_source(1, np.array([5.0, 5.0, 5.0]), np.ones(3))
    b.close()


def test_autotune_keeps_state_and_results():
    """The autotuner's dt = 0 trial steps leave state and time unchanged, and
    whichever schedule it keeps gives the solo solvers' results bitwise."""
    insts = _instances(32, seed=11)
    b = _batch(insts, 32)
    b.step(1e-3, 2)
    before = [b.get_state(i, with_res=False) for i in range(len(insts))]
    t0 = b.time()
    sched, ms = b.autotune(2)
    assert 0 <= sched < 4 and ms > 0
    assert b.time() == t0
    for i in range(len(insts)):
        assert np.array_equal(b.get_state(i), before[i])
    b.step(1e-3, 3)
    for i, d in enumerate(insts):
        s = _solo(d, 32)
        s.step(1e-3, 5)
        assert np.array_equal(b.get_state(i), s.get_state()[0]), i
        s.close()
    b.close()


@pytest.mark.parametrize("prec,graph", [(32, True), (64, False)])
def test_per_instance_dt_and_step_budgets_match_solo_runs(prec, graph):
    """Each instance steps with its own dt (half its CFL step) and stops after
    its own step budget; it then equals its solo solver run with that dt for
    that many steps, bitwise (state and residual), while the batch goes on;
    an autotuner pass in between leaves all of that unchanged."""
    insts = _instances(prec, seed=3)
    b = _batch(insts, prec)
    n = len(insts)
    dts = np.array([0.5 * b.member_cfl_dt(i, 0.5) for i in range(n)])
    assert np.isclose(dts.min(), 0.5 * b.cfl_dt(0.5), rtol=0, atol=0)
    budgets = np.array([2 + i % 3 for i in range(n)], dtype=np.int64)
    b.set_instance_steps(dts, budgets)
    b.step(1.0, 2, graph=graph)  # the common dt is not used
    b.autotune(1)
    b.step(1.0, int(budgets.max()) + 1 - 2, graph=graph)
    b.sync()
    for i, d in enumerate(insts):
        t, steps = b.instance_time(i)
        assert steps == budgets[i] and abs(t - budgets[i] * dts[i]) <= 1e-12 * t
        s = _solo(d, prec)
        s.step(float(dts[i]), int(budgets[i]))
        qs, rs, _ = s.get_state(with_res=True)
        qb, rb = b.get_state(i, with_res=True)
        assert np.array_equal(qb, qs), (i, rel_l2(qb, qs))
        assert np.array_equal(rb, rs), (i, rel_l2(rb, rs))
        s.close()
    with pytest.raises(B.BBWError):
        b.set_instance_steps(np.full(n, np.nan))
    with pytest.raises(B.BBWError):
        b.set_instance_steps(None, np.full(n, -1))
    b.close()
