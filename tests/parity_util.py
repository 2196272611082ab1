"""Helpers shared by the GPU parity tests: seeded cases and oracle evaluation.

Inputs are drawn in FP64, rounded to the GPU precision and handed, rounded,
to both sides, so the only difference left is the arithmetic.
"""
from __future__ import annotations

import numpy as np

from oracle import bernstein as bb
from oracle.acoustic import AcousticOracle
from paper_1808_08645_gb300 import inputs

#: per-stage tolerance on relative L2 (all four fields concatenated)
TOL_STAGE = {32: 1e-5, 64: 1e-11}
#: final-time tolerance on relative L2
TOL_FINAL = {32: 1e-4, 64: 1e-10}


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def stage_times():
    """The RK stage times c_s as floats (the oracle's exact rationals)."""
    from oracle.acoustic import lsrk_stage_times
    return [float(c) for c in lsrk_stage_times()]


def rounded(x, precision: int):
    return np.asarray(x, dtype=np.float32 if precision == 32 else np.float64).astype(np.float64)


def random_case(hexes: int, N: int, M: int, precision: int, seed: int = 0,
                jitter: float = 0.15, shuffle: bool = True):
    """Mesh, positive c2, random q and res, all rounded to ``precision``."""
    vxyz, etov = inputs.cube_mesh(hexes, jitter=jitter, shuffle=shuffle, seed=seed)
    rng = np.random.default_rng(seed + 1000 * N + 100 * M)
    K = len(etov)
    Np, Mp = bb.np_count(N), bb.np_count(M)
    c2 = rounded(rng.uniform(0.5, 2.0, (K, Mp)), precision)
    q = rounded(rng.standard_normal((4, K, Np)), precision)
    res = rounded(rng.standard_normal((4, K, Np)), precision)
    return vxyz, etov, c2, q, res


def patch(etoe: np.ndarray, e: int):
    """Element e followed by its face neighbours (e's full stencil)."""
    out = [int(e)]
    for nb in etoe[e]:
        if nb >= 0 and int(nb) not in out:
            out.append(int(nb))
    return out


def oracle_stage_on_patch(vxyz, etov, etoe, e, N, M, c2, q, res, s, dt, step=0,
                          tau=(1.0, 1.0), source=None):
    """Oracle stage for element e alone, on the sub-mesh of e and its neighbours.

    The right-hand side of e depends only on e and its face neighbours, and
    e's walls are walls of the sub-mesh too, so e's result equals its result
    on the full mesh. ``source`` = (x, amplitude samples) is applied only if
    e holds it; ``step`` is the RK step the stage belongs to.
    Returns (q_out[:, e], res_out[:, e]).
    """
    els = patch(etoe, e)
    sub_etov = np.asarray(etov)[els]
    verts, inv = np.unique(sub_etov, return_inverse=True)
    sub_etov = inv.reshape(sub_etov.shape)
    sub_vxyz = np.asarray(vxyz)[verts]
    orc = AcousticOracle(sub_vxyz, sub_etov, N, M, c2[els], tau_p=tau[0], tau_u=tau[1])
    if source is not None:
        orc.set_point_source(source[0], source[1])
    qo, ro = orc.stage(q[:, els], res[:, els], s, dt, step)
    return qo[:, 0], ro[:, 0]
