"""The range-checked build (libbbwadg_checked.so, kernels compiled with
BBW_CHECKED) runs the same acoustic and elastic cases clean -- no neighbour word or table index out
of range -- and agrees with the normal build. It stands in for a device
memory checker: the checks skip a bad access and report it through the
device status word instead of faulting."""
from __future__ import annotations

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1808_08645_gb300 import build as libbuild
from parity_util import TOL_STAGE, rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = textwrap.dedent("""
    import sys, numpy as np
    sys.path.insert(0, {root!r})
    from paper_1808_08645_gb300 import binding as B, inputs
    lib = {lib!r}
    if lib:
        B.lib_path = lambda: lib
    out = {{}}
    for N, hexes in ((2, 2), (5, 2), (9, 1)):
        vxyz, etov = inputs.cube_mesh(hexes, jitter=0.15, shuffle=True, seed=N)
        rng = np.random.default_rng(N)
        K, Np = len(etov), (N + 1) * (N + 2) * (N + 3) // 6
        s = B.Solver(vxyz, etov, N, 2, 32)
        s.set_c2(rng.uniform(0.5, 2.0, (K, 10)))
        s.set_state(rng.standard_normal((4, K, Np)))
        s.set_point_source([0.5, 0.5, 0.5], B.ricker_samples(1e-3, 2, f0=10.0, t0=0.05))
        s.step(1e-3, 2)
        s.sync()
        out["solo%d" % N] = s.get_state()[0]
        s.close()
    meshes = [inputs.cube_mesh(h, jitter=0.1, shuffle=True, seed=h) for h in (1, 2, 2)]
    b = B.Batch(meshes, [3, 3, 6], 2, 32)
    for i, (v, e) in enumerate(meshes):
        Np = b.np_(i)
        b.set_c2(i, np.full((len(e), 10), 1.5))
        b.set_state(i, np.random.default_rng(i).standard_normal((4, len(e), Np)))
    b.set_point_source(1, [0.4, 0.6, 0.5], B.ricker_samples(1e-3, 2, f0=10.0, t0=0.05))
    b.step(1e-3, 3)
    b.sync()
    for i in range(3):
        out["batch%d" % i] = b.get_state(i)
    b.close()
    ve, ee = inputs.cube_mesh(2, jitter=0.15, shuffle=True, seed=4)
    for N in (3, 9):
        K, Np = len(ee), (N + 1) * (N + 2) * (N + 3) // 6
        e = B.ElasticSolver(ve, ee, N, 2, 32)
        e.set_media(*inputs.elastic_media(ve, ee, 2))
        e.set_state(np.random.default_rng(N).standard_normal((9, K, Np)))
        e.step(1e-3, 2)
        e.sync()
        out["elastic%d" % N] = e.get_state()[0]
        e.close()
    np.savez({path!r}, **out)
""")


def _run(tmp_path, lib, name):
    path = str(tmp_path / f"{name}.npz")
    script = tmp_path / f"{name}.py"
    script.write_text(CASES.format(root=ROOT, lib=lib, path=path))
    p = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-2000:]
    return np.load(path)


def test_checked_build_runs_clean_and_agrees(tmp_path):
    checked = libbuild.build(checked=True)
    libbuild.build()
    got = _run(tmp_path, checked, "checked")
    want = _run(tmp_path, "", "normal")
    assert sorted(got.files) == sorted(want.files)
    for k in want.files:
        assert rel_l2(got[k], want[k]) <= TOL_STAGE[32], k
