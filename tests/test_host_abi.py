"""Host-side tests of libbbwadg (no GPU): symbols, constants, mesh logic, errors.

The library is built by the session fixture (nvcc cross-compiles without a
GPU); no call here launches a kernel or allocates device memory.
"""
import os
import re

import numpy as np
import pytest

from oracle import bernstein as bb
from oracle.acoustic import LSRK_A, LSRK_B, lsrk_stage_times
from oracle.mesh import FACE_VERTS, connectivity, face_node_map, geometry
from paper_1808_08645_gb300 import binding as B
from paper_1808_08645_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_1808_08645_gb300 import build
    build.build()
    return B.lib()


def _header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bbw_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported_and_bound():
    declared = _header_functions()
    assert declared, "no declarations found"
    L = B.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(B.EXPORTS), declared - set(B.EXPORTS)


def test_version():
    assert B.lib().bbw_version() >= 100


@pytest.mark.parametrize("N,M", [(1, 1), (2, 2), (3, 1), (3, 2), (5, 2), (7, 2), (9, 2), (9, 3)])
def test_projection_coeffs_match_oracle(N, M):
    c = B.projection_coeffs(N, M)
    co, _ = bb.projection_coeffs(N, M)
    assert np.allclose(c, co, rtol=1e-8, atol=1e-9)


def test_projection_coeffs_table1():
    # Table 1, N=4 M=2 (printed to 4 decimals)
    assert np.allclose(B.projection_coeffs(4, 2), [2.8846, -2.7972, 0.9441, -0.1119, 0.0029], atol=5.1e-5)


def test_lsrk_coeffs_match_oracle():
    a, b, c = B.lsrk_coeffs()
    assert np.allclose(a, [float(x) for x in LSRK_A], rtol=1e-15, atol=0)
    assert np.allclose(b, [float(x) for x in LSRK_B], rtol=1e-15, atol=0)
    assert np.allclose(c, [float(x) for x in lsrk_stage_times()], rtol=1e-14, atol=1e-16)


def _oracle_nmap_in_face_order(vxyz, etov, N):
    etoe, etof = connectivity(etov)
    nm = face_node_map(vxyz, etov, etoe, etof, N)
    out = np.empty((len(etov), 4, bb.np_count(N, 2)), np.int64)
    for f in range(4):
        vol_idx = []
        for b in bb.face_multi_indices(N):
            al = [0, 0, 0, 0]
            for x, v in enumerate(FACE_VERTS[f]):
                al[v] = b[x]
            vol_idx.append(bb.index_of(al))
        out[:, f, :] = nm[:, f, vol_idx]
    return etoe, etof, out


@pytest.mark.parametrize("N", [1, 2, 4, 6, 9])
def test_connectivity_and_face_map_bit_exact(N):
    vxyz, etov = inputs.cube_mesh(2, jitter=0.15, shuffle=True, seed=N)
    m = B.mesh_analyze(vxyz, etov, N)
    etoe, etof, nmap = _oracle_nmap_in_face_order(vxyz, etov, N)
    assert np.array_equal(m["etoe"], etoe)
    assert np.array_equal(m["etof"], etof)
    assert np.array_equal(m["nmap"], nmap)
    assert set(np.unique(m["fperm"][m["fperm"] >= 0])) == set(range(6))
    assert np.all(m["fperm"][m["etoe"] < 0] == -1)


def test_geometry_matches_oracle():
    vxyz, etov = inputs.cube_mesh(3, jitter=0.2, shuffle=True, seed=9)
    m = B.mesh_analyze(vxyz, etov, 2)
    geo = geometry(vxyz, etov)
    assert np.allclose(m["grad"], geo["grad"], rtol=0, atol=1e-12)
    assert np.allclose(m["vol"], geo["vol"], rtol=1e-13, atol=0)


def test_single_element_is_all_walls():
    vxyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    m = B.mesh_analyze(vxyz, np.array([[0, 1, 2, 3]]), 3)
    assert np.all(m["etoe"] == -1) and np.all(m["nmap"] == -1)


def test_mesh_errors():
    vxyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0], [1, 1, 1]])
    with pytest.raises(B.BBWError) as ei:                      # inverted element
        B.mesh_analyze(vxyz, np.array([[0, 2, 1, 3]]), 2)
    assert ei.value.status == -2
    with pytest.raises(B.BBWError) as ei:                      # degenerate (repeated vertex)
        B.mesh_analyze(vxyz, np.array([[0, 1, 1, 3]]), 2)
    assert ei.value.status == -2
    with pytest.raises(B.BBWError) as ei:                      # vertex id out of range
        B.mesh_analyze(vxyz, np.array([[0, 1, 2, 7]]), 2)
    assert ei.value.status == -2
    # three tets sharing the face (0, 1, 2): non-manifold
    v = np.vstack([vxyz, [[0.2, 0.2, -1.0], [0.3, 0.3, 2.0]]])
    et = np.array([[0, 1, 2, 3], [0, 2, 1, 5], [0, 1, 2, 6]])
    with pytest.raises(B.BBWError) as ei:
        B.mesh_analyze(v, et, 1)
    assert ei.value.status == -2
    with pytest.raises(B.BBWError) as ei:
        B.mesh_analyze(vxyz, np.array([[0, 1, 2, 3]]), 10)
    assert ei.value.status == -7


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "_LIB", None)
    monkeypatch.setattr(B, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        B.projection_coeffs(2, 1)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("M", [0, 1, 2, 3])
def test_operator_tables_agree_with_brute_force(M, prec):
    """Every stencil word, product index, face map and lift slot the kernels
    use, for all N, recomputed by enumeration of the multi-index lattice
    (host only)."""
    for N in range(1, 10):
        B.validate_tables(N, M, prec)


def test_table_validation_rejects_bad_arguments():
    with pytest.raises(B.BBWError, match="BBW_ERR_UNSUPPORTED"):
        B.validate_tables(10, 2, 32)
    with pytest.raises(B.BBWError, match="BBW_ERR_ARG"):
        B.validate_tables(3, 2, 16)


def test_elastic_argument_and_mesh_errors_need_no_device():
    """bbw_elastic_create validates sizes, precision and the mesh on the host
    before any device work; every call rejects a NULL handle."""
    vxyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    with pytest.raises(B.BBWError, match="BBW_ERR_UNSUPPORTED"):
        B.ElasticSolver(vxyz, np.array([[0, 1, 2, 3]]), 10, 2)
    with pytest.raises(B.BBWError, match="BBW_ERR_UNSUPPORTED"):
        B.ElasticSolver(vxyz, np.array([[0, 1, 2, 3]]), 3, 4)
    with pytest.raises(B.BBWError, match="BBW_ERR_ARG"):
        B.ElasticSolver(vxyz, np.array([[0, 1, 2, 3]]), 3, 2, precision=16)
    with pytest.raises(B.BBWError, match="BBW_ERR_MESH"):        # inverted element
        B.ElasticSolver(vxyz, np.array([[0, 2, 1, 3]]), 3, 2)
    L = B.lib()
    assert L.bbw_elastic_stage(None, 0, 1e-3) == -1
    assert L.bbw_elastic_step(None, 1e-3, 1) == -1
    assert L.bbw_elastic_set_params(None, 1.0, 1.0) == -1
    assert L.bbw_elastic_set_media(None, None, None, None) == -1
    assert L.bbw_elastic_set_state(None, None, None, 0.0) == -1
    assert L.bbw_elastic_get_state(None, None, None, None) == -1
    assert L.bbw_elastic_sync(None) == -1
    assert L.bbw_elastic_get_time(None, None, None) == -1
    assert L.bbw_elastic_info(None, None, None, None, None, None, None) == -1
    L.bbw_elastic_destroy(None)  # no-op


def test_surrogate_and_batch_argument_errors_need_no_device():
    """The bbw_nn_* calls and the per-instance batch calls validate their
    arguments on the host and return BBW_ERR_ARG (-1) before any device work."""
    L = B.lib()
    p = 4096  # a dummy non-NULL address: never dereferenced on these paths
    # GEMM: negative sizes, NULL matrices, split-K with an epilogue, batch x splits beyond the grid
    assert L.bbw_nn_gemm(-1, 4, 4, p, 4, 0, 0, p, 4, 0, 0, p, 4, 0, 1, 1.0, 0.0, None, None, 0, 1, None) == -1
    assert L.bbw_nn_gemm(4, 4, 4, None, 4, 0, 0, p, 4, 0, 0, p, 4, 0, 1, 1.0, 0.0, None, None, 0, 1, None) == -1
    assert L.bbw_nn_gemm(4, 4, 4, p, 4, 0, 0, p, 4, 0, 0, p, 4, 0, 1, 1.0, 1.0, None, None, 0, 2, None) == -1
    assert L.bbw_nn_gemm(4, 4, 4, p, 4, 0, 0, p, 4, 0, 0, p, 4, 0, 1, 1.0, 0.0, None, None, 2, 1, None) == -1
    assert L.bbw_nn_gemm(4, 4, 4, p, 4, 0, 0, p, 4, 0, 0, p, 4, 0, 1000, 1.0, 0.0, None, None, 0, 100, None) == -1
    # transforms: modes beyond 16, a contraction with an epilogue
    assert L.bbw_nn_axis_transform(p, 64, 17, p, p + 64, 1, 32, 0, 0.0, None, 0, None) == -1
    assert L.bbw_nn_axis_transform(p, 64, 6, p, p + 64, 1, 32, 0, 1.0, None, 0, None) == -1
    # shifts in place, bias gradients of width 0, receivers without arrays
    assert L.bbw_nn_shift_traces(p, p, p, None, 3, 8, None) == -1
    assert L.bbw_nn_bias_grad(p, p, 10, 0, None) == -1
    assert L.bbw_nn_gather_receivers(p, p, None, p, p, 1, 8, 8, 8, 4, 2, 0, None) == -1
    assert L.bbw_nn_mse(p, p, None, None, 10, None) == -1
    assert L.bbw_nn_adam(p, p, p, p, 10, 0, 1e-3, 0.9, 0.999, 1e-8, None) == -1
    # per-instance batch calls on a NULL batch
    assert L.bbw_batch_set_instance_steps(None, None, None) == -1
    assert L.bbw_batch_instance_time(None, 0, None, None) == -1
    assert L.bbw_batch_member_cfl_dt(None, 0, 0.5, None) == -1
