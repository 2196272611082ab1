"""Host-side checks of the measurement script and the seeded input
generators (CPU only): the reference arm's JSON line, the traffic lookup's
source check, and the batched / adjoint workload recipes."""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1808_08645_gb300 import inputs  # noqa: E402

REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config")


def test_reference_arm_line_has_the_contract_keys():
    args = argparse.Namespace(Ns="1,3", ref_hexes=1, steps=1, warmup=0, gpus=1)
    out = bench.run_reference(args)
    json.dumps(out)
    for k in REQUIRED:
        assert k in out, k
    assert out["impl"] == "reference" and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0


def test_traffic_lookup_tracks_the_kernel_sources(tmp_path, monkeypatch):
    """A committed traffic figure is reported only for the sources it was
    measured on."""
    assert bench.load_traffic(9) is None or bench.load_traffic(9) > 0
    prof = tmp_path / "profiles"
    prof.mkdir()
    line = {"N": 4, "traffic_bytes_per_launch": 123.0, "kernel_sources_sha256": bench.kernel_sources_sha256()}
    (prof / "stage_kernel_n4_test_dram_traffic.md").write_text("x\nmachine-readable: " + json.dumps(line) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the sources are read from the real tree
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: line["kernel_sources_sha256"])
    assert bench.load_traffic(4) == 123.0
    line["K"] = 196608
    (prof / "stage_kernel_n4_test_dram_traffic.md").write_text("x\nmachine-readable: " + json.dumps(line) + "\n")
    assert bench.load_traffic(4, 196608) == 123.0
    assert bench.load_traffic(4, 10368) is None  # captured on another mesh
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: "0" * 64)
    assert bench.load_traffic(4) is None
    assert bench.load_traffic(5) is None


def test_algorithmic_bytes_formula():
    # q_in read, q_out and res written, res read on 4 of 5 stages, c2, geometry, connectivity
    N, M = 9, 2
    np3 = lambda n: (n + 1) * (n + 2) * (n + 3) // 6
    want = 4 * ((12 + 16 / 5) * np3(N) + np3(M) + 9) + 16
    assert abs(bench.algorithmic_bytes_per_element(N, M) - want) < 1e-9


def test_batched_instances_recipe():
    a = inputs.batched_instances()
    b = inputs.batched_instances()
    assert all(x["hexes"] == y["hexes"] and x["N"] == y["N"] and x["c2_seed"] == y["c2_seed"]
               and np.array_equal(x["source"], y["source"]) for x, y in zip(a, b))
    cfg = inputs.BATCH_CONFIG
    assert len(a) == cfg["instances"]
    tets = [6 * d["hexes"] ** 3 for d in a]
    assert 2000 <= min(tets) and max(tets) <= 60000
    assert {d["N"] for d in a} <= set(range(cfg["Ns"][0], cfg["Ns"][1] + 1))
    assert len({d["c2_seed"] for d in a}) == len(a)
    for d in a:
        assert np.all((d["source"] >= 0.25) & (d["source"] <= 0.75))


def test_top_face_receivers():
    r = inputs.top_face_receivers(8)
    assert r.shape == (64, 3)
    assert np.all(r[:, 2] == 1.0)
    assert np.all((r[:, :2] > 0) & (r[:, :2] < 1))
    assert len({tuple(x) for x in r}) == 64


def test_elastic_reference_line_and_bytes():
    args = argparse.Namespace(Ns="1,2", steps=1, warmup=0, gpus=1)
    out = bench.run_elastic_reference(args)
    json.dumps(out)
    for k in REQUIRED:
        assert k in out, k
    assert out["impl"] == "reference" and out["value"] > 0
    N, M = 9, 2
    np3 = lambda n: (n + 1) * (n + 2) * (n + 3) // 6
    want = 4 * ((27 + 36 / 5) * np3(N) + 3 * np3(M) + 9) + 16
    assert abs(bench.elastic_bytes_per_element(N, M) - want) < 1e-9
    assert bench.load_elastic_traffic(9) is None or bench.load_elastic_traffic(9) > 0


def test_elastic_inputs_recipe():
    vxyz, etov = inputs.cube_mesh(2)
    rho_inv, lam, mu = inputs.elastic_media(vxyz, etov, 2)
    assert rho_inv.shape == lam.shape == mu.shape == (48, 10)
    assert rho_inv.min() > 0 and lam.min() > 0 and mu.min() > 0
    assert np.allclose(lam, mu)  # Poisson ratio 1/4
    q = inputs.elastic_pulse(vxyz, etov, 3)
    assert q.shape == (9, 48, 20)
    assert np.all(q[:3] == 0) and np.all(q[6:] == 0)
    assert np.array_equal(q[3], q[4]) and np.array_equal(q[4], q[5]) and q[3].min() < 0



def test_ricker_samples_are_the_wavelet_at_the_stage_times():
    """Sample 5 n + s is the (separately pinned) oracle wavelet at
    t_start + (n + c_s) dt, for the test helper and the library's helper."""
    from oracle.acoustic import lsrk_stage_times, ricker
    from paper_1808_08645_gb300 import binding as B
    c = [float(x) for x in lsrk_stage_times()]
    f0, t0, dt, n, ts = 10.0, 0.07, 3e-3, 9, 0.011
    want = [ricker(ts + (k // 5 + c[k % 5]) * dt, f0, t0) for k in range(5 * n)]
    got = inputs.ricker_samples(f0, t0, dt, n, c, t_start=ts)
    assert np.allclose(got, want, rtol=0, atol=1e-15)
    lib_got = B.ricker_samples(dt, n, f0=f0, t0=t0, t_start=ts)
    assert np.allclose(lib_got, want, rtol=0, atol=1e-14)


def test_manufactured_forcing_makes_the_manufactured_solution_exact():
    """(1/c^2) dp/dt + div u = f and du/dt + grad p = 0 for
    p = sin sin sin cos(pi t), u = -(cos sin sin, sin cos sin, sin sin cos) sin(pi t),
    checked by central differences at random points and times."""
    rng = np.random.default_rng(0)
    x = rng.uniform(0.05, 0.95, (40, 3))
    t = rng.uniform(0.0, 2.0, 40)
    c2 = inputs.c2_config_small
    g = inputs.manufactured_forcing(c2)(x)

    def p(x, t):
        s = np.sin(np.pi * x)
        return s[:, 0] * s[:, 1] * s[:, 2] * np.cos(np.pi * t)

    def u(x, t):
        s, c = np.sin(np.pi * x), np.cos(np.pi * x)
        return -np.stack([c[:, 0] * s[:, 1] * s[:, 2], s[:, 0] * c[:, 1] * s[:, 2],
                          s[:, 0] * s[:, 1] * c[:, 2]], 1) * np.sin(np.pi * t)[:, None]

    h = 1e-5
    pt = (p(x, t + h) - p(x, t - h)) / (2 * h)
    div = sum((u(x + h * np.eye(3)[i], t)[:, i] - u(x - h * np.eye(3)[i], t)[:, i]) / (2 * h) for i in range(3))
    assert np.allclose(pt / c2(x) + div, g * np.sin(np.pi * t), atol=1e-8)
    ut = (u(x, t + h) - u(x, t - h)) / (2 * h)
    gp = np.stack([(p(x + h * np.eye(3)[i], t) - p(x - h * np.eye(3)[i], t)) / (2 * h) for i in range(3)], 1)
    assert np.allclose(ut + gp, 0.0, atol=1e-8)
