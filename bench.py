"""Throughput of the fused BBWADG LSRK stage on the FP32 sweep workload.

Workload (synthetic, seeded): the unit cube cut into 32^3 hexes x 6 = 196,608
affine tetrahedra, degrees N = 1..9, c^2 of degree M = 2 (a smooth random
medium in [0.5, 2] with a planar x1.5 layer jump cutting through elements,
sampled at the degree-2 domain points), a 10 Hz Ricker point source at the
cube centre, Gaussian initial pressure.

One bench step = one full LSRK4 step (5 stages) for each of the nine degrees,
interleaved by stage (stage s for N = 1..9, then s+1), so every stage kernel
starts with the other degrees' data (>= 6 GB) having streamed through the
129 MB L2. The metric is DOF-updates per second per RK stage,
4 K N_p / t_stage, aggregated over the sweep (sum of DOF updates / sum of
kernel time); per-degree values are in ``sweep``.

``--impl reference`` times the FP64 CPU oracle (one stage per degree on a
bounded sub-mesh per step) on the host cores instead.

``--workload batched`` measures the batched form instead: 256 seeded
instances (cube refinements of 2k-60k tets, N in 3..7, M = 2, FP32, one medium
and Ricker source per instance) advanced together by graph-replayed batch
steps, against the same instances stepped one after another by solo solvers
("plain"); the line reports the speedup, both throughputs and the largest
relative L2 difference between the two final states.

``--workload elastic`` measures the elastic stage kernel (the velocity-stress
system of Sec. 2.2, nine fields, matrix-weighted update) on the same mesh:
N = 1..9, M = 2 media (rho^{-1}, lambda, mu from seeded smooth random fields),
a Gaussian compressional pulse, interleaved by stage as above; the metric is
9 K N_p / t_stage. ``--impl reference --workload elastic`` times the FP64
elastic oracle on a sub-cube.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1808_08645_gb300 import inputs  # noqa: E402

METRIC = "DOF-updates/s per RK stage vs N"
UNIT = "DOF-updates/s"


def np3(n):
    return (n + 1) * (n + 2) * (n + 3) // 6


def algorithmic_bytes_per_element(N: int, M: int, real: int = 4) -> float:
    """Bytes one stage must move per element, averaged over the five stages.

    q_in read, q_out and res written (12 N_p values) on every stage; res read
    (4 N_p) on stages 1-4 only (a_0 = 0); c^2 (M_p values), geometry (9 values)
    and the packed connectivity (16 B). Neighbour traces are re-reads of q_in
    and not counted.
    """
    vals = (12 + 4 * 4 / 5) * np3(N) + np3(M) + 9
    return vals * real + 16


def elastic_bytes_per_element(N: int, M: int, real: int = 4) -> float:
    """Bytes one elastic stage must move per element, averaged over the five
    stages: q_in read, q_out and res written (27 N_p values), res read
    (9 N_p) on stages 1-4, the three media polynomials (3 M_p values),
    geometry (9 values) and the packed connectivity (16 B)."""
    vals = (27 + 9 * 4 / 5) * np3(N) + 3 * np3(M) + 9
    return vals * real + 16


# ---------------------------------------------------------------------------
# clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs),
                "reasons": sorted(reasons), "samples": len(sms)}


# ---------------------------------------------------------------------------
# GPU arm

def make_c2(M: int, vxyz, etov, c2_field):
    """(c2, recipe) of the sweep workload: the L2 projection of the medium onto
    P^M per element, every Bernstein coefficient checked positive (tools
    layer). On meshes where the projection of the layer jump undershoots
    below zero (coarser than the default 32^3 hexes, e.g. 16^3), the medium
    is sampled at the domain points instead, and the recipe says so."""
    from paper_1808_08645_gb300 import project
    try:
        return project.project_c2(vxyz, etov, M, c2_field), "L2 projection onto P^M"
    except project.NonPositiveC2:
        return (inputs.sample_at_domain_points(vxyz, etov, M, c2_field),
                "sampled at the domain points (the L2 projection has a coefficient <= 0 on this mesh)")


def make_workload(N: int, M: int, vxyz, etov, c2, pulse):
    """(c2, q0): the projected c^2 and the initial pulse (sampled at the
    domain points: the throughput does not depend on it)."""
    K = len(etov)
    q0 = np.zeros((4, K, np3(N)))
    q0[0] = inputs.sample_at_domain_points(vxyz, etov, N, pulse)
    return c2, q0


def run_gpu(args):
    import torch

    from paper_1808_08645_gb300 import binding as B
    from paper_1808_08645_gb300 import build as libbuild

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        libbuild.build()
    if dist is not None:
        dist.barrier()

    cfg = inputs.SWEEP_CONFIG
    Ns = [int(x) for x in args.Ns.split(",")]
    M = cfg["M"]
    vxyz, etov = inputs.cube_mesh(args.hexes)
    K = len(etov)
    field = inputs.c2_smooth_random(seed=0)
    pulse = inputs.gaussian_pulse()
    stream = torch.cuda.Stream()
    solvers, host_q0 = {}, {}
    c2p, c2_recipe = make_c2(M, vxyz, etov, field)
    for N in Ns:
        c2, q0 = make_workload(N, M, vxyz, etov, c2p, pulse)
        s = B.Solver(vxyz, etov, N, M, B.F32, stream=stream.cuda_stream)
        s.set_c2(c2)
        s.set_state(q0)
        solvers[N] = s
        host_q0[N] = q0
    dts = {N: solvers[N].cfl_dt(0.5) for N in Ns}
    # the Ricker source's amplitude samples, one per stage, for every step the
    # bench runs (warm-up, timed, end to end)
    horizon = args.warmup + args.steps + args.e2e_steps + 1
    for N in Ns:
        solvers[N].set_point_source(np.array(cfg["source"]), B.ricker_samples(dts[N], horizon, f0=cfg["f0"]))

    def sweep_step(events=None):
        for st in range(5):
            for N in Ns:
                if events is not None:
                    events[N][st][0].record(stream)
                solvers[N].stage(st, dts[N])
                if events is not None:
                    events[N][st][1].record(stream)

    # warm-up
    for _ in range(args.warmup):
        sweep_step()
    torch.cuda.synchronize()

    ev = [{N: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(5)] for N in Ns} for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for k in range(args.steps):
        sweep_step(ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    for s in solvers.values():
        s.sync()  # surfaces any asynchronous error (e.g. a non-finite state)

    total_ms = t0.elapsed_time(t1)
    kern_ms = {N: [sum(ev[k][N][st][0].elapsed_time(ev[k][N][st][1]) for st in range(5))
                   for k in range(args.steps)] for N in Ns}
    dof_stage = {N: 4 * K * np3(N) for N in Ns}
    per_n = {}
    for N in Ns:
        t_stage = statistics.median(kern_ms[N]) / 5 / 1e3
        per_n[str(N)] = {"dof_updates_per_s": dof_stage[N] / t_stage,
                         "us_per_stage": t_stage * 1e6,
                         "achieved_gbs": algorithmic_bytes_per_element(N, M) * K / t_stage / 1e9}
    dofs_total = sum(5 * dof_stage[N] for N in Ns) * args.steps
    total_ms, value = aggregate_ranks(total_ms, dofs_total, dist, device="cuda")

    # dominant kernel: the largest share of kernel time
    top = max(Ns, key=lambda N: statistics.median(kern_ms[N]))
    t_launch = statistics.mean([x / 5 for x in kern_ms[top]]) / 1e3  # mean launch, seconds
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = algorithmic_bytes_per_element(top, M) * K / t_launch / 1e9
    traffic = load_traffic(top, K)

    # end to end through the public API with host buffers
    e2e = run_e2e(solvers, host_q0, Ns, dts, K, args.e2e_steps, stream)

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": f"BBWADG acoustic LSRK4 stage sweep, {args.hexes}^3 hexes x 6 = {K} "
                            f"affine tets, N={Ns[0]}..{Ns[-1]}, M={M}, smooth random c2 in [0.5,2] "
                            "with planar layer jump, Ricker point source",
                "mesh_elements": K, "Ns": Ns, "M": M, "c2": c2_recipe,
                "step": "one LSRK4 step (5 stages) per degree, interleaved by stage",
                "l2": "inputs larger than L2: between two stages of one degree the other "
                      "degrees stream >= 6 GB through the 129 MB L2",
                "parallelism": f"replicas x{world}",
            },
            "sweep": per_n,
            "roofline": {"bound": "hbm", "kernel": f"stage_kernel N={top} M={M} f32",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                                         "(RK stages 1-2, which read res) from the committed summary; "
                                         "null once the kernel sources change",
                         "algorithmic_bytes_per_launch": algorithmic_bytes_per_element(top, M) * K,
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"},
            "e2e": e2e,
            "gpu_launches": 5 * len(Ns) * args.steps,
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args)
    for s in solvers.values():
        s.close()
    if dist is not None:
        dist.destroy_process_group()
    return out


def aggregate_ranks(local_ms: float, local_units: float, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: every rank processed
    ``local_units`` in ``local_ms``; the job time is the maximum over ranks
    and the value is the units of all ranks over that time. Returns
    (job_ms, value). ``dist`` is torch.distributed (or None for one rank)."""
    if dist is not None:
        import torch
        t = torch.tensor([float(local_ms), float(local_units)], dtype=torch.float64, device=device)
        u = t[1:].clone()
        dist.all_reduce(t[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        local_ms, units = float(t[0].item()), float(u[0].item())
    else:
        units = float(local_units)
    return local_ms, units / (local_ms / 1e3)


def run_e2e(solvers, host_q0, Ns, dts, K, steps, stream):
    """Upload the initial state from pinned host memory, run ``steps`` RK
    steps, read the final state back into pinned host memory, per degree;
    wall-clock timed."""
    import torch
    pinned_in, pinned_out = {}, {}
    for N in Ns:
        n = host_q0[N].size
        pinned_in[N] = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        pinned_in[N][:] = host_q0[N].ravel()
        pinned_out[N] = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        pinned_out[N][:] = 0.0
    torch.cuda.synchronize()
    t = time.perf_counter()
    h2d = d2h = 0
    for N in Ns:
        s = solvers[N]
        s.set_state(pinned_in[N])
        s.step(dts[N], steps)
        s.get_state(out=pinned_out[N])
        h2d += pinned_in[N].nbytes
        d2h += pinned_out[N].nbytes
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    dofs = sum(5 * steps * 4 * K * np3(N) for N in Ns)
    return {"value": dofs / wall, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps,
            "note": f"per degree: bbw_set_state from pinned host FP64 (copied as is, regrouped and rounded "
                    f"to FP32 on the device), {steps} RK steps, bbw_get_state into pinned host FP64; "
                    "bytes per step amortised over the run"}


# the sources that decide the stage kernel's memory traffic: the kernel and
# its tables, and the host code that lays out and orders the elements
KERNEL_SOURCES = ("bbw_stage.cuh", "bbw_common.h", "bbw_stage_inst.cuh", "bbw_api.cu")
# the same for the elastic stage kernel
ELASTIC_SOURCES = ("bbw_elastic.cuh", "bbw_stage.cuh", "bbw_common.h", "bbw_elastic_inst.cuh",
                   "bbw_elastic.cu", "bbw_api.cu")


def sources_sha256(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1808_08645_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_sources_sha256() -> str:
    return sources_sha256(KERNEL_SOURCES)


def _traffic_from_profiles(pattern: str, N: int, sha: str, K=None):
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", pattern))):
        with open(path) as fh:
            for line in fh:
                if line.startswith("machine-readable:"):
                    try:
                        data = json.loads(line.split(":", 1)[1])
                    except ValueError:
                        continue
                    if K is not None and data.get("K", K) != K:
                        continue  # captured on another mesh
                    if data.get("N") == N and data.get("kernel_sources_sha256") == sha:
                        return float(data["traffic_bytes_per_launch"])
    return None


def load_traffic(N: int, K=None):
    """DRAM bytes per launch of the degree-N stage kernel from a committed ncu
    summary (profiles/stage_kernel_n<N>_*dram_traffic.md, its
    ``machine-readable:`` line). None when there is no capture for N (on a
    mesh of K elements, if K is given) or when the kernel sources changed
    since the counters were taken."""
    return _traffic_from_profiles(f"stage_kernel_n{N}_*dram_traffic.md", N, kernel_sources_sha256(), K)


def load_elastic_traffic(N: int, K=None):
    """As load_traffic, for the elastic stage kernel
    (profiles/elastic_stage_kernel_n<N>_*dram_traffic.md)."""
    return _traffic_from_profiles(f"elastic_stage_kernel_n{N}_*dram_traffic.md", N,
                                  sources_sha256(ELASTIC_SOURCES), K)


# ---------------------------------------------------------------------------
# CPU oracle arms

def _oracle_stage_times():
    from oracle.acoustic import lsrk_stage_times
    return [float(c) for c in lsrk_stage_times()]


def _oracle_sample(hexes: int, Ns, reps: int):
    """Time one oracle stage per degree on a hexes^3 x 6 sub-mesh; returns
    (DOF updates, seconds)."""
    from oracle.acoustic import AcousticOracle
    cfg = inputs.SWEEP_CONFIG
    vxyz, etov = inputs.cube_mesh(hexes)
    field = inputs.c2_smooth_random(seed=0)
    pulse = inputs.gaussian_pulse()
    K = len(etov)
    dofs, secs = 0, 0.0
    # the medium projected onto this coarser sub-cube (the oracle takes any
    # c^2; on elements this large the layer jump can undershoot below zero)
    from paper_1808_08645_gb300 import project
    c2p = project.l2_project(vxyz, etov, cfg["M"], field, q=cfg["M"] + 4)
    for N in Ns:
        c2, q0 = make_workload(N, cfg["M"], vxyz, etov, c2p, pulse)
        orc = AcousticOracle(vxyz, etov, N, cfg["M"], c2)
        orc.set_point_source(np.array(cfg["source"]),
                             inputs.ricker_samples(cfg["f0"], 1.0 / cfg["f0"], 1e-4, reps, _oracle_stage_times()))
        res = np.zeros_like(q0)
        orc.stage(q0, res, 0, 1e-4)  # warm caches
        t = time.perf_counter()
        q, r = q0, res
        for i in range(reps):
            q, r = orc.stage(q, r, i % 5, 1e-4, i // 5)
        secs += time.perf_counter() - t
        dofs += reps * 4 * K * np3(N)
    return dofs, secs


def cpu_baseline(args):
    """The FP64 oracle on one host core, in a fresh process (spawned)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    Ns = [int(x) for x in args.Ns.split(",")]
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"d, s = bench._oracle_sample({args.cpu_hexes}, {Ns!r}, {args.cpu_reps}); print(json.dumps([d, s]))")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if p.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "failed: " + p.stderr.strip().splitlines()[-1] if p.stderr else "failed"}
    d, s = json.loads(p.stdout.strip().splitlines()[-1])
    K = 6 * args.cpu_hexes ** 3
    out = {"value": d / s, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{args.cpu_reps} FP64 oracle stages per degree N={Ns[0]}..{Ns[-1]} on the "
                     f"{args.cpu_hexes}^3 x 6 = {K}-tet sub-cube of the same workload "
                     f"(same c2 field, source, pulse); {s:.1f} s of CPU work, 1 thread"}
    out["all_cores"] = cpu_baseline_all_cores(code, env)
    return out


def cpu_baseline_all_cores(code: str, env: dict):
    """The same sample in nproc concurrent single-threaded oracle processes
    (the oracle is not parallel; replicas use every host core): total
    DOF-updates over the slowest process's time."""
    cores = os.cpu_count() or 1
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=env) for _ in range(cores)]
    dofs, worst = 0, 0.0
    for p in procs:
        out, err = p.communicate(timeout=1800)
        if p.returncode != 0:
            return {"value": None, "cores": cores, "note": "failed: " + (err.strip().splitlines() or [""])[-1]}
        d, s = json.loads(out.strip().splitlines()[-1])
        dofs += d
        worst = max(worst, s)
    return {"value": dofs / worst, "unit": UNIT, "cores": cores,
            "note": f"{cores} concurrent single-threaded oracle processes (os.cpu_count) on the same sample; "
                    "total DOF-updates / slowest process time"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    Ns = [int(x) for x in args.Ns.split(",")]
    for _ in range(args.warmup):
        _oracle_sample(args.ref_hexes, Ns, 1)
    per = []
    dofs_total, secs_total = 0, 0.0
    for _ in range(args.steps):
        d, s = _oracle_sample(args.ref_hexes, Ns, 1)
        dofs_total += d
        secs_total += s
        per.append(s)
    value = dofs_total / secs_total
    K = 6 * args.ref_hexes ** 3
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"FP64 oracle: one stage per degree N={Ns[0]}..{Ns[-1]} on the "
                               f"{args.ref_hexes}^3 x 6 = {K}-tet sub-cube of the sweep workload",
                   "Ns": Ns, "M": inputs.SWEEP_CONFIG["M"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{K}-tet sub-cube, one stage per degree per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_batched(args):
    """Batched instances against plain one-by-one solving on the same GPU."""
    import torch

    from paper_1808_08645_gb300 import binding as B
    from paper_1808_08645_gb300 import build as libbuild

    libbuild.build()
    cfg = inputs.BATCH_CONFIG
    M = cfg["M"]
    specs = inputs.batched_instances(args.instances)
    meshes, c2s = [], []
    cache = {}
    for d in specs:
        if d["hexes"] not in cache:
            cache[d["hexes"]] = inputs.cube_mesh(d["hexes"])
        vxyz, etov = cache[d["hexes"]]
        meshes.append((vxyz, etov))
        c2s.append(inputs.sample_at_domain_points(vxyz, etov, M, inputs.c2_smooth_random(seed=d["c2_seed"])))
    Ns = [d["N"] for d in specs]
    stream = torch.cuda.Stream()
    t_setup = time.perf_counter()
    batch = B.Batch(meshes, Ns, M, B.F32, stream=stream.cuda_stream)
    solos = []
    for i, d in enumerate(specs):
        batch.set_c2(i, c2s[i])
        s = B.Solver(meshes[i][0], meshes[i][1], d["N"], M, B.F32, stream=stream.cuda_stream)
        s.set_c2(c2s[i])
        solos.append(s)
    dt = batch.cfl_dt(cfg["cfl"])
    amp = B.ricker_samples(dt, 4 * (args.warmup + args.steps) + 16, f0=cfg["f0"])
    for i, d in enumerate(specs):
        batch.set_point_source(i, d["source"], amp)
        solos[i].set_point_source(d["source"], amp)
    t_setup = time.perf_counter() - t_setup
    schedule, tuned_ms = batch.autotune(3)
    dofs_step = sum(5 * 4 * len(m[1]) * np3(N) for m, N in zip(meshes, Ns))

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            fn(steps)
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def run_batch(n):
        batch.step(dt, n, graph=True)

    def run_plain(n):
        for s in solos:
            s.step(dt, n)

    clk = ClockSampler(torch.cuda.current_device())
    timed(run_batch, args.warmup)
    timed(run_plain, args.warmup)
    clk.start()
    ms_batch = timed(run_batch, args.steps)
    ms_plain = timed(run_plain, args.steps)
    clocks = clk.stop()
    batch.sync()
    err = 0.0
    for i, s in enumerate(solos):
        qb = batch.get_state(i)
        qs, _ = s.get_state()
        err = max(err, float(np.linalg.norm(qb - qs) / max(np.linalg.norm(qs), 1e-300)))
    n, nbuckets, elements = batch.info()
    for s in solos:
        s.close()
    to_T = _batched_to_time(batch, specs, meshes, Ns, dt, cfg, timed, max(args.steps, 20) * dt, B)
    batch.close()
    value_b = dofs_step * args.steps / (ms_batch / 1e3)
    value_p = dofs_step * args.steps / (ms_plain / 1e3)
    return {
        "metric": "batched speedup vs plain BBWADG at L2 tolerance", "impl": "ours", "workload": "batched",
        "value": ms_plain / ms_batch, "unit": "x", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_batch / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{n} instances, cube refinements of {min(len(m[1]) for m in meshes)}-"
                               f"{max(len(m[1]) for m in meshes)} tets ({sum(len(m[1]) for m in meshes)} "
                               f"in total), N in 3..7, M=2, per-instance seeded c2 and Ricker source, "
                               f"common CFL dt", "buckets": nbuckets, "elements_with_padding": elements,
                   "l2": "inputs larger than L2 (tens of GB of state)"},
        "batched": {"dof_updates_per_s": value_b, "ms_per_step": ms_batch / args.steps,
                    "launch": "one CUDA graph per step: 5 persistent stage launches per degree bucket",
                    "schedule": {0: "concurrent branches, solo grids", 1: "buckets in sequence, solo grids",
                                 2: "concurrent branches, half grids",
                                 3: "concurrent branches, double grids"}.get(schedule, str(schedule)),
                    "autotune_ms_per_step": tuned_ms},
        "plain": {"dof_updates_per_s": value_p, "ms_per_step": ms_plain / args.steps,
                  "launch": "one solo solver per instance, bbw_step per instance, one after another"},
        "max_rel_l2_batched_vs_plain": err,
        "to_time_T": to_T,
        "gpu_launches": 5 * nbuckets * args.steps + args.steps,
        "setup_s": t_setup, "clocks": clocks,
    }


def _batched_to_time(batch, specs, meshes, Ns, dt, cfg, timed, T, B):
    """Every instance from rest to time T: with the batch's common (smallest)
    CFL step, and with each instance's own CFL step and step count
    (bbw_batch_set_instance_steps); each source sampled at its own stage
    times. Returns the two times, the DOF-updates each needs and the largest
    relative L2 difference of the final states (the two dt's discretisation
    errors)."""
    import math
    n = len(specs)
    Np = [np3(N) for N in Ns]
    K = [len(m[1]) for m in meshes]

    def start(dts, steps):
        batch.set_instance_steps(dts, steps)
        for i, d in enumerate(specs):
            batch.set_state(i, np.zeros((4, K[i], Np[i])))
            h = dt if dts is None else dts[i]
            batch.set_point_source(i, d["source"], B.ricker_samples(h, int(math.ceil(T / h)) + 1, f0=cfg["f0"]))
        batch.set_time(0.0)

    n_common = int(math.ceil(T / dt))
    start(None, None)
    ms_common = timed(lambda k: batch.step(dt, k, graph=True), n_common)
    q_common = [batch.get_state(i) for i in range(n)]
    own = np.array([batch.member_cfl_dt(i, cfg["cfl"]) for i in range(n)])
    steps = np.ceil(T / own).astype(np.int64)
    dts = T / steps
    start(dts, steps)
    ms_own = timed(lambda k: batch.step(dt, k, graph=True), int(steps.max()))
    diff = max(float(np.linalg.norm(batch.get_state(i) - q_common[i]) / max(np.linalg.norm(q_common[i]), 1e-300))
               for i in range(n))
    batch.set_instance_steps(None, None)
    per = [5 * 4 * K[i] * Np[i] for i in range(n)]
    return {"T": T, "common_dt": {"ms": ms_common, "steps": n_common,
                                  "dof_updates": sum(per) * n_common},
            "own_dt": {"ms": ms_own, "steps_min": int(steps.min()), "steps_max": int(steps.max()),
                       "dof_updates": int(sum(p * k for p, k in zip(per, steps)))},
            "speedup": ms_common / ms_own, "max_rel_l2_final_states": diff}


def run_adjoint(args):
    """Receiver-misfit gradient with respect to c^2 on the adjoint workload:
    forward steps alone, the recorded forward run (checkpoints, traces) and
    the adjoint sweep, timed on the solver's stream."""
    import torch

    from paper_1808_08645_gb300 import binding as B
    from paper_1808_08645_gb300 import build as libbuild

    libbuild.build()
    cfg = inputs.ADJOINT_CONFIG
    N, M = cfg["N"], cfg["M"]
    nsteps = args.adjoint_steps
    vxyz, etov = inputs.cube_mesh(cfg["hexes"])
    K = len(etov)
    # media sampled at the domain points: on this mesh the L2 projection of the
    # seed-0 medium undershoots below zero next to its layer jump
    c2_true = inputs.sample_at_domain_points(vxyz, etov, M, inputs.c2_smooth_random(seed=cfg["true_seed"]))
    c2 = inputs.sample_at_domain_points(vxyz, etov, M, inputs.c2_smooth_random(seed=cfg["model_seed"]))
    rec = inputs.top_face_receivers()
    stream = torch.cuda.Stream()
    s = B.Solver(vxyz, etov, N, M, B.F32, stream=stream.cuda_stream)
    s.set_receivers(rec)
    q0 = np.zeros((4, K, np3(N)))
    s.set_c2(c2_true)
    s.set_state(q0)
    dt = s.cfl_dt(cfg["cfl"])
    s.set_c2(c2)
    dt = min(dt, s.cfl_dt(cfg["cfl"]))
    s.set_point_source(np.array(cfg["source"]), B.ricker_samples(dt, nsteps, f0=cfg["f0"]))
    every = max(1, int(round(np.sqrt(nsteps))))

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, out

    # data: traces of the true medium
    s.set_c2(c2_true)
    s.set_state(q0)
    data = s.record(dt, nsteps, every)
    # warm-up (one checkpoint segment of record + adjoint: first-use set-up of
    # the adjoint's buffers and of cuBLAS), then forward alone
    s.set_c2(c2)
    s.set_state(q0)
    s.step(dt, 3)
    s.set_state(q0)
    s.record(dt, every, every)
    s.adjoint(np.zeros((every, len(rec))))
    s.set_state(q0)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    t_fwd, _ = timed(lambda: s.step(dt, nsteps))
    s.set_state(q0)
    t_rec, tr = timed(lambda: s.record(dt, nsteps, every))
    resid = tr - data
    t_adj, (gc, _) = timed(lambda: s.adjoint(resid))
    # every stage's pressure bracket kept in HBM (5 nsteps pressure fields):
    # the adjoint recomputes nothing (warm-up record: the buffer's allocation)
    s.set_state(q0)
    s.record(dt, nsteps, 0)
    s.set_state(q0)
    t_rec0, tr0 = timed(lambda: s.record(dt, nsteps, 0))
    t_adj0, (gc0, _) = timed(lambda: s.adjoint(tr0 - data))
    clocks = clk.stop()
    s.close()
    dofs = 4 * K * np3(N) * 5 * nsteps
    kept_gb = 5 * nsteps * K * np3(N) * 4 / 1e9
    return {
        "metric": "receiver-misfit gradient w.r.t. c2: time relative to the forward run", "impl": "ours",
        "workload": "adjoint", "value": (t_rec0 + t_adj0) / t_fwd, "unit": "x forward time", "n_gpus": 1,
        "steps": nsteps, "warmup": 3, "ms_per_step": 1e3 * (t_rec0 + t_adj0) / nsteps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{cfg['hexes']}^3 hexes x 6 = {K} tets, N={N}, M={M}, {len(rec)} receivers on "
                               f"the top face, {nsteps} steps, every stage's pressure bracket kept "
                               f"({kept_gb:.1f} GB of HBM), Ricker source "
                               f"at {tuple(cfg['source'])}, data from the seed-{cfg['true_seed']} medium, "
                               f"model the seed-{cfg['model_seed']} medium", "dt": dt},
        "forward_s": t_fwd, "record_s": t_rec0, "adjoint_s": t_adj0,
        "forward_dof_updates_per_s": dofs / t_fwd, "adjoint_dof_updates_per_s": dofs / t_adj0,
        "checkpointed": {"checkpoint_every": every, "record_s": t_rec, "adjoint_s": t_adj,
                         "x_forward": (t_rec + t_adj) / t_fwd,
                         "bitwise_equal_gradient": bool(np.array_equal(gc, gc0))},
        "misfit": 0.5 * float(np.sum(resid ** 2)), "grad_norm": float(np.linalg.norm(gc0)),
        "timing": "wall clock around each call with device synchronisation (each call ends with a device wait)",
        "clocks": clocks,
    }


# ---------------------------------------------------------------------------
# elastic workload

def _elastic_setup(hexes: int, N: int, M: int):
    vxyz, etov = inputs.cube_mesh(hexes)
    media = inputs.elastic_media(vxyz, etov, M, seed=inputs.ELASTIC_CONFIG["seed"])
    return vxyz, etov, media, inputs.elastic_pulse(vxyz, etov, N)


def _elastic_oracle_sample(hexes: int, Ns, reps: int):
    """Time `reps` FP64 elastic oracle stages per degree on a hexes^3 x 6
    sub-cube; returns (DOF updates, seconds)."""
    from oracle.elastic import ElasticOracle
    M = inputs.ELASTIC_CONFIG["M"]
    dofs, secs = 0, 0.0
    for N in Ns:
        vxyz, etov, media, q0 = _elastic_setup(hexes, N, M)
        orc = ElasticOracle(vxyz, etov, N, M, *media)
        res = np.zeros_like(q0)
        orc.stage(q0, res, 0, 1e-4)  # warm caches
        t = time.perf_counter()
        q, r = q0, res
        for i in range(reps):
            q, r = orc.stage(q, r, i % 5, 1e-4)
        secs += time.perf_counter() - t
        dofs += reps * 9 * len(etov) * np3(N)
    return dofs, secs


def elastic_cpu_baseline(args):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    Ns = [int(x) for x in args.Ns.split(",")]
    hexes, reps = 3, 15  # about 10 s of FP64 work on the GPU machine's host cores
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"d, s = bench._elastic_oracle_sample({hexes}, {Ns!r}, {reps}); print(json.dumps([d, s]))")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if p.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "failed: " + p.stderr.strip().splitlines()[-1] if p.stderr else "failed"}
    d, s = json.loads(p.stdout.strip().splitlines()[-1])
    return {"value": d / s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} FP64 elastic oracle stages per degree N={Ns[0]}..{Ns[-1]} on the "
                      f"{hexes}^3 x 6 = {6 * hexes ** 3}-tet sub-cube of the same workload (same media "
                      f"recipe and pulse); {s:.1f} s of CPU work, 1 thread"}


def run_elastic_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return None
    Ns = [int(x) for x in args.Ns.split(",")]
    hexes = 2
    for _ in range(args.warmup):
        _elastic_oracle_sample(hexes, Ns, 1)
    dofs_total, secs_total = 0, 0.0
    for _ in range(args.steps):
        d, s = _elastic_oracle_sample(hexes, Ns, 1)
        dofs_total += d
        secs_total += s
    value = dofs_total / secs_total
    K = 6 * hexes ** 3
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"FP64 elastic oracle: one stage per degree N={Ns[0]}..{Ns[-1]} on the "
                               f"{hexes}^3 x 6 = {K}-tet sub-cube of the elastic workload",
                   "Ns": Ns, "M": inputs.ELASTIC_CONFIG["M"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{K}-tet sub-cube, one stage per degree per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _meta_rows(meta: dict, n: int) -> dict:
    return dict(meta, gain=meta["gain"][:n], shift=meta["shift"][:n])


def run_surrogate(args):
    """The neural-operator surrogate: BBWADG runs generate the training and
    held-out data, the network is trained by the library's kernels, and its
    trace error on held-out runs (measured against BBWADG) and its inference time
    are reported against plain BBWADG."""
    import torch

    from paper_1808_08645_gb300 import binding as B
    from paper_1808_08645_gb300 import build as libbuild
    from paper_1808_08645_gb300 import surrogate as S

    libbuild.build()
    dcfg = dict(inputs.SURROGATE_CONFIG, grid=args.sur_grid)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    t = time.perf_counter()
    X, Y, meta = S.generate(dcfg, 0, args.sur_runs)
    Xt, Yt, mt = S.generate(dcfg, args.sur_runs, args.sur_test)
    t_gen = time.perf_counter() - t
    A = S.encode(Y, meta)
    scale = float(A.std())
    net = S.Net(S.default_config(grid=dcfg["grid"], nt=Y.shape[2], rec_z=dcfg["rec_z"]), seed=0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    losses = S.train(net, X, A, args.sur_iters, scale=scale, lr=args.sur_lr, log_every=max(1, args.sur_iters // 20))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t
    pred = S.predict(net, Xt, scale, mt)
    err = S.relative_errors(pred, Yt)
    # device time per run: the network (forward + decode, batches of 8, CUDA
    # events) against one BBWADG time integration (record of a prepared solver)
    xb = Xt[:8].contiguous()
    m8 = _meta_rows(mt, 8)

    def infer(x, m):
        y, _ = net.forward(x)
        return S.decode(y * scale, m)

    for _ in range(3):
        infer(xb, m8)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 10
    for _ in range(reps):
        infer(xb, m8)
    e1.record()
    e1.synchronize()
    t_nn = e0.elapsed_time(e1) / 1e3 / (reps * 8)
    vxyz, etov, rec, dt, amp = S._bbwadg_setup(dcfg)
    stream = torch.cuda.Stream()
    sol = B.Solver(vxyz, etov, dcfg["N"], dcfg["M"], B.F32, stream=stream.cuda_stream)
    sol.set_receivers(rec)
    run0 = inputs.surrogate_runs(args.sur_runs, 1, dcfg)[0]
    S.bbwadg_traces(sol, vxyz, etov, dcfg, run0, dt, amp)  # warm-up
    reps_b = 3
    t_rec = []
    for _ in range(reps_b):
        S.bbwadg_traces(sol, vxyz, etov, dcfg, run0, dt, amp, timings=t_rec)
    t_bbw = float(np.median(t_rec))
    # end to end per run from the run's description (medium seed, source) to
    # host traces: host features / coefficients, copies, device work
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps_b):
        S.bbwadg_traces(sol, vxyz, etov, dcfg, run0, dt, amp)
    t_bbw_e2e = (time.perf_counter() - t) / reps_b
    sol.close()
    runs8 = inputs.surrogate_runs(args.sur_runs, 8, dcfg)
    torch.cuda.synchronize()
    t = time.perf_counter()
    feats = np.stack([inputs.surrogate_features(inputs.c2_smooth_random(r["c2_seed"]), r["source"], dcfg["grid"],
                                                dcfg["sigma"]) for r in runs8])
    xh = torch.from_numpy(feats).pin_memory()
    m8e = S.run_meta(dcfg, runs8, [inputs.c2_smooth_random(r["c2_seed"]) for r in runs8], rec, meta["dt"])
    out8 = infer(xh.to("cuda", non_blocking=True), m8e).cpu()
    t_nn_e2e = (time.perf_counter() - t) / 8
    h2d = xh.numel() * 4 / 8
    d2h = out8.numel() * 4 / 8
    # the fallback: a run outside the training box goes to BBWADG
    c2min = float(X[..., 0].min()) * 0.75 + 1.25
    c2max = float(X[..., 0].max()) * 0.75 + 1.25
    sur = S.Surrogate(net, dcfg, scale, float(np.quantile(err, 0.95)), (c2min, c2max), meta["dt"])
    out_run = dict(run0, source=np.array([0.5, 0.5, 0.3]))
    _, used_out, _ = sur.predict(out_run)
    _, used_in, _ = sur.predict(run0, tol=float(np.quantile(err, 0.95)))
    clocks = clk.stop()
    return {
        "metric": "surrogate speedup vs plain BBWADG @ receiver-trace L2 error", "impl": "ours",
        "workload": "surrogate", "value": t_bbw / t_nn, "unit": "x (BBWADG run time / surrogate time per run)",
        "n_gpus": 1, "steps": args.sur_iters, "warmup": 3, "ms_per_step": 1e3 * t_train / max(args.sur_iters, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
        "data": "synthetic (BBWADG runs)",
        "config": {"workload": f"neural operator: c2 on a {dcfg['grid']}^3 grid + source xyz -> {len(rec)} "
                               f"receiver traces x {Y.shape[2]} samples; 4 spectral layers, width 32, "
                               f"{S.default_config()['modes']} cosine modes; trained on {args.sur_runs} BBWADG "
                               f"N={dcfg['N']} runs on {dcfg['hexes']}^3 x 6 tets, {args.sur_test} held out",
                   "iters": args.sur_iters, "batch": 8, "lr": args.sur_lr},
        "heldout_rel_l2": {"all_traces": float(((pred - Yt).double().norm() / Yt.double().norm()).item()),
                           "per_run_median": float(np.median(err)), "per_run_p95": float(np.quantile(err, 0.95)),
                           "per_run_max": float(np.max(err))},
        "train_runs_rel_l2_all_traces": float(((S.predict(net, X[:256], scale, _meta_rows(meta, 256)) - Y[:256])
                                                .double().norm()
                                                / Y[:256].double().norm()).item()),
        "e2e": {"value": t_bbw_e2e / t_nn_e2e, "unit": "x (per run, from the run's medium and source to host "
                                                         "traces, host preparation included on both sides)",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "time_s": {"bbwadg_run_device": t_bbw, "surrogate_per_run_device": t_nn, "bbwadg_run_e2e": t_bbw_e2e,
                   "surrogate_per_run_e2e": t_nn_e2e, "generate": t_gen, "train": t_train},
        "loss_curve": losses,
        "fallback": {"out_of_box_source": used_out, "in_box_at_p95_tol": used_in},
        "clocks": clocks,
    }


def run_elastic(args):
    import torch

    from paper_1808_08645_gb300 import binding as B
    from paper_1808_08645_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = inputs.ELASTIC_CONFIG
    M = cfg["M"]
    Ns = [int(x) for x in args.Ns.split(",")]
    vxyz, etov = inputs.cube_mesh(args.hexes)
    K = len(etov)
    media = inputs.elastic_media(vxyz, etov, M, seed=cfg["seed"])
    stream = torch.cuda.Stream()
    solvers = {}
    for N in Ns:
        s = B.ElasticSolver(vxyz, etov, N, M, B.F32, stream=stream.cuda_stream)
        s.set_media(*media)
        s.set_state(inputs.elastic_pulse(vxyz, etov, N))
        solvers[N] = s
    dts = {N: solvers[N].cfl_dt(cfg["cfl"]) for N in Ns}

    def sweep_step(events=None):
        for st in range(5):
            for N in Ns:
                if events is not None:
                    events[N][st][0].record(stream)
                solvers[N].stage(st, dts[N])
                if events is not None:
                    events[N][st][1].record(stream)

    for _ in range(args.warmup):
        sweep_step()
    torch.cuda.synchronize()
    ev = [{N: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(5)] for N in Ns} for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for k in range(args.steps):
        sweep_step(ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    for s in solvers.values():
        s.sync()
    total_ms = t0.elapsed_time(t1)
    kern_ms = {N: [sum(ev[k][N][st][0].elapsed_time(ev[k][N][st][1]) for st in range(5))
                   for k in range(args.steps)] for N in Ns}
    per_n = {}
    for N in Ns:
        t_stage = statistics.median(kern_ms[N]) / 5 / 1e3
        per_n[str(N)] = {"dof_updates_per_s": 9 * K * np3(N) / t_stage, "us_per_stage": t_stage * 1e6,
                         "achieved_gbs": elastic_bytes_per_element(N, M) * K / t_stage / 1e9}
    value = sum(5 * 9 * K * np3(N) for N in Ns) * args.steps / (total_ms / 1e3)
    top = max(Ns, key=lambda N: statistics.median(kern_ms[N]))
    t_launch = statistics.mean([x / 5 for x in kern_ms[top]]) / 1e3
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = elastic_bytes_per_element(top, M) * K / t_launch / 1e9

    # end to end, one degree at a time: pinned host FP64 in, steps, pinned host FP64 out
    e2e_steps = max(1, args.e2e_steps // 4)
    wall, h2d, d2h, dofs = 0.0, 0, 0, 0
    for N in Ns:
        q0 = inputs.elastic_pulse(vxyz, etov, N)
        pin_in = torch.empty(q0.size, dtype=torch.float64, pin_memory=True).numpy()
        pin_in[:] = q0.ravel()
        pin_out = torch.empty(q0.size, dtype=torch.float64, pin_memory=True).numpy()
        pin_out[:] = 0.0
        torch.cuda.synchronize()
        t = time.perf_counter()
        solvers[N].set_state(pin_in)
        solvers[N].step(dts[N], e2e_steps)
        solvers[N].get_state(out=pin_out)
        torch.cuda.synchronize()
        wall += time.perf_counter() - t
        h2d += pin_in.nbytes
        d2h += pin_out.nbytes
        dofs += 5 * e2e_steps * 9 * K * np3(N)
        del pin_in, pin_out
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": f"BBWADG elastic (velocity-stress, 9 fields) LSRK4 stage sweep, {args.hexes}^3 hexes "
                        f"x 6 = {K} affine tets, N={Ns[0]}..{Ns[-1]}, M={M}, smooth random rho, lambda, mu "
                        "with planar layer jump, Gaussian compressional pulse",
            "mesh_elements": K, "Ns": Ns, "M": M,
            "step": "one LSRK4 step (5 stages) per degree, interleaved by stage",
            "l2": "inputs larger than L2: between two stages of one degree the other degrees stream "
                  "several GB through the 129 MB L2",
            "parallelism": "replicas x1"},
        "sweep": per_n,
        "roofline": {"bound": "hbm", "kernel": f"elastic_stage_kernel N={top} M={M} f32",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": load_elastic_traffic(top, K),
                     "algorithmic_bytes_per_launch": elastic_bytes_per_element(top, M) * K,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"},
        "e2e": {"value": dofs / wall, "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_steps,
                "d2h_bytes_per_step": d2h / e2e_steps,
                "note": f"per degree: bbw_elastic_set_state from pinned host FP64, {e2e_steps} RK steps, "
                        "bbw_elastic_get_state into pinned host FP64"},
        "gpu_launches": 5 * len(Ns) * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = elastic_cpu_baseline(args)
    for s in solvers.values():
        s.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--Ns", default="1,2,3,4,5,6,7,8,9")
    ap.add_argument("--hexes", type=int, default=inputs.SWEEP_CONFIG["hexes"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-hexes", type=int, default=5)
    ap.add_argument("--cpu-reps", type=int, default=15)
    ap.add_argument("--ref-hexes", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["sweep", "batched", "adjoint", "elastic", "surrogate"], default="sweep")
    ap.add_argument("--sur-runs", type=int, default=inputs.SURROGATE_CONFIG["runs"])
    ap.add_argument("--sur-test", type=int, default=inputs.SURROGATE_CONFIG["test_runs"])
    ap.add_argument("--sur-iters", type=int, default=8000)
    ap.add_argument("--sur-grid", type=int, default=inputs.SURROGATE_CONFIG["grid"])
    ap.add_argument("--sur-lr", type=float, default=2e-3)
    ap.add_argument("--adjoint-steps", type=int, default=inputs.ADJOINT_CONFIG["steps"])
    ap.add_argument("--instances", type=int, default=inputs.BATCH_CONFIG["instances"])
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.workload == "adjoint":
        out = run_adjoint(args) if args.impl == "ours" else {
            "impl": "reference", "workload": "adjoint",
            "unavailable": "the FP64 oracle adjoint is dense (small meshes only); its check is in the tests"}
    elif args.workload == "surrogate":
        out = run_surrogate(args) if args.impl == "ours" else {
            "impl": "reference", "workload": "surrogate",
            "unavailable": "the surrogate's reference is plain BBWADG, timed in the same line"}
    elif args.workload == "batched":
        out = run_batched(args) if args.impl == "ours" else {
            "impl": "reference", "workload": "batched",
            "unavailable": "the batched form has no oracle counterpart; its reference is plain one-by-one "
                           "solving, reported in the same line"}
    elif args.workload == "elastic":
        out = run_elastic_reference(args) if args.impl == "reference" else run_elastic(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
