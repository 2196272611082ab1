"""Neural-operator surrogate of BBWADG: c^2 field + source position -> receiver traces.

The learned part (the paper has none): a Fourier-type neural operator on a
G^3 grid (G = 64, width 32, four spectral layers in a truncated orthonormal
cosine basis), a decoder that reads the top layer at the receivers, and two
dense layers to the trace samples. It is trained on runs of this library's
BBWADG solver, which also measures its error on held-out runs and is its
fallback (``Surrogate.predict``).

The contractions, forward and backward, are calls of ``bbw_nn_gemm`` (BF16
tensor cores, FP32 accumulation), except the transforms along z, the
innermost axis: they touch every grid value for a 64 -> 6 contraction and
run as FP32 pencil kernels (``bbw_nn_axis_transform``), bound by HBM. GELU
backward, bias gradients, the receiver gather and its transpose, the loss
and Adam are the library's other ``bbw_nn_*`` kernels. torch tensors only
hold device memory; this module is argument marshalling and the order of
the calls. The spectral transform of one layer is separable: one transform
per direction (z, y, x) with the truncated DCT-II matrices, one batched GEMM
over the modes for the mode weights, three transforms back.

Layouts: fields [B, X, Y, Z, C] (C fastest) viewed as a [B X Y Z, C] matrix;
modes [B, mx, my, mz, C]; receiver features [B, R, C]; traces [B, R, T].
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B

__all__ = ["Net", "default_config", "receiver_corners", "cosine_basis", "receiver_gain", "straight_ray_times",
           "encode", "decode", "run_meta", "generate", "train", "predict", "relative_errors", "Surrogate"]


def default_config(grid: int = 64, width: int = 32, modes=(6, 6, 6), layers: int = 4, cin: int = 6,
                   hidden: int = 128, nt: int = 512, receivers: int = 8, rec_z: float = 0.9) -> dict:
    rx, ry, rz = receiver_corners(grid, receivers, rec_z)
    return dict(grid=grid, width=width, modes=tuple(modes), layers=layers, cin=cin, hidden=hidden, nt=nt,
                rx=rx, ry=ry, rz=rz)


def receiver_corners(grid: int, n: int, z: float):
    """Lower grid corners of the 2 x 2 x 2 stencils around an n x n receiver
    grid at the cell centres (i + 1/2)/n of the plane at height z (grid
    points at (i + 1/2)/grid), x-major like ``inputs.surrogate_receivers``."""
    c = [int(math.floor(((i + 0.5) / n) * grid - 0.5)) for i in range(n)]
    zc = min(max(int(math.floor(z * grid - 0.5)), 0), grid - 2)
    rx = [a for a in c for _ in c]
    ry = [b for _ in c for b in c]
    return rx, ry, [zc] * len(rx)


def cosine_basis(n: int, m: int) -> np.ndarray:
    """[n, m] truncated orthonormal DCT-II basis c_k cos(pi k (i + 1/2) / n)."""
    i = np.arange(n)[:, None] + 0.5
    k = np.arange(m)[None, :]
    phi = np.cos(np.pi * k * i / n) * math.sqrt(2.0 / n)
    phi[:, 0] = math.sqrt(1.0 / n)
    return phi


def _ptr(t):
    return None if t is None else t.data_ptr()


def gemm(M, N, K, A, lda, sA, tA, Bm, ldb, sB, tB, Cm, ldc, sC, batch=1, alpha=1.0, beta=0.0, bias=None, pre=None,
         act=0, splits=1, stream=None):
    """bbw_nn_gemm on torch tensors (their data pointers; views keep their offset)."""
    B._check(B.lib().bbw_nn_gemm(M, N, K, A.data_ptr(), lda, sA, tA, Bm.data_ptr(), ldb, sB, tB, Cm.data_ptr(), ldc,
                                 sC, batch, alpha, beta, _ptr(bias), _ptr(pre), act, splits, stream),
             "bbw_nn_gemm")


def axis(basis, L, m, x, out, pencils, C, expand=0, beta=0.0, pre=None, act=0, stream=None):
    """bbw_nn_axis_transform: along the innermost spatial axis (FP32 pencils)."""
    B._check(B.lib().bbw_nn_axis_transform(basis.data_ptr(), L, m, x.data_ptr(), out.data_ptr(), pencils, C, expand,
                                           beta, _ptr(pre), act, stream), "bbw_nn_axis_transform")


def _splits(k: int) -> int:
    """K-splits of a weight-gradient GEMM: about 2048 rows per thread block."""
    return int(min(1024, max(1, k // 2048)))


class Net:
    """Parameters, forward, backward and Adam of the surrogate network on cuda."""

    def __init__(self, cfg: dict, params: dict | None = None, seed: int = 0, device: str = "cuda"):
        self.cfg = dict(cfg)
        self.dev = torch.device(device)
        G = cfg["grid"]
        mx, my, mz = cfg["modes"]
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.phi = [torch.tensor(cosine_basis(G, m), **f32).contiguous() for m in (mx, my, mz)]
        self.rx = torch.tensor(cfg["rx"], dtype=torch.int32, device=self.dev)
        self.ry = torch.tensor(cfg["ry"], dtype=torch.int32, device=self.dev)
        self.rz = torch.tensor(cfg["rz"], dtype=torch.int32, device=self.dev)
        if params is None:
            params = self.init_params(seed)
        self.p = {k: torch.tensor(np.asarray(v), **f32).contiguous() for k, v in params.items()}
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.steps = 0

    def init_params(self, seed: int) -> dict:
        cfg = self.cfg
        rng = np.random.default_rng(seed)
        C, cin, H, T, L = cfg["width"], cfg["cin"], cfg["hidden"], cfg["nt"], cfg["layers"]
        nm = int(np.prod(cfg["modes"]))
        p = {"W0": rng.uniform(-1, 1, (cin, C)) / math.sqrt(cin), "b0": np.zeros(C)}
        for l in range(L):
            p[f"W{l}_pw"] = rng.uniform(-1, 1, (C, C)) / math.sqrt(C)
            p[f"b{l}_pw"] = np.zeros(C)
            p[f"W{l}_sp"] = rng.uniform(-1, 1, (nm, C, C)) / C
        p["W1"] = rng.uniform(-1, 1, (C, H)) / math.sqrt(C)
        p["b1"] = np.zeros(H)
        p["W2"] = rng.uniform(-1, 1, (H, T)) / math.sqrt(H)
        p["b2"] = np.zeros(T)
        return p

    def numpy_params(self) -> dict:
        return {k: v.double().cpu().numpy() for k, v in self.p.items()}

    # -- the spectral convolution of layer l (forward), accumulated into out --
    def _spectral(self, l: int, u, out, pre, nb: int, cache: dict):
        cfg = self.cfg
        G, C = cfg["grid"], cfg["width"]
        mx, my, mz = cfg["modes"]
        nm = mx * my * mz
        Px, Py, Pz = self.phi
        e = dict(dtype=torch.float32, device=self.dev)
        s1 = torch.empty(nb * G * G * mz * C, **e)
        s2 = torch.empty(nb * G * my * mz * C, **e)
        s3 = torch.empty(nb * nm * C, **e)
        t3 = torch.empty(nb * nm * C, **e)
        # forward transform z, y, x: S = Phi^T u along each axis
        axis(Pz, G, mz, u, s1, nb * G * G, C)
        gemm(my, mz * C, G, Py, my, 0, 1, s1, mz * C, G * mz * C, 0, s2, mz * C, my * mz * C, batch=nb * G)
        gemm(mx, my * mz * C, G, Px, mx, 0, 1, s2, my * mz * C, G * my * mz * C, 0, s3, my * mz * C,
             mx * my * mz * C, batch=nb)
        # one C x C matrix per mode
        W = self.p[f"W{l}_sp"]
        gemm(nb, C, C, s3, nm * C, C, 0, W, C, C * C, 0, t3, nm * C, C, batch=nm)
        # back: x, y, z (the last one accumulates into out, adds GELU, keeps pre)
        t2 = torch.empty(nb * G * my * mz * C, **e)
        t1 = torch.empty(nb * G * G * mz * C, **e)
        gemm(G, my * mz * C, mx, Px, mx, 0, 0, t3, my * mz * C, nm * C, 0, t2, my * mz * C, G * my * mz * C,
             batch=nb)
        gemm(G, mz * C, my, Py, my, 0, 0, t2, mz * C, my * mz * C, 0, t1, mz * C, G * mz * C, batch=nb * G)
        axis(Pz, G, mz, t1, out, nb * G * G, C, expand=1, beta=1.0, pre=pre, act=1)
        cache[f"s3_{l}"] = s3

    def forward(self, x, cache: dict | None = None):
        """traces [nb, R, T] of inputs x [nb, G, G, G, cin] (float32 cuda)."""
        cfg = self.cfg
        G, C, L, H, T = cfg["grid"], cfg["width"], cfg["layers"], cfg["hidden"], cfg["nt"]
        R = len(cfg["rx"])
        nb = x.shape[0]
        P = nb * G ** 3
        cache = {} if cache is None else cache
        xin = x.reshape(P, cfg["cin"]).contiguous()
        e = dict(dtype=torch.float32, device=self.dev)
        u = torch.empty(P, C, **e)
        gemm(P, C, cfg["cin"], xin, cfg["cin"], 0, 0, self.p["W0"], C, 0, 0, u, C, 0, bias=self.p["b0"])
        cache["x"] = xin
        cache["u0"] = u
        for l in range(L):
            out = torch.empty(P, C, **e)
            pre = torch.empty(P, C, **e)
            gemm(P, C, C, u, C, 0, 0, self.p[f"W{l}_pw"], C, 0, 0, out, C, 0, bias=self.p[f"b{l}_pw"])
            self._spectral(l, u, out, pre, nb, cache)
            cache[f"pre{l}"] = pre
            u = out
            cache[f"u{l + 1}"] = u
        r = torch.empty(nb * R, C, **e)
        B._check(B.lib().bbw_nn_gather_receivers(u.data_ptr(), r.data_ptr(), self.rx.data_ptr(), self.ry.data_ptr(),
                                                 self.rz.data_ptr(), nb, G, G, G, C, R, 0, None),
                 "bbw_nn_gather_receivers")
        h = torch.empty(nb * R, H, **e)
        hpre = torch.empty(nb * R, H, **e)
        gemm(nb * R, H, C, r, C, 0, 0, self.p["W1"], H, 0, 0, h, H, 0, bias=self.p["b1"], pre=hpre, act=1)
        y = torch.empty(nb * R, T, **e)
        gemm(nb * R, T, H, h, H, 0, 0, self.p["W2"], T, 0, 0, y, T, 0, bias=self.p["b2"])
        cache.update(r=r, h=h, hpre=hpre, nb=nb)
        return y.reshape(nb, R, T), cache

    def backward(self, cache: dict, dy):
        """Parameter gradients (into self.g) of sum(dy * traces)."""
        cfg = self.cfg
        G, C, L, H, T = cfg["grid"], cfg["width"], cfg["layers"], cfg["hidden"], cfg["nt"]
        mx, my, mz = cfg["modes"]
        nm = mx * my * mz
        R = len(cfg["rx"])
        nb = cache["nb"]
        P = nb * G ** 3
        Px, Py, Pz = self.phi
        e = dict(dtype=torch.float32, device=self.dev)
        for v in self.g.values():
            v.zero_()
        dy = dy.reshape(nb * R, T).contiguous()
        h, hpre, r = cache["h"], cache["hpre"], cache["r"]
        gemm(H, T, nb * R, h, H, 0, 1, dy, T, 0, 0, self.g["W2"], T, 0)
        self._bias(dy, self.g["b2"], nb * R, T)
        dh = torch.empty(nb * R, H, **e)
        gemm(nb * R, H, T, dy, T, 0, 0, self.p["W2"], T, 0, 1, dh, H, 0)
        B._check(B.lib().bbw_nn_gelu_backward(hpre.data_ptr(), dh.data_ptr(), dh.numel(), None), "gelu_backward")
        gemm(C, H, nb * R, r, C, 0, 1, dh, H, 0, 0, self.g["W1"], H, 0)
        self._bias(dh, self.g["b1"], nb * R, H)
        dr = torch.empty(nb * R, C, **e)
        gemm(nb * R, C, H, dh, H, 0, 0, self.p["W1"], H, 0, 1, dr, C, 0)
        du = torch.zeros(P, C, **e)
        B._check(B.lib().bbw_nn_gather_receivers(du.data_ptr(), dr.data_ptr(), self.rx.data_ptr(),
                                                 self.ry.data_ptr(), self.rz.data_ptr(), nb, G, G, G, C, R, 1, None),
                 "bbw_nn_gather_receivers")
        for l in reversed(range(L)):
            u = cache[f"u{l}"]
            B._check(B.lib().bbw_nn_gelu_backward(cache[f"pre{l}"].data_ptr(), du.data_ptr(), du.numel(), None),
                     "gelu_backward")
            dpre = du
            gemm(C, C, P, u, C, 0, 1, dpre, C, 0, 0, self.g[f"W{l}_pw"], C, 0, splits=_splits(P))
            self._bias(dpre, self.g[f"b{l}_pw"], P, C)
            dprev = torch.empty(P, C, **e)
            gemm(P, C, C, dpre, C, 0, 0, self.p[f"W{l}_pw"], C, 0, 1, dprev, C, 0)
            # the spectral branch: transforms are orthogonal-basis contractions
            dt1 = torch.empty(nb * G * G * mz * C, **e)
            dt2 = torch.empty(nb * G * my * mz * C, **e)
            dt3 = torch.empty(nb * nm * C, **e)
            axis(Pz, G, mz, dpre, dt1, nb * G * G, C)
            gemm(my, mz * C, G, Py, my, 0, 1, dt1, mz * C, G * mz * C, 0, dt2, mz * C, my * mz * C, batch=nb * G)
            gemm(mx, my * mz * C, G, Px, mx, 0, 1, dt2, my * mz * C, G * my * mz * C, 0, dt3, my * mz * C,
                 nm * C, batch=nb)
            s3 = cache[f"s3_{l}"]
            gemm(C, C, nb, s3, nm * C, C, 1, dt3, nm * C, C, 0, self.g[f"W{l}_sp"], C, C * C, batch=nm)
            ds3 = torch.empty(nb * nm * C, **e)
            gemm(nb, C, C, dt3, nm * C, C, 0, self.p[f"W{l}_sp"], C, C * C, 1, ds3, nm * C, C, batch=nm)
            ds2 = torch.empty(nb * G * my * mz * C, **e)
            ds1 = torch.empty(nb * G * G * mz * C, **e)
            gemm(G, my * mz * C, mx, Px, mx, 0, 0, ds3, my * mz * C, nm * C, 0, ds2, my * mz * C,
                 G * my * mz * C, batch=nb)
            gemm(G, mz * C, my, Py, my, 0, 0, ds2, mz * C, my * mz * C, 0, ds1, mz * C, G * mz * C, batch=nb * G)
            axis(Pz, G, mz, ds1, dprev, nb * G * G, C, expand=1, beta=1.0)
            du = dprev
        gemm(cfg["cin"], C, P, cache["x"], cfg["cin"], 0, 1, du, C, 0, 0, self.g["W0"], C, 0, splits=_splits(P))
        self._bias(du, self.g["b0"], P, C)
        return self.g

    def _bias(self, dY, db, rows, N):
        B._check(B.lib().bbw_nn_bias_grad(dY.data_ptr(), db.data_ptr(), rows, N, None), "bbw_nn_bias_grad")

    def loss(self, y, target, want_grad: bool = True):
        """(mean squared error as a device scalar, its gradient or None)."""
        lo = torch.zeros(1, dtype=torch.float32, device=self.dev)
        dy = torch.empty_like(y) if want_grad else None
        B._check(B.lib().bbw_nn_mse(y.data_ptr(), target.data_ptr(), _ptr(dy), lo.data_ptr(), y.numel(), None),
                 "bbw_nn_mse")
        return lo, dy

    def adam(self, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.steps += 1
        for k in self.p:
            B._check(B.lib().bbw_nn_adam(self.p[k].data_ptr(), self.g[k].data_ptr(), self.m[k].data_ptr(),
                                         self.v[k].data_ptr(), self.p[k].numel(), self.steps, lr, b1, b2, eps,
                                         None), "bbw_nn_adam")


# ---------------------------------------------------------------------------
# data, training, evaluation and the BBWADG fallback


def receiver_gain(sources, rec, d_ref: float = 0.25) -> np.ndarray:
    """[n, R] gains d_ref / |x_r - x_s| of the traces (the 1/r spreading of a
    point source in 3D). The network is trained on the traces divided by
    them, so near and far receivers and sources weigh alike, and its output
    is multiplied by them."""
    s = np.asarray(sources, dtype=np.float64).reshape(-1, 1, 3)
    r = np.asarray(rec, dtype=np.float64).reshape(1, -1, 3)
    return d_ref / np.linalg.norm(r - s, axis=2)


def straight_ray_times(c2_field, sources, rec, nseg: int = 32) -> np.ndarray:
    """[n, R] travel times along the straight segments from each source to
    each receiver through the medium, int ds / c (midpoint rule, nseg
    pieces). By Fermat's principle the first arrival comes no later; in the
    smooth layer the sources sit in, the difference is second order."""
    xs = np.asarray(sources, dtype=np.float64).reshape(-1, 1, 1, 3)
    xr = np.asarray(rec, dtype=np.float64).reshape(1, -1, 1, 3)
    u = ((np.arange(nseg) + 0.5) / nseg).reshape(1, 1, -1, 1)
    pts = xs + u * (xr - xs)
    c = np.sqrt(np.asarray(c2_field(pts.reshape(-1, 3)), dtype=np.float64)).reshape(pts.shape[:3])
    length = np.linalg.norm(xr - xs, axis=3)[..., 0]
    return length * np.mean(1.0 / c, axis=2)


def _shift(Y, shift, scale):
    out = torch.empty_like(Y)
    rows = Y.numel() // Y.shape[-1]
    B._check(B.lib().bbw_nn_shift_traces(Y.data_ptr(), out.data_ptr(), shift.data_ptr(), _ptr(scale), rows,
                                         Y.shape[-1], None), "bbw_nn_shift_traces")
    return out


def encode(Y, meta: dict):
    """Network targets from traces Y [n, R, T]: every trace moved earlier by its
    straight-ray travel time (in samples) and divided by its receiver gain, so
    that the direct arrival sits at the wavelet's own delay and near and far
    receivers weigh alike."""
    return _shift(Y.contiguous(), meta["shift"], 1.0 / meta["gain"])


def decode(A, meta: dict):
    """Traces from network outputs A [n, R, T] (the inverse of ``encode`` where
    the traces are known: samples past the end of the recorded window were
    zero-filled by ``encode``)."""
    return _shift(A.contiguous(), -meta["shift"], meta["gain"])


def run_meta(dcfg: dict, runs, c2_fields, rec, dt: float, device: str = "cuda") -> dict:
    """Receiver gains and straight-ray shifts (samples) [n, R] of the runs."""
    gain = receiver_gain([r["source"] for r in runs], rec)
    tau = np.stack([straight_ray_times(f, [r["source"]], rec)[0] for r, f in zip(runs, c2_fields)])
    f32 = dict(dtype=torch.float32, device=device)
    return dict(gain=torch.tensor(gain, **f32).contiguous(),
                shift=torch.tensor(tau / (dt * dcfg["every"]), **f32).contiguous())


def _bbwadg_setup(dcfg: dict):
    """Mesh, receivers, the common time step (CFL of c^2 <= c2_max) and the
    source amplitude samples of the surrogate workload."""
    from . import inputs
    vxyz, etov = inputs.cube_mesh(dcfg["hexes"])
    rec = inputs.surrogate_receivers(z=dcfg["rec_z"])
    probe = B.Solver(vxyz, etov, dcfg["N"], dcfg["M"], B.F32)
    probe.set_c2(np.full((len(etov), (dcfg["M"] + 1) * (dcfg["M"] + 2) * (dcfg["M"] + 3) // 6), dcfg["c2_max"]))
    dt = probe.cfl_dt(dcfg["cfl"])
    probe.close()
    amp = B.ricker_samples(dt, dcfg["steps"], f0=dcfg["f0"], t0=dcfg["t0"])
    return vxyz, etov, rec, dt, amp


def bbwadg_traces(solver, vxyz, etov, dcfg, run, dt, amp, timings: list | None = None):
    """Receiver traces [R, T] of one run with a prepared solver (BBWADG, FP32);
    timings (if given) receives the seconds of the time integration alone."""
    import time

    from . import inputs
    field = inputs.c2_smooth_random(run["c2_seed"])
    solver.set_c2(inputs.sample_at_domain_points(vxyz, etov, dcfg["M"], field))
    solver.set_state(np.zeros((4, len(etov), (dcfg["N"] + 1) * (dcfg["N"] + 2) * (dcfg["N"] + 3) // 6)))
    solver.set_point_source(run["source"], amp)
    if timings is not None:
        solver.sync()
        t = time.perf_counter()
    tr = solver.record(dt, dcfg["steps"], dcfg["steps"])
    if timings is not None:
        timings.append(time.perf_counter() - t)
    return np.ascontiguousarray(tr[dcfg["every"] - 1::dcfg["every"]].T)


def generate(dcfg: dict, first: int, n: int, threads: int = 8, device: str = "cuda"):
    """(X [n, G, G, G, 6], Y [n, R, T], meta) on the device for runs first ..
    first + n - 1: each target is a BBWADG run (solvers on `threads` streams
    run concurrently), each input the run's c^2 on the grid plus its source;
    meta holds dt, the runs and their receiver gains and shifts [n, R]
    (``run_meta``, used by ``encode`` / ``decode``)."""
    import concurrent.futures as cf
    import threading

    from . import inputs
    vxyz, etov, rec, dt, amp = _bbwadg_setup(dcfg)
    G = dcfg["grid"]
    runs = inputs.surrogate_runs(first, n, dcfg)
    X = torch.empty((n, G, G, G, 6), dtype=torch.float32, device=device)
    Y = torch.empty((n, len(rec), dcfg["steps"] // dcfg["every"]), dtype=torch.float32, device=device)
    local = threading.local()
    streams = [torch.cuda.Stream() for _ in range(threads)]
    counter = iter(range(threads))
    lock = threading.Lock()

    def solver():
        if not hasattr(local, "s"):
            with lock:
                k = next(counter)
            local.s = B.Solver(vxyz, etov, dcfg["N"], dcfg["M"], B.F32, stream=streams[k].cuda_stream)
            local.s.set_receivers(rec)
        return local.s

    def work(j):
        run = runs[j]
        tr = bbwadg_traces(solver(), vxyz, etov, dcfg, run, dt, amp)
        ft = inputs.surrogate_features(inputs.c2_smooth_random(run["c2_seed"]), run["source"], G, dcfg["sigma"])
        return j, tr, ft

    with cf.ThreadPoolExecutor(threads) as ex:
        for j, tr, ft in ex.map(work, range(n)):
            Y[j].copy_(torch.from_numpy(tr.astype(np.float32)))
            X[j].copy_(torch.from_numpy(ft))
    torch.cuda.synchronize()
    meta = run_meta(dcfg, runs, [inputs.c2_smooth_random(r["c2_seed"]) for r in runs], rec, dt, device)
    return X, Y, dict(meta, dt=dt, runs=runs)


def train(net: Net, X, Y, iters: int, batch: int = 8, lr: float = 1e-3, seed: int = 0, scale: float = 1.0,
          log_every: int = 0):
    """Adam on the mean squared error of the targets Y / scale (Y: ``encode``d
    traces), random batches; the learning rate decays by a cosine to lr / 20.
    Returns the losses (host floats, read every log_every iterations)."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    losses = []
    for it in range(iters):
        idx = torch.from_numpy(rng.choice(n, batch, replace=False)).to(X.device)
        xb = X.index_select(0, idx)
        yb = Y.index_select(0, idx) / scale
        y, cache = net.forward(xb)
        lo, dy = net.loss(y, yb)
        net.backward(cache, dy)
        lr_it = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * it / max(iters, 1))))
        net.adam(lr=lr_it)
        if log_every and (it % log_every == 0 or it == iters - 1):
            losses.append((it, float(lo)))
    return losses


def predict(net: Net, X, scale: float, meta: dict | None = None, batch: int = 8):
    """Network outputs [n, R, T] for inputs X, times scale; with the runs'
    meta (``generate``), decoded to traces."""
    out = []
    for k in range(0, X.shape[0], batch):
        y, _ = net.forward(X[k:k + batch].contiguous())
        out.append(y * scale)
    out = torch.cat(out)
    return out if meta is None else decode(out, meta)


def relative_errors(pred, Y) -> np.ndarray:
    """Per-run relative L2 trace error ||pred - Y|| / ||Y||."""
    d = (pred - Y).reshape(Y.shape[0], -1).double()
    return (d.norm(dim=1) / Y.reshape(Y.shape[0], -1).double().norm(dim=1)).cpu().numpy()


class Surrogate:
    """The trained network with BBWADG as its error reference and fallback.

    ``predict(run, tol)`` returns (traces [R, T], "surrogate" | "bbwadg", err)
    where err is the held-out error quantile the surrogate is trusted to: the
    network answers only when the source lies in the box it was trained on,
    the medium's grid values lie in the training range and tol (a relative L2
    trace error) is at least the calibrated quantile; otherwise the run is
    solved by BBWADG."""

    def __init__(self, net: Net, dcfg: dict, scale: float, calib_err: float, c2_range, dt: float):
        self.net, self.dcfg, self.scale, self.err = net, dict(dcfg), scale, float(calib_err)
        self.c2_range, self.dt = c2_range, float(dt)
        self._bbw = None

    def _in_domain(self, run, feat) -> bool:
        lo, hi = np.asarray(self.dcfg["src_lo"]), np.asarray(self.dcfg["src_hi"])
        xs = np.asarray(run["source"])
        c2 = feat[..., 0] * 0.75 + 1.25
        return bool(np.all(xs >= lo) and np.all(xs <= hi) and c2.min() >= self.c2_range[0] and
                    c2.max() <= self.c2_range[1])

    def predict(self, run: dict, tol: float | None = None):
        from . import inputs
        field = inputs.c2_smooth_random(run["c2_seed"]) if "c2_field" not in run else run["c2_field"]
        feat = inputs.surrogate_features(field, run["source"], self.dcfg["grid"], self.dcfg["sigma"])
        if self._in_domain(run, feat) and (tol is None or tol >= self.err):
            x = torch.from_numpy(feat[None]).to(self.net.dev)
            y, _ = self.net.forward(x)
            rec = inputs.surrogate_receivers(z=self.dcfg["rec_z"])
            meta = run_meta(self.dcfg, [run], [field], rec, self.dt, device=str(self.net.dev))
            return decode(y * self.scale, meta)[0].double().cpu().numpy(), "surrogate", self.err
        if self._bbw is None:
            vxyz, etov, rec, dt, amp = _bbwadg_setup(self.dcfg)
            s = B.Solver(vxyz, etov, self.dcfg["N"], self.dcfg["M"], B.F32)
            s.set_receivers(rec)
            self._bbw = (s, vxyz, etov, dt, amp)
        s, vxyz, etov, dt, amp = self._bbw
        run2 = dict(run)
        if "c2_field" in run:
            raise ValueError("the fallback solves media given by their seed (c2_seed)")
        return bbwadg_traces(s, vxyz, etov, self.dcfg, run2, dt, amp), "bbwadg", 0.0
