"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method: it only builds meshes, samples
scalar fields at points and draws random numbers. It imports neither the
CUDA binding nor the oracle.

Recipes (the paper's GMSH meshes and media are not available):
  * ``cube_mesh(n)``: the unit cube cut into n^3 hexahedra, each split into six
    tetrahedra around its main diagonal (Kuhn/Freudenthal split), hexes in
    lexicographic order with x fastest and the six tets of a hex consecutive;
    ``jitter`` moves interior vertices, ``shuffle`` permutes each element's
    local vertex order (keeping positive orientation) so that every face
    orientation code occurs.
  * Fields are turned into per-element coefficients by *sampling at domain
    points* x_alpha = sum_i alpha_i v_i / n of each element (the Bezier
    control-point positions), which is a synthetic recipe, not a projection;
    the paper's L2 projection is ``project.py`` (host tools of the package).
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "cube_mesh", "multi_index_points", "sample_at_domain_points",
    "c2_smooth_random", "c2_config_small", "gaussian_pulse", "random_state",
    "PARITY_CONFIG", "SWEEP_CONFIG", "BATCH_CONFIG", "batched_instances", "ADJOINT_CONFIG",
    "top_face_receivers", "ELASTIC_CONFIG", "elastic_media", "elastic_pulse",
    "ricker", "ricker_samples", "manufactured_forcing",
    "SURROGATE_CONFIG", "surrogate_runs", "surrogate_receivers", "grid_centres", "surrogate_features",
]

#: the FP64 parity workload: 4^3 hexes x 6 = 384 tets, N=3, M=1, T=0.5
PARITY_CONFIG = dict(hexes=4, N=3, M=1, T=0.5, cfl=0.5)
#: the FP32 throughput workload: 32^3 hexes x 6 = 196,608 tets, N=1..9, M=2
SWEEP_CONFIG = dict(hexes=32, Ns=tuple(range(1, 10)), M=2, steps=100,
                    source=(0.5, 0.5, 0.5), f0=10.0)


#: the batched workload: 256 instances, cube refinements of 2k-60k tets
#: (7^3 x 6 = 2,058 .. 21^3 x 6 = 55,566), N in 3..7, M = 2, FP32, one seeded
#: medium and Ricker source position per instance
BATCH_CONFIG = dict(instances=256, hexes=(7, 21), Ns=(3, 7), M=2, f0=10.0, cfl=0.5)


#: the adjoint workload: 16^3 hexes x 6 = 24,576 tets, N = 5, M = 2, FP32,
#: 64 receivers on the top face (8 x 8 grid at z = 1), 2000 steps, data from
#: the medium of seed 0, model medium of seed 1, Ricker source at (0.5, 0.5, 0.7)
ADJOINT_CONFIG = dict(hexes=16, N=5, M=2, steps=2000, receivers=8, source=(0.5, 0.5, 0.7), f0=10.0,
                      cfl=0.5, true_seed=0, model_seed=1)


def top_face_receivers(n: int = ADJOINT_CONFIG["receivers"]) -> np.ndarray:
    """n x n receiver points at the cell centres of a uniform grid on z = 1."""
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.ones(n * n)], axis=1)


def surrogate_receivers(n: int = 8, z: float = 0.9) -> np.ndarray:
    """n x n receiver points at the cell centres of a uniform grid on the
    plane at height z (below the p = 0 top wall, so that they record the
    wave and not the wall's weak residual)."""
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(n * n, float(z))], axis=1)


def batched_instances(n: int = BATCH_CONFIG["instances"], seed: int = 0):
    """Seeded instance descriptions of the batched workload: for each, the
    cube refinement (hexes per side), the degree N, the seed of its c^2
    medium (``c2_smooth_random``) and its source position."""
    rng = np.random.default_rng(seed)
    lo, hi = BATCH_CONFIG["hexes"]
    nlo, nhi = BATCH_CONFIG["Ns"]
    out = []
    for i in range(n):
        out.append(dict(hexes=int(rng.integers(lo, hi + 1)), N=int(rng.integers(nlo, nhi + 1)),
                        c2_seed=int(1000 + i), source=rng.uniform(0.25, 0.75, 3)))
    return out


def cube_mesh(n: int, jitter: float = 0.0, shuffle: bool = False, seed: int = 0,
              lo: float = 0.0, hi: float = 1.0):
    """Return (vxyz (nv,3) float64, etov (K,4) int64) for n^3 hexes x 6 tets."""
    rng = np.random.default_rng(seed)
    g = np.linspace(lo, hi, n + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")  # vertex (i, j, k)
    vxyz = np.stack([X, Y, Z], axis=-1).transpose(2, 1, 0, 3).reshape(-1, 3).copy()
    if jitter:
        h = (hi - lo) / n
        inner = np.ones(len(vxyz), dtype=bool)
        for d in range(3):
            inner &= (vxyz[:, d] > lo + 1e-12) & (vxyz[:, d] < hi - 1e-12)
        vxyz[inner] += rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 3))

    def vid(i, j, k):
        return i + (n + 1) * (j + (n + 1) * k)

    unit = np.eye(3, dtype=int)
    tets = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                base = np.array([i, j, k])
                for perm in itertools.permutations(range(3)):
                    c = base.copy()
                    vs = [vid(*c)]
                    for ax in perm:
                        c = c + unit[ax]
                        vs.append(vid(*c))
                    tets.append(vs)
    etov = np.array(tets, dtype=np.int64)
    if shuffle:
        for e in range(len(etov)):
            etov[e] = etov[e][rng.permutation(4)]
    # positive orientation: swap two vertices where the volume is negative
    P = vxyz[etov]
    det = np.einsum("ki,ki->k", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    neg = det < 0
    etov[neg, 2], etov[neg, 3] = etov[neg, 3].copy(), etov[neg, 2].copy()
    return vxyz, etov


def multi_index_points(n: int) -> np.ndarray:
    """(N_p, 4) array of alpha / n in the library's multi-index order.

    Order: for l in 0..n, for k in 0..n-l, for j in 0..n-l-k, alpha =
    (n-j-k-l, j, k, l). For n = 0 the single point is the centroid.
    """
    out = []
    for l in range(n + 1):
        for k in range(n - l + 1):
            for j in range(n - l - k + 1):
                out.append((n - j - k - l, j, k, l))
    a = np.array(out, dtype=np.float64)
    if n == 0:
        return np.full((1, 4), 0.25)
    return a / n


#: the elastic workload (the velocity-stress system of Sec. 2.2): the
#: throughput mesh (32^3 hexes x 6 = 196,608 tets), N = 1..9, M = 2 media
#: (rho^{-1}, lambda, mu from seeded smooth random fields with a layer jump),
#: a Gaussian compressional pulse as initial state, FP32
ELASTIC_CONFIG = dict(hexes=32, Ns=tuple(range(1, 10)), M=2, cfl=0.5, seed=0)


def elastic_media(vxyz, etov, M: int, seed: int = 0):
    """(rho_inv, lam, mu), each [K, M_p] Bernstein coefficients of degree M
    (field values at the domain points, so every coefficient is positive).

    c_p^2 = 2 f_0(x) in [1, 6] (f_0 the smooth random medium of seed ``seed``
    with its layer jump), c_s^2 = c_p^2 / 3 (Poisson ratio 1/4, lambda = mu),
    rho = f_1(x) in [0.5, 3] (seed + 1); lambda = rho (c_p^2 - 2 c_s^2),
    mu = rho c_s^2."""
    f0 = c2_smooth_random(seed)
    rho = c2_smooth_random(seed + 1)

    def rho_inv(x):
        return 1.0 / rho(x)

    def mu(x):  # rho c_s^2 = rho (2 f_0) / 3
        return rho(x) * 2.0 * f0(x) / 3.0

    def lam(x):  # rho (c_p^2 - 2 c_s^2) = rho (2 f_0) / 3
        return rho(x) * 2.0 * f0(x) / 3.0

    return tuple(sample_at_domain_points(vxyz, etov, M, f) for f in (rho_inv, lam, mu))


def elastic_pulse(vxyz, etov, N: int, center=(0.5, 0.5, 0.5), width: float = 0.1) -> np.ndarray:
    """Initial state [9, K, N_p]: v = 0, sigma = -g I with g the Gaussian
    pulse (an isotropic pressure-like load that radiates a P wave); the
    Bernstein coefficients are the pulse values at the domain points."""
    g = sample_at_domain_points(vxyz, etov, N, gaussian_pulse(center, width))
    q = np.zeros((9,) + g.shape)
    q[3:6] = -g
    return q


def sample_at_domain_points(vxyz, etov, n: int, field) -> np.ndarray:
    """field(x (P,3)) sampled at every element's degree-n domain points, (K, N_p)."""
    X = np.asarray(vxyz, dtype=np.float64)[np.asarray(etov)]
    pts = np.einsum("pa,kai->kpi", multi_index_points(n), X)
    K, P = pts.shape[:2]
    return np.asarray(field(pts.reshape(-1, 3)), dtype=np.float64).reshape(K, P)


def c2_config_small(x: np.ndarray) -> np.ndarray:
    """c^2 = 1 + 0.5 sin(pi x) sin(pi y) sin(pi z) (the paper's 3D medium)."""
    s = np.sin(np.pi * x)
    return 1.0 + 0.5 * s[:, 0] * s[:, 1] * s[:, 2]


def c2_smooth_random(seed: int = 0, modes: int = 8, jump: float = 1.5,
                     plane=(0.3, 0.2, 1.0, 0.55)):
    """A seeded smooth random medium in [0.5, 2] with a planar layer jump.

    Sum of ``modes`` random low-frequency Fourier modes, affinely rescaled to
    [0.5, 2] over a fixed probe grid, times ``jump`` where
    a x + b y + c z > d (a plane not aligned with any mesh face).
    """
    rng = np.random.default_rng(seed)
    kvec = rng.integers(1, 4, size=(modes, 3)) * np.pi
    phase = rng.uniform(0, 2 * np.pi, size=modes)
    amp = rng.normal(size=modes)

    def raw(x):
        return np.sum(amp[None, :] * np.cos(x @ kvec.T + phase[None, :]), axis=1)

    g = np.linspace(0.0, 1.0, 33)
    probe = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r = raw(probe)
    lo, hi = r.min(), r.max()
    a, b, c, d = plane

    def field(x):
        v = 0.5 + 1.5 * np.clip((raw(x) - lo) / (hi - lo), 0.0, 1.0)
        above = a * x[:, 0] + b * x[:, 1] + c * x[:, 2] > d
        return np.where(above, jump * v, v)

    return field


def gaussian_pulse(center=(0.5, 0.5, 0.5), width: float = 0.1):
    """p0 = exp(-|x - center|^2 / width^2)."""
    c = np.asarray(center, dtype=np.float64)

    def field(x):
        return np.exp(-np.sum((x - c) ** 2, axis=1) / width ** 2)

    return field


def random_state(K: int, Np: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """Standard-normal state of shape (4, K, Np), rounded to ``dtype``."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, K, Np)).astype(dtype)


def ricker(t, f0: float, t0: float):
    """Ricker wavelet (1 - 2 a) exp(-a), a = (pi f0 (t - t0))^2 (a source time
    signature; not part of the method)."""
    a = (np.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def ricker_samples(f0: float, t0: float, dt: float, nsteps: int, stage_times, t_start: float = 0.0,
                   signal=None) -> np.ndarray:
    """Amplitude samples of a source time function, one per RK stage:
    sample 5 n + s = signal(t_start + (n + c_s) dt) for n < nsteps, with
    c_s = stage_times[s] (the RK scheme's stage times, passed in) and
    signal the Ricker wavelet of (f0, t0) unless given."""
    c = np.asarray(stage_times, dtype=np.float64).reshape(1, 5)
    t = t_start + (np.arange(nsteps, dtype=np.float64)[:, None] + c) * dt
    sig = signal if signal is not None else (lambda x: ricker(x, f0, t0))
    return np.asarray(sig(t), dtype=np.float64).reshape(-1)


def manufactured_forcing(c2):
    """The spatial part g(x) of a separable forcing f(x, t) = g(x) sin(pi t):
    g = (3 - 1/c^2(x)) pi sin(pi x) sin(pi y) sin(pi z), the forcing for which
    p = sin(pi x) sin(pi y) sin(pi z) cos(pi t) solves the 3D acoustic system
    with wave speed c^2 (the manufactured solution of the convergence study,
    Sec. 6.1). Returns g as a field of points (P, 3)."""
    def field(x):
        s = np.sin(np.pi * x)
        return (3.0 - 1.0 / c2(x)) * np.pi * s[:, 0] * s[:, 1] * s[:, 2]
    return field


#: the surrogate workload: BBWADG N = 4 runs on 16^3 x 6 tets (the adjoint's
#: mesh) with 64 receivers on the plane z = rec_z (``surrogate_receivers``),
#: each run a seeded smooth random medium (the sweep's recipe with its layer
#: jump, seed 5000 + run) and a Ricker source (peak frequency f0, delay t0) at
#: a seeded position in the box [src_lo, src_hi] (above the layer jump);
#: traces of `steps` RK steps at the common CFL step of c^2 <= c2_max, every
#: `every`-th kept (512 samples over 0.37 time units, in which the direct
#: wave reaches the receivers nearest the source); f0 = 12 keeps about 7
#: nodes per wavelength at the median wave speed of that layer; the network
#: sees c^2 on the centres of a grid^3 grid plus the source position
SURROGATE_CONFIG = dict(runs=4096, test_runs=256, hexes=16, N=4, M=2, steps=1024, every=2, f0=12.0, t0=1.0 / 12.0,
                        src_lo=(0.25, 0.25, 0.55), src_hi=(0.75, 0.75, 0.75), rec_z=0.9, grid=64, c2_max=3.0,
                        cfl=0.5, sigma=0.05)


def surrogate_runs(first: int, n: int, cfg: dict = SURROGATE_CONFIG):
    """Descriptions (medium seed, source position) of runs first .. first + n - 1."""
    out = []
    for i in range(first, first + n):
        rng = np.random.default_rng(5000 + i)
        out.append(dict(c2_seed=5000 + i, source=rng.uniform(cfg["src_lo"], cfg["src_hi"])))
    return out


def grid_centres(G: int) -> np.ndarray:
    """[G^3, 3] cell centres (i + 1/2)/G of a G^3 grid on the unit cube, x outermost."""
    c = (np.arange(G) + 0.5) / G
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([X, Y, Z], -1).reshape(-1, 3)


def surrogate_features(c2_field, xs, G: int, sigma: float) -> np.ndarray:
    """[G, G, G, 6] float32 network input: (c^2 - 1.25)/0.75 on the grid, the
    coordinates mapped to [-1, 1], a Gaussian bump of width sigma at the
    source xs and the distance to it (times 2)."""
    x = grid_centres(G)
    f = np.empty((len(x), 6), dtype=np.float32)
    f[:, 0] = (c2_field(x) - 1.25) / 0.75
    f[:, 1:4] = 2.0 * x - 1.0
    d2 = np.sum((x - np.asarray(xs)) ** 2, axis=1)
    f[:, 4] = np.exp(-d2 / (2.0 * sigma ** 2))
    f[:, 5] = 2.0 * np.sqrt(d2)
    return f.reshape(G, G, G, 6)

