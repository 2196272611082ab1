"""The surrogate network's kernels on the GPU against the FP64 reference
network (oracle/fno.py): forward traces and every parameter gradient, the
GEMM kernel against numpy on ragged shapes, MSE and Adam.

Tolerance: the GEMM rounds both operands to BF16 (unit roundoff 2^-9), so
each contraction carries a relative error of a few 1e-3 and the network's
chain of ~10 of them about 1e-2: outputs and gradients are compared in
relative L2 at 2e-2."""
import numpy as np
import pytest

from oracle import fno
from parity_util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_08645_gb300 import build
    build.build()


def _cfg():
    from paper_1808_08645_gb300 import surrogate as S
    return S.default_config(grid=8, width=8, modes=(3, 3, 2), layers=2, cin=6, hidden=16, nt=12, receivers=2)


@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_bf16_against_numpy(tA, tB):
    from paper_1808_08645_gb300 import surrogate as S
    rng = np.random.default_rng(tA * 2 + tB)
    for M, N, K, batch, splits in [(70, 45, 37, 3, 1), (5, 33, 130, 2, 1), (33, 17, 3000, 1, 7)]:
        A = rng.standard_normal((batch, K, M) if tA else (batch, M, K))
        Bm = rng.standard_normal((batch, N, K) if tB else (batch, K, N))
        want = np.einsum("bmk,bkn->bmn", A.transpose(0, 2, 1) if tA else A, Bm.transpose(0, 2, 1) if tB else Bm)
        # BF16-rounded operands give the reference the kernel can reach exactly up to FP32 sums
        rA = torch.tensor(A, dtype=torch.float32).bfloat16().double().numpy()
        rB = torch.tensor(Bm, dtype=torch.float32).bfloat16().double().numpy()
        want_r = np.einsum("bmk,bkn->bmn", rA.transpose(0, 2, 1) if tA else rA, rB.transpose(0, 2, 1) if tB else rB)
        dA = torch.tensor(A, dtype=torch.float32, device="cuda")
        dB = torch.tensor(Bm, dtype=torch.float32, device="cuda")
        dC = torch.zeros((batch, M, N), dtype=torch.float32, device="cuda")
        S.gemm(M, N, K, dA, M if tA else K, A[0].size, tA, dB, K if tB else N, Bm[0].size, tB, dC, N, M * N,
               batch=batch, splits=splits)
        got = dC.double().cpu().numpy()
        assert rel_l2(got, want_r) < 1e-5
        assert rel_l2(got, want) < 1e-2


@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_vector_paths_with_ragged_edges(tA, tB):
    """Operands padded to leading dimensions that are multiples of 4 floats
    (the 16-byte load path) while M, N, K are not multiples of the tile or of
    4: partial quads at every edge, an odd N for the scalar store path, and
    split-K."""
    from paper_1808_08645_gb300 import surrogate as S
    rng = np.random.default_rng(10 + tA * 2 + tB)
    for M, N, K, batch, splits in [(70, 44, 38, 2, 1), (67, 45, 61, 1, 1), (33, 30, 2050, 1, 5)]:
        pm, pn, pk = -(-M // 4) * 4 + 4, -(-N // 4) * 4 + 4, -(-K // 4) * 4 + 4  # padded leading dims
        Ap = rng.standard_normal((batch, pk, pm) if tA else (batch, pm, pk))
        Bp = rng.standard_normal((batch, pn, pk) if tB else (batch, pk, pn))
        A = Ap[:, :K, :M] if tA else Ap[:, :M, :K]
        Bm = Bp[:, :N, :K] if tB else Bp[:, :K, :N]
        rA = torch.tensor(A, dtype=torch.float32).bfloat16().double().numpy()
        rB = torch.tensor(Bm, dtype=torch.float32).bfloat16().double().numpy()
        want = np.einsum("bmk,bkn->bmn", rA.transpose(0, 2, 1) if tA else rA, rB.transpose(0, 2, 1) if tB else rB)
        dA = torch.tensor(Ap, dtype=torch.float32, device="cuda")
        dB = torch.tensor(Bp, dtype=torch.float32, device="cuda")
        ldc = N + (N % 2)
        dC = torch.zeros((batch, M, ldc), dtype=torch.float32, device="cuda")
        S.gemm(M, N, K, dA, Ap.shape[2], Ap[0].size, tA, dB, Bp.shape[2], Bp[0].size, tB, dC, ldc, M * ldc,
               batch=batch, splits=splits)
        got = dC.double().cpu().numpy()[:, :, :N]
        assert rel_l2(got, want) < 1e-5, (M, N, K)


def test_axis_transform_against_numpy():
    """bbw_nn_axis_transform: contraction and expansion along the innermost
    axis with beta, the pre-activation copy and GELU, FP32."""
    from math import erf

    from paper_1808_08645_gb300 import surrogate as S
    rng = np.random.default_rng(12)
    f32 = dict(dtype=torch.float32, device="cuda")
    for P, L, m, C in [(37, 64, 6, 32), (5, 9, 16, 3), (1, 1, 1, 1)]:
        basis = rng.standard_normal((L, m))
        x = rng.standard_normal((P, L, C))
        want = np.einsum("zk,pzc->pkc", basis, x)
        out = torch.full((P, m, C), float("nan"), **f32)
        S.axis(torch.tensor(basis, **f32), L, m, torch.tensor(x, **f32), out, P, C)
        assert np.allclose(out.double().cpu().numpy(), want, rtol=1e-5, atol=1e-5 * np.abs(want).max())
        t = rng.standard_normal((P, m, C))
        o0 = rng.standard_normal((P, L, C))
        v = np.einsum("zk,pkc->pzc", basis, t) + 0.5 * o0
        o = torch.tensor(o0, **f32)
        pre = torch.empty_like(o)
        S.axis(torch.tensor(basis, **f32), L, m, torch.tensor(t, **f32), o, P, C, expand=1, beta=0.5, pre=pre, act=1)
        gelu = np.vectorize(lambda a: 0.5 * a * (1.0 + erf(a / np.sqrt(2.0))))
        tol = 1e-5 * max(1.0, np.abs(v).max())
        assert np.allclose(pre.double().cpu().numpy(), v, rtol=1e-5, atol=tol)
        assert np.allclose(o.double().cpu().numpy(), gelu(v), rtol=1e-5, atol=tol)


def test_forward_and_gradients_match_the_reference_network():
    from paper_1808_08645_gb300 import surrogate as S
    cfg = _cfg()
    rng = np.random.default_rng(1)
    p = fno.init_params(cfg, seed=2)
    x = rng.standard_normal((2, 8, 8, 8, 6))
    dy = rng.standard_normal((2, len(cfg["rx"]), cfg["nt"]))
    y_ref, cache = fno.forward(p, cfg, x)
    g_ref = fno.backward(p, cfg, cache, dy)
    net = S.Net(cfg, params=p)
    y, c = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda"))
    assert rel_l2(y.double().cpu().numpy(), y_ref) <= TOL
    g = net.backward(c, torch.tensor(dy, dtype=torch.float32, device="cuda"))
    for k in p:
        assert rel_l2(g[k].double().cpu().numpy(), g_ref[k]) <= TOL, k


def test_shift_traces_kernel():
    """bbw_nn_shift_traces against numpy's linear interpolation of the
    zero-extended samples, fractional shifts of both signs and beyond the
    window; integer shifts there and back restore the overlapping samples."""
    from paper_1808_08645_gb300 import surrogate as S
    rng = np.random.default_rng(9)
    rows, T = 37, 29
    Y = rng.standard_normal((rows, T))
    sh = np.concatenate([rng.uniform(-40, 40, rows - 5), [0.0, -0.5, 28.7, -28.3, 3.0]])
    sc = rng.uniform(0.5, 2.0, rows)
    xp = np.arange(-1, T + 1)
    want = np.stack([sc[i] * np.interp(np.arange(T) + sh[i], xp, np.concatenate([[0.0], Y[i], [0.0]]),
                                       left=0.0, right=0.0) for i in range(rows)])
    f32 = dict(dtype=torch.float32, device="cuda")
    meta = dict(shift=torch.tensor(sh, **f32), gain=torch.tensor(1.0 / sc, **f32))
    got = S.encode(torch.tensor(Y, **f32), meta).double().cpu().numpy()
    assert np.allclose(got, want, atol=1e-5)
    ish = np.round(sh)
    meta = dict(shift=torch.tensor(ish, **f32), gain=torch.tensor(1.0 / sc, **f32))
    back = S.decode(S.encode(torch.tensor(Y, **f32), meta), meta).double().cpu().numpy()
    for i in range(rows):
        keep = (np.arange(T) - ish[i] >= 0) & (np.arange(T) - ish[i] < T)
        assert np.allclose(back[i][keep], Y[i][keep], atol=1e-5)


def test_mse_and_adam_kernels():
    from paper_1808_08645_gb300 import surrogate as S
    cfg = _cfg()
    net = S.Net(cfg, seed=0)
    rng = np.random.default_rng(3)
    y = torch.tensor(rng.standard_normal((3, 4, 5)), dtype=torch.float32, device="cuda")
    t = torch.tensor(rng.standard_normal((3, 4, 5)), dtype=torch.float32, device="cuda")
    lo, dy = net.loss(y, t)
    yn, tn = y.double().cpu().numpy(), t.double().cpu().numpy()
    assert abs(float(lo) - np.mean((yn - tn) ** 2)) < 1e-5
    assert np.allclose(dy.double().cpu().numpy(), 2 * (yn - tn) / yn.size, atol=1e-6)
    # two Adam steps against the update in FP64
    p0 = {k: v.double().cpu().numpy() for k, v in net.p.items()}
    m = {k: np.zeros_like(v) for k, v in p0.items()}
    v2 = {k: np.zeros_like(v) for k, v in p0.items()}
    grads = [{k: rng.standard_normal(v.shape) for k, v in p0.items()} for _ in range(2)]
    for s, gr in enumerate(grads, 1):
        for k in net.g:
            net.g[k].copy_(torch.tensor(gr[k]))
            m[k] = 0.9 * m[k] + 0.1 * gr[k]
            v2[k] = 0.999 * v2[k] + 0.001 * gr[k] ** 2
            # the efficient form of Kingma & Ba: bias corrections folded into the step
            lr_t = 1e-2 * np.sqrt(1 - 0.999 ** s) / (1 - 0.9 ** s)
            p0[k] -= lr_t * m[k] / (np.sqrt(v2[k]) + 1e-8)
        net.adam(lr=1e-2)
    for k in p0:
        assert np.allclose(net.p[k].double().cpu().numpy(), p0[k], atol=2e-6), k


def test_training_follows_the_reference_adam_trajectory():
    """120 Adam steps on a fixed batch: the GPU loss follows the FP64
    reference network trained by the same Adam update (within 10 % over the
    first 90 steps, BF16 operands) and falls below a quarter of its start."""
    from paper_1808_08645_gb300 import surrogate as S
    cfg = _cfg()
    p0 = fno.init_params(cfg, seed=4)
    rng = np.random.default_rng(5)
    xn = rng.standard_normal((2, 8, 8, 8, 6))
    tn = rng.standard_normal((2, len(cfg["rx"]), cfg["nt"]))
    # the reference: FP64 network, Adam in the efficient form of Kingma & Ba
    p = {k: v.copy() for k, v in p0.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v2 = {k: np.zeros_like(v) for k, v in p.items()}
    ref = []
    for it in range(120):
        y, c = fno.forward(p, cfg, xn)
        d = y - tn
        ref.append(np.mean(d ** 2))
        g = fno.backward(p, cfg, c, 2 * d / d.size)
        for k in p:
            m[k] = 0.9 * m[k] + 0.1 * g[k]
            v2[k] = 0.999 * v2[k] + 0.001 * g[k] ** 2
            p[k] -= 3e-3 * np.sqrt(1 - 0.999 ** (it + 1)) / (1 - 0.9 ** (it + 1)) * m[k] / (np.sqrt(v2[k]) + 1e-8)
    net = S.Net(cfg, params=p0)
    x = torch.tensor(xn, dtype=torch.float32, device="cuda")
    t = torch.tensor(tn, dtype=torch.float32, device="cuda")
    got = []
    for _ in range(120):
        y, c = net.forward(x)
        lo, dy = net.loss(y, t)
        got.append(float(lo))
        net.backward(c, dy)
        net.adam(lr=3e-3)
    for it in (0, 30, 60, 90):
        assert abs(got[it] - ref[it]) <= 0.1 * ref[it], (it, got[it], ref[it])
    assert got[-1] < 0.25 * got[0]


def test_small_pipeline_generate_train_calibrate_and_fall_back():
    """A reduced surrogate workload end to end: BBWADG runs make the data, the
    network fits its training runs, held-out errors are finite, and runs
    outside the training box (or asked for a tolerance below the calibrated
    error) are solved by BBWADG (bitwise the direct solve)."""
    from paper_1808_08645_gb300 import inputs
    from paper_1808_08645_gb300 import surrogate as S
    dcfg = dict(inputs.SURROGATE_CONFIG, hexes=3, N=2, steps=48, grid=16)
    X, Y, meta = S.generate(dcfg, 0, 24, threads=4)
    Xt, Yt, mt = S.generate(dcfg, 24, 6, threads=2)
    assert torch.isfinite(Y).all() and float(Y.abs().max()) > 0
    assert meta["gain"].shape == (24, 64) and float(meta["gain"].min()) > 0
    assert meta["shift"].shape == (24, 64) and float(meta["shift"].min()) > 0
    A = S.encode(Y, meta)
    scale = float(A.std())
    net = S.Net(S.default_config(grid=16, width=8, modes=(3, 3, 3), layers=2, hidden=16, nt=Y.shape[2],
                                 rec_z=dcfg["rec_z"]), seed=1)

    def train_mse():
        return float(((S.predict(net, X, scale) - A) ** 2).mean())

    m0 = train_mse()
    S.train(net, X, A, 300, scale=scale, lr=1e-2)
    assert train_mse() < 0.7 * m0  # it learns its training runs
    e1 = S.relative_errors(S.predict(net, Xt, scale, mt), Yt)  # held out (far too few runs here to generalise)
    assert np.isfinite(e1).all()
    sur = S.Surrogate(net, dcfg, scale, float(np.quantile(e1, 0.95)), (0.4, 3.5), meta["dt"])
    run = inputs.surrogate_runs(24, 1, dcfg)[0]
    out_run = dict(run, source=np.array([0.5, 0.5, 0.3]))
    tr, used, _ = sur.predict(out_run)
    assert used == "bbwadg"
    vxyz, etov, rec, dt, amp = S._bbwadg_setup(dcfg)
    from paper_1808_08645_gb300 import binding as B
    s = B.Solver(vxyz, etov, dcfg["N"], dcfg["M"], B.F32)
    s.set_receivers(rec)
    assert np.array_equal(tr, S.bbwadg_traces(s, vxyz, etov, dcfg, out_run, dt, amp))
    s.close()
    _, used, _ = sur.predict(run, tol=sur.err)  # the calibrated error is accepted
    assert used == "surrogate"
    _, used, _ = sur.predict(run, tol=0.5 * sur.err)  # a tighter tolerance falls back
    assert used == "bbwadg"
