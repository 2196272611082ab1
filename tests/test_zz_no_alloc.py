"""The allocation-free weight-adjusted update (bbw_wadg_update_noalloc).

Callers that cannot allocate device memory (code running while a CUDA graph
is captured on another stream, frameworks that own the whole memory pool,
latency-critical loops) use this entry point; it keeps its operator tables in
the library's static device memory instead of a cache it allocates. These
tests call it through the C ABI and compare it with bbw_wadg_update on two
calls in a row and with the FP64 oracle's M^{-1} M_{c2} r, check that a call
after the set-up leaves the device's free memory unchanged, and run it on a
side stream while a CUDA graph is being captured on another stream. The file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1808_08645_gb300 import binding as B

from oracle import bernstein as bb
from parity_util import TOL_STAGE, rel_l2, rounded

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_08645_gb300 import build
    build.build()


def _np3(n):
    return (n + 1) * (n + 2) * (n + 3) // 6


def _run(fn, N, M, prec, r, c2):
    dt = torch.float32 if prec == 32 else torch.float64
    dr = torch.tensor(r, dtype=dt, device="cuda")
    dc = torch.tensor(c2, dtype=dt, device="cuda")
    out = torch.full_like(dr, float("nan"))
    fn(N, M, prec, r.shape[0], dr, dc, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("prec", [32, 64])
def test_noalloc_matches_wadg_update_on_consecutive_calls(prec):
    rng = np.random.default_rng(5)
    # consecutive calls with different (N, M) so the second overwrites the
    # first call's tables in the shared static array
    for N, M, K in [(7, 2, 41), (3, 1, 70), (7, 2, 41), (9, 2, 19)]:
        r = rounded(rng.standard_normal((K, _np3(N))), prec)
        c2 = rounded(rng.uniform(0.5, 2.0, (K, _np3(M))), prec)
        want = _run(B.wadg_update, N, M, prec, r, c2)
        got = _run(B.wadg_update_noalloc, N, M, prec, r, c2)
        assert rel_l2(got, want) <= TOL_STAGE[prec]
        again = _run(B.wadg_update_noalloc, N, M, prec, r, c2)
        assert rel_l2(again, want) <= TOL_STAGE[prec]


def test_noalloc_rejects_tables_beyond_its_static_capacity():
    K, N, M = 4, 9, 3
    r = torch.zeros((K, _np3(N)), device="cuda")
    c2 = torch.ones((K, _np3(M)), device="cuda")
    out = torch.zeros_like(r)
    with pytest.raises(B.BBWError) as ei:
        B.wadg_update_noalloc(N, M, 32, K, r, c2, out)
    assert ei.value.status == -1 and "static scratch" in str(ei.value)


@pytest.mark.parametrize("prec", [32, 64])
def test_noalloc_matches_the_oracle(prec):
    """out = P^{N+M}_N(c2 * r) equals the oracle's dense M^{-1} M_{c2} r."""
    rng = np.random.default_rng(11)
    for N, M, K in [(9, 2, 23), (4, 3, 50), (1, 0, 9)]:
        r = rounded(rng.standard_normal((K, _np3(N))), prec)
        c2 = rounded(rng.uniform(0.5, 2.0, (K, _np3(M))), prec)
        want = np.linalg.solve(bb.mass(N), np.einsum("kb,bij,kj->ki", c2, bb.weighted_mass_terms(N, M), r).T).T
        got = _run(B.wadg_update_noalloc, N, M, prec, r, c2)
        assert rel_l2(got, want) <= TOL_STAGE[prec]


def test_noalloc_call_after_setup_allocates_no_device_memory():
    """After a first (set-up) call, further calls for the same and for other
    (N, M) leave cudaMemGetInfo's free bytes unchanged."""
    rng = np.random.default_rng(2)
    cases = [(6, 2, 64), (3, 1, 128)]
    bufs = []
    for N, M, K in cases:
        dr = torch.tensor(rng.standard_normal((K, _np3(N))), dtype=torch.float32, device="cuda")
        dc = torch.tensor(rng.uniform(0.5, 2.0, (K, _np3(M))), dtype=torch.float32, device="cuda")
        bufs.append((N, M, K, dr, dc, torch.empty_like(dr)))
    for N, M, K, dr, dc, out in bufs:  # set-up calls
        B.wadg_update_noalloc(N, M, 32, K, dr, dc, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for N, M, K, dr, dc, out in bufs:
            B.wadg_update_noalloc(N, M, 32, K, dr, dc, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_on_a_side_stream_during_another_streams_capture():
    """A graph is captured on torch's capture stream while the entry point runs
    on a separate non-blocking stream; its result equals bbw_wadg_update."""
    rng = np.random.default_rng(4)
    N, M, K = 5, 2, 77
    r = rounded(rng.standard_normal((K, _np3(N))), 32)
    c2 = rounded(rng.uniform(0.5, 2.0, (K, _np3(M))), 32)
    want = _run(B.wadg_update, N, M, 32, r, c2)
    dr = torch.tensor(r, dtype=torch.float32, device="cuda")
    dc = torch.tensor(c2, dtype=torch.float32, device="cuda")
    out = torch.full_like(dr, float("nan"))
    B.wadg_update_noalloc(N, M, 32, K, dr, dc, out)  # set-up before any capture
    torch.cuda.synchronize()
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    x = torch.ones(1024, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        y = x * 2.0
        B.wadg_update_noalloc(N, M, 32, K, dr, dc, out, stream=side.cuda_stream)
    side.synchronize()
    torch.cuda.synchronize()
    assert rel_l2(out.double().cpu().numpy(), want) <= TOL_STAGE[32]
    graph.replay()
    torch.cuda.synchronize()
    assert float(y[0]) == 2.0
