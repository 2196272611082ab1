"""The allocation-free weight-adjusted update (bbw_wadg_update_noalloc).

Callers that cannot allocate device memory (code running while a CUDA graph
is captured on another stream, frameworks that own the whole memory pool,
latency-critical loops) use this entry point; it keeps its operator tables in
the library's static device memory instead of a cache it allocates. These
tests call it through the C ABI and compare it with bbw_wadg_update on two
calls in a row. The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1808_08645_gb300 import binding as B

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
