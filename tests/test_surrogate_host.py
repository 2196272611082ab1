"""Host-side pieces of the surrogate (no GPU): the straight-ray travel
times, receiver gains and receiver stencils that shape its targets and its
decoder, pinned by closed forms."""
import numpy as np

from paper_1808_08645_gb300 import inputs
from paper_1808_08645_gb300 import surrogate as S


def test_straight_ray_times_closed_forms():
    rng = np.random.default_rng(0)
    xs = rng.uniform(0.2, 0.8, (3, 3))
    rec = inputs.surrogate_receivers(4, 0.9)
    dist = np.linalg.norm(rec[None, :, :] - xs[:, None, :], axis=2)
    # constant medium c^2 = 4: time = distance / 2
    tau = S.straight_ray_times(lambda x: np.full(len(x), 4.0), xs, rec)
    assert np.allclose(tau, dist / 2.0, rtol=1e-14, atol=0)
    # slowness linear in z, 1/c = 0.7 + 0.5 z: the midpoint rule is exact,
    # time = distance x slowness at the segment's midpoint
    tau = S.straight_ray_times(lambda x: 1.0 / (0.7 + 0.5 * x[:, 2]) ** 2, xs, rec, nseg=7)
    zmid = 0.5 * (xs[:, None, 2] + rec[None, :, 2])
    assert np.allclose(tau, dist * (0.7 + 0.5 * zmid), rtol=1e-13, atol=0)


def test_receiver_gain_is_reference_distance_over_distance():
    xs = np.array([[0.5, 0.5, 0.6]])
    rec = np.array([[0.5, 0.5, 0.9], [0.1, 0.5, 0.9]])
    g = S.receiver_gain(xs, rec, d_ref=0.25)
    assert np.allclose(g[0], [0.25 / 0.3, 0.25 / 0.5], rtol=1e-14)


def test_receiver_stencils_bracket_the_receivers():
    """Each receiver's 2 x 2 x 2 grid stencil has cell centres on both sides of
    it in every direction, in the receivers' own order (x-major)."""
    for G, n, z in [(64, 8, 0.9), (16, 8, 0.9), (8, 2, 0.9)]:
        rec = inputs.surrogate_receivers(n, z)
        rx, ry, rz = S.receiver_corners(G, n, z)
        centre = lambda i: (np.asarray(i) + 0.5) / G
        for d, ix in enumerate((rx, ry, rz)):
            ix = np.asarray(ix)
            assert np.all(ix >= 0) and np.all(ix + 1 < G)
            assert np.all(centre(ix) <= rec[:, d] + 1e-12) and np.all(rec[:, d] <= centre(ix + 1) + 1e-12)
        cfg = S.default_config(grid=G, receivers=n, rec_z=z)
        assert (cfg["rx"], cfg["ry"], cfg["rz"]) == (rx, ry, rz)


def test_cosine_basis_matches_the_reference_network():
    from oracle import fno
    for n, m in ((64, 6), (16, 3)):
        assert np.allclose(S.cosine_basis(n, m), fno.cosine_basis(n, m), rtol=0, atol=1e-15)
