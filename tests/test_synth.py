"""The seeded input generators follow the stated recipe of each workload:
int32 (n, 2) arrays in [1, p]^2, a pure function of (n, p, seed), and each
distribution's defining property (the inscribed disc, the Gaussian's centre
and spread, the annulus radii, the clustered projected shells, the boxes of
the bounding-box workload, the size laws of the batched workload)."""
import numpy as np
import pytest

from paper_1505_00914_gb300 import synth


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
@pytest.mark.parametrize("p", [1, 7, 1024, 65536])
def test_shape_range_and_determinism(dist, p):
    n = 20_000
    a = synth.points(dist, n, p, seed=3)
    assert a.dtype == np.int32 and a.shape == (n, 2) and a.flags.c_contiguous
    assert a.min() >= 1 and a.max() <= p
    np.testing.assert_array_equal(a, synth.points(dist, n, p, seed=3))
    if p >= 1024:
        assert not np.array_equal(a, synth.points(dist, n, p, seed=4))
    assert synth.points(dist, 0, p, seed=3).shape == (0, 2)


def test_disc_is_uniform_over_the_inscribed_disc():
    p = 4096
    P = synth.disc(200_000, p, seed=1).astype(np.int64)
    d = (2 * P[:, 0] - (p + 1)) ** 2 + (2 * P[:, 1] - (p + 1)) ** 2  # (2 * distance)^2
    assert (d <= p * p).all()
    # uniform over the area: a quarter of the points within half the radius
    assert abs((d <= p * p // 4).mean() - 0.25) < 0.01


def test_gaussian_centre_and_spread():
    p = 65536
    P = synth.gaussian(400_000, p, seed=2).astype(np.float64)
    assert np.all(np.abs(P.mean(0) - (p + 1) / 2) < 0.005 * p)
    assert np.all(np.abs(P.std(0) - p / 8) < 0.005 * p)


def test_annulus_radii():
    p = 65536
    P = synth.annulus(200_000, p, seed=3).astype(np.float64)
    r = np.hypot(P[:, 0] - (p + 1) / 2, P[:, 1] - (p + 1) / 2)
    assert r.min() >= 0.45 * p - 1 and r.max() <= 0.5 * p + 1
    # uniform over the ring's area: half the points inside the radius that
    # splits the area in two
    r_med = np.sqrt(((0.45 * p) ** 2 + (0.5 * p) ** 2) / 2)
    assert abs((r <= r_med).mean() - 0.5) < 0.01


def test_shells_are_clustered_with_duplicates():
    """Against uniform points of the same n and p: fewer distinct points and
    far more uneven column counts (the stand-in's clustered columns)."""
    p, n = 4096, 1_000_000
    S = synth.shells(n, p, seed=0)
    U = synth.uniform(n, p, seed=0)

    def distinct(P):
        return np.unique(P[:, 0].astype(np.int64) * (p + 1) + P[:, 1]).size / n

    def column_cv(P):
        c = np.bincount(P[:, 0], minlength=p + 1)[1:]
        return c.std() / c.mean()

    assert distinct(S) < distinct(U) - 0.03
    assert column_cv(S) > 5 * column_cv(U)


def test_boxed_points_fill_their_box():
    sx, sy, x0, y0 = 120_000, 40_000, 1_000_000_000, -2_000_000_000
    P = synth.boxed("uniform", 300_000, sx, sy, x0, y0, seed=1).astype(np.int64)
    assert P[:, 0].min() >= x0 and P[:, 0].max() <= x0 + sx - 1
    assert P[:, 1].min() >= y0 and P[:, 1].max() <= y0 + sy - 1
    # uniform on the square, scaled: the box's corners are reached closely
    assert P[:, 0].min() - x0 < sx // 1000 and x0 + sx - 1 - P[:, 0].max() < sx // 1000
    assert P[:, 1].min() - y0 < sy // 1000 and y0 + sy - 1 - P[:, 1].max() < sy // 1000


def test_batched_size_laws():
    n, p, d = synth.batched_spec(10_000, seed=4)
    assert n.min() >= 100 and n.max() <= 1_000_000
    assert abs(np.log10(n).mean() - 4.0) < 0.05  # log-uniform over four decades
    sides, counts = np.unique(p, return_counts=True)
    assert tuple(sides) == (256, 1024, 4096, 16384)
    assert (np.abs(counts / 10_000 - 0.25) < 0.03).all()
    assert set(d) == {"uniform", "disc", "gaussian"}
    pts, offsets, ps, dists = synth.batched(50, seed=9)
    assert offsets[0] == 0 and offsets[-1] == pts.shape[0] and (np.diff(offsets) >= 0).all()
    for s in range(50):
        Q = pts[offsets[s]:offsets[s + 1]]
        assert Q.shape[0] == 0 or (Q.min() >= 1 and Q.max() <= ps[s])


def test_affine_keeps_the_square_and_the_seed():
    p = 16384
    P = synth.points("disc", 50_000, p, seed=5)
    A = synth.affine(P, p, seed=1)
    assert A.dtype == np.int32 and A.shape == P.shape and A.min() >= 1 and A.max() <= p
    np.testing.assert_array_equal(A, synth.affine(P, p, seed=1))
    assert not np.array_equal(A, synth.affine(P, p, seed=2))
