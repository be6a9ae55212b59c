"""Steps 1-2 of the paper's general procedure on the GPU: the bounding box,
then Algorithm 1 on the translated points with the columns along the shorter
side, and the hull back in the input's coordinates.  The reference is the
oracle's hull of the raw points (sort + Andrew, 64-bit orientation), which
needs no box at all; every comparison is exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

I32_MIN, I32_MAX = -(2 ** 31), 2 ** 31 - 1


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def check(P):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    d = dev(P).reshape(-1, 2)
    box = host(ch.ch_bbox(d))
    if P.shape[0]:
        np.testing.assert_array_equal(box, [P[:, 0].min(), P[:, 0].max(), P[:, 1].min(),
                                            P[:, 1].max()])
    h = host(ch.convex_hull(d))
    np.testing.assert_array_equal(h, oracle.hull_points(P))
    return box


def stretched(n, sx, sy, x0, y0, seed, dist="uniform"):
    """n points of a shape scaled to sx by sy and shifted to (x0, y0)."""
    base = synth.points(dist, n, 65536, seed=seed).astype(np.int64) - 1
    x = x0 + (base[:, 0] * (sx - 1)) // 65535
    y = y0 + (base[:, 1] * (sy - 1)) // 65535
    return np.stack([x, y], 1).astype(np.int32)


def test_bbox_of_nothing():
    box = host(ch.ch_bbox(torch.empty((0, 2), dtype=torch.int32, device="cuda")))
    np.testing.assert_array_equal(box, [I32_MAX, I32_MIN, I32_MAX, I32_MIN])


@pytest.mark.parametrize("sx,sy", [(1000, 1000), (5000, 300), (300, 5000), (1, 700), (700, 1),
                                   (1, 1), (16384, 16384), (16384, 16385), (16385, 16384),
                                   (12000, 40000), (29056, 70000), (70000, 29056), (70000, 300000),
                                   (300000, 70000), (130000, 200000), (200000, 130000)])
@pytest.mark.parametrize("dist", ["uniform", "disc", "gaussian", "shells"])
def test_any_box_matches_the_oracle(sx, sy, dist):
    rng = np.random.default_rng(sx * 7 + sy)
    x0 = int(rng.integers(-2 ** 30, 2 ** 30 - 300000))
    y0 = int(rng.integers(-2 ** 30, 2 ** 30 - 300000))
    check(stretched(400_001, sx, sy, x0, y0, seed=sx + sy, dist=dist))


def test_extreme_coordinates_and_small_sets():
    rng = np.random.default_rng(3)
    for n in (1, 2, 3, 7, 100):
        check(rng.integers(-50, 50, size=(n, 2)))
    # near both ends of int32, sides up to 2^30
    lo = np.array([I32_MIN, I32_MIN], np.int64)
    P = lo + rng.integers(0, 2 ** 30, size=(50_000, 2))
    check(P)
    hi = np.array([I32_MAX, I32_MAX], np.int64)
    check(hi - rng.integers(0, 2 ** 30, size=(50_000, 2)))
    check(np.array([[I32_MAX, I32_MIN]] * 10))


def test_point_outside_the_given_box_is_reported():
    P = stretched(10_000, 500, 400, 100, 200, seed=1)
    d = dev(P).reshape(-1, 2)
    box = [P[:, 0].min(), P[:, 0].max() - 1, P[:, 1].min(), P[:, 1].max()]  # x range one short
    ch.ch_convex_hull_box(d, box)
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE


def test_box_sides_beyond_the_limit_are_rejected():
    d = dev(np.zeros((4, 2), np.int32)).reshape(-1, 2)
    with pytest.raises(ch.ChError) as e:
        ch.ch_convex_hull_box(d, [0, 2 ** 30, 0, 10])
    assert e.value.code == ch.CH_ERR_ARG
    with pytest.raises(ch.ChError):
        ch.ch_convex_hull_box(d, [5, 4, 0, 10])  # empty box


@pytest.mark.slow
def test_box_path_at_bench_size():
    """The bench's Steps 1-2 workload, one instance at full size (2^26 points
    of a 120000 x 40000 box at (1e9, -2e9), columns along y): the box, the
    hull through the user call, against the oracle's Steps 1-2."""
    P = synth.boxed("disc", 1 << 26, 120_000, 40_000, 1_000_000_000, -2_000_000_000, seed=32)
    H = oracle.hull_box(P)
    d = dev(P).reshape(-1, 2)
    box = host(ch.ch_bbox(d))
    np.testing.assert_array_equal(box, [P[:, 0].min(), P[:, 0].max(), P[:, 1].min(), P[:, 1].max()])
    del P
    np.testing.assert_array_equal(host(ch.convex_hull(d)), H)
