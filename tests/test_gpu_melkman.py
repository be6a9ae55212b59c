"""Parity of the Lemma 1 polyline and of Melkman's hull on the GPU with the
oracle (Section 2.1; Section 3, Fig. 10).  Integer work: the polyline, its
length and every hull are compared bit-exactly."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def gpu_polyline(L, p):
    poly, cnt = ch.ch_polyline(dev(L).reshape(-1, 2), p)
    c = int(host(cnt)[0])
    return host(poly)[:c]


def gpu_melkman(poly, p):
    poly = np.ascontiguousarray(poly, dtype=np.int32).reshape(-1, 2)
    d = dev(poly).reshape(-1, 2) if poly.shape[0] else torch.empty((1, 2), dtype=torch.int32,
                                                                   device="cuda")
    cnt = torch.tensor([poly.shape[0]], dtype=torch.int32, device="cuda")
    h, hc = ch.ch_hull_melkman(d, cnt, p)
    return host(h)[: int(host(hc)[0])]


def star(rng, m, r, p):
    """A simple open polyline of about m vertices inside [1, p]^2: integer
    points of distinct directions around the box centre, in angular order,
    every angular gap below pi."""
    c = np.array([(p + 1) // 2, (p + 1) // 2])
    while True:
        d = rng.integers(-r, r + 1, size=(2 * m, 2))
        d = d[np.any(d != 0, axis=1)]
        g = np.gcd(d[:, 0], d[:, 1])
        _, first = np.unique(d // g[:, None], axis=0, return_index=True)
        d = d[np.sort(first)][:m]
        ang = np.arctan2(d[:, 1], d[:, 0])
        o = np.argsort(ang)
        d, ang = d[o], ang[o]
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2 * np.pi]))
        if len(d) >= 3 and np.all(gaps < np.pi - 1e-9):
            k = int(rng.integers(0, len(d)))
            d = np.roll(d, -k, axis=0)[:-1]
            return (d + c).astype(np.int32)


DISTS = ("uniform", "disc", "gaussian", "annulus", "shells")


@pytest.mark.parametrize("dist", DISTS)
@pytest.mark.parametrize("p,n", [(1024, 100_000), (4096, 262_145), (3000, 50_000),
                                 (65536, 2_000_001), (300_000, 1_000_000)])
def test_polyline_and_melkman_match_the_oracle(dist, p, n):
    P = synth.points(dist, n, p, seed=p + n)
    L = oracle.reduce(P, p)
    poly = gpu_polyline(L, p)
    np.testing.assert_array_equal(poly, oracle.polyline(L))
    H = oracle.hull_points(P)
    np.testing.assert_array_equal(oracle.melkman(poly), H)
    np.testing.assert_array_equal(gpu_melkman(poly, p), H)
    fused_matches(P, p, poly, H)


def fused_matches(P, p, poly_full, H):
    """ch_convex_hull_melkman: the hull is exact; its polyline is the Lemma 1
    polyline with some non-vertices removed (a subsequence holding every hull
    vertex), and Melkman on it alone gives the hull again."""
    d = dev(P).reshape(-1, 2) if P.shape[0] else torch.empty((0, 2), dtype=torch.int32,
                                                             device="cuda")
    poly = torch.empty((2 * p, 2), dtype=torch.int32, device="cuda")
    pc = torch.empty(1, dtype=torch.int32, device="cuda")
    h, hc = ch.ch_convex_hull_melkman(d, p, poly=poly, poly_count=pc)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)
    sub = host(poly)[: int(host(pc)[0])]
    assert sub.shape[0] <= poly_full.shape[0]
    # subsequence of the full polyline
    key = lambda a: a[:, 0].astype(np.int64) * (1 << 32) + a[:, 1]
    kf, ks = key(poly_full), key(sub)
    pos = np.searchsorted(kf, ks)  # the Lemma 1 polyline is sorted by (x, y)
    assert np.all(pos < kf.shape[0]) and np.all(kf[np.minimum(pos, kf.shape[0] - 1)] == ks)
    assert np.all(np.diff(pos) > 0)
    # every hull vertex kept, and Melkman on the shorter polyline agrees
    assert set(map(tuple, H)) <= set(map(tuple, sub))
    np.testing.assert_array_equal(oracle.melkman(sub), H)
    return sub


@pytest.mark.parametrize("p", [1, 2, 3, 5, 33, 1025])
@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000])
def test_small_and_degenerate(p, n):
    rng = np.random.default_rng(p * 100 + n)
    P = rng.integers(1, p + 1, size=(n, 2)).astype(np.int32)
    L = oracle.reduce(P, p)
    poly = gpu_polyline(L, p)
    np.testing.assert_array_equal(poly, oracle.polyline(L))
    np.testing.assert_array_equal(gpu_melkman(poly, p), oracle.hull_points(P))
    fused_matches(P, p, poly, oracle.hull_points(P))


def _segments_meet(a, b, c, d):
    def orient(o, u, v):
        return int(np.sign((int(u[0]) - o[0]) * (int(v[1]) - o[1]) - (int(u[1]) - o[1]) * (int(v[0]) - o[0])))

    def on(o, u, v):
        return min(o[0], u[0]) <= v[0] <= max(o[0], u[0]) and min(o[1], u[1]) <= v[1] <= max(o[1], u[1])
    o1, o2, o3, o4 = orient(a, b, c), orient(a, b, d), orient(c, d, a), orient(c, d, b)
    if o1 * o2 < 0 and o3 * o4 < 0:
        return True
    return ((o1 == 0 and on(a, b, c)) or (o2 == 0 and on(a, b, d)) or
            (o3 == 0 and on(c, d, a)) or (o4 == 0 and on(c, d, b)))


@pytest.mark.parametrize("dist", DISTS)
def test_filtered_polyline_is_simple(dist):
    """The polyline the fused path hands to Melkman is still simple."""
    p, n = 40, 3000
    P = synth.points(dist, n, p, seed=77)
    L = oracle.reduce(P, p)
    sub = fused_matches(P, p, oracle.polyline(L), oracle.hull_points(P))
    e = [(sub[i], sub[i + 1]) for i in range(sub.shape[0] - 1)]
    for i in range(len(e)):
        for j in range(i + 2, len(e)):
            assert not _segments_meet(e[i][0], e[i][1], e[j][0], e[j][1]), (i, j)


def test_collinear_and_walk_back_polylines():
    p = 100
    cases = [
        [[1, 1], [2, 1], [3, 1], [4, 1], [2, 5]],
        [[4, 1], [3, 1], [2, 1], [1, 1], [2, 7]],
        [[1, 2], [2, 4], [3, 6], [50, 100]],
        [[10, 10], [12, 7], [14, 10], [12, 10]],
        [[5, 5], [6, 6], [7, 7], [8, 8]],
        [[9, 9]],
    ]
    for c in cases:
        c = np.asarray(c, np.int32)
        np.testing.assert_array_equal(gpu_melkman(c, p), oracle.melkman(c))
        np.testing.assert_array_equal(gpu_melkman(c, p), oracle.hull_points(c))


def test_star_shaped_and_monotone_polylines():
    rng = np.random.default_rng(12)
    p = 8192
    for m, r in ((10, 3), (200, 40), (5000, 400), (60_000, 1500)):
        for _ in range(3):
            poly = star(rng, m, r, p)
            H = oracle.hull_points(poly)
            np.testing.assert_array_equal(oracle.melkman(poly), H)
            np.testing.assert_array_equal(gpu_melkman(poly, p), H)
            np.testing.assert_array_equal(gpu_melkman(poly[::-1], p), H)
    # x-monotone polylines over several staging rounds
    for m in (31, 32, 33, 1023, 1024, 1025, 5000):
        xs = np.sort(rng.choice(np.arange(1, p + 1), size=m, replace=False))
        poly = np.stack([xs, rng.integers(1, p + 1, size=m)], 1).astype(np.int32)
        np.testing.assert_array_equal(gpu_melkman(poly, p), oracle.hull_points(poly))
    # vertices of a convex polygon, from any start, both directions
    C = oracle.hull_points(synth.points("disc", 400_000, p, seed=3))
    for k in (0, 7, len(C) // 2):
        R = np.roll(C, -k, axis=0)
        np.testing.assert_array_equal(gpu_melkman(R, p), C)
        np.testing.assert_array_equal(gpu_melkman(R[::-1], p), C)


def test_deque_in_global_memory_for_large_sides():
    """Above p of about 2^17 the largest lattice hull outgrows the shared-memory
    deque and the deque moves to the workspace."""
    p = 1 << 21
    assert ch.ch_hull_melkman_workspace_size(p) > 0
    assert ch.ch_hull_melkman_workspace_size(65536) == 0
    P = synth.points("disc", 3_000_000, p, seed=8)
    L = oracle.reduce(P, p)
    poly = gpu_polyline(L, p)
    np.testing.assert_array_equal(poly, oracle.polyline(L))
    np.testing.assert_array_equal(gpu_melkman(poly, p), oracle.hull_points(P))


def test_vertex_outside_the_square_is_reported():
    p = 64
    poly = np.asarray([[1, 1], [5, 2], [65, 3]], np.int32)
    d = dev(poly)
    cnt = torch.tensor([3], dtype=torch.int32, device="cuda")
    h, hc = ch.ch_hull_melkman(d, cnt, p)
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    assert int(host(hc)[0]) == 0


@pytest.mark.slow
@pytest.mark.parametrize("dist", ("uniform", "disc", "gaussian"))
def test_melkman_path_full_size(dist):
    """n = 2^26 at p = 65536 (the plain path's timed size): the hull through
    the polyline and Melkman equals the oracle's and the plain path's."""
    p, n = 65536, 1 << 26
    P = synth.points(dist, n, p, seed=21)
    H = oracle.hull(P, p)
    d = dev(P).reshape(-1, 2)
    del P
    h, hc = ch.ch_convex_hull_melkman(d, p)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)


@pytest.mark.parametrize("p", [32768, 32769])
def test_full_scale_coordinates_at_the_32_bit_boundary(p):
    """Up to p = 2^15 the orientation runs in 32-bit arithmetic; polylines
    spanning the whole square, with near-collinear triples, at both sides of
    that boundary."""
    rng = np.random.default_rng(p)
    for m in (50, 4000):
        poly = star(rng, m, (p - 2) // 2, p)
        np.testing.assert_array_equal(gpu_melkman(poly, p), oracle.hull_points(poly))
    # long thin fans: every triple nearly collinear over the full width
    xs = np.arange(1, p + 1, 97)
    lo = np.stack([xs, 1 + (xs * 3) // p], 1)
    hi = np.stack([xs[::-1], p - (xs[::-1] * 5) // p], 1)
    poly = np.concatenate([lo, hi]).astype(np.int32)
    np.testing.assert_array_equal(oracle.melkman(poly), oracle.hull_points(poly))
    np.testing.assert_array_equal(gpu_melkman(poly, p), oracle.hull_points(poly))


def test_coordinates_up_to_two_to_the_thirty():
    """p = 2^30, the largest side: the deque in global memory and the 64-bit
    orientation, on star-shaped polylines spanning the whole square (vertices
    in angular order around the centre, every gap below pi, so simple)."""
    p = 1 << 30
    rng = np.random.default_rng(30)
    c = (p + 1) // 2
    for m in (5, 300, 20_000):
        ang = np.sort(rng.uniform(-np.pi, np.pi, size=m))
        ang = ang[np.concatenate([[True], np.diff(ang) > 1e-6])]
        r = rng.uniform(0.2, 0.499, size=ang.shape[0]) * p
        poly = np.stack([c + np.rint(r * np.cos(ang)), c + np.rint(r * np.sin(ang))], 1)
        poly = poly.astype(np.int64)
        d = poly - c
        a2 = np.arctan2(d[:, 1], d[:, 0])
        gaps = np.diff(np.concatenate([a2, a2[:1] + 2 * np.pi]))
        assert np.all(np.diff(a2) > 0) and np.all(gaps < np.pi)  # still a star in angular order
        poly = poly[:-1].astype(np.int32)  # open
        assert poly.min() >= 1 and poly.max() <= p
        H = oracle.hull_points(poly)
        np.testing.assert_array_equal(oracle.melkman(poly), H)
        np.testing.assert_array_equal(gpu_melkman(poly, p), H)
