"""Pins for two more oracle functions, each against hulls computed another
way (brute force from the definition of a hull edge, or sort + Andrew):

* Melkman's hull of a simple polyline (the hull algorithm the paper runs on
  its reduced set in Section 3, Fig. 10), on Lemma 1 polylines and on other
  simple polylines (star-shaped, x-monotone, convex in either orientation);
* Steps 1-2 of the general procedure (Section 2): bounding box, translation,
  Algorithm 1 along the shorter side, for points anywhere in int32."""
import numpy as np
import pytest

import oracle
from paper_1505_00914_gb300 import synth
from test_oracle import _fig1_points, _segments_cross, _tiny_sets

I32_MIN, I32_MAX = -(2 ** 31), 2 ** 31 - 1


def _simple(poly):
    e = [(poly[i], poly[i + 1]) for i in range(len(poly) - 1)]
    return all(not _segments_cross(e[i][0], e[i][1], e[j][0], e[j][1])
               for i in range(len(e)) for j in range(i + 2, len(e)))


def _star(rng, m, r):
    """m integer points with distinct directions from an integer centre,
    ordered by angle around it with every angular gap (the closing one
    included) below pi, so each edge stays in its own convex sector: any run
    of consecutive vertices of the ring is a simple open polyline."""
    c = rng.integers(-r, r + 1, size=2)
    while True:
        d = rng.integers(-r, r + 1, size=(4 * m, 2))
        d = d[np.any(d != 0, axis=1)]
        g = np.gcd(d[:, 0], d[:, 1])
        prim = d // g[:, None]
        _, first = np.unique(prim, axis=0, return_index=True)
        d = d[np.sort(first)][:m]
        ang = np.arctan2(d[:, 1], d[:, 0])
        o = np.argsort(ang)
        d, ang = d[o], ang[o]
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2 * np.pi]))
        if len(d) >= 3 and np.all(gaps < np.pi - 1e-9):
            k = int(rng.integers(0, len(d)))  # start anywhere along the ring
            d = np.roll(d, -k, axis=0)
            d = d[: len(d) - 1] if len(d) > 3 else d  # open: drop the closing vertex
            return (d + c).astype(np.int32)


def test_melkman_fig1_is_the_pentagon():
    L = oracle.reduce(_fig1_points(), 5)
    np.testing.assert_array_equal(oracle.melkman(oracle.polyline(L)),
                                  [[1, 1], [5, 2], [5, 3], [3, 5], [1, 4]])


def test_melkman_on_lemma1_polylines_matches_brute_force():
    for P, p in _tiny_sets(6000, seed=3):
        poly = oracle.polyline(oracle.reduce(P, p))
        np.testing.assert_array_equal(oracle.melkman(poly), oracle.hull_brute(P))


def test_melkman_on_star_shaped_polylines():
    rng = np.random.default_rng(5)
    for it in range(1500):
        m = int(rng.integers(3, 14))
        poly = _star(rng, m, int(rng.integers(2, 6)))
        assert _simple(poly)
        np.testing.assert_array_equal(oracle.melkman(poly), oracle.hull_brute(poly), err_msg=str(poly))
        np.testing.assert_array_equal(oracle.melkman(poly[::-1]), oracle.hull_brute(poly))


def test_melkman_on_x_monotone_and_convex_polylines():
    rng = np.random.default_rng(6)
    for it in range(800):
        m = int(rng.integers(1, 16))
        xs = np.sort(rng.choice(np.arange(-20, 21), size=m, replace=False))
        P = np.stack([xs, rng.integers(-4, 5, size=m)], 1).astype(np.int32)
        np.testing.assert_array_equal(oracle.melkman(P), oracle.hull_brute(P))
        np.testing.assert_array_equal(oracle.melkman(P[::-1]), oracle.hull_brute(P))
    # vertices of a strictly convex polygon, from any start, either direction
    C = oracle.hull_points(synth.points("disc", 5000, 200, seed=2))
    for k in (0, 1, len(C) // 2, len(C) - 1):
        R = np.roll(C, -k, axis=0)
        np.testing.assert_array_equal(oracle.melkman(R), C)
        np.testing.assert_array_equal(oracle.melkman(R[::-1]), C)


def test_melkman_collinear_walk_back_is_dropped():
    # the path returns along a hull edge: the returning vertex is not strict
    poly = np.asarray([[0, 0], [2, -3], [4, 0], [2, 0]], np.int32)
    assert _simple(poly)
    np.testing.assert_array_equal(oracle.melkman(poly), [[0, 0], [2, -3], [4, 0]])


def test_melkman_degenerate():
    assert oracle.melkman(np.zeros((0, 2), np.int32)).shape == (0, 2)
    np.testing.assert_array_equal(oracle.melkman([[3, 4]]), [[3, 4]])
    np.testing.assert_array_equal(oracle.melkman([[3, 4], [1, 2]]), [[1, 2], [3, 4]])
    line = np.asarray([[k, 2 * k] for k in (3, 4, 5, 2, 1)], np.int32)  # simple: a zigzag on one line is not
    np.testing.assert_array_equal(oracle.melkman([[1, 2], [2, 4], [3, 6]]), [[1, 2], [3, 6]])
    # a collinear prefix, then a vertex off its line
    poly = np.asarray([[1, 1], [2, 1], [3, 1], [4, 1], [2, 5]], np.int32)
    np.testing.assert_array_equal(oracle.melkman(poly), [[1, 1], [4, 1], [2, 5]])
    poly = np.asarray([[4, 1], [3, 1], [2, 1], [1, 1], [2, -5]], np.int32)
    np.testing.assert_array_equal(oracle.melkman(poly), [[1, 1], [2, -5], [4, 1]])
    del line


@pytest.mark.parametrize("dist", ["uniform", "disc", "gaussian", "annulus", "shells"])
def test_melkman_on_synthetic_lemma1_polylines(dist):
    for p, n in ((64, 5000), (1024, 200_000), (4096, 300_000)):
        P = synth.points(dist, n, p, seed=p)
        poly = oracle.polyline(oracle.reduce(P, p))
        np.testing.assert_array_equal(oracle.melkman(poly), oracle.hull_points(P))


def _stretched(n, sx, sy, x0, y0, seed, dist="uniform"):
    base = synth.points(dist, n, 65536, seed=seed).astype(np.int64) - 1
    x = x0 + (base[:, 0] * (sx - 1)) // 65535
    y = y0 + (base[:, 1] * (sy - 1)) // 65535
    return np.stack([x, y], 1).astype(np.int32)


def test_hull_box_matches_brute_force_on_tiny_sets():
    rng = np.random.default_rng(8)
    for P, p in _tiny_sets(4000, seed=9):
        if P.shape[0] == 0:
            continue
        off = rng.integers(-2 ** 31, 2 ** 31 - 16, size=2)
        Q = (P.astype(np.int64) + off).astype(np.int32)
        if rng.integers(0, 2):
            Q = Q[:, ::-1].copy()
        np.testing.assert_array_equal(oracle.hull_box(Q), oracle.hull_brute(Q))


@pytest.mark.parametrize("sx,sy", [(1000, 1000), (5000, 300), (300, 5000), (1, 700), (700, 1),
                                   (1, 1), (70000, 300000), (300000, 70000)])
@pytest.mark.parametrize("dist", ["uniform", "disc", "gaussian", "shells"])
def test_hull_box_matches_sort_and_andrew(sx, sy, dist):
    rng = np.random.default_rng(sx * 3 + sy)
    x0 = int(rng.integers(I32_MIN, I32_MAX - 300000))
    y0 = int(rng.integers(I32_MIN, I32_MAX - 300000))
    P = _stretched(100_003, sx, sy, x0, y0, seed=sx + sy, dist=dist)
    np.testing.assert_array_equal(oracle.hull_box(P), oracle.hull_points(P))


def test_hull_box_at_the_ends_of_int32_and_on_the_plain_square():
    P = np.asarray([[I32_MIN, I32_MIN], [I32_MIN + 5, I32_MIN + 1], [I32_MIN + 2, I32_MIN + 9]],
                   np.int32)
    np.testing.assert_array_equal(oracle.hull_box(P), oracle.hull_brute(P))
    Q = np.asarray([[I32_MAX, I32_MAX], [I32_MAX - 7, I32_MAX], [I32_MAX - 3, I32_MAX - 2]], np.int32)
    np.testing.assert_array_equal(oracle.hull_box(Q), oracle.hull_brute(Q))
    # a set that spans [1, p]^2 exactly is the plain path's input
    p = 1024
    S = np.concatenate([synth.points("disc", 50_000, p, seed=1), [[1, 1], [p, p]]]).astype(np.int32)
    np.testing.assert_array_equal(oracle.hull_box(S), oracle.hull(S, p))
    with pytest.raises(ValueError):
        oracle.hull_box(np.asarray([[0, 0], [2 ** 30, 5]], np.int32))


def test_chain_points_equals_the_scan_of_L():
    """The chains taken from the points directly (for sides too large for L)
    equal the Lemma 1 scan of Algorithm 1's array."""
    for P, p in _tiny_sets(3000, seed=17):
        lo, up = oracle.chain_points(P)
        lo2, up2 = oracle.chain(oracle.reduce(P, p))
        np.testing.assert_array_equal(lo, lo2)
        np.testing.assert_array_equal(up, up2)
    for dist in ("uniform", "gaussian", "shells"):
        P = synth.points(dist, 200_000, 70_000, seed=4)
        lo, up = oracle.chain_points(P)
        lo2, up2 = oracle.chain(oracle.reduce(P, 70_000))
        np.testing.assert_array_equal(lo, lo2)
        np.testing.assert_array_equal(up, up2)


def test_second_scan_on_fig1():
    """Fig. 1's L: the rx points are (1,1) (1,4) (2,2) (2,4) (3,2) (3,5)
    (4,3) (5,2) (5,3); scanning them along y keeps, per row, the leftmost
    and rightmost: row 1 (1,1); row 2 x in {2,3,5}; row 3 x in {4,5}; row 4
    x in {1,2}; row 5 (3,5).  One point, (3,2), goes; the pentagon stays."""
    L = oracle.reduce(_fig1_points(), 5)
    R = oracle.reduce_rows(L)
    np.testing.assert_array_equal(R, [[1, 1], [2, 5], [4, 5], [1, 2], [3, 3]])
    rxy = oracle.rxy_points(R)
    assert rxy.shape[0] == 8 and oracle.rx_points(L).shape[0] == 9
    np.testing.assert_array_equal(oracle.hull_points(rxy), [[1, 1], [5, 2], [5, 3], [3, 5], [1, 4]])


def test_second_scan_is_algorithm1_on_the_transposed_rx_points():
    """The second scan is Algorithm 1 over the rx points with x and y
    exchanged; the rxy set is a subset of rx, at most min(2q, |rx|) points,
    and keeps the hull (brute force)."""
    for P, p in _tiny_sets(3000, seed=23):
        L = oracle.reduce(P, p)
        rx = oracle.rx_points(L)
        R = oracle.reduce_rows(L)
        np.testing.assert_array_equal(R, oracle.reduce(rx[:, ::-1], p))
        rxy = oracle.rxy_points(R)
        assert rxy.shape[0] <= min(2 * p, rx.shape[0])
        assert set(map(tuple, rxy)) <= set(map(tuple, rx))
        np.testing.assert_array_equal(oracle.hull_brute(rxy), oracle.hull_brute(P))
    # full lattice square: rx is the top and bottom of every column, rxy the corners
    p = 9
    P = np.asarray([(x, y) for x in range(1, p + 1) for y in range(1, p + 1)], np.int32)
    rxy = oracle.rxy_points(oracle.reduce_rows(oracle.reduce(P, p)))
    np.testing.assert_array_equal(rxy, [[1, 1], [p, 1], [1, p], [p, p]])
    for dist in ("disc", "shells"):
        P = synth.points(dist, 300_000, 4096, seed=5)
        L = oracle.reduce(P, 4096)
        rxy = oracle.rxy_points(oracle.reduce_rows(L))
        assert rxy.shape[0] < oracle.rx_points(L).shape[0]
        np.testing.assert_array_equal(oracle.hull_points(rxy), oracle.hull_points(P))


def test_tree_sizes_printed_in_the_paper():
    """Section 4: for p = 2^24 and 64-bit words the tree has height 3 above
    its leaf words and 266305 words, 4161 more than the flat array of 262144
    words; height h = log_w((w - 1) p + w) - 2 and m = (w^(h+1) - 1)/(w - 1)."""
    import math
    p, w = 1 << 24, 64
    words = oracle.tree_words(p, w)
    assert words == [262144, 4096, 64, 1]
    assert sum(words) == 266305 and sum(words) - words[0] == 4161
    h = len(words) - 1
    assert h == 3 == math.ceil(math.log((w - 1) * p + w, w) - 2)
    assert sum(words) == (w ** (h + 1) - 1) // (w - 1)
    assert oracle.tree_words(1, 32) == [1] and oracle.tree_words(33, 32) == [2, 1]
