"""Pins for the CPU oracle: values the paper prints, brute force on tiny inputs,
closed forms and invariants.  None of these re-types the oracle's own formulas:
each checks it against something the paper or the mathematics fixes."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1505_00914_gb300 import synth
from _golden import read

pytestmark = pytest.mark.filterwarnings("ignore")


def _fig1_points(gapped=False, seed=0):
    """A point set consistent with Fig. 1: every (x, y) with ly <= y <= hy of
    the printed L (the paper draws P but prints only L), duplicated and
    shuffled.  Interior points of a column cannot change its (min, max)."""
    _, L = read("fig1_gapped_L.txt" if gapped else "fig1_L.txt")
    pts = []
    for x, (ly, hy) in enumerate(L, start=1):
        if ly > hy:
            continue
        for y in range(ly, hy + 1):
            pts += [(x, y)] * (1 + (x + y) % 3)
    pts = np.asarray(pts, dtype=np.int32)
    return np.random.default_rng(seed).permutation(pts)


def test_fig1_reduction_matches_paper():
    keys, L = read("fig1_L.txt")
    for seed in range(5):
        got = oracle.reduce(_fig1_points(seed=seed), keys["p"])
        np.testing.assert_array_equal(got, L)


def test_fig1_gapped_reduction_and_mask():
    keys, L = read("fig1_gapped_L.txt")
    got = oracle.reduce(_fig1_points(gapped=True), keys["p"])
    np.testing.assert_array_equal(got, L)
    np.testing.assert_array_equal(oracle.mask(got), np.asarray([keys["mask"]], np.uint32))
    lo, up = oracle.chain(got)
    np.testing.assert_array_equal(lo[:, 0], [1, 3, 5])
    np.testing.assert_array_equal(lo[:, 1], [1, 2, 2])
    np.testing.assert_array_equal(up[:, 1], [4, 5, 3])


def test_table1_ctz_walk_over_mask():
    keys, _ = read("table1_ctz.txt")
    gk, L = read("fig1_gapped_L.txt")
    word = int(oracle.mask(L)[0])
    assert word == keys["word"]
    pos, x = [], word
    while x:
        b = (x & -x).bit_length() - 1  # count trailing zeros
        pos.append(b)
        x ^= 1 << b
    assert pos == keys["positions"]


def test_block_bit_index_example():
    keys, _ = read("block_index.txt")
    i = keys["i"]
    p = 1 << 17
    L = oracle.reduce(np.asarray([[i, 7]], np.int32), p)
    M = oracle.mask(L)
    nz = np.flatnonzero(M)
    assert list(nz) == [keys["block"]]
    assert int(M[keys["block"]]) == 1 << keys["bit"]
    assert keys["block"] * keys["w"] + keys["bit"] + 1 == i


def test_fig1_hull_is_the_pentagon():
    keys, H = read("fig1_hull.txt")
    P = _fig1_points()
    L = oracle.reduce(P, 5)
    for h in (oracle.hull_chain(L), oracle.hull_points(P), oracle.hull_brute(P)):
        assert h.shape[0] == keys["count"]
        np.testing.assert_array_equal(h, H)


def _tiny_sets(count, seed):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        p = int(rng.integers(1, 9))
        n = int(rng.integers(0, 13))
        mode = rng.integers(0, 4)
        if mode == 0:  # random
            P = rng.integers(1, p + 1, size=(n, 2))
        elif mode == 1:  # collinear on a random lattice line
            dx, dy = rng.integers(-2, 3, size=2)
            x0, y0 = rng.integers(1, p + 1, size=2)
            t = rng.integers(-p, p + 1, size=n)
            P = np.stack([x0 + t * dx, y0 + t * dy], 1)
            P = P[(P.min(1) >= 1) & (P.max(1) <= p)]
        elif mode == 2:  # few distinct points, many duplicates
            base = rng.integers(1, p + 1, size=(3, 2))
            P = base[rng.integers(0, 3, size=n)]
        else:  # one or two columns only
            xs = rng.integers(1, p + 1, size=2)
            P = np.stack([xs[rng.integers(0, 2, size=n)], rng.integers(1, p + 1, size=n)], 1)
        yield np.asarray(P, np.int32).reshape(-1, 2), p


def test_andrew_matches_brute_force_on_tiny_sets():
    for P, p in _tiny_sets(10000, seed=1):
        hb = oracle.hull_brute(P)
        np.testing.assert_array_equal(oracle.hull_points(P), hb)
        # the paper's claim (Appendix): the hull of L's points is the hull of P
        np.testing.assert_array_equal(oracle.hull_chain(oracle.reduce(P, p)), hb)


def test_brute_force_closed_forms():
    # full lattice square: the four corners
    p = 6
    P = np.asarray(list(itertools.product(range(1, p + 1), repeat=2)), np.int32)
    corners = np.asarray([[1, 1], [p, 1], [p, p], [1, p]], np.int32)
    np.testing.assert_array_equal(oracle.hull_brute(P), corners)
    np.testing.assert_array_equal(oracle.hull_points(P), corners)
    L = oracle.reduce(P, p)
    np.testing.assert_array_equal(L, np.tile([1, p], (p, 1)))
    np.testing.assert_array_equal(oracle.hull_chain(L), corners)
    # lattice triangle with collinear edge points: only the three corners
    T = np.asarray([(x, y) for x in range(1, 8) for y in range(1, 8) if y <= x], np.int32)
    np.testing.assert_array_equal(oracle.hull_points(T), [[1, 1], [7, 1], [7, 7]])
    # strictly convex lower chain y = k(k-1)/2 + 1: every point is a vertex
    m = 9
    C = np.asarray([(k, k * (k - 1) // 2 + 1) for k in range(1, m + 1)], np.int32)
    h = oracle.hull_points(C)
    assert h.shape[0] == m
    np.testing.assert_array_equal(oracle.hull_brute(C), h)


def test_degenerate_cases():
    p = 7
    empty = np.zeros((0, 2), np.int32)
    L = oracle.reduce(empty, p)
    np.testing.assert_array_equal(L, np.tile([p + 1, -1], (p, 1)))
    lo, up = oracle.chain(L)
    assert lo.shape == (0, 2) and up.shape == (0, 2)
    assert oracle.hull_chain(L).shape == (0, 2)
    assert oracle.hull_points(empty).shape == (0, 2)
    one = np.asarray([[3, 4]] * 5, np.int32)
    np.testing.assert_array_equal(oracle.hull_chain(oracle.reduce(one, p)), [[3, 4]])
    col = np.asarray([[2, 5], [2, 1], [2, 3]], np.int32)
    np.testing.assert_array_equal(oracle.hull_chain(oracle.reduce(col, p)), [[2, 1], [2, 5]])
    diag = np.asarray([[k, k] for k in range(1, 8)], np.int32)
    np.testing.assert_array_equal(oracle.hull_chain(oracle.reduce(diag, p)), [[1, 1], [7, 7]])
    flat = np.asarray([[k, 3] for k in (5, 1, 4)], np.int32)
    np.testing.assert_array_equal(oracle.hull_chain(oracle.reduce(flat, p)), [[1, 3], [5, 3]])
    anti = np.asarray([[k, 8 - k] for k in range(1, 8)], np.int32)
    np.testing.assert_array_equal(oracle.hull_chain(oracle.reduce(anti, p)), [[1, 7], [7, 1]])


def test_out_of_range_points_are_rejected():
    for bad in ([0, 1], [1, 0], [6, 1], [1, 6], [-3, 2]):
        with pytest.raises(oracle.OracleRangeError):
            oracle.reduce(np.asarray([[1, 1], bad], np.int32), 5)


def test_order_independence_and_merge_property():
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = int(rng.integers(1, 200))
        P = rng.integers(1, p + 1, size=(int(rng.integers(0, 2000)), 2)).astype(np.int32)
        L = oracle.reduce(P, p)
        np.testing.assert_array_equal(oracle.reduce(rng.permutation(P), p), L)
        k = int(rng.integers(0, P.shape[0] + 1))
        L1, L2 = oracle.reduce(P[:k], p), oracle.reduce(P[k:], p)
        merged = np.stack([np.minimum(L1[:, 0], L2[:, 0]), np.maximum(L1[:, 1], L2[:, 1])], 1)
        np.testing.assert_array_equal(merged, L)


def _segments_cross(a, b, c, d):
    """Proper or touching intersection of segments ab and cd (exact ints)."""
    def orient(o, u, v):
        return int(np.sign((u[0] - o[0]) * (v[1] - o[1]) - (u[1] - o[1]) * (v[0] - o[0])))

    def on(o, u, v):
        return min(o[0], u[0]) <= v[0] <= max(o[0], u[0]) and min(o[1], u[1]) <= v[1] <= max(o[1], u[1])
    o1, o2, o3, o4 = orient(a, b, c), orient(a, b, d), orient(c, d, a), orient(c, d, b)
    if o1 != o2 and o3 != o4 and o1 * o2 <= 0 and o3 * o4 <= 0:
        if o1 != 0 or o2 != 0:
            return True
    if o1 == 0 and on(a, b, c):
        return True
    if o2 == 0 and on(a, b, d):
        return True
    if o3 == 0 and on(c, d, a):
        return True
    if o4 == 0 and on(c, d, b):
        return True
    return False


@pytest.mark.parametrize("dist", ["uniform", "disc", "gaussian", "annulus", "shells"])
def test_invariants_on_synthetic_sets(dist):
    p, n = 48, 3000
    P = synth.points(dist, n, p, seed=11)
    L = oracle.reduce(P, p)
    lo, up = oracle.chain(L)
    s_cols = lo.shape[0]
    assert np.all(np.diff(lo[:, 0]) > 0) and np.all(np.diff(up[:, 0]) > 0)
    assert np.all(lo[:, 1] <= up[:, 1])
    poly = oracle.polyline(L)
    assert poly.shape[0] <= min(n, 2 * p)
    assert s_cols <= poly.shape[0] <= 2 * s_cols
    # Lemma 1: the polyline is simple (non-adjacent edges do not meet)
    e = [(poly[i], poly[i + 1]) for i in range(poly.shape[0] - 1)]
    for i in range(len(e)):
        for j in range(i + 2, len(e)):
            assert not _segments_cross(e[i][0], e[i][1], e[j][0], e[j][1]), (i, j)
    # every hull vertex survives the reduction, and the hull is unchanged
    H = oracle.hull_points(P)
    np.testing.assert_array_equal(oracle.hull_chain(L), H)
    survivors = {tuple(v) for v in poly}
    assert all(tuple(v) in survivors for v in H)
    # each surviving point is an input point and is the min or max of its column
    inputs = {tuple(v) for v in P}
    assert survivors <= inputs


def test_culling_polygon_start_array_against_point_in_polygon():
    """polygon_init marks exactly the lattice points strictly inside the
    polygon: checked against a direct strict point-in-convex-polygon test."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        p = int(rng.integers(3, 40))
        P = rng.integers(1, p + 1, size=(int(rng.integers(3, 12)), 2)).astype(np.int32)
        Q = oracle.hull_points(P)
        if Q.shape[0] < 3:
            continue
        Linit = oracle.polygon_init(Q, p)
        for x in range(1, p + 1):
            for y in range(1, p + 1):
                inside = True
                for i in range(Q.shape[0]):
                    a, b = Q[i], Q[(i + 1) % Q.shape[0]]
                    cr = (int(b[0]) - a[0]) * (y - int(a[1])) - (int(b[1]) - a[1]) * (x - int(a[0]))
                    if cr <= 0:
                        inside = False
                        break
                culled = Linit[x - 1, 0] <= y <= Linit[x - 1, 1]
                assert culled == inside, (p, Q.tolist(), x, y)


def test_culled_reduction_keeps_the_hull():
    rng = np.random.default_rng(6)
    for dist in ("uniform", "disc", "gaussian", "annulus"):
        p = 64
        P = synth.points(dist, 4000, p, seed=int(rng.integers(1 << 30)))
        H = oracle.hull_points(P)
        # culling polygon: hull of a few input points (extremes of a sample)
        S = P[rng.choice(P.shape[0], size=12, replace=False)]
        Q = oracle.hull_points(S)
        if Q.shape[0] < 3:
            continue
        Linit = oracle.polygon_init(Q, p)
        Lc = oracle.reduce_from(P, p, Linit)
        lo, up = oracle.chain_from(Lc, Linit)
        kept = np.concatenate([lo, up])
        np.testing.assert_array_equal(oracle.hull_points(kept), H)
