"""Parity of the culling proposal and of the culled path with the oracle.

Every integer result is compared bit-exactly: the sample histogram, the
extreme-point indices (given the GPU's float32 directions, both sides take
the argmax in float32 with the same two roundings), the polygon, the start
array Linit, L, both culled chains and the hull.  The hull must also equal
the plain hull for any network output, NaN included."""
import numpy as np
import pytest
import torch

import oracle
from oracle import learned as Lm
from paper_1505_00914_gb300 import ch, synth
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    w = Lm.init_params(seed) * scale
    d = Lm.unpack(w)
    d["b3"][:] = rng.normal(0, 1.0, Lm.K)
    return torch.from_numpy(w.astype(np.float32)).cuda()


def check_proposal(P, p, params=None):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    n = P.shape[0]
    out = ch.ch_cull_propose(dev(P).reshape(-1, 2), p, params=params)
    o = {k: host(v) for k, v in out.items()}
    idx = Lm.sample_index(n)
    np.testing.assert_array_equal(o["features"], Lm.histogram(P[idx], p))
    th0 = 2 * np.pi * np.arange(16) / 16
    np.testing.assert_allclose(o["dirs"][0][0], np.cos(th0), atol=2e-6)
    np.testing.assert_allclose(o["dirs"][0][1], np.sin(th0), atol=2e-6)
    if params is not None:
        y = o["net_out"].astype(np.float64)
        Y = Lm.forward(host(params).astype(np.float64), o["features"])[2][0]
        if np.all(np.isfinite(Y)):  # NaN weights: the directions fall back (checked below)
            assert np.max(np.abs(y - Y)) <= 2.0 ** -6 * (np.max(np.abs(Y)) + 1)
        th = Lm.directions(np.where(np.isnan(y), 0.0, y))
        np.testing.assert_allclose(o["dirs"][1][0], np.cos(th), atol=4e-6)
        np.testing.assert_allclose(o["dirs"][1][1], np.sin(th), atol=4e-6)
    else:
        assert o["chosen"][0] == -1
    if n == 0:
        assert np.all(o["extremes"] == -1) and o["poly_count"][0] == 0
        np.testing.assert_array_equal(o["Linit"], oracle.polygon_init(np.zeros((0, 2)), p))
        return o
    # both sides take the argmax with the GPU's float32 directions
    poly, sel, ext = Lm.choose_polygon(P, idx, o["dirs"], params is not None)
    for s_, e in enumerate(ext):
        np.testing.assert_array_equal(o["extremes"][s_], e)
    if params is not None:
        assert o["chosen"][0] == sel
    assert o["poly_count"][0] == poly.shape[0]
    np.testing.assert_array_equal(o["poly"][: poly.shape[0]], poly)
    np.testing.assert_array_equal(o["Linit"], oracle.polygon_init(poly, p))
    return o


def check_learned(P, p, params=None):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    H = oracle.hull(P, p)
    d = dev(P).reshape(-1, 2)
    L = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    Li = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    lo = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    up = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    cnt = torch.empty(2, dtype=torch.int32, device="cuda")
    stats = ch.cull_stats_tensor()
    h, hc = ch.ch_hull_learned(d, p, params=params, L=L, Linit=Li, lower=lo, upper=up, counts=cnt,
                               stats=stats)
    Li, L = host(Li), host(L)
    Lr = oracle.reduce_from(P, p, Li)
    np.testing.assert_array_equal(L, Lr)
    lo_o, up_o = oracle.chain_from(Lr, Li)
    cnt = host(cnt)
    assert cnt[0] == lo_o.shape[0] and cnt[1] == up_o.shape[0]
    np.testing.assert_array_equal(host(lo)[: cnt[0]], lo_o)
    np.testing.assert_array_equal(host(up)[: cnt[1]], up_o)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)
    # the start array is the proposal's, whose polygon is checked against the oracle
    o = check_proposal(P, p, params)
    np.testing.assert_array_equal(Li, o["Linit"])
    # the call's statistics: the polygon used, and the points strictly inside it
    st = ch.cull_stats(stats)
    k = int(o["poly_count"][0])
    assert st["poly_vertices"] == k and st["chosen"] == int(o["chosen"][0])
    assert st["culled"] == strictly_inside(P, o["poly"][:k])
    if P.shape[0]:
        lo_i, hi_i = Li[P[:, 0] - 1, 0], Li[P[:, 0] - 1, 1]
        assert st["culled"] == int(np.count_nonzero((lo_i <= P[:, 1]) & (P[:, 1] <= hi_i)))
    return H, Li


def strictly_inside(P, poly):
    """Points strictly inside the convex counter-clockwise polygon: strictly
    left of every edge (int64 orientation); none for fewer than 3 vertices."""
    k = poly.shape[0]
    if k < 3 or P.shape[0] == 0:
        return 0
    q = P.astype(np.int64)
    v = poly.astype(np.int64)
    inside = np.ones(P.shape[0], bool)
    for i in range(k):
        a, b = v[i], v[(i + 1) % k]
        inside &= (b[0] - a[0]) * (q[:, 1] - a[1]) - (b[1] - a[1]) * (q[:, 0] - a[0]) > 0
    return int(np.count_nonzero(inside))


DISTS = ("uniform", "disc", "gaussian", "annulus", "shells")


@pytest.mark.parametrize("dist", DISTS)
@pytest.mark.parametrize("p,n", [(1024, 100_000), (65536, 1_000_003), (4096, 262_144),
                                 (4096, 262_145)])
def test_proposal_matches_oracle(dist, p, n):
    P = synth.points(dist, n, p, seed=5)
    check_proposal(P, p)
    check_proposal(P, p, params=_params(1))


@pytest.mark.parametrize("dist", DISTS)
@pytest.mark.parametrize("p,n", [(1024, 100_000), (29056, 500_000), (29057, 500_000),
                                 (65536, 2_000_001), (116225, 300_000)])
def test_learned_path_matches_oracle(dist, p, n):
    P = synth.points(dist, n, p, seed=9)
    check_learned(P, p)
    check_learned(P, p, params=_params(2))


@pytest.mark.parametrize("dist", ("uniform", "disc", "annulus"))
def test_learned_path_long_chains(dist):
    """p = 262144: the global-L reduction form and 256 runs per chain, so the
    survivors take the second filter pass before the final CTA."""
    P = synth.points(dist, 2_000_000, 262_144, seed=12)
    check_learned(P, 262_144)
    check_learned(P, 262_144, params=_params(5))


@pytest.mark.parametrize("p", [1, 2, 3, 5, 31, 33, 1025])
@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000])
def test_learned_small_and_degenerate(p, n):
    rng = np.random.default_rng(p * 1000 + n)
    P = rng.integers(1, p + 1, size=(n, 2)).astype(np.int32)
    check_proposal(P, p)
    check_learned(P, p)
    check_learned(P, p, params=_params(3))


def test_learned_adversarial_shapes():
    p = 4096
    t = np.linspace(0, 2 * np.pi, 5000, endpoint=False)
    circle = np.stack([2048 + 2000 * np.cos(t), 2048 + 2000 * np.sin(t)], 1).round().astype(np.int32)
    line = np.stack([np.arange(1, p + 1), np.arange(1, p + 1)], 1).astype(np.int32)
    vertical = np.stack([np.full(3000, 77), np.arange(1, 3001)], 1).astype(np.int32)
    same = np.full((4000, 2), 1234, np.int32)
    square = np.array([[1, 1], [p, 1], [p, p], [1, p]] * 300, np.int32)
    rng = np.random.default_rng(4)
    tri = np.concatenate([square[:3], rng.integers(1, p + 1, (10000, 2))]).astype(np.int32)
    tri = tri[(tri[:, 1] <= tri[:, 0])]  # lower-right triangle, corners included
    for P in (circle, line, vertical, same, square, tri):
        check_proposal(P, p)
        check_learned(P, p)


def test_nan_and_huge_network_outputs_keep_the_hull_exact():
    p = 65536
    P = synth.points("disc", 500_000, p, seed=3)
    nan = torch.full((ch.CH_MLP_PARAMS,), float("nan"), device="cuda")
    H, Li = check_learned(P, p, params=nan)
    H2, _ = check_learned(P, p, params=_params(4, scale=1e3))
    np.testing.assert_array_equal(H, H2)
    # NaN falls back to the sector centres: the same start array as no network
    _, Li0 = check_learned(P, p)
    np.testing.assert_array_equal(Li, Li0)


@pytest.mark.slow
@pytest.mark.parametrize("dist", ("uniform", "disc", "gaussian", "annulus"))
def test_learned_full_size(dist):
    """The evaluation size of the learned form: n = 2^27 at p = 65536, in the
    configuration the benchmark times; hull, chain counts and Linit exact."""
    p, n = 65536, 1 << 27
    P = synth.points(dist, n, p, seed=17)
    H = oracle.hull(P, p)
    d = dev(P).reshape(-1, 2)
    del P
    Li = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    h, hc = ch.ch_hull_learned(d, p, Linit=Li)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)
    hp, hpc = ch.ch_convex_hull(d, p)
    np.testing.assert_array_equal(host(hp)[: int(host(hpc)[0])], H)
