"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work: every comparison is bit-exact (L, chains, counts, mask, the hull
vertex list and its order)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from _golden import read
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def gpu_all(P, p):
    """ch_reduce, ch_chain, ch_hull one by one (numpy in/out)."""
    L = ch.ch_reduce(dev(P).reshape(-1, 2), p)
    lo, up, cnt, M = ch.ch_chain(L, p, with_mask=True)
    h, hc = ch.ch_hull(lo, up, cnt, p)
    L, lo, up, cnt, M, h, hc = map(host, (L, lo, up, cnt, M, h, hc))
    s = int(cnt[0])
    return L, lo[:s], up[:s], cnt, M.view(np.uint32), h[: int(hc[0])]


def check_against_oracle(P, p, fused=True):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    Lo = oracle.reduce(P, p)
    lo_o, up_o = oracle.chain(Lo)
    H = oracle.hull_chain(Lo)
    L, lo, up, cnt, M, h = gpu_all(P, p)
    np.testing.assert_array_equal(L, Lo)
    assert cnt[0] == cnt[1] == lo_o.shape[0]
    np.testing.assert_array_equal(lo, lo_o)
    np.testing.assert_array_equal(up, up_o)
    np.testing.assert_array_equal(M, oracle.mask(Lo))
    np.testing.assert_array_equal(h, H)
    if fused:
        Lf = torch.empty((p, 2), dtype=torch.int32, device="cuda")
        hf, hcf = ch.ch_convex_hull(dev(P).reshape(-1, 2), p, L=Lf)
        np.testing.assert_array_equal(host(Lf), Lo)
        np.testing.assert_array_equal(host(hf)[: int(host(hcf)[0])], H)
    return H


def test_fig1_worked_example():
    keys, L = read("fig1_L.txt")
    _, H = read("fig1_hull.txt")
    P = np.asarray([(x, y) for x, (a, b) in enumerate(L, 1) for y in range(a, b + 1)], np.int32)
    Lg, lo, up, cnt, M, h = gpu_all(np.random.default_rng(0).permutation(P), keys["p"])
    np.testing.assert_array_equal(Lg, L)
    np.testing.assert_array_equal(h, H)
    assert int(M[0]) == 0b11111


def test_fig1_gapped_mask_word():
    keys, L = read("fig1_gapped_L.txt")
    P = np.asarray([(x, y) for x, (a, b) in enumerate(L, 1) if a <= b for y in range(a, b + 1)],
                   np.int32)
    Lg, lo, up, cnt, M, h = gpu_all(P, keys["p"])
    np.testing.assert_array_equal(Lg, L)
    assert int(M[0]) == keys["mask"]


def test_block_bit_index_on_gpu():
    keys, _ = read("block_index.txt")
    p = 1 << 17
    _, _, _, _, M, _ = gpu_all(np.asarray([[keys["i"], 5]], np.int32), p)
    assert list(np.flatnonzero(M)) == [keys["block"]]
    assert int(M[keys["block"]]) == 1 << keys["bit"]


@pytest.mark.parametrize("p", [1, 2, 5, 31, 32, 33, 1000, 1024, 1025, 4096, 4097, 16384, 20480,
                               20481, 29056, 29057, 65535, 65536, 116224, 116225])
def test_tile_boundaries_and_layouts(p):
    rng = np.random.default_rng(p)
    for n in (0, 1, 2, 3, 1001, 50_000):
        P = rng.integers(1, p + 1, size=(n, 2)).astype(np.int32)
        check_against_oracle(P, p, fused=(n % 2 == 1))


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
def test_distributions_small(dist):
    for p in (64, 1024, 4096):
        check_against_oracle(synth.points(dist, 200_000, p, seed=7), p)


def test_misaligned_point_array():
    p = 4096
    P = synth.uniform(100_001, p, seed=3)
    big = dev(P)
    for off in (1, 3):
        sub = big[off:]
        assert sub.data_ptr() % 16 == 8
        L = host(ch.ch_reduce(sub, p))
        np.testing.assert_array_equal(L, oracle.reduce(P[off:], p))


def test_config_small_uniform_exact():
    """p=1024, n=100,000 uniform on [1,1024]^2 from seed 0."""
    P = synth.uniform(100_000, 1024, seed=0)
    H = check_against_oracle(P, 1024)
    np.testing.assert_array_equal(H, oracle.hull_points(P))


def _convex_arcs(p, arc, rng):
    """Sawtooth of strictly convex arcs: many local hull vertices."""
    pts = []
    x = 1
    while x + arc <= p:
        base = int(rng.integers(1, max(2, p - arc * arc // 2)))
        for k in range(arc):
            pts.append((x + k, base + k * (k - 1) // 2 % p))
            pts.append((x + k, min(p, base + arc * arc)))
        x += arc
    P = np.asarray(pts, np.int32)
    P[:, 1] = np.clip(P[:, 1], 1, p)
    return P


def test_adversarial_hulls():
    rng = np.random.default_rng(9)
    p = 65536
    # parabola: every column is a lower-hull vertex
    xs = np.arange(1, 361)
    P = np.stack([xs * 100, 1 + (xs - 1) * (xs - 2) // 2], 1).astype(np.int32)
    check_against_oracle(P, p)
    # convex arcs of 32 (one thread segment each) and of 45 (straddling)
    for arc in (8, 32, 45):
        check_against_oracle(_convex_arcs(4096, arc, rng), 4096)
    # lattice circle: many hull vertices at full p
    t = np.linspace(0, 2 * np.pi, 200_000, endpoint=False)
    C = np.stack([32768.5 + 32767 * np.cos(t), 32768.5 + 32767 * np.sin(t)], 1)
    check_against_oracle(np.clip(np.rint(C), 1, p).astype(np.int32), p)
    # heavy collinearity: points on a few lattice lines
    for _ in range(20):
        q = int(rng.integers(3, 300))
        lines = []
        for _ in range(int(rng.integers(1, 4))):
            dx, dy = rng.integers(-3, 4, size=2)
            x0, y0 = rng.integers(1, q + 1, size=2)
            tt = rng.integers(-q, q + 1, size=500)
            lines.append(np.stack([x0 + tt * dx, y0 + tt * dy], 1))
        Q = np.concatenate(lines)
        Q = Q[(Q.min(1) >= 1) & (Q.max(1) <= q)].astype(np.int32)
        check_against_oracle(Q, q)


def test_degenerate_inputs():
    for P, p in (([[3, 4]] * 9, 7), ([[2, 5], [2, 1], [2, 3]], 7), ([[k, k] for k in range(1, 8)], 7),
                 ([[k, 3] for k in (5, 1, 4)], 7), ([[k, 8 - k] for k in range(1, 8)], 7),
                 ([[1, 1]], 1), ([[1, 1], [1, 1]], 1)):
        check_against_oracle(np.asarray(P, np.int32), p)


def test_out_of_range_points_set_status():
    p = 100
    for bad in ([0, 5], [5, 0], [101, 5], [5, 101], [-7, 3]):
        P = np.asarray([[1, 1], bad, [3, 4]] * 1000, np.int32)
        ch.ch_reduce(dev(P), p)
        assert ch.ch_sync_status() == ch.CH_ERR_RANGE
        ch.ch_convex_hull(dev(P), p)
        assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    P = np.asarray([[1, 1], [70001, 5]], np.int32)
    ch.ch_reduce(dev(P), 70000)
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    assert ch.ch_sync_status() == ch.CH_OK  # the status word clears on read


def test_reduction_forms_switch_at_their_limits():
    """The private form up to 160 KB of shared memory (p = 20480), the
    filtered form up to the opt-in limit (p = 116224), the global form
    beyond (form numbers of ch_plan_info)."""
    n = 1 << 22
    assert ch.ch_plan_info(n, 20480)[0] == 0
    assert ch.ch_plan_info(n, 20481)[0] == 1
    assert ch.ch_plan_info(n, 116224)[0] == 1
    assert ch.ch_plan_info(n, 116225)[0] == 2


def test_argument_errors():
    P = dev(np.ones((10, 2), np.int32))
    with pytest.raises(ch.ChError) as e:
        ch.ch_reduce(P, 0)
    assert e.value.code == ch.CH_ERR_ARG
    with pytest.raises(ch.ChError) as e:
        ch.ch_reduce(P, (1 << 30) + 1)
    assert e.value.code == ch.CH_ERR_ARG
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ch.ChError) as e:
        ch.ch_convex_hull(P, 4096, workspace=small)
    assert e.value.code == ch.CH_ERR_WORKSPACE
    # a workspace that does not start on a 256-byte boundary
    for fn, size in ((ch.ch_convex_hull, ch.ch_convex_hull_workspace_size(10, 4096)),
                     (ch.ch_reduce, ch.ch_reduce_workspace_size(10, 70000))):
        buf = torch.empty(size + 512, dtype=torch.uint8, device="cuda")
        for off in (8, 16, 128):
            with pytest.raises(ch.ChError) as e:
                fn(P, 4096 if fn is ch.ch_convex_hull else 70000, workspace=buf[off:])
            assert e.value.code == ch.CH_ERR_ARG
        fn(P, 4096 if fn is ch.ch_convex_hull else 70000, workspace=buf[256:])


def test_host_entry_point_matches():
    """Page-locked and pageable host points; a page-locked array starting 8
    bytes into its buffer (not 16-byte aligned) and short lengths."""
    p = 4096
    P = synth.shells(300_001, p, seed=2)
    nbytes = ch.ch_convex_hull_host_workspace_size(P.shape[0], p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    hp = torch.from_numpy(P).pin_memory()
    np.testing.assert_array_equal(ch.ch_convex_hull_host(hp, p, ws).numpy(), oracle.hull_points(P))
    pageable = torch.from_numpy(P.copy())
    np.testing.assert_array_equal(ch.ch_convex_hull_host(pageable, p, ws).numpy(),
                                  oracle.hull_points(P))
    big = torch.from_numpy(np.concatenate([P[:1], P])).pin_memory()
    sub = big[1:]
    assert sub.data_ptr() % 16 == 8 and sub.is_contiguous()
    np.testing.assert_array_equal(ch.ch_convex_hull_host(sub, p, ws).numpy(), oracle.hull_points(P))
    for n in (0, 1, 2, 3, 1001):
        Q = torch.from_numpy(P[:n].copy()).pin_memory()
        np.testing.assert_array_equal(ch.ch_convex_hull_host(Q, p, ws).numpy(),
                                      oracle.hull_points(P[:n]))


@pytest.mark.parametrize("dist", ["uniform", "disc", "gaussian"])
def test_plain_at_scale_full_size(dist):
    """p=65536, n=2^26: the launch configuration the benchmark times."""
    p, n = 65536, 1 << 26
    P = synth.points(dist, n, p, seed=1)
    Lo = oracle.reduce(P, p)
    H = oracle.hull_chain(Lo)
    d = dev(P)
    L = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    lo = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    up = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    cnt = torch.empty(2, dtype=torch.int32, device="cuda")
    h, hc = ch.ch_convex_hull(d, p, L=L, lower=lo, upper=up, counts=cnt)
    np.testing.assert_array_equal(host(L), Lo)
    lo_o, up_o = oracle.chain(Lo)
    s = int(host(cnt)[0])
    assert s == lo_o.shape[0]
    np.testing.assert_array_equal(host(lo)[:s], lo_o)
    np.testing.assert_array_equal(host(up)[:s], up_o)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)


@pytest.mark.parametrize("p", [1, 2, 33, 1023, 1024, 1025, 4096, 9999, 16384, 16385])
def test_fused_path_with_and_without_chain_outputs(p):
    """ch_convex_hull with chain outputs (the chain step ranks and writes both
    chains) and without (it writes only the pre-filter's candidates), on
    sides around the tile size and the 16384 limit of the 32-bit orientation
    tests: a uniform set, a disc and a circle (a hull vertex in most columns),
    each compared with the oracle."""
    rng = np.random.default_rng(p)
    t = np.linspace(0, 2 * np.pi, 50_000, endpoint=False)
    r = (p - 1) / 2
    circle = np.stack([np.rint(1 + r + r * np.cos(t)), np.rint(1 + r + r * np.sin(t))], 1)
    sets = [rng.integers(1, p + 1, size=(300_001, 2)), synth.points("disc", 200_000, p, seed=p),
            circle]
    for P in sets:
        P = np.ascontiguousarray(np.clip(P, 1, p), dtype=np.int32)
        Lo = oracle.reduce(P, p)
        H = oracle.hull_chain(Lo)
        lo_o, up_o = oracle.chain(Lo)
        d = dev(P)
        h0, hc0 = ch.ch_convex_hull(d, p)
        np.testing.assert_array_equal(host(h0)[: int(host(hc0)[0])], H)
        lo = torch.empty((p, 2), dtype=torch.int32, device="cuda")
        up = torch.empty((p, 2), dtype=torch.int32, device="cuda")
        cnt = torch.empty(2, dtype=torch.int32, device="cuda")
        h1, hc1 = ch.ch_convex_hull(d, p, lower=lo, upper=up, counts=cnt)
        np.testing.assert_array_equal(host(h1)[: int(host(hc1)[0])], H)
        s = int(host(cnt)[0])
        assert s == int(host(cnt)[1]) == lo_o.shape[0]
        np.testing.assert_array_equal(host(lo)[:s], lo_o)
        np.testing.assert_array_equal(host(up)[:s], up_o)


def test_projected_shells_full_size():
    """p=4096, n=10^7 projected shells and cylinders."""
    p = 4096
    P = synth.shells(10_000_000, p, seed=3)
    check_against_oracle(P, p)


@pytest.mark.parametrize("p", [131071, 131072, 262145, 1 << 20, 1 << 22])
def test_long_chains_second_filter_pass(p):
    """From 128 runs of 1024 columns per chain on, the survivors of the
    in-tile filter are packed and filtered again before the final CTA: sparse
    and dense uniform sets, a disc, and a circle whose every column holds a
    hull vertex region."""
    rng = np.random.default_rng(p)
    sets = [rng.integers(1, p + 1, size=(200_000, 2)),
            synth.points("uniform", 3_000_000, p, seed=1),
            synth.points("disc", 2_000_000, p, seed=2)]
    t = np.linspace(0, 2 * np.pi, 400_000, endpoint=False)
    r = (p - 3) / 2
    circ = np.stack([(p + 1) / 2 + r * np.cos(t), (p + 1) / 2 + r * np.sin(t)], 1)
    sets.append(np.clip(np.rint(circ), 1, p))
    for P in sets:
        P = np.ascontiguousarray(P, dtype=np.int32)
        H = oracle.hull_points(P)
        h, hc = ch.ch_convex_hull(dev(P).reshape(-1, 2), p)
        np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)
        lo, up, cnt = ch.ch_chain(ch.ch_reduce(dev(P).reshape(-1, 2), p), p)
        h2, hc2 = ch.ch_hull(lo, up, cnt, p)
        np.testing.assert_array_equal(host(h2)[: int(host(hc2)[0])], H)
