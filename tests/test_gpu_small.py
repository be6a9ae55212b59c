"""The single-launch path of ch_convex_hull for small problems (p <= 16384,
up to 8192 points per CTA, the partial rows of all CTAs small enough for
one CTA to merge): one kernel folds, merges and finishes the set.  Every
hull and L against the oracle (Algorithm 1, then the hull of its chains),
including empty, degenerate and misaligned inputs, range errors, repeated
calls on one stream and concurrent calls on several."""
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


def small(n, p):
    form, kernels = ch.ch_plan_info(n, p)
    return form == 3 and kernels == 1


def check(P, p, d=None):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    Lo = oracle.reduce(P, p)
    H = oracle.hull_chain(Lo)
    d = dev(P) if d is None else d
    L = torch.full((p, 2), -3, dtype=torch.int32, device="cuda")
    h, hc = ch.ch_convex_hull(d, p, L=L)
    np.testing.assert_array_equal(host(L), Lo)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)
    h2, hc2 = ch.ch_convex_hull(d, p)  # without L
    np.testing.assert_array_equal(host(h2)[: int(host(hc2)[0])], H)
    return H


def test_plan_reports_one_launch():
    assert small(100_000, 1024)  # the small configuration: p = 1024, n = 10^5
    assert small(0, 1) and small(32_768, 16384) and small(524_288, 1024)
    assert not small(32_769, 16384)  # five CTAs' rows of 16384 words: too many to merge
    assert not small(524_289, 1024)
    assert not small(100_000, 16385)
    assert not small(1 << 26, 65536)


@pytest.mark.parametrize("p", [1, 2, 5, 31, 33, 256, 1000, 1024, 1025, 4096, 16384])
@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 8191, 8192, 8193, 32_768, 100_000, 524_288])
def test_small_path_matches_oracle(p, n):
    if not small(n, p):
        pytest.skip("not a single-launch case")
    rng = np.random.default_rng(p * 7919 + n)
    P = rng.integers(1, p + 1, size=(n, 2)).astype(np.int32)
    check(P, p)


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
def test_small_config_distributions(dist):
    """The small configuration's size (p = 1024, n = 10^5) in every distribution."""
    check(synth.points(dist, 100_000, 1024, seed=3), 1024)


def test_small_adversarial_shapes():
    p = 4096
    t = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    circle = np.stack([2048 + 2000 * np.cos(t), 2048 + 2000 * np.sin(t)], 1).round().astype(np.int32)
    line = np.stack([np.arange(1, p + 1), np.arange(1, p + 1)], 1).astype(np.int32)
    vertical = np.stack([np.full(3000, 77), np.arange(1, 3001)], 1).astype(np.int32)
    same = np.full((40000, 2), 1234, np.int32)
    for P in (circle, line, vertical, same):
        check(P, p)
    # every column of a 16384-wide set on its hull's boundary: survivors beyond
    # the shared-memory capacity of the finishing step
    q = 16384
    x = np.arange(1, q + 1)
    para = np.stack([x, 1 + ((x - 8192) ** 2) // 16384], 1).astype(np.int32)
    check(np.concatenate([para, np.stack([x, q - para[:, 1] + 1], 1)]), q)


def test_small_misaligned_points():
    p = 1024
    P = synth.uniform(100_001, p, seed=8)
    big = dev(np.concatenate([np.zeros((1, 2), np.int32), P]))
    check(P, p, d=big[1:])  # 8 bytes past a 16-byte boundary


def test_small_range_error_and_recovery():
    p = 1024
    P = synth.uniform(100_000, p, seed=9)
    bad = P.copy()
    bad[77_777] = (p + 1, 3)
    ch.ch_convex_hull(dev(bad), p)
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    check(P, p)  # the next call is unaffected


def test_small_repeated_and_concurrent_calls():
    """Calls back to back on one stream (the ticket returns to zero each
    time) and on four streams at once (each stream has its own ticket)."""
    p = 1024
    sets = [synth.points(d, 100_000 + k, p, seed=k) for k, d in enumerate(synth.DISTRIBUTIONS)]
    H = [oracle.hull_chain(oracle.reduce(P, p)) for P in sets]
    ds = [dev(P) for P in sets]
    streams = [torch.cuda.Stream() for _ in sets]
    hulls = [torch.empty((2 * p, 2), dtype=torch.int32, device="cuda") for _ in sets]
    cnts = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in sets]
    wss = [torch.empty(ch.ch_convex_hull_workspace_size(P.shape[0], p), dtype=torch.uint8,
                       device="cuda") for P in sets]
    torch.cuda.synchronize()
    for _ in range(5):
        for d, h, c, w, st in zip(ds, hulls, cnts, wss, streams):
            ch.ch_convex_hull(d, p, hull=h, hull_count=c, workspace=w, stream=st)
            ch.ch_convex_hull(d, p, hull=h, hull_count=c, workspace=w, stream=st)
        for k, st in enumerate(streams):
            assert ch.ch_sync_status(st) == ch.CH_OK
            np.testing.assert_array_equal(host(hulls[k])[: int(host(cnts[k])[0])], H[k])


def test_small_path_in_a_cuda_graph():
    p = 1024
    P = synth.disc(100_000, p, seed=10)
    H = oracle.hull_chain(oracle.reduce(P, p))
    d = dev(P)
    h = torch.empty((2 * p, 2), dtype=torch.int32, device="cuda")
    c = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(ch.ch_convex_hull_workspace_size(P.shape[0], p), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ch.ch_convex_hull(d, p, hull=h, hull_count=c, workspace=ws, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ch.ch_convex_hull(d, p, hull=h, hull_count=c, workspace=ws, stream=s)
    for _ in range(3):
        h.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(h)[: int(host(c)[0])], H)
    assert ch.ch_sync_status(s) == ch.CH_OK
