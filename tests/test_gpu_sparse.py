"""Parity of the sparse-regime path (the tree of bit words of Section 4,
"Extraction using a tree structure") with the oracle: the chains, their
counts and the hull bit-exactly, and the persistent part of the workspace
back to all-zero after every call."""
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


def run_sparse(P, p, ws, offset=False):
    n = P.shape[0]
    if offset:  # an 8-byte but not 16-byte aligned point array
        buf = torch.empty((n + 1, 2), dtype=torch.int32, device="cuda")
        buf[1:] = dev(P).reshape(-1, 2) if n else buf[1:]
        d = buf[1:]
    else:
        d = dev(P).reshape(-1, 2) if n else torch.empty((0, 2), dtype=torch.int32, device="cuda")
    cap = max(1, min(p, n))
    lo = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    up = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    cnt = torch.empty(2, dtype=torch.int32, device="cuda")
    h, hc = ch.ch_convex_hull_sparse(d, p, ws, lower=lo, upper=up, counts=cnt)
    cnt = host(cnt)
    assert cnt[0] == cnt[1]
    s = int(cnt[0])
    return host(lo)[:s], host(up)[:s], host(h)[: int(host(hc)[0])]


def check(P, p, ws=None, offset=False):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    if ws is None:
        ws = ch.ch_sparse_workspace(P.shape[0], p)
    lo, up, h = run_sparse(P, p, ws, offset)
    lo_o, up_o = oracle.chain_points(P)
    np.testing.assert_array_equal(lo, lo_o)
    np.testing.assert_array_equal(up, up_o)
    np.testing.assert_array_equal(h, oracle.hull_points(P))
    _, persistent = ch.ch_sparse_workspace_size(P.shape[0], p)
    assert int(torch.count_nonzero(ws[:persistent]).item()) == 0
    return ws


@pytest.mark.parametrize("dist", ("uniform", "disc", "gaussian", "annulus", "shells"))
@pytest.mark.parametrize("p,n", [(1 << 20, 100_000), (1 << 24, 1 << 20), (1_000_003, 300_001),
                                 (4096, 1_000_000), (33, 5000), (1 << 30, 200_000)])
def test_sparse_path_matches_the_oracle(dist, p, n):
    check(synth.points(dist, n, p, seed=p % 1000 + n), p)


def test_workspace_is_reused_across_calls_and_sizes():
    p = 1 << 22
    ws = ch.ch_sparse_workspace(1 << 20, p)
    for i, n in enumerate((1 << 20, 5, 0, 777_777, 1, 1 << 20)):
        P = synth.points(("uniform", "gaussian", "disc")[i % 3], n, p, seed=i)
        check(P, p, ws, offset=bool(i & 1))


@pytest.mark.parametrize("p", [1, 2, 31, 32, 33, 1023, 1024, 1025, 32768, 32769])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 100])
def test_small_and_level_boundaries(p, n):
    rng = np.random.default_rng(p * 7 + n)
    P = rng.integers(1, p + 1, size=(n, 2)).astype(np.int32)
    check(P, p)
    check(P, p, offset=True)


def test_columns_at_the_ends_and_one_per_word():
    p = 1 << 25
    xs = np.concatenate([[1, 2, p - 1, p], np.arange(1, p + 1, 32 * 32 * 32 + 7)])
    P = np.stack([xs, (xs * 7919) % p + 1], 1).astype(np.int32)
    check(P, p)


def test_point_outside_is_reported_and_skipped():
    p = 1 << 20
    P = synth.points("uniform", 10_000, p, seed=1)
    bad = np.concatenate([P, [[p + 1, 5]]]).astype(np.int32)
    ws = ch.ch_sparse_workspace(bad.shape[0], p)
    run_sparse(bad, p, ws)
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    # the bad point was skipped: the workspace is clean and the next call exact
    check(P, p, ws)
