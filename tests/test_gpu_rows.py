"""Parity of the second scan along y (Section 2, Fig. 4: rx -> rxy) with the
oracle: R bit-exactly, and the hull of the rxy path."""
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


def check(P, p):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    L = oracle.reduce(P, p)
    Ro = oracle.reduce_rows(L)
    np.testing.assert_array_equal(host(ch.ch_reduce_rows(dev(L).reshape(-1, 2), p)), Ro)
    d = dev(P).reshape(-1, 2) if P.shape[0] else torch.empty((0, 2), dtype=torch.int32,
                                                             device="cuda")
    Lg = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    Rg = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    h, hc = ch.ch_convex_hull_rxy(d, p, L=Lg, R=Rg)
    np.testing.assert_array_equal(host(Lg), L)
    np.testing.assert_array_equal(host(Rg), Ro)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], oracle.hull_points(P))


@pytest.mark.parametrize("dist", ("uniform", "disc", "gaussian", "annulus", "shells"))
@pytest.mark.parametrize("p,n", [(1024, 100_000), (4096, 10_000_000), (29057, 500_000),
                                 (65536, 2_000_001), (200_000, 1_000_000)])
def test_rxy_path_matches_the_oracle(dist, p, n):
    check(synth.points(dist, n, p, seed=n % 977), p)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 33, 1025])
@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000])
def test_small_and_degenerate(p, n):
    rng = np.random.default_rng(p * 31 + n)
    check(rng.integers(1, p + 1, size=(n, 2)), p)


def test_lines_and_the_full_square():
    p = 300
    diag = np.stack([np.arange(1, p + 1)] * 2, 1)
    row = np.stack([np.arange(1, p + 1), np.full(p, 7)], 1)
    col = np.stack([np.full(p, 9), np.arange(1, p + 1)], 1)
    sq = np.stack(np.meshgrid(np.arange(1, 41), np.arange(1, 41)), -1).reshape(-1, 2)
    for P in (diag, row, col, sq):
        check(P, p)


def test_entry_that_is_not_from_algorithm_1_is_reported():
    p = 16
    L = np.tile(np.array([[p + 1, -1]], np.int32), (p, 1))
    L[3] = [5, 2]  # ly > hy: no input makes this
    R = ch.ch_reduce_rows(dev(L).reshape(-1, 2), p)
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    np.testing.assert_array_equal(host(R), np.tile([[p + 1, -1]], (p, 1)))
