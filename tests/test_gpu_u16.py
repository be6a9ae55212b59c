"""Parity of the packed 16-bit point format (int16x2 loads: one 32-bit word
(x - 1) | (y - 1) << 16 per point) with the oracle: L and the hull
bit-exactly, every alignment of the array start, ragged tails, the forms of
the reduction, and the full size of the plain path.  The packing is done
here with numpy; the oracle sees the plain int32 points."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from gpu_util import host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def packed(P, offset=0):
    """Device int32 view of the packed points, starting `offset` words after
    a 16-byte aligned allocation."""
    P = np.asarray(P, dtype=np.int64).reshape(-1, 2)
    w = (((P[:, 1] - 1) << 16) | (P[:, 0] - 1)).astype(np.uint32).view(np.int32)
    buf = torch.zeros(w.shape[0] + offset + 4, dtype=torch.int32, device="cuda")
    assert buf.data_ptr() % 16 == 0
    d = buf[offset:offset + w.shape[0]]
    d.copy_(torch.from_numpy(w))
    return d


def check(P, p, offset=0):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    d = packed(P, offset)
    Lo = oracle.reduce(P, p)
    np.testing.assert_array_equal(host(ch.ch_reduce_u16(d, p)), Lo)
    L = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    h, hc = ch.ch_convex_hull_u16(d, p, L=L)
    np.testing.assert_array_equal(host(L), Lo)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], oracle.hull_chain(Lo))


@pytest.mark.parametrize("p", [1, 2, 31, 1024, 1025, 4096, 20480, 20481, 29056, 29057, 65535,
                               65536])
@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_every_alignment_and_tail(p, offset):
    rng = np.random.default_rng(p * 4 + offset)
    for n in (0, 1, 2, 3, 5, 7, 1001, 50_003):
        check(rng.integers(1, p + 1, size=(n, 2)), p, offset)


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
def test_distributions(dist):
    for p, n in ((1024, 100_000), (4096, 10**6), (65536, 2_000_001)):
        check(synth.points(dist, n, p, seed=p + 7), p)


def test_point_outside_and_side_limit():
    p = 1000
    P = np.asarray([[1, 1], [1001, 5], [3, 3]], np.int32)
    ch.ch_reduce_u16(packed(P), p)
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    with pytest.raises(ch.ChError):
        ch.ch_convex_hull_u16(packed(np.asarray([[1, 1]])), 65537)


@pytest.mark.slow
@pytest.mark.parametrize("dist", ("uniform", "disc", "gaussian"))
def test_full_size(dist):
    """n = 2^26 at p = 65536, the plain path's timed size, in this format."""
    p, n = 65536, 1 << 26
    P = synth.points(dist, n, p, seed=23)
    H = oracle.hull(P, p)
    d = packed(P)
    del P
    h, hc = ch.ch_convex_hull_u16(d, p)
    np.testing.assert_array_equal(host(h)[: int(host(hc)[0])], H)
