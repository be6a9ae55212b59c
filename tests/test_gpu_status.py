"""The error status is kept per stream: a data error recorded by a call on
one stream is reported by ch_sync_status on that stream only, never to a
caller on another stream, and is cleared by that read."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

P = 65536


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield


def _inputs():
    good = synth.uniform(1 << 24, P, seed=71)
    bad = good.copy()
    bad[(1 << 23) + 5] = (P + 1, 7)  # one point outside [1,p]^2
    return good, bad


def _ws(n):
    return torch.empty(ch.ch_convex_hull_workspace_size(n, P), dtype=torch.uint8, device="cuda")


def test_two_streams_each_see_only_their_own_status():
    good, bad = _inputs()
    d_good, d_bad = dev(good), dev(bad)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    wa, wb = _ws(bad.shape[0]), _ws(good.shape[0])
    ha, hb = (torch.empty((2 * P, 2), dtype=torch.int32, device="cuda") for _ in range(2))
    ca, cb = (torch.empty(1, dtype=torch.int32, device="cuda") for _ in range(2))
    torch.cuda.synchronize()
    H = oracle.hull_chain(oracle.reduce(good, P))
    for order in ("good_first", "bad_first"):
        for _ in range(3):
            # both calls in flight at once, on their own streams
            ch.ch_convex_hull(d_bad, P, hull=ha, hull_count=ca, workspace=wa, stream=sa)
            ch.ch_convex_hull(d_good, P, hull=hb, hull_count=cb, workspace=wb, stream=sb)
            if order == "good_first":  # read b while a may still be running
                assert ch.ch_sync_status(sb) == ch.CH_OK
                assert ch.ch_sync_status(sa) == ch.CH_ERR_RANGE
            else:
                assert ch.ch_sync_status(sa) == ch.CH_ERR_RANGE
                assert ch.ch_sync_status(sb) == ch.CH_OK
            assert ch.ch_sync_status(sa) == ch.CH_OK  # cleared by the read
            assert ch.ch_sync_status() == ch.CH_OK  # the current stream saw nothing
            k = int(host(cb)[0])
            np.testing.assert_array_equal(host(hb)[:k], H)


def test_status_of_a_captured_call_goes_to_its_capture_stream():
    good, bad = _inputs()
    d_bad = dev(bad[: 1 << 20])
    sc = torch.cuda.Stream()
    ws = _ws(1 << 20)
    h = torch.empty((2 * P, 2), dtype=torch.int32, device="cuda")
    c = torch.empty(1, dtype=torch.int32, device="cuda")
    sc.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(sc):
        ch.ch_convex_hull(d_bad, P, hull=h, hull_count=c, workspace=ws, stream=sc)  # set-up
    assert ch.ch_sync_status(sc) == ch.CH_OK  # the point outside is beyond the first 2^20
    d_bad2 = dev(bad[(1 << 23) - (1 << 19): (1 << 23) + (1 << 19)])
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=sc):
        ch.ch_convex_hull(d_bad2, P, hull=h, hull_count=c, workspace=ws, stream=sc)
    g.replay()
    torch.cuda.synchronize()
    assert ch.ch_sync_status() == ch.CH_OK
    assert ch.ch_sync_status(sc) == ch.CH_ERR_RANGE
    assert ch.ch_sync_status(sc) == ch.CH_OK


def test_clear_status_is_per_stream():
    _, bad = _inputs()
    d_bad = dev(bad[(1 << 23):(1 << 23) + 1024])
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ws_a, ws_b = _ws(1024), _ws(1024)
    ch.ch_convex_hull(d_bad, P, workspace=ws_a, stream=sa)
    ch.ch_convex_hull(d_bad, P, workspace=ws_b, stream=sb)
    ch.ch_clear_status(sa)
    assert ch.ch_sync_status(sa) == ch.CH_OK
    assert ch.ch_sync_status(sb) == ch.CH_ERR_RANGE
