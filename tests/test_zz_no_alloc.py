"""ch_chain_noalloc, the chain step for callers that cannot hand the library
device memory (it uses a fixed scratch array inside the library instead of a
caller workspace).  Each case runs it twice in a row on different inputs,
back to back on one stream, and checks the chains, counts and bit array M of
both calls against the CPU oracle (Lemma 1 scan and the bit array of
Section 4) and against ch_chain with a caller workspace.  The cases reach
the array's limit: p = CH_CHAIN_NOALLOC_MAX_P (L of 128 MB) and a p just
below it that is not a multiple of the 1024-column tile.  Collected last, so
that it also runs after every other GPU test in the same process."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


def _outputs(p):
    return (torch.full((p, 2), -5, dtype=torch.int32, device="cuda"),
            torch.full((p, 2), -5, dtype=torch.int32, device="cuda"),
            torch.full((2,), -5, dtype=torch.int32, device="cuda"),
            torch.full(((p + 31) // 32,), -5, dtype=torch.int32, device="cuda"))


def _check_pair(cases):
    Ls = [oracle.reduce(P, p) for p, P in cases]
    dLs = [dev(L) for L in Ls]
    outs = [_outputs(p) for p, _ in cases]
    for (p, _), dL, (lo, up, cnt, M) in zip(cases, dLs, outs):  # back to back, one stream
        ch.ch_chain_noalloc(dL, p, lo, up, cnt, M)
    for (p, _), L, dL, (lo, up, cnt, M) in zip(cases, Ls, dLs, outs):
        olo, oup = oracle.chain(L)
        s = olo.shape[0]
        c = host(cnt)
        assert c[0] == s and c[1] == s, (p, c, s)
        np.testing.assert_array_equal(host(lo)[:s], olo)
        np.testing.assert_array_equal(host(up)[:s], oup)
        np.testing.assert_array_equal(host(M).view(np.uint32), oracle.mask(L))
        rlo, rup, rcnt, rM = ch.ch_chain(dL, p, with_mask=True)
        np.testing.assert_array_equal(host(rcnt), c)
        np.testing.assert_array_equal(host(rlo)[:s], olo)
        np.testing.assert_array_equal(host(rup)[:s], oup)
        np.testing.assert_array_equal(host(rM), host(M))
    assert ch.ch_sync_status() == ch.CH_OK


def test_noalloc_chain_matches_oracle_twice_in_a_row():
    need_gpu()
    _check_pair([(65536, synth.points("disc", 300_000, 65536, seed=41)),
                 (5000, synth.points("gaussian", 40_000, 5000, seed=42))])


def test_noalloc_chain_at_its_size_limit():
    """p = CH_CHAIN_NOALLOC_MAX_P (every scratch word in use), then p just
    below it and not a multiple of 1024 (a ragged last tile)."""
    need_gpu()
    pmax = ch.CH_CHAIN_NOALLOC_MAX_P
    _check_pair([(pmax, synth.points("uniform", 1 << 21, pmax, seed=43)),
                 (pmax - 1000, synth.points("disc", 1 << 21, pmax - 1000, seed=44))])


def test_noalloc_chain_rejects_p_above_its_scratch():
    need_gpu()
    L = torch.empty((1, 2), dtype=torch.int32, device="cuda")
    lo, up, cnt, _ = _outputs(1)
    with pytest.raises(ch.ChError) as e:  # checked before any device access
        ch.ch_chain_noalloc(L, ch.CH_CHAIN_NOALLOC_MAX_P + 1, lo, up, cnt)
    assert e.value.code == ch.CH_ERR_CAPACITY
