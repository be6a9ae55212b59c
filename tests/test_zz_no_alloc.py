"""ch_chain_noalloc (fixed library scratch, no workspace) against ch_chain
(caller workspace): two calls in a row on different inputs must give the
same chains, counts and bit array as the workspace form.  Collected last so
that it also runs after every other GPU test in the same process."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


def _outputs(p):
    return (torch.empty((p, 2), dtype=torch.int32, device="cuda"),
            torch.empty((p, 2), dtype=torch.int32, device="cuda"),
            torch.empty(2, dtype=torch.int32, device="cuda"),
            torch.empty(((p + 31) // 32,), dtype=torch.int32, device="cuda"))


def test_noalloc_chain_matches_workspace_form_twice_in_a_row():
    need_gpu()
    cases = [(65536, synth.points("disc", 300_000, 65536, seed=41)),
             (5000, synth.points("gaussian", 40_000, 5000, seed=42))]
    Ls = [dev(oracle.reduce(P, p)) for p, P in cases]
    outs = [_outputs(p) for p, _ in cases]
    for (p, _), L, (lo, up, cnt, M) in zip(cases, Ls, outs):  # back to back, one stream
        ch.ch_chain_noalloc(L, p, lo, up, cnt, M)
    for (p, _), L, (lo, up, cnt, M) in zip(cases, Ls, outs):
        rlo, rup, rcnt, rM = ch.ch_chain(L, p, with_mask=True)
        c = host(cnt)
        np.testing.assert_array_equal(c, host(rcnt))
        s = int(c[0])
        np.testing.assert_array_equal(host(lo)[:s], host(rlo)[:s])
        np.testing.assert_array_equal(host(up)[:s], host(rup)[:s])
        np.testing.assert_array_equal(host(M), host(rM))
    assert ch.ch_sync_status() == ch.CH_OK


def test_noalloc_chain_rejects_p_above_its_scratch():
    need_gpu()
    L = torch.empty((1, 2), dtype=torch.int32, device="cuda")
    lo, up, cnt, _ = _outputs(1)
    with pytest.raises(ch.ChError) as e:  # checked before any device access
        ch.ch_chain_noalloc(L, ch.CH_CHAIN_NOALLOC_MAX_P + 1, lo, up, cnt)
    assert e.value.code == ch.CH_ERR_CAPACITY
