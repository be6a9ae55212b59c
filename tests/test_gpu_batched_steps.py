"""Parity of the batched reduce and chain steps (ch_reduce_batched,
ch_chain_batched) with the CPU oracle, set by set: each set's L bit-exactly
against Algorithm 1 (Section 2.1), and its chains and counts against the
Lemma 1 scan of that L."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import ch, synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def reduce_batch(pts, offsets, ps, chunk_mult=64):
    d_pts = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 2)).cuda()
    d_off = torch.from_numpy(np.asarray(offsets, np.int64)).cuda()
    d_ps = torch.from_numpy(np.asarray(ps, np.int32)).cuda()
    loff = ch.L_offsets_of(ps)
    d_loff = torch.from_numpy(loff).cuda()
    L = torch.full((int(loff[-1]), 2), -9, dtype=torch.int32, device="cuda")
    nws = ch.ch_batched_workspace_size(offsets, ps, chunk_mult)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    ch.ch_batched_prepare(offsets, ps, ws, chunk_mult)
    ch.ch_reduce_batched(d_pts, d_off, d_ps, L, d_loff, ws)
    return L, d_loff, d_ps, loff


def chain_batch(L, d_loff, d_ps, total):
    lo = torch.full((total, 2), -9, dtype=torch.int32, device="cuda")
    up = torch.full((total, 2), -9, dtype=torch.int32, device="cuda")
    cnt = torch.full((d_ps.shape[0], 2), -7, dtype=torch.int32, device="cuda")
    ch.ch_chain_batched(L, d_loff, d_ps, lo, up, cnt)
    torch.cuda.synchronize()
    return lo.cpu().numpy(), up.cpu().numpy(), cnt.cpu().numpy()


def check(pts, offsets, ps, chunk_mult=64):
    L, d_loff, d_ps, loff = reduce_batch(pts, offsets, ps, chunk_mult)
    lo, up, cnt = chain_batch(L, d_loff, d_ps, int(loff[-1]))
    L = L.cpu().numpy()
    for s in range(len(ps)):
        p = int(ps[s])
        Lo = oracle.reduce(pts[offsets[s]:offsets[s + 1]], p)
        np.testing.assert_array_equal(L[loff[s]:loff[s] + p], Lo, err_msg=f"L of set {s}")
        clo, cup = oracle.chain(Lo)
        k = clo.shape[0]
        assert tuple(cnt[s]) == (k, k), (s, cnt[s], k)
        np.testing.assert_array_equal(lo[loff[s]:loff[s] + k], clo, err_msg=f"lower chain of set {s}")
        np.testing.assert_array_equal(up[loff[s]:loff[s] + k], cup, err_msg=f"upper chain of set {s}")


def test_mixed_batch_matches_the_oracle():
    rng = np.random.default_rng(14)
    B = 240
    ps = rng.choice([1, 2, 5, 31, 256, 1000, 1024, 1025, 4096, 16384], size=B).astype(np.int32)
    ns = np.rint(10 ** rng.uniform(0, 5.2, size=B)).astype(np.int64)
    ns[rng.random(B) < 0.05] = 0
    dists = ["uniform", "disc", "gaussian", "annulus"]
    parts = [synth.points(dists[i % 4], int(ns[i]), int(ps[i]), seed=200 + i) for i in range(B)]
    offsets = np.zeros(B + 1, np.int64)
    np.cumsum(ns, out=offsets[1:])
    check(np.concatenate(parts), offsets, ps)


def test_multi_chunk_sets_and_misaligned_starts():
    """chunk_mult = 1 cuts every set of more than 65536 points into chunks
    merged through the packed partial rows; odd set lengths make most sets
    start 8 bytes into a 16-byte vector."""
    ps = np.asarray([256, 16384, 7, 4096, 1, 300], np.int32)
    ns = np.asarray([400_001, 150_003, 3, 200_000, 5, 131_073], np.int64)
    parts = [synth.points(["uniform", "disc", "gaussian", "annulus"][i % 4], int(ns[i]), int(ps[i]),
                          seed=70 + i) for i in range(len(ps))]
    offsets = np.zeros(len(ps) + 1, np.int64)
    np.cumsum(ns, out=offsets[1:])
    pts = np.concatenate(parts)
    for cm in (1, 64):
        check(pts, offsets, ps, chunk_mult=cm)


def test_chain_batched_takes_any_side():
    """The chain step reads L only, so sides above the batch limit work."""
    ps = np.asarray([20_000, 1, 70_001, 3, 65_536], np.int32)
    Ls = [oracle.reduce(synth.points(d, n, int(p), seed=9 + i), int(p))
          for i, (d, n, p) in enumerate(zip(["uniform", "disc", "gaussian", "annulus", "uniform"],
                                            [30_000, 0, 500_000, 2, 1000], ps))]
    loff = ch.L_offsets_of(ps)
    L = torch.from_numpy(np.concatenate(Ls)).cuda()
    lo, up, cnt = chain_batch(L, torch.from_numpy(loff).cuda(), torch.from_numpy(ps).cuda(),
                              int(loff[-1]))
    for s, Lo in enumerate(Ls):
        clo, cup = oracle.chain(Lo)
        k = clo.shape[0]
        assert tuple(cnt[s]) == (k, k)
        np.testing.assert_array_equal(lo[loff[s]:loff[s] + k], clo)
        np.testing.assert_array_equal(up[loff[s]:loff[s] + k], cup)


def test_range_error_and_arguments():
    pts = np.asarray([[1, 1], [9, 2], [3, 3]], np.int32)
    L, _, _, _ = reduce_batch(pts, np.asarray([0, 3]), np.asarray([8], np.int32))
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    # the bad point was skipped: the others are in L
    Lh = L.cpu().numpy()
    assert tuple(Lh[0]) == (1, 1) and tuple(Lh[2]) == (3, 3)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    z = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(ch.ChError) as e:  # no plan prepared in this workspace
        ch.ch_reduce_batched(torch.zeros((3, 2), dtype=torch.int32, device="cuda"), z,
                             torch.ones(3, dtype=torch.int32, device="cuda"),
                             torch.zeros((8, 2), dtype=torch.int32, device="cuda"), z, ws)
    assert e.value.code == ch.CH_ERR_ARG
