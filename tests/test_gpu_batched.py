"""Parity of the batched path (one persistent launch over many sets) with the
CPU oracle, set by set; bit-exact hull vertex lists."""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_00914_gb300 import autotune, ch, synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def run_batch(pts, offsets, ps, chunk_mult=64, fold=None):
    d_pts = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 2)).cuda()
    d_off = torch.from_numpy(np.asarray(offsets, np.int64)).cuda()
    d_ps = torch.from_numpy(np.asarray(ps, np.int32)).cuda()
    hoff = ch.hull_capacity_offsets(offsets, ps)
    d_hoff = torch.from_numpy(hoff).cuda()
    hull = torch.zeros((max(1, int(hoff[-1])), 2), dtype=torch.int32, device="cuda")
    cnt = torch.full((len(ps),), -7, dtype=torch.int32, device="cuda")
    nws = ch.ch_batched_workspace_size(offsets, ps, chunk_mult)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    ch.ch_batched_prepare(offsets, ps, ws, chunk_mult, fold_threads=fold)
    ch.ch_hull_batched(d_pts, d_off, d_ps, hull, d_hoff, cnt, ws)
    torch.cuda.synchronize()
    return hull.cpu().numpy(), hoff, cnt.cpu().numpy()


def check_sets(pts, offsets, ps, hull, hoff, cnt, sets=None):
    for s in (range(len(ps)) if sets is None else sets):
        P = pts[offsets[s]:offsets[s + 1]]
        H = oracle.hull_chain(oracle.reduce(P, int(ps[s])))
        got = hull[hoff[s]:hoff[s] + cnt[s]]
        assert cnt[s] == H.shape[0], (s, cnt[s], H.shape[0])
        np.testing.assert_array_equal(got, H, err_msg=f"set {s}")


def test_mixed_small_batch():
    rng = np.random.default_rng(4)
    B = 300
    ps = rng.choice([1, 2, 5, 31, 256, 1000, 1024, 4096, 16384], size=B).astype(np.int32)
    ns = np.rint(10 ** rng.uniform(0, 5.3, size=B)).astype(np.int64)
    ns[rng.random(B) < 0.05] = 0
    dists = ["uniform", "disc", "gaussian", "annulus"]
    parts = [synth.points(dists[i % 4], int(ns[i]), int(ps[i]), seed=i) for i in range(B)]
    offsets = np.zeros(B + 1, np.int64)
    np.cumsum(ns, out=offsets[1:])
    pts = np.concatenate(parts) if parts else np.zeros((0, 2), np.int32)
    for fold in ch.CH_BATCH_FOLD_SHAPES:
        hull, hoff, cnt = run_batch(pts, offsets, ps, fold=fold)
        check_sets(pts, offsets, ps, hull, hoff, cnt)


def test_multi_chunk_sets_merge():
    """chunk_mult = 1 cuts every set of more than 65536 points into chunks."""
    rng = np.random.default_rng(5)
    ps = np.asarray([256, 1024, 4096, 16384, 16384, 300, 7], np.int32)
    ns = np.asarray([400_000, 300_001, 200_003, 150_000, 70_000, 1_000_000, 131_073], np.int64)
    parts = [synth.points(["uniform", "disc", "gaussian", "annulus"][i % 4], int(ns[i]), int(ps[i]),
                          seed=50 + i) for i in range(len(ps))]
    offsets = np.zeros(len(ps) + 1, np.int64)
    np.cumsum(ns, out=offsets[1:])
    pts = np.concatenate(parts)
    for cm in (1, 3, 64):
        for fold in ch.CH_BATCH_FOLD_SHAPES:
            hull, hoff, cnt = run_batch(pts, offsets, ps, chunk_mult=cm, fold=fold)
            check_sets(pts, offsets, ps, hull, hoff, cnt)


def test_misaligned_set_starts_and_degenerate_sets():
    # sets of odd lengths so that most start 8 (not 16) bytes into a pair
    sets = [np.asarray([[3, 4]] * 5, np.int32), np.asarray([[2, 5], [2, 1], [2, 3]], np.int32),
            np.asarray([[k, k] for k in range(1, 8)], np.int32), np.zeros((0, 2), np.int32),
            np.asarray([[1, 1]], np.int32), synth.disc(999, 64, seed=3), synth.uniform(1001, 33, 4)]
    ps = np.asarray([7, 7, 7, 9, 1, 64, 33], np.int32)
    offsets = np.zeros(len(sets) + 1, np.int64)
    np.cumsum([s.shape[0] for s in sets], out=offsets[1:])
    pts = np.concatenate(sets)
    for fold in ch.CH_BATCH_FOLD_SHAPES:
        hull, hoff, cnt = run_batch(pts, offsets, ps, fold=fold)
        check_sets(pts, offsets, ps, hull, hoff, cnt)


def test_batched_range_error_and_arguments():
    pts = np.asarray([[1, 1], [9, 2], [3, 3]], np.int32)
    run_batch(pts, np.asarray([0, 3]), np.asarray([8], np.int32))
    assert ch.ch_sync_status() == ch.CH_ERR_RANGE
    with pytest.raises(ch.ChError) as e:
        ch.ch_batched_workspace_size(np.asarray([0, 3]), np.asarray([20000], np.int32))
    assert e.value.code == ch.CH_ERR_ARG
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    z = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(ch.ChError) as e:  # no plan prepared in this workspace
        ch.ch_hull_batched(torch.zeros((3, 2), dtype=torch.int32, device="cuda"), z,
                           torch.ones(3, dtype=torch.int32, device="cuda"),
                           torch.zeros((8, 2), dtype=torch.int32, device="cuda"), z,
                           torch.zeros(3, dtype=torch.int32, device="cuda"), ws)
    assert e.value.code == ch.CH_ERR_ARG


def test_batched_config_full_size_sampled():
    """10,000 sets, n log-uniform in [1e2, 1e6], p in {256, 1024, 4096, 16384},
    uniform/disc/Gaussian (the benchmark's batch), one direct launch at the
    default chunk multiplier 64; 200 sets and the largest checked.  The
    benchmark's own launch (autotuned multiplier, CUDA-graph replay) is
    checked by test_batched_graph_replay_as_benchmarked."""
    pts, offsets, ps, _ = synth.batched(10_000, seed=4)
    hull, hoff, cnt = run_batch(pts, offsets, ps)
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(len(ps), size=200, replace=False).tolist())
                    | {int(np.argmax(np.diff(offsets)))})
    check_sets(pts, offsets, ps, hull, hoff, cnt, sets=sample)
    assert np.all(cnt >= 1)


def test_culling_polygon_shapes():
    """Sets for which the extreme-point polygon of the finishing step is
    degenerate, tight or full of boundary points: every hull exact."""
    rng = np.random.default_rng(21)
    sets, ps = [], []
    p = 4096
    t = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    circle = np.stack([2048 + 2000 * np.cos(t), 2048 + 2000 * np.sin(t)], 1).round().astype(np.int32)
    sets.append(circle); ps.append(p)
    g = np.arange(1, 65)
    sets.append(np.stack(np.meshgrid(g, g), -1).reshape(-1, 2).astype(np.int32)); ps.append(64)
    tri = rng.integers(1, p + 1, size=(200_000, 2))
    sets.append(tri[tri[:, 1] <= tri[:, 0]].astype(np.int32)); ps.append(p)
    diag = np.stack([np.arange(1, 5001), np.arange(1, 5001)], 1).astype(np.int32)
    sets.append(diag); ps.append(5000)
    two = np.asarray([[5, 1], [5, 9], [9, 3], [9, 4], [5, 5]], np.int32)
    sets.append(two); ps.append(9)
    # points on the octagon-like boundary of a square with cut corners, plus interior
    sq = rng.integers(100, 3900, size=(100_000, 2))
    edge = np.concatenate([np.stack([np.arange(100, 3900), np.full(3800, 100)], 1),
                           np.stack([np.full(3800, 3899), np.arange(100, 3900)], 1)])
    sets.append(np.concatenate([sq, edge]).astype(np.int32)); ps.append(p)
    for d in ("uniform", "disc", "gaussian", "annulus"):
        sets.append(synth.points(d, 300_000, 16384, seed=len(sets))); ps.append(16384)
    ps = np.asarray(ps, np.int32)
    offsets = np.zeros(len(sets) + 1, np.int64)
    np.cumsum([s.shape[0] for s in sets], out=offsets[1:])
    pts = np.concatenate(sets)
    for cm in (1, 64):
        for fold in ch.CH_BATCH_FOLD_SHAPES:
            hull, hoff, cnt = run_batch(pts, offsets, ps, chunk_mult=cm, fold=fold)
            check_sets(pts, offsets, ps, hull, hoff, cnt)


def _device_batch(pts, offsets, ps):
    d_pts = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 2)).cuda()
    d_off = torch.from_numpy(np.asarray(offsets, np.int64)).cuda()
    d_ps = torch.from_numpy(np.asarray(ps, np.int32)).cuda()
    hoff = ch.hull_capacity_offsets(offsets, ps)
    d_hoff = torch.from_numpy(hoff).cuda()
    hull = torch.zeros((max(1, int(hoff[-1])), 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(len(ps), dtype=torch.int32, device="cuda")
    return d_pts, d_off, d_ps, hoff, d_hoff, hull, cnt


def run_batch_graph(dev_batch, offsets, ps, chunk_mult, replays=2, fold=None):
    """The benchmark's launch: prepare the plan, a first call on a side stream
    (set-up), capture one ch_hull_batched in a CUDA graph on that stream, then
    replay the graph; the outputs are overwritten with garbage before every
    replay, so each replay's result is its own.  Returns one (hull, counts)
    per replay."""
    d_pts, d_off, d_ps, hoff, d_hoff, hull, cnt = dev_batch
    ws = torch.empty(ch.ch_batched_workspace_size(offsets, ps, chunk_mult), dtype=torch.uint8,
                     device="cuda")
    ch.ch_batched_prepare(offsets, ps, ws, chunk_mult, fold_threads=fold)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        ch.ch_hull_batched(d_pts, d_off, d_ps, hull, d_hoff, cnt, ws)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        ch.ch_hull_batched(d_pts, d_off, d_ps, hull, d_hoff, cnt, ws)
    out = []
    for _ in range(replays):
        hull.fill_(-9)
        cnt.fill_(-7)
        graph.replay()
        torch.cuda.synchronize()
        out.append((hull.cpu().numpy(), cnt.cpu().numpy()))
    assert ch.ch_sync_status(stream) == ch.CH_OK
    del graph
    return out


class _OracleHulls:
    """Oracle hull of each set (Algorithm 1, then the hull of its chains),
    computed once per set."""

    def __init__(self, pts, offsets, ps):
        self.pts, self.off, self.ps, self.h = pts, offsets, ps, {}

    def __call__(self, s):
        if s not in self.h:
            P = self.pts[self.off[s]:self.off[s + 1]]
            self.h[s] = oracle.hull_chain(oracle.reduce(P, int(self.ps[s])))
        return self.h[s]


def _check_against(hulls, hoff, hull, cnt, sets, where):
    for s in sets:
        H = hulls(s)
        assert cnt[s] == H.shape[0], (where, s, int(cnt[s]), H.shape[0])
        np.testing.assert_array_equal(hull[hoff[s]:hoff[s] + cnt[s]], H, err_msg=f"{where} set {s}")


def test_batched_graph_replay_as_benchmarked():
    """The launch the benchmark times: the 10,000-set batch, the chunk
    multiplier and CTA shape chosen by the autotuner on this batch (and 4096
    with the default shape), one ch_hull_batched captured in a CUDA graph and
    replayed twice; 200 sampled sets and the largest against the oracle."""
    pts, offsets, ps, _ = synth.batched(10_000, seed=4)
    db = _device_batch(pts, offsets, ps)
    d_pts, d_off, d_ps, hoff, d_hoff, hull, cnt = db
    (best, fold), times = autotune.tune_batched(d_pts, offsets, ps, d_off, d_ps, hull, d_hoff,
                                                cnt, use_cache=False)
    assert best in autotune.CANDIDATES and fold in autotune.SHAPES
    assert len(times) == len(autotune.CANDIDATES) * len(autotune.SHAPES)
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(len(ps), size=200, replace=False).tolist())
                    | {int(np.argmax(np.diff(offsets)))})
    hulls = _OracleHulls(pts, offsets, ps)
    for cm, fd in sorted({(best, fold), (4096, ch.CH_BATCH_FOLD_DEFAULT)}):
        for r, (h, c) in enumerate(run_batch_graph(db, offsets, ps, cm, fold=fd)):
            assert np.all(c >= 1)
            _check_against(hulls, hoff, h, c, sample, f"chunk_mult {cm} fold {fd} replay {r}")


def test_batched_graph_replay_every_candidate():
    """Every chunk multiplier and CTA shape the autotuner may choose, each as
    a CUDA-graph replay (twice) on a 1,000-set batch of the benchmark's
    recipe: every set against the oracle."""
    pts, offsets, ps, _ = synth.batched(1_000, seed=11)
    db = _device_batch(pts, offsets, ps)
    hoff = db[3]
    hulls = _OracleHulls(pts, offsets, ps)
    for cm in autotune.CANDIDATES:
        for fd in autotune.SHAPES:
            for r, (h, c) in enumerate(run_batch_graph(db, offsets, ps, cm, fold=fd)):
                _check_against(hulls, hoff, h, c, range(len(ps)),
                               f"chunk_mult {cm} fold {fd} replay {r}")
