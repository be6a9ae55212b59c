"""Training set of the culling network, written from the oracle alone.

TEST AND TRAINING INFRASTRUCTURE: it imports only the oracle and the seeded
input generators; the CUDA library never runs here.

Set i draws m points of one of the plain workloads' shapes (uniform square,
inscribed disc, Gaussian sigma = p/8, projected 3D shells) at a side p from
{1024, 4096, 16384, 65536}, both by a seeded choice; three sets in four are
then stretched and rotated by a seeded random map (synth.affine).  Its features are the
occupancy histogram counts (oracle/learned.py's cells; the network input is
count * fl32(1024 / m)) and its label the K per-sector direction offsets that
maximise the area of the polygon of the extreme hull vertices
(oracle_best_offsets, on the hull the oracle computes for the set).

    python -m oracle.labels --sets 1000000 --out train.npz [--workers 16]

writes counts (uint16, sets x 1024), labels (float32, sets x 16), ps, dists
and m.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import time

import numpy as np

DISTS = ("uniform", "disc", "gaussian", "shells")
PS = (1024, 4096, 16384, 65536)


def set_spec(i: int, seed: int):
    """(distribution, p, stretched): three sets in four go through a seeded
    random stretch and rotation (synth.affine), so that the network sees
    tilted, elongated variants of the shapes as well as the shapes."""
    rng = np.random.default_rng([seed, i, 7])
    d = DISTS[int(rng.integers(0, len(DISTS)))]
    p = PS[int(rng.integers(0, len(PS)))]
    return d, p, bool(rng.random() < 0.75)


def _chunk(args):
    lo, hi, m, seed, k = args
    import oracle
    from oracle import learned as Lm
    from paper_1505_00914_gb300 import synth
    n = hi - lo
    counts = np.zeros((n, Lm.IN), dtype=np.uint16)
    pts = np.empty((n * m, 2), dtype=np.int32)
    ps = np.empty(n, dtype=np.int32)
    dist_ix = np.empty(n, dtype=np.int8)
    for j, i in enumerate(range(lo, hi)):
        d, p, stretched = set_spec(i, seed)
        P = synth.points(d, m, p, seed=seed * 1_000_003 + i)
        if stretched:
            P = synth.affine(P, p, seed=seed * 1_000_003 + i)
        pts[j * m:(j + 1) * m] = P
        ps[j] = p
        dist_ix[j] = DISTS.index(d)
        counts[j] = Lm.histogram_counts(P, p)
    offsets = np.arange(n + 1, dtype=np.int64) * m
    labels, _ = oracle.label_batch(pts, offsets, ps, K=k)
    return lo, counts, labels, ps, dist_ix


def build(sets: int, m: int = 8192, seed: int = 1, k: int = 16, workers: int | None = None,
          chunk: int = 1024):
    workers = workers or os.cpu_count() or 1
    jobs = [(lo, min(sets, lo + chunk), m, seed, k) for lo in range(0, sets, chunk)]
    counts = np.zeros((sets, 1024), dtype=np.uint16)
    labels = np.zeros((sets, k), dtype=np.float32)
    ps = np.zeros(sets, dtype=np.int32)
    dist_ix = np.zeros(sets, dtype=np.int8)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for lo, c, lab, pp, di in pool.imap_unordered(_chunk, jobs):
            hi = lo + c.shape[0]
            counts[lo:hi], labels[lo:hi], ps[lo:hi], dist_ix[lo:hi] = c, lab, pp, di
    return counts, labels, ps, dist_ix


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=1_000_000)
    ap.add_argument("--m", type=int, default=8192, help="points per training set")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--workers", type=int, default=None)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    t0 = time.time()
    counts, labels, ps, dist_ix = build(a.sets, a.m, a.seed, workers=a.workers)
    np.savez(a.out, counts=counts, labels=labels, ps=ps, dists=dist_ix, m=np.int64(a.m),
             seed=np.int64(a.seed))
    print(f"labels: {a.sets} sets of {a.m} points in {time.time() - t0:.1f} s -> {a.out}", flush=True)


if __name__ == "__main__":
    main()
