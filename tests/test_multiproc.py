"""Multi-process path on CPU (gloo, world size 2).

A single problem shards by points: each rank reduces its slice with
Algorithm 1, and one all-reduce MIN over (lo, -hi) merges the partial arrays
(min and max commute, so the merge is exact and the empty sentinel (p+1, -1)
is the identity).  The merged L must equal the oracle's L of all points, and
its hull the oracle hull."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, p, n, out):
    import oracle
    from paper_1505_00914_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = synth.points("disc", n, p, seed=77)
        lo_i, hi_i = rank * n // world, (rank + 1) * n // world
        L = oracle.reduce(P[lo_i:hi_i], p).astype(np.int64)
        t = torch.from_numpy(np.stack([L[:, 0], -L[:, 1]], 1).copy())
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        merged = np.stack([t[:, 0].numpy(), -t[:, 1].numpy()], 1).astype(np.int32)
        if rank == 0:
            np.save(out, merged)
    finally:
        dist.destroy_process_group()


def test_sharded_reduce_merges_exactly(tmp_path):
    import oracle
    from paper_1505_00914_gb300 import synth
    p, n = 4096, 200_001
    out = str(tmp_path / "L.npy")
    mp.start_processes(_worker, args=(2, _free_port(), p, n, out), nprocs=2, join=True,
                       start_method="spawn")
    merged = np.load(out)
    P = synth.points("disc", n, p, seed=77)
    L = oracle.reduce(P, p)
    np.testing.assert_array_equal(merged, L)
    np.testing.assert_array_equal(oracle.hull_chain(merged), oracle.hull_points(P))


def _bench_worker(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the slowest rank's time is the job's time
        t = bench._max_over_ranks(torch, dist, world, 1.5 + rank)
        # weak scaling: every rank draws its own instances of the same shape
        p, n, inputs = bench.gen_inputs("plain_small", rank)
        h = [int(np.frombuffer(P.tobytes(), np.uint8).sum()) for _, P in inputs]
        np.save(out + f".{rank}.npy", np.array([t, p, n] + h, dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_bench_ranks_time_and_inputs(tmp_path):
    out = str(tmp_path / "r")
    mp.start_processes(_bench_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    r0, r1 = np.load(out + ".0.npy"), np.load(out + ".1.npy")
    assert r0[0] == r1[0] == 2.5
    assert tuple(r0[1:3]) == tuple(r1[1:3])
    assert not np.array_equal(r0[3:], r1[3:])
