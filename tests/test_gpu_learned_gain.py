"""What the trained network gains over the culling proposal without it.

Held-out seeded sets (seeds the training set never used) of the training
family: the four plain workload shapes, stretched and rotated.  With the
trained weights the proposal keeps the larger of the network's polygon and
the sector-centre polygon, so it never culls a smaller area; the test asks
that it culls more points on average and that the network's polygon is the
one used on a good share of the stretched shapes.  Cull rate = share of the
input points strictly inside the culling polygon (Linit.lo <= y <= Linit.hi
in their column)."""
import os

import numpy as np
import pytest
import torch

from paper_1505_00914_gb300 import ch, synth, train
from gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(__file__), os.pardir, "paper_1505_00914_gb300", "weights",
                       "cull_mlp_k16.npz")


def cull_rate(d, Linit):
    li = Linit.long()
    x = d[:, 0].long() - 1
    y = d[:, 1].long()
    col = li[x]
    return float(((y >= col[:, 0]) & (y <= col[:, 1])).float().mean().item())


def test_trained_network_culls_more_than_sector_centres():
    need_gpu()
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights in the package")
    params = train.load_params(WEIGHTS)
    rng = np.random.default_rng(20261204)
    gains, chosen = [], 0
    for t in range(40):
        dist = ("uniform", "disc", "gaussian", "shells")[t % 4]
        p = int(rng.choice([1024, 4096, 16384, 65536]))
        seed = 10_000_000 + t  # training sets use seeds 1_000_003 + i, i < 10^6
        P = synth.affine(synth.points(dist, 300_000, p, seed=seed), p, seed=seed)
        d = dev(P).reshape(-1, 2)
        with_net = ch.ch_cull_propose(d, p, params=params)
        without = ch.ch_cull_propose(d, p)
        a, b = cull_rate(d, with_net["Linit"]), cull_rate(d, without["Linit"])
        gains.append(a - b)
        chosen += int(with_net["chosen"].item() == 1)
    gains = np.asarray(gains)
    assert ch.ch_sync_status() == ch.CH_OK
    assert gains.mean() > 0, gains
    assert chosen >= 8, chosen
