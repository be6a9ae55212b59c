"""Trains the culling network on the GPU with the library's own kernels.

Every step runs ch_mlp_forward (three bf16 tensor-core GEMMs with fused bias
and ReLU), ch_mlp_loss (tanh-MSE against the label offsets), ch_mlp_backward
(six GEMMs and three column sums) and ch_mlp_adam; PyTorch only holds the
tensors.  The training set (histogram counts and label offsets) is a file
written beforehand by the oracle's label generator; nothing here computes a
label.

    python -m paper_1505_00914_gb300.train --data train.npz --out weights.npz

The weights file holds the float32 parameter vector (ch.CH_MLP_PARAMS values,
the C ABI's layout) and the training record.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import ch


def init_params(seed: int) -> torch.Tensor:
    """He-uniform weights, zero biases, in the C ABI's parameter layout."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for fan_in, fan_out in ((ch.CH_MLP_IN, ch.CH_MLP_HID), (ch.CH_MLP_HID, ch.CH_MLP_HID),
                            (ch.CH_MLP_HID, ch.CH_MLP_K)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append((torch.rand(fan_in * fan_out, generator=g) * 2 - 1) * lim)
        parts.append(torch.zeros(fan_out))
    w = torch.cat(parts).float()
    assert w.numel() == ch.CH_MLP_PARAMS
    return w


def load_params(path: str, device="cuda") -> torch.Tensor:
    d = np.load(path)
    w = torch.from_numpy(np.ascontiguousarray(d["params"], dtype=np.float32))
    if w.numel() != ch.CH_MLP_PARAMS:
        raise ValueError(f"{path}: {w.numel()} parameters, expected {ch.CH_MLP_PARAMS}")
    return w.to(device)


def evaluate(params, X, T, batch: int = 4096) -> float:
    tot, n = 0.0, 0
    for i in range(0, X.shape[0], batch):
        xb, tb = X[i:i + batch], T[i:i + batch]
        _, _, Y = ch.ch_mlp_forward(params, xb)
        loss, _ = ch.ch_mlp_loss(Y, tb)
        tot += float(loss.item()) * xb.shape[0]
        n += xb.shape[0]
    return tot / max(n, 1)


def train(counts: np.ndarray, labels: np.ndarray, m: int, epochs: int = 8, batch: int = 1024,
          lr: float = 1e-3, holdout: float = 0.05, seed: int = 0, log=print):
    dev = torch.device("cuda")
    scale = np.float32(1024.0) / np.float32(m)
    N = counts.shape[0]
    nh = max(1, int(N * holdout))
    X = (torch.from_numpy(counts.astype(np.float32)).to(dev) * float(scale)).contiguous()
    T = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.float32)).to(dev)
    Xtr, Ttr, Xho, Tho = X[:-nh], T[:-nh], X[-nh:], T[-nh:]
    params = init_params(seed).to(dev)
    mom = torch.zeros_like(params)
    vel = torch.zeros_like(params)
    zero = torch.zeros(ch.CH_MLP_PARAMS, device=dev)
    base = evaluate(zero, Xho, Tho)  # the sector centres: what the path does without a network
    g = torch.Generator(device=dev).manual_seed(seed)
    steps_per_epoch = max(1, Xtr.shape[0] // batch)
    total = epochs * steps_per_epoch
    H1 = torch.empty((batch, ch.CH_MLP_HID), device=dev)
    H2 = torch.empty_like(H1)
    Y = torch.empty((batch, ch.CH_MLP_K), device=dev)
    ws = torch.empty(2 * batch * ch.CH_MLP_HID * 4, dtype=torch.uint8, device=dev)
    grads = torch.empty_like(params)
    record = {"holdout_loss_sector_centres": base, "epochs": []}
    step = 0
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(Xtr.shape[0], device=dev, generator=g)
        run = 0.0
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            xb, tb = Xtr.index_select(0, idx), Ttr.index_select(0, idx)
            step += 1
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / total))
            ch.ch_mlp_forward(params, xb, H1, H2, Y)
            loss, dY = ch.ch_mlp_loss(Y, tb)
            ch.ch_mlp_backward(params, xb, H1, H2, dY, grads=grads, workspace=ws)
            ch.ch_mlp_adam(params, grads, mom, vel, step, lr_t)
            if b % 64 == 0:
                run = float(loss.item())
        ho = evaluate(params, Xho, Tho)
        record["epochs"].append({"epoch": ep + 1, "train_loss_last": run, "holdout_loss": ho})
        log(f"epoch {ep + 1}: train {run:.4f} holdout {ho:.4f} (sector centres {base:.4f}) "
            f"{time.time() - t0:.1f} s")
    rc = ch.ch_sync_status()
    if rc != ch.CH_OK:
        raise ch.ChError(rc, "train")
    record.update({"sets": int(N), "holdout_sets": nh, "batch": batch, "lr": lr, "steps": step,
                   "seconds": time.time() - t0, "holdout_loss": record["epochs"][-1]["holdout_loss"]})
    return params, record


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    d = np.load(a.data)
    params, rec = train(d["counts"], d["labels"], int(d["m"]), a.epochs, a.batch, a.lr, seed=a.seed)
    rec["data_seed"] = int(d["seed"])
    np.savez_compressed(a.out, params=params.cpu().numpy(), record=json.dumps(rec))
    print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
