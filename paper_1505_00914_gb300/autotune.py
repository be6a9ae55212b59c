"""Autotuner for the batched launch: picks the work plan's chunk size per
column (``chunk_mult``) and the persistent kernel's CTA shape
(``fold_threads``: how many of a CTA's 1024 threads fold points while the
others finish the previous set, 0 for no split) by timing the real launch on
the batch at hand, and caches the winner per (device, batch shape) in a JSON
file.

The chunk size trades load balance (small chunks, more items for the
persistent CTAs to share) against per-item overhead (every item initialises a
private L of p columns and, when a set has several chunks, writes and merges a
partial row of p words).  The CTA shape trades streaming width (threads with
loads in flight) against how much of a set's finishing hides behind the next
set's folding.  Everything timed here is the library's own launch; no kernel
is written in Python.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import ch

CANDIDATES = (8, 16, 32, 64, 128, 256, 1024, 4096)
SHAPES = ch.CH_BATCH_FOLD_SHAPES  # fold_threads of the CTA (0: no split)


def _cache_path() -> str:
    return os.environ.get("CH_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "chull_gb300", "autotune.json"))


def _kernel_digest() -> str:
    """Digest of the batched kernel's source, so that a tuning measured on
    another version of the kernel is not reused."""
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "batched.cu")
    try:
        with open(src, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:12]
    except OSError:
        return "unknown"


def batch_key(offsets, ps, candidates=CANDIDATES, shapes=SHAPES) -> str:
    """Device name + digests of the batch's shape (n and p per set), of the
    candidate chunk sizes and CTA shapes and of the kernel source."""
    off = np.asarray(offsets, np.int64)
    pp = np.asarray(ps, np.int32)
    h = hashlib.sha256(np.diff(off).tobytes() + pp.tobytes()).hexdigest()[:16]
    c = ",".join(str(int(x)) for x in candidates)
    f = ",".join(str(int(x)) for x in shapes)
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "no-device"
    return f"{dev}|B={pp.shape[0]}|{h}|C={c}|F={f}|K={_kernel_digest()}"


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(db):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only loses the cache


def tune_batched(d_pts, offsets, ps, d_off, d_ps, hull, d_hoff, counts, candidates=CANDIDATES,
                 shapes=SHAPES, reps: int = 3, use_cache: bool = True):
    """Returns ((chunk_mult, fold_threads), {"chunk_mult/fold_threads": ms})
    for this batch: every pair timed on the real launch.  The host arrays
    offsets/ps describe the batch, the device tensors are those the caller
    will launch with."""
    key = batch_key(offsets, ps, candidates, shapes)
    db = _load() if use_cache else {}
    if key in db:
        e = db[key]
        return (int(e["chunk_mult"]), int(e["fold_threads"])), dict(e["ms"])
    need = max(ch.ch_batched_workspace_size(offsets, ps, c) for c in candidates)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    times = {}
    for c in candidates:
        for f in shapes:
            ch.ch_batched_prepare(offsets, ps, ws, c, fold_threads=f)
            ch.ch_hull_batched(d_pts, d_off, d_ps, hull, d_hoff, counts, ws)  # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                ch.ch_hull_batched(d_pts, d_off, d_ps, hull, d_hoff, counts, ws)
            b.record()
            torch.cuda.synchronize()
            times[f"{c}/{f}"] = a.elapsed_time(b) / reps
    rc = ch.ch_sync_status()
    if rc != ch.CH_OK:
        raise ch.ChError(rc, "tune_batched")
    best = min(times, key=times.get)
    cm, fold = (int(x) for x in best.split("/"))
    db[key] = {"chunk_mult": cm, "fold_threads": fold, "ms": times}
    if use_cache:
        _store(db)
    return (cm, fold), times
