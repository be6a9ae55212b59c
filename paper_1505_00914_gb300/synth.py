"""Seeded synthetic point sets shaped like the paper's workloads.

This module only draws inputs: it holds none of the method's arithmetic, and it
is the one module that both the CUDA path's tests/benchmark and the CPU oracle's
tests consume.  Every generator returns a C-contiguous numpy int32 array of
shape (n, 2) holding (x, y) with 1 <= x, y <= p (the square of side p of
Section 2.1), and is a pure function of its arguments (numpy PCG64 seeded from
``numpy.random.SeedSequence``).

Distributions:
  * ``uniform``  - i.i.d. uniform on [1, p]^2, duplicates allowed;
  * ``disc``     - uniform over the lattice points of the inscribed disc
                   (centre ((p+1)/2, (p+1)/2), radius p/2), by rejection;
  * ``gaussian`` - isotropic normal, sigma = p/8, at the centre, rounded and
                   clamped to [1, p];
  * ``annulus``  - uniform over the ring p*[0.45, 0.5] about the centre,
                   rounded and clamped;
  * ``shells``   - stand-in for the paper's projected 3D skeleton scans
                   (Section 2.4, Fig. 2; the dataset itself is not available):
                   64 random elongated ellipsoidal shells and cylinders,
                   surface-sampled, projected orthographically onto xy and
                   quantised to the p-grid.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

DISTRIBUTIONS = ("uniform", "disc", "gaussian", "annulus", "shells")


def _rng(seed, *stream) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), *map(int, stream)])))


def uniform(n: int, p: int, seed: int = 0) -> np.ndarray:
    rng = _rng(seed, 1)
    return rng.integers(1, p + 1, size=(n, 2), dtype=np.int32)


def disc(n: int, p: int, seed: int = 0) -> np.ndarray:
    rng = _rng(seed, 2)
    out = np.empty((n, 2), dtype=np.int32)
    got = 0
    c2 = p + 1  # 2 * centre
    while got < n:
        m = max(1024, int((n - got) * 1.30) + 1024)
        q = rng.integers(1, p + 1, size=(m, 2), dtype=np.int64)
        d = (2 * q[:, 0] - c2) ** 2 + (2 * q[:, 1] - c2) ** 2
        q = q[d <= np.int64(p) * p]
        k = min(n - got, q.shape[0])
        out[got:got + k] = q[:k]
        got += k
    return out


def gaussian(n: int, p: int, seed: int = 0, sigma: float | None = None) -> np.ndarray:
    rng = _rng(seed, 3)
    s = p / 8.0 if sigma is None else float(sigma)
    c = (p + 1) / 2.0
    out = np.empty((n, 2), dtype=np.int32)
    step = 1 << 22
    for a in range(0, n, step):
        b = min(n, a + step)
        z = rng.standard_normal(size=(b - a, 2)) * s + c
        np.clip(np.rint(z), 1, p, out=z)
        out[a:b] = z
    return out


def annulus(n: int, p: int, seed: int = 0, r0: float = 0.45, r1: float = 0.5) -> np.ndarray:
    rng = _rng(seed, 4)
    c = (p + 1) / 2.0
    out = np.empty((n, 2), dtype=np.int32)
    step = 1 << 22
    for a in range(0, n, step):
        b = min(n, a + step)
        u = rng.random(b - a)
        r = np.sqrt((r0 * p) ** 2 + u * ((r1 * p) ** 2 - (r0 * p) ** 2))
        t = rng.random(b - a) * (2.0 * np.pi)
        z = np.empty((b - a, 2))
        z[:, 0] = c + r * np.cos(t)
        z[:, 1] = c + r * np.sin(t)
        np.clip(np.rint(z), 1, p, out=z)
        out[a:b] = z
    return out


def _rotation(rng) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def shells(n: int, p: int, seed: int = 0, k: int = 64) -> np.ndarray:
    """k random elongated shapes in the unit cube (half ellipsoidal shells,
    half open cylinders), lengths 0.1-0.6 of the box, random orientations;
    points sampled on their surfaces in proportion to a rough area, projected
    onto xy and quantised to [1, p]."""
    rng = _rng(seed, 5)
    kinds = rng.integers(0, 2, size=k)
    lengths = rng.uniform(0.1, 0.6, size=k)
    radii = lengths * rng.uniform(0.08, 0.25, size=k)
    centres = rng.uniform(0.25, 0.75, size=(k, 3))
    area = lengths * radii
    counts = np.floor(area / area.sum() * n).astype(np.int64)
    counts[: n - counts.sum()] += 1
    out = np.empty((n, 2), dtype=np.int32)
    pos = 0
    for i in range(k):
        m = int(counts[i])
        if m == 0:
            continue
        R = _rotation(rng)
        half = lengths[i] / 2.0
        if kinds[i] == 0:  # ellipsoidal shell, semi-axes (half, r, r)
            v = rng.standard_normal(size=(m, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            v *= np.array([half, radii[i], radii[i]])
        else:  # open cylinder of radius r along the local x axis
            t = rng.uniform(-half, half, size=m)
            a = rng.uniform(0.0, 2.0 * np.pi, size=m)
            v = np.stack([t, radii[i] * np.cos(a), radii[i] * np.sin(a)], axis=1)
        w = v @ R.T + centres[i]
        xy = np.floor(w[:, :2] * p) + 1
        np.clip(xy, 1, p, out=xy)
        out[pos:pos + m] = xy
        pos += m
    perm = rng.permutation(n)
    return out[perm]


_GEN = {"uniform": uniform, "disc": disc, "gaussian": gaussian,
        "annulus": annulus, "shells": shells}


def affine(pts: np.ndarray, p: int, seed: int = 0, min_scale: float = 0.25) -> np.ndarray:
    """The set under a seeded random similarity-plus-stretch: scaled by
    (s1, s2) in [min_scale, 1] along its own axes, rotated by a uniform angle
    about the box centre, shifted by a random offset that keeps it inside,
    then rounded and clamped to [1, p] (elongated, tilted variants of a
    shape)."""
    rng = _rng(seed, 7)
    s = rng.uniform(min_scale, 1.0, size=2)
    t = rng.uniform(0.0, 2.0 * np.pi)
    c = (p + 1) / 2.0
    z = (np.asarray(pts, dtype=np.float64) - c) * s
    R = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
    z = z @ R.T
    lo, hi = z.min(axis=0) if len(z) else np.zeros(2), z.max(axis=0) if len(z) else np.zeros(2)
    room = np.maximum(0.0, (p - 1) / 2.0 - np.maximum(-lo, hi))
    z += c + rng.uniform(-1.0, 1.0, size=2) * room
    out = np.clip(np.rint(z), 1, p).astype(np.int32)
    return np.ascontiguousarray(out)


def points(dist: str, n: int, p: int, seed: int = 0) -> np.ndarray:
    """Dispatch by distribution name."""
    return _GEN[dist](n, p, seed)


def boxed(dist: str, n: int, sx: int, sy: int, x0: int, y0: int, seed: int = 0) -> np.ndarray:
    """n points of a distribution drawn on the 65536 x 65536 square, scaled
    (integer arithmetic) to an sx by sy box and shifted to start at (x0, y0):
    int32 points anywhere, the input of the bounding-box steps.  The box must
    fit in int32."""
    base = points(dist, n, 65536, seed=seed).astype(np.int64) - 1
    x = x0 + (base[:, 0] * (sx - 1)) // 65535
    y = y0 + (base[:, 1] * (sy - 1)) // 65535
    return np.ascontiguousarray(np.stack([x, y], 1).astype(np.int32))


def batched_spec(B: int, seed: int = 0, n_lo: float = 1e2, n_hi: float = 1e6,
                 ps=(256, 1024, 4096, 16384), dists=("uniform", "disc", "gaussian")):
    """Per-set sizes of the batched workload: n log-uniform in [n_lo, n_hi],
    p drawn from ``ps``, distribution drawn from ``dists``."""
    rng = _rng(seed, 6)
    n = np.rint(10.0 ** rng.uniform(np.log10(n_lo), np.log10(n_hi), size=B)).astype(np.int64)
    p = np.asarray(ps, dtype=np.int32)[rng.integers(0, len(ps), size=B)]
    d = rng.integers(0, len(dists), size=B)
    return n, p, [dists[j] for j in d]


def batched(B: int, seed: int = 0, threads: int | None = None, **kw):
    """Ragged batch of B independent sets: returns (pts (sum n, 2) int32,
    offsets (B+1,) int64, ps (B,) int32, dists list)."""
    n, p, d = batched_spec(B, seed, **kw)
    offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(n, out=offsets[1:])
    pts = np.empty((int(offsets[-1]), 2), dtype=np.int32)

    def one(i):
        pts[offsets[i]:offsets[i + 1]] = points(d[i], int(n[i]), int(p[i]), seed=(seed * 1000003 + i))

    nt = threads or min(32, os.cpu_count() or 1)
    with _cf.ThreadPoolExecutor(nt) as ex:
        list(ex.map(one, range(B)))
    return pts, offsets, p, d
