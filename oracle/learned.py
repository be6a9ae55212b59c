"""Floating-point part of the learned culling proposal, restated in numpy.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU legs may import it; it never imports the CUDA library.

The paper has no learned part.  Its culling idea is what this serves: a convex
polygon whose vertices are input points is drawn inside the hull and the
points strictly inside it cannot be hull vertices, so Algorithm 1 may skip
them (the polygon only decides how much is skipped, never what the hull is).
Here the polygon's vertices are the sample points extreme in K directions
proposed by a small network from an occupancy histogram of the sample:

  sample     runs of R = 1024 consecutive points at J = 256 evenly spaced
             starts (the whole set when n <= R * J);
  histogram  32 x 32 cells, cell (bx, by) = ((x-1)*32 // p, (y-1)*32 // p),
             feature index by*32 + bx, value count * fl32(1024 / m) in float32
             (m = sample size);
  network    1024 -> 256 (ReLU) -> 256 (ReLU) -> K, every product computed
             with both operands rounded to bf16 and accumulated in float
             (here: float64 sums of the bf16-rounded operands);
  directions theta_k = 2 pi k / K + (pi / K) tanh(y_k);
  extremes   argmax over the sample of fl32(fl32(c_k x) + fl32(s_k y)),
             c_k, s_k float32, ties to the smallest point index;
  loss       mean over the batch and K outputs of (tanh(y) - t)^2.

`exact=True` drops the bf16 rounding, which makes the forward and backward
passes the textbook float64 ones; the tests pin those by finite differences.
"""
from __future__ import annotations

import numpy as np

IN, HID, K = 1024, 256, 16
R_RUN, J_RUNS = 1024, 256

# parameter vector layout: W[i][j] maps input i to output j
_SHAPES = (("W1", (IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
           ("W3", (HID, K)), ("b3", (K,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in _SHAPES)


def unpack(params):
    """Views W1, b1, W2, b2, W3, b3 of the flat parameter vector."""
    out, o = {}, 0
    for name, shape in _SHAPES:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in _SHAPES])


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, float32 values in a float64 vector."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in _SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[0])
            d[name] = rng.uniform(-lim, lim, size=shape).astype(np.float32)
        else:
            d[name] = np.zeros(shape, dtype=np.float32)
    return pack(d)


# ------------------------------------------------------------------ rounding
def to_f32(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float64).astype(np.float32)


def bf16(a) -> np.ndarray:
    """Round to float32, then to bf16 (round to nearest, ties to even);
    returned as float64.  NaN/Inf are not expected here."""
    f = np.ascontiguousarray(to_f32(a))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _op(a, exact):
    return np.asarray(a, dtype=np.float64) if exact else bf16(a)


# ------------------------------------------------------------------ features
def sample_index(n: int) -> np.ndarray:
    """Indices of the sample: all points when n <= R*J, else R consecutive
    points starting at j * (n // J), j = 0..J-1."""
    if n <= R_RUN * J_RUNS:
        return np.arange(n, dtype=np.int64)
    step = n // J_RUNS
    starts = np.arange(J_RUNS, dtype=np.int64) * step
    return (starts[:, None] + np.arange(R_RUN, dtype=np.int64)[None, :]).reshape(-1)


def histogram_counts(pts, p: int) -> np.ndarray:
    """Points per cell of the 32 x 32 occupancy grid: int64 (1024,)."""
    pts = np.asarray(pts, dtype=np.int64).reshape(-1, 2)
    bx = ((pts[:, 0] - 1) * 32) // p
    by = ((pts[:, 1] - 1) * 32) // p
    return np.bincount(by * 32 + bx, minlength=IN)


def histogram(pts, p: int) -> np.ndarray:
    """Occupancy histogram of the given points (no sampling): float32 (1024,),
    count * fl32(1024 / m)."""
    m = np.asarray(pts).reshape(-1, 2).shape[0]
    counts = histogram_counts(pts, p).astype(np.float32)
    if m == 0:
        return counts
    scale = np.float32(1024.0) / np.float32(m)
    return (counts * scale).astype(np.float32)


# ------------------------------------------------------------------ network
def forward(params, X, exact: bool = False):
    """H1 = relu(X W1 + b1), H2 = relu(H1 W2 + b2), Y = H2 W3 + b3 (float64)."""
    w = unpack(np.asarray(params, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64).reshape(-1, IN)
    H1 = np.maximum(_op(X, exact) @ _op(w["W1"], exact) + w["b1"], 0.0)
    H2 = np.maximum(_op(H1, exact) @ _op(w["W2"], exact) + w["b2"], 0.0)
    Y = _op(H2, exact) @ _op(w["W3"], exact) + w["b3"]
    return H1, H2, Y


def loss(Y, T):
    """mean((tanh(Y) - T)^2) and its gradient with respect to Y."""
    Y = np.asarray(Y, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    th = np.tanh(Y)
    d = th - T
    cnt = Y.size
    return float(np.sum(d * d) / cnt), 2.0 * d * (1.0 - th * th) / cnt


def backward(params, X, H1, H2, dY, exact: bool = False) -> np.ndarray:
    """Gradient of the loss with respect to every parameter (flat, float64),
    by the chain rule through the three layers; the ReLU gradient is taken as
    [h > 0].  Each product rounds its operands like the forward pass does."""
    w = unpack(np.asarray(params, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64).reshape(-1, IN)
    H1 = np.asarray(H1, dtype=np.float64)
    H2 = np.asarray(H2, dtype=np.float64)
    dY = np.asarray(dY, dtype=np.float64)
    g = {}
    g["W3"] = _op(H2, exact).T @ _op(dY, exact)
    g["b3"] = dY.sum(axis=0)
    dH2 = (_op(dY, exact) @ _op(w["W3"], exact).T) * (H2 > 0)
    g["W2"] = _op(H1, exact).T @ _op(dH2, exact)
    g["b2"] = dH2.sum(axis=0)
    dH1 = (_op(dH2, exact) @ _op(w["W2"], exact).T) * (H1 > 0)
    g["W1"] = _op(X, exact).T @ _op(dH1, exact)
    g["b1"] = dH1.sum(axis=0)
    return pack(g)


def adam(params, grads, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999,
         eps: float = 1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1 of their paper) with the
    bias correction folded into the step size; returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    lr_t = lr * np.sqrt(1 - b2 ** step) / (1 - b1 ** step)
    return params - lr_t * m / (np.sqrt(v) + eps), m, v


# ------------------------------------------------------------------ culling
def directions(Y, k: int = K):
    """theta_k = 2 pi k / K + (pi / K) tanh(y_k), float64."""
    Y = np.asarray(Y, dtype=np.float64).reshape(-1)
    kk = np.arange(k, dtype=np.float64)
    return 2.0 * np.pi * kk / k + (np.pi / k) * np.tanh(Y[:k])


def extremes(pts, index, c, s) -> np.ndarray:
    """For each direction (c_k, s_k) (float32), the index (from `index`) of the
    point of pts[index] with the largest fl32(fl32(c x) + fl32(s y)); ties go
    to the smallest index."""
    pts = np.asarray(pts).reshape(-1, 2)
    index = np.asarray(index, dtype=np.int64)
    x = pts[index, 0].astype(np.float32)
    y = pts[index, 1].astype(np.float32)
    out = np.empty(len(c), dtype=np.int64)
    for k, (ck, sk) in enumerate(zip(np.asarray(c, np.float32), np.asarray(s, np.float32))):
        score = (np.float32(ck) * x).astype(np.float32) + (np.float32(sk) * y).astype(np.float32)
        score = score.astype(np.float32)
        out[k] = index[score == score.max()].min()
    return out


def area2(poly) -> int:
    """Twice the area of a counter-clockwise polygon (exact integers); 0 for
    fewer than three vertices."""
    P = [(int(x), int(y)) for x, y in np.asarray(poly).reshape(-1, 2)]
    if len(P) < 3:
        return 0
    return sum(P[i][0] * P[(i + 1) % len(P)][1] - P[i][1] * P[(i + 1) % len(P)][0]
               for i in range(len(P)))


def choose_polygon(pts, index, dirs, has_net: bool):
    """The culling polygon: the strict hull of the sample points extreme in
    the sector-centre directions (dirs[0] = (cos, sin)), or, with a network,
    that of its directions (dirs[1]) when its area is strictly larger.
    Returns (polygon, chosen set, extremes of both sets)."""
    import oracle
    pts = np.asarray(pts).reshape(-1, 2)
    sets = 2 if has_net else 1
    ext = [extremes(pts, index, dirs[s][0], dirs[s][1]) if len(index) else
           np.full(len(dirs[s][0]), -1, np.int64) for s in range(sets)]
    polys = [oracle.hull_points(pts[e[e >= 0]]) for e in ext]
    sel = 1 if sets == 2 and area2(polys[1]) > area2(polys[0]) else 0
    return polys[sel], sel, ext
