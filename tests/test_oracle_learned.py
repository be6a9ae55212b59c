"""Pins of the learned culling oracle (oracle/learned.py and the label
routines of oracle.c) against things other than itself: a library bf16
conversion, finite differences, closed forms, brute-force loops."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import learned as Lm


def test_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    vals = np.concatenate([
        rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
        # exact halfway cases: ties to even
        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -130, 0.0, -0.0, 65504.0]),
    ]).astype(np.float32)
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(Lm.bf16(vals), ref)


def _small_problem(seed, M=3):
    rng = np.random.default_rng(seed)
    params = Lm.init_params(seed) * 0.5
    w = Lm.unpack(params)
    w["b1"][:] = rng.normal(0, 0.1, Lm.HID)
    w["b2"][:] = rng.normal(0, 0.1, Lm.HID)
    w["b3"][:] = rng.normal(0, 0.1, Lm.K)
    X = rng.uniform(0, 3, size=(M, Lm.IN))
    T = rng.uniform(-1, 1, size=(M, Lm.K))
    return params, X, T


def test_backward_matches_finite_differences():
    params, X, T = _small_problem(1)

    def f(theta):
        return Lm.loss(Lm.forward(theta, X, exact=True)[2], T)[0]

    H1, H2, Y = Lm.forward(params, X, exact=True)
    _, dY = Lm.loss(Y, T)
    g = Lm.backward(params, X, H1, H2, dY, exact=True)
    rng = np.random.default_rng(2)
    # coordinates from every block: W1, b1, W2, b2, W3, b3
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in Lm._SHAPES])
    idx = np.concatenate([rng.integers(offs[i], offs[i + 1], 8) for i in range(6)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        fd = (f(params + e) - f(params - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_forward_closed_forms():
    params = np.zeros(Lm.N_PARAMS)
    w = Lm.unpack(params)
    w["b1"][:] = np.linspace(-1, 1, Lm.HID)
    w["b3"][:] = np.arange(Lm.K) * 0.25
    X = np.random.default_rng(3).uniform(0, 5, size=(4, Lm.IN))
    for exact in (True, False):
        H1, H2, Y = Lm.forward(params, X, exact=exact)
        np.testing.assert_array_equal(H1, np.tile(np.maximum(w["b1"], 0), (4, 1)))
        np.testing.assert_array_equal(H2, 0)
        np.testing.assert_array_equal(Y, np.tile(w["b3"], (4, 1)))
    # one path: y_0 = relu(relu(x_5) * 2) * 3 + 1
    params = np.zeros(Lm.N_PARAMS)
    w = Lm.unpack(params)
    w["W1"][5, 7] = 1.0
    w["W2"][7, 9] = 2.0
    w["W3"][9, 0] = 3.0
    w["b3"][0] = 1.0
    X = np.zeros((2, Lm.IN))
    X[0, 5], X[1, 5] = 1.5, -2.0
    Y = Lm.forward(params, X)[2]
    assert Y[0, 0] == 1.5 * 6 + 1 and Y[1, 0] == 1.0


def test_bf16_forward_close_to_exact():
    params, X, _ = _small_problem(4, M=8)
    Ye = Lm.forward(params, X, exact=True)[2]
    Yb = Lm.forward(params, X, exact=False)[2]
    assert np.max(np.abs(Ye - Yb)) <= 0.05 * np.max(np.abs(Ye)) + 1e-3
    assert not np.array_equal(Ye, Yb)


def test_loss_closed_form():
    Y = np.array([[0.0, math.atanh(0.5)]])
    T = np.array([[1.0, 0.5]])
    l, dY = Lm.loss(Y, T)
    assert l == pytest.approx(0.5)  # ((0 - 1)^2 + 0) / 2
    assert dY[0, 0] == pytest.approx(2 * (-1) * 1 / 2) and dY[0, 1] == pytest.approx(0.0)


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3])
    p0 = np.array([1.0, 2.0, 3.0])
    p1, m, v = Lm.adam(p0, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # lr_t m / (sqrt(v) + eps) = lr g / (|g| + eps / sqrt(1 - b2)) at step 1
    np.testing.assert_allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8 / np.sqrt(0.001)),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_histogram_brute_force():
    rng = np.random.default_rng(5)
    for p in (1, 7, 32, 100, 1000):
        pts = rng.integers(1, p + 1, size=(333, 2))
        counts = {}
        for x, y in pts.tolist():
            cell = int(math.floor((y - 1) * 32 / p)) * 32 + int(math.floor((x - 1) * 32 / p))
            counts[cell] = counts.get(cell, 0) + 1
        h = Lm.histogram(pts, p)
        scale = np.float32(1024) / np.float32(333)
        for c in range(1024):
            assert h[c] == np.float32(counts.get(c, 0)) * scale
        assert h.dtype == np.float32


def test_sample_index():
    np.testing.assert_array_equal(Lm.sample_index(1000), np.arange(1000))
    n = 10 ** 7 + 3
    s = Lm.sample_index(n)
    assert s.shape[0] == Lm.R_RUN * Lm.J_RUNS
    assert np.all(np.diff(s) > 0) and s[0] == 0 and s[-1] < n
    assert s[Lm.R_RUN] == n // Lm.J_RUNS


def test_extremes_brute_force():
    rng = np.random.default_rng(6)
    pts = rng.integers(1, 50, size=(400, 2)).astype(np.int32)
    idx = np.arange(0, 400, 3)
    ang = rng.uniform(0, 2 * np.pi, 12)
    c, s = np.cos(ang).astype(np.float32), np.sin(ang).astype(np.float32)
    c[0], s[0] = 1.0, 0.0  # axis direction: many ties
    got = Lm.extremes(pts, idx, c, s)
    for k in range(12):
        best, bi = None, None
        for i in idx.tolist():
            v = np.float32(np.float32(c[k]) * np.float32(pts[i, 0])) + np.float32(
                np.float32(s[k]) * np.float32(pts[i, 1]))
            if best is None or v > best:
                best, bi = v, i
        assert got[k] == bi
    assert pts[got[0], 0] == pts[idx, 0].max()


def _area2(H, sel):
    sel = sorted(set(sel))
    s = 0
    for a, b in zip(sel, sel[1:] + sel[:1]):
        s += int(H[a, 0]) * int(H[b, 1]) - int(H[a, 1]) * int(H[b, 0])
    return s


def _extreme(H, a):
    return int(np.argmax(np.cos(a) * H[:, 0] + np.sin(a) * H[:, 1]))


def test_best_offsets_coordinate_ascent_bounds():
    rng = np.random.default_rng(7)
    Kk, sub = 3, 5
    for t in range(20):
        pts = rng.integers(1, 200, size=(60, 2))
        H = oracle.hull_points(pts)
        if H.shape[0] < 3:
            continue
        got = oracle.best_offsets(H, K=Kk, sub=sub, rounds=3)
        offs = [-1 + 2 * j / (sub - 1) for j in range(sub)]
        ang = lambda k, o: 2 * np.pi * k / Kk + o * np.pi / Kk
        area = lambda os_: _area2(H, [_extreme(H, ang(k, o)) for k, o in enumerate(os_)])
        brute = max(area(c) for c in itertools.product(offs, repeat=Kk))
        a_got = area(got.tolist())
        assert area([0.0] * Kk) <= a_got <= brute
        assert np.all(np.abs(got) <= 1)


def test_label_batch_shapes_and_hull_sizes():
    rng = np.random.default_rng(8)
    sets = [rng.integers(1, p + 1, size=(n, 2)).astype(np.int32)
            for p, n in ((64, 500), (1024, 3000), (5, 40))]
    ps = [64, 1024, 5]
    off = np.concatenate([[0], np.cumsum([s.shape[0] for s in sets])])
    lab, hs = oracle.label_batch(np.concatenate(sets), off, ps)
    assert lab.shape == (3, 16) and np.all(np.abs(lab) <= 1)
    for s, p, h in zip(sets, ps, hs):
        assert h == oracle.hull(s, p).shape[0]
