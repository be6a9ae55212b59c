"""The network's CUDA kernels (forward, loss, backward, Adam) against the
float64 oracle of oracle/learned.py.

Tolerances come from the arithmetic: a GEMM multiplies bf16-rounded operands
exactly in float32 and accumulates K products in float32, so its error is at
most gamma_K = K * 2^-23 times sum |a| |b| (rounding of every partial sum,
with room for the tensor core's accumulation order).  Each layer is checked
from the GPU's own inputs, so the oracle rounds the same float32 values to
bf16.  Where an intermediate that the GPU keeps in float32 is rounded to bf16
inside the backward pass, a one-ulp difference of that rounding (2^-8
relative) is allowed on top."""
import numpy as np
import pytest
import torch

from oracle import learned as Lm
from paper_1505_00914_gb300 import ch
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()
    yield
    assert ch.ch_sync_status() == ch.CH_OK


def _gamma(K):
    return K * 2.0 ** -23


def _problem(seed, M):
    rng = np.random.default_rng(seed)
    params = Lm.init_params(seed)
    w = Lm.unpack(params)
    w["b1"][:] = rng.normal(0, 0.1, Lm.HID).astype(np.float32)
    w["b2"][:] = rng.normal(0, 0.1, Lm.HID).astype(np.float32)
    w["b3"][:] = rng.normal(0, 0.1, Lm.K).astype(np.float32)
    X = rng.gamma(0.7, 1.5, size=(M, Lm.IN)).astype(np.float32)
    X[:, rng.random(Lm.IN) < 0.2] = 0.0
    T = rng.uniform(-1, 1, size=(M, Lm.K)).astype(np.float32)
    return params.astype(np.float32), X, T


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


def _bound(A, B, K):
    return _gamma(K) * (np.abs(Lm.bf16(A)) @ np.abs(Lm.bf16(B)))


@pytest.mark.parametrize("M", [1, 63, 200])
def test_forward_layers(M):
    params, X, _ = _problem(M, M)
    w = Lm.unpack(params.astype(np.float64))
    H1, H2, Y = ch.ch_mlp_forward(_cuda(params), _cuda(X))
    H1, H2, Y = _np(H1), _np(H2), _np(Y)
    ref1 = np.maximum(Lm.bf16(X) @ Lm.bf16(w["W1"]) + w["b1"], 0)
    assert np.all(np.abs(H1 - ref1) <= _bound(X, w["W1"], Lm.IN) + 1e-6)
    ref2 = np.maximum(Lm.bf16(H1) @ Lm.bf16(w["W2"]) + w["b2"], 0)
    assert np.all(np.abs(H2 - ref2) <= _bound(H1, w["W2"], Lm.HID) + 1e-6)
    ref3 = Lm.bf16(H2) @ Lm.bf16(w["W3"]) + w["b3"]
    assert np.all(np.abs(Y - ref3) <= _bound(H2, w["W3"], Lm.HID) + 1e-6)
    # whole pass from X alone: bf16 roundings of the hidden layers may differ
    # by one ulp, so only closeness is asked for
    Yo = Lm.forward(params, X)[2]
    assert np.max(np.abs(Y - Yo)) <= 2.0 ** -6 * (np.max(np.abs(Yo)) + 1)
    assert ref1.shape == (M, Lm.HID) and Y.shape == (M, Lm.K)


def test_loss_and_gradient_of_loss():
    params, X, T = _problem(7, 100)
    _, _, Y = ch.ch_mlp_forward(_cuda(params), _cuda(X))
    loss, dY = ch.ch_mlp_loss(Y, _cuda(T))
    lo, dYo = Lm.loss(_np(Y), T)
    assert abs(float(_np(loss)[0]) - lo) <= 1e-5 * lo + 1e-7
    np.testing.assert_allclose(_np(dY), dYo, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("M", [1, 130])
def test_backward_against_oracle(M):
    params, X, T = _problem(11 + M, M)
    dp, dX = _cuda(params), _cuda(X)
    H1, H2, Y = ch.ch_mlp_forward(dp, dX)
    _, dY = ch.ch_mlp_loss(Y, _cuda(T))
    g = _np(ch.ch_mlp_backward(dp, dX, H1, H2, dY))
    H1n, H2n, dYn = _np(H1), _np(H2), _np(dY)
    ref = Lm.backward(params, X, H1n, H2n, dYn)
    G, R = Lm.unpack(g), Lm.unpack(ref)
    w = Lm.unpack(params.astype(np.float64))
    # output layer: direct products of GPU tensors
    assert np.all(np.abs(G["W3"] - R["W3"]) <= _bound(H2n.T, dYn, M) + 1e-12)
    assert np.all(np.abs(G["b3"] - R["b3"]) <= _gamma(M) * np.abs(dYn).sum(0) + 1e-12)
    # hidden layers: dH2, dH1 are float32 on the GPU and rounded to bf16 as
    # operands of the next product
    dH2 = (Lm.bf16(dYn) @ Lm.bf16(w["W3"]).T) * (H2n > 0)
    dH1 = (Lm.bf16(dH2) @ Lm.bf16(w["W2"]).T) * (H1n > 0)
    for name, A, B, K in (("W2", H1n.T, dH2, M), ("W1", X.T.astype(np.float64), dH1, M)):
        tol = (2.0 ** -7 + _gamma(K)) * (np.abs(Lm.bf16(A)) @ np.abs(B)) + 1e-12
        assert np.all(np.abs(G[name] - R[name]) <= tol), name
    for name, D, K in (("b2", dH2, M), ("b1", dH1, M)):
        tol = (2.0 ** -7 + _gamma(K)) * np.abs(D).sum(0) + 1e-12
        assert np.all(np.abs(G[name] - R[name]) <= tol), name
    # and close to the exact (float64, unrounded) gradient
    exact = Lm.backward(params, X, *Lm.forward(params, X, exact=True)[:2],
                        Lm.loss(Lm.forward(params, X, exact=True)[2], T)[1], exact=True)
    assert np.linalg.norm(g - exact) <= 0.05 * np.linalg.norm(exact)


def test_adam_step():
    """Hyper-parameters cross the C ABI as float32, so the oracle gets the
    float32 values; the bounds are a few float32 roundings of each term."""
    rng = np.random.default_rng(3)
    n = ch.CH_MLP_PARAMS
    p0 = rng.normal(0, 1, n).astype(np.float32)
    g = rng.normal(0, 1e-2, n).astype(np.float32)
    m0 = rng.normal(0, 1e-3, n).astype(np.float32)
    v0 = np.abs(rng.normal(0, 1e-4, n)).astype(np.float32)
    dp, dg, dm, dv = map(_cuda, (p0, g, m0, v0))
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1e-3, 0.9, 0.999, 1e-8))
    ch.ch_mlp_adam(dp, dg, dm, dv, 5, lr, b1, b2, eps)
    pr, mr, vr = Lm.adam(p0.astype(np.float64), g, m0, v0, 5, lr, b1, b2, eps)
    u = 2.0 ** -24
    m_gpu, v_gpu, p_gpu = _np(dm), _np(dv), _np(dp)
    assert np.all(np.abs(m_gpu - mr) <= 4 * u * (b1 * np.abs(m0) + (1 - b1) * np.abs(g)))
    assert np.all(np.abs(v_gpu - vr) <= 4 * u * (b2 * v0 + (1 - b2) * g.astype(np.float64) ** 2))
    step = np.abs(pr - p0)
    assert np.all(np.abs(p_gpu - pr) <= 2 * u * np.abs(p0) + 1e-5 * step + 1e-12)


def test_training_reduces_loss():
    """A few hundred Adam steps on a fixed batch drive the loss down."""
    params, X, _ = _problem(21, 256)
    rng = np.random.default_rng(22)
    # targets that depend on the input: tanh of a random projection
    T = np.tanh(X @ rng.normal(0, 0.05, (Lm.IN, Lm.K))).astype(np.float32)
    dp, dX, dT = _cuda(params), _cuda(X), _cuda(T)
    m, v = torch.zeros_like(dp), torch.zeros_like(dp)
    losses = []
    for step in range(1, 301):
        H1, H2, Y = ch.ch_mlp_forward(dp, dX)
        loss, dY = ch.ch_mlp_loss(Y, dT)
        grads = ch.ch_mlp_backward(dp, dX, H1, H2, dY)
        ch.ch_mlp_adam(dp, grads, m, v, step, 1e-3)
        if step in (1, 300):
            losses.append(float(_np(loss)[0]))
    assert losses[1] < 0.2 * losses[0]
