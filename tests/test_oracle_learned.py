"""Pins of the learned-loading oracle (CPU): hand-worked features, finite-
difference gradients, the closed-form first Adam step, and the two limits of
the SINR-optimal loading."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import learned_loading as LL

RNG = np.random.default_rng(77)


def crandn(*s):
    return (RNG.standard_normal(s) + 1j * RNG.standard_normal(s)) / math.sqrt(2)


def test_features_golden(golden):
    vals = [float(l) for l in open(golden("features_W2.txt")) if l.strip() and not l.startswith("#")]
    R = np.array([[2, 1 - 1j], [1 + 1j, 4]])
    f = LL.window_features(R, np.array([1, 1j]), K=6)
    np.testing.assert_allclose(f, vals, atol=1e-15)


def test_mlp_forward_golden(golden):
    """Hand-worked forward pass of a 2-2-2-1 network (ReLU between layers)."""
    rows = np.array([[float(v) for v in l.split()] for l in open(golden("mlp_2221.txt"))
                     if l.strip() and not l.startswith("#")])
    p = {"W1": np.array([[1.0, -1.0], [0.5, 2.0]]), "b1": np.array([0.0, -1.0]),
         "W2": np.array([[1.0, 1.0], [-1.0, 0.5]]), "b2": np.array([0.5, 0.0]),
         "W3": np.array([[2.0, -1.0]]), "b3": np.array([0.25])}
    Y, _ = LL.mlp_forward(p, rows[:, :2])
    np.testing.assert_allclose(Y[:, 0], rows[:, 2], atol=1e-15)


def test_features_scale_invariance():
    W, K = 9, 18
    Z = crandn(K, W)
    R = O.window_covariance(Z, 0.0)
    a = crandn(W)
    f1 = LL.window_features(R, a, K)
    f2 = LL.window_features(37.0 * R, 5.0 * a, K)
    assert f1.size == W * W + 2 * W + 2
    np.testing.assert_allclose(f2[:-2], f1[:-2], atol=1e-12)
    assert f2[-2] == pytest.approx(f1[-2] + math.log10(37.0))


def test_gradients_finite_differences():
    p = LL.mlp_init(7, 5, 3, seed=1)
    for k in p:                         # non-zero biases so every term is exercised
        if k.startswith("b"):
            p[k] = RNG.standard_normal(p[k].shape) * 0.1
    X = RNG.standard_normal((4, 7))
    T = RNG.standard_normal((4, 3))
    Y, cache = LL.mlp_forward(p, X)
    g = LL.mlp_backward(p, cache, Y, T)
    h = 1e-6
    for k in p:
        it = np.nditer(p[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[k][idx]
            p[k][idx] = old + h
            lp = LL.mlp_loss(LL.mlp_forward(p, X)[0], T)
            p[k][idx] = old - h
            lm = LL.mlp_loss(LL.mlp_forward(p, X)[0], T)
            p[k][idx] = old
            assert g[k][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9), (k, idx)


def test_adam_first_step_is_signed_lr():
    """At t = 1 the bias-corrected moments are g and g^2, so each parameter
    moves by -lr g / (|g| + eps)."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    LL.adam_step(p, g, m, v, t=1, lr=0.1)
    gw = np.array([0.5, -4.0, 1e-3])
    np.testing.assert_allclose(p["w"], np.array([1.0, -2.0, 3.0]) - 0.1 * gw / (np.abs(gw) + 1e-8), rtol=1e-13)


def test_optimal_loading_limits():
    W = 6
    a = np.exp(1j * 0.3 * np.arange(W))
    # judged against the covariance it was estimated from: no loading is best
    Q, _ = np.linalg.qr(crandn(W, W))
    R = (Q * np.array([1, 3, 10, 30, 100, 300.0])) @ Q.conj().T
    d, s = LL.optimal_loading(R, a, R)
    assert d == LL.LOADING_GRID[0] and np.argmax(s) == 0
    # white-noise truth, noisy estimate: the largest loading (matched filter) is best
    Rhat = O.window_covariance(crandn(W + 1, W) * 3.0, 0.0)
    d2, s2 = LL.optimal_loading(Rhat, a, np.eye(W))
    assert d2 == LL.LOADING_GRID[-1]


def test_loading_targets():
    R = np.diag([1.0, 3.0]).astype(complex)
    t = LL.loading_targets(R, 1.0)
    np.testing.assert_allclose(t, [0.0, math.log10(2 ** -0.5), math.log10(4 ** -0.5)], atol=1e-15)


def test_preconditioned_mvdr_is_invariant_and_equilibrates():
    """The scaled solve gives the plain MVDR correlator for any positive d
    (exact-arithmetic invariance, to FP64 rounding); d = 1 is the plain
    solve; Jacobi scaling d = diag(R)^-1/2 gives a unit diagonal and, for a
    badly scaled R, a far smaller condition number."""
    W = 9
    Z = crandn(40, W) * np.logspace(0, 3, W)[None, :]      # columns 1 .. 1000 in scale
    R = O.window_covariance(Z, 0.5)
    a = crandn(W)
    c = O.mvdr_weights(R, a)
    for d in (np.ones(W), np.exp(RNG.standard_normal(W)), 2.0 ** RNG.integers(-9, 9, size=W)):
        np.testing.assert_allclose(LL.mvdr_weights_preconditioned(R, a, d), c, rtol=0, atol=1e-9 * np.abs(c).max())
    dj = np.real(np.diag(R)) ** -0.5
    Rs = dj[:, None] * R * dj[None, :]
    np.testing.assert_allclose(np.real(np.diag(Rs)), 1.0, atol=1e-14)
    assert np.linalg.cond(Rs) < 1e-3 * np.linalg.cond(R)
    with pytest.raises(ValueError):
        LL.mvdr_weights_preconditioned(R, a, -np.ones(W))
