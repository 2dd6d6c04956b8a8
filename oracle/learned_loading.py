"""FP64 oracle of the learned diagonal loading (test infrastructure only).

The paper loads nothing and learns nothing; this part follows the workload's
"learned loading" direction: from a window covariance estimated with few
training vectors (K = 2W), a small MLP predicts the diagonal loading delta
and a diagonal preconditioner d for the MVDR solve (Eq. BeamCorrMVDR).
Definitions (restated in the design notes):

* features of one window (W entries, K training vectors, unloaded sample
  covariance R of Eq. EmpiricalCov, windowed steering vector a):
  tau = tr(R) / W;  [diag(R)/tau (W), Re R_ij/tau (i > j, row-major),
  Im R_ij/tau (i > j), Re a/|a| (W), Im a/|a| (W), log10 tau, log10(K/W)]
  -> W^2 + 2W + 2 values;
* label: delta* = the grid value maximising the output SINR
  |c^H a|^2 / (c^H R_ref c) of c = mvdr(R + delta I, a), judged against a
  reference covariance R_ref of the same window from many more training
  vectors; targets [log10 delta*, log10 d*_i] with
  d*_i = (R_ii + delta*)^(-1/2);
* network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (3 layers);
* loss: mean squared error over batch and outputs;
* optimiser: Adam (Kingma and Ba, 2015), bias-corrected;
* preconditioner: with D = diag(d), d > 0, the correlator is solved as
  (D R D) y = D a, c = D y / (a^H D y) -- the same c as Eq. BeamCorrMVDR in
  exact arithmetic (R^-1 a = D (D R D)^-1 D a), with a better-scaled
  matrix for the finite-precision Cholesky when d equilibrates R.
"""
from __future__ import annotations

import numpy as np

from .beamspace_mvdr import mvdr_weights, output_sinr

__all__ = [
    "LOADING_GRID",
    "window_features",
    "optimal_loading",
    "loading_targets",
    "mlp_init",
    "mlp_forward",
    "mlp_loss",
    "mlp_backward",
    "adam_step",
    "mvdr_weights_preconditioned",
]

# 61 log-spaced loading values from 1e-1 to 1e4 (noise variance units)
LOADING_GRID = 10.0 ** np.linspace(-1.0, 4.0, 61)


def window_features(R: np.ndarray, a: np.ndarray, K: int) -> np.ndarray:
    """Feature vector of one window from its unloaded sample covariance."""
    R = np.asarray(R, np.complex128)
    a = np.asarray(a, np.complex128)
    W = R.shape[0]
    tau = float(np.real(np.trace(R))) / W
    il, jl = np.tril_indices(W, -1)
    an = a / np.linalg.norm(a)
    return np.concatenate([
        np.real(np.diag(R)) / tau,
        np.real(R[il, jl]) / tau,
        np.imag(R[il, jl]) / tau,
        np.real(an), np.imag(an),
        [np.log10(tau), np.log10(K / W)],
    ])


def optimal_loading(R: np.ndarray, a: np.ndarray, R_ref: np.ndarray, grid=LOADING_GRID):
    """(delta*, SINR per grid value) for the window: argmax over the grid of
    the output SINR of mvdr(R + delta I, a) judged against R_ref (first
    maximum on ties)."""
    W = R.shape[0]
    s = np.array([output_sinr(mvdr_weights(R + d * np.eye(W), a), a, R_ref) for d in grid])
    return float(grid[int(np.argmax(s))]), s


def loading_targets(R: np.ndarray, delta: float) -> np.ndarray:
    """[log10 delta, log10 d_i], d_i = (R_ii + delta)^(-1/2)."""
    d = (np.real(np.diag(R)) + delta) ** -0.5
    return np.concatenate([[np.log10(delta)], np.log10(d)])


def mlp_init(n_in: int, n_hidden: int, n_out: int, seed: int) -> dict:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    g = np.random.default_rng(seed)

    def lin(fo, fi):
        b = np.sqrt(6.0 / fi)
        return g.uniform(-b, b, size=(fo, fi))

    return {"W1": lin(n_hidden, n_in), "b1": np.zeros(n_hidden),
            "W2": lin(n_hidden, n_hidden), "b2": np.zeros(n_hidden),
            "W3": lin(n_out, n_hidden), "b3": np.zeros(n_out)}


def mlp_forward(p: dict, X: np.ndarray):
    """Returns (Y, cache); X is [batch][n_in]."""
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def mlp_loss(Y: np.ndarray, T: np.ndarray) -> float:
    """Mean squared error over batch and outputs."""
    return float(np.mean((Y - T) ** 2))


def mlp_backward(p: dict, cache, Y: np.ndarray, T: np.ndarray) -> dict:
    """Gradients of mlp_loss with respect to every parameter (chain rule)."""
    X, Z1, H1, Z2, H2 = cache
    dY = 2.0 * (Y - T) / Y.size
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dH2 = dY @ p["W3"]
    dZ2 = dH2 * (Z2 > 0)
    g["W2"], g["b2"] = dZ2.T @ H1, dZ2.sum(0)
    dH1 = dZ2 @ p["W2"]
    dZ1 = dH1 * (Z1 > 0)
    g["W1"], g["b1"] = dZ1.T @ X, dZ1.sum(0)
    return g


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place (t counts from 1)."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def mvdr_weights_preconditioned(R: np.ndarray, a: np.ndarray, d: np.ndarray) -> np.ndarray:
    """MVDR correlator through the diagonally scaled system: solve
    (D R D) y = D a with D = diag(d), then c = D y / (a^H D y)."""
    R = np.asarray(R, np.complex128)
    a = np.asarray(a, np.complex128)
    d = np.asarray(d, np.float64)
    if np.any(~(d > 0)):
        raise ValueError("the preconditioner must be positive")
    y = np.linalg.solve(d[:, None] * R * d[None, :], d * a)
    v = d * y
    return v / (np.conj(a) @ v)
