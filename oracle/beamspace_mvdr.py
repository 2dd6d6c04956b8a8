"""FP64 oracle of windowed beamspace MVDR (test infrastructure only).

Section / equation names refer to the paper "Scaling Wideband Massive MIMO
Radar via Beamspace Dimension Reduction" (arXiv 2508.11790).  The array is
the linear (ULA) case of the paper's planar array: N_z = 1, elevation 0, so
the 2-D beamspace transform D = D_h^T (x) D_v of Eq. OverallDFT reduces to
one truncated M-point DFT and the selector S_k of Eq. OverallWindow to one
run of W consecutive beams.

Readings of points the paper leaves open (all stated once more in the
design notes of the repository):
* channeliser: critically sampled, rectangular, unitary F-point FFT of each
  record; FFT bin with signed index j belongs to subband s = (j + F/2) // B
  (B = F/L bins per subband), which is the subband l = s - L/2 + 1 whose
  centre is f(l) of Eq. SubChannelFreq; channelise first, beamspace second
  (the paper notes both orders are equal since both are linear);
* the FFT bin "corresponding to target k" is the beam nearest to the
  squinted spatial frequency x = Omega^(l) M / (2 pi) of Eq. SubOmegaX; the
  window is the W consecutive beams (mod M) whose centre is nearest to x,
  start = floor(x - W/2 + 1) mod M (ties round up);
* training vectors of a (target, subband) pair are the windowed beamspace
  vectors of the target-free training records, taken in record-major,
  bin-minor order; the first K of them enter Eq. EmpiricalCov;
* diagonal loading delta*I is added to the windowed covariance (the paper
  does not load; the workloads do, delta = 10 sigma^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "subband_center_freq",
    "squinted_omega",
    "steering_vector",
    "truncated_dft_matrix",
    "channelize",
    "beamspace",
    "window_start",
    "window_beams",
    "windowed_steering",
    "window_covariance",
    "mvdr_weights",
    "beamformer_output",
    "lifted_correlator",
    "lifted_output",
    "beam_pattern_grid",
    "beam_pattern",
    "output_sinr",
    "sinr_loss_db",
    "antenna_mvdr",
    "reference_covariances",
    "PairTable",
    "pair_table",
    "PipelineResult",
    "run_pipeline",
]


# --------------------------------------------------------------------------
# Sec. II-A: subbands, spatial frequencies, steering vectors
# --------------------------------------------------------------------------
def subband_center_freq(s: int, L: int, fc: float, fs: float) -> float:
    """Centre frequency of subband index s (Eq. SubChannelFreq).

    f(l) = f_c + ((l - 1/2) / L) f_s with l = -L/2 + 1, ..., L/2 and
    s = l + L/2 - 1 (s = 0 is the lowest subband).  Evaluated in exactly this
    order in float64.
    """
    ell = s - L // 2 + 1
    return fc + ((ell - 0.5) / L) * fs


def squinted_omega(u: float, f: float, fd: float) -> float:
    """Spatial frequency at subband frequency f (Eq. OmegaX, Eq. SubOmegaX).

    Omega^ref = pi cos(theta) sin(phi) with theta = 0 (linear array), u =
    sin(phi); Omega^(l) = Omega^ref * f(l) / f_d.
    """
    return math.pi * u * (f / fd)


def steering_vector(omega: float, N: int) -> np.ndarray:
    """a(Omega) = [1, e^{j Omega}, ..., e^{j Omega (N-1)}]^T (Eq. ArrayX)."""
    return np.exp(1j * omega * np.arange(N, dtype=np.float64))


def truncated_dft_matrix(M: int, N: int, rows=None) -> np.ndarray:
    """[D]_{m,n} = M^{-1/2} e^{-j 2 pi m n / M}, m < M, n < N (Eq. VerDFT).

    Zero-based indices; ``rows`` selects a subset of the M rows.
    """
    m = np.arange(M) if rows is None else np.asarray(rows)
    n = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(m, n) / M) / math.sqrt(M)


# --------------------------------------------------------------------------
# Sec. III-A: channelisation and beamspace transform
# --------------------------------------------------------------------------
def channelize(x: np.ndarray, L: int, subbands=None) -> np.ndarray:
    """FFT channeliser (Sec. III-A; L subbands as in Sec. IV-B).

    x[p, t, n]: records p, fast-time samples t < F, elements n.
    Returns Xc[p, s', i, n] = F^{-1/2} sum_t x[p, t, n] e^{-j 2 pi k t / F}
    for the bin k = j mod F with signed index j = (s - L/2) B + i, where s is
    the s'-th entry of ``subbands`` (all L subbands by default).

    With all subbands the numpy FFT gives every bin; with a subset the same
    sum is taken directly for just the bins of those subbands.
    """
    x = np.asarray(x, dtype=np.complex128)
    P, F, N = x.shape
    if F % L:
        raise ValueError("F must be a multiple of L")
    B = F // L
    sel = list(range(L)) if subbands is None else [int(s) for s in subbands]
    out = np.empty((P, len(sel), B, N), dtype=np.complex128)
    if subbands is None:
        X = np.fft.fft(x, axis=1) / math.sqrt(F)
        for si, s in enumerate(sel):
            for i in range(B):
                j = (s - L // 2) * B + i
                out[:, si, i, :] = X[:, j % F, :]
        return out
    t = np.arange(F)
    for si, s in enumerate(sel):
        k = np.array([((s - L // 2) * B + i) % F for i in range(B)])
        E = np.exp(-2j * np.pi * np.outer(k, t) / F) / math.sqrt(F)   # [B][F]
        out[:, si] = np.matmul(E[None], x)
    return out


def beamspace(y: np.ndarray, M: int) -> np.ndarray:
    """Beamspace vectors y_hat = D y (Eq. BeamTransform) along the last axis.

    D is the M x N truncated DFT of Eq. VerDFT; numpy's FFT of the vector
    zero-padded to M points, times M^{-1/2}, is that product.
    """
    y = np.asarray(y, dtype=np.complex128)
    if M < y.shape[-1]:
        raise ValueError("M must be >= N")
    return np.fft.fft(y, n=M, axis=-1) / math.sqrt(M)


# --------------------------------------------------------------------------
# Sec. III-B: window (selector S_k) and windowed steering vector
# --------------------------------------------------------------------------
def window_start(u: float, s: int, W: int, L: int, M: int,
                 fc: float, fs: float, fd: float) -> int:
    """First beam of the W-beam window of a target at subband index s.

    Eq. OverallWindow / Eq. ApplyWindow: the window is centred on the FFT bin
    of the target.  With x = Omega^(l) M / (2 pi) (Eq. SubOmegaX), the window
    is the W consecutive beams (circular in M) whose centre is nearest to x:
    start = floor(x - W/2 + 1) mod M.  The decision is taken in float64 in
    this order of operations.
    """
    f = subband_center_freq(s, L, fc, fs)
    omega = squinted_omega(u, f, fd)
    x = omega * M / (2.0 * math.pi)
    return int(math.floor(x - W / 2.0 + 1.0)) % M


def window_beams(start: int, W: int, M: int) -> np.ndarray:
    """Beams selected by S_k: start, start+1, ..., start+W-1 (mod M)."""
    return (start + np.arange(W)) % M


def windowed_steering(omega: float, N: int, M: int, beams) -> np.ndarray:
    """a_tilde = S D a(Omega) (Sec. III-C, below Eq. BeamCorrMVDR).

    Direct product of the selected rows of D (Eq. VerDFT) with a (Eq. ArrayX).
    """
    return truncated_dft_matrix(M, N, rows=beams) @ steering_vector(omega, N)


# --------------------------------------------------------------------------
# Sec. II-B / III-C: covariance, MVDR correlator, output
# --------------------------------------------------------------------------
def window_covariance(z: np.ndarray, delta: float) -> np.ndarray:
    """R_tilde = (1/K) sum_k z_k z_k^H + delta I (Eq. EmpiricalCov on the
    windowed vectors of Eq. ApplyWindow, plus diagonal loading).

    z[k, w]: K training vectors of length W.  sum_k z_k z_k^H is z^T conj(z).
    """
    z = np.asarray(z, dtype=np.complex128)
    K, W = z.shape
    if K < 1:
        raise ValueError("need at least one training vector")
    return (z.T @ z.conj()) / K + delta * np.eye(W)


def mvdr_weights(R: np.ndarray, a: np.ndarray) -> np.ndarray:
    """c = R^{-1} a / (a^H R^{-1} a) (Eq. CorrMVDR, Eq. BeamCorrMVDR)."""
    Ria = np.linalg.solve(np.asarray(R, np.complex128), np.asarray(a, np.complex128))
    return Ria / (np.conj(a) @ Ria)


def beamformer_output(c: np.ndarray, y: np.ndarray) -> np.ndarray:
    """c^H y[n] for every vector y[n] = y[n, :] (Sec. II-B)."""
    return np.asarray(y, np.complex128) @ np.conj(c)


def lifted_correlator(c_tilde: np.ndarray, N: int, M: int, beams) -> np.ndarray:
    """c_hat = D^H S^T c_tilde (Eq. AntennaEqCorr)."""
    Dw = truncated_dft_matrix(M, N, rows=beams)          # S D, W x N
    return Dw.conj().T @ np.asarray(c_tilde, np.complex128)


def beam_pattern(c: np.ndarray, a: np.ndarray) -> float:
    """|<c, a>| / (||c|| ||a||) (Eq. Cosine Sim), <c, a> = c^H a."""
    return float(abs(np.vdot(c, a)) / (np.linalg.norm(c) * np.linalg.norm(a)))


def lifted_output(c_hat: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Output of the lifted correlator applied in antenna space (Sec. III-C,
    below Eq. AntennaEqCorr): c_hat^H y for each row y of the channelised
    antenna-domain snapshots, without the spatial FFT and window."""
    return np.asarray(y, np.complex128) @ np.conj(np.asarray(c_hat, np.complex128))


def beam_pattern_grid(c_hat: np.ndarray, u, f: float, fd: float) -> np.ndarray:
    """Eq. Cosine Sim of c_hat against the steering vector of every direction
    sine in u at frequency f (squinted spatial frequency, Eq. SubOmegaX)."""
    N = len(c_hat)
    return np.array([beam_pattern(c_hat, steering_vector(squinted_omega(float(uk), f, fd), N)) for uk in u])


def output_sinr(c: np.ndarray, a: np.ndarray, R_in: np.ndarray) -> float:
    """Output SINR of correlator c for a unit-power signal with response a
    against interference-plus-noise covariance R_in: |c^H a|^2 / (c^H R_in c)."""
    num = abs(np.vdot(c, a)) ** 2
    den = float(np.real(np.vdot(c, R_in @ c)))
    return num / den


def sinr_loss_db(c: np.ndarray, c_ref: np.ndarray, a: np.ndarray,
                 R_in: np.ndarray) -> float:
    """10 log10(SINR(c_ref) / SINR(c)) against the same R_in."""
    return 10.0 * math.log10(output_sinr(c_ref, a, R_in) / output_sinr(c, a, R_in))


def antenna_mvdr(y: np.ndarray, a: np.ndarray, delta: float) -> np.ndarray:
    """Full-dimensional MVDR (Sec. II-B): R_hat = (1/n_t) sum y y^H + delta I
    (Eq. EmpiricalCov plus loading) and c = R_hat^{-1} a / (a^H R_hat^{-1} a)."""
    return mvdr_weights(window_covariance(y, delta), a)


# --------------------------------------------------------------------------
# Whole path over (target, subband) pairs
# --------------------------------------------------------------------------
@dataclass
class PairTable:
    """Per (target, subband) pair g = t * L + s: window and steering."""

    t: np.ndarray
    s: np.ndarray
    start: np.ndarray
    W: np.ndarray
    K: np.ndarray
    a_tilde: list = field(default_factory=list)


def pair_table(cfg, u, subbands=None, targets=None) -> PairTable:
    """Window starts and windowed steering vectors of the selected pairs.

    ``cfg`` carries N, F, L, M, T, W[t], K[t], fc, fs, fd; ``u[t]`` is the
    direction sine of target t.
    """
    L = cfg.L
    subs = list(range(L)) if subbands is None else [int(s) for s in subbands]
    tgts = list(range(cfg.T)) if targets is None else [int(t) for t in targets]
    ts, ss, st, Ws, Ks, at = [], [], [], [], [], []
    for t in tgts:
        for s in subs:
            W = int(cfg.W[t])
            start = window_start(float(u[t]), s, W, L, cfg.M, cfg.fc, cfg.fs, cfg.fd)
            omega = squinted_omega(float(u[t]),
                                   subband_center_freq(s, L, cfg.fc, cfg.fs), cfg.fd)
            ts.append(t); ss.append(s); st.append(start); Ws.append(W)
            Ks.append(int(cfg.K[t]))
            at.append(windowed_steering(omega, cfg.N, cfg.M, window_beams(start, W, cfg.M)))
    return PairTable(np.array(ts), np.array(ss), np.array(st), np.array(Ws),
                     np.array(Ks), at)


@dataclass
class PipelineResult:
    pairs: PairTable
    z_train: list          # per pair [K][W]
    z_test: list           # per pair [P_te*B][W]
    R: list                # per pair [W][W]
    c: list                # per pair [W]
    out: list              # per pair [P_te*B]


def run_pipeline(x: np.ndarray, cfg, u, subbands=None, targets=None,
                 delta=None) -> PipelineResult:
    """Channelise -> beamspace -> window -> loaded covariance -> MVDR -> apply.

    x[p, t, n] holds cfg.P_tr training records followed by cfg.P_te test
    records.  ``delta`` overrides cfg.delta; it may be a callable of the pair
    index in the returned table.
    """
    L, B, M = cfg.L, cfg.F // cfg.L, cfg.M
    subs = list(range(L)) if subbands is None else [int(s) for s in subbands]
    tab = pair_table(cfg, u, subs, targets)
    xc = channelize(x, L, subs if subbands is not None else None)  # [P][S][B][N]
    yb = beamspace(xc, M)                                          # [P][S][B][M]
    P = x.shape[0]
    zt, ze, Rs, cs, outs = [], [], [], [], []
    for gi in range(len(tab.t)):
        si = subs.index(int(tab.s[gi]))
        beams = window_beams(int(tab.start[gi]), int(tab.W[gi]), M)
        z_all = yb[:, si][:, :, beams].reshape(P * B, -1)   # record-major, bin-minor
        K = int(tab.K[gi])
        z_tr = z_all[:K]
        z_te = z_all[cfg.P_tr * B:]
        d = cfg.delta if delta is None else (delta(gi) if callable(delta) else delta)
        R = window_covariance(z_tr, d)
        c = mvdr_weights(R, tab.a_tilde[gi])
        zt.append(z_tr); ze.append(z_te); Rs.append(R); cs.append(c)
        outs.append(beamformer_output(c, z_te))
    return PipelineResult(tab, zt, ze, Rs, cs, outs)


def reference_covariances(x_ref: np.ndarray, cfg, u, subbands=None, targets=None) -> list:
    """Interference-plus-noise covariance of every selected pair, estimated
    from target-free records x_ref[p, t, n] that the weights never saw:
    R_ref = (1/K_ref) sum z z^H over all K_ref = P_ref B windowed vectors of
    the pair (Eq. EmpiricalCov, no loading), in the order of pair_table.
    Output SINR judged against R_ref measures how well a correlator
    suppresses the scene's interference, not how well it fits its own
    training sample."""
    L, B, M = cfg.L, cfg.F // cfg.L, cfg.M
    subs = list(range(L)) if subbands is None else [int(s) for s in subbands]
    tab = pair_table(cfg, u, subs, targets)
    yb = beamspace(channelize(x_ref, L, subs if subbands is not None else None), M)   # [P][S][B][M]
    P = yb.shape[0]
    out = []
    for gi in range(len(tab.t)):
        si = subs.index(int(tab.s[gi]))
        beams = window_beams(int(tab.start[gi]), int(tab.W[gi]), M)
        z = yb[:, si][:, :, beams].reshape(P * B, -1)
        out.append(window_covariance(z, 0.0))
    return out
