"""FP64 oracle of the processing after the beamformer (test infrastructure
only): synthesis of each target's wideband output from its subband outputs,
range compression, Doppler processing and CFAR detection.

The paper hands the beamformed subbands to a synthesis IFFT and to standard
range-Doppler processing (Sec. II, Fig. 1) and declares detections 10 dB
above the noise floor (Sec. IV).  Readings taken here:

* the beamformed output of pair (t, s) at test vector v' = r B + i is the
  value of bin q = s B + i of test record r, i.e. of FFT bin
  k = (q - F/2) mod F (the channeliser's signed-frequency order);
* range compression is the matched filter of the transmitted pulse, applied
  in the frequency domain before the synthesis IFFT (orthonormal scaling):
  rp[t][r][tau] = IFFT_k(Y[t][r][k] conj(P[k]))[tau];
* Doppler is the unnormalised DFT over the test records:
  map[t][d][tau] = |sum_r rp[t][r][tau] e^{-j 2 pi d r / P_te}|^2;
* CFAR: a one-dimensional CFAR across the velocity bins of the map
  (Sec. IV-B): the noise floor of cell (d, tau) is the mean of the other
  P_te - 1 velocity bins of the same range cell tau (cell averaging with the
  cell under test left out; with it included, a target alone in its range
  cell could never clear 10 dB once P_te <= 10); a cell is a detection when
  it exceeds its floor by the threshold (10 dB).  Needs P_te >= 2;
* detection accuracy (Sec. IV-B: range and velocity error): a target's
  detection is its strongest detected cell; its range error is the signed
  difference of range bins and its velocity error the signed difference of
  velocity bins taken modulo P_te into [-P_te/2, P_te/2); a target with no
  detected cell is missed.
"""
from __future__ import annotations

import numpy as np

__all__ = ["beamformed_spectrum", "range_profiles", "doppler_map", "cfar_detect", "detection_errors"]


def beamformed_spectrum(out: np.ndarray, T: int, L: int, B: int, P_te: int) -> np.ndarray:
    """Y[t][r][k] (complex128, FFT order) from the pair outputs out[g][v'],
    g = t L + s, v' = r B + i."""
    F = L * B
    out = np.asarray(out, np.complex128).reshape(T, L, P_te, B)
    Y = np.empty((T, P_te, F), np.complex128)
    for s in range(L):
        for i in range(B):
            k = (s * B + i - F // 2) % F
            Y[:, :, k] = out[:, s, :, i]
    return Y


def range_profiles(Y: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Matched filter and synthesis IFFT: IFFT_k(Y conj(P)), orthonormal."""
    return np.fft.ifft(Y * np.conj(np.asarray(P, np.complex128)), axis=-1, norm="ortho")


def doppler_map(rp: np.ndarray) -> np.ndarray:
    """|DFT over the records|^2 of the range profiles: [t][d][tau]."""
    return np.abs(np.fft.fft(rp, axis=1)) ** 2


def cfar_detect(m: np.ndarray, threshold_db: float = 10.0):
    """(mask, floor), both [t][d][tau]: floor = mean of the other velocity
    bins of the same range cell, mask = m > floor * 10^(threshold_db / 10)."""
    m = np.asarray(m, np.float64)
    Pd = m.shape[1]
    if Pd < 2:
        raise ValueError("a CFAR across velocity bins needs at least two bins")
    floor = np.empty_like(m)
    for d in range(Pd):
        others = [e for e in range(Pd) if e != d]
        floor[:, d, :] = m[:, others, :].sum(axis=1) / (Pd - 1)
    return m > floor * 10.0 ** (threshold_db / 10.0), floor


def detection_errors(mask: np.ndarray, m: np.ndarray, delay, doppler):
    """Per target: (detected, peak cell (d, tau), range error, velocity
    error).  The peak is the strongest detected cell (the first in
    (d, tau) order on ties); errors are None for a missed target."""
    T, Pd, _ = m.shape
    out = []
    for t in range(T):
        if not mask[t].any():
            out.append((False, None, None, None))
            continue
        masked = np.where(mask[t], m[t], -np.inf)
        d, tau = np.unravel_index(int(np.argmax(masked)), masked.shape)
        dv = (int(d) - int(doppler[t]) + Pd // 2) % Pd - Pd // 2
        out.append((True, (int(d), int(tau)), int(tau) - int(delay[t]), dv))
    return out
