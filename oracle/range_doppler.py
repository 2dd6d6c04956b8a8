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
* CFAR: the noise floor of a target's map is its mean over all cells; a cell
  is a detection when it exceeds the floor by the threshold (10 dB).
"""
from __future__ import annotations

import numpy as np

__all__ = ["beamformed_spectrum", "range_profiles", "doppler_map", "cfar_detect"]


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
    """(mask, floor): cells of each target's map above its mean times
    10^(threshold_db / 10)."""
    floor = m.mean(axis=(1, 2))
    return m > floor[:, None, None] * 10.0 ** (threshold_db / 10.0), floor
