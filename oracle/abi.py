"""The oracle behind the five calls of the C boundary (test infrastructure
only), one function per call with the ``oracle_`` prefix, on host FP64
arrays and per-pair lists:

    bs_channelize  -> oracle_channelize   (Sec. II-A, Eq. SubChannelFreq)
    bs_beamspace   -> oracle_beamspace    (Eq. VerDFT, Eq. BeamTransform,
                                           Eq. OverallWindow, Eq. ApplyWindow)
    bs_window_cov  -> oracle_window_cov   (Eq. EmpiricalCov plus loading)
    bs_mvdr_solve  -> oracle_mvdr_solve   (Eq. CorrMVDR, Eq. BeamCorrMVDR)
    bs_apply       -> oracle_apply        (Sec. II-B)

Pairs are ordered g = t L + s as in the library; each function delegates to
the step of ``beamspace_mvdr`` that defines it, so composing the five gives
``run_pipeline`` exactly.
"""
from __future__ import annotations

import numpy as np

from .beamspace_mvdr import (beamformer_output, beamspace, channelize, mvdr_weights, pair_table, window_beams,
                             window_covariance)

__all__ = ["oracle_channelize", "oracle_beamspace", "oracle_window_cov", "oracle_mvdr_solve", "oracle_apply",
           "oracle_pairs"]


def oracle_pairs(cfg, u):
    """The plan's pair table: window start, W, K and windowed steering vector
    of every pair g = t L + s (Eq. OverallWindow, Eq. SubOmegaX)."""
    return pair_table(cfg, u)


def oracle_channelize(x: np.ndarray, L: int) -> np.ndarray:
    """x[P][F][N] -> xc[P][F][N] with bin q = s B + i of subband s (the
    library's layout of bs_channelize's output)."""
    xc = channelize(np.asarray(x, np.complex128), L)   # [P][L][B][N]
    return xc.reshape(xc.shape[0], -1, xc.shape[-1])


def oracle_beamspace(xc: np.ndarray, cfg, pairs) -> tuple[list, list]:
    """Windows of every pair from the channelised cube: per pair the first K
    training vectors [K][W] (record-major, then bin) and the P_te B test
    vectors [P_te B][W], as bs_beamspace packs them."""
    P, F, N = xc.shape
    L, B, M = cfg.L, F // cfg.L, cfg.M
    yb = beamspace(np.asarray(xc, np.complex128).reshape(P, L, B, N), M)   # [P][L][B][M]
    z_train, z_test = [], []
    for g in range(len(pairs.t)):
        beams = window_beams(int(pairs.start[g]), int(pairs.W[g]), M)
        z_all = yb[:, int(pairs.s[g])][:, :, beams].reshape(P * B, -1)
        z_train.append(z_all[:int(pairs.K[g])])
        z_test.append(z_all[cfg.P_tr * B:])
    return z_train, z_test


def oracle_window_cov(z_train: list, delta) -> list:
    """Loaded covariance of every pair; ``delta`` is the plan's loading or a
    per-pair sequence (bs_window_cov's delta_pair)."""
    d = [delta] * len(z_train) if np.isscalar(delta) else list(delta)
    return [window_covariance(z, float(dg)) for z, dg in zip(z_train, d)]


def oracle_mvdr_solve(R: list, a_tilde: list) -> list:
    """MVDR weights of every pair."""
    return [mvdr_weights(Rg, ag) for Rg, ag in zip(R, a_tilde)]


def oracle_apply(c: list, z_test: list) -> list:
    """Beamformer output of every pair on its test vectors."""
    return [beamformer_output(cg, zg) for cg, zg in zip(c, z_test)]
