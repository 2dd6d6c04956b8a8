"""FP64 oracle of the planar-array path (test infrastructure only).

Uniform planar array of Nx x Nz elements, element n = n_x Nz + n_z (the
order of a = a_x (x) a_z, Eq. ArrayFactor).  The 2-D beamspace transform is
D = D_h^T (x) D_v (Eq. VerDFT, Eq. HorDFT, Eq. OverallDFT), beam
m = m_x Mz + m_z.  The window of target k selects W_x x W_z beams; the
printed selector S_h^T (x) S_v with S_h in R^{W_x x M_x} does not have the
W x M shape the text states, so it is read as S = S_h (x) S_v (window entry
w = w_x W_z + w_z), the Kronecker order that matches D.  Each axis' window is
centred as in the linear case (Eq. OverallWindow) on its own squinted
spatial frequency, Omega_x = pi u f / f_d, Omega_z = pi v f / f_d with
u = cos(theta) sin(phi), v = sin(theta) (Eq. OmegaX, Eq. OmegaZ,
Eq. SubOmegaX, Eq. SubOmegaZ).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .beamspace_mvdr import (beamformer_output, channelize, mvdr_weights, squinted_omega, steering_vector,
                             subband_center_freq, truncated_dft_matrix, window_beams, window_covariance,
                             window_start)

__all__ = ["steering2d", "dft2d", "beamspace2d", "window_beams2d", "run_pipeline2d"]


def steering2d(om_x: float, om_z: float, Nx: int, Nz: int) -> np.ndarray:
    """a = a_x(Omega_x) (x) a_z(Omega_z) (Eq. ArrayFactor)."""
    return np.kron(steering_vector(om_x, Nx), steering_vector(om_z, Nz))


def dft2d(Mx: int, Nx: int, Mz: int, Nz: int) -> np.ndarray:
    """D = D_h^T (x) D_v, M x N (Eq. OverallDFT); D_h^T is the M_x x N_x
    truncated DFT, D_v the M_z x N_z one."""
    return np.kron(truncated_dft_matrix(Mx, Nx), truncated_dft_matrix(Mz, Nz))


def beamspace2d(y: np.ndarray, Mx: int, Mz: int, Nx: int, Nz: int) -> np.ndarray:
    """D y for every vector y[..., N] (Eq. BeamTransform), by zero-padded
    orthonormal FFTs along both axes; [..., M]."""
    y = np.asarray(y, np.complex128).reshape(y.shape[:-1] + (Nx, Nz))
    yb = np.fft.fft(np.fft.fft(y, n=Mz, axis=-1), n=Mx, axis=-2) / np.sqrt(Mx * Mz)
    return yb.reshape(yb.shape[:-2] + (Mx * Mz,))


def window_beams2d(sx: int, Wx: int, Mx: int, sz: int, Wz: int, Mz: int) -> np.ndarray:
    """Beams of the W_x x W_z window, entry w = w_x W_z + w_z."""
    bx = window_beams(sx, Wx, Mx)
    bz = window_beams(sz, Wz, Mz)
    return (bx[:, None] * Mz + bz[None, :]).reshape(-1)


@dataclass
class Pipeline2DResult:
    t: np.ndarray
    s: np.ndarray
    start_x: np.ndarray
    start_z: np.ndarray
    a_tilde: list
    R: list
    c: list
    out: list


def run_pipeline2d(x: np.ndarray, cfg, u, v, subbands=None) -> Pipeline2DResult:
    """Channelise -> 2-D beamspace -> W_x x W_z window -> loaded covariance ->
    MVDR -> apply, for every (target, subband) pair of a planar-array
    workload (cfg: a synth.SceneConfig with Nz, Mz, Wz)."""
    L, B = cfg.L, cfg.F // cfg.L
    Nx, Nz, Mx, Mz = cfg.Nx, cfg.Nz, cfg.Mx, cfg.Mz
    subs = list(range(L)) if subbands is None else [int(s) for s in subbands]
    xc = channelize(x, L)                                  # [P][L][B][N]
    yb = beamspace2d(xc, Mx, Mz, Nx, Nz)                   # [P][L][B][M]
    D = dft2d(Mx, Nx, Mz, Nz)
    P = x.shape[0]
    res = Pipeline2DResult(*([] for _ in range(8)))
    for t in range(cfg.T):
        Wz = cfg.Wz_t[t]
        Wx = cfg.W[t] // Wz
        for s in subs:
            f = subband_center_freq(s, L, cfg.fc, cfg.fs)
            sx = window_start(float(u[t]), s, Wx, L, Mx, cfg.fc, cfg.fs, cfg.fd)
            sz = window_start(float(v[t]), s, Wz, L, Mz, cfg.fc, cfg.fs, cfg.fd)
            beams = window_beams2d(sx, Wx, Mx, sz, Wz, Mz)
            z = yb[:, s][:, :, beams].reshape(P * B, -1)
            a = D[beams] @ steering2d(squinted_omega(float(u[t]), f, cfg.fd),
                                      squinted_omega(float(v[t]), f, cfg.fd), Nx, Nz)
            R = window_covariance(z[:cfg.K[t]], cfg.delta)
            c = mvdr_weights(R, a)
            res.t.append(t); res.s.append(s); res.start_x.append(sx); res.start_z.append(sz)
            res.a_tilde.append(a); res.R.append(R); res.c.append(c)
            res.out.append(beamformer_output(c, z[cfg.P_tr * B:]))
    res.t, res.s = np.array(res.t), np.array(res.s)
    res.start_x, res.start_z = np.array(res.start_x), np.array(res.start_z)
    return res
