"""Pins of the planar-array oracle: the 2-D transform against the explicit
Kronecker matrix, the Kronecker structure of the windowed steering vector,
the reduction to the linear array for Nz = 1, and full-dimensional antenna
MVDR for a full window of the unitary (unpadded) transform."""
import numpy as np

import oracle as O
from oracle import upa as U
from synth import all_configs, make_scene, scaled_config

RNG = np.random.default_rng(7)


def crandn(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


def test_beamspace2d_is_the_kronecker_transform():
    Nx, Nz, Mx, Mz = 6, 3, 16, 4
    y = crandn(5, Nx * Nz)
    D = U.dft2d(Mx, Nx, Mz, Nz)
    # brute force entries: D[m_x Mz + m_z, n_x Nz + n_z]
    mx, mz, nx, nz = 5, 3, 4, 2
    ref = np.exp(-2j * np.pi * (mx * nx / Mx + mz * nz / Mz)) / np.sqrt(Mx * Mz)
    assert abs(D[mx * Mz + mz, nx * Nz + nz] - ref) < 1e-14
    np.testing.assert_allclose(U.beamspace2d(y, Mx, Mz, Nx, Nz), y @ D.T, atol=1e-12)


def test_windowed_steering_is_kronecker_of_the_axes():
    Nx, Nz, Mx, Mz = 8, 4, 16, 8
    omx, omz = 0.7, -0.4
    sx, Wx, sz, Wz = 14, 4, 6, 3   # both windows wrap
    beams = U.window_beams2d(sx, Wx, Mx, sz, Wz, Mz)
    a2 = U.dft2d(Mx, Nx, Mz, Nz)[beams] @ U.steering2d(omx, omz, Nx, Nz)
    ax = O.windowed_steering(omx, Nx, Mx, O.window_beams(sx, Wx, Mx))
    az = O.windowed_steering(omz, Nz, Mz, O.window_beams(sz, Wz, Mz))
    np.testing.assert_allclose(a2, np.kron(ax, az), atol=1e-12)


def test_linear_array_is_the_nz_1_case():
    cfg = scaled_config(all_configs()["C1"], name="ula-as-upa", N=16, F=128, L=4, M=32, T=2, W=5, K=40,
                        P_tr=2, P_te=1, n_jam=1)
    sc = make_scene(cfg)
    ref = O.run_pipeline(sc.x, cfg, sc.u_tgt)
    res = U.run_pipeline2d(sc.x, cfg, sc.u_tgt, np.zeros(cfg.T))
    for k in range(len(ref.pairs.t)):
        j = int(np.nonzero((res.t == ref.pairs.t[k]) & (res.s == ref.pairs.s[k]))[0][0])
        assert res.start_x[j] == ref.pairs.start[k]
        np.testing.assert_allclose(res.c[j], ref.c[k], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(res.out[j], ref.out[k], rtol=1e-12, atol=1e-14)


def test_full_window_of_unitary_transform_is_antenna_mvdr():
    """Mx = Nx, Mz = Nz, W = N: D is unitary, and the lifted windowed MVDR
    weights D^H S^T c equal full-dimensional antenna MVDR (Sec. II-B)."""
    Nx, Nz, K, delta = 4, 2, 30, 0.5
    y = crandn(K, Nx * Nz)
    a = U.steering2d(0.9, -0.3, Nx, Nz)
    D = U.dft2d(Nx, Nx, Nz, Nz)
    np.testing.assert_allclose(D.conj().T @ D, np.eye(Nx * Nz), atol=1e-12)
    c_b = O.mvdr_weights(O.window_covariance(y @ D.T, delta), D @ a)
    np.testing.assert_allclose(D.conj().T @ c_b, O.antenna_mvdr(y, a, delta), atol=1e-12)
