"""Pins of the oracle's processing after the beamformer (synthesis, matched
filter, Doppler, CFAR) to closed forms and to the channeliser, on the CPU."""
import numpy as np
import pytest

import oracle as O
from oracle import range_doppler as RD
from synth import pulse

RNG = np.random.default_rng(99)


def test_noise_free_target_peak_closed_form():
    """A target of amplitude a, delay tau0 and Doppler bin d0 (phase
    advancing by 2 pi d0 / P_te per record) gives one map peak at (d0, tau0)
    of value (a Tp P_te / sqrt(F))^2: the pulse energy is Tp (orthonormal
    FFT), the synthesis IFFT is orthonormal, the Doppler DFT is not."""
    F, P_te, a, tau0, d0, psi = 64, 8, 0.7, 13, 3, 0.4
    P = np.fft.fft(pulse(F), norm="ortho")
    k = np.arange(F)
    r = np.arange(P_te)[:, None]
    Y = (a * np.exp(1j * (psi + 2 * np.pi * d0 * r / P_te)) * P[None, :] * np.exp(-2j * np.pi * k * tau0 / F))[None]
    m = RD.doppler_map(RD.range_profiles(Y, P))
    Tp = F // 2
    assert np.unravel_index(np.argmax(m[0]), m[0].shape) == (d0, tau0)
    assert m[0, d0, tau0] == pytest.approx((a * Tp * P_te / np.sqrt(F)) ** 2, rel=1e-12)
    # all other Doppler bins of the peak's range cell vanish
    np.testing.assert_allclose(np.delete(m[0, :, tau0], d0), 0.0, atol=1e-18 * m[0, d0, tau0] + 1e-20)


def test_beamformed_spectrum_follows_the_channeliser_bins():
    """A pair output equal to the channelised value of element 0 at every
    (subband, bin) reassembles the record's orthonormal FFT in FFT order."""
    F, L, P_te, T = 32, 4, 3, 2
    B = F // L
    x = (RNG.standard_normal((P_te, F, 1)) + 1j * RNG.standard_normal((P_te, F, 1)))
    xc = O.channelize(x, L)                       # [P][L][B][1]
    out = np.empty((T, L, P_te, B), np.complex128)
    for t in range(T):
        out[t] = xc[:, :, :, 0].transpose(1, 0, 2)  # [L][P][B]
    Y = RD.beamformed_spectrum(out.reshape(T * L, P_te * B), T, L, B, P_te)
    for t in range(T):
        np.testing.assert_allclose(Y[t], np.fft.fft(x[:, :, 0], axis=-1, norm="ortho"), atol=1e-12)


def test_range_profile_of_unit_spectrum_is_the_pulse_autocorrelation():
    """With Y = P (zero delay) the range profile is the pulse's circular
    autocorrelation / sqrt(F), computed here by a direct sum."""
    F = 32
    s = pulse(F)
    P = np.fft.fft(s, norm="ortho")
    rp = RD.range_profiles(P[None, None, :], P)[0, 0]
    acf = np.array([np.sum(s * np.conj(np.roll(s, tau))) for tau in range(F)]) / np.sqrt(F)
    np.testing.assert_allclose(rp, acf, atol=1e-12)


def test_cfar_threshold_and_floor():
    m = np.ones((2, 4, 8))
    m[0, 1, 2] = 20.0     # floor (31 + 20) / 32 = 1.59: threshold 15.9
    m[1, 3, 7] = 12.0     # floor (31 + 12) / 32 = 1.34: threshold 13.4
    mask, floor = RD.cfar_detect(m, 10.0)
    assert floor[0] == pytest.approx((31 + 20.0) / 32) and floor[1] == pytest.approx((31 + 12.0) / 32)
    assert mask[0].sum() == 1 and mask[0, 1, 2]
    assert mask[1].sum() == 0
