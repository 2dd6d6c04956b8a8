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


def _read_cfar_golden(path):
    rows = [[float(v) for v in l.split()] for l in open(path) if l.strip() and not l.startswith("#")]
    return np.array(rows)


def test_cfar_across_velocity_bins_golden(golden):
    """Hand-worked 1-D CFAR (Sec. IV-B) on a 4-velocity-bin x 3-range-cell
    map: each cell against the mean of the other velocity bins of its
    range cell."""
    tab = _read_cfar_golden(golden("cfar_P4_F3.txt"))
    m = tab[:, 2].reshape(1, 4, 3)
    mask, floor = RD.cfar_detect(m, 10.0)
    np.testing.assert_allclose(floor.reshape(-1), tab[:, 3], rtol=1e-15)
    assert (mask.reshape(-1) == tab[:, 4].astype(bool)).all()


def test_cfar_target_alone_in_its_range_cell_is_detected():
    """With the cell under test left out of its own floor, a target 20 dB
    above flat noise is detected at P_te = 4..8 (a floor that included it
    would reach m / P_te + noise and hide it at 10 dB for P_te <= 10), and
    nothing else is."""
    for Pd in (4, 5, 8):
        m = np.ones((1, Pd, 16))
        m[0, Pd - 1, 9] = 100.0
        mask, floor = RD.cfar_detect(m, 10.0)
        assert mask.sum() == 1 and mask[0, Pd - 1, 9]
        assert floor[0, Pd - 1, 9] == pytest.approx(1.0)
        assert floor[0, 0, 9] == pytest.approx((Pd - 2 + 100.0) / (Pd - 1))
    with pytest.raises(ValueError):
        RD.cfar_detect(np.ones((1, 1, 4)))


def test_detection_errors():
    m = np.ones((3, 4, 10))
    mask = np.zeros(m.shape, bool)
    m[0, 1, 6] = 50.0; mask[0, 1, 6] = True          # exact
    m[1, 3, 2] = 30.0; mask[1, 3, 2] = True          # velocity wraps: 3 - 0 -> -1
    m[1, 2, 2] = 40.0; mask[1, 2, 2] = True          # the stronger detection wins
    det = RD.detection_errors(mask, m, delay=[6, 4, 0], doppler=[1, 0, 0])
    assert det[0] == (True, (1, 6), 0, 0)
    assert det[1] == (True, (2, 2), -2, 2 - 4)
    assert det[2] == (False, None, None, None)
