"""Pins of the FP64 oracle to things other than itself (no GPU needed).

Each test ties one oracle function to a hand-worked fixture, a brute-force
sum written from the paper's definition in a different form, a closed form,
an invariant of the method, or a textbook special case.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import all_configs, make_scene, reference_records, scaled_config

RNG = np.random.default_rng(1234)


def crandn(*shape, rng=RNG):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def read_golden(path):
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


# --------------------------------------------------------------- fixtures
def test_subband_freqs_golden(golden):
    tab = read_golden(golden("subband_freqs_L4.txt"))
    for s, ell, f in tab:
        assert int(s) - 4 // 2 + 1 == int(ell)
        assert O.subband_center_freq(int(s), 4, 10.0, 1.0) == pytest.approx(f, abs=1e-15)


def test_dft_matrix_golden(golden):
    tab = read_golden(golden("dft_M4_N2.txt"))
    D = O.truncated_dft_matrix(4, 2)
    for m, n, re, im in tab:
        assert D[int(m) - 1, int(n) - 1] == pytest.approx(re + 1j * im, abs=1e-15)


def test_mvdr_golden(golden):
    tab = read_golden(golden("mvdr_2x2.txt"))
    c = O.mvdr_weights(np.diag([2.0, 1.0]).astype(complex), np.array([1.0, 1.0]))
    np.testing.assert_allclose(c, tab[:, 1] + 1j * tab[:, 2], atol=1e-15)


# --------------------------------------------------------------- channeliser
def _brute_channelize(x, L):
    """Triple loop from the definition with the signed frequency of each bin."""
    P, F, N = x.shape
    B = F // L
    out = np.zeros((P, L, B, N), complex)
    for p in range(P):
        for s in range(L):
            for i in range(B):
                nu = ((s - L // 2) * B + i) / F          # cycles / sample, signed
                for n in range(N):
                    acc = 0j
                    for t in range(F):
                        acc += x[p, t, n] * np.exp(-2j * np.pi * nu * t)
                    out[p, s, i, n] = acc / math.sqrt(F)
    return out


def test_channelize_bruteforce():
    x = crandn(2, 16, 3)
    ref = _brute_channelize(x, 4)
    np.testing.assert_allclose(O.channelize(x, 4), ref, atol=1e-12)
    np.testing.assert_allclose(O.channelize(x, 4, subbands=[3, 1]), ref[:, [3, 1]], atol=1e-12)


@pytest.mark.parametrize("ell", [-3, 0, 1, 4])
def test_channelize_tone_at_subband_centre(ell):
    """A tone at f(l) - f_c (Eq. SubChannelFreq) lands on the middle bin of
    subband s = l + L/2 - 1 and nowhere else."""
    F, L, N = 64, 8, 2
    B = F // L
    fs, fc = 1.0, 0.0
    f_off = O.subband_center_freq(ell + L // 2 - 1, L, fc, fs) - fc   # = (l - 1/2) fs / L
    t = np.arange(F)
    x = np.exp(2j * np.pi * f_off / fs * t)[None, :, None] * np.ones((1, 1, N))
    Xc = O.channelize(x, L)
    s = ell + L // 2 - 1
    mag = np.abs(Xc[0, :, :, 0])
    assert mag[s, B // 2] == pytest.approx(math.sqrt(F), rel=1e-12)
    mag[s, B // 2] = 0
    assert mag.max() < 1e-9


def test_channelize_parseval():
    x = crandn(3, 32, 5)
    Xc = O.channelize(x, 4)
    assert np.sum(abs(Xc) ** 2) == pytest.approx(np.sum(abs(x) ** 2), rel=1e-12)


# --------------------------------------------------------------- beamspace
def test_beamspace_bruteforce():
    N, M = 5, 8
    y = crandn(3, N)
    ref = np.zeros((3, M), complex)
    for v in range(3):
        for m in range(M):
            for n in range(N):
                ref[v, m] += y[v, n] * np.exp(-2j * np.pi * m * n / M) / math.sqrt(M)
    np.testing.assert_allclose(O.beamspace(y, M), ref, atol=1e-13)
    np.testing.assert_allclose(O.truncated_dft_matrix(M, N) @ y.T, ref.T, atol=1e-13)


def test_beamspace_unitary_when_not_padded():
    y = crandn(4, 16)
    yb = O.beamspace(y, 16)
    np.testing.assert_allclose(np.sum(abs(yb) ** 2, -1), np.sum(abs(y) ** 2, -1), rtol=1e-12)


# --------------------------------------------------------------- window and steering
@pytest.mark.parametrize("N,M", [(8, 8), (16, 64), (100, 256)])
def test_windowed_steering_dirichlet(N, M):
    """a_tilde = S D a equals the closed-form Dirichlet kernel
    M^-1/2 e^{j(N-1)d/2} sin(N d/2)/sin(d/2), d = Omega - 2 pi m / M."""
    for omega in RNG.uniform(-np.pi, np.pi, size=5):
        beams = np.arange(M)
        at = O.windowed_steering(omega, N, M, beams)
        d = omega - 2 * np.pi * beams / M
        assert np.min(np.abs(np.sin(d / 2))) > 1e-9      # random omega: no 0/0 case
        closed = np.exp(1j * (N - 1) * d / 2) * np.sin(N * d / 2) / np.sin(d / 2) / math.sqrt(M)
        np.testing.assert_allclose(at, closed, atol=1e-10)


@pytest.mark.parametrize("W", [1, 3, 5, 9, 4])
def test_window_is_centred_on_target_beam(W):
    """The window holds the beam of largest |D a| (odd W: at its centre) and
    its centre is within half a beam of the squinted frequency."""
    N, M, L = 32, 128, 8
    fc, fs, fd = 10e9, 1e9, 10e9
    for u in RNG.uniform(-0.87, 0.87, size=20):
        for s in (0, 3, 7):
            start = O.window_start(u, s, W, L, M, fc, fs, fd)
            beams = O.window_beams(start, W, M)
            omega = O.squinted_omega(u, O.subband_center_freq(s, L, fc, fs), fd)
            full = np.abs(O.windowed_steering(omega, N, M, np.arange(M)))
            assert int(np.argmax(full)) in set(beams.tolist())
            if W % 2 == 1:
                assert beams[W // 2] == int(np.argmax(full))
            x = omega * M / (2 * np.pi)
            centre = start + (W - 1) / 2.0
            dist = (x - centre + M / 2) % M - M / 2
            assert abs(dist) <= 0.5 + 1e-9


def test_squint_moves_window_with_frequency():
    """Eq. SubOmegaX: the spatial frequency scales with f(l)/f_d, so a target
    off broadside drifts across beams from the lowest to the highest subband."""
    N, M, L = 64, 512, 16
    u = 0.8
    x = [O.squinted_omega(u, O.subband_center_freq(s, L, 10e9, 5e9), 10e9) * M / (2 * np.pi)
         for s in range(L)]
    assert np.all(np.diff(x) > 0)
    # x(s) = u M f(l) / (2 f_d): the span over the band is u M ((L-1)/L) f_s / (2 f_d)
    assert x[-1] - x[0] == pytest.approx(u * M * ((L - 1) / L) * 5e9 / (2 * 10e9), rel=1e-12)


# --------------------------------------------------------------- covariance
def test_window_covariance_properties():
    K, W, delta = 40, 6, 0.5
    z = crandn(K, W)
    R = O.window_covariance(z, delta)
    np.testing.assert_allclose(R, R.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(R).min() >= delta - 1e-12
    assert np.trace(R).real == pytest.approx(np.mean(np.sum(abs(z) ** 2, 1)) + W * delta, rel=1e-12)
    brute = np.zeros((W, W), complex)
    for k in range(K):
        for i in range(W):
            for j in range(W):
                brute[i, j] += z[k, i] * np.conj(z[k, j])
    np.testing.assert_allclose(R, brute / K + delta * np.eye(W), atol=1e-13)


def test_window_covariance_is_window_of_beamspace_covariance():
    """R_tilde = S (D R_hat D^H) S^T + delta I, with R_hat the antenna-space
    sample covariance (Eq. EmpiricalCov) and D, S as in Sec. III-B."""
    N, M, K, delta = 12, 32, 30, 2.0
    y = crandn(K, N)
    beams = O.window_beams(30, 5, M)                  # wraps around M
    z = O.beamspace(y, M)[:, beams]
    Rhat = O.window_covariance(y, 0.0)
    D = O.truncated_dft_matrix(M, N)
    ref = (D @ Rhat @ D.conj().T)[np.ix_(beams, beams)] + delta * np.eye(5)
    np.testing.assert_allclose(O.window_covariance(z, delta), ref, atol=1e-12)


# --------------------------------------------------------------- MVDR
def _rand_pd(W, cond=1e3):
    Q, _ = np.linalg.qr(crandn(W, W))
    ev = np.logspace(0, math.log10(cond), W)
    return (Q * ev) @ Q.conj().T


@pytest.mark.parametrize("W", [1, 2, 5, 9, 16])
def test_mvdr_constraint_power_and_optimality(W):
    R = _rand_pd(W)
    a = crandn(W)
    c = O.mvdr_weights(R, a)
    assert np.vdot(c, a) == pytest.approx(1.0, abs=1e-10)            # Eq. DefMVDR constraint
    p = np.real(np.vdot(c, R @ c))
    q = np.real(np.vdot(a, np.linalg.inv(R) @ a))
    assert p == pytest.approx(1.0 / q, rel=1e-9)                      # min output power
    for _ in range(10):                                              # any other feasible c is worse
        d = crandn(W)
        d -= a * (np.vdot(a, d) / np.vdot(a, a))                     # keep c'^H a = 1
        c2 = c + 0.1 * d
        assert np.vdot(c2, a) == pytest.approx(1.0, abs=1e-10)
        assert np.real(np.vdot(c2, R @ c2)) >= p * (1 - 1e-12)


def test_mvdr_one_interferer_sherman_morrison():
    """R = s I + q b b^H: R^-1 a is proportional to a - q (b^H a)/(s + q ||b||^2) b."""
    W, s, q = 7, 3.0, 500.0
    a, b = crandn(W), crandn(W)
    R = s * np.eye(W) + q * np.outer(b, b.conj())
    v = a - q * np.vdot(b, a) / (s + q * np.vdot(b, b).real) * b
    c_closed = v / np.vdot(a, v)
    np.testing.assert_allclose(O.mvdr_weights(R, a), c_closed, atol=1e-12)


def test_mvdr_white_noise_is_matched_filter():
    a = crandn(6)
    np.testing.assert_allclose(O.mvdr_weights(4.0 * np.eye(6), a), a / np.vdot(a, a).real,
                               atol=1e-14)


def test_full_window_equals_antenna_mvdr():
    """W = M = N: D is unitary, so windowed beamspace MVDR lifted by
    Eq. AntennaEqCorr equals antenna-space MVDR (Eq. CorrMVDR) with the same
    loading."""
    N, K, delta = 16, 50, 1.5
    y = crandn(K, N) + 3.0 * np.outer(crandn(K), O.steering_vector(0.9, N))
    omega = -0.4
    a = O.steering_vector(omega, N)
    beams = np.arange(N)
    z = O.beamspace(y, N)
    at = O.windowed_steering(omega, N, N, beams)
    ct = O.mvdr_weights(O.window_covariance(z, delta), at)
    np.testing.assert_allclose(O.lifted_correlator(ct, N, N, beams), O.antenna_mvdr(y, a, delta),
                               atol=1e-11)


def test_lifted_correlator_is_distortionless():
    N, M, K = 20, 64, 40
    y = crandn(K, N)
    omega = 1.1
    start = int(round(omega * M / (2 * np.pi))) - 2
    beams = O.window_beams(start, 5, M)
    at = O.windowed_steering(omega, N, M, beams)
    ct = O.mvdr_weights(O.window_covariance(O.beamspace(y, M)[:, beams], 1.0), at)
    ch = O.lifted_correlator(ct, N, M, beams)
    assert np.vdot(ch, O.steering_vector(omega, N)) == pytest.approx(1.0, abs=1e-12)
    assert O.beam_pattern(ch, O.steering_vector(omega, N)) <= 1.0 + 1e-12
    assert O.beam_pattern(O.steering_vector(omega, N), O.steering_vector(omega, N)) == pytest.approx(1.0)


def test_sinr_loss_of_mvdr_is_non_negative():
    W = 5
    R = _rand_pd(W, 1e4)
    a = crandn(W)
    c = O.mvdr_weights(R, a)
    assert O.sinr_loss_db(c, c, a, R) == pytest.approx(0.0, abs=1e-12)
    for _ in range(5):
        assert O.sinr_loss_db(c + 0.01 * crandn(W), c, a, R) >= -1e-12


def _read_output_golden(path):
    outs, sinr = {}, None
    with open(path) as fh:
        for line in fh:
            f = line.split()
            if not f or f[0].startswith("#"):
                continue
            if f[0] == "out":
                outs[int(f[1])] = float(f[2]) + 1j * float(f[3])
            elif f[0] == "sinr":
                sinr = float(f[1])
    return outs, sinr


def test_beamformer_output_and_sinr_golden(golden):
    """Hand-worked c^H y (Sec. II-B) and |c^H a|^2 / (c^H R c) for W = 2."""
    outs, sinr = _read_output_golden(golden("output_2x2.txt"))
    c = np.array([1.0, 1j])
    y = np.array([[1.0, 1.0], [1j, 0.0], [2.0, 3j]])
    got = O.beamformer_output(c, y)
    for k, v in outs.items():
        assert got[k] == pytest.approx(v, abs=1e-15)
    R = np.array([[2.0, 1j], [-1j, 2.0]])
    assert O.output_sinr(c, np.array([1.0, 1.0]), R) == pytest.approx(sinr, abs=1e-15)


@pytest.mark.parametrize("W", [1, 3, 9, 16])
def test_beamformer_output_of_mvdr_is_distortionless(W):
    """Eq. DefMVDR: the MVDR correlator passes its own steering vector with
    unit gain, so the output for y = a~ is exactly 1 (a dropped conjugate or
    a transposed product gives c^T a instead)."""
    R = _rand_pd(W, 1e3)
    a = crandn(W)
    c = O.mvdr_weights(R, a)
    out = O.beamformer_output(c, a[None, :])
    assert out.shape == (1,)
    assert out[0] == pytest.approx(1.0, abs=1e-10)
    # linearity in the snapshots and anti-linearity in the weights
    y = crandn(4, W)
    np.testing.assert_allclose(O.beamformer_output(2j * c, y), -2j * O.beamformer_output(c, y), atol=1e-12)


@pytest.mark.parametrize("W", [1, 4, 9])
def test_output_sinr_of_mvdr_is_closed_form(W):
    """Against its own covariance the MVDR output SINR is a^H R^-1 a
    (distortionless gain 1 over output power 1/(a^H R^-1 a), Eq. CorrMVDR);
    for R = s I + q b b^H, a^H R^-1 a follows from Sherman-Morrison in closed
    form, independent of any solve."""
    s, q = 2.5, 300.0
    a, b = crandn(W), crandn(W)
    R = s * np.eye(W) + q * np.outer(b, b.conj())
    aa, ba, bb = np.vdot(a, a).real, np.vdot(b, a), np.vdot(b, b).real
    closed = (aa - q * abs(ba) ** 2 / (s + q * bb)) / s
    c = O.mvdr_weights(R, a)
    assert O.output_sinr(c, a, R) == pytest.approx(closed, rel=1e-10)
    # the conventional beamformer c = a: ||a||^4 / (s ||a||^2 + q |b^H a|^2)
    assert O.output_sinr(a, a, R) == pytest.approx(aa ** 2 / (s * aa + q * abs(ba) ** 2), rel=1e-12)
    # invariant to any complex scaling of the weights (|k|^2 over |k|^2)
    assert O.output_sinr((0.3 - 2j) * c, a, R) == pytest.approx(closed, rel=1e-10)


# --------------------------------------------------------------- whole path
def test_pipeline_consistency_small():
    cfg = scaled_config(all_configs()["C1"], T=3, L=8, P_tr=2, P_te=2, K=40, W=(5, 3, 1))
    sc = make_scene(cfg)
    res = O.run_pipeline(sc.x, cfg, sc.u_tgt)
    B = cfg.B
    yb = O.beamspace(O.channelize(sc.x, cfg.L), cfg.M)
    for g in range(len(res.pairs.t)):
        t, s = int(res.pairs.t[g]), int(res.pairs.s[g])
        W, K = int(res.pairs.W[g]), int(res.pairs.K[g])
        beams = O.window_beams(int(res.pairs.start[g]), W, cfg.M)
        # training vector k = record p, bin i with k = p * B + i
        for k in (0, K - 1):
            p, i = divmod(k, B)
            np.testing.assert_allclose(res.z_train[g][k], yb[p, s, i, beams], atol=1e-12)
        assert res.z_train[g].shape == (K, W)
        assert res.z_test[g].shape == (cfg.P_te * B, W)
        np.testing.assert_allclose(res.z_test[g][0], yb[cfg.P_tr, s, 0, beams], atol=1e-12)
        assert np.vdot(res.c[g], res.pairs.a_tilde[g]) == pytest.approx(1.0, abs=1e-10)
        np.testing.assert_allclose(res.out[g], res.z_test[g] @ res.c[g].conj(), atol=1e-12)


def test_scene_noise_only_covariance():
    """With jammers and targets off, channelised noise is white with power
    sigma^2 per bin (unitary FFT), so R_tilde -> sigma^2 S D D^H S^T + delta I."""
    base = all_configs()["C1"]
    cfg = scaled_config(base, n_jam=0, T=1, L=4, P_tr=64, P_te=0, K=64 * 128, W=5)
    sc = make_scene(cfg)
    res = O.run_pipeline(sc.x, cfg, sc.u_tgt, subbands=[1])
    beams = O.window_beams(int(res.pairs.start[0]), 5, cfg.M)
    D = O.truncated_dft_matrix(cfg.M, cfg.N, rows=beams)
    expect = cfg.sigma2 * D @ D.conj().T + cfg.delta * np.eye(5)
    tol = 5.0 / math.sqrt(cfg.K[0])
    assert np.max(np.abs(res.R[0] - expect)) < tol * np.max(np.abs(expect - cfg.delta * np.eye(5)))


def test_scene_training_records_are_target_free():
    """Training records hold jammers + noise only: with jammers off the
    training data is pure noise of variance sigma^2."""
    cfg = scaled_config(all_configs()["C1"], n_jam=0, P_tr=4, P_te=2, snr_db=20.0)
    sc = make_scene(cfg)
    tr = sc.x[: cfg.P_tr]
    assert np.mean(np.abs(tr) ** 2) == pytest.approx(cfg.sigma2, rel=0.02)
    assert np.mean(np.abs(sc.x[cfg.P_tr:]) ** 2) > 5 * cfg.sigma2


def test_lifted_output_equals_windowed_beamspace_output():
    """c_hat^H y = c~^H (S D y) (Sec. III-C, below Eq. AntennaEqCorr): the
    lifted correlator applied in antenna space gives the windowed beamspace
    output; the beamspace side is a brute-force DFT sum."""
    N, M, W, start = 12, 32, 5, 29   # window wraps past beam M-1
    ct = crandn(W)
    y = crandn(7, N)
    beams = O.window_beams(start, W, M)
    ch = O.lifted_correlator(ct, N, M, beams)
    n = np.arange(N)
    zb = np.array([[np.sum(yy * np.exp(-2j * np.pi * m * n / M)) / np.sqrt(M) for m in beams] for yy in y])
    np.testing.assert_allclose(O.lifted_output(ch, y), zb @ np.conj(ct), rtol=1e-12, atol=1e-12)


def test_beam_pattern_grid_closed_forms():
    """Eq. Cosine Sim: a matched filter c = a(Omega0) has the Dirichlet
    pattern |sin(N d/2) / (N sin(d/2))|, d = Omega - Omega0; a distortionless
    lifted MVDR correlator has pattern 1 / (||c_hat|| sqrt(N)) at its target."""
    N, fd, f = 16, 10e9, 9.6e9
    u = np.linspace(-0.95, 0.95, 41)
    u0 = 0.3
    om0 = O.squinted_omega(u0, f, fd)
    pat = O.beam_pattern_grid(O.steering_vector(om0, N), u, f, fd)
    d = np.array([O.squinted_omega(uk, f, fd) for uk in u]) - om0
    with np.errstate(invalid="ignore", divide="ignore"):
        dir_ = np.abs(np.sin(N * d / 2) / (N * np.sin(d / 2)))
    dir_[np.abs(d) < 1e-12] = 1.0
    np.testing.assert_allclose(pat, dir_, atol=1e-12)
    # lifted MVDR weights of a window around u0
    M, W = 32, 5
    x = om0 * M / (2 * np.pi)
    start = int(np.floor(x - W / 2 + 1)) % M
    beams = O.window_beams(start, W, M)
    at = O.windowed_steering(om0, N, M, beams)
    R = _rand_pd(W, cond=50.0)
    ch = O.lifted_correlator(O.mvdr_weights(R, at), N, M, beams)
    p0 = O.beam_pattern_grid(ch, [u0], f, fd)[0]
    assert p0 == pytest.approx(1.0 / (np.linalg.norm(ch) * np.sqrt(N)), rel=1e-12)


def test_boundary_functions_compose_to_the_pipeline():
    """The oracle_ functions of the five boundary calls, chained, give the
    pipeline's windows, covariances, weights and outputs exactly."""
    cfg = scaled_config(all_configs()["C1"], name="abi", T=3, W=(5, 3, 7), K=(40, 20, 64), L=8)
    sc = make_scene(cfg)
    ref = O.run_pipeline(sc.x, cfg, sc.u_tgt)
    pairs = O.oracle_pairs(cfg, sc.u_tgt)
    xc = O.oracle_channelize(sc.x, cfg.L)
    assert xc.shape == sc.x.shape
    ztr, zte = O.oracle_beamspace(xc, cfg, pairs)
    R = O.oracle_window_cov(ztr, cfg.delta)
    c = O.oracle_mvdr_solve(R, pairs.a_tilde)
    out = O.oracle_apply(c, zte)
    for g in range(len(pairs.t)):
        assert int(pairs.t[g]) * cfg.L + int(pairs.s[g]) == g
        np.testing.assert_array_equal(ztr[g], ref.z_train[g])
        np.testing.assert_array_equal(zte[g], ref.z_test[g])
        np.testing.assert_array_equal(R[g], ref.R[g])
        np.testing.assert_array_equal(c[g], ref.c[g])
        np.testing.assert_array_equal(out[g], ref.out[g])


def test_reference_covariance_sees_the_jammer():
    """The reference covariance (independent target-free records of the
    same scene) of a window centred on a strong jammer is dominated by that
    jammer: its principal eigenvector is the windowed steering vector
    S D a(Omega_j) of the jammer at the subband centre (closed-form
    Dirichlet kernel, Sec. III-C) up to the narrowband approximation (the
    jammer's spread over the subband's bins leaves a second, much smaller
    eigenvalue), its noise eigenvalues sit at the beam noise floor
    sigma^2 N / M, and the
    records are a new realisation (not the training records)."""
    cfg = scaled_config(all_configs()["C1"], T=2, L=8, n_jam=1, jnr_db=(30.0, 30.0), P_tr=4, P_te=1, K=64)
    sc = make_scene(cfg)
    xr = reference_records(cfg, 16)
    assert xr.shape == (16, cfg.F, cfg.N)
    assert not np.allclose(xr[0], sc.x[0])
    one = scaled_config(cfg, T=1, W=7, K=64)
    subs = [0, 3, 7]
    Rs = O.reference_covariances(xr, one, [float(sc.u_jam[0])], subbands=subs)
    tab = O.pair_table(one, [float(sc.u_jam[0])], subs)
    M, N = cfg.M, cfg.N
    for k, R in enumerate(Rs):
        ev, V = np.linalg.eigh(R)
        s = int(tab.s[k])
        om = O.squinted_omega(float(sc.u_jam[0]), O.subband_center_freq(s, cfg.L, cfg.fc, cfg.fs), cfg.fd)
        m = (int(tab.start[k]) + np.arange(7)) % M
        d = om - 2 * np.pi * m / M
        a = np.exp(1j * (N - 1) * d / 2) * np.sin(N * d / 2) / np.sin(d / 2) / math.sqrt(M)
        cos = abs(np.vdot(V[:, -1], a)) / np.linalg.norm(a)
        assert cos >= 0.99, (s, cos)
        assert ev[-1] >= 10 * ev[-2]        # the rest of the jammer: its spread over the subband's bins
        assert 0.5 * N / M <= np.median(ev[:-3]) <= 2.0 * N / M


def test_sinr_against_reference_covariance_rewards_nulling():
    """Judged against the independent reference covariance, loaded MVDR
    weights from the training records beat the matched filter a~ / ||a~||^2
    (which does not null the jammers) by a wide margin."""
    cfg = scaled_config(all_configs()["C1"], T=3, L=8, P_tr=4, P_te=1, K=64)
    sc = make_scene(cfg)
    res = O.run_pipeline(sc.x, cfg, sc.u_tgt, subbands=[2, 5])
    Rr = O.reference_covariances(reference_records(cfg, 16), cfg, sc.u_tgt, subbands=[2, 5])
    gains = []
    for k in range(len(res.pairs.t)):
        a = res.pairs.a_tilde[k]
        gains.append(10 * math.log10(O.output_sinr(res.c[k], a, Rr[k]) / O.output_sinr(a, a, Rr[k])))
    assert np.median(gains) > 10.0, gains
