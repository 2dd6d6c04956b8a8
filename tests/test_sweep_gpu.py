"""GPU parity of the window-size / zero-padding SINR sweep: every pair's
output SINR (weights from K training vectors, judged against the
no-loading covariance of all K_ref target-free training vectors of the same
window) against the FP64 oracle, and the W = M = N point against
full-dimensional antenna-space MVDR (Sec. II-B), which it equals because the
unpadded beamspace is unitary (Eq. AntennaEqCorr).
"""
import numpy as np
import pytest

import oracle as O
from oracle import range_doppler as RD
from synth import all_configs, make_scene, pulse, scaled_config

pytestmark = pytest.mark.gpu

SINR_TOL_DB = 0.01


def _scene():
    cfg = scaled_config(all_configs()["C1"], name="sweep-small", N=16, F=256, L=8, M=16, T=4, W=5, K=48,
                        P_tr=4, P_te=1, n_jam=2)
    return cfg, make_scene(cfg)


@pytest.mark.parametrize("W,M", [(3, 16), (8, 32), (16, 64), (16, 16)])
def test_sweep_point_matches_oracle(W, M):
    from paper_2508_11790_gb300.sweep import sweep_point
    cfg, sc = _scene()
    K = int(cfg.K[0])
    r = sweep_point(cfg, sc.x, sc.u_tgt, W, M, K)
    assert (r["info"] == 0).all()
    c = scaled_config(cfg, W=W, M=M, K=K)
    ref = O.run_pipeline(sc.x, c, sc.u_tgt)
    B = c.F // c.L
    K_ref = c.P_tr * B
    yb = O.beamspace(O.channelize(sc.x, c.L), M)   # [P][L][B][M]
    xc = O.channelize(sc.x, c.L)                    # [P][L][B][N]
    worst = 0.0
    for k in range(len(ref.pairs.t)):
        t, s = int(ref.pairs.t[k]), int(ref.pairs.s[k])
        g = t * c.L + s
        beams = O.window_beams(int(ref.pairs.start[k]), W, M)
        z_ref = yb[:c.P_tr, s][:, :, beams].reshape(K_ref, W)
        R_ref = O.window_covariance(z_ref, 0.0)
        a = ref.pairs.a_tilde[k]
        s_or = 10 * np.log10(O.output_sinr(ref.c[k], a, R_ref))
        s_gpu = 10 * np.log10(r["sinr"][g])
        worst = max(worst, abs(s_gpu - s_or))
        # MVDR on the reference covariance with the method's loading
        c_ref = O.mvdr_weights(R_ref + c.delta * np.eye(W), a)
        s_opt = 10 * np.log10(O.output_sinr(c_ref, a, R_ref))
        assert abs(10 * np.log10(r["sinr_opt"][g]) - s_opt) <= SINR_TOL_DB, (g, s_opt)
        if W == M == c.N:
            # full-dimensional antenna MVDR on the channelised element vectors
            y = xc[:c.P_tr, s].reshape(K_ref, c.N)
            omega = O.squinted_omega(float(sc.u_tgt[t]), O.subband_center_freq(s, c.L, c.fc, c.fs), c.fd)
            a_ant = O.steering_vector(omega, c.N)
            c_ant = O.antenna_mvdr(y[:K], a_ant, c.delta)
            s_ant = 10 * np.log10(O.output_sinr(c_ant, a_ant, O.window_covariance(y, 0.0)))
            assert abs(s_gpu - s_ant) <= SINR_TOL_DB, (g, s_gpu, s_ant)
    assert worst <= SINR_TOL_DB, worst


def test_sweep_rows():
    """The sweep's summary rows: one per (M, W <= min(M, 32)), finite, with
    the full-dimensional point flagged."""
    from paper_2508_11790_gb300.sweep import sinr_sweep
    cfg, sc = _scene()
    rows = sinr_sweep(cfg, sc.x, sc.u_tgt, [3, 9, 16], [16, 32], int(cfg.K[0]))
    assert [(r["M"], r["W"]) for r in rows] == [(16, 3), (16, 9), (16, 16), (32, 3), (32, 9), (32, 16)]
    assert [r["full_dimensional"] for r in rows] == [False, False, True, False, False, False]
    for r in rows:
        assert np.isfinite(r["mean_sinr_db"]) and np.isfinite(r["mean_reference_mvdr_sinr_db"])
        assert r["mean_gap_db"] == pytest.approx(r["mean_reference_mvdr_sinr_db"] - r["mean_sinr_db"])


def _coherent_scene():
    cfg = scaled_config(all_configs()["C1"], name="detect-small", N=32, F=256, L=8, M=32, T=4, W=5, K=48,
                        P_tr=4, P_te=6, n_jam=3, jnr_db=(40.0, 50.0), snr_db=-18.0, coherent_targets=True)
    return cfg, make_scene(cfg)


@pytest.mark.parametrize("W,M", [(3, 32), (9, 64), (32, 64)])
def test_detection_point_matches_oracle(W, M):
    """The GPU detection of every target (pass, range-Doppler map, CFAR
    across velocity bins, strongest detected cell) equals the oracle's FP64
    chain on the same scene wherever the oracle's decision is clear (its
    peak cell beats the CFAR threshold and the runner-up detection by more
    than 1e-3)."""
    from paper_2508_11790_gb300.sweep import detection_point
    cfg, sc = _coherent_scene()
    ps = np.fft.fft(pulse(cfg.F), norm="ortho")
    K = int(cfg.K[0])
    r = detection_point(cfg, sc.x, sc.u_tgt, sc.tgt_delay, sc.tgt_doppler, ps, W, M, K)
    c = scaled_config(cfg, W=W, M=M, K=K)
    ref = O.run_pipeline(sc.x, c, sc.u_tgt)
    out = np.stack(ref.out)                                      # [T L][P_te B]
    m = RD.doppler_map(RD.range_profiles(RD.beamformed_spectrum(out, c.T, c.L, c.B, c.P_te), ps))
    mask, floor = RD.cfar_detect(m, 10.0)
    det = RD.detection_errors(mask, m, sc.tgt_delay, sc.tgt_doppler)
    checked = 0
    for t in range(c.T):
        got = r["targets"][t]
        ok, cell, re, ve = det[t]
        if ok:
            vals = np.sort(m[t][mask[t]])[::-1]
            thr = floor[t][cell] * 10.0
            clear = m[t][cell] > thr * (1 + 1e-3) and (len(vals) < 2 or vals[0] > vals[1] * (1 + 1e-3))
        else:
            clear = (m[t] < floor[t] * 10.0 * (1 - 1e-3)).all()
        if not clear:
            continue
        checked += 1
        assert got["detected"] == ok, t
        if ok:
            assert (got["velocity_bin"], got["range_bin"]) == cell, (t, got, cell)
            assert (got["range_error"], got["velocity_error"]) == (re, ve)
    assert checked >= c.T - 1


def test_detection_sweep_rows():
    """Rows of the detection sweep for linear windows up to 32 and FFT sizes
    N and 2N: every target counted, errors finite where detected."""
    from paper_2508_11790_gb300.sweep import detection_sweep
    cfg, sc = _coherent_scene()
    ps = np.fft.fft(pulse(cfg.F), norm="ortho")
    rows = detection_sweep(cfg, sc.x, sc.u_tgt, sc.tgt_delay, sc.tgt_doppler, ps, [1, 5, 32], [32, 64],
                           int(cfg.K[0]))
    assert [(r["fft"], r["window"]) for r in rows] == [("32", "1"), ("32", "5"), ("32", "32"), ("64", "1"),
                                                       ("64", "5"), ("64", "32")]
    for r in rows:
        assert r["targets"] == cfg.T and r["detected"] + len(r["missed"]) == cfg.T
        assert r["exact"] <= r["detected"]
