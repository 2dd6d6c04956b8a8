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
from synth import all_configs, make_scene, scaled_config

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
    """The sweep's summary rows: one per (M, W <= min(M, 16)), finite, with
    the full-dimensional point flagged."""
    from paper_2508_11790_gb300.sweep import sinr_sweep
    cfg, sc = _scene()
    rows = sinr_sweep(cfg, sc.x, sc.u_tgt, [3, 9, 16], [16, 32], int(cfg.K[0]))
    assert [(r["M"], r["W"]) for r in rows] == [(16, 3), (16, 9), (16, 16), (32, 3), (32, 9), (32, 16)]
    assert [r["full_dimensional"] for r in rows] == [False, False, True, False, False, False]
    for r in rows:
        assert np.isfinite(r["mean_sinr_db"]) and np.isfinite(r["mean_reference_mvdr_sinr_db"])
        assert r["mean_gap_db"] == pytest.approx(r["mean_reference_mvdr_sinr_db"] - r["mean_sinr_db"])
