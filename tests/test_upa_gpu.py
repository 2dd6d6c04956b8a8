"""GPU parity of the planar-array path (the paper's 4 x 32 UPA, 8 x 64 beams)
against the FP64 planar oracle: window starts and windowed steering
vectors, every training and test window (2-D transform of the GPU's
channelised data, Eq. OverallDFT, Wx x Wz windows read as S_h (x) S_v), and
end to end the weights, SINR loss and outputs.

Tolerances as for the linear array: windows within FFT_TOL of the subband's
largest beam norm, weights within 1e-3 and SINR loss within 0.1 dB of the
FP64 pipeline, outputs within 2e-3.
"""
import numpy as np
import pytest

import oracle as O
import paper_2508_11790_gb300 as P
from gpu_helpers import rel, run_gpu
from oracle import upa as U
from synth import all_configs, make_scene, scaled_config

pytestmark = pytest.mark.gpu

FFT_TOL = 5e-6


def _upa_config(kind="paper"):
    if kind == "paper":
        # window sizes W_z x W_x: 2 x 4 and 4 x 4 (the paper's), 2 x 2, 3 x 3, 1 x 5
        return scaled_config(all_configs()["C1"], name="upa-4x32", N=128, Nz=4, M=512, Mz=8, T=5,
                             W=(8, 16, 4, 9, 5), Wz=(2, 4, 2, 3, 1), K=64, P_tr=2, P_te=1, n_jam=2)
    if kind == "wide":
        # the paper's 4 x 8 window (E2) and other windows above 16 beams:
        # 4 x 8, 4 x 6, 4 x 4, 2 x 4
        return scaled_config(all_configs()["C1"], name="upa-4x32-wide", N=128, Nz=4, M=512, Mz=8, T=4,
                             W=(32, 24, 16, 8), Wz=(4, 4, 4, 2), K=64, P_tr=2, P_te=1, n_jam=2)
    if kind == "large":
        # 4 x 128 elements, 8 x 256 beams: one vector per CTA (its buffers fill the shared memory)
        return scaled_config(all_configs()["C1"], name="upa-4x128", N=512, Nz=4, M=2048, Mz=8, T=3,
                             W=(16, 8, 6), Wz=(4, 2, 3), K=64, P_tr=2, P_te=1, n_jam=2)
    # a single column (Nx = Mx = 1): no horizontal transform, windows 4 x 1 and 2 x 1
    return scaled_config(all_configs()["C1"], name="upa-4x1", N=4, Nz=4, M=16, Mz=16, T=2,
                         W=(4, 2), Wz=(4, 2), K=16, P_tr=1, P_te=1, n_jam=1)


@pytest.mark.parametrize("kind,precision", [("paper", P.BS_PREC_FP32), ("paper", P.BS_PREC_FP16),
                                            ("wide", P.BS_PREC_FP32), ("wide", P.BS_PREC_FP16),
                                            ("large", P.BS_PREC_FP32), ("column", P.BS_PREC_FP32)])
def test_planar_pipeline_matches_oracle(kind, precision):
    cfg = _upa_config(kind)
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, v=sc.v_tgt)
    ref = U.run_pipeline2d(sc.x, cfg, sc.u_tgt, sc.v_tgt)
    B = cfg.B
    yb = U.beamspace2d(res.xc.astype(np.complex128), cfg.Mx, cfg.Mz, cfg.Nx, cfg.Nz)   # [P][F][M]
    worst_w, worst_loss = 0.0, 0.0
    for k in range(len(ref.t)):
        t, s = int(ref.t[k]), int(ref.s[k])
        g = t * cfg.L + s
        pr = res.pair(g)
        assert pr["start"] == int(ref.start_x[k])
        np.testing.assert_allclose(pr["a"], ref.a_tilde[k], atol=1e-12 * max(1.0, np.abs(ref.a_tilde[k]).max()))
        if precision == P.BS_PREC_FP32:
            Wz = cfg.Wz_t[t]
            beams = U.window_beams2d(int(ref.start_x[k]), cfg.W[t] // Wz, cfg.Mx, int(ref.start_z[k]), Wz, cfg.Mz)
            zall = yb[:, s * B:(s + 1) * B][:, :, beams].reshape(cfg.P * B, cfg.W[t])
            scale = np.linalg.norm(yb[:, s * B:(s + 1) * B], axis=-1).max()
            assert np.abs(pr["z_train"] - zall[:pr["K"]]).max() <= FFT_TOL * scale, g
            assert np.abs(pr["z_test"] - zall[cfg.P_tr * B:]).max() <= FFT_TOL * scale, g
        assert pr["info"] in (0, -2)
        e = rel(pr["c"], ref.c[k])
        loss = O.sinr_loss_db(pr["c"].astype(np.complex128), ref.c[k], ref.a_tilde[k], ref.R[k])
        worst_w, worst_loss = max(worst_w, e), max(worst_loss, abs(loss))
        assert abs(loss) <= 0.1, (g, loss)
        if precision == P.BS_PREC_FP32:
            assert e <= 1e-3, (g, e)
            assert rel(pr["out"], ref.out[k]) <= 2e-3, g
    print(f"UPA {kind} precision {precision}: max weight rel err {worst_w:.2e}, max |SINR loss| {worst_loss:.2e} dB")


def test_planar_rejects_linear_only_calls():
    cfg = _upa_config()
    sc = make_scene(cfg)
    plan = P.Plan.from_scene_config(cfg, sc.u_tgt, v=sc.v_tgt)
    import torch
    c = torch.zeros(plan.sizes.c_elems, dtype=torch.complex64, device="cuda")
    ch = torch.zeros(plan.sizes.pairs * plan.N, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.BsError, match="linear arrays only"):
        P.bs_lift(plan, c, ch)
