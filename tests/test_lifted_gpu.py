"""GPU parity of the lifted correlator (Sec. III-C, Eq. AntennaEqCorr), its
antenna-space application and its beam pattern (Eq. Cosine Sim) against the
FP64 oracle, each on the GPU's own inputs of that step.

Tolerances: the lift is a W <= 16 term FP32 sum with table twiddles
(LIFT_TOL = 1e-5 relative per pair); c_hat^H y sums N FP32 products
(APPLY_TOL = 2e-5 relative per pair); the beam pattern is a cosine in [0, 1]
(PATTERN_TOL = 2e-5 absolute); the antenna-space output equals the windowed
beamspace output of bs_apply up to the FP32 rounding of both paths
(IDENTITY_TOL = 2e-4 relative per pair).
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_11790_gb300 as P
from gpu_helpers import rel, run_gpu
from synth import all_configs, make_scene, scaled_config

pytestmark = pytest.mark.gpu

LIFT_TOL = 1e-5
APPLY_TOL = 2e-5
PATTERN_TOL = 2e-5
IDENTITY_TOL = 2e-4


def _configs():
    c2 = all_configs()["C2"]
    ragged = scaled_config(all_configs()["C1"], name="lift-ragged", N=100, F=256, L=8, M=128, T=37,
                           W=(1, 16, 5, 4, 9, 7), K=(40, 64, 100, 33, 120, 64), P_tr=7, P_te=3, n_jam=2)
    return {"C2": c2, "ragged": ragged}


@pytest.mark.parametrize("name", ["C2", "ragged"])
def test_lift_apply_and_pattern(name):
    cfg = _configs()[name]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt)
    plan, off = res.plan, res.off
    N, M, G, Vte = cfg.N, cfg.M, plan.sizes.pairs, plan.sizes.Vte
    c = torch.from_numpy(res.c).cuda()
    c_hat = torch.empty(G * N, dtype=torch.complex64, device="cuda")
    P.bs_lift(plan, c, c_hat)
    xc = torch.from_numpy(res.xc.reshape(-1)).cuda()
    out_l = torch.empty(max(G * Vte, 1), dtype=torch.complex64, device="cuda")
    P.bs_apply_lifted(plan, xc, c_hat, out_l)
    u = torch.linspace(-0.99, 0.99, 67, dtype=torch.float64)
    u[10] = 0.0
    ud = u.cuda()
    pattern = torch.empty(G * len(u), dtype=torch.float32, device="cuda")
    P.bs_beam_pattern(plan, c_hat, ud, pattern)
    torch.cuda.synchronize()
    ch = c_hat.cpu().numpy().reshape(G, N).astype(np.complex128)
    ol = out_l.cpu().numpy()[: G * Vte].reshape(G, Vte)
    pat = pattern.cpu().numpy().reshape(G, len(u))
    B = cfg.B
    worst = {"lift": 0.0, "apply": 0.0, "identity": 0.0, "pattern": 0.0}
    for g in range(G):
        pr = res.pair(g)
        t, s = divmod(g, cfg.L)
        beams = O.window_beams(pr["start"], pr["W"], M)
        ref = O.lifted_correlator(pr["c"].astype(np.complex128), N, M, beams)
        worst["lift"] = max(worst["lift"], rel(ch[g], ref))
        # antenna-space output on the GPU's channelised test vectors
        y = res.xc[cfg.P_tr:, s * B:(s + 1) * B].reshape(Vte, N).astype(np.complex128)
        oref = O.lifted_output(ch[g], y)
        worst["apply"] = max(worst["apply"], rel(ol[g], oref))
        worst["identity"] = max(worst["identity"], rel(ol[g], pr["out"]))
        f = O.subband_center_freq(s, cfg.L, cfg.fc, cfg.fs)
        pref = O.beam_pattern_grid(ch[g], u.numpy(), f, cfg.fd)
        worst["pattern"] = max(worst["pattern"], float(np.abs(pat[g] - pref).max()))
    print(name, {k: f"{v:.2e}" for k, v in worst.items()})
    assert worst["lift"] <= LIFT_TOL
    assert worst["apply"] <= APPLY_TOL
    assert worst["identity"] <= IDENTITY_TOL
    assert worst["pattern"] <= PATTERN_TOL
