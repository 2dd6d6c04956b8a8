"""GPU parity of the processing after the beamformer: range-Doppler power
maps (synthesis IFFT + matched filter + Doppler DFT) and CFAR detection
against the FP64 oracle on the GPU's own beamformed outputs, and detection
of every target of a coherent pulse-train scene at its delay and Doppler.

Tolerances: map cells within 1e-4 of the target's largest cell (FP32 row
FFTs of F points and a P_test-point DFT); the per-cell noise floors of the
CFAR across velocity bins, computed from the GPU's own map, within 1e-5
relative (plus 1e-7 of the largest cell for floors near zero); CFAR
decisions identical except for cells within 1e-3 of the threshold (the two
sides decide in FP32 and FP64); the strongest detected cell equal to the
oracle's wherever the decision is clear.
"""
import numpy as np
import pytest
import torch

import paper_2508_11790_gb300 as P
from gpu_helpers import run_gpu
from oracle import range_doppler as RD
from synth import all_configs, make_scene, pulse, scaled_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("P_te,T", [(8, 4), (5, 3)])
def test_range_doppler_and_cfar(P_te, T):
    cfg = scaled_config(all_configs()["C1"], name="radar", T=T, W=7, K=64, P_tr=2, P_te=P_te,
                        coherent_targets=True)
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, keep_xc=False)
    plan = res.plan
    F, L, B = cfg.F, cfg.L, cfg.B
    Pspec = np.fft.fft(pulse(F), norm="ortho")
    out = torch.from_numpy(res.out.reshape(-1)).cuda()
    pd = torch.from_numpy(Pspec.astype(np.complex64)).cuda()
    n = T * P_te * F
    work = torch.empty(2 * n, dtype=torch.complex64, device="cuda")
    rd_map = torch.empty(n, dtype=torch.float32, device="cuda")
    P.bs_range_doppler(plan, out, pd, work, rd_map)
    floor = torch.empty(n, dtype=torch.float32, device="cuda")
    count = torch.empty(T, dtype=torch.int32, device="cuda")
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    peak = torch.empty(T, dtype=torch.int32, device="cuda")
    P.bs_cfar(plan, rd_map, 10.0, floor, count, mask, peak)
    torch.cuda.synchronize()
    m = rd_map.cpu().numpy().reshape(T, P_te, F)
    ref = RD.doppler_map(RD.range_profiles(
        RD.beamformed_spectrum(res.out.astype(np.complex128), T, L, B, P_te), Pspec))
    for t in range(T):
        assert np.abs(m[t] - ref[t]).max() <= 1e-4 * ref[t].max(), t
    # the CFAR from the GPU's own map (FP32 cells), decided by the oracle in FP64
    rmask, rfloor = RD.cfar_detect(m.astype(np.float64), 10.0)
    gf = floor.cpu().numpy().reshape(T, P_te, F)
    for t in range(T):
        assert np.all(np.abs(gf[t] - rfloor[t]) <= 1e-5 * rfloor[t] + 1e-7 * m[t].max()), t
    gm = mask.cpu().numpy().reshape(T, P_te, F).astype(bool)
    thr = rfloor * 10.0
    clear = np.abs(m - thr) > 1e-3 * thr
    assert (gm[clear] == rmask[clear]).all()
    assert (count.cpu().numpy() == gm.reshape(T, -1).sum(axis=1)).all()
    det = RD.detection_errors(rmask, m.astype(np.float64), sc.tgt_delay, sc.tgt_doppler)
    pk = peak.cpu().numpy()
    # every target: detected at its own delay and Doppler bin (zero range
    # and velocity error), the strongest detection the GPU reports
    for t in range(T):
        d0, tau0 = int(sc.tgt_doppler[t]), int(sc.tgt_delay[t])
        assert gm[t, d0, tau0], (t, d0, tau0)
        assert det[t] == (True, (d0, tau0), 0, 0), det[t]
        assert pk[t] == d0 * F + tau0, (t, pk[t])


def test_cfar_peak_and_misses_on_a_planted_map():
    """A map with one planted cell per target (at chosen strengths) and a
    flat floor: the peak output is that cell where it clears 10 dB over the
    other velocity bins of its range cell and -1 where it does not; ties
    keep the smaller index."""
    cfg = scaled_config(all_configs()["C1"], name="cfar-plant", T=4, W=5, K=64, P_tr=2, P_te=6)
    plan = P.Plan.from_scene_config(cfg, [0.1, -0.2, 0.3, 0.0])
    T, Pd, F = 4, 6, cfg.F
    m = np.full((T, Pd, F), 2.0, np.float32)
    m[0, 4, 17] = 200.0            # clear
    m[1, 0, F - 1] = 15.0          # below 10 x 2: missed
    m[2, 2, 5] = 80.0; m[2, 3, 9] = 80.0   # tie: the smaller index d F + tau wins
    rd_map = torch.from_numpy(m.reshape(-1)).cuda()
    n = T * Pd * F
    floor = torch.empty(n, dtype=torch.float32, device="cuda")
    count = torch.empty(T, dtype=torch.int32, device="cuda")
    peak = torch.empty(T, dtype=torch.int32, device="cuda")
    P.bs_cfar(plan, rd_map, 10.0, floor, count, None, peak)
    torch.cuda.synchronize()
    assert peak.cpu().tolist() == [4 * F + 17, -1, 2 * F + 5, -1]
    assert count.cpu().tolist() == [1, 0, 2, 0]
