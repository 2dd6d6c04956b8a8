"""GPU parity of the processing after the beamformer: range-Doppler power
maps (synthesis IFFT + matched filter + Doppler DFT) and CFAR detection
against the FP64 oracle on the GPU's own beamformed outputs, and detection
of every target of a coherent pulse-train scene at its delay and Doppler.

Tolerances: map cells within 1e-4 of the target's largest cell (FP32 row
FFTs of F points and a P_test-point DFT); noise floors within 1e-5
relative; CFAR decisions identical except for cells within 1e-3 of the
threshold (the two sides decide in FP32 and FP64).
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
    floor = torch.empty(T, dtype=torch.float32, device="cuda")
    count = torch.empty(T, dtype=torch.int32, device="cuda")
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    P.bs_cfar(plan, rd_map, 10.0, floor, count, mask)
    torch.cuda.synchronize()
    m = rd_map.cpu().numpy().reshape(T, P_te, F)
    ref = RD.doppler_map(RD.range_profiles(
        RD.beamformed_spectrum(res.out.astype(np.complex128), T, L, B, P_te), Pspec))
    for t in range(T):
        assert np.abs(m[t] - ref[t]).max() <= 1e-4 * ref[t].max(), t
    rmask, rfloor = RD.cfar_detect(ref, 10.0)
    np.testing.assert_allclose(floor.cpu().numpy(), rfloor, rtol=1e-5)
    gm = mask.cpu().numpy().reshape(T, P_te, F).astype(bool)
    thr = rfloor[:, None, None] * 10.0
    clear = np.abs(ref - thr) > 1e-3 * thr
    assert (gm[clear] == rmask[clear]).all()
    assert (count.cpu().numpy() == gm.reshape(T, -1).sum(axis=1)).all()
    # every target: detected at its own delay and Doppler bin, the map's peak
    for t in range(T):
        d0, tau0 = int(sc.tgt_doppler[t]), int(sc.tgt_delay[t])
        assert gm[t, d0, tau0], (t, d0, tau0)
        assert np.unravel_index(np.argmax(m[t]), m[t].shape) == (d0, tau0)
