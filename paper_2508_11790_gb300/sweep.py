"""Window-size and zero-padding sweep on a synthetic scene: output SINR of
the windowed beamspace MVDR against W and M (the synthetic analogue of the
paper's window-size comparisons, Sec. IV).

For every (M, W) the library runs the pass on the scene's raw cube (weights
from the first K training vectors of each pair) and judges each pair's
weights c with bs_output_sinr against the reference covariance of the same
window estimated from all target-free training vectors (K_ref = P_tr B,
no loading): SINR = |c^H a~|^2 / (c^H R_ref c).  Beside it: the SINR of
MVDR with the same diagonal loading on the reference covariance, i.e. what
the few-snapshot estimate converges to (without loading that solve is
ill-posed for zero-padded windows, whose beams are nearly linearly
dependent; with it, it is a reference point, not a bound).
Because the beamspace SINR of c equals the antenna-space SINR of its lifted
correlator D^H S^T c (Eq. AntennaEqCorr), the numbers compare across W and
M; with W = M = N the window is the whole unitary beamspace and the point is
full-dimensional antenna MVDR.

    python -m paper_2508_11790_gb300.sweep --config C1 --W 3,5,9,15 --M 64,128,256

Detection (the paper's measure, Sec. IV-B and IV-C: range and velocity
error of CFAR detections against window size and FFT size): on a coherent
pulse-train scene (each target one delay and one Doppler bin over the test
records) the pass, the range-Doppler maps and the 1-D CFAR across velocity
bins run on the GPU for every window; each target's strongest detection is
compared with its true delay and Doppler bin.  Planar windows are given as
W_z x W_x pairs on a planar scene (the paper's 2 x 4, 4 x 4 and 4 x 8 on a
4 x 32 array).

    python -m paper_2508_11790_gb300.sweep --detect --config C1 --W 1,3,5,9,17,32
    python -m paper_2508_11790_gb300.sweep --detect --planar --W 2x4,4x4,4x8 --M 4x32,8x64
"""
from __future__ import annotations

import numpy as np
import torch

from . import (BS_PREC_FP32, Plan, _check, _stream, alloc_buffers, bs_beamspace, bs_cfar, bs_channelize,
               bs_mvdr_solve, bs_range_doppler, bs_run, bs_window_cov, lib)


def sweep_point(cfg, x: np.ndarray, u, W: int, M: int, K: int, device="cuda") -> dict:
    """Per-pair SINR (linear) of the K-snapshot weights and of MVDR on the
    loaded reference covariance, for window size W and spatial FFT size M."""
    T = len(u)
    B = cfg.F // cfg.L
    K_ref = cfg.P_tr * B
    common = dict(N=cfg.N, F=cfg.F, L=cfg.L, M=M, u=list(u), W=[W] * T, P_train=cfg.P_tr, P_test=cfg.P_te,
                  fc=cfg.fc, fs=cfg.fs, fd=cfg.fd, delta=cfg.delta, precision=BS_PREC_FP32)
    ps = Plan(K=[K] * T, **common)
    pr = Plan(K=[K_ref] * T, **common)
    b = alloc_buffers(ps, device)
    b.x.copy_(torch.from_numpy(np.ascontiguousarray(x).reshape(-1)))
    G = ps.sizes.pairs
    ztr_r = torch.empty(pr.sizes.ztrain_elems, dtype=torch.complex64, device=device)
    Rr = torch.empty(pr.sizes.r_elems, dtype=torch.complex128, device=device)
    bs_channelize(ps, b.x, b.xc)
    bs_beamspace(ps, b.xc, b.z_train, b.z_test)
    bs_beamspace(pr, b.xc, ztr_r, b.z_test)
    bs_window_cov(ps, b.z_train, b.R)
    bs_mvdr_solve(ps, b.R, b.c, b.info)
    bs_window_cov(pr, ztr_r, Rr, delta_pair=torch.zeros(G, dtype=torch.float32, device=device))
    L = lib()
    sinr = torch.empty(G, dtype=torch.float64, device=device)
    _check(L.bs_output_sinr(ps.handle, b.c.data_ptr(), Rr.data_ptr(), sinr.data_ptr(), _stream(None)),
           "bs_output_sinr")
    Rl = torch.empty_like(Rr)
    bs_window_cov(pr, ztr_r, Rl)   # the plan's loading
    c_opt = torch.empty_like(b.c)
    info_opt = torch.empty_like(b.info)
    bs_mvdr_solve(ps, Rl, c_opt, info_opt)
    sinr_opt = torch.empty(G, dtype=torch.float64, device=device)
    _check(L.bs_output_sinr(ps.handle, c_opt.data_ptr(), Rr.data_ptr(), sinr_opt.data_ptr(), _stream(None)),
           "bs_output_sinr")
    torch.cuda.synchronize()
    return {"sinr": sinr.cpu().numpy(), "sinr_opt": sinr_opt.cpu().numpy(), "info": b.info.cpu().numpy(),
            "info_opt": info_opt.cpu().numpy(), "pairs": G}


def sinr_sweep(cfg, x: np.ndarray, u, Ws, Ms, K: int, device="cuda") -> list:
    """Mean over pairs of the SINR (dB) for every (M, W) with W <= min(M, 32)."""
    rows = []
    for M in Ms:
        for W in Ws:
            if W > min(M, 32):
                continue
            r = sweep_point(cfg, x, u, W, M, K, device)
            db, db_opt = 10 * np.log10(r["sinr"]), 10 * np.log10(r["sinr_opt"])
            rows.append({"M": M, "W": W, "K": K, "pairs": r["pairs"], "mean_sinr_db": float(np.mean(db)),
                         "mean_reference_mvdr_sinr_db": float(np.mean(db_opt)),
                         "mean_gap_db": float(np.mean(db_opt - db)),
                         "full_dimensional": bool(W == M == cfg.N)})
    return rows


def detection_point(cfg, x: np.ndarray, u, delay, doppler, pulse_spectrum: np.ndarray, W: int, M: int,
                    K: int, Wz: int = 1, Mz: int = 1, v=None, threshold_db: float = 10.0, device="cuda") -> dict:
    """Detections of one window / FFT size on a coherent scene: the pass
    (bs_run), each target's range-Doppler map (bs_range_doppler) and the
    CFAR across velocity bins (bs_cfar).  W is the whole window (W_x W_z for
    a planar array, Wz its vertical part), M the whole FFT size (M_x M_z).
    Per target: detected, the strongest detection's range bin and velocity
    bin, and their signed errors against the truth (velocity modulo P_te
    into [-P_te/2, P_te/2))."""
    T = len(u)
    kw = dict(N=cfg.N, F=cfg.F, L=cfg.L, M=M, u=list(u), W=[W] * T, K=[K] * T, P_train=cfg.P_tr,
              P_test=cfg.P_te, fc=cfg.fc, fs=cfg.fs, fd=cfg.fd, delta=cfg.delta, precision=BS_PREC_FP32)
    if Mz > 1 or getattr(cfg, "Nz", 1) > 1:
        kw.update(Nz=cfg.Nz, Mz=Mz, Wz=[Wz] * T, v=list(v))
    plan = Plan(**kw)
    b = alloc_buffers(plan, device)
    b.x.copy_(torch.from_numpy(np.ascontiguousarray(x).reshape(-1)))
    bs_run(plan, b)
    P_te, F = cfg.P_te, cfg.F
    n = T * P_te * F
    work = torch.empty(2 * n, dtype=torch.complex64, device=device)
    rmap = torch.empty(n, dtype=torch.float32, device=device)
    pd = torch.from_numpy(np.asarray(pulse_spectrum, np.complex64)).to(device)
    bs_range_doppler(plan, b.out, pd, work, rmap)
    floor = torch.empty(n, dtype=torch.float32, device=device)
    count = torch.empty(T, dtype=torch.int32, device=device)
    peak = torch.empty(T, dtype=torch.int32, device=device)
    bs_cfar(plan, rmap, threshold_db, floor, count, None, peak)
    torch.cuda.synchronize()
    pk = peak.cpu().numpy()
    rows = []
    for t in range(T):
        if pk[t] < 0:
            rows.append({"detected": False, "range_bin": None, "velocity_bin": None,
                         "range_error": None, "velocity_error": None})
            continue
        d, tau = divmod(int(pk[t]), F)
        dv = (d - int(doppler[t]) + P_te // 2) % P_te - P_te // 2
        rows.append({"detected": True, "range_bin": tau, "velocity_bin": d,
                     "range_error": tau - int(delay[t]), "velocity_error": dv})
    return {"targets": rows, "detections": count.cpu().numpy(), "info": b.info.cpu().numpy()}


def detection_sweep(cfg, x: np.ndarray, u, delay, doppler, pulse_spectrum, windows, ffts, K: int,
                    v=None, device="cuda") -> list:
    """Detection against window and FFT size: windows as W (linear) or
    (W_z, W_x) pairs, FFT sizes as M or (M_z, M_x) pairs; one row per
    (FFT size, window) that fits.  A target counts as detected exactly when
    its strongest detection has zero range and velocity error."""
    rows = []
    for ff in ffts:
        Mz, Mx = (ff if isinstance(ff, tuple) else (1, ff))
        for win in windows:
            Wz, Wx = (win if isinstance(win, tuple) else (1, win))
            if Wx > Mx or Wz > Mz or Wx * Wz > 32:
                continue
            r = detection_point(cfg, x, u, delay, doppler, pulse_spectrum, Wx * Wz, Mx * Mz, K, Wz=Wz, Mz=Mz,
                                v=v, device=device)
            tg = r["targets"]
            det = [t for t in tg if t["detected"]]
            exact = [t for t in det if t["range_error"] == 0 and t["velocity_error"] == 0]
            rows.append({"window": f"{Wz}x{Wx}" if Mz > 1 else str(Wx), "fft": f"{Mz}x{Mx}" if Mz > 1 else str(Mx),
                         "targets": len(tg), "detected": len(det), "exact": len(exact),
                         "missed": [i for i, t in enumerate(tg) if not t["detected"]],
                         "mean_abs_range_error": float(np.mean([abs(t["range_error"]) for t in det])) if det else None,
                         "mean_abs_velocity_error": (float(np.mean([abs(t["velocity_error"]) for t in det]))
                                                     if det else None)})
    return rows


def main(argv=None) -> list:
    import argparse
    import json

    from synth import all_configs, make_scene, scaled_config
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--config", default="C1")
    ap.add_argument("--W", default="3,5,7,9,11,13,15")
    ap.add_argument("--M", default="")
    ap.add_argument("--K", type=int, default=0, help="training vectors of the weights (default: the config's)")
    ap.add_argument("--P-train", type=int, default=16, help="target-free records (reference covariance)")
    ap.add_argument("--detect", action="store_true", help="detection sweep on a coherent pulse-train scene")
    ap.add_argument("--planar", action="store_true", help="the paper's 4 x 32 planar array (with --detect)")
    ap.add_argument("--snr", type=float, default=-20.0, help="per-element target SNR, dB (with --detect)")
    ap.add_argument("--targets", type=int, default=8, help="targets of the detection scene")
    ap.add_argument("--jammers", type=int, default=6, help="jammers of the detection scene (40-60 dB JNR)")
    a = ap.parse_args(argv)
    if a.detect:
        return _detect_main(a)
    base = all_configs()[a.config]
    cfg = scaled_config(base, P_tr=max(a.P_train, base.P_tr))
    Ws = [int(v) for v in a.W.split(",")]
    Ms = [int(v) for v in a.M.split(",")] if a.M else [cfg.N, 2 * cfg.N, 4 * cfg.N]
    K = a.K or int(base.K[0])
    sc = make_scene(cfg)
    rows = sinr_sweep(cfg, sc.x, sc.u_tgt, Ws, Ms, K)
    print(json.dumps({"config": a.config, "N": cfg.N, "records_train": cfg.P_tr, "rows": rows}))
    return rows


def detection_scene(config: str = "C1", planar: bool = False, snr_db: float = -20.0, T: int = 8, P_te: int = 8,
                    n_jam: int = 6):
    """A coherent pulse-train scene for the detection sweep: the config's
    linear array (or the paper's 4 x 32 planar array with 16 subbands),
    T targets at snr_db per element, n_jam jammers at 40-60 dB JNR."""
    from synth import all_configs, make_scene, scaled_config
    base = all_configs()[config]
    if planar:
        cfg = scaled_config(base, name="detect-4x32", N=128, Nz=4, M=128, Mz=4, F=512, L=16, T=T, W=4, Wz=2,
                            K=64, P_tr=8, P_te=P_te, n_jam=n_jam, jnr_db=(40.0, 60.0), snr_db=snr_db,
                            coherent_targets=True)
    else:
        cfg = scaled_config(base, name="detect", T=T, W=5, K=int(base.K[0]), P_te=P_te, n_jam=n_jam,
                            jnr_db=(40.0, 60.0), snr_db=snr_db, coherent_targets=True)
    return cfg, make_scene(cfg)


def _detect_main(a) -> list:
    import json

    from synth import pulse
    cfg, sc = detection_scene(a.config, a.planar, a.snr, T=a.targets, n_jam=a.jammers)
    ps = np.fft.fft(pulse(cfg.F), norm="ortho")   # the transmitted pulse's spectrum: an input of range processing

    def pairs(text):
        out = []
        for v in text.split(","):
            out.append(tuple(int(w) for w in v.split("x")) if "x" in v else int(v))
        return out
    windows = pairs(a.W) if a.W != "3,5,7,9,11,13,15" else ([(2, 4), (4, 4), (4, 8)] if a.planar else
                                                            [1, 3, 5, 9, 17, 32])
    ffts = pairs(a.M) if a.M else ([(4, 32), (8, 64)] if a.planar else [cfg.N, 2 * cfg.N, 4 * cfg.N])
    K = a.K or int(cfg.K[0])
    rows = detection_sweep(cfg, sc.x, sc.u_tgt, sc.tgt_delay, sc.tgt_doppler, ps, windows, ffts, K,
                           v=sc.v_tgt)
    print(json.dumps({"config": cfg.name, "N": cfg.N, "targets": cfg.T, "snr_db": cfg.snr_db,
                      "jnr_db": list(cfg.jnr_db), "rows": rows}))
    return rows


if __name__ == "__main__":
    main()
