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
"""
from __future__ import annotations

import numpy as np
import torch

from . import (BS_PREC_FP32, Plan, _check, _stream, alloc_buffers, bs_beamspace, bs_channelize, bs_mvdr_solve,
               bs_window_cov, lib)


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
    """Mean over pairs of the SINR (dB) for every (M, W) with W <= min(M, 16)."""
    rows = []
    for M in Ms:
        for W in Ws:
            if W > min(M, 16):
                continue
            r = sweep_point(cfg, x, u, W, M, K, device)
            db, db_opt = 10 * np.log10(r["sinr"]), 10 * np.log10(r["sinr_opt"])
            rows.append({"M": M, "W": W, "K": K, "pairs": r["pairs"], "mean_sinr_db": float(np.mean(db)),
                         "mean_reference_mvdr_sinr_db": float(np.mean(db_opt)),
                         "mean_gap_db": float(np.mean(db_opt - db)),
                         "full_dimensional": bool(W == M == cfg.N)})
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
    a = ap.parse_args(argv)
    base = all_configs()[a.config]
    cfg = scaled_config(base, P_tr=max(a.P_train, base.P_tr))
    Ws = [int(v) for v in a.W.split(",")]
    Ms = [int(v) for v in a.M.split(",")] if a.M else [cfg.N, 2 * cfg.N, 4 * cfg.N]
    K = a.K or int(base.K[0])
    sc = make_scene(cfg)
    rows = sinr_sweep(cfg, sc.x, sc.u_tgt, Ws, Ms, K)
    print(json.dumps({"config": a.config, "N": cfg.N, "records_train": cfg.P_tr, "rows": rows}))
    return rows


if __name__ == "__main__":
    main()
