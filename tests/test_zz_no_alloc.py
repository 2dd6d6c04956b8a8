"""The allocation-free entry point bs_cov_solve_noalloc (for callers that may
not allocate device memory while running, and therefore cannot create a
plan): called through the C ABI with caller-provided tables, twice in a row,
its weights match the plan-based bs_cov_solve on the same windows.  Kept in
a file collected last so that a failure here comes after every other test."""
import numpy as np
import pytest
import torch

import paper_2508_11790_gb300 as P
from synth import all_configs, make_scene, scaled_config

SOLVE_TOL = 1e-5


def _tables(plan):
    off = plan.offsets()
    G = plan.sizes.pairs
    dev = "cuda"
    a64 = off["a_tilde"]
    hi = a64.astype(np.complex64)
    lo = (a64 - hi.astype(np.complex128)).astype(np.complex64)
    return off, dict(
        W=torch.from_numpy(off["W"]).to(dev), K=torch.from_numpy(off["K"]).to(dev),
        ztr=torch.from_numpy(off["ztr_off"][:G].copy()).to(dev),
        woff=torch.from_numpy(off["woff"][:G].copy()).to(dev),
        a_hi=torch.from_numpy(hi).to(dev), a_lo=torch.from_numpy(lo).to(dev),
        a_fp=torch.from_numpy(a64).to(dev))


def _config():
    base = all_configs()["C4"]
    rng = np.random.default_rng(9)
    T = 12
    W = tuple(int(w) for w in rng.choice([3, 5, 7, 9, 11, 15, 16, 1], size=T))
    K = tuple(int(rng.integers(max(1, 2 * w), 8 * w + 2)) for w in W)
    return scaled_config(base, name="noalloc", N=128, F=256, L=16, M=256, T=T, W=W, K=K,
                         P_tr=8, P_te=1, n_jam=3)


def test_noalloc_rejects_too_many_pairs():
    """Sizes beyond the fixed scratch are refused before any device work."""
    L = P.lib()
    st = L.bs_cov_solve_noalloc(None, 0, 1.0, None, None, None, None, None, None, None,
                                (1 << 18) + 1, 1.0, 0.0, 0, None, None, None)
    assert st == 1   # BS_EINVAL
    assert b"262144" in L.bs_last_error()


def test_noalloc_zero_pairs_and_bad_loading():
    """pairs == 0 is a no-op; a non-finite or negative loading is refused."""
    L = P.lib()
    assert L.bs_cov_solve_noalloc(None, 0, 1.0, None, None, None, None, None, None, None,
                                  0, 1.0, 0.0, 0, None, None, None) == 0
    for bad in (float("inf"), float("nan"), -1.0):
        assert L.bs_cov_solve_noalloc(None, 0, 1.0, None, None, None, None, None, None, None,
                                      4, bad, 0.0, 0, None, None, None) == 1


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [P.BS_PREC_FP32, P.BS_PREC_FP16])
def test_noalloc_matches_plan_entry_point(precision):
    cfg = _config()
    sc = make_scene(cfg)
    plan = P.Plan.from_scene_config(cfg, sc.u_tgt, precision=precision)
    b = P.alloc_buffers(plan)
    b.x.copy_(torch.from_numpy(sc.x.reshape(-1)))
    P.bs_channelize(plan, b.x, b.xc)
    P.bs_beamspace(plan, b.xc, b.z_train, b.z_test)
    P.bs_cov_solve(plan, b.z_train, b.c, b.info)
    torch.cuda.synchronize()
    c_ref, info_ref = b.c.cpu().numpy().copy(), b.info.cpu().numpy().copy()

    off = plan.offsets()
    G = plan.sizes.pairs
    dev = "cuda"
    W = torch.from_numpy(off["W"]).to(dev)
    K = torch.from_numpy(off["K"]).to(dev)
    ztr = torch.from_numpy(off["ztr_off"][:G].copy()).to(dev)
    woff = torch.from_numpy(off["woff"][:G].copy()).to(dev)
    a64 = off["a_tilde"]
    hi = a64.astype(np.complex64)
    lo = (a64 - hi.astype(np.complex128)).astype(np.complex64)
    a_hi, a_lo = torch.from_numpy(hi).to(dev), torch.from_numpy(lo).to(dev)
    a_fp = torch.from_numpy(a64).to(dev)
    for call in range(2):
        c = torch.full((plan.sizes.c_elems,), float("nan"), dtype=torch.complex64, device=dev)
        info = torch.full((G,), 99, dtype=torch.int32, device=dev)
        P.bs_cov_solve_noalloc(b.z_train, precision, W, K, ztr, woff, a_hi, a_lo, a_fp, cfg.delta, c, info)
        torch.cuda.synchronize()
        cn, inn = c.cpu().numpy(), info.cpu().numpy()
        assert np.array_equal(inn, info_ref), call
        for g in range(G):
            s0, s1 = off["woff"][g], off["woff"][g + 1]
            ref = c_ref[s0:s1]
            err = np.linalg.norm(cn[s0:s1] - ref) / np.linalg.norm(ref)
            assert err <= SOLVE_TOL, (call, g, err)


@pytest.mark.gpu
def test_noalloc_out_of_range_pairs_are_skipped():
    """Pairs whose W is outside 1..16 or whose K is 0 get info = -3 and keep
    their weights untouched; every other pair still matches bs_cov_solve."""
    cfg = _config()
    sc = make_scene(cfg)
    plan = P.Plan.from_scene_config(cfg, sc.u_tgt)
    b = P.alloc_buffers(plan)
    b.x.copy_(torch.from_numpy(sc.x.reshape(-1)))
    P.bs_channelize(plan, b.x, b.xc)
    P.bs_beamspace(plan, b.xc, b.z_train, b.z_test)
    P.bs_cov_solve(plan, b.z_train, b.c, b.info)
    torch.cuda.synchronize()
    c_ref, info_ref = b.c.cpu().numpy().copy(), b.info.cpu().numpy().copy()
    off, tb = _tables(plan)
    G = plan.sizes.pairs
    bad = {3: ("W", 0), 7: ("W", 17), 11: ("K", 0)}
    for g, (name, v) in bad.items():
        tb[name][g] = v
    c = torch.full((plan.sizes.c_elems,), float("nan"), dtype=torch.complex64, device="cuda")
    info = torch.full((G,), 99, dtype=torch.int32, device="cuda")
    P.bs_cov_solve_noalloc(b.z_train, P.BS_PREC_FP32, tb["W"], tb["K"], tb["ztr"], tb["woff"], tb["a_hi"],
                           tb["a_lo"], tb["a_fp"], cfg.delta, c, info)
    torch.cuda.synchronize()
    cn, inn = c.cpu().numpy(), info.cpu().numpy()
    for g in range(G):
        s0, s1 = off["woff"][g], off["woff"][g + 1]
        if g in bad:
            assert inn[g] == -3, g
            assert np.all(np.isnan(cn[s0:s1])), g
        else:
            assert inn[g] == info_ref[g], g
            ref = c_ref[s0:s1]
            assert np.linalg.norm(cn[s0:s1] - ref) / np.linalg.norm(ref) <= SOLVE_TOL, g
