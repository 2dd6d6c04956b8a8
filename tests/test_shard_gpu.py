"""Subband-shard plans on the GPU (bs_config.s_begin / s_count): the plans a
rank runs for its block of subbands reproduce, bit for bit, the same pairs
of the unsharded plan on the same raw records -- channelised bins,
windows, covariances, weights, info and outputs -- and so do the lifted
correlator, its antenna-space output and its beam pattern (each subband's
own centre frequency).  The shards run one after the other on one GPU
(each rank's work, without the ranks).  Both plans take the same covariance
kernel here (few pairs: one CTA per pair), so equality is exact."""
import numpy as np
import pytest
import torch

import paper_2508_11790_gb300 as P
from gpu_helpers import run_gpu
from paper_2508_11790_gb300.shard import shard_plan_blocks
from synth import all_configs, make_scene, scaled_config

pytestmark = pytest.mark.gpu


def _config():
    return scaled_config(all_configs()["C1"], name="shard", N=64, F=512, L=16, M=128, T=3,
                         W=(5, 7, 3), K=(64, 40, 100), P_tr=4, P_te=2, n_jam=2)


@pytest.mark.parametrize("precision", [P.BS_PREC_FP32, P.BS_PREC_FP16])
def test_shards_reproduce_the_full_plan(precision):
    cfg = _config()
    sc = make_scene(cfg)
    kw = {"store_scale": 4.0} if precision != P.BS_PREC_FP32 else {}
    full = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, **kw)
    B, L = cfg.B, cfg.L
    for world in (2, 4, 3):
        for rank in range(world):
            for s0, n in shard_plan_blocks(L, world, rank):
                part = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, s_begin=s0, s_count=n, **kw)
                assert part.plan.sizes.pairs == cfg.T * n
                assert np.array_equal(part.xc, full.xc[:, s0 * B:(s0 + n) * B])
                for t in range(cfg.T):
                    for j in range(n):
                        a, b = part.pair(t * n + j), full.pair(t * L + s0 + j)
                        assert a["start"] == b["start"] and a["info"] == b["info"]
                        for k in ("a", "z_train", "z_test", "R", "c", "out"):
                            assert np.array_equal(a[k], b[k]), (world, rank, t, j, k)


def test_shard_lifted_correlator_and_host_path():
    cfg = _config()
    sc = make_scene(cfg)
    dirs = torch.linspace(-0.9, 0.9, 37, dtype=torch.float64, device="cuda")

    def lifted(**kw):
        plan = P.Plan.from_scene_config(cfg, sc.u_tgt, **kw)
        b = P.alloc_buffers(plan)
        b.x.copy_(torch.from_numpy(sc.x.reshape(-1)))
        P.bs_run(plan, b)
        ch = torch.empty(plan.sizes.pairs * cfg.N, dtype=torch.complex64, device="cuda")
        P.bs_lift(plan, b.c, ch)
        out = torch.empty(max(1, plan.sizes.out_elems), dtype=torch.complex64, device="cuda")
        P.bs_apply_lifted(plan, b.xc, ch, out)
        pat = torch.empty(plan.sizes.pairs * dirs.numel(), dtype=torch.float32, device="cuda")
        P.bs_beam_pattern(plan, ch, dirs, pat)
        # the whole pass from pinned host memory equals bs_run on the shard too
        xh = torch.from_numpy(sc.x.reshape(-1)).pin_memory()
        oh = torch.empty(max(1, plan.sizes.out_elems), dtype=torch.complex64).pin_memory()
        ref_out = b.out.cpu().clone()
        P.bs_run_host(plan, xh, oh, b)
        assert torch.equal(oh[: plan.sizes.out_elems], ref_out[: plan.sizes.out_elems])
        torch.cuda.synchronize()
        assert plan.device_status() == 0
        return (plan, ch.cpu().numpy().reshape(plan.sizes.pairs, cfg.N),
                out.cpu().numpy()[: plan.sizes.out_elems].reshape(plan.sizes.pairs, -1),
                pat.cpu().numpy().reshape(plan.sizes.pairs, -1))

    _, ch_f, out_f, pat_f = lifted()
    s0, n = 8, 4
    plan, ch_s, out_s, pat_s = lifted(s_begin=s0, s_count=n)
    for t in range(cfg.T):
        for j in range(n):
            g, gs = t * cfg.L + s0 + j, t * n + j
            assert np.array_equal(ch_s[gs], ch_f[g])
            assert np.array_equal(out_s[gs], out_f[g])
            assert np.array_equal(pat_s[gs], pat_f[g])
    # the range-Doppler map needs every subband of a target
    work = torch.empty(2 * cfg.T * cfg.P_te * cfg.F, dtype=torch.complex64, device="cuda")
    rmap = torch.empty(cfg.T * cfg.P_te * cfg.F, dtype=torch.float32, device="cuda")
    pulse = torch.zeros(cfg.F, dtype=torch.complex64, device="cuda")
    outs = torch.zeros(plan.sizes.out_elems, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.BsError, match="shard"):
        P.bs_range_doppler(plan, outs, pulse, work, rmap)
