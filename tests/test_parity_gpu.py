"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances, from the arithmetic:
* FFT stages (FP32, unitary, radix 16/8/4/2 with correctly rounded twiddle
  tables): error of one transform ~ eps32 * c * log2(n) * ||x|| with
  eps32 = 6e-8; bound the norm-wise relative error of each transform by
  FFT_TOL = 5e-6 (n <= 4096).
* covariance: FP32 products in blocks of <= 16 combined in double-float, so
  every entry is within a few eps32 of the FP64 sum of the same inputs,
  relative to the largest entry: COV_TOL = 1e-6.
* solve of the GPU's own R: FP32 Cholesky + one FP64-residual refinement
  step (or FP64): SOLVE_TOL = 1e-5 (norm-wise, per pair).
* end to end, weights against the oracle's FP64 pipeline: the stated target
  WEIGHT_TOL = 1e-3 per pair and SINR_TOL_DB = 0.1 dB per pair.
* outputs c^H y: OUT_TOL = 2e-3 norm-wise per pair (weights error plus
  FP32 windows).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_11790_gb300 as P
from synth import all_configs, make_scene, reference_records, scaled_config
from gpu_helpers import GpuResult, rel, run_gpu, ztrain_to_complex

pytestmark = pytest.mark.gpu

FFT_TOL = 5e-6
COV_TOL = 1e-6
SOLVE_TOL = 1e-5
WEIGHT_TOL = 1e-3
SINR_TOL_DB = 0.1
OUT_TOL = 2e-3


def ragged_config():
    """N not a multiple of the 8-column tile, W in {1, 16, even}, K < W, K = 1."""
    base = all_configs()["C1"]
    return scaled_config(base, name="ragged", N=100, F=256, L=8, M=128, T=5,
                         W=(1, 16, 5, 4, 9), K=(1, 3, 40, 64, 200), P_tr=7, P_te=3,
                         n_jam=2, jnr_db=(25.0, 35.0))


def check_end_to_end(cfg, sc, res, subbands=None, weight_tol=WEIGHT_TOL, check_out=True, P_ref=None):
    """Weights, SINR loss and outputs of every (selected) pair against the
    oracle's FP64 pipeline on the same raw data.

    The SINR loss 10 log10(SINR(c_oracle) / SINR(c_gpu)) is judged twice:
    against the oracle's loaded sample covariance of the same training
    windows (both sides solve with that matrix, so the loss isolates the GPU
    arithmetic; it is second order in the weight error), and against an
    interference-plus-noise covariance estimated from P_ref independent
    target-free records of the same scene (reference_records), which the
    weights never saw, so that the loss is first order in the weight error
    and measures the suppression of the scene's interference.  Returns
    (max weight error, max |loss| sample, max |loss| reference)."""
    ref = O.run_pipeline(sc.x, cfg, sc.u_tgt, subbands=subbands)
    if P_ref is None:
        P_ref = max(4, min(16, cfg.P_tr))
    R_in = O.reference_covariances(reference_records(cfg, P_ref), cfg, sc.u_tgt, subbands=subbands)
    worst = 0.0
    worst_loss = 0.0
    worst_ref = 0.0
    for k in range(len(ref.pairs.t)):
        g = int(ref.pairs.t[k]) * cfg.L + int(ref.pairs.s[k])
        pr = res.pair(g)
        assert pr["start"] == int(ref.pairs.start[k])
        assert pr["info"] in (0, -2), (g, pr["info"])
        np.testing.assert_allclose(pr["a"], ref.pairs.a_tilde[k], rtol=0, atol=1e-12 * max(1.0, np.abs(ref.pairs.a_tilde[k]).max()))
        e = rel(pr["c"], ref.c[k])
        cg = pr["c"].astype(np.complex128)
        loss = O.sinr_loss_db(cg, ref.c[k], ref.pairs.a_tilde[k], ref.R[k])
        loss_ref = O.sinr_loss_db(cg, ref.c[k], ref.pairs.a_tilde[k], R_in[k])
        worst, worst_loss, worst_ref = max(worst, e), max(worst_loss, abs(loss)), max(worst_ref, abs(loss_ref))
        assert e <= weight_tol, (g, e)
        assert abs(loss) <= SINR_TOL_DB, (g, loss)
        assert abs(loss_ref) <= SINR_TOL_DB, (g, loss_ref)
        if check_out and cfg.P_te:
            assert rel(pr["out"], ref.out[k]) <= OUT_TOL, g
    return worst, worst_loss, worst_ref


def check_stages(cfg, sc, res):
    """Each stage against the oracle applied to the GPU's input of that stage."""
    # channelise: all records, every element column
    Xo = O.channelize(sc.x, cfg.L).reshape(cfg.P, cfg.F, cfg.N)
    err = np.linalg.norm(res.xc - Xo, axis=1) / np.maximum(np.linalg.norm(Xo, axis=1), 1e-30)
    assert err.max() <= FFT_TOL, err.max()
    # beamspace + window, from the GPU's channelised data
    yb = O.beamspace(res.xc.astype(np.complex128), cfg.M)        # [P][F][M]
    B = cfg.B
    for g in range(res.plan.sizes.pairs):
        pr = res.pair(g)
        t, s = divmod(g, cfg.L)
        beams = O.window_beams(pr["start"], pr["W"], cfg.M)
        zall = yb[:, s * B:(s + 1) * B][:, :, beams].reshape(cfg.P * B, pr["W"])
        ztr = zall[: pr["K"]]
        zte = zall[cfg.P_tr * B:]
        scale = np.linalg.norm(yb[:, s * B:(s + 1) * B], axis=-1).max()
        assert np.abs(pr["z_train"] - ztr).max() <= FFT_TOL * scale
        if cfg.P_te:
            assert np.abs(pr["z_test"] - zte).max() <= FFT_TOL * scale
        # covariance from the GPU's own windows
        Ro = O.window_covariance(pr["z_train"].astype(np.complex128), cfg.delta)
        assert np.abs(pr["R"] - Ro).max() <= COV_TOL * np.abs(Ro).max(), g
        np.testing.assert_allclose(pr["R"], pr["R"].conj().T, atol=0)
        # solve from the GPU's own covariance
        co = O.mvdr_weights(pr["R"], pr["a"])
        assert rel(pr["c"], co) <= SOLVE_TOL, (g, rel(pr["c"], co))
        # apply
        if cfg.P_te:
            oo = O.beamformer_output(pr["c"].astype(np.complex128), pr["z_test"])
            assert rel(pr["out"], oo) <= 1e-5, g


@pytest.fixture(scope="module")
def c1():
    cfg = all_configs()["C1"]
    sc = make_scene(cfg)
    return cfg, sc, run_gpu(cfg, sc.x, sc.u_tgt)


def test_c1_stages(c1):
    cfg, sc, res = c1
    check_stages(cfg, sc, res)


def test_c1_end_to_end(c1):
    cfg, sc, res = c1
    check_end_to_end(cfg, sc, res)


def test_ragged_stages_and_end_to_end():
    cfg = ragged_config()
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt)
    check_stages(cfg, sc, res)
    check_end_to_end(cfg, sc, res)


def test_c2_end_to_end():
    cfg = all_configs()["C2"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, keep_xc=False)
    worst, loss, lref = check_end_to_end(cfg, sc, res)
    print(f"C2 FP32: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), {lref:.2e} dB (reference R)")


def test_c2_fp16_windows():
    """FP16 training windows (tensor-core covariance inputs) meet the weight
    and SINR targets on C2."""
    cfg = all_configs()["C2"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=P.BS_PREC_FP16, keep_xc=False)
    worst, loss, lref = check_end_to_end(cfg, sc, res)
    print(f"C2 FP16: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), {lref:.2e} dB (reference R)")


def test_c2_bf16_windows_sinr():
    """BF16 windows keep the SINR loss within 0.1 dB but their 8-bit
    mantissa misses the 1e-3 weight target on some pairs (reported)."""
    cfg = all_configs()["C2"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=P.BS_PREC_BF16, keep_xc=False)
    worst, loss, lref = check_end_to_end(cfg, sc, res, weight_tol=2e-2, check_out=False)
    print(f"C2 BF16: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), {lref:.2e} dB (reference R)")


def test_plain_path_c2():
    """The plain FP32 per-pair path (benchmark baseline) on C2: SINR within
    target; its weight error is reported."""
    cfg = all_configs()["C2"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, flags=P.BS_FLAG_PLAIN, keep_xc=False)
    worst, loss, lref = check_end_to_end(cfg, sc, res, weight_tol=1e-2, check_out=False)
    print(f"C2 plain FP32: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), {lref:.2e} dB (reference R)")


@pytest.mark.parametrize("N,M", [(1, 16), (16, 16), (100, 128), (1024, 2048), (700, 4096), (64, 64)])
def test_beamspace_full(N, M):
    rng = np.random.default_rng(N + M)
    nvec = 37
    y = (rng.standard_normal((nvec, N)) + 1j * rng.standard_normal((nvec, N))).astype(np.complex64)
    plan = P.Plan(N=N, F=64, L=4, M=M, u=[0.1], W=[1], K=[1], P_train=1, P_test=0,
                  fc=10e9, fs=1e9, fd=10e9, delta=1.0)
    yd = torch.from_numpy(y.reshape(-1)).cuda()
    yb = torch.empty(nvec * M, dtype=torch.complex64, device="cuda")
    P.bs_beamspace_full(plan, yd, yb, nvec)
    torch.cuda.synchronize()
    got = yb.cpu().numpy().reshape(nvec, M)
    ref = O.beamspace(y, M)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= FFT_TOL


@pytest.mark.parametrize("F,N", [(16, 1), (64, 7), (512, 33), (4096, 12), (2048, 9),
                                 (2048, 10), (1024, 6), (512, 34), (2048, 1024)])
def test_channelize_sizes(F, N):
    """Odd N takes the plain kernel; even N with F in 512..2048 the persistent
    TMA-staged kernel (ragged last column tile when N % 4 != 0)."""
    rng = np.random.default_rng(F + N)
    Pn, L = 3, min(F, 16)
    x = (rng.standard_normal((Pn, F, N)) + 1j * rng.standard_normal((Pn, F, N))).astype(np.complex64)
    plan = P.Plan(N=N, F=F, L=L, M=max(16, 1 << (N - 1).bit_length()), u=[0.0], W=[1], K=[1],
                  P_train=Pn, P_test=0, fc=10e9, fs=1e9, fd=10e9, delta=1.0)
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    xc = torch.empty_like(xd)
    P.bs_channelize(plan, xd, xc, P=Pn)
    torch.cuda.synchronize()
    got = xc.cpu().numpy().reshape(Pn, F, N)
    assert plan.device_status() == 0
    ref = O.channelize(x, L).reshape(Pn, F, N)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= FFT_TOL


def test_channelize_tma_matches_plain_kernel():
    """The TMA-staged persistent channeliser and the plain one do the same
    arithmetic in the same order: identical bits."""
    rng = np.random.default_rng(11)
    Pn, F, N = 5, 2048, 1022
    x = (rng.standard_normal((Pn, F, N)) + 1j * rng.standard_normal((Pn, F, N))).astype(np.complex64)
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    outs = []
    for flags in (0, P.BS_FLAG_NO_TMA):
        plan = P.Plan(N=N, F=F, L=128, M=1024, u=[0.0], W=[1], K=[1], P_train=Pn, P_test=0,
                      fc=10e9, fs=1e9, fd=10e9, delta=1.0, flags=flags)
        xc = torch.empty_like(xd)
        P.bs_channelize(plan, xd, xc, P=Pn)
        torch.cuda.synchronize()
        assert plan.device_status() == 0
        outs.append(xc.cpu())
    assert torch.equal(outs[0], outs[1])


def _solve_only(R_list, a_list, **plan_kw):
    """Run bs_mvdr_solve on given covariances (one target, L pairs)."""
    L = len(R_list)
    W = R_list[0].shape[0]
    plan = P.Plan(N=16, F=16 * L, L=L, M=16, u=[0.0], W=[W], K=[1], P_train=1, P_test=0,
                  fc=10e9, fs=1e9, fd=10e9, delta=1.0, **plan_kw)
    off = plan.offsets()
    R = torch.from_numpy(np.concatenate([r.reshape(-1) for r in R_list]).astype(np.complex128)).cuda()
    c = torch.empty(plan.sizes.c_elems, dtype=torch.complex64, device="cuda")
    info = torch.empty(plan.sizes.pairs, dtype=torch.int32, device="cuda")
    P.bs_mvdr_solve(plan, R, c, info)
    torch.cuda.synchronize()
    return off, c.cpu().numpy(), info.cpu().numpy()


def test_solve_info_codes():
    """info: -1 non-finite input, k+1 for a non-positive pivot, -2 for an
    FP64 escalation of an ill-conditioned pair; 0 otherwise."""
    rng = np.random.default_rng(3)
    W = 6
    Q, _ = np.linalg.qr(rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W)))
    good = (Q * np.array([1, 2, 3, 4, 5, 6.0])) @ Q.conj().T
    illc = (Q * np.array([1, 1e3, 1e5, 1e6, 1e7, 1e8])) @ Q.conj().T
    nan = good.copy(); nan[2, 3] = np.nan
    notpd = good.copy(); notpd[0, 0] = -1.0
    Rs = [good, illc, nan, notpd]
    off, c, info = _solve_only(Rs, None)
    assert list(info) == [0, -2, -1, 1]
    at = off["a_tilde"]
    for g in (0, 1):
        a = at[off["woff"][g]:off["woff"][g + 1]]
        co = O.mvdr_weights(Rs[g], a)
        assert rel(c[off["woff"][g]:off["woff"][g + 1]], co) <= SOLVE_TOL
    assert np.isnan(c[off["woff"][2]:off["woff"][3]]).all()
    assert np.isnan(c[off["woff"][3]:off["woff"][4]]).all()


def test_solve_scale_invariance_and_split_edges():
    """MVDR weights do not change when R is scaled (Eq. BeamCorrMVDR): the
    solve reads its FP64 covariance through an integer-operation hi/lo split,
    so scales 2^-40 .. 2^40 (the FP32 solve's range: a^H R^-1 a is squared in
    FP32), entries whose low mantissa bits round the high part up into the
    next binade, and an infinite entry (info -1) are checked against the
    oracle."""
    rng = np.random.default_rng(17)
    W = 7
    Q, _ = np.linalg.qr(rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W)))
    base = (Q * np.linspace(1.0, 30.0, W)) @ Q.conj().T
    # diagonal 2^24 - 2^-29 ... : the FP32 high part rounds up to a power of two
    edge = base.copy()
    edge[np.arange(W), np.arange(W)] += 2.0 ** 24 - 2.0 ** -28 - np.real(np.diag(base)).max()
    scales = [2.0 ** -40, 2.0 ** -17, 1.0, 3.0 ** 20, 2.0 ** 35, 2.0 ** 40]
    inf = base.copy(); inf[1, 1] = np.inf
    Rs = [base * sc_ for sc_ in scales] + [edge, inf]
    off, c, info = _solve_only(Rs, None)
    assert list(info[:-1]) == [0] * (len(Rs) - 1) and info[-1] == -1
    at = off["a_tilde"]
    for g in range(len(Rs) - 1):
        a = at[off["woff"][g]:off["woff"][g + 1]]
        co = O.mvdr_weights(Rs[g], a)
        assert rel(c[off["woff"][g]:off["woff"][g + 1]], co) <= SOLVE_TOL, (g, rel(c[off["woff"][g]:off["woff"][g + 1]], co))


@pytest.mark.parametrize("name,precision,records", [("C1", P.BS_PREC_FP32, None), ("C2", P.BS_PREC_FP16, None),
                                                    ("C2", P.BS_PREC_FP32, (13, 6)), ("C1", P.BS_PREC_FP32, (3, 0)),
                                                    ("C1", P.BS_PREC_FP16, (2, 1)), ("C2", P.BS_PREC_FP32, (5, 2))])
def test_run_host_matches_run(name, precision, records):
    """bs_run_host pipelines the host copy with channelisation and beamspace
    in record chunks that end at P_train (covariance and solve then run
    under the copy of the test records; the last chunk is one record):
    training-record counts below and above the chunk count, 0, 1, 2 and
    more test records; every intermediate and the output equal bs_run's
    bit for bit."""
    cfg = all_configs()[name]
    if records:
        cfg = scaled_config(cfg, P_tr=records[0], P_te=records[1], K=min(cfg.K[0], records[0] * cfg.B))
    sc = make_scene(cfg)
    plan = P.Plan.from_scene_config(cfg, sc.u_tgt, precision=precision)
    b = P.alloc_buffers(plan)
    keys = ("xc", "z_train", "z_test", "R", "c", "out")
    for k in keys:   # parts a pass does not write (no test records) compare as zeros
        getattr(b, k).zero_()
    b.x.copy_(torch.from_numpy(sc.x.reshape(-1)))
    P.bs_run(plan, b)
    torch.cuda.synchronize()
    ref = {k: getattr(b, k).cpu().clone() for k in keys}
    xh = torch.from_numpy(sc.x.reshape(-1)).pin_memory()
    oh = torch.empty(max(1, plan.sizes.out_elems), dtype=torch.complex64).pin_memory()
    for k in ref:
        getattr(b, k).zero_()
    b.x.zero_()
    P.bs_run_host(plan, xh, oh, b)
    assert plan.device_status() == 0
    assert torch.equal(oh[: plan.sizes.out_elems], ref["out"][: plan.sizes.out_elems])
    for k in ref:
        assert torch.equal(getattr(b, k).cpu(), ref[k]), k


def test_no_test_records_and_single_subband_bins():
    """P_test = 0 (no test windows, apply is a no-op) and B = 1 (L = F)."""
    base = all_configs()["C1"]
    cfg = scaled_config(base, name="degenerate", F=64, L=64, T=2, W=(3, 1), K=(4, 2),
                        P_tr=4, P_te=0, N=20, M=32)
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt)
    check_end_to_end(cfg, sc, res)


@pytest.mark.parametrize("precision", [P.BS_PREC_FP32, P.BS_PREC_FP16])
def test_full_size_c3_sampled(precision):
    """The benchmark workload (N=1024, F=2048, L=128, M=2048, W=9, K=512,
    T=64) through bs_run at full size; the oracle checks 4 subbands x 64
    targets = 256 pairs."""
    cfg = all_configs()["C3"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, keep_xc=False)
    assert set(np.unique(res.info)).issubset({0, -2})
    worst, loss, lref = check_end_to_end(cfg, sc, res, subbands=[0, 37, 64, 127])
    print(f"C3 prec={precision}: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), {lref:.2e} dB (reference R)")


def uneven_small_config():
    """C4-like: uneven W in {3,5,7,9,11,15} and K in [2W, 8W], scaled down."""
    base = all_configs()["C4"]
    rng = np.random.default_rng(5)
    T = 24
    W = tuple(int(w) for w in rng.choice([3, 5, 7, 9, 11, 15], size=T))
    K = tuple(int(rng.integers(2 * w, 8 * w + 1)) for w in W)
    return scaled_config(base, name="uneven-small", N=256, F=512, L=16, M=512, T=T, W=W, K=K,
                         P_tr=8, P_te=2, n_jam=4)


@pytest.mark.parametrize("precond", [False, True])
def test_escalation_every_pair(precond):
    """Stand-alone solve with every pair escalated (kappa_max just above 1):
    1536 pairs, W from 2 to 16 in both lane-group widths, each solved again
    on the escalation path.  Weights against the oracle's FP64 solve of the
    GPU's own covariances (Eq. BeamCorrMVDR; with a diagonal preconditioner
    the same weights in exact arithmetic), info -2."""
    base = all_configs()["C4"]
    rng = np.random.default_rng(11)
    T = 24
    W = tuple(int(w) for w in rng.choice([2, 3, 5, 8, 9, 12, 16], size=T))
    K = tuple(int(rng.integers(2 * w, 6 * w + 1)) for w in W)
    cfg = scaled_config(base, name="escalate-all", N=256, F=1024, L=64, M=512, T=T, W=W, K=K, P_te=1, n_jam=4)
    sc = make_scene(cfg)
    plan = P.Plan.from_scene_config(cfg, sc.u_tgt, kappa_max=1.0001)
    assert plan.sizes.pairs == 1536
    b = P.alloc_buffers(plan)
    b.x.copy_(torch.from_numpy(sc.x.reshape(-1)))
    P.bs_channelize(plan, b.x, b.xc)
    P.bs_beamspace(plan, b.xc, b.z_train, b.z_test)
    P.bs_window_cov(plan, b.z_train, b.R)
    b.info.fill_(99)
    off = plan.offsets()
    if precond:
        d = (2.0 ** np.random.default_rng(12).uniform(-6, 6, size=plan.sizes.c_elems)).astype(np.float32)
        P.bs_mvdr_solve_precond(plan, b.R, torch.from_numpy(d).cuda(), b.c, b.info)
    else:
        P.bs_mvdr_solve(plan, b.R, b.c, b.info)
    torch.cuda.synchronize()
    R, c, info = b.R.cpu().numpy(), b.c.cpu().numpy(), b.info.cpu().numpy()
    assert (info == -2).all(), np.unique(info, return_counts=True)
    worst = 0.0
    for g in range(plan.sizes.pairs):
        Wg = int(off["W"][g])
        Rg = R[off["roff"][g]:off["roff"][g + 1]].reshape(Wg, Wg)
        a = off["a_tilde"][off["woff"][g]:off["woff"][g + 1]]
        worst = max(worst, rel(c[off["woff"][g]:off["woff"][g + 1]], O.mvdr_weights(Rg, a)))
    assert worst <= SOLVE_TOL, worst


@pytest.mark.parametrize("precision", [P.BS_PREC_FP32, P.BS_PREC_FP16])
def test_fused_cov_solve_matches_unfused(precision):
    """bs_cov_solve (persistent, work queue) against bs_window_cov +
    bs_mvdr_solve on the same windows, uneven W and K."""
    cfg = uneven_small_config()
    sc = make_scene(cfg)
    out = {}
    for flags in (0, P.BS_FLAG_FUSED):
        res = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, flags=flags, keep_xc=False)
        out[flags] = res
    a, b = out[0], out[P.BS_FLAG_FUSED]
    assert np.array_equal(a.z_train, b.z_train)
    np.testing.assert_allclose(a.R, b.R, rtol=0, atol=1e-6 * np.abs(b.R).max())
    # the two kernels sum in different orders: agreement within the sum of
    # their errors against the oracle (each far below the 1e-3 target)
    worst = 0.0
    for g in range(a.plan.sizes.pairs):
        pa, pb = a.pair(g), b.pair(g)
        assert pa["info"] == pb["info"]
        worst = max(worst, rel(pa["c"], pb["c"]))
    print(f"fused vs unfused (prec {precision}): max weight difference {worst:.2e}")
    assert worst <= 2e-4


def test_uneven_end_to_end():
    cfg = uneven_small_config()
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, flags=P.BS_FLAG_FUSED, keep_xc=False)
    worst, loss, lref = check_end_to_end(cfg, sc, res)
    print(f"uneven-small FP32: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), {lref:.2e} dB (reference R)")


def test_full_size_c4_sampled():
    """The batched-uneven workload at full size (N=1024, 256 targets, W in
    {3..15}, K in [2W, 8W], 32768 pairs) through bs_run with the fused
    persistent kernel; the oracle checks 2 subbands x 256 targets."""
    cfg = all_configs()["C4"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, flags=P.BS_FLAG_FUSED, keep_xc=False)
    assert set(np.unique(res.info)).issubset({0, -2})
    worst, loss, lref = check_end_to_end(cfg, sc, res, subbands=[5, 100])
    print(f"C4 FP32: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), {lref:.2e} dB (reference R)")


def test_full_size_c4_default_path_sampled():
    """The batched-uneven workload at full size through the default bs_run
    (no fused kernel): the warp-per-pair FP32 covariance (K <= 128, 128 pairs
    per SM) followed by the solve that visits pairs grouped by W; the oracle
    checks 2 subbands x 256 targets."""
    cfg = all_configs()["C4"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, keep_xc=False)
    assert set(np.unique(res.info)).issubset({0, -2})
    worst, loss, lref = check_end_to_end(cfg, sc, res, subbands=[17, 90])
    print(f"C4 FP32 (default path): max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), "
          f"{lref:.2e} dB (reference R)")


def test_full_size_c5_sampled():
    """The few-snapshot workload at full size (N=1024, 128 targets, W=9,
    K=2W=18, 16384 pairs) through the default bs_run with the fixed loading;
    the oracle checks 3 subbands x 128 targets."""
    cfg = all_configs()["C5"]
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, keep_xc=False)
    assert set(np.unique(res.info)).issubset({0, -2})
    worst, loss, lref = check_end_to_end(cfg, sc, res, subbands=[3, 64, 120])
    print(f"C5 FP32: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB (sample R), "
          f"{lref:.2e} dB (reference R)")


def test_device_error_word_reaches_caller():
    """A set device error word (what a kernel whose bounded wait gave up
    leaves) is reported as BS_ETIMEOUT by bs_plan_device_status and cleared
    by the read; injected from the host, no device wait runs out."""
    cfg = scaled_config(all_configs()["C1"], name="err-word", T=1, L=4, P_tr=1, P_te=1, K=8)
    plan = P.Plan.from_scene_config(cfg, [0.1])
    assert plan.device_status() == 0
    plan.set_device_flags(1)
    with pytest.raises(P.BsError, match="timed out"):
        plan.device_status()
    assert plan.device_status() == 0


def wide_config():
    """Windows above 16 beams (17..32, the whole-warp solve) beside a small
    one, K below and above W, windows wrapping around beam M - 1."""
    return scaled_config(all_configs()["C1"], name="wide", N=64, F=256, L=8, M=128, T=6,
                         W=(17, 32, 24, 25, 5, 20), K=(40, 64, 30, 100, 10, 33), P_tr=7, P_te=2,
                         n_jam=3, jnr_db=(25.0, 35.0))


@pytest.mark.parametrize("precision", [P.BS_PREC_FP32, P.BS_PREC_FP16])
def test_wide_windows_stages_and_end_to_end(precision):
    cfg = wide_config()
    sc = make_scene(cfg)
    kw = {"store_scale": 2.0} if precision != P.BS_PREC_FP32 else {}
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, **kw)
    if precision == P.BS_PREC_FP32:
        check_stages(cfg, sc, res)
    # FP16 windows of streams only about 2W long: the 2^-11 rounding of the
    # windows, amplified by the conditioning of the loaded covariance, puts
    # the weights near 1e-3 of the FP64 ones (as on the K = 2W..8W workloads);
    # the SINR bars stay at 0.1 dB
    wtol = WEIGHT_TOL if precision == P.BS_PREC_FP32 else 5e-3
    worst, loss, lref = check_end_to_end(cfg, sc, res, weight_tol=wtol, check_out=precision == P.BS_PREC_FP32)
    print(f"W up to 32, prec {precision}: max weight rel err {worst:.2e}, max |SINR loss| {loss:.2e} dB "
          f"(sample R), {lref:.2e} dB (reference R)")


@pytest.mark.parametrize("kappa_max,flags", [(1.0001, 0), (0.0, P.BS_FLAG_NO_FP64), (0.0, P.BS_FLAG_NO_REFINE)])
def test_wide_windows_escalation_paths(kappa_max, flags):
    """The whole-warp solve's FP64 path (every pair escalated by a tiny
    kappa_max), its FP32 path without escalation and without refinement:
    each against the FP64 solve of the GPU's own covariances."""
    cfg = wide_config()
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, flags=flags, kappa_max=kappa_max, keep_xc=False)
    tol = 1e-4 if flags & P.BS_FLAG_NO_REFINE else SOLVE_TOL
    for g in range(res.plan.sizes.pairs):
        pr = res.pair(g)
        assert pr["info"] == (-2 if kappa_max > 0 else 0), (g, pr["info"])
        co = O.mvdr_weights(pr["R"], pr["a"])
        assert rel(pr["c"], co) <= tol, (g, rel(pr["c"], co))


def test_wide_windows_plain_path():
    """The plain FP32 per-pair path (BS_FLAG_PLAIN) with windows up to 32."""
    cfg = wide_config()
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, flags=P.BS_FLAG_PLAIN, keep_xc=False)
    worst, loss, lref = check_end_to_end(cfg, sc, res, weight_tol=1e-2, check_out=False)
    print(f"W up to 32, plain FP32: max weight rel err {worst:.2e}")


@pytest.mark.parametrize("precision", [P.BS_PREC_FP32, P.BS_PREC_FP16])
def test_pass_autotuner(precision):
    """bs_autotune_pass times every beamspace and covariance variant that
    applies and the fused launch, keeps the fastest, and the tuned pass (and
    its CUDA graph) still meets the oracle's tolerances."""
    cfg = scaled_config(uneven_small_config(), name="tune", M=1024, N=256, F=512, L=16)
    sc = make_scene(cfg)
    kw = {"store_scale": 2.0} if precision != P.BS_PREC_FP32 else {}
    plan = P.Plan.from_scene_config(cfg, sc.u_tgt, precision=precision, **kw)
    b = P.alloc_buffers(plan)
    b.x.copy_(torch.from_numpy(sc.x.reshape(-1)))
    st = torch.cuda.Stream()
    rep = P.bs_autotune_pass(plan, b, stream=st)
    bms, cms = rep["beamspace_ms"], rep["covariance_ms"]
    assert all(bms[k] is not None and bms[k] > 0 for k in P.BEAMSPACE_VARIANTS[:3])   # M = 1024: these three apply
    assert bms["tensor-core DFT"] is None                                            # N = 1024, M = 2048 only
    assert cms["CTA per pair"] > 0 and cms["warp per pair"] > 0         # K <= 128
    assert (cms["tensor cores"] is not None) == (precision != P.BS_PREC_FP32)
    assert rep["beamspace"] == min((v, k) for k, v in bms.items() if v is not None)[1]
    assert rep["covariance"] == min((v, k) for k, v in cms.items() if v is not None)[1]
    assert rep["solve_ms"] > 0 and rep["fused_ms"] > 0
    g = P.Graph(plan, b, st)
    g.launch(st)
    st.synchronize()
    res = GpuResult(plan=plan, off=plan.offsets(), xc=None,
                    z_train=ztrain_to_complex(plan, b.z_train, kw.get("store_scale", 1.0)),
                    z_test=b.z_test.cpu().numpy(), R=b.R.cpu().numpy(), c=b.c.cpu().numpy(),
                    info=b.info.cpu().numpy(),
                    out=b.out.cpu().numpy()[: plan.sizes.out_elems].reshape(plan.sizes.pairs, -1))
    wtol = WEIGHT_TOL if precision == P.BS_PREC_FP32 else 5e-3
    check_end_to_end(cfg, sc, res, weight_tol=wtol, check_out=precision == P.BS_PREC_FP32)
    assert plan.device_status() == 0


def test_graph_and_autotune():
    """The autotuner picks a launch shape; a captured CUDA graph of the whole
    pass then reproduces bs_run (same shape) bit for bit."""
    cfg = uneven_small_config()
    sc = make_scene(cfg)
    plan = P.Plan.from_scene_config(cfg, sc.u_tgt, flags=P.BS_FLAG_FUSED)
    b = P.alloc_buffers(plan)
    b.x.copy_(torch.from_numpy(sc.x.reshape(-1)))
    st = torch.cuda.Stream()
    tuned = P.bs_autotune(plan, b, stream=st)
    assert tuned["threads"] in (64, 128) and 1 <= tuned["ctas_per_sm"] <= 8 and tuned["ms"] > 0
    P.bs_run(plan, b, stream=st)
    st.synchronize()
    ref_out, ref_c = b.out.clone(), b.c.clone()
    b.out.zero_(); b.c.zero_()
    g = P.Graph(plan, b, st)
    for _ in range(3):
        g.launch(st)
    st.synchronize()
    assert torch.equal(b.out, ref_out)
    assert torch.equal(b.c, ref_c)
    assert plan.device_status() == 0


# (W, K, training records): K up to 128 with ragged 16-vector blocks, and
# K < 8, K not a multiple of the 64-vector stage and K beyond the ring of
# stages (the ring wraps)
TC_COV_CASES = {
    "short": ((1, 2, 3, 5, 8, 9, 12, 15, 16), (1, 7, 17, 40, 64, 65, 100, 127, 128), 1),
    "wrapping": ((1, 2, 3, 4, 5, 8, 9, 12, 15, 16), (4, 2, 4, 1, 8, 65, 4, 100, 128, 300), 3),
}


@pytest.mark.parametrize("case", list(TC_COV_CASES))
@pytest.mark.parametrize("precision", [P.BS_PREC_FP16, P.BS_PREC_BF16])
def test_tensor_core_covariance(precision, case):
    """16-bit windows: the tensor-core covariance equals the FP64 covariance
    of the same (dequantised) windows to COV_TOL, for W = 1..16 and K not a
    multiple of 16 (ragged last k-block)."""
    base = all_configs()["C1"]
    W, K, ptr = TC_COV_CASES[case]
    cfg = scaled_config(base, name="tc-cov", N=64, F=512, L=4, M=64, T=len(W), W=W, K=K,
                        P_tr=ptr, P_te=1, n_jam=2)
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, keep_xc=False)
    for g in range(res.plan.sizes.pairs):
        pr = res.pair(g)
        Ro = O.window_covariance(pr["z_train"].astype(np.complex128), cfg.delta)
        assert np.abs(pr["R"] - Ro).max() <= COV_TOL * np.abs(Ro).max(), (g, np.abs(pr["R"] - Ro).max())
        np.testing.assert_allclose(pr["R"], pr["R"].conj().T, atol=0)


@pytest.mark.parametrize("precision,flags", [(P.BS_PREC_FP32, 0), (P.BS_PREC_FP16, P.BS_FLAG_SIMT_COV)])
def test_short_stream_covariance_warp_per_pair(precision, flags):
    """Short window streams over many pairs (K <= 128, 1024 pairs) take the
    warp-per-pair covariance: W = 1..16 (one to five lower-triangle entries
    per lane), K = 1..128 across the 64-vector chunk boundary; R equals the
    FP64 covariance of the same windows to COV_TOL."""
    base = all_configs()["C1"]
    W = (1, 2, 7, 8, 11, 13, 15, 16)
    K = (1, 5, 63, 64, 65, 17, 128, 100)
    cfg = scaled_config(base, name="warp-cov", N=64, F=512, L=128, M=64, T=len(W), W=W, K=K,
                        P_te=1, n_jam=2)
    sc = make_scene(cfg)
    kw = {"store_scale": 4.0} if precision != P.BS_PREC_FP32 else {}
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, flags=flags, keep_xc=False, **kw)
    assert res.plan.sizes.pairs == 1024
    for g in range(res.plan.sizes.pairs):
        pr = res.pair(g)
        Ro = O.window_covariance(pr["z_train"].astype(np.complex128), cfg.delta)
        assert np.abs(pr["R"] - Ro).max() <= COV_TOL * np.abs(Ro).max(), (g, np.abs(pr["R"] - Ro).max())
        np.testing.assert_allclose(pr["R"], pr["R"].conj().T, atol=0)


@pytest.mark.parametrize("precision", [P.BS_PREC_FP16, P.BS_PREC_BF16])
def test_tensor_core_covariance_long_streams(precision):
    """K of several hundred vectors: the per-warp ring of window stages wraps
    several times (4 stages of 48-byte rows for 2W <= 24, 2 stages of
    80-byte rows above), with ragged last chunks."""
    base = all_configs()["C1"]
    W = (9, 12, 13, 16, 3)
    K = (1000, 513, 300, 257, 640)
    cfg = scaled_config(base, name="tc-cov-long", N=64, F=512, L=4, M=64, T=len(W), W=W, K=K,
                        P_te=1, n_jam=2)
    sc = make_scene(cfg)
    res = run_gpu(cfg, sc.x, sc.u_tgt, precision=precision, keep_xc=False)
    for g in range(res.plan.sizes.pairs):
        pr = res.pair(g)
        Ro = O.window_covariance(pr["z_train"].astype(np.complex128), cfg.delta)
        assert np.abs(pr["R"] - Ro).max() <= COV_TOL * np.abs(Ro).max(), (g, np.abs(pr["R"] - Ro).max())
