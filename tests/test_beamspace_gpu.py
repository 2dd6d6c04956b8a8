"""GPU parity of the window beamspace stage (bs_beamspace) for the
three-pass sizes M = 512 .. 4096: the tensor-core kernel (N = 1024,
M = 2048), the warp-per-transform kernel (M = 1024, 2048, 4096 with
N <= 1024, and BS_FLAG_SIMT_FFT), the persistent bulk-copy kernel (the other
sizes, and BS_FLAG_STAGED_FFT) and the one-shot kernel (BS_FLAG_NO_TMA):
every training and test window against the oracle's zero-padded DFT
(Eq. VerDFT, Eq. BeamTransform) and window selection (Eq. OverallWindow,
Eq. ApplyWindow) of the same channelised input.

Tolerances: FP32 windows within FFT_TOL (norm-wise FFT error bound of the
transform, relative to the largest beam norm of the subband); 16-bit
windows additionally within one rounding of the stored value (2^-11
relative for FP16, 2^-8 for BF16).
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_11790_gb300 as P

pytestmark = pytest.mark.gpu

FFT_TOL = 5e-6
ROUND = {P.BS_PREC_FP32: 0.0, P.BS_PREC_FP16: 2.0 ** -11, P.BS_PREC_BF16: 2.0 ** -8}


def _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, precision, flags, xc, store_scale=0.0):
    plan = P.Plan(N=N, F=F, L=L, M=M, u=u, W=W, K=K, P_train=Ptr, P_test=Pte, fc=10e9, fs=1e9,
                  fd=10e9, delta=1.0, precision=precision, flags=flags, store_scale=store_scale)
    b = P.alloc_buffers(plan)
    b.xc.copy_(torch.from_numpy(xc.reshape(-1)))
    b.z_train.zero_()
    b.z_test.zero_()
    P.bs_beamspace(plan, b.xc, b.z_train, b.z_test)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    sc = store_scale if store_scale > 0 else 1.0
    if precision == P.BS_PREC_FP32:
        ztr = b.z_train.cpu().numpy().astype(np.complex128)
    else:
        f = b.z_train.float().cpu().numpy().reshape(-1, 2) / sc
        ztr = f[:, 0] + 1j * f[:, 1]
    return plan, plan.offsets(), ztr, b.z_test.cpu().numpy().astype(np.complex128)


def _check_windows(plan, off, ztr, zte, xc, M, L, Ptr, Pte, precision):
    Pn, F, _ = xc.shape
    B = F // L
    yb = O.beamspace(xc.astype(np.complex128), M)     # [P][F][M]
    Vte = Pte * B
    tol_r = ROUND[precision]
    for g in range(plan.sizes.pairs):
        s = g % L
        W, K, st = int(off["W"][g]), int(off["K"][g]), int(off["start"][g])
        beams = O.window_beams(st, W, M)
        zall = yb[:, s * B:(s + 1) * B][:, :, beams].reshape(Pn * B, W)
        scale = np.linalg.norm(yb[:, s * B:(s + 1) * B], axis=-1).max()
        got_tr = ztr[off["ztr_off"][g]:off["ztr_off"][g + 1]].reshape(K, W)
        ref_tr = zall[:K]
        assert np.all(np.abs(got_tr - ref_tr) <= FFT_TOL * scale + tol_r * np.abs(ref_tr)), g
        if Pte:
            got_te = zte[off["zte_off"][g]:off["zte_off"][g + 1]].reshape(Vte, W)
            assert np.abs(got_te - zall[Ptr * B:]).max() <= FFT_TOL * scale, g


# (N, M, F, L, P_train, P_test, W per target, K per target): zero-padded
# (N <= M/2) and unpadded-half (N > M/2) inputs, N short of the tile, several
# groups per resident CTA (the loop wraps the staging double buffer), W up
# to 16 with windows that wrap around beam M-1 -> 0, K cutting a group.
CASES = [
    (256, 512, 512, 16, 9, 2, [7, 16, 1], [200, 288, 5]),
    (1024, 2048, 1024, 64, 3, 1, [9, 3], [48, 33]),
    (1022, 2048, 512, 32, 2, 2, [9, 16, 5], [31, 32, 17]),
    (1500, 2048, 512, 32, 2, 1, [9], [25]),
    (2048, 2048, 256, 16, 2, 1, [4], [31]),
    (400, 1024, 1024, 32, 3, 1, [11, 2], [64, 95]),
    (2000, 4096, 256, 16, 2, 1, [9, 13], [32, 7]),
    (4096, 4096, 128, 8, 2, 0, [6], [20]),
    (1024, 4096, 256, 16, 2, 1, [9, 16, 2], [32, 17, 3]),
    (700, 4096, 256, 16, 3, 2, [5, 12], [48, 40]),
    (1000, 1024, 512, 32, 2, 1, [15, 4], [9, 32]),
]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[0]}_M{c[1]}_F{c[2]}" for c in CASES])
@pytest.mark.parametrize("precision", [P.BS_PREC_FP32, P.BS_PREC_FP16])
def test_window_beamspace(case, precision):
    N, M, F, L, Ptr, Pte, W, K = case
    rng = np.random.default_rng(N * 7 + M + F)
    Pn = Ptr + Pte
    xc = (rng.standard_normal((Pn, F, N)) + 1j * rng.standard_normal((Pn, F, N))).astype(np.complex64)
    u = list(rng.uniform(-0.95, 0.95, size=len(W)))
    u[0] = 0.0   # broadside: the window wraps from beam M-1 to beam 0
    store_scale = 4.0 if precision != P.BS_PREC_FP32 else 0.0
    plan, off, ztr, zte = _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, precision, 0, xc, store_scale)
    _check_windows(plan, off, ztr, zte, xc, M, L, Ptr, Pte, precision)


KERNEL_CASES = CASES[:3] + CASES[-3:]


@pytest.mark.parametrize("case", KERNEL_CASES, ids=[f"N{c[0]}_M{c[1]}" for c in KERNEL_CASES])
def test_kernels_agree(case):
    """The default kernel (tensor cores or warp-per-transform where they
    apply), the warp-per-transform kernel (BS_FLAG_SIMT_FFT), the
    bulk-copy-staged kernel (BS_FLAG_STAGED_FFT) and the one-shot kernel
    (BS_FLAG_NO_TMA) factor the transform differently and read their
    twiddles differently (table values, products of table values, folded
    constants) but agree to within twice the FFT bound; each meets the
    oracle bound on its own."""
    N, M, F, L, Ptr, Pte, W, K = case
    rng = np.random.default_rng(5 + N)
    Pn = Ptr + Pte
    xc = (rng.standard_normal((Pn, F, N)) + 1j * rng.standard_normal((Pn, F, N))).astype(np.complex64)
    u = list(rng.uniform(-0.9, 0.9, size=len(W)))
    outs = []
    for flags in (0, P.BS_FLAG_SIMT_FFT, P.BS_FLAG_STAGED_FFT, P.BS_FLAG_NO_TMA):
        plan, off, ztr, zte = _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, P.BS_PREC_FP32, flags, xc)
        _check_windows(plan, off, ztr, zte, xc, M, L, Ptr, Pte, P.BS_PREC_FP32)
        outs.append((ztr, zte))
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            if a.size:
                assert np.linalg.norm(a - b) <= 2 * FFT_TOL * np.linalg.norm(b)


def test_warp_kernel_many_targets():
    """256 targets (the most the warp-per-transform kernel stages per
    vector) with W up to 16 at M = 1024 and M = 2048: gather entries beyond
    the ones each lane keeps in registers, windows of every residue class."""
    rng = np.random.default_rng(256)
    T = 256
    W = list(rng.integers(1, 17, size=T))
    for N, M, F, L, Ptr, Pte in ((512, 1024, 64, 4, 2, 1), (1024, 2048, 32, 2, 2, 1)):
        K = list(rng.integers(1, Ptr * (F // L) + 1, size=T))
        Pn = Ptr + Pte
        xc = (rng.standard_normal((Pn, F, N)) + 1j * rng.standard_normal((Pn, F, N))).astype(np.complex64)
        u = list(rng.uniform(-0.99, 0.99, size=T))
        for precision in (P.BS_PREC_FP32, P.BS_PREC_FP16):
            ss = 2.0 if precision != P.BS_PREC_FP32 else 0.0
            plan, off, ztr, zte = _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, precision, 0, xc, ss)
            _check_windows(plan, off, ztr, zte, xc, M, L, Ptr, Pte, precision)


def test_many_targets_gather_paths():
    """300 targets at M = 512 (8 vectors per group): gather entries beyond
    the ones each thread keeps in registers, and targets beyond the 256
    whose per-group entries are staged in shared memory."""
    N, M, F, L, Ptr, Pte = 128, 512, 64, 4, 2, 1
    rng = np.random.default_rng(77)
    T = 300
    W = list(rng.integers(1, 17, size=T))
    K = list(rng.integers(1, Ptr * (F // L) + 1, size=T))
    Pn = Ptr + Pte
    xc = (rng.standard_normal((Pn, F, N)) + 1j * rng.standard_normal((Pn, F, N))).astype(np.complex64)
    u = list(rng.uniform(-0.99, 0.99, size=T))
    for precision in (P.BS_PREC_FP32, P.BS_PREC_BF16):
        ss = 2.0 if precision != P.BS_PREC_FP32 else 0.0
        plan, off, ztr, zte = _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, precision, 0, xc, ss)
        _check_windows(plan, off, ztr, zte, xc, M, L, Ptr, Pte, precision)


def test_tensor_core_input_scale():
    """The tensor-core kernel scales every vector by a power of two before
    splitting it into FP16 parts, so inputs scaled by 2^-40 or 2^40 (far
    outside FP16's range) give windows scaled by exactly that power of two,
    and any other scale factor stays within the FFT bound of the oracle."""
    N, M, F, L, Ptr, Pte, W, K = 1024, 2048, 256, 16, 2, 1, [9, 32, 1], [32, 17, 5]
    rng = np.random.default_rng(2048)
    Pn = Ptr + Pte
    xc = (rng.standard_normal((Pn, F, N)) + 1j * rng.standard_normal((Pn, F, N))).astype(np.complex64)
    xc[:, :, :7] *= 3e3   # a strong component on a few elements
    u = [0.0, 0.37, -0.8]
    _, _, ztr0, zte0 = _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, P.BS_PREC_FP32, 0, xc)
    for e in (-40, 40):
        _, _, ztr, zte = _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, P.BS_PREC_FP32, 0,
                                        (xc * np.float32(2.0 ** e)).astype(np.complex64))
        assert np.array_equal(ztr, ztr0 * 2.0 ** e) and np.array_equal(zte, zte0 * 2.0 ** e)
    for f in (1e-30, 7.3e25):
        xs = (xc * np.float32(f)).astype(np.complex64)
        plan, off, ztr, zte = _run_beamspace(N, M, F, L, Ptr, Pte, W, K, u, P.BS_PREC_FP32, 0, xs)
        _check_windows(plan, off, ztr, zte, xs, M, L, Ptr, Pte, P.BS_PREC_FP32)
