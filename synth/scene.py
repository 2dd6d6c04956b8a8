"""Wideband ULA scenes: LFM jammers, LFM target echoes and white noise.

The signal model is the paper's received-signal model (Sec. II-A,
Eq. ReceivedSignal) for the linear-array case of its planar array (N_z = 1,
elevation 0): per record the array sees

    y[t] = sum_k alpha_k a_k p_k[t] + I[t] + n[t],   n ~ CN(0, sigma^2 I),

with half-wavelength spacing at the design frequency f_d.  The wideband
array response is applied exactly at every FFT bin of the record (a true time
delay): a plane wave with direction sine u reaches element n with phase
exp(j*pi*n*u*(f_c + f)/f_d) at baseband frequency f.  Records are built in
the frequency domain and brought to raw IQ by a unitary inverse FFT, so the
element-0 waveform is exactly the source waveform.  The narrowband steering
vector the method uses per subband is therefore an approximation that the
data really exercise, not an assumption baked into them.

Training records (the first P_tr) hold jammers and noise only; test records
hold targets, jammers and noise.  Jammers are LFM sweeps over a random
50-100 % of the band with random start frequency, sweep and phase per record;
targets are full-band LFM pulses of half a record with a random delay.

Nothing here computes a step of the beamspace MVDR method.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

BASE_SEED = 20250811
WINDOW_CHOICES_UNEVEN = (3, 5, 7, 9, 11, 15)


@dataclass(frozen=True)
class SceneConfig:
    """One workload: array, channeliser, beamspace, targets, windows, data.

    W[t] and K[t] are the window size and the number of training vectors of
    target t (the same for every subband of that target).
    """

    name: str
    N: int                      # array elements (ULA)
    F: int                      # fast-time samples per record (FFT size)
    L: int                      # subbands
    M: int                      # spatial FFT size (zero-padded, M >= N)
    T: int                      # targets
    W: tuple                    # window size per target
    K: tuple                    # training vectors per target
    n_jam: int                  # wideband LFM jammers
    jnr_db: tuple               # (lo, hi) per-element jammer-to-noise ratio, dB
    snr_db: float               # per-element target SNR, dB
    P_tr: int                   # training records (target-free)
    P_te: int                   # test records (targets present)
    seed: int
    fc: float = 10e9            # carrier frequency, Hz
    fs: float = 1e9             # sampling rate, Hz
    fd: float = 10e9            # design frequency of the half-wavelength spacing, Hz
    sigma2: float = 1.0         # noise variance per element per sample
    delta: float = 10.0         # diagonal loading (10 sigma^2)
    description: str = ""
    # Coherent pulse train: each target keeps one delay over all test records
    # and its echo phase advances by 2 pi nu_t per record (nu_t: Doppler in
    # cycles per record, drawn on the grid k / P_te so that it falls on a
    # Doppler bin); the default draws an independent delay and phase per record.
    coherent_targets: bool = False
    # Uniform planar array (Eq. ArrayFactor): N = Nx Nz elements ordered
    # n = n_x Nz + n_z, M = Mx Mz beams ordered m = m_x Mz + m_z, and a
    # W_x x W_z window per target (W[t] = W_x W_z, Wz[t] = W_z).  Nz = 1 is
    # the uniform linear array.
    Nz: int = 1
    Mz: int = 1
    Wz: tuple = ()

    @property
    def B(self) -> int:
        """Bins per subband."""
        return self.F // self.L

    @property
    def P(self) -> int:
        return self.P_tr + self.P_te

    @property
    def pairs(self) -> int:
        return self.T * self.L

    @property
    def Nx(self) -> int:
        return self.N // self.Nz

    @property
    def Mx(self) -> int:
        return self.M // self.Mz

    @property
    def Wz_t(self) -> tuple:
        """Vertical window size per target (1 for a linear array)."""
        return tuple(self.Wz) if self.Wz else (1,) * self.T

    def validate(self) -> None:
        if self.F % self.L:
            raise ValueError("F must be a multiple of L")
        if self.M < self.N:
            raise ValueError("M must be >= N")
        if len(self.W) != self.T or len(self.K) != self.T:
            raise ValueError("W and K need one entry per target")
        kmax = max(self.K) if self.K else 0
        if kmax > self.P_tr * self.B:
            raise ValueError("P_tr * B training vectors cannot cover max(K)")
        if self.Nz < 1 or self.N % self.Nz or self.Mz < self.Nz or self.M % self.Mz or self.Mx < self.Nx:
            raise ValueError("planar array: Nz | N, Mz | M, Mz >= Nz, M/Mz >= N/Nz")
        if len(self.Wz_t) != self.T or any(w % wz or wz > self.Mz or w // wz > self.Mx
                                           for w, wz in zip(self.W, self.Wz_t)):
            raise ValueError("planar windows: Wz | W, Wz <= Mz, W/Wz <= M/Mz")


def _uniform(name, idx, N, F, L, M, T, W, K, n_jam, jnr_db, P_tr, P_te, desc):
    return SceneConfig(
        name=name, N=N, F=F, L=L, M=M, T=T, W=(W,) * T, K=(K,) * T,
        n_jam=n_jam, jnr_db=jnr_db, snr_db=0.0, P_tr=P_tr, P_te=P_te,
        seed=BASE_SEED + idx, description=desc,
    )


def _uneven_c4() -> SceneConfig:
    T = 256
    g = np.random.default_rng(BASE_SEED + 3 + 1000)
    W = tuple(int(w) for w in g.choice(WINDOW_CHOICES_UNEVEN, size=T))
    K = tuple(int(g.integers(2 * w, 8 * w + 1)) for w in W)
    F, L = 2048, 128
    B = F // L
    P_tr = -(-max(K) // B)
    return SceneConfig(
        name="C4", N=1024, F=F, L=L, M=2048, T=T, W=W, K=K, n_jam=8,
        jnr_db=(20.0, 40.0), snr_db=0.0, P_tr=P_tr, P_te=8,
        seed=BASE_SEED + 3,
        description="batched uneven: N=1024, L=128, 256 targets, W in "
                    "{3,5,7,9,11,15}, K in [2W, 8W]",
    )


def all_configs() -> dict:
    """The five workloads, smallest first."""
    cfgs = [
        _uniform("C1", 0, N=64, F=512, L=16, M=64, T=4, W=5, K=128, n_jam=2,
                 jnr_db=(30.0, 30.0), P_tr=4, P_te=8,
                 desc="plain FP32: N=64, F=512, L=16, M=64, W=5, K=128, T=4, "
                      "2 jammers at +30 dB"),
        _uniform("C2", 1, N=256, F=1024, L=64, M=512, T=16, W=7, K=256, n_jam=4,
                 jnr_db=(20.0, 40.0), P_tr=16, P_te=8,
                 desc="grid: N=256, F=1024, L=64, M=512, W=7, K=256, T=16, "
                      "4 jammers at 20-40 dB"),
        _uniform("C3", 2, N=1024, F=2048, L=128, M=2048, T=64, W=9, K=512, n_jam=8,
                 jnr_db=(20.0, 40.0), P_tr=32, P_te=8,
                 desc="mixed precision: N=1024, F=2048, L=128, M=2048, W=9, "
                      "K=512, T=64, 8 jammers at 20-40 dB"),
        _uneven_c4(),
        _uniform("C5", 4, N=1024, F=2048, L=128, M=2048, T=128, W=9, K=18, n_jam=8,
                 jnr_db=(20.0, 40.0), P_tr=2, P_te=8,
                 desc="learned loading: N=1024, F=2048, L=128, M=2048, W=9, "
                      "K=2W=18, T=128"),
    ]
    for c in cfgs:
        c.validate()
    return {c.name: c for c in cfgs}


def config_by_name(name: str) -> SceneConfig:
    return all_configs()[name]


def scaled_config(cfg: SceneConfig, **changes) -> SceneConfig:
    """A copy of cfg with fields replaced; P_tr grows to cover max(K) if needed.

    W or K given as an int is expanded to one entry per target.
    """
    T = changes.get("T", cfg.T)
    if "Wz" in changes or (cfg.Wz and T != cfg.T):
        v = changes.get("Wz", cfg.Wz)
        if isinstance(v, (int, np.integer)):
            v = (int(v),) * T
        elif len(v) != T:
            v = tuple(int(v[i % len(v)]) for i in range(T))
        changes["Wz"] = tuple(int(a) for a in v)
    for key in ("W", "K"):
        v = changes.get(key, getattr(cfg, key))
        if isinstance(v, (int, np.integer)):
            v = (int(v),) * T
        elif len(v) != T:
            v = tuple(int(v[i % len(v)]) for i in range(T))
        changes[key] = tuple(int(a) for a in v)
    out = dataclasses.replace(cfg, **changes)
    need = -(-max(out.K) // out.B) if out.K else 0
    if out.P_tr < need:
        out = dataclasses.replace(out, P_tr=need)
    out.validate()
    return out


@dataclass
class Scene:
    cfg: SceneConfig
    x: np.ndarray                 # [P][F][N] complex64 raw IQ, training records first
    u_tgt: np.ndarray             # [T] direction sines of the targets (float64)
    u_jam: np.ndarray             # [J] direction sines of the jammers
    jnr_db: np.ndarray            # [J]
    x_interf: Optional[np.ndarray] = None  # [P][F][N] complex64 noise-free jammer part
    v_tgt: Optional[np.ndarray] = None        # [T] vertical sines sin(theta) (planar arrays)
    v_jam: Optional[np.ndarray] = None        # [J]
    tgt_delay: Optional[np.ndarray] = None    # [T] delays (samples), coherent_targets only
    tgt_doppler: Optional[np.ndarray] = None  # [T] Doppler bins (cycles per record x P_te)


def _directions(g, T, J, N):
    """Target and jammer direction sines in +-60 deg.

    Jammers keep at least 4/N (two 3-dB beamwidths) in sine space from every
    target; the spacing is halved if a draw cannot meet it (dense scenes).
    """
    u_t = np.sin(np.deg2rad(g.uniform(-60.0, 60.0, size=T)))
    u_j = np.empty(J)
    sep = 4.0 / N
    for j in range(J):
        for _attempt in range(100000):
            cand = math.sin(math.radians(g.uniform(-60.0, 60.0)))
            if T == 0 or np.min(np.abs(u_t - cand)) >= sep:
                u_j[j] = cand
                break
            if _attempt % 1000 == 999:
                sep *= 0.5
        else:  # pragma: no cover - unreachable for the configs here
            u_j[j] = cand
    return u_t, u_j


def _plane_wave(theta: np.ndarray, N: int, blk: int = 32) -> np.ndarray:
    """exp(j*theta*n) for n < N, shape theta.shape + (N,).

    Written as exp(j*theta*n0) * exp(j*theta*blk*n1) with n = blk*n1 + n0, so
    only 2*sqrt(N)-ish exponentials are taken per theta.
    """
    n0 = np.arange(blk, dtype=np.float64)
    n1 = np.arange(-(-N // blk), dtype=np.float64) * blk
    lo = np.exp(1j * theta[..., None] * n0)                  # [..][blk]
    hi = np.exp(1j * theta[..., None] * n1)                  # [..][nb]
    out = (hi[..., :, None] * lo[..., None, :]).reshape(theta.shape + (n1.size * blk,))
    return out[..., :N]


def pulse(F: int) -> np.ndarray:
    """The targets' transmitted waveform, [F] complex128: a full-band LFM
    pulse of Tp = F/2 samples (phase 2 pi (-tau/2 + tau^2 / (2 Tp))), zero
    after it.  Matched filtering needs its spectrum, an input of the
    processing after the beamformer."""
    Tp = max(F // 2, 1)
    tau = np.arange(F, dtype=np.float64)
    return np.where(tau < Tp, np.exp(1j * 2 * np.pi * (-0.5 * tau + 0.5 * tau * tau / Tp)), 0.0)


def make_scene(cfg: SceneConfig, keep_interference: bool = False,
               k_chunk: int = 64, realisation: int = 0) -> Scene:
    """Synthesise the raw IQ records x[p][t][n] of one workload (seeded).

    realisation > 0 keeps the geometry of the workload's scene (target and
    jammer directions, jammer powers) and draws new jammer waveforms, target
    echoes and noise: an independent realisation of the same scene.
    """
    cfg.validate()
    N, F, P, J, T = cfg.N, cfg.F, cfg.P, cfg.n_jam, cfg.T
    ss = np.random.SeedSequence(cfg.seed)
    g_geom, g_jam, g_tgt, g_noise, g_vert = [np.random.default_rng(s) for s in ss.spawn(5)]
    if realisation:
        g_jam, g_tgt, g_noise = [np.random.default_rng(s)
                                 for s in np.random.SeedSequence([cfg.seed, int(realisation)]).spawn(3)]

    u_t, u_j = _directions(g_geom, T, J, cfg.Nx)
    v_t = v_j = None
    if cfg.Nz > 1:   # elevations within +-20 deg
        v_t = np.sin(np.deg2rad(g_vert.uniform(-20.0, 20.0, size=T)))
        v_j = np.sin(np.deg2rad(g_vert.uniform(-20.0, 20.0, size=J)))

    def response(scale, u, v):
        """Array response at each bin: [kc][src][N], n = n_x Nz + n_z."""
        ex = _plane_wave(scale[:, None] * u[None, :], cfg.Nx)
        if v is None:
            return ex.astype(np.complex64)
        ez = _plane_wave(scale[:, None] * v[None, :], cfg.Nz)
        return (ex[..., :, None] * ez[..., None, :]).reshape(ex.shape[:-1] + (N,)).astype(np.complex64)
    jnr = g_geom.uniform(cfg.jnr_db[0], cfg.jnr_db[1], size=J) if J else np.zeros(0)

    t = np.arange(F, dtype=np.float64)
    # Jammer waveforms per (record, jammer): LFM over a random 50-100 % of the band.
    bw = g_jam.uniform(0.5, 1.0, size=(P, J))
    nu0 = g_jam.uniform(0.0, 1.0, size=(P, J)) * (1.0 - bw) - 0.5
    psi = g_jam.uniform(0.0, 2 * np.pi, size=(P, J))
    amp_j = np.sqrt(cfg.sigma2 * 10.0 ** (jnr / 10.0))
    s_jam = amp_j[None, :, None] * np.exp(1j * (
        2 * np.pi * (nu0[..., None] * t + 0.5 * bw[..., None] * t * t / F) + psi[..., None]))
    S_jam = np.fft.fft(s_jam, axis=-1, norm="ortho")            # [P][J][F]

    # Target echoes (test records): full-band LFM pulse of F/2 samples, random delay.
    Tp = max(F // 2, 1)
    tgt_delay = tgt_doppler = None
    if cfg.coherent_targets:
        tgt_delay = g_tgt.integers(0, F - Tp + 1, size=T)
        tgt_doppler = g_tgt.integers(0, max(cfg.P_te, 1), size=T)
        psi0 = g_tgt.uniform(0.0, 2 * np.pi, size=T)
        delay = np.broadcast_to(tgt_delay, (cfg.P_te, T))
        rec = np.arange(cfg.P_te, dtype=np.float64)[:, None]
        psi_t = psi0[None, :] + 2 * np.pi * rec * tgt_doppler[None, :] / max(cfg.P_te, 1)
    else:
        delay = g_tgt.integers(0, F - Tp + 1, size=(cfg.P_te, T))
        psi_t = g_tgt.uniform(0.0, 2 * np.pi, size=(cfg.P_te, T))
    amp_t = math.sqrt(cfg.sigma2 * 10.0 ** (cfg.snr_db / 10.0))
    tau = t[None, None, :] - delay[..., None]
    inside = (tau >= 0) & (tau < Tp)
    s_tgt = np.where(inside, amp_t * np.exp(1j * (
        2 * np.pi * (-0.5 * tau + 0.5 * tau * tau / Tp) + psi_t[..., None])), 0.0)
    S_tgt = np.fft.fft(s_tgt, axis=-1, norm="ortho")            # [P_te][T][F]

    # Baseband frequency of FFT bin k (signed bin index).
    k = np.arange(F)
    f_bin = np.where(k < F // 2, k, k - F) * (cfg.fs / F)

    X = np.empty((P, F, N), dtype=np.complex64)
    XJ = np.empty((P, F, N), dtype=np.complex64) if keep_interference else None
    SJ = np.ascontiguousarray(S_jam.transpose(2, 0, 1)).astype(np.complex64)  # [F][P][J]
    ST = np.ascontiguousarray(S_tgt.transpose(2, 0, 1)).astype(np.complex64)  # [F][P_te][T]
    for k0 in range(0, F, k_chunk):
        k1 = min(F, k0 + k_chunk)
        scale = np.pi * (cfg.fc + f_bin[k0:k1]) / cfg.fd           # [kc]
        # true-time-delay response of each source at each bin: [kc][src][N]
        Ej = response(scale, u_j, v_j)
        xj = np.matmul(SJ[k0:k1], Ej)                               # [kc][P][N]
        if XJ is not None:
            XJ[:, k0:k1, :] = xj.transpose(1, 0, 2)
        if T and cfg.P_te:
            Et = response(scale, u_t, v_t)
            xj[:, cfg.P_tr:, :] += np.matmul(ST[k0:k1], Et)         # [kc][P_te][N]
        X[:, k0:k1, :] = xj.transpose(1, 0, 2)

    # White noise CN(0, sigma^2): seeded torch CPU generator (much faster than
    # numpy's for hundreds of millions of samples); real and imaginary parts
    # each have variance sigma^2 / 2.
    tg = torch.Generator(device="cpu")
    tg.manual_seed(int(g_noise.integers(0, 2**62)))
    noise = torch.randn((P, F, N, 2), generator=tg, dtype=torch.float32)
    noise.mul_(math.sqrt(cfg.sigma2 / 2.0))
    x = noise.numpy().view(np.complex64)[..., 0]
    for p in range(P):
        x[p] += np.fft.ifft(X[p], axis=0, norm="ortho").astype(np.complex64)
    del X
    x_interf = None
    if XJ is not None:
        x_interf = np.empty_like(XJ)
        for p in range(P):
            x_interf[p] = np.fft.ifft(XJ[p], axis=0, norm="ortho").astype(np.complex64)
    return Scene(cfg=cfg, x=np.ascontiguousarray(x), u_tgt=u_t, u_jam=u_j,
                 jnr_db=jnr, x_interf=x_interf, v_tgt=v_t, v_jam=v_j, tgt_delay=tgt_delay,
                 tgt_doppler=tgt_doppler)


def reference_records(cfg: SceneConfig, P_ref: int, realisation: int = 1) -> np.ndarray:
    """P_ref target-free records [P_ref][F][N] (complex64) of an independent
    realisation of cfg's scene: the same jammer directions and powers, new
    jammer waveforms and noise.  They are not used for the weights, so a
    covariance estimated from them judges output SINR independently of the
    training data."""
    need = -(-max(cfg.K) // cfg.B) if cfg.K else 1
    ref = dataclasses.replace(cfg, P_tr=max(int(P_ref), need), P_te=0)
    return make_scene(ref, realisation=realisation).x[:P_ref]
