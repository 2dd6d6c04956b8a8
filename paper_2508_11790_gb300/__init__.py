"""Windowed beamspace MVDR hot path on GB300: Python binding of the C ABI.

The functions here have the names of the C entry points in ``include/bs.h``
and only marshal arguments: every step of the path runs in the CUDA kernels
of ``libbs_mvdr.so``.  PyTorch supplies device memory and streams.  If the
library is missing the import fails with an error; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from .build import lib_path

__all__ = [
    "BS_PREC_FP32", "BS_PREC_FP16", "BS_PREC_BF16",
    "BS_FLAG_PLAIN", "BS_FLAG_NO_REFINE", "BS_FLAG_NO_FP64", "BS_FLAG_NO_TMA", "BS_FLAG_FUSED", "BS_FLAG_SIMT_COV",
    "BS_FLAG_STAGED_FFT", "BS_FLAG_SIMT_FFT",
    "bs_cov_solve", "bs_autotune", "bs_autotune_pass", "bs_set_launch", "Graph", "bs_cov_solve_noalloc",
    "BsError", "Plan", "Buffers", "alloc_buffers", "lib", "bs_plan_tables_host",
    "bs_channelize", "bs_beamspace", "bs_beamspace_full", "bs_window_cov",
    "bs_mvdr_solve", "bs_mvdr_solve_precond", "bs_apply", "bs_run", "bs_run_host",
    "bs_lift", "bs_apply_lifted", "bs_beam_pattern", "bs_range_doppler", "bs_cfar",
]

BS_PREC_FP32, BS_PREC_FP16, BS_PREC_BF16 = 0, 1, 2
BS_FLAG_PLAIN, BS_FLAG_NO_REFINE, BS_FLAG_NO_FP64, BS_FLAG_NO_TMA, BS_FLAG_FUSED = 1, 2, 4, 8, 16
BS_FLAG_SIMT_COV = 32
BS_FLAG_STAGED_FFT = 64
BS_FLAG_SIMT_FFT = 128


class BsError(RuntimeError):
    pass


class _Config(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("F", ctypes.c_int32), ("L", ctypes.c_int32),
        ("M", ctypes.c_int32), ("T", ctypes.c_int32), ("P_train", ctypes.c_int32),
        ("P_test", ctypes.c_int32), ("fc", ctypes.c_double), ("fs", ctypes.c_double),
        ("fd", ctypes.c_double), ("u", ctypes.POINTER(ctypes.c_double)),
        ("W", ctypes.POINTER(ctypes.c_int32)), ("K", ctypes.POINTER(ctypes.c_int32)),
        ("delta", ctypes.c_double), ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("kappa_max", ctypes.c_double), ("store_scale", ctypes.c_float),
        ("Nz", ctypes.c_int32), ("Mz", ctypes.c_int32),
        ("Wz", ctypes.POINTER(ctypes.c_int32)), ("v", ctypes.POINTER(ctypes.c_double)),
        ("s_begin", ctypes.c_int32), ("s_count", ctypes.c_int32),
    ]


class _Sizes(ctypes.Structure):
    _fields_ = [
        ("pairs", ctypes.c_int64), ("B", ctypes.c_int32), ("Vte", ctypes.c_int32),
        ("W_max", ctypes.c_int32), ("K_max", ctypes.c_int32), ("x_elems", ctypes.c_int64),
        ("xc_elems", ctypes.c_int64), ("ztrain_elems", ctypes.c_int64),
        ("ztrain_bytes", ctypes.c_int64), ("ztest_elems", ctypes.c_int64),
        ("r_elems", ctypes.c_int64), ("c_elems", ctypes.c_int64), ("out_elems", ctypes.c_int64),
    ]


class _Buffers(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("x", "xc", "z_train", "z_test", "R", "c", "info", "out")]


_P = ctypes.c_void_p
_SIGS = {
    "bs_plan_create": ([ctypes.POINTER(_P), ctypes.POINTER(_Config)], ctypes.c_int),
    "bs_plan_destroy": ([_P], None),
    "bs_plan_sizes": ([_P, ctypes.POINTER(_Sizes)], ctypes.c_int),
    "bs_plan_offsets": ([_P] + [_P] * 8, ctypes.c_int),
    "bs_channelize": ([_P, _P, ctypes.c_int32, _P, _P], ctypes.c_int),
    "bs_beamspace": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "bs_beamspace_full": ([_P, _P, ctypes.c_int64, _P, _P], ctypes.c_int),
    "bs_window_cov": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "bs_mvdr_solve": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "bs_apply": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "bs_lift": ([_P, _P, _P, _P], ctypes.c_int),
    # SINR judge, features and loading labels (also used by learned.py)
    "bs_features": ([_P, _P, _P, _P], ctypes.c_int),
    "bs_output_sinr": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "bs_loading_labels": ([_P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
    "bs_apply_lifted": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "bs_beam_pattern": ([_P, _P, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
    "bs_range_doppler": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "bs_cfar": ([_P, _P, ctypes.c_float, _P, _P, _P, _P, _P], ctypes.c_int),
    "bs_run": ([_P, ctypes.POINTER(_Buffers), _P], ctypes.c_int),
    "bs_run_host": ([_P, _P, _P, ctypes.POINTER(_Buffers), _P], ctypes.c_int),
    "bs_plan_tables_host": ([ctypes.POINTER(_Config), _P, _P], ctypes.c_int),
    "bs_plan_device_status": ([_P, _P], ctypes.c_int),
    "bs_plan_set_device_flags": ([_P, ctypes.c_int32], ctypes.c_int),
    "bs_mvdr_solve_precond": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "bs_cov_solve": ([_P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "bs_autotune": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "bs_set_launch": ([_P, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "bs_autotune_pass": ([_P, ctypes.POINTER(_Buffers), _P, _P], ctypes.c_int),
    "bs_cov_solve_noalloc": ([_P, ctypes.c_int32, ctypes.c_float, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int64,
                              ctypes.c_double, ctypes.c_double, ctypes.c_uint32, _P, _P, _P], ctypes.c_int),
    "bs_graph_create": ([_P, ctypes.POINTER(_Buffers), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "bs_graph_launch": ([_P, _P], ctypes.c_int),
    "bs_graph_destroy": ([_P], None),
    "bs_graph_kernel_count": ([_P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "bs_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "bs_last_error": ([], ctypes.c_char_p),
}

_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """The loaded C library (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise BsError(f"CUDA library {path} is missing: run "
                          "`python -m paper_2508_11790_gb300.build` first")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int, what: str) -> None:
    if status != 0:
        L = lib()
        raise BsError(f"{what}: {L.bs_status_string(status).decode()} "
                      f"({L.bs_last_error().decode()})")


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: Optional[torch.Tensor], dtype=None, numel=None, name="buffer") -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise BsError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise BsError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise BsError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if numel is not None and t.numel() < numel:
        raise BsError(f"{name} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


@dataclass
class Sizes:
    pairs: int
    B: int
    Vte: int
    W_max: int
    K_max: int
    x_elems: int
    xc_elems: int
    ztrain_elems: int
    ztrain_bytes: int
    ztest_elems: int
    r_elems: int
    c_elems: int
    out_elems: int


def _make_config(N, F, L, M, u, W, K, P_train, P_test, fc, fs, fd, delta, precision=BS_PREC_FP32,
                 flags=0, kappa_max=0.0, store_scale=0.0, Nz=1, Mz=1, Wz=None, v=None, s_begin=0, s_count=0):
    """ctypes config plus the numpy arrays it points into (keep both alive).
    Nz > 1 (with Mz, per-target Wz and vertical sines v) makes it planar;
    0 < s_count < L restricts it to subbands s_begin .. s_begin + s_count - 1."""
    ua = np.ascontiguousarray(u, dtype=np.float64)
    Wa = np.ascontiguousarray(W, dtype=np.int32)
    Ka = np.ascontiguousarray(K, dtype=np.int32)
    planar = Nz > 1 or Mz > 1
    Wza = np.ascontiguousarray(Wz if Wz is not None else np.ones(len(ua)), dtype=np.int32)
    va = np.ascontiguousarray(v if v is not None else np.zeros(len(ua)), dtype=np.float64)
    cfg = _Config(N, F, L, M, len(ua), P_train, P_test, fc, fs, fd,
                  ua.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  Wa.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                  Ka.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                  delta, precision, flags, kappa_max, store_scale, Nz, Mz,
                  Wza.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if planar else None,
                  va.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if planar else None,
                  int(s_begin), int(s_count))
    return cfg, (ua, Wa, Ka, Wza, va)


def bs_plan_tables_host(**kw):
    """Window starts [T*L] and windowed steering vectors (packed, complex128)
    computed by the library on the host (no device needed)."""
    cfg, keep = _make_config(**kw)
    Ls = cfg.s_count if 0 < cfg.s_count < cfg.L else cfg.L
    G = cfg.T * Ls
    start = np.empty(G, np.int32)
    at = np.empty(int(np.repeat(keep[1], Ls).sum()), np.complex128)
    _check(lib().bs_plan_tables_host(ctypes.byref(cfg), start.ctypes.data, at.ctypes.data),
           "bs_plan_tables_host")
    return start, at


class Plan:
    """A bs_plan: per-pair window tables and steering vectors on the device."""

    def __init__(self, *, N: int, F: int, L: int, M: int, u: Sequence[float],
                 W: Sequence[int], K: Sequence[int], P_train: int, P_test: int,
                 fc: float, fs: float, fd: float, delta: float,
                 precision: int = BS_PREC_FP32, flags: int = 0,
                 kappa_max: float = 0.0, store_scale: float = 0.0,
                 Nz: int = 1, Mz: int = 1, Wz: Optional[Sequence[int]] = None,
                 v: Optional[Sequence[float]] = None, s_begin: int = 0, s_count: int = 0):
        self.T = len(u)
        cfg, self._keep = _make_config(N, F, L, M, u, W, K, P_train, P_test, fc, fs, fd, delta,
                                       precision, flags, kappa_max, store_scale, Nz, Mz, Wz, v,
                                       s_begin, s_count)
        self.Nz, self.Mz = Nz, Mz
        self.N, self.F, self.L, self.M = N, F, L, M
        shard = 0 < s_count < L
        self.s_begin, self.s_count = (int(s_begin), int(s_count)) if shard else (0, L)
        self.P_train, self.P_test = P_train, P_test
        self.precision, self.flags = precision, flags
        h = _P()
        _check(lib().bs_plan_create(ctypes.byref(h), ctypes.byref(cfg)), "bs_plan_create")
        self._h = h
        s = _Sizes()
        _check(lib().bs_plan_sizes(h, ctypes.byref(s)), "bs_plan_sizes")
        self.sizes = Sizes(**{f: getattr(s, f) for f, _ in _Sizes._fields_})

    @classmethod
    def from_scene_config(cls, cfg, u, precision=BS_PREC_FP32, flags=0, v=None, **kw):
        """Plan for a ``synth.SceneConfig`` workload with target sines u (and,
        for a planar array, vertical sines v)."""
        planar = getattr(cfg, "Nz", 1) > 1
        if planar:
            kw.update(Nz=cfg.Nz, Mz=cfg.Mz, Wz=cfg.Wz_t, v=v)
        return cls(N=cfg.N, F=cfg.F, L=cfg.L, M=cfg.M, u=u, W=cfg.W, K=cfg.K,
                   P_train=cfg.P_tr, P_test=cfg.P_te, fc=cfg.fc, fs=cfg.fs, fd=cfg.fd,
                   delta=cfg.delta, precision=precision, flags=flags, **kw)

    @property
    def handle(self):
        return self._h

    @property
    def P(self) -> int:
        return self.P_train + self.P_test

    def offsets(self) -> dict:
        G = self.sizes.pairs
        out = {
            "start": np.empty(G, np.int32), "W": np.empty(G, np.int32), "K": np.empty(G, np.int32),
            "woff": np.empty(G + 1, np.int64), "ztr_off": np.empty(G + 1, np.int64),
            "zte_off": np.empty(G + 1, np.int64), "roff": np.empty(G + 1, np.int64),
            "a_tilde": np.empty(self.sizes.c_elems, np.complex128),
        }
        args = [out[k].ctypes.data for k in ("start", "W", "K", "woff", "ztr_off", "zte_off", "roff", "a_tilde")]
        _check(lib().bs_plan_offsets(self._h, *args), "bs_plan_offsets")
        return out

    def device_status(self) -> int:
        """Synchronise, return and clear the device error word (raises on a
        bounded-wait timeout)."""
        flags = ctypes.c_int32(0)
        st = lib().bs_plan_device_status(self._h, ctypes.byref(flags))
        _check(st, "bs_plan_device_status")
        return flags.value

    def set_device_flags(self, flags: int) -> None:
        """Write the device error word from the host (0 clears it)."""
        _check(lib().bs_plan_set_device_flags(self._h, int(flags)), "bs_plan_set_device_flags")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().bs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ztrain_dtype(plan: Plan):
    return torch.complex64 if plan.precision == BS_PREC_FP32 else (
        torch.float16 if plan.precision == BS_PREC_FP16 else torch.bfloat16)


@dataclass
class Buffers:
    x: torch.Tensor
    xc: torch.Tensor
    z_train: torch.Tensor
    z_test: torch.Tensor
    R: torch.Tensor
    c: torch.Tensor
    info: torch.Tensor
    out: torch.Tensor


def alloc_buffers(plan: Plan, device="cuda") -> Buffers:
    """Caller-owned device buffers of one whole pass (allocated by torch)."""
    s = plan.sizes
    zt = _ztrain_dtype(plan)
    ztr = (torch.empty(s.ztrain_elems, dtype=zt, device=device) if zt == torch.complex64
           else torch.empty(s.ztrain_elems * 2, dtype=zt, device=device))
    return Buffers(
        x=torch.empty(s.x_elems, dtype=torch.complex64, device=device),
        xc=torch.empty(s.xc_elems, dtype=torch.complex64, device=device),
        z_train=ztr,
        z_test=torch.empty(max(s.ztest_elems, 1), dtype=torch.complex64, device=device),
        R=torch.empty(s.r_elems, dtype=torch.complex128, device=device),
        c=torch.empty(s.c_elems, dtype=torch.complex64, device=device),
        info=torch.empty(s.pairs, dtype=torch.int32, device=device),
        out=torch.empty(max(s.out_elems, 1), dtype=torch.complex64, device=device),
    )


def _ztr_check(plan: Plan, z: torch.Tensor, name="z_train") -> int:
    s = plan.sizes
    dt = _ztrain_dtype(plan)
    n = s.ztrain_elems if dt == torch.complex64 else 2 * s.ztrain_elems
    return _ptr(z, dt, n, name)


def bs_channelize(plan: Plan, x: torch.Tensor, xc: torch.Tensor, P: Optional[int] = None, stream=None):
    P = plan.P if P is None else P
    n = P * plan.F * plan.N
    _check(lib().bs_channelize(plan.handle, _ptr(x, torch.complex64, n, "x"), P,
                               _ptr(xc, torch.complex64, n, "xc"), _stream(stream)), "bs_channelize")


def bs_beamspace(plan: Plan, xc: torch.Tensor, z_train: torch.Tensor, z_test: Optional[torch.Tensor],
                 stream=None):
    s = plan.sizes
    _check(lib().bs_beamspace(plan.handle, _ptr(xc, torch.complex64, s.xc_elems, "xc"),
                              _ztr_check(plan, z_train),
                              _ptr(z_test, torch.complex64, s.ztest_elems, "z_test"),
                              _stream(stream)), "bs_beamspace")


def bs_beamspace_full(plan: Plan, y: torch.Tensor, yb: torch.Tensor, nvec: int, stream=None):
    _check(lib().bs_beamspace_full(plan.handle, _ptr(y, torch.complex64, nvec * plan.N, "y"), nvec,
                                   _ptr(yb, torch.complex64, nvec * plan.M, "yb"), _stream(stream)),
           "bs_beamspace_full")


def bs_window_cov(plan: Plan, z_train: torch.Tensor, R: torch.Tensor,
                  delta_pair: Optional[torch.Tensor] = None, stream=None):
    s = plan.sizes
    _check(lib().bs_window_cov(plan.handle, _ztr_check(plan, z_train),
                               _ptr(delta_pair, torch.float32, s.pairs, "delta_pair"),
                               _ptr(R, torch.complex128, s.r_elems, "R"), _stream(stream)),
           "bs_window_cov")


def bs_mvdr_solve(plan: Plan, R: torch.Tensor, c: torch.Tensor, info: torch.Tensor, stream=None):
    s = plan.sizes
    _check(lib().bs_mvdr_solve(plan.handle, _ptr(R, torch.complex128, s.r_elems, "R"),
                               _ptr(c, torch.complex64, s.c_elems, "c"),
                               _ptr(info, torch.int32, s.pairs, "info"), _stream(stream)),
           "bs_mvdr_solve")


def bs_mvdr_solve_precond(plan: Plan, R: torch.Tensor, d: torch.Tensor, c: torch.Tensor, info: torch.Tensor,
                          stream=None):
    """bs_mvdr_solve with the diagonal preconditioner d (float32, packed
    like c; each entry rounded to a power of two by the library)."""
    s = plan.sizes
    _check(lib().bs_mvdr_solve_precond(plan.handle, _ptr(R, torch.complex128, s.r_elems, "R"),
                                       _ptr(d, torch.float32, s.c_elems, "d"),
                                       _ptr(c, torch.complex64, s.c_elems, "c"),
                                       _ptr(info, torch.int32, s.pairs, "info"), _stream(stream)),
           "bs_mvdr_solve_precond")


def bs_cov_solve(plan: Plan, z_train: torch.Tensor, c: torch.Tensor, info: torch.Tensor,
                 R: Optional[torch.Tensor] = None, delta_pair: Optional[torch.Tensor] = None, stream=None):
    s = plan.sizes
    _check(lib().bs_cov_solve(plan.handle, _ztr_check(plan, z_train),
                              _ptr(delta_pair, torch.float32, s.pairs, "delta_pair"),
                              _ptr(R, torch.complex128, s.r_elems, "R"),
                              _ptr(c, torch.complex64, s.c_elems, "c"),
                              _ptr(info, torch.int32, s.pairs, "info"), _stream(stream)), "bs_cov_solve")


def bs_cov_solve_noalloc(z_train: torch.Tensor, precision: int, W: torch.Tensor, K: torch.Tensor,
                         ztr_off: torch.Tensor, woff: torch.Tensor, a_hi: torch.Tensor, a_lo: torch.Tensor,
                         a_fp64: torch.Tensor, delta: float, c: torch.Tensor, info: torch.Tensor,
                         store_scale: float = 1.0, kappa_max: float = 0.0, flags: int = 0, stream=None):
    """Allocation-free covariance + solve (no plan): every per-pair table is a
    caller-provided device tensor; see bs_cov_solve_noalloc in include/bs.h."""
    pairs = W.numel()
    zt = torch.complex64 if precision == BS_PREC_FP32 else (
        torch.float16 if precision == BS_PREC_FP16 else torch.bfloat16)
    _check(lib().bs_cov_solve_noalloc(
        _ptr(z_train, zt, None, "z_train"), precision, store_scale,
        _ptr(W, torch.int32, pairs, "W"), _ptr(K, torch.int32, pairs, "K"),
        _ptr(ztr_off, torch.int64, pairs, "ztr_off"), _ptr(woff, torch.int64, pairs, "woff"),
        _ptr(a_hi, torch.complex64, None, "a_hi"), _ptr(a_lo, torch.complex64, None, "a_lo"),
        _ptr(a_fp64, torch.complex128, None, "a_fp64"), pairs, delta, kappa_max, flags,
        _ptr(c, torch.complex64, None, "c"), _ptr(info, torch.int32, pairs, "info"), _stream(stream)),
        "bs_cov_solve_noalloc")


def bs_autotune(plan: Plan, bufs: "Buffers", stream=None) -> dict:
    """Time the launch shapes of bs_cov_solve on these buffers; the fastest
    is kept in the plan."""
    s = plan.sizes
    thr, cps, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(lib().bs_autotune(plan.handle, _ztr_check(plan, bufs.z_train),
                             _ptr(bufs.R, torch.complex128, s.r_elems, "R"),
                             _ptr(bufs.c, torch.complex64, s.c_elems, "c"),
                             _ptr(bufs.info, torch.int32, s.pairs, "info"), _stream(stream),
                             ctypes.byref(thr), ctypes.byref(cps), ctypes.byref(ms)), "bs_autotune")
    return {"threads": thr.value, "ctas_per_sm": cps.value, "ms": ms.value}


class _TuneReport(ctypes.Structure):
    _fields_ = [("beamspace", ctypes.c_int32), ("covariance", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("beamspace_ms", ctypes.c_float * 4),
                ("covariance_ms", ctypes.c_float * 3), ("solve_ms", ctypes.c_float), ("fused_ms", ctypes.c_float)]


BEAMSPACE_VARIANTS = ("warp per beam residue", "bulk-copy-staged radix-16", "one-shot CTA per group",
                      "tensor-core DFT")
COVARIANCE_VARIANTS = ("CTA per pair", "warp per pair", "tensor cores")


def bs_autotune_pass(plan: Plan, bufs: "Buffers", stream=None) -> dict:
    """Time every kernel variant of the beamspace and covariance stages and
    the fused covariance + solve on these buffers (bufs.x holds the raw
    cube); the fastest of each is kept in the plan.  Returns the choices and
    the candidate times (ms, None where a variant does not apply)."""
    r = _TuneReport()
    _check(lib().bs_autotune_pass(plan.handle, ctypes.byref(_cbuf(plan, bufs)), _stream(stream), ctypes.byref(r)),
           "bs_autotune_pass")

    def ms(v):
        return None if v < 0 else float(v)
    return {
        "beamspace": BEAMSPACE_VARIANTS[r.beamspace] if r.beamspace >= 0 else None,
        "covariance": COVARIANCE_VARIANTS[r.covariance] if r.covariance >= 0 else None,
        "fused": bool(r.fused), "ctas_per_sm": r.ctas_per_sm,
        "beamspace_ms": {BEAMSPACE_VARIANTS[k]: ms(r.beamspace_ms[k]) for k in range(4)},
        "covariance_ms": {COVARIANCE_VARIANTS[k]: ms(r.covariance_ms[k]) for k in range(3)},
        "solve_ms": ms(r.solve_ms), "fused_ms": ms(r.fused_ms),
    }


def bs_set_launch(plan: Plan, threads: int, ctas_per_sm: int):
    _check(lib().bs_set_launch(plan.handle, threads, ctas_per_sm), "bs_set_launch")


def bs_apply(plan: Plan, z_test: torch.Tensor, c: torch.Tensor, out: torch.Tensor, stream=None):
    s = plan.sizes
    _check(lib().bs_apply(plan.handle, _ptr(z_test, torch.complex64, s.ztest_elems, "z_test"),
                          _ptr(c, torch.complex64, s.c_elems, "c"),
                          _ptr(out, torch.complex64, s.out_elems, "out"), _stream(stream)), "bs_apply")


def bs_lift(plan: Plan, c: torch.Tensor, c_hat: torch.Tensor, stream=None):
    """Lifted correlators c_hat [pairs * N] (complex64) from the weights c."""
    s = plan.sizes
    _check(lib().bs_lift(plan.handle, _ptr(c, torch.complex64, s.c_elems, "c"),
                         _ptr(c_hat, torch.complex64, s.pairs * plan.N, "c_hat"), _stream(stream)), "bs_lift")


def bs_apply_lifted(plan: Plan, xc: torch.Tensor, c_hat: torch.Tensor, out: torch.Tensor, stream=None):
    """out [pairs * Vte] = c_hat^H y on the channelised test vectors xc."""
    s = plan.sizes
    _check(lib().bs_apply_lifted(plan.handle, _ptr(xc, torch.complex64, s.xc_elems, "xc"),
                                 _ptr(c_hat, torch.complex64, s.pairs * plan.N, "c_hat"),
                                 _ptr(out, torch.complex64, s.out_elems, "out"), _stream(stream)),
           "bs_apply_lifted")


def bs_beam_pattern(plan: Plan, c_hat: torch.Tensor, u: torch.Tensor, pattern: torch.Tensor, stream=None):
    """pattern [pairs * len(u)] (float32) of every lifted correlator at the
    direction sines u (float64 device tensor)."""
    s = plan.sizes
    n = u.numel()
    _check(lib().bs_beam_pattern(plan.handle, _ptr(c_hat, torch.complex64, s.pairs * plan.N, "c_hat"), n,
                                 _ptr(u, torch.float64, n, "u"), _ptr(pattern, torch.float32, s.pairs * n, "pattern"),
                                 _stream(stream)), "bs_beam_pattern")


def bs_range_doppler(plan: Plan, out: torch.Tensor, pulse: torch.Tensor, work: torch.Tensor, rd_map: torch.Tensor,
                     stream=None):
    """Range-Doppler power maps [T * P_test * F] (float32) of the beamformed
    outputs; pulse: [F] complex64 spectrum; work: >= 2 T P_test F complex64."""
    s = plan.sizes
    n = plan.T * plan.P_test * plan.F
    _check(lib().bs_range_doppler(plan.handle, _ptr(out, torch.complex64, s.out_elems, "out"),
                                  _ptr(pulse, torch.complex64, plan.F, "pulse"),
                                  _ptr(work, torch.complex64, 2 * n, "work"),
                                  _ptr(rd_map, torch.float32, n, "map"), _stream(stream)), "bs_range_doppler")


def bs_cfar(plan: Plan, rd_map: torch.Tensor, threshold_db: float, floor: torch.Tensor, count: torch.Tensor,
            mask: Optional[torch.Tensor] = None, peak: Optional[torch.Tensor] = None, stream=None):
    """CFAR across the velocity bins of each target's map: floor
    [T * P_test * F] float32 (per cell), count [T] int32, optional mask
    [T * P_test * F] uint8 and peak [T] int32 (strongest detected cell
    d F + tau, -1 if none)."""
    n = plan.T * plan.P_test * plan.F
    _check(lib().bs_cfar(plan.handle, _ptr(rd_map, torch.float32, n, "map"), float(threshold_db),
                         _ptr(floor, torch.float32, n, "floor"), _ptr(count, torch.int32, plan.T, "count"),
                         _ptr(mask, torch.uint8, n, "mask"), _ptr(peak, torch.int32, plan.T, "peak"),
                         _stream(stream)), "bs_cfar")


def _cbuf(plan: Plan, b: Buffers) -> _Buffers:
    s = plan.sizes
    return _Buffers(_ptr(b.x, torch.complex64, s.x_elems, "x"),
                    _ptr(b.xc, torch.complex64, s.xc_elems, "xc"),
                    _ztr_check(plan, b.z_train),
                    _ptr(b.z_test, torch.complex64, s.ztest_elems, "z_test"),
                    _ptr(b.R, torch.complex128, s.r_elems, "R"),
                    _ptr(b.c, torch.complex64, s.c_elems, "c"),
                    _ptr(b.info, torch.int32, s.pairs, "info"),
                    _ptr(b.out, torch.complex64, s.out_elems, "out"))


def bs_run(plan: Plan, bufs: Buffers, stream=None):
    cb = _cbuf(plan, bufs)
    _check(lib().bs_run(plan.handle, ctypes.byref(cb), _stream(stream)), "bs_run")


def bs_run_host(plan: Plan, x_host: torch.Tensor, out_host: torch.Tensor, bufs: Buffers, stream=None):
    s = plan.sizes
    for t, n, name in ((x_host, s.x_elems, "x_host"), (out_host, s.out_elems, "out_host")):
        if t.is_cuda or not t.is_contiguous() or t.dtype != torch.complex64 or t.numel() < n:
            raise BsError(f"{name} must be a contiguous complex64 host tensor of >= {n} elements")
    cb = _cbuf(plan, bufs)
    _check(lib().bs_run_host(plan.handle, x_host.data_ptr(), out_host.data_ptr(), ctypes.byref(cb),
                             _stream(stream)), "bs_run_host")


class Graph:
    """CUDA graph of one whole pass on fixed buffers (bs_graph_create)."""

    def __init__(self, plan: Plan, bufs: Buffers, stream):
        if stream is None:
            raise BsError("graph capture needs a non-default stream")
        self._plan, self._bufs = plan, bufs
        self._cb = _cbuf(plan, bufs)
        h = _P()
        _check(lib().bs_graph_create(plan.handle, ctypes.byref(self._cb), _stream(stream), ctypes.byref(h)),
               "bs_graph_create")
        self._h = h

    def launch(self, stream):
        _check(lib().bs_graph_launch(self._h, _stream(stream)), "bs_graph_launch")

    def kernel_count(self) -> int:
        """Kernels one launch of the graph runs (bs_graph_kernel_count)."""
        n = ctypes.c_int32()
        _check(lib().bs_graph_kernel_count(self._h, ctypes.byref(n)), "bs_graph_kernel_count")
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().bs_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
