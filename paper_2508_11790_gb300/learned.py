"""Learned diagonal loading: binding of the MLP entry points, training-data
pipeline and training loop.

All arithmetic runs in the library's kernels (features, SINR judge, labels,
MLP forward / backward / Adam, minibatch gather); torch only allocates
device memory and the host only draws shuffling permutations and the
initial weights.

Training data (one scene at a time): two plans over the same raw records
share the channelised cube: one with the few-snapshot training count
K = 2W (the features and the candidate weights) and one with K_ref >> K
(the reference covariance that judges the output SINR).  For every loading
on a 61-point grid (0.1 .. 1e4, noise-variance units) the few-snapshot
weights are solved and judged; the label is the best loading and the
diagonal preconditioner it implies.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import (BS_PREC_FP32, BsError, Plan, _P, _check, _ptr, _stream, lib)

LOADING_GRID = 10.0 ** np.linspace(-1.0, 4.0, 61)


class _Mlp(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("n_out", ctypes.c_int32),
                ("step", ctypes.c_int32), ("master", ctypes.c_void_p), ("weights_bf16", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p)]


class _Work(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64)] + [(n, ctypes.c_void_p) for n in
                                                 ("z1", "h1", "z2", "h2", "y", "dy", "dh1", "dh2")]


_SIGS = {
    "bs_mlp_param_count": ([ctypes.c_int32] * 3, ctypes.c_int64),
    "bs_mlp_forward": ([ctypes.POINTER(_Mlp), _P, ctypes.c_int64, _P, ctypes.POINTER(_Work), _P], ctypes.c_int),
    "bs_mlp_train_step": ([ctypes.POINTER(_Mlp), _P, _P, ctypes.c_int64, ctypes.POINTER(_Work), ctypes.c_float, _P,
                           _P], ctypes.c_int),
    "bs_mlp_sync_bf16": ([ctypes.POINTER(_Mlp), _P], ctypes.c_int),
    "bs_gather_rows": ([_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P], ctypes.c_int),
    "bs_loading_from_mlp": ([_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             _P, _P], ctypes.c_int),
    "bs_precond_from_mlp": ([_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P, _P], ctypes.c_int),
}
_bound = False


def _lib():
    global _bound
    L = lib()
    if not _bound:
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _bound = True
    return L


def feature_count(W: int) -> int:
    return W * W + 2 * W + 2


def he_uniform_params(n_in: int, n_hidden: int, n_out: int, seed: int) -> np.ndarray:
    """Flat FP32 parameter vector in the library's layout, He-uniform weights
    (bound sqrt(6 / fan_in)) and zero biases, drawn in the order W1, W2, W3."""
    g = np.random.default_rng(seed)
    parts = []
    for fo, fi in ((n_hidden, n_in), (n_hidden, n_hidden), (n_out, n_hidden)):
        b = np.sqrt(6.0 / fi)
        parts += [g.uniform(-b, b, size=(fo, fi)).ravel(), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)


def unflatten(p: np.ndarray, n_in: int, n_hidden: int, n_out: int) -> dict:
    """Flat vector -> {W1, b1, W2, b2, W3, b3} (views, float64 copies)."""
    out, o = {}, 0
    for k, shape in (("W1", (n_hidden, n_in)), ("b1", (n_hidden,)), ("W2", (n_hidden, n_hidden)),
                     ("b2", (n_hidden,)), ("W3", (n_out, n_hidden)), ("b3", (n_out,))):
        n = int(np.prod(shape))
        out[k] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


class LoadingMLP:
    """The MLP's device buffers and its C entry points."""

    def __init__(self, n_in: int, n_out: int, n_hidden: int = 256, capacity: int = 4096, seed: int = 1,
                 device="cuda", params: Optional[np.ndarray] = None):
        L = _lib()
        self.n_in, self.n_hidden, self.n_out, self.capacity = n_in, n_hidden, n_out, capacity
        P = int(L.bs_mlp_param_count(n_in, n_hidden, n_out))
        self.P = P
        init = he_uniform_params(n_in, n_hidden, n_out, seed) if params is None else params.astype(np.float32)
        if init.size != P:
            raise BsError("parameter vector has the wrong size")
        f32 = dict(dtype=torch.float32, device=device)
        self.master = torch.from_numpy(init).to(device)
        self.bf16 = torch.empty(P, dtype=torch.bfloat16, device=device)
        self.grad = torch.zeros(P, **f32)
        self.m = torch.zeros(P, **f32)
        self.v = torch.zeros(P, **f32)
        self.work = {k: torch.empty(capacity * (n_out if k in ("y", "dy") else n_hidden), **f32)
                     for k in ("z1", "h1", "z2", "h2", "y", "dy", "dh1", "dh2")}
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self._m = _Mlp(n_in, n_hidden, n_out, 0, self.master.data_ptr(), self.bf16.data_ptr(),
                       self.grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr())
        self._w = _Work(capacity, *[self.work[k].data_ptr() for k in
                                    ("z1", "h1", "z2", "h2", "y", "dy", "dh1", "dh2")])
        _check(L.bs_mlp_sync_bf16(ctypes.byref(self._m), _stream(None)), "bs_mlp_sync_bf16")

    @property
    def step(self) -> int:
        return self._m.step

    def forward(self, X: torch.Tensor, batch: int, Y: torch.Tensor, stream=None):
        _check(_lib().bs_mlp_forward(ctypes.byref(self._m), _ptr(X, torch.float32, batch * self.n_in, "X"), batch,
                                     _ptr(Y, torch.float32, batch * self.n_out, "Y"), ctypes.byref(self._w),
                                     _stream(stream)), "bs_mlp_forward")

    def train_step(self, X: torch.Tensor, T: torch.Tensor, batch: int, lr: float, stream=None):
        _check(_lib().bs_mlp_train_step(ctypes.byref(self._m), _ptr(X, torch.float32, batch * self.n_in, "X"),
                                        _ptr(T, torch.float32, batch * self.n_out, "T"), batch,
                                        ctypes.byref(self._w), lr, self.loss.data_ptr(), _stream(stream)),
               "bs_mlp_train_step")

    def predict(self, X: torch.Tensor, n: int, stream=None) -> torch.Tensor:
        """Network outputs [n][n_out] for feature rows X (chunks of capacity)."""
        Y = torch.empty(n * self.n_out, dtype=torch.float32, device=X.device)
        for s in range(0, n, self.capacity):
            b = min(self.capacity, n - s)
            self.forward(X[s * self.n_in:], b, Y[s * self.n_out:], stream)
        return Y

    def precond(self, Y: torch.Tensor, n: int, W: int, stream=None) -> torch.Tensor:
        """The preconditioner seed d [n * W] (10^ of outputs 1..W)."""
        d = torch.empty(n * W, dtype=torch.float32, device=Y.device)
        _check(_lib().bs_precond_from_mlp(_ptr(Y, torch.float32, n * self.n_out, "Y"), self.n_out, n, W,
                                          d.data_ptr(), _stream(stream)), "bs_precond_from_mlp")
        return d

    def loading(self, Y: torch.Tensor, n: int, lo=0.1, hi=1e4, fallback=10.0, stream=None) -> torch.Tensor:
        d = torch.empty(n, dtype=torch.float32, device=Y.device)
        _check(_lib().bs_loading_from_mlp(_ptr(Y, torch.float32, n * self.n_out, "Y"), self.n_out, n, lo, hi,
                                          fallback, d.data_ptr(), _stream(stream)), "bs_loading_from_mlp")
        return d


@dataclass
class WindowData:
    X: torch.Tensor            # [n][n_in] features
    T: torch.Tensor            # [n][n_out] targets
    sinr: torch.Tensor         # [ngrid][n] SINR of each grid loading (reference covariance)
    best: torch.Tensor         # [n] grid loading of the label
    n: int


def scene_windows(cfg, x: np.ndarray, u, K_small: int, grid=LOADING_GRID, device="cuda") -> WindowData:
    """Features, labels and the SINR of every grid loading for all pairs of
    one scene.  cfg must give every target the same W; its P_tr records give
    the reference covariance (K_ref = P_tr * B vectors)."""
    from . import (alloc_buffers, bs_beamspace, bs_channelize, bs_mvdr_solve, bs_window_cov)
    W = int(cfg.W[0])
    T = cfg.T
    B = cfg.F // cfg.L
    K_ref = cfg.P_tr * B
    common = dict(N=cfg.N, F=cfg.F, L=cfg.L, M=cfg.M, u=u, W=[W] * T, P_train=cfg.P_tr, P_test=cfg.P_te,
                  fc=cfg.fc, fs=cfg.fs, fd=cfg.fd, delta=cfg.delta, precision=BS_PREC_FP32)
    ps = Plan(K=[K_small] * T, **common)
    pr = Plan(K=[K_ref] * T, **common)
    bs_ = alloc_buffers(ps, device)
    ztr_r = torch.empty(pr.sizes.ztrain_elems, dtype=torch.complex64, device=device)
    Rr = torch.empty(pr.sizes.r_elems, dtype=torch.complex128, device=device)
    bs_.x.copy_(torch.from_numpy(np.ascontiguousarray(x).reshape(-1)))
    G = ps.sizes.pairs
    zeros = torch.zeros(G, dtype=torch.float32, device=device)
    bs_channelize(ps, bs_.x, bs_.xc)
    bs_beamspace(ps, bs_.xc, bs_.z_train, bs_.z_test)
    bs_beamspace(pr, bs_.xc, ztr_r, bs_.z_test)
    Rs = torch.empty_like(bs_.R)
    bs_window_cov(ps, bs_.z_train, Rs, delta_pair=zeros)
    bs_window_cov(pr, ztr_r, Rr, delta_pair=zeros)
    L = _lib()
    nin, nout = feature_count(W), 1 + W
    X = torch.empty(G * nin, dtype=torch.float32, device=device)
    _check(L.bs_features(ps.handle, Rs.data_ptr(), X.data_ptr(), _stream(None)), "bs_features")
    sinr = torch.empty(len(grid) * G, dtype=torch.float64, device=device)
    dl = torch.empty(G, dtype=torch.float32, device=device)
    for k, d in enumerate(grid):
        dl.fill_(float(d))
        bs_window_cov(ps, bs_.z_train, bs_.R, delta_pair=dl)
        bs_mvdr_solve(ps, bs_.R, bs_.c, bs_.info)
        _check(L.bs_output_sinr(ps.handle, bs_.c.data_ptr(), Rr.data_ptr(), sinr[k * G:].data_ptr(),
                                _stream(None)), "bs_output_sinr")
    gd = torch.from_numpy(np.asarray(grid, dtype=np.float64)).to(device)
    Tt = torch.empty(G * nout, dtype=torch.float32, device=device)
    best = torch.empty(G, dtype=torch.float32, device=device)
    _check(L.bs_loading_labels(ps.handle, sinr.data_ptr(), len(grid), gd.data_ptr(), Rs.data_ptr(), nout,
                               Tt.data_ptr(), best.data_ptr(), _stream(None)), "bs_loading_labels")
    torch.cuda.synchronize()
    return WindowData(X, Tt, sinr.view(len(grid), G), best, G)


def concat(parts) -> WindowData:
    return WindowData(torch.cat([p.X for p in parts]), torch.cat([p.T for p in parts]),
                      torch.cat([p.sinr for p in parts], dim=1), torch.cat([p.best for p in parts]),
                      sum(p.n for p in parts))


def train(mlp: LoadingMLP, data: WindowData, epochs: int, batch: int, lr: float, seed: int = 0,
          stream=None) -> list:
    """Adam over shuffled minibatches; returns the mean loss of every epoch."""
    g = np.random.default_rng(seed)
    dev = data.X.device
    xb = torch.empty(batch * mlp.n_in, dtype=torch.float32, device=dev)
    tb = torch.empty(batch * mlp.n_out, dtype=torch.float32, device=dev)
    L = _lib()
    hist = []
    for _ in range(epochs):
        perm = torch.from_numpy(g.permutation(data.n).astype(np.int64)).to(dev)
        mlp.loss.zero_()
        nb = 0
        for s in range(0, data.n - batch + 1, batch):
            idx = perm[s:s + batch]
            _check(L.bs_gather_rows(data.X.data_ptr(), idx.data_ptr(), batch, mlp.n_in, xb.data_ptr(),
                                    _stream(stream)), "bs_gather_rows")
            _check(L.bs_gather_rows(data.T.data_ptr(), idx.data_ptr(), batch, mlp.n_out, tb.data_ptr(),
                                    _stream(stream)), "bs_gather_rows")
            mlp.train_step(xb, tb, batch, lr, stream)
            nb += 1
        torch.cuda.synchronize()
        hist.append(float(mlp.loss.item()) / max(nb, 1))
    return hist


def grid_sinr_at(data: WindowData, delta: float) -> torch.Tensor:
    """SINR of the grid loading nearest to delta (per pair)."""
    k = int(np.argmin(np.abs(np.log10(LOADING_GRID) - np.log10(delta))))
    return data.sinr[k]


def evaluate_scene(cfg, x: np.ndarray, u, K_small: int, mlp: LoadingMLP, base_delta: float = 10.0,
                   device="cuda") -> dict:
    """Runs the path on one scene with the network's per-pair loading and with
    the fixed loading base_delta; both weight sets are judged by the output
    SINR against the reference covariance (K_ref = P_tr * B vectors).  The
    learned loading is solved twice more with the network's preconditioner
    seed and with exact Jacobi scaling (diag(R + delta)^-1/2): their weights
    are compared with the unscaled solve's (the scaling is by powers of two,
    under which the FP32 Cholesky is exactly equivariant, so pairs solved in
    FP32 both ways agree bit for bit), the FP64 escalations (info = -2) of
    each are counted, and for the pairs that only the scaled pivot test
    escalates, the distance of the unscaled FP32 weights from the FP64 ones
    is reported.  Returns per-pair SINRs (numpy), the mean gain in dB and
    those counts."""
    from . import (alloc_buffers, bs_beamspace, bs_channelize, bs_mvdr_solve, bs_mvdr_solve_precond,
                   bs_window_cov)
    W = int(cfg.W[0])
    T = cfg.T
    B = cfg.F // cfg.L
    common = dict(N=cfg.N, F=cfg.F, L=cfg.L, M=cfg.M, u=u, W=[W] * T, P_train=cfg.P_tr, P_test=cfg.P_te,
                  fc=cfg.fc, fs=cfg.fs, fd=cfg.fd, delta=base_delta, precision=BS_PREC_FP32)
    ps = Plan(K=[K_small] * T, **common)
    pr = Plan(K=[cfg.P_tr * B] * T, **common)
    b = alloc_buffers(ps, device)
    ztr_r = torch.empty(pr.sizes.ztrain_elems, dtype=torch.complex64, device=device)
    Rr = torch.empty(pr.sizes.r_elems, dtype=torch.complex128, device=device)
    b.x.copy_(torch.from_numpy(np.ascontiguousarray(x).reshape(-1)))
    G = ps.sizes.pairs
    zeros = torch.zeros(G, dtype=torch.float32, device=device)
    bs_channelize(ps, b.x, b.xc)
    bs_beamspace(ps, b.xc, b.z_train, b.z_test)
    bs_beamspace(pr, b.xc, ztr_r, b.z_test)
    bs_window_cov(pr, ztr_r, Rr, delta_pair=zeros)
    L = _lib()
    Ru = torch.empty_like(b.R)
    bs_window_cov(ps, b.z_train, Ru, delta_pair=zeros)
    X = torch.empty(G * feature_count(W), dtype=torch.float32, device=device)
    _check(L.bs_features(ps.handle, Ru.data_ptr(), X.data_ptr(), _stream(None)), "bs_features")
    Y = mlp.predict(X, G)
    dhat = mlp.loading(Y, G, fallback=base_delta)
    seed = mlp.precond(Y, G, W)
    out = {}
    for name, dpair in (("learned", dhat), ("fixed", None)):
        bs_window_cov(ps, b.z_train, b.R, delta_pair=dpair)
        bs_mvdr_solve(ps, b.R, b.c, b.info)
        s = torch.empty(G, dtype=torch.float64, device=device)
        _check(L.bs_output_sinr(ps.handle, b.c.data_ptr(), Rr.data_ptr(), s.data_ptr(), _stream(None)),
               "bs_output_sinr")
        out[name] = s.cpu().numpy()
        out["escalations_" + name] = int((b.info == -2).sum().item())
    # the learned loading again (b.R holds the fixed loading now)
    bs_window_cov(ps, b.z_train, b.R, delta_pair=dhat)
    bs_mvdr_solve(ps, b.R, b.c, b.info)
    c_plain, info_plain = b.c.clone(), b.info.clone()
    Rd = b.R.view(G, W, W).diagonal(dim1=1, dim2=2).real
    jacobi = Rd.clamp_min(1e-30).rsqrt().to(torch.float32).reshape(-1).contiguous()
    for name, dvec in (("seed", seed), ("jacobi", jacobi)):
        c2 = torch.empty_like(b.c)
        info2 = torch.empty_like(b.info)
        bs_mvdr_solve_precond(ps, b.R, dvec, c2, info2)
        both = ((info2 == 0) & (info_plain == 0)).repeat_interleave(W)
        diff = (c2 - c_plain).abs().view(G, W).norm(dim=1) / c_plain.view(G, W).abs().norm(dim=1)
        out["escalations_learned_" + name] = int((info2 == -2).sum().item())
        out["max_weight_change_" + name] = float(diff[both.view(G, W)[:, 0]].max().item()) if both.any() else 0.0
        # pairs the scaled pivot test sends to FP64 that the unscaled test
        # left in FP32: how far the FP32 weights were from the FP64 ones
        moved = ((info2 == -2) & (info_plain == 0))
        out["fp32_error_where_" + name + "_escalates"] = float(diff[moved].max().item()) if moved.any() else 0.0
        # pairs the scaled pivot test sends to FP64 that the unscaled test
        # left in FP32: how far the FP32 weights were from the FP64 ones
        moved = ((info2 == -2) & (info_plain == 0))
        out["fp32_error_where_" + name + "_escalates"] = float(diff[moved].max().item()) if moved.any() else 0.0
    out["delta_hat"] = dhat.cpu().numpy()
    out["gain_db"] = float(np.mean(10.0 * np.log10(out["learned"] / out["fixed"])))
    return out


def _c5_scene_config(index: int):
    """The C5 geometry (N=1024, F=2048, L=128, M=2048, T=128, W=9, K=2W) with
    32 target-free training records for the reference covariance; one seed
    per scene index."""
    import dataclasses

    from synth import config_by_name, scaled_config
    base = config_by_name("C5")
    c = scaled_config(base, name="C5-learned", P_tr=32, P_te=0)
    return dataclasses.replace(c, seed=c.seed + 1000 + index)


def main(argv=None) -> dict:
    """Train the loading network on windows of `--scenes` scenes of the C5
    geometry and report the held-out gain over the fixed loading (JSON)."""
    import argparse
    import json
    import time

    from synth import make_scene
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--scenes", type=int, default=61)
    ap.add_argument("--test-scenes", type=int, default=2)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--save", default="")
    a = ap.parse_args(argv)
    t0 = time.time()
    parts = []
    for k in range(a.scenes):
        cfg = _c5_scene_config(k)
        sc = make_scene(cfg)
        parts.append(scene_windows(cfg, sc.x, sc.u_tgt, K_small=2 * int(cfg.W[0])))
    data = concat(parts)
    del parts
    t_data = time.time() - t0
    mlp = LoadingMLP(feature_count(9), 10, 256, capacity=a.batch, seed=7)
    t1 = time.time()
    hist = train(mlp, data, epochs=a.epochs, batch=a.batch, lr=a.lr)
    t_train = time.time() - t1
    gains, uppers = [], []
    for k in range(a.test_scenes):
        cfg = _c5_scene_config(10_000 + k)
        sc = make_scene(cfg)
        ev = evaluate_scene(cfg, sc.x, sc.u_tgt, K_small=18, mlp=mlp)
        held = scene_windows(cfg, sc.x, sc.u_tgt, K_small=18)
        best = held.sinr.max(dim=0).values.cpu().numpy()
        gains.append(ev["gain_db"])
        uppers.append(float(np.mean(10 * np.log10(best / ev["fixed"]))))
    out = {"windows": data.n, "scenes": a.scenes, "epochs": a.epochs, "batch": a.batch, "lr": a.lr,
           "loss_per_epoch": hist, "heldout_gain_db": gains, "heldout_grid_optimum_gain_db": uppers,
           "data_seconds": t_data, "train_seconds": t_train, "train_steps": mlp.step}
    if a.save:
        np.save(a.save, mlp.master.cpu().numpy())
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
