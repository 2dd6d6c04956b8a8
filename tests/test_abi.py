"""C-ABI library: builds, loads and exports every declared entry point; host
logic (argument checks, window tables) checked without a GPU."""
import os
import re

import numpy as np
import pytest

import oracle as O
from synth import all_configs, make_scene

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_11790_gb300 import build as B
    B.build()
    import paper_2508_11790_gb300 as P
    return P


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bs_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(pkg):
    names = declared_functions()
    assert "bs_channelize" in names and "bs_mvdr_solve" in names
    L = pkg.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_every_declared_function_has_a_ctypes_signature(pkg):
    """A declared entry point called through ctypes without argtypes would pass
    64-bit device pointers as 32-bit C ints: every one has a registered
    signature (the package table, or learned.py's for the network structs)."""
    from paper_2508_11790_gb300 import learned
    sigs = set(pkg._SIGS) | set(learned._SIGS)
    missing = [n for n in declared_functions() if n not in sigs]
    assert not missing, missing


def test_status_strings(pkg):
    L = pkg.lib()
    assert L.bs_status_string(0) == b"ok"
    assert L.bs_status_string(6) == b"unsupported size"


def _kw(cfg, u=None, **over):
    u = [0.1, -0.2, 0.3, 0.5][: cfg.T] if u is None else u
    kw = dict(N=cfg.N, F=cfg.F, L=cfg.L, M=cfg.M, u=u, W=cfg.W, K=cfg.K, P_train=cfg.P_tr,
              P_test=cfg.P_te, fc=cfg.fc, fs=cfg.fs, fd=cfg.fd, delta=cfg.delta)
    kw.update(over)
    return kw


@pytest.mark.parametrize("over,code", [
    (dict(F=1000), 6), (dict(M=48), 6), (dict(L=3), 1), (dict(W=[33] * 4), 6),
    (dict(K=[10 ** 6] * 4), 1), (dict(u=[2.0, 0, 0, 0]), 1), (dict(delta=-1.0), 1),
    (dict(N=128), 6),
])
def test_config_validation(pkg, over, code):
    cfg = all_configs()["C1"]
    with pytest.raises(pkg.BsError) as ei:
        pkg.bs_plan_tables_host(**_kw(cfg, **over))
    assert pkg.lib().bs_status_string(code).decode() in str(ei.value)


@pytest.mark.parametrize("name", ["C1", "C2", "C3", "C4", "C5"])
def test_window_tables_match_oracle(pkg, name):
    """Window starts are bit-exact with the oracle's FP64 decision; the
    closed-form steering vectors match the oracle's direct sum."""
    cfg = all_configs()[name]
    rng = np.random.default_rng(7)
    u = np.sin(np.deg2rad(rng.uniform(-60, 60, size=cfg.T)))
    start, at = pkg.bs_plan_tables_host(**_kw(cfg, u))
    subs = range(cfg.L) if cfg.N * cfg.M <= 2 ** 18 else [0, 1, cfg.L // 2, cfg.L - 1]
    woff = np.concatenate([[0], np.cumsum(np.repeat(cfg.W, cfg.L))])
    for t in range(cfg.T):
        for s in subs:
            g = t * cfg.L + s
            st = O.window_start(u[t], s, cfg.W[t], cfg.L, cfg.M, cfg.fc, cfg.fs, cfg.fd)
            assert start[g] == st, (t, s)
            if t < 8:
                om = O.squinted_omega(u[t], O.subband_center_freq(s, cfg.L, cfg.fc, cfg.fs), cfg.fd)
                ref = O.windowed_steering(om, cfg.N, cfg.M, O.window_beams(st, cfg.W[t], cfg.M))
                got = at[woff[g]:woff[g + 1]]
                assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_window_ties_round_up(pkg):
    """x exactly on a half beam (u chosen so that x - W/2 + 1 is an integer):
    both sides pick the same start (ties round up)."""
    N, F, L, M = 16, 64, 4, 64
    fc = fs = fd = 1.0
    # subband s=2 (l=1): f = 1 + 0.5/4 = 1.125; x = u * M * f / 2 = 36 u
    u = [0.125, -0.125, 0.5]   # x = 4.5, -4.5, 18
    kw = dict(N=N, F=F, L=L, M=M, u=u, W=[4, 1, 3], K=[4, 4, 4], P_train=1, P_test=0,
              fc=fc, fs=fs, fd=fd, delta=1.0)
    start, _ = pkg.bs_plan_tables_host(**kw)
    for t in range(3):
        for s in range(L):
            assert start[t * L + s] == O.window_start(u[t], s, kw["W"][t], L, M, fc, fs, fd)


def test_planar_window_tables_match_oracle(pkg):
    """Planar plans: horizontal window starts and the windowed steering
    vectors (Kronecker of the two axes) computed by the library on the host
    equal the planar oracle's."""
    from oracle import upa as U
    from synth import scaled_config
    cfg = scaled_config(all_configs()["C1"], name="upa-tables", N=128, Nz=4, M=512, Mz=8, T=5,
                        W=(8, 16, 4, 2, 6), Wz=(2, 4, 4, 1, 3), K=40, P_tr=2, P_te=1)
    sc = make_scene(cfg)
    start, at = pkg.bs_plan_tables_host(N=cfg.N, F=cfg.F, L=cfg.L, M=cfg.M, u=sc.u_tgt, W=cfg.W, K=cfg.K,
                                        P_train=cfg.P_tr, P_test=cfg.P_te, fc=cfg.fc, fs=cfg.fs, fd=cfg.fd,
                                        delta=cfg.delta, Nz=cfg.Nz, Mz=cfg.Mz, Wz=cfg.Wz_t, v=sc.v_tgt)
    D = U.dft2d(cfg.Mx, cfg.Nx, cfg.Mz, cfg.Nz)
    e = 0
    for t in range(cfg.T):
        Wz = cfg.Wz_t[t]
        Wx = cfg.W[t] // Wz
        for s in range(cfg.L):
            f = O.subband_center_freq(s, cfg.L, cfg.fc, cfg.fs)
            sx = O.window_start(float(sc.u_tgt[t]), s, Wx, cfg.L, cfg.Mx, cfg.fc, cfg.fs, cfg.fd)
            sz = O.window_start(float(sc.v_tgt[t]), s, Wz, cfg.L, cfg.Mz, cfg.fc, cfg.fs, cfg.fd)
            assert start[t * cfg.L + s] == sx
            beams = U.window_beams2d(sx, Wx, cfg.Mx, sz, Wz, cfg.Mz)
            a = D[beams] @ U.steering2d(O.squinted_omega(float(sc.u_tgt[t]), f, cfg.fd),
                                        O.squinted_omega(float(sc.v_tgt[t]), f, cfg.fd), cfg.Nx, cfg.Nz)
            np.testing.assert_allclose(at[e:e + cfg.W[t]], a, atol=1e-12)
            e += cfg.W[t]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 5])
def test_subband_shard_tables_concatenate(pkg, world):
    """Plans restricted to aligned power-of-two subband blocks (the blocks of
    each rank's share, shard_plan_blocks) hold exactly the window starts and
    steering vectors of the same pairs of the unsharded plan: pair
    (t, s_begin + j) of a shard is pair t s_count + j of its tables."""
    from paper_2508_11790_gb300.shard import shard_plan_blocks
    base = all_configs()["C2"]
    u = np.sin(np.deg2rad(np.random.default_rng(3).uniform(-60, 60, size=base.T)))
    start, at = pkg.bs_plan_tables_host(**_kw(base, u))
    L, T, W = base.L, base.T, np.asarray(base.W)
    woff = np.concatenate([[0], np.cumsum(np.repeat(W, L))])
    seen = np.zeros((T, L), bool)
    for rank in range(world):
        for s0, n in shard_plan_blocks(L, world, rank):
            st, a = pkg.bs_plan_tables_host(**_kw(base, u, s_begin=s0, s_count=n))
            assert st.shape == (T * n,)
            wo = np.concatenate([[0], np.cumsum(np.repeat(W, n))])
            for t in range(T):
                for j in range(n):
                    g, gl = t * L + s0 + j, t * n + j
                    assert st[gl] == start[g]
                    assert np.array_equal(a[wo[gl]:wo[gl + 1]], at[woff[g]:woff[g + 1]])
                    assert not seen[t, s0 + j]
                    seen[t, s0 + j] = True
    assert seen.all()


@pytest.mark.parametrize("s_begin,s_count", [(2, 4), (0, 3), (-4, 4), (60, 8)])
def test_subband_shard_validation(pkg, s_begin, s_count):
    """A shard must be an aligned power-of-two block inside the L subbands."""
    base = all_configs()["C2"]
    with pytest.raises(pkg.BsError):
        pkg.bs_plan_tables_host(**_kw(base, s_begin=s_begin, s_count=s_count))
