"""Multi-rank logic on CPU (gloo, world size 2): each rank builds the
library's host tables of its subband shard (bs_config.s_begin / s_count, the
plan a rank would run) and the gathered shards equal the unsharded plan's
tables; the oracle, sharded the same way, reproduces the unsharded result;
the bench's rank helpers (barrier, max over ranks) behave."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2508_11790_gb300.shard import aligned_blocks, shard_plan_blocks, shard_range, shard_subbands


def test_shard_range_partitions():
    for n in (0, 1, 7, 16, 128):
        for world in (1, 2, 3, 8):
            parts = [shard_range(n, world, r) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def test_aligned_blocks_cover_each_share():
    for L in (1, 8, 16, 128):
        for world in (1, 2, 3, 5, 8):
            covered = []
            for r in range(world):
                blocks = shard_plan_blocks(L, world, r)
                for s0, n in blocks:
                    assert n >= 1 and n & (n - 1) == 0 and s0 % n == 0
                    covered += list(range(s0, s0 + n))
                assert [i for s0, n in blocks for i in range(s0, s0 + n)] == list(shard_range(L, world, r))
            assert covered == list(range(L))
    assert aligned_blocks(0, 128) == [(0, 128)]
    assert shard_plan_blocks(128, 2, 1) == [(64, 64)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from synth import all_configs, make_scene, scaled_config
        import bench

        import paper_2508_11790_gb300 as P

        cfg = scaled_config(all_configs()["C1"], T=2, L=8, K=(32, 20), W=(5, 3))
        sc = make_scene(cfg)
        kw = dict(N=cfg.N, F=cfg.F, L=cfg.L, M=cfg.M, u=list(sc.u_tgt), W=cfg.W, K=cfg.K, P_train=cfg.P_tr,
                  P_test=cfg.P_te, fc=cfg.fc, fs=cfg.fs, fd=cfg.fd, delta=cfg.delta)
        # the library's tables of this rank's shard plans, keyed by (t, s)
        lib_tabs = {}
        for s0, n in shard_plan_blocks(cfg.L, world, rank):
            st, at = P.bs_plan_tables_host(**kw, s_begin=s0, s_count=n)
            wo = np.concatenate([[0], np.cumsum(np.repeat(cfg.W, n))])
            for t in range(cfg.T):
                for j in range(n):
                    g = t * n + j
                    lib_tabs[(t, s0 + j)] = (int(st[g]), at[wo[g]:wo[g + 1]])
        lib_gathered = [None] * world
        dist.all_gather_object(lib_gathered, lib_tabs)
        subs = shard_subbands(cfg.L, world, rank)
        res = O.run_pipeline(sc.x, cfg, sc.u_tgt, subbands=subs)
        mine = {(int(t), int(s)): c for t, s, c in zip(res.pairs.t, res.pairs.s, res.c)}
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        bench.barrier(world)
        m = bench.max_over_ranks(world, float(rank + 1))
        if rank == 0:
            merged = {}
            for part in gathered:
                assert not (set(part) & set(merged))
                merged.update(part)
            full = O.run_pipeline(sc.x, cfg, sc.u_tgt)
            ok = len(merged) == len(full.pairs.t)
            lib_merged = {}
            for part in lib_gathered:
                ok = ok and not (set(part) & set(lib_merged))
                lib_merged.update(part)
            st_full, at_full = P.bs_plan_tables_host(**kw)
            wo = np.concatenate([[0], np.cumsum(np.repeat(cfg.W, cfg.L))])
            ok = ok and len(lib_merged) == cfg.T * cfg.L
            for t in range(cfg.T):
                for s in range(cfg.L):
                    g = t * cfg.L + s
                    st, at = lib_merged[(t, s)]
                    ok = ok and st == int(st_full[g]) and np.array_equal(at, at_full[wo[g]:wo[g + 1]])
            for t, s, c in zip(full.pairs.t, full.pairs.s, full.c):
                ok = ok and np.allclose(merged[(int(t), int(s))], c, rtol=0, atol=1e-12)
            out.put((ok, m))
    finally:
        dist.destroy_process_group()


def test_subband_sharding_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    ok, m = q.get(timeout=10)
    assert ok
    assert m == 2.0
