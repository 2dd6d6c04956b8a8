"""Multi-rank logic on CPU (gloo, world size 2): subband sharding of the path
reproduces the unsharded result, and the bench's rank helpers (barrier,
max over ranks) behave."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2508_11790_gb300.shard import shard_range, shard_subbands


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

        cfg = scaled_config(all_configs()["C1"], T=2, L=8, K=(32, 20), W=(5, 3))
        sc = make_scene(cfg)
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
