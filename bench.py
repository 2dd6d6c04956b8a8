#!/usr/bin/env python
"""Benchmark of the windowed beamspace MVDR hot path on GB300.

One step = one whole pass of the path over one synthetic batch: channelise
(F-point FFT of every element of every record), beamspace + window gather
(zero-padded M-point spatial FFT), loaded window covariance, Cholesky MVDR
solve and apply, for every (target, subband) pair.  Metric: (target,
subband) MVDR solves per second = pairs / step time.

Default workload: N=1024 elements, F=2048, L=128 subbands, M=2048, W=9,
K=512, T=64 targets (8192 pairs), 32 training + 8 test records (671 MB raw
cube, larger than L2, so no flush is needed between steps), FP16 training
windows (the mixed-precision configuration); --precision fp32 for FP32.
The other workloads (--workload C1, C2, C4, C5) default to FP32 windows,
the precision their configurations name.

Arms:  --impl ours (default): the CUDA path through the C ABI.
       --impl reference: the FP64 CPU oracle on the host cores, one bounded
       sample of the workload per step.
Under torchrun every rank runs its own batch (independent problems, weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import all_configs, make_scene  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="C3")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16"], default=None,
                    help="window precision (default: fp16 for C3, fp32 otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time bs_run calls instead of a CUDA graph")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the pass (kernel variant per stage, fused or not) before timing")
    ap.add_argument("--fused", action="store_true", help="fused persistent covariance + solve kernel")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="budget of the oracle sample timed for cpu_baseline")
    a = ap.parse_args()
    if a.precision is None:
        a.precision = "fp16" if a.workload == "C3" else "fp32"
    return a


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload_desc(cfg):
    return {
        "workload": f"{cfg.name}: {cfg.description}",
        "pairs": cfg.pairs, "N": cfg.N, "F": cfg.F, "L": cfg.L, "M": cfg.M, "T": cfg.T,
        "W": cfg.W[0] if len(set(cfg.W)) == 1 else "per-target",
        "K": cfg.K[0] if len(set(cfg.K)) == 1 else "per-target",
        "P_train": cfg.P_tr, "P_test": cfg.P_te,
        "l2": "no flush: raw cube %.0f MB > 129 MB L2" % (cfg.P * cfg.F * cfg.N * 8 / 1e6),
    }


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- distributed
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, value: float) -> float:
    if ws == 1:
        return value
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------- oracle leg
def oracle_sample(cfg, scene, seconds: float, subband_order=None):
    """Run the oracle subband by subband (all targets) until `seconds` pass.
    Returns (pairs done, elapsed seconds, results by subband)."""
    import oracle as O
    order = subband_order if subband_order is not None else list(range(cfg.L))
    done, results = 0, {}
    t0 = time.perf_counter()
    for s in order:
        res = O.run_pipeline(scene.x, cfg, scene.u_tgt, subbands=[s])
        results[s] = res
        done += len(res.pairs.t)
        if time.perf_counter() - t0 >= seconds:
            break
    return done, time.perf_counter() - t0, results


def run_reference(args):
    ws, rank, _ = dist_init()
    cfg = all_configs()[args.workload]
    if rank != 0:
        return
    scene = make_scene(cfg)
    import oracle as O
    times, pairs = [], []
    order = [(7 * i) % cfg.L for i in range(args.warmup + args.steps)]
    for i, s in enumerate(order):
        t0 = time.perf_counter()
        res = O.run_pipeline(scene.x, cfg, scene.u_tgt, subbands=[s])
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            pairs.append(len(res.pairs.t))
    value = sum(pairs) / sum(times)
    cores = os.cpu_count()
    sample = (f"one subband (all {cfg.T} targets, all records and elements) per step; "
              f"value = pairs / oracle time")
    line = {
        "impl": "reference", "metric": "(target,subband) MVDR solves/sec", "value": value,
        "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_desc(cfg), precision=args.precision,
                       parallelism=f"{ws} independent batch(es)"),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- our arm
def algorithmic_bytes(plan, cfg):
    s = plan.sizes
    raw = cfg.P * cfg.F * cfg.N * 8
    return {
        "channelize": 2 * raw,
        "beamspace": raw + s.ztrain_bytes + 8 * s.ztest_elems,
        "window_cov": s.ztrain_bytes + 16 * s.r_elems,
        "cov_solve": s.ztrain_bytes + 16 * s.r_elems + 24 * s.c_elems + 8 * s.c_elems + 4 * s.pairs,
        "mvdr_solve": 16 * s.r_elems + 24 * s.c_elems + 8 * s.c_elems + 4 * s.pairs,
        "apply": 8 * s.ztest_elems + 8 * s.c_elems + 8 * s.out_elems,
    }


def kernel_traffic(stage, workload):
    """DRAM bytes per launch of a stage from the committed ncu summary, if it
    was taken on this workload and precision and the kernel source has not
    changed since (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    ent = d.get(workload, {}).get(stage)
    if not ent:
        return None
    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return ent["bytes_per_launch"] if h == ent["source_sha256_16"] else None


def run_ours(args):
    ws, rank, local = dist_init()
    import paper_2508_11790_gb300 as P

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = all_configs()[args.workload]
    scene = make_scene(cfg)
    prec = {"fp32": P.BS_PREC_FP32, "fp16": P.BS_PREC_FP16, "bf16": P.BS_PREC_BF16}[args.precision]
    plan = P.Plan.from_scene_config(cfg, scene.u_tgt, precision=prec,
                                    flags=P.BS_FLAG_FUSED if args.fused else 0)
    b = P.alloc_buffers(plan, dev)
    b.x.copy_(torch.from_numpy(scene.x.reshape(-1)))
    stream = torch.cuda.Stream(dev)

    tune = None
    if args.autotune:
        tune = P.bs_autotune_pass(plan, b, stream=stream)
    fused = args.fused or bool(tune and tune["fused"])

    def stages_for(pl, bb):
        return [
            ("channelize", lambda: P.bs_channelize(pl, bb.x, bb.xc, stream=stream)),
            ("beamspace", lambda: P.bs_beamspace(pl, bb.xc, bb.z_train, bb.z_test, stream=stream)),
        ] + ([
            ("cov_solve", lambda: P.bs_cov_solve(pl, bb.z_train, bb.c, bb.info, R=bb.R, stream=stream)),
        ] if fused else [
            ("window_cov", lambda: P.bs_window_cov(pl, bb.z_train, bb.R, stream=stream)),
            ("mvdr_solve", lambda: P.bs_mvdr_solve(pl, bb.R, bb.c, bb.info, stream=stream)),
        ]) + [
            ("apply", lambda: P.bs_apply(pl, bb.z_test, bb.c, bb.out, stream=stream)),
        ]

    stages = stages_for(plan, b)

    def plain_stages(pl, bb):
        return [
            ("channelize", lambda: P.bs_channelize(pl, bb.x, bb.xc, stream=stream)),
            ("beamspace", lambda: P.bs_beamspace(pl, bb.xc, bb.z_train, bb.z_test, stream=stream)),
            ("window_cov", lambda: P.bs_window_cov(pl, bb.z_train, bb.R, stream=stream)),
            ("mvdr_solve", lambda: P.bs_mvdr_solve(pl, bb.R, bb.c, bb.info, stream=stream)),
            ("apply", lambda: P.bs_apply(pl, bb.z_test, bb.c, bb.out, stream=stream)),
        ]

    graph = None if args.no_graph else P.Graph(plan, b, stream)
    # kernels one pass launches, read from a captured graph of the pass
    kernels_per_step = (graph or P.Graph(plan, b, stream)).kernel_count()

    def step():
        if graph is not None:
            graph.launch(stream)
        else:
            P.bs_run(plan, b, stream=stream)

    def timed_loop(fn, K):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
        return e0.elapsed_time(e1)

    def stage_breakdown(stg, K):
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in stg] for _ in range(K)]
        torch.cuda.synchronize(dev)
        for k in range(K):
            for (name, fn), (a, z) in zip(stg, ev[k]):
                a.record(stream)
                fn()
                z.record(stream)
        torch.cuda.synchronize(dev)
        return {name: float(np.mean([ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(K)]))
                for i, (name, _) in enumerate(stg)}

    sampler = ClockSampler(dev.index)
    sampler.start()
    plain = None
    if not args.no_plain:
        pplan = P.Plan.from_scene_config(cfg, scene.u_tgt, precision=P.BS_PREC_FP32,
                                         flags=P.BS_FLAG_PLAIN)
        pb = P.alloc_buffers(pplan, dev)
        pb.x.copy_(b.x)
        for _ in range(args.warmup):
            P.bs_run(pplan, pb, stream=stream)
        pms = timed_loop(lambda: P.bs_run(pplan, pb, stream=stream), args.steps) / args.steps
        pbd = stage_breakdown(plain_stages(pplan, pb), max(3, args.steps // 4))
        p_core = pbd["window_cov"] + pbd["mvdr_solve"]
        plain = {"ms_per_step": pms, "value": cfg.pairs / (pms / 1e3),
                 "solve_core_ms": p_core, "solve_core_pairs_per_s": cfg.pairs / (p_core / 1e3),
                 "path": "one CTA per pair, FP32 sums, one thread per Cholesky, no refinement"}
        del pb, pplan
    # the tuned FP32 path (FP32 windows through the library's own covariance
    # and solve kernels) as a second, harder denominator
    fp32_tuned = None
    if not args.no_plain and prec != P.BS_PREC_FP32:
        tplan = P.Plan.from_scene_config(cfg, scene.u_tgt, precision=P.BS_PREC_FP32)
        tb = P.alloc_buffers(tplan, dev)
        tb.x.copy_(b.x)
        P.bs_run(tplan, tb, stream=stream)
        tbd = stage_breakdown([
            ("window_cov", lambda: P.bs_window_cov(tplan, tb.z_train, tb.R, stream=stream)),
            ("mvdr_solve", lambda: P.bs_mvdr_solve(tplan, tb.R, tb.c, tb.info, stream=stream)),
        ], max(3, args.steps // 4))
        t_core = tbd["window_cov"] + tbd["mvdr_solve"]
        fp32_tuned = {"solve_core_ms": t_core, "solve_core_pairs_per_s": cfg.pairs / (t_core / 1e3),
                      "path": "FP32 windows through the library's FP32 covariance and solve kernels"}
        del tb, tplan

    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(scene.x.reshape(-1)).pin_memory()
        oh = torch.empty(plan.sizes.out_elems, dtype=torch.complex64).pin_memory()
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):   # first host-to-device copies map the pinned pages
                P.bs_run_host(plan, xh, oh, b, stream=stream)
            barrier(ws)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                P.bs_run_host(plan, xh, oh, b, stream=stream)
            dt = (time.perf_counter() - t0) / args.steps
        dt = max_over_ranks(ws, dt)
        e2e = {"value": ws * cfg.pairs / dt, "unit": "pairs/s", "api": "bs_run_host",
               "h2d_bytes_per_step": xh.numel() * 8, "d2h_bytes_per_step": oh.numel() * 8,
               "ms_per_step": dt * 1e3}

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    # keep the GPU loaded for ~1 s right before the timed region so that the
    # clock samples (every 100 ms) describe the clocks it runs at
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 1.0:
        for _ in range(20):
            step()
        torch.cuda.synchronize(dev)
    total_ms = timed_loop(step, args.steps)
    ms_step = max_over_ranks(ws, total_ms / args.steps)
    value = ws * cfg.pairs / (ms_step / 1e3)
    breakdown = stage_breakdown(stages, args.steps)
    other = stage_breakdown([
        ("cov_solve", lambda: P.bs_cov_solve(plan, b.z_train, b.c, b.info, R=b.R, stream=stream)),
    ] if not fused else [
        ("window_cov", lambda: P.bs_window_cov(plan, b.z_train, b.R, stream=stream)),
        ("mvdr_solve", lambda: P.bs_mvdr_solve(plan, b.R, b.c, b.info, stream=stream)),
    ], max(3, args.steps // 4))
    step()   # leave the timed path's results in the buffers
    # lifted correlator (a row beyond the hot path): timed on its own, after
    # the pass, on the pass's weights and channelised cube
    lifted = None
    if rank == 0:
        c_hat = torch.empty(cfg.pairs * cfg.N, dtype=torch.complex64, device=dev)
        out_l = torch.empty(max(plan.sizes.out_elems, 1), dtype=torch.complex64, device=dev)
        n_dirs = 181
        u_dirs = torch.linspace(-1.0, 1.0, n_dirs, dtype=torch.float64, device=dev)
        pattern = torch.empty(cfg.pairs * n_dirs, dtype=torch.float32, device=dev)
        lb = stage_breakdown([
            ("lift", lambda: P.bs_lift(plan, b.c, c_hat, stream=stream)),
            ("apply_lifted", lambda: P.bs_apply_lifted(plan, b.xc, c_hat, out_l, stream=stream)),
            ("beam_pattern", lambda: P.bs_beam_pattern(plan, c_hat, u_dirs, pattern, stream=stream)),
        ], max(3, args.steps // 4))
        vte = plan.sizes.Vte
        lift_bytes = cfg.pairs * cfg.N * 8 + plan.sizes.c_elems * 8
        al_flops = 8.0 * cfg.pairs * vte * cfg.N
        bp_flops = 8.0 * cfg.pairs * n_dirs * cfg.N
        lifted = {"lift_ms": lb["lift"], "lift_GB/s": lift_bytes / (lb["lift"] / 1e3) / 1e9,
                  "apply_lifted_ms": lb["apply_lifted"],
                  "apply_lifted_TFLOP/s_fp32": al_flops / (lb["apply_lifted"] / 1e3) / 1e12,
                  "beam_pattern_ms": lb["beam_pattern"], "beam_pattern_directions": n_dirs,
                  "beam_pattern_TFLOP/s_fp32": bp_flops / (lb["beam_pattern"] / 1e3) / 1e12}
        del c_hat, out_l, pattern
    # range-Doppler maps and CFAR of the pass's outputs (rows beyond the hot
    # path; the synthetic pulse is the scene's)
    radar = None
    if rank == 0 and cfg.P_te > 0:
        from synth import pulse
        nmap = cfg.T * cfg.P_te * cfg.F
        pspec = torch.from_numpy(np.fft.fft(pulse(cfg.F), norm="ortho").astype(np.complex64)).to(dev)
        work = torch.empty(2 * nmap, dtype=torch.complex64, device=dev)
        rmap = torch.empty(nmap, dtype=torch.float32, device=dev)
        rfloor = torch.empty(nmap, dtype=torch.float32, device=dev)
        rpeak = torch.empty(cfg.T, dtype=torch.int32, device=dev)
        rcount = torch.empty(cfg.T, dtype=torch.int32, device=dev)
        rmask = torch.empty(nmap, dtype=torch.uint8, device=dev)
        rb = stage_breakdown([
            ("range_doppler", lambda: P.bs_range_doppler(plan, b.out, pspec, work, rmap, stream=stream)),
            ("cfar", lambda: P.bs_cfar(plan, rmap, 10.0, rfloor, rcount, rmask, rpeak, stream=stream)),
        ], max(3, args.steps // 4))
        radar = {"range_doppler_ms": rb["range_doppler"], "cfar_ms": rb["cfar"], "map_cells": nmap}
        del work, rmap, rmask, rfloor
    clocks = sampler.stop()
    clocks["window"] = "plain-path, e2e, 1 s load soak, timed and per-stage loops (100 ms samples)"
    info = b.info.cpu().numpy()
    peaks, peak_kind = load_peaks()
    abytes = algorithmic_bytes(plan, cfg)
    dom = max(breakdown, key=breakdown.get)
    achieved = abytes[dom] / (breakdown[dom] / 1e3) / 1e9
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": kernel_traffic(dom, f"{args.workload}/{args.precision}"),
                "peak_source": f"{peak_kind} HBM copy bandwidth",
                "algorithmic_bytes": abytes[dom]}
    per_stage = {k: {"ms": v, "GB/s": abytes[k] / (v / 1e3) / 1e9,
                     "frac_hbm": abytes[k] / (v / 1e3) / 1e9 / peaks["hbm_gbs"]}
                 for k, v in breakdown.items()}
    solve_core_ms = (breakdown["cov_solve"] if fused
                     else breakdown["window_cov"] + breakdown["mvdr_solve"])
    if plain is not None:
        plain["solve_core_speedup_of_ours"] = plain["solve_core_ms"] / solve_core_ms
        plain["step_speedup_of_ours"] = plain["ms_per_step"] / ms_step
    if fp32_tuned is not None:
        fp32_tuned["solve_core_speedup_of_ours"] = fp32_tuned["solve_core_ms"] / solve_core_ms

    cpu = None
    accuracy = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        order = [0, cfg.L // 2, cfg.L - 1] + [s for s in range(1, cfg.L) if s not in (cfg.L // 2, cfg.L - 1)]
        done, el, results = oracle_sample(cfg, scene, args.cpu_seconds, order)
        cpu = {"value": done / el, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(results)} subband(s) x {cfg.T} targets = {done} pairs of the same "
                         f"workload (all records and elements), FP64 numpy, {el:.1f} s"}
        import oracle as O
        off = plan.offsets()
        cc = b.c.cpu().numpy()
        errs, losses = [], []
        for s, res in results.items():
            for k in range(len(res.pairs.t)):
                g = int(res.pairs.t[k]) * cfg.L + int(res.pairs.s[k])
                cg = cc[off["woff"][g]:off["woff"][g + 1]].astype(np.complex128)
                errs.append(float(np.linalg.norm(cg - res.c[k]) / np.linalg.norm(res.c[k])))
                losses.append(abs(O.sinr_loss_db(cg, res.c[k], res.pairs.a_tilde[k], res.R[k])))
        # the same loss judged against an interference-plus-noise covariance
        # from 8 independent target-free records of the scene (never seen by
        # the weights), on the first subbands of the sample
        from synth import reference_records
        x_ref = reference_records(cfg, 8)
        ref_losses = []
        for s in list(results)[:4]:
            res = results[s]
            Rin = O.reference_covariances(x_ref, cfg, scene.u_tgt, subbands=[s])
            for k in range(len(res.pairs.t)):
                g = int(res.pairs.t[k]) * cfg.L + int(res.pairs.s[k])
                cg = cc[off["woff"][g]:off["woff"][g + 1]].astype(np.complex128)
                ref_losses.append(abs(O.sinr_loss_db(cg, res.c[k], res.pairs.a_tilde[k], Rin[k])))
        del x_ref
        accuracy = {"pairs_checked": len(errs), "max_weight_rel_err": max(errs),
                    "median_weight_rel_err": float(np.median(errs)),
                    "max_abs_sinr_loss_db": max(losses),
                    "sinr_judge": "sample: the oracle's loaded covariance of the same training windows",
                    "max_abs_sinr_loss_db_reference_cov": max(ref_losses),
                    "reference_cov_pairs": len(ref_losses),
                    "reference_cov": "unloaded covariance of 8 independent target-free records of the same scene"}

    if rank == 0:
        dtype = {"fp32": "f32", "fp16": "f16 windows, f32/f64 solve", "bf16": "bf16 windows, f32/f64 solve"}[args.precision]
        line = {
            "metric": "(target,subband) MVDR solves/sec", "value": value, "unit": "pairs/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic",
            "config": dict(workload_desc(cfg), precision=args.precision,
                           parallelism=f"{ws} independent batch(es)"),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": kernels_per_step * args.steps,
            "timed_as": "CUDA graph of the whole pass" if graph is not None else "bs_run calls",
            "autotune": tune,
            "clocks": clocks, "stages": per_stage, "solve_core_ms": solve_core_ms,
            "other_solve_core_ms": other,
            "plain_fp32": plain, "fp32_tuned": fp32_tuned, "accuracy": accuracy, "lifted_correlator": lifted, "range_doppler": radar,
            "info_counts": {str(k): int(v) for k, v in zip(*np.unique(info, return_counts=True))},
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
