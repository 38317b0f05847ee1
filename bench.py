#!/usr/bin/env python3
"""Benchmark of the batched explicit patch update on GB300.

Workload: 3D compressible Euler (5 variables, gamma = 1.4), first-order FV
with the Rusanov flux and SSP-RK3, on the AMR-like patch mix
4096 x 8^3 + 1024 x 16^3 + 128 x 32^3 voxels (10,485,760 voxels, halo 1),
seeded smooth Fourier-mode initial data.  One benchmark step is one replay of
a CUDA graph of 100 time steps; each time step is the device-side CFL time
step (CFL 0.4) followed by three batched stage launches (one per SSP-RK3
stage).  Metric: FP64 cell-updates per second (voxels x time steps / s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain C++ implementation the
CUDA path is checked against) on the host cores: a deliberately slow
baseline, not a target.  Under torchrun every rank runs an independent
replica (the patch update of one rank needs no data from another).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_19273_gb300 import synth  # noqa: E402

METRIC = "FP64 cell-updates/s + % of roofline; learned-seed vs plain con2prim at 1e-12"
UNIT = "cell-updates/s"
INNER_STEPS = 100
CFL = 0.4
FLOPS_FILE = os.path.join(ROOT, "oracle", "flop_counts.json")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload_config(mesh):
    return {"workload": "euler3d_fv_rusanov_ssprk3_amr_mix", "pde": "3D Euler (5 vars, gamma 1.4)",
            "patches": "4096x8^3 + 1024x16^3 + 128x32^3", "voxels": mesh.nvox, "halo": 1,
            "time_steps_per_step": INNER_STEPS, "rk": "SSP-RK3", "cfl": CFL, "cuda_graph": True,
            "l2": "no flush: each state array (420 MB) is larger than L2 (129 MB)",
            "seed": synth.SEED_BASE + 1}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for_smi(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        first = vis.split(",")[dev] if vis else str(dev)
        return first


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(mesh, prim, budget_s, threads=0):
    """Oracle SSP-RK3 steps on the full workload for about budget_s seconds (at least one step)."""
    import oracle
    cores = oracle.num_threads(threads)
    q = oracle.prim2con(synth.PDE_EULER3D, prim, mesh.var_stride)
    steps, t0 = 0, time.perf_counter()
    while True:
        oracle.rk_steps(0, synth.PDE_EULER3D, 3, mesh.patches, 1, mesh.var_stride, q, rk=3, steps=1, cfl=CFL)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el / steps * (steps + 1) > 2.5 * budget_s:
            break
    return mesh.nvox * steps / el, cores, steps, el


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    w = synth.workload("euler3d")
    mesh = w.mesh
    prim = synth.euler_prims(mesh, w.seed)
    import oracle
    cores = oracle.num_threads(0)
    q = oracle.prim2con(synth.PDE_EULER3D, prim, mesh.var_stride)
    for _ in range(args.warmup):
        oracle.rk_steps(0, 3, 3, mesh.patches, 1, mesh.var_stride, q, rk=3, steps=1, cfl=CFL)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rk_steps(0, 3, 3, mesh.patches, 1, mesh.var_stride, q, rk=3, steps=1, cfl=CFL)
    el = time.perf_counter() - t0
    value = mesh.nvox * args.steps / el
    cfg = workload_config(mesh)
    cfg["time_steps_per_step"] = 1
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one full SSP-RK3 time step of the whole workload per bench step "
                                       f"({mesh.nvox} voxels), OpenMP over patches"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def measure_fp64_peak(torch, dh, stream, sms):
    n = sms * 8 * 256
    iters = 4096
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    best = None
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dh.dh_probe_dfma(out, n, iters, stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return 16.0 * iters * n / (best * 1e-3) / 1e12  # TFLOP/s


def our_arm(args, rank, world, local_rank):
    import torch
    from paper_2608_19273_gb300 import dh
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU: there is no CPU fallback")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    w = synth.workload("euler3d")
    mesh = w.mesh
    prim = synth.euler_prims(mesh, w.seed)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = dh.Plan(synth.PDE_EULER3D, 3, mesh.patches, 1, mesh.var_stride)
        d_prim = torch.from_numpy(prim).to("cuda")
        Q = torch.empty_like(d_prim)
        dh.dh_prim2con(plan, d_prim, Q, stream)
        del d_prim
        U1, U2 = torch.empty_like(Q), torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        Q_init = Q.clone()
        dh.max_wave_speed(plan, Q, None, lam, stream)
        lam_init = lam.clone()
        # eager warm-up step (sets kernel attributes outside of capture), then reset
        dh.dh_rk_step(plan, 0, 3, Q, U1, U2, None, None, dt, lam, CFL, 0.1, stream)
        Q.copy_(Q_init)
        lam.copy_(lam_init)
        stream.synchronize()
        dh.dh_graph_capture(plan, 0, 3, INNER_STEPS, Q, U1, U2, None, None, dt, lam, CFL, 0.1, True, stream)
        n_kernels, n_timed = dh.dh_graph_info(plan)
        peak = measure_fp64_peak(torch, dh, stream, sms)
        for _ in range(args.warmup):
            dh.dh_graph_launch(plan, stream)
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(gpu_id_for_smi(torch, dev))
        sampler.start()
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            dh.dh_graph_launch(plan, stream)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        stage_ms = dh.dh_graph_stage_times(plan, n_timed)
        if dist:
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        finite = bool(torch.isfinite(Q).all().item())

        # end-to-end through the public API with host buffers: H2D of the state,
        # one graph replay (100 time steps), D2H of the result, every step
        h_in = torch.empty(Q.shape, dtype=torch.float64, pin_memory=True)
        h_in.copy_(Q_init)
        h_out = torch.empty_like(h_in, pin_memory=True)
        n_e2e = max(2, args.steps // 2)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_host = time.perf_counter()
        f0.record(stream)
        for _ in range(n_e2e):
            Q.copy_(h_in, non_blocking=True)
            dh.max_wave_speed(plan, Q, None, lam, stream)
            dh.dh_graph_launch(plan, stream)
            h_out.copy_(Q, non_blocking=True)
        f1.record(stream)
        f1.synchronize()
        t_host = time.perf_counter() - t_host
        e2e_ms = f0.elapsed_time(f1)

    nvox = mesh.nvox
    value = world * nvox * INNER_STEPS * args.steps / (ms * 1e-3)
    flops_voxel_step = json.load(open(FLOPS_FILE))["fv/euler3d/ssprk3_step"]["flops_per_voxel"]
    # dominant kernel: the FV stage; average over the 3 x 100 stage launches of the last replay
    ach = flops_voxel_step * nvox * INNER_STEPS / (float(stage_ms.sum()) * 1e-3) / 1e12
    stage_share = float(stage_ms.sum()) / (ms / args.steps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(mesh), parallelism="replicas" if world > 1 else "single-gpu"),
        "roofline": {"bound": "alu", "kernel": "k_fv_stage<Euler3D>", "achieved": ach,
                     "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                     "peak_source": "FP64 FMA peak measured live by dh_probe_dfma on this GPU",
                     "flops_per_voxel_step": flops_voxel_step,
                     "stage_ms_mean": float(stage_ms.mean()), "stage_share_of_step": stage_share,
                     "hbm_bound_frac": None},
        "e2e": {"value": world * nvox * INNER_STEPS * n_e2e / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(Q.numel() * 8), "d2h_bytes_per_step": int(Q.numel() * 8),
                "host_wall_s": t_host},
        "gpu_launches": int(n_kernels * args.steps),
        "clocks": clocks,
        "state_finite": finite,
    }
    # HBM side of the roofline: 320 algorithmic bytes per voxel-step (see DESIGN)
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs") if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6701.5
    line["roofline"]["hbm_bound_frac"] = (320.0 * nvox * INNER_STEPS / (float(stage_ms.sum()) * 1e-3) / 1e9) / hbm
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, steps, el = oracle_rate(mesh, prim, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{steps} full SSP-RK3 time step(s) of the whole workload "
                                          f"({nvox} voxels) in {el:.1f} s, OpenMP over patches"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    rank, world, local_rank = env_rank()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    return our_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
