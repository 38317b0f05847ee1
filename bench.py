#!/usr/bin/env python3
"""Benchmark of the batched explicit patch update on GB300.

Default workload (the headline line): 3D compressible Euler (5 variables,
gamma = 1.4), first-order FV with the Rusanov flux and SSP-RK3 on the AMR-like
patch mix 4096 x 8^3 + 1024 x 16^3 + 128 x 32^3 (10,485,760 voxels, halo 1),
seeded smooth Fourier-mode initial data.  One benchmark step is one replay of
a CUDA graph of 100 time steps; a time step is the device-side CFL time step
(CFL 0.4) plus three batched stage launches (one per SSP-RK3 stage).
Metric: FP64 cell-updates per second (voxels x time steps / s).  The line
also carries the learned-seed vs plain con2prim comparison at 1e-12.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload euler3d|euler2d|wave3d|srhd3d|gw59]

The other workloads (2D Euler forward Euler; wave system FD4+KO RK4; SRHD
FV + con2prim SSP-RK3; 59-unknown GW59 FD4+KO RK4) print the same line for
their own configuration.  --impl reference times the FP64 CPU oracle (the
plain C++ implementation the CUDA path is checked against) on the host
cores: a deliberately slow baseline, not a target.  Under torchrun every rank
runs an independent replica of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
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
FLOPS_FILE = os.path.join(ROOT, "oracle", "flop_counts.json")
# DRAM bytes per voxel and launch of each workload's dominant kernel, read from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum), with the hash of the kernel sources profiled
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")

# name: pde, scheme (0 FV, 1 FD), rk, time steps per graph replay, CFL, flop-count key,
# algorithmic bytes per voxel-step (state reads and writes of all stages, materials,
# RK4 accumulator copies, SRHD primitive reads/writes), description
WORKLOADS = {
    "euler3d": dict(pde=3, scheme=0, rk=3, inner=100, cfl=0.4, flops="fv/euler3d/ssprk3_step", bytes=320,
                    kernel="k_fv_stage<Euler3D>",
                    desc="3D Euler (5 vars, gamma 1.4), FV Rusanov, SSP-RK3; 4096x8^3 + 1024x16^3 + 128x32^3 "
                         "patches, halo 1"),
    "euler3d_muscl": dict(pde=3, scheme=2, rk=3, inner=20, cfl=0.4, flops="fv2/euler3d/ssprk3_step", bytes=320,
                          kernel="k_fv2_stage<Euler3D>",
                          desc="3D Euler, second-order FV (MUSCL-minmod + Rusanov), SSP-RK3; 4096x8^3 + 1024x16^3 + "
                               "128x32^3 patches, halo 2"),
    "euler3d_amr2": dict(pde=3, scheme=0, rk=3, inner=20, cfl=0.4, flops="fv/euler3d/ssprk3_step", bytes=320,
                         kernel="k_fv_stage<Euler3D> + k_reflux + k_restrict",
                         desc="3D Euler on two coupled refinement levels (512 coarse 16^3 patches, dx 1/128, with the "
                              "central 4^3 block refined into 512 patches of 16^3, dx 1/256): FV Rusanov with "
                              "prolongation, reflux and restriction, SSP-RK3; halo 1"),
    "euler3d_p6": dict(pde=3, scheme=0, rk=3, inner=20, cfl=0.4, flops="fv/euler3d/ssprk3_step", bytes=320,
                       kernel="k_fv_any<Euler3D>",
                       desc="3D Euler on the paper's typical 6^3 cells: 32x32x16 patches of 6^3 (16,384 cells of "
                            "216 voxels), FV Rusanov through the generic stage (one patch per CTA), "
                            "SSP-RK3; halo 1"),
    "euler3d_p3": dict(pde=3, scheme=0, rk=3, inner=20, cfl=0.4, flops="fv/euler3d/ssprk3_step", bytes=320,
                       kernel="k_fv_any<Euler3D>",
                       desc="3D Euler on the paper's typical 3^3 cells: 64x64x32 patches of 3^3 (131,072 cells of 27 "
                            "voxels), FV Rusanov through the generic stage (2x2x2 blocks of patches as one 6^3 box "
                            "per CTA), SSP-RK3; halo 1"),
    "euler2d": dict(pde=2, scheme=0, rk=1, inner=10, cfl=0.4, flops="fv/euler2d/fe_step", bytes=128,
                    kernel="k_fv_stage<Euler2D>",
                    desc="2D Euler (4 vars), FV Rusanov, forward Euler; 64 patches of 16^2, halo 1"),
    "wave3d": dict(pde=4, scheme=1, rk=4, inner=10, cfl=0.25, flops="fd/wave3d/rk4_step", bytes=872,
                   kernel="k_fd_stage<Wave>",
                   desc="first-order wave system with c(x) in [0.5, 2], FD4 + KO sigma 0.1, RK4; 2048 patches of "
                        "16^3, halo 3"),
    "srhd3d": dict(pde=5, scheme=0, rk=3, inner=10, cfl=0.4, flops="fv/srhd3d/ssprk3_step", bytes=1040,
                   kernel="k_fv_stage<SRHD> (the timed stage launches; con2prim runs between them)",
                   desc="3D SRHD (Gamma 5/3), FV Rusanov + per-voxel con2prim Newton (tol 1e-12, max 50 "
                        "iterations; seed: the previous pressure refined by 2 FP32 Newton steps), SSP-RK3; "
                        "4096 patches of 16^3, halo 1"),
    "gw59": dict(pde=6, scheme=1, rk=4, inner=5, cfl=0.25, flops="fd/gw59/rk4_step", bytes=9912,
                 kernel="k_fd_stage<GW59>",
                 desc="59-unknown GW stand-in, FD4 + KO sigma 0.1, RK4; 512x24^3 + 1728x16^3 + 4096x16^3 patches "
                      "(3 levels), halo 3"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="euler3d")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-con2prim", action="store_true", help="skip the con2prim seed comparison")
    ap.add_argument("--no-aoas", action="store_true", help="skip the AoAoS gather/scatter measurement")
    ap.add_argument("--no-offload", action="store_true", help="skip the offload-mode measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: skip the per-configuration entries (C1, C3-C5, MUSCL, coupled)")
    ap.add_argument("--config-cpu-seconds", type=float, default=3.0,
                    help="budget of the oracle CPU baseline of each per-configuration entry")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (JSON lines): reuse a previous choice, else time and append")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the patch counts per axis by this factor (small cases for profiling); 1 = full size")
    return ap.parse_args()


# sources of each workload's dominant kernel (besides the shared headers)
_FV = ["dh_fv.cu", "dh_fv_stage.cuh", "dh_tma.cuh"]
KERNEL_SOURCES = {
    "euler3d": _FV + ["dh_fv_euler3.cu", "dh_fv_euler3_tma.cu"], "euler2d": _FV + ["dh_fv_euler2.cu"],
    "euler3d_amr2": _FV + ["dh_fv_euler3.cu", "dh_fv_euler3_tma.cu", "dh_amr.cu"],
    "euler3d_muscl": ["dh_fv2.cu"], "srhd3d": _FV + ["dh_fv_srhd.cu"],
    "euler3d_p6": _FV + ["dh_fv_euler3.cu", "dh_fv_any.cuh"],
    "euler3d_p3": _FV + ["dh_fv_euler3.cu", "dh_fv_any.cuh"],
    "wave3d": ["dh_fd.cu"], "gw59": ["dh_fd.cu"],
}


def _code_only(text):
    """C/C++ source without comments and blank lines (string literals here hold no comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash(name):
    """Hash of the code (comments excluded) of a workload's dominant kernel: its .cu files, the
    shared device headers, the plan code that builds its work lists and the C header; identifies
    the kernel a stored ncu capture describes."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2608_19273_gb300", "csrc")
    # dh_api.cu builds the tile work lists the launches run
    files = [os.path.join(csrc, f) for f in sorted(KERNEL_SOURCES[name] + ["dh_internal.cuh", "dh_pde.cuh", "dh_api.cu"])]
    files.append(os.path.join(ROOT, "include", "dh.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_traffic(name, nvox):
    """DRAM bytes per launch of the workload's dominant kernel from the stored ncu capture, scaled to
    this workload's voxel count; None when no capture exists or that kernel's sources changed since."""
    try:
        with open(TRAFFIC_FILE) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get("workloads", {}).get(name)
    if not e or e.get("source_hash") != kernel_source_hash(name):
        return None
    return float(e["bytes_per_voxel_launch"]) * nvox


def max_over_ranks(value, dist=None, device=None):
    """Largest value over all ranks (the timed region of the slowest rank); identity without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, nvox, time_steps, ms):
    """Cell-updates per second of the whole job: every rank advanced nvox voxels by time_steps in ms."""
    return world * nvox * time_steps / (ms * 1e-3)


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload_config(name, w, mesh, inner=None):
    spec = WORKLOADS[name]
    return {"workload": name, "description": spec["desc"], "voxels": mesh.nvox, "patches": int(mesh.K),
            "time_steps_per_step": spec["inner"] if inner is None else inner, "cfl": spec["cfl"], "cuda_graph": True,
            "time_integrator": {1: "forward Euler", 4: "classical RK4"}.get(
                spec["rk"], "SSP-RK3, stage-sum (Butcher) form: acc holds the raw face-flux sums"
                if spec["scheme"] == 0 else "SSP-RK3, Shu-Osher form"),
            "l2": "no flush: every state array is larger than L2 (129 MB)" if mesh.nvox * 40 > 129e6
            else "state fits in L2 (small workload)",
            "seed": int(w.seed)}


# ------------------------------------------------------------------ inputs
def host_inputs(name, w):
    """(prim or cons on host, material on host or None, kind) of the workload."""
    mesh = w.mesh
    if name in ("euler3d", "euler2d", "euler3d_muscl", "euler3d_p6", "euler3d_p3"):
        return synth.euler_prims(mesh, w.seed), None, "prim"
    if name == "euler3d_amr2":
        return synth.euler_prims_coupled(mesh, w.seed), None, "prim"
    if name == "wave3d":
        q, mat = synth.wave_initial(mesh, w.seed)
        return q, mat, "cons"
    if name == "srhd3d":
        return synth.srhd_initial(mesh, w.seed), None, "prim"
    if name == "gw59":
        return synth.gw59_initial(mesh, w.seed), None, "cons"
    raise KeyError(name)


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
        s = str(torch.cuda.get_device_properties(dev).uuid)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


# ------------------------------------------------------------------ CPU oracle
def oracle_step(name, w, mesh, q, mat, prim):
    """One time step of the oracle on the given mesh (q, prim updated in place)."""
    import oracle
    spec = WORKLOADS[name]
    if name == "srhd3d":
        # con2prim before every stage, warm-started from the previous primitives
        vs = mesh.var_stride
        pr, _, _, _ = oracle.con2prim(q, vs, p_prev=np.ascontiguousarray(prim[4]), refine=SRHD_STEP_REFINE)
        prim[:] = pr
        lam = oracle.max_wave_speed(5, 3, mesh.patches, vs, q, mat=prim, params=w.params)
        dt = oracle.cfl_dt(spec["cfl"], float(mesh.patches["dx"].min()), 3, lam)
        u1, u2 = np.zeros_like(q), np.zeros_like(q)
        for qs, q0, out, a, b, g in ((q, None, u1, 0, 1, 1), (u1, q, u2, 0.75, 0.25, 0.25),
                                     (u2, q, q, 1 / 3, 2 / 3, 2 / 3)):
            if qs is not q:
                pr, _, _, _ = oracle.con2prim(qs, vs, p_prev=np.ascontiguousarray(prim[4]), refine=SRHD_STEP_REFINE)
                prim[:] = pr
            oracle.stage(0, 5, 3, mesh.patches, 1, vs, qs, q0=q0, out=out, mat=prim, dt=dt, a=a, b=b, g=g,
                         params=w.params)
        return
    oracle.rk_steps(spec["scheme"], spec["pde"], mesh.dim, mesh.patches, w.halo, mesh.var_stride, q, mat=mat,
                    rk=spec["rk"], steps=1, cfl=spec["cfl"], sigma=0.1, params=w.params)


# The oracle's CPU samples run each workload with its box scaled down by this factor per axis
# (same patch sizes) where the whole workload would take too long on the host cores.
ORACLE_SCALE = {"euler3d": 1, "euler3d_muscl": 2, "euler3d_amr2": 1, "euler2d": 1, "wave3d": 2, "srhd3d": 2,
                "gw59": 4, "euler3d_p6": 1, "euler3d_p3": 1}


def oracle_sample(name, budget_s):
    """The oracle on a bounded sample of the workload: the full mesh when it is small enough,
    else the same patch sizes with fewer patches per level (scaled box)."""
    import oracle
    cores = oracle.num_threads(0)
    scale = ORACLE_SCALE[name]
    w = synth.workload(name, scale=scale)
    mesh = w.mesh
    h, mat, kind = host_inputs(name, w)
    prim = None
    if name == "srhd3d":
        prim = h.copy()
        q = oracle.prim2con(5, h, mesh.var_stride, params=w.params)
    elif kind == "prim":
        q = oracle.prim2con(WORKLOADS[name]["pde"], h, mesh.var_stride, params=w.params)
    else:
        q = h
    steps, t0 = 0, time.perf_counter()
    while True:
        oracle_step(name, w, mesh, q, mat, prim)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el / steps * (steps + 1) > 2.5 * budget_s:
            break
    sample = (f"{steps} full time step(s) of the {'whole' if scale == 1 else f'1/{scale**3} (box scaled 1/{scale} per axis)'} "
              f"workload ({mesh.nvox} voxels) in {el:.1f} s, OpenMP over patches{oracle_form(w)}")
    return mesh.nvox * steps / el, cores, sample, el / steps


def oracle_form(w):
    """How the oracle evaluates the time step, where that differs from the GPU arm's evaluation."""
    return "; SSP-RK3 in the Shu-Osher form (the same scheme)" if w.rk == 3 and w.scheme == synth.SCHEME_FV else ""


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    name = args.workload
    import oracle
    # under torchrun every rank starts with one OpenMP thread; rank 0 runs alone here, so it takes
    # the host's cores
    cores = oracle.num_threads(len(os.sched_getaffinity(0)) if world > 1 else 0)
    scale = ORACLE_SCALE[name]
    w = synth.workload(name, scale=scale)
    mesh = w.mesh
    h, mat, kind = host_inputs(name, w)
    prim = h.copy() if name == "srhd3d" else None
    q = oracle.prim2con(WORKLOADS[name]["pde"], h, mesh.var_stride, params=w.params) if kind == "prim" else h
    for _ in range(args.warmup):
        oracle_step(name, w, mesh, q, mat, prim)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(name, w, mesh, q, mat, prim)
    el = time.perf_counter() - t0
    value = mesh.nvox * args.steps / el
    cfg = workload_config(name, w, mesh)
    cfg["time_steps_per_step"] = 1
    sample = (f"one full time step per bench step of the {'whole' if scale == 1 else f'1/{scale**3}'} workload "
              f"({mesh.nvox} voxels), OpenMP over patches{oracle_form(w)}")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
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


def train_seed(torch, dh, stream, n=1 << 20, steps=6000, seed=synth.SEED_BASE + 3):
    """Train the con2prim seed MLP on n (conserved, pressure) pairs with the library's kernels.
    The pairs come from the library's prim2con kernel on i.i.d. primitives (the tests pin that
    kernel, and the training itself, to the oracle's prim2con)."""
    mesh = synth.make_mesh([synth.Level((8, 8, 4), 16, 1.0 / 256, 0)], dim=3)
    prim = synth.srhd_iid_prims(mesh.var_stride, seed)
    plan = dh.Plan(5, 3, mesh.patches, 1, mesh.var_stride)
    d_prim = torch.from_numpy(prim).to("cuda")
    cons = torch.empty_like(d_prim)
    dh.dh_prim2con(plan, d_prim, cons, stream)
    n = mesh.var_stride
    x = torch.empty(n * 3, dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    dh.dh_mlp_features(cons, d_prim[4], n, n, x, y, stream)
    rng = np.random.default_rng(seed)
    w = np.zeros(1224, dtype=np.float32)
    for off, fi, fo in ((0, 3, 32), (128, 32, 32), (1184, 32, 1)):
        lim = math.sqrt(6.0 / (fi + fo))
        w[off:off + fi * fo] = rng.uniform(-lim, lim, fi * fo)
    d_w = torch.from_numpy(w).to("cuda")
    scratch = torch.zeros(6 * 1024, dtype=torch.float64, device="cuda")
    dh.dh_mlp_standardize(x, n, d_w, scratch, stream)
    m, v = torch.zeros(1224, device="cuda"), torch.zeros(1224, device="cuda")
    B = 4096
    part = torch.zeros((B // 64) * 1224, device="cuda")
    grad = torch.zeros(1224, device="cuda")
    loss = torch.zeros(steps, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dh.dh_mlp_train(d_w, m, v, x, y, n, B, steps, 0, 1e-3, part, grad, loss, stream)
    e1.record(stream)
    e1.synchronize()
    plan.close()
    lh = loss.cpu().numpy()
    return d_w, {"samples": n, "steps": steps, "batch": B, "train_ms": e0.elapsed_time(e1),
                 "loss_first": float(lh[:20].mean()), "loss_last": float(lh[-100:].mean())}


# FP32 Newton steps that refine the learned seed before the FP64 iteration
C2P_REFINE = 3
# FP32 Newton steps that refine the previous pressure, the seed of every con2prim of the SRHD
# workload's time steps (the oracle's steps refine it the same way)
SRHD_STEP_REFINE = 3


def con2prim_compare(torch, dh, stream):
    """Plain vs MLP-seeded Newton at tol 1e-12: cold (i.i.d. states, no previous pressure)
    and warm (the first SSP-RK3 stage of the SRHD workload, seeded by the previous pressure)."""
    d_w, train = train_seed(torch, dh, stream)
    res = {"tol": 1e-12, "max_iter": 50, "training": train}
    w = synth.workload("srhd3d")
    mesh = w.mesh
    n = mesh.var_stride
    plan = dh.Plan(5, 3, mesh.patches, 1, mesh.var_stride, w.params)

    def run(cons, p_prev, mlp, refine=0):
        prim = torch.empty_like(cons)
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        fails = torch.zeros(1, dtype=torch.int32, device="cuda")
        dh.con2prim(plan, cons, prim, p_prev, mlp, 1e-12, 50, None, it, fails, stream, seed_refine=refine)  # warm-up
        fails.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = 5
        for _ in range(reps):
            dh.con2prim(plan, cons, prim, p_prev, mlp, 1e-12, 50, None, it, fails, stream, seed_refine=refine)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        hist = torch.bincount(it.long().clamp(0, 101)).cpu().tolist()
        return prim, {"ns_per_voxel": ms * 1e6 / mesh.nvox, "iters_mean": float(it.double().mean().item()),
                      "iters_hist": [[k, c] for k, c in enumerate(hist) if c], "fails": int(fails.item()) // reps}

    with torch.cuda.stream(stream):
        # cold: i.i.d. primitives (rho, p log-uniform on [0.1, 10], W uniform on [1, 10])
        prim_iid = torch.from_numpy(synth.srhd_iid_prims(n, synth.SEED_BASE + 13)).to("cuda")
        cons = torch.empty_like(prim_iid)
        dh.dh_prim2con(plan, prim_iid, cons, stream)
        _, plain = run(cons, None, None)
        _, mlp = run(cons, None, d_w)
        _, mlp_r = run(cons, None, d_w, C2P_REFINE)
        _, plain_r = run(cons, None, None, C2P_REFINE)
        res["cold_iid"] = {"voxels": mesh.nvox, "plain": plain, "mlp": mlp_r, "mlp_unrefined": mlp,
                           "ablation_plain_refined": plain_r,
                           "speedup": plain["ns_per_voxel"] / mlp_r["ns_per_voxel"]}
        del prim_iid
        # warm: smooth workload state after one FV stage; seed = previous pressure
        prim0 = torch.from_numpy(synth.srhd_initial(mesh, w.seed)).to("cuda")
        q0 = torch.empty_like(prim0)
        dh.dh_prim2con(plan, prim0, q0, stream)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, q0, prim0, lam, stream)
        dh.dh_cfl_dt(plan, lam, 0.4, dt, stream)
        u1 = torch.empty_like(q0)
        dh.patch_update_fv(plan, q0, None, u1, None, prim0, dt, 0, 1, 1, 0, None, stream)
        p_prev = prim0[4].contiguous()
        _, plain = run(u1, p_prev, None)
        _, mlp = run(u1, p_prev, d_w)
        _, mlp_r = run(u1, p_prev, d_w, C2P_REFINE)
        abl = {f"refine_{k}": run(u1, p_prev, None, k)[1] for k in (1, 2, 3)}
        res["warm_stage"] = {"voxels": mesh.nvox, "plain": plain, "mlp": mlp_r, "mlp_unrefined": mlp,
                             "ablation_plain_refined": abl,
                             "speedup": plain["ns_per_voxel"] / mlp_r["ns_per_voxel"]}
    plan.close()
    res["winner_cold"] = "mlp" if res["cold_iid"]["speedup"] > 1 else "plain"
    res["winner_warm"] = "mlp" if res["warm_stage"]["speedup"] > 1 else "plain"
    res["mlp_seed"] = (f"network seed refined by {C2P_REFINE} FP32 Newton steps, then FP64 Newton; plain = FP64 "
                       "Newton from the previous pressure (cold: from the cold seed), unrefined; the ablation rows "
                       "refine the plain seed the same way")
    return res


def measure_aoas(torch, dh, plan, mesh, nq, halo, stream, reps=5):
    """Gather prologue / scatter epilogue (AoAoS <-> SoA arena) throughput on the workload's patches:
    nq quantities per voxel, blocks of (p + 2 halo)^3 voxels as shuffled views of one buffer."""
    lens = [(int(pt["p"]) + 2 * halo) ** mesh.dim * nq for pt in mesh.patches]
    order = np.random.default_rng(synth.SEED_BASE).permutation(len(lens))
    starts = np.zeros(len(lens), dtype=np.int64)
    pos = 0
    for k in order:
        starts[k] = pos
        pos += lens[k] + 1
    buf = torch.empty(pos, dtype=torch.float64, device="cuda")
    buf.normal_()
    ptrs = torch.tensor([buf.data_ptr() + 8 * int(starts[k]) for k in range(len(lens))], dtype=torch.int64,
                        device="cuda")
    arena = torch.empty(nq * mesh.var_stride, dtype=torch.float64, device="cuda")
    out = {}
    for what in ("gather", "scatter"):
        call = ((lambda: dh.dh_gather_aoas(plan, ptrs, nq, halo, arena, stream)) if what == "gather" else
                (lambda: dh.dh_scatter_aoas(plan, arena, ptrs, nq, halo, stream)))
        for _ in range(3):
            call()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            call()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[what + "_ms"] = ms
        out[what + "_gbs"] = 16.0 * nq * mesh.nvox / (ms * 1e-3) / 1e9
    del buf, arena, ptrs
    torch.cuda.empty_cache()
    out.update(nq=nq, aos_halo=halo, bytes_per_call=16 * nq * mesh.nvox,
               note="algorithmic bytes: one read and one write of every interior element; "
                    "every buffer is larger than L2")
    return out


def measure_offload(torch, dh, plan, mesh, spec, w, arena_init, U1, U2, ACC, stream, inner, compute_ms_per_step):
    """Offload mode: the state lives in host page-locked AoAoS blocks (one per patch, halo included, shuffled
    in one buffer); each call gathers it over NVLink-C2C, advances n steps on the GPU and scatters it back."""
    nq, h = plan.nq + plan.nm, w.halo
    lens = [(int(pt["p"]) + 2 * h) ** mesh.dim * nq for pt in mesh.patches]
    order = np.random.default_rng(synth.SEED_BASE + 7).permutation(len(lens))
    starts = np.zeros(len(lens), dtype=np.int64)
    pos = 0
    for k in order:
        starts[k] = pos
        pos += lens[k] + 1
    hbuf = torch.zeros(pos, dtype=torch.float64).pin_memory()
    addrs = [hbuf.data_ptr() + 8 * int(starts[k]) for k in range(len(lens))]
    table = torch.tensor(addrs, dtype=torch.int64, device="cuda")
    arena = arena_init.clone()
    dh.dh_scatter_aoas(plan, arena, table, nq, h, stream)       # initial state into the host blocks
    dh.dh_offload_bind(plan, addrs, nq, h)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros(1, dtype=torch.float64, device="cuda")
    nq_back = nq if spec["pde"] == synth.PDE_SRHD3D else plan.nq
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps):
        fn()
        stream.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    g_ms = timed(lambda: dh.dh_gather_aoas(plan, table, nq, h, arena, stream), 3)
    s_ms = timed(lambda: dh.dh_scatter_aoas(plan, arena, table, nq_back, h, stream), 3)
    run = lambda n: dh.dh_offload_run(plan, spec["scheme"], spec["rk"], n, arena, U1, U2, ACC, dt, lam, spec["cfl"],
                                      0.1, nq_back, stream)
    one_ms = timed(lambda: run(1), 3)
    many_ms = timed(lambda: run(inner), 1)
    small = 8.0 * nq * mesh.nvox <= 4e9
    two = two_st = None
    if small:
        two = measure_two_offload_problems(torch, dh, plan, mesh, spec, w, arena_init, U1, U2, ACC, stream, starts, pos,
                                           nq, h, nq_back, run, timed, compute_ms_per_step, False)
    # staged: the blocks' host span moved by the copy engine (one cudaMemcpyAsync each way)
    dh.dh_offload_bind_staged(plan, addrs, nq, h)
    one_st = timed(lambda: run(1), 3)
    many_st = timed(lambda: run(inner), 1)
    if small:
        two_st = measure_two_offload_problems(torch, dh, plan, mesh, spec, w, arena_init, U1, U2, ACC, stream, starts,
                                              pos, nq, h, nq_back, run, timed, compute_ms_per_step, True)
    finite = bool(torch.isfinite(hbuf).all().item())
    del hbuf, table, arena
    torch.cuda.empty_cache()
    nvox = mesh.nvox
    return {"two_problems_two_streams": two,
            "staged": {"total_ms_1_step": one_st, "total_ms_%d_steps" % inner: many_st,
                       "total_over_compute_1_step": one_st / compute_ms_per_step,
                       "total_over_compute_%d_steps" % inner: many_st / (inner * compute_ms_per_step),
                       "two_problems_two_streams": two_st},"nq": nq, "nq_back": nq_back, "aos_halo": h, "blocks": "page-locked host memory, one block per patch",
            "gather_ms": g_ms, "scatter_ms": s_ms,
            "c2c_read_gbs": 8.0 * nq * nvox / (g_ms * 1e-3) / 1e9,
            "c2c_write_gbs": 8.0 * nq_back * nvox / (s_ms * 1e-3) / 1e9,
            "total_ms_1_step": one_ms, "total_ms_%d_steps" % inner: many_ms,
            "compute_ms_per_step": compute_ms_per_step,
            "total_over_compute_1_step": one_ms / compute_ms_per_step,
            "total_over_compute_%d_steps" % inner: many_ms / (inner * compute_ms_per_step),
            "host_blocks_finite": finite}


def measure_two_offload_problems(torch, dh, plan, mesh, spec, w, arena_init, U1, U2, ACC, stream, starts, pos, nq, h,
                                 nq_back, run_a, timed, compute_ms_per_step, staged):
    """A second, independent problem (own plan, host blocks and device buffers), one time step per call:
    the two calls on one stream one after the other, then on two streams at once, so that each
    problem's host transfers can overlap the other's compute."""
    plan_b = dh.Plan(spec["pde"], mesh.dim, mesh.patches, w.halo, mesh.var_stride, w.params)
    hbuf_b = torch.zeros(pos, dtype=torch.float64).pin_memory()
    addrs_b = [hbuf_b.data_ptr() + 8 * int(starts[k]) for k in range(len(starts))]
    table_b = torch.tensor(addrs_b, dtype=torch.int64, device="cuda")
    arena_b = arena_init.clone()
    dh.dh_scatter_aoas(plan_b, arena_b, table_b, nq, h, stream)
    (dh.dh_offload_bind_staged if staged else dh.dh_offload_bind)(plan_b, addrs_b, nq, h)
    like = lambda t: torch.empty_like(t) if t is not None else None
    u1b, u2b, accb = like(U1), like(U2), like(ACC)
    dt_b = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam_b = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream_b = torch.cuda.Stream()
    run_b = lambda s: dh.dh_offload_run(plan_b, spec["scheme"], spec["rk"], 1, arena_b, u1b, u2b, accb, dt_b, lam_b,
                                        spec["cfl"], 0.1, nq_back, s)
    seq_ms = timed(lambda: (run_a(1), run_b(stream)), 3)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def both():
        fork.record(stream)
        stream_b.wait_event(fork)
        run_a(1)
        run_b(stream_b)
        join.record(stream_b)
        stream.wait_event(join)
    par_ms = timed(both, 3)
    stream.synchronize()
    stream_b.synchronize()
    plan_b.close()
    del hbuf_b, table_b, arena_b, u1b, u2b, accb
    return {"sequential_ms": seq_ms, "concurrent_ms": par_ms, "overlap_gain": seq_ms / par_ms,
            "total_over_compute_1_step_concurrent": par_ms / (2 * compute_ms_per_step)}


# Settings of the per-configuration entries of the default line (`configs`): time steps per
# graph replay, warm-up and timed replays (every state array is larger than L2 except C1's).
CONFIGS = {
    "euler2d": dict(label="C1", inner=10, warmup=3, steps=20),
    "wave3d": dict(label="C3", inner=10, warmup=3, steps=3),
    "srhd3d": dict(label="C4", inner=10, warmup=3, steps=3),
    "gw59": dict(label="C5", inner=1, warmup=3, steps=3),
    "euler3d_muscl": dict(label="C2, second order (MUSCL-minmod)", inner=10, warmup=3, steps=3),
    "euler3d_amr2": dict(label="C2-like, two coupled refinement levels", inner=20, warmup=3, steps=3),
    "euler3d_p6": dict(label="the paper's typical 6^3 cells (generic FV stage)", inner=20, warmup=3, steps=3),
    "euler3d_p3": dict(label="the paper's typical 3^3 cells (generic FV stage, 2x2x2 blocks of patches)", inner=20,
                       warmup=3, steps=3),
}


def flop_table():
    with open(FLOPS_FILE) as fh:
        return json.load(fh)


def hbm_peak():
    hbm, src = 6800.0, "fallback"
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        with open(mp) as fh:
            hbm, src = float(json.load(fh).get("hbm_gbs", hbm)), "measured"
    return hbm, src


def offload_blocks(torch, mesh, nq, halo, seed):
    """Page-locked host AoAoS blocks (one per patch, halo included, back to back in a shuffled
    order in one buffer): (host buffer, block addresses, device pointer table).  The buffer is
    zeroed only where the blocks have halo entries (nothing else leaves entries unwritten)."""
    lens = [(int(pt["p"]) + 2 * halo) ** mesh.dim * nq for pt in mesh.patches]
    order = np.random.default_rng(seed).permutation(len(lens))
    starts = np.zeros(len(lens), dtype=np.int64)
    pos = 0
    for k in order:
        starts[k] = pos
        pos += lens[k]
    hbuf = torch.empty(pos, dtype=torch.float64, pin_memory=True)
    if halo > 0:
        hbuf.zero_()
    addrs = [hbuf.data_ptr() + 8 * int(starts[k]) for k in range(len(lens))]
    table = torch.tensor(addrs, dtype=torch.int64, device="cuda")
    return hbuf, addrs, table


def measure_e2e(torch, dh, plan, mesh, spec, w, arena_init, U1, U2, ACC, stream, inner, calls):
    """End to end through the library's host-buffer entry point: the state lives in page-locked
    host AoAoS blocks (the paper's layout, Sec. II-B); every call of dh_offload_run gathers all
    quantities from them over NVLink-C2C, advances `inner` time steps on the GPU and scatters
    the evolved quantities back into them (paper Sec. III-C/D).  GW59 uses blocks without halo
    (aos_halo 0) so that its page-locked copy stays at 14.6 GB."""
    nq = plan.nq + plan.nm
    halo = 0 if spec["pde"] == synth.PDE_GW59 else w.halo
    hbuf, addrs, table = offload_blocks(torch, mesh, nq, halo, synth.SEED_BASE + 17)
    arena = arena_init.clone()
    dh.dh_scatter_aoas(plan, arena, table, nq, halo, stream)  # the initial state into the host blocks
    dh.dh_offload_bind(plan, addrs, nq, halo)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros(1, dtype=torch.float64, device="cuda")
    nq_back = nq if spec["pde"] == synth.PDE_SRHD3D else plan.nq
    run = lambda: dh.dh_offload_run(plan, spec["scheme"], spec["rk"], inner, arena, U1, U2, ACC, dt, lam,
                                    spec["cfl"], 0.1, nq_back, stream)
    run()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(calls):
        run()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    finite = bool(torch.isfinite(hbuf).all().item())
    del hbuf, table, arena
    return {"value": mesh.nvox * inner * calls / (ms * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": int(8 * nq * mesh.nvox), "d2h_bytes_per_step": int(8 * nq_back * mesh.nvox),
            "api": f"dh_offload_run: gather from page-locked host AoAoS blocks (aos_halo {halo}) over NVLink-C2C, "
                   f"{inner} time steps, scatter back, per call",
            "calls": calls, "time_steps_per_call": inner, "ms_per_call": ms / calls, "host_blocks_finite": finite}


def run_workload(torch, dh, name, args, stream, world, dist, peak, warmup, steps, inner, e2e_calls, headline):
    """Build, autotune, capture and time one workload (a graph of `inner` time steps, `warmup`
    untimed and `steps` timed replays); roofline of its dominant kernel, end-to-end rate through
    the host-buffer entry point.  Returns (line fields, objects kept for the headline's extras)."""
    spec = WORKLOADS[name]
    w = synth.workload(name, scale=args.scale)
    mesh = w.mesh
    h, h_mat, kind = host_inputs(name, w)
    srhd = name == "srhd3d"
    dev = torch.cuda.current_device()
    with torch.cuda.stream(stream):
        plan = dh.Plan(spec["pde"], mesh.dim, mesh.patches, w.halo, mesh.var_stride, w.params)
        if srhd:
            dh.dh_plan_set_con2prim(plan, None, 1e-12, 50, None, seed_refine=SRHD_STEP_REFINE)
        d_h = torch.from_numpy(h).to("cuda")
        del h
        if kind == "prim":
            Q = torch.empty_like(d_h)
            dh.dh_prim2con(plan, d_h, Q, stream)
        else:
            Q = d_h
        mat = d_h if srhd else (torch.from_numpy(h_mat).to("cuda") if h_mat is not None else None)
        if not srhd and kind == "prim":
            del d_h
        U1 = torch.empty_like(Q)
        U2 = torch.empty_like(Q) if spec["rk"] >= 3 else None
        # RK4 accumulator; for SSP-RK3 FV steps the raw face-flux sums of the stage-sum form
        ACC = torch.empty_like(Q) if spec["rk"] == 4 or (spec["rk"] == 3 and spec["scheme"] == 0) else None
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        Q_init = Q.clone()
        M_init = mat.clone() if mat is not None else None
        dh.max_wave_speed(plan, Q, mat, lam, stream)
        lam_init = lam.clone()
        dh.dh_cfl_dt(plan, lam, spec["cfl"], dt, stream)
        if spec["scheme"] == 0 and spec["pde"] in (synth.PDE_EULER2D, synth.PDE_EULER3D):
            # FV, Euler: tune whole time steps as the graph runs them (stage-sum form, derived
            # quantities handed between stages), on scratch copies of the state
            Qt = Q.clone()
            Mt = mat.clone() if mat is not None else None
            lam_t = lam.clone()
            # (two steps per call: the hand-over of derived quantities starts with the second stage)
            tv, tz, tf, cached, ttimes = dh.dh_autotune_steps(plan, spec["scheme"], spec["rk"], 2, Qt, U1, U2, ACC, Mt,
                                                              dt, lam_t,
                                                              spec["cfl"], 0.1, reps=2, cache_path=args.tune_cache,
                                                              stream=stream)
            del Qt, Mt, lam_t
            tune = ({"fv2_var": tv} if spec["scheme"] == 2 else {"fv_var": tv, "fv_zs": tz, "fd_var": tf})
            tune.update({"from_cache": cached, "timed": "two time steps per call",
                         "candidate_ms": [round(t, 4) for t in ttimes if t > 0]})
        else:
            # the other stages hand nothing from stage to stage: one stage per call, on the same state
            # for every candidate (for SRHD the steps' con2prim work would vary from candidate to
            # candidate as the state advanced)
            tv, tz, tf, cached, ttimes = dh.dh_autotune(plan, spec["scheme"], Q, U1, mat, dt, reps=3,
                                                        cache_path=args.tune_cache, stream=stream)
            tune = ({"fv2_var": tv} if spec["scheme"] == 2 else {"fv_var": tv, "fv_zs": tz, "fd_var": tf})
            tune.update({"from_cache": cached, "timed": "one stage per call",
                         "candidate_ms": [round(t, 4) for t in ttimes if t > 0]})
        # eager warm-up step (sets kernel attributes outside of capture), then reset
        dh.dh_rk_step(plan, spec["scheme"], spec["rk"], Q, U1, U2, ACC, mat, dt, lam, spec["cfl"], 0.1, stream)
        Q.copy_(Q_init)
        lam.copy_(lam_init)
        if mat is not None:
            mat.copy_(M_init)
        stream.synchronize()
        # per-stage device times (the roofline's kernel time) from a graph with event records
        # around every stage launch, replayed once after a warm-up replay; the bench value from
        # the same graph captured without them (on short steps the event nodes cost time)
        dh.dh_graph_capture(plan, spec["scheme"], spec["rk"], inner, Q, U1, U2, ACC, mat, dt, lam, spec["cfl"], 0.1,
                            True, stream)
        n_kernels, n_timed = dh.dh_graph_info(plan)
        for _ in range(2):
            dh.dh_graph_launch(plan, stream)
        stream.synchronize()
        stage_ms = dh.dh_graph_stage_times(plan, n_timed)
        Q.copy_(Q_init)
        lam.copy_(lam_init)
        if mat is not None:
            mat.copy_(M_init)
        stream.synchronize()
        dh.dh_graph_capture(plan, spec["scheme"], spec["rk"], inner, Q, U1, U2, ACC, mat, dt, lam, spec["cfl"], 0.1,
                            False, stream)
        for _ in range(warmup):
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
        for _ in range(steps):
            dh.dh_graph_launch(plan, stream)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        if dist:
            ms = max_over_ranks(ms, dist, device="cuda")
            dist.barrier()
        finite = bool(torch.isfinite(Q).all().item())
        it_mean = None
        if srhd:
            # Newton iterations of a recovery as the step runs it (the evolved state, seeded by
            # the pressure of the previous stage input), for the whole-step operation count
            its = torch.empty(mesh.var_stride, dtype=torch.int32, device="cuda")
            its.zero_()
            dh.con2prim(plan, Q, U1, mat[4], None, 1e-12, 50, None, its, None, stream, seed_refine=SRHD_STEP_REFINE)
            stream.synchronize()
            it_mean = float(its.double().sum().item()) / mesh.nvox
        a0 = Q_init if M_init is None else torch.cat([Q_init, M_init])
        e2e = measure_e2e(torch, dh, plan, mesh, spec, w, a0.contiguous(), U1, U2, ACC, stream, inner, e2e_calls)

    nvox = mesh.nvox
    table = flop_table()
    flops_vs = table[spec["flops"]]["flops_per_voxel"]
    stage_sum_s = float(stage_ms.sum()) * 1e-3
    # The event records around every stage launch cost time of their own (about 4 us per launch):
    # where the per-stage times add up to more than the replay without them, the replay's time per
    # stage launch (which still includes the gaps between launches and the steps' CFL kernels,
    # where there are any) is the smaller, and closer, bound on the stage kernel's duration.
    step_s = ms * 1e-3 / steps
    duration_source = "per-stage CUDA events in a graph replay"
    if stage_sum_s > step_s:
        stage_sum_s = step_s
        duration_source = ("CUDA events around the timed replays / stage launches (the replay holds only the "
                           "stage launches and the steps' CFL kernels; per-stage event records would add their own time)")
    ach = flops_vs * nvox * inner / stage_sum_s / 1e12
    hbm, hbm_src = hbm_peak()
    roof = {"bound": "alu", "kernel": spec["kernel"], "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": measured_traffic(name, nvox),
            "peak_source": "FP64 FMA peak measured live on this GPU (dh_probe_dfma, 2 FLOP per FMA)",
            "flops_per_voxel_step": flops_vs, "timed_launches": int(n_timed),
            "stage_ms_mean": float(stage_ms.mean()),
            "stage_share_of_step": float(stage_ms.sum()) / (ms / steps),
            "duration_source": duration_source,
            "hbm": {"bytes_per_voxel_step": spec["bytes"], "peak_gbs": hbm, "peak_source": hbm_src,
                    "achieved_gbs": spec["bytes"] * nvox * inner / stage_sum_s / 1e9,
                    "frac": spec["bytes"] * nvox * inner / stage_sum_s / 1e9 / hbm}}
    out = {"value": whole_job_rate(world, nvox, inner * steps, ms), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "warmup": warmup, "config": workload_config(name, w, mesh, inner),
           "roofline": roof, "e2e": e2e, "gpu_launches": int(n_kernels * steps), "autotune": tune,
           "clocks": clocks, "state_finite": finite}
    if srhd:
        # the whole SSP-RK3 step: three recoveries (the step start's and those of stages 2 and
        # 3), the step start's wave speed and the three FV stages, all in the timed graph
        c2p = table["c2p/srhd3d/voxel"]["flops_per_voxel"] + it_mean * table["c2p/srhd3d/newton_iteration"][
            "flops_per_voxel"]
        # the wave speed kernel evaluates one direction (that of the largest |v_d|, whose speed is the
        # largest), so its count is the derived quantities and one speed, not the three-direction 68
        wave = table["speed/srhd3d/voxel_one_direction"]["flops_per_voxel"]
        whole = flops_vs + 3 * c2p + wave
        step_s = ms * 1e-3 / (steps * inner)
        ach_w = whole * nvox / step_s / 1e12
        out["roofline_stage"] = roof
        out["roofline"] = {"bound": "alu", "kernel": "whole SSP-RK3 step: con2prim (k_con2prim_patches) x 3, "
                                                      "wave speed, CFL dt, k_fv_stage<SRHD> x 3",
                           "achieved": ach_w, "peak": peak, "unit": "TFLOP/s", "frac": ach_w / peak,
                           "traffic": None, "peak_source": roof["peak_source"],
                           "flops_per_voxel_step": whole,
                           "flops_breakdown": {"fv_stages": flops_vs, "con2prim_per_call": c2p,
                                               "con2prim_calls": 3, "newton_iterations_mean": it_mean,
                                               "wave_speed": wave},
                           "hbm": {"bytes_per_voxel_step": spec["bytes"], "peak_gbs": hbm,
                                   "achieved_gbs": spec["bytes"] * nvox / step_s / 1e9,
                                   "frac": spec["bytes"] * nvox / step_s / 1e9 / hbm}}
    keep = None
    if headline:
        keep = dict(plan=plan, mesh=mesh, spec=spec, w=w, Q_init=Q_init, M_init=M_init, U1=U1, U2=U2, ACC=ACC)
    else:
        plan.close()
    del Q, U1, U2, ACC, mat
    return out, keep


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
    name = args.workload
    spec = WORKLOADS[name]
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.Stream()
    peak = measure_fp64_peak(torch, dh, stream, sms)
    inner = spec["inner"]
    main_, keep = run_workload(torch, dh, name, args, stream, world, dist, peak, args.warmup, args.steps, inner,
                               max(3, args.steps // 4), headline=True)
    plan, mesh, w = keep["plan"], keep["mesh"], keep["w"]
    offload = None
    if rank == 0 and not args.no_offload and spec["pde"] != synth.PDE_GW59:
        with torch.cuda.stream(stream):
            Q_init, M_init = keep["Q_init"], keep["M_init"]
            a0 = Q_init if M_init is None else torch.cat([Q_init, M_init])
            offload = measure_offload(torch, dh, plan, mesh, spec, w, a0.contiguous(), keep["U1"], keep["U2"],
                                      keep["ACC"], stream, inner, main_["ms_per_step"] / inner)
    keep.clear()
    torch.cuda.empty_cache()
    hbm, _ = hbm_peak()
    line = {
        "metric": METRIC, "value": main_["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(main_["config"], parallelism="replicas" if world > 1 else "single-gpu", scale=args.scale),
        "roofline": main_["roofline"], "e2e": main_["e2e"], "gpu_launches": main_["gpu_launches"],
        "autotune": main_["autotune"], "offload": offload, "clocks": main_["clocks"],
        "state_finite": main_["state_finite"],
    }
    if "roofline_stage" in main_:
        line["roofline_stage"] = main_["roofline_stage"]
    if rank == 0 and not args.no_aoas:
        ao = measure_aoas(torch, dh, plan, mesh, plan.nq + plan.nm, w.halo, stream)
        ao["gather_frac"] = ao["gather_gbs"] / hbm
        ao["scatter_frac"] = ao["scatter_gbs"] / hbm
        line["aoas"] = ao
    plan.close()
    torch.cuda.empty_cache()
    if rank == 0 and name in ("euler3d", "srhd3d") and not args.no_con2prim:
        line["con2prim"] = con2prim_compare(torch, dh, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample, _ = oracle_sample(name, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    # every other configuration: same measurement with fewer replays, each with its own oracle sample
    if name == "euler3d" and not args.no_configs:
        configs = {}
        for cname, cs in CONFIGS.items():
            out, _ = run_workload(torch, dh, cname, args, stream, world, dist, peak, cs["warmup"], cs["steps"],
                                  cs["inner"], 2, headline=False)
            torch.cuda.empty_cache()
            out["config"]["label"] = cs["label"]
            if rank == 0 and world == 1 and not args.no_cpu_baseline:
                rate, cores, sample, _ = oracle_sample(cname, args.config_cpu_seconds)
                out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": sample}
            configs[cname] = out
        line["configs"] = configs
        line["gpu_launches_configs"] = int(sum(c["gpu_launches"] for c in configs.values()))
    if rank == 0:
        print(json.dumps(line), flush=True)
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
