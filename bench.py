#!/usr/bin/env python
"""Benchmark: MACE iterations/s on a 4D volume on one GB300 (learned multi-slice
fusion vs the plain q-GGMRF prior), plus projector throughput.

One step = one Mann iteration of Algorithm 1 (all agents + consensus) of the
full multi-slice-fusion workload: 384^3 voxels x 16 time-points, 512x384
detector, 24 views per time-point interlaced over 360 deg, seeded moving
ellipsoid phantom, Poisson noise at 1e4 photons.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl msf|reference]
For N > 1 launch with torch.distributed.run: every rank reconstructs its own
independent problem (different seed), so the work per GPU is fixed (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

I0 = 1e4
METRIC = "MACE iters/s on 4D volume, learned vs plain prior, 1 GB300; projector GB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="msf", choices=["msf", "reference"])
    ap.add_argument("--workload", default="full", choices=["full", "proj", "tiny"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(name):
    from paper_2008_01567_gb300 import synth
    return {"full": synth.FULL, "proj": synth.PROJ, "tiny": synth.TINY}[name]


# settings of the plain and learned runs (rho, sigma and agent weights of Eq. (9))
PLAIN = dict(rho=0.8, sigma=0.1, mu=[0.25, 0.75], n_cg=5, n_sweeps=2, sx=0.1, T=1.0, bt=0.5, q=1.2)
LEARNED = dict(rho=0.8, sigma=0.1, mu=[0.25, 0.25, 0.25, 0.25], n_cg=5)


# ---------------------------------------------------------------- clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- problem set-up

def make_problem(scan, seed, n_ell=6):
    """Phantom, photon counts and (y, Lambda) on the device.  The phantom and its
    exact line integrals come from the library's phantom kernels; the Poisson
    draw uses the seeded generator of synth."""
    import torch
    from paper_2008_01567_gb300 import msf, synth
    P = msf.Projector(scan)
    ell = synth.ellipsoids(seed, n_ell, scan)
    x_true = torch.empty((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    msf.msf_phantom_voxelize(P.vol, ell, x_true, ss=2)
    p = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    msf.msf_phantom_project(P, ell, p)
    mean = I0 * np.exp(-p.cpu().numpy().astype(np.float64))
    counts_h = torch.from_numpy(synth.poisson(seed + 1, mean).astype(np.float32)).pin_memory()
    counts = counts_h.cuda()
    y = torch.empty_like(counts)
    lam = torch.empty_like(counts)
    msf.msf_weights(counts, y, lam, I0, I0)
    del p
    torch.cuda.synchronize()
    return dict(P=P, x_true=x_true, counts_h=counts_h, counts=counts, y=y, lam=lam)


def timed(fn, steps, warmup, dist):
    import torch
    for _ in range(warmup):
        fn()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = t.item()
    return ms


# ---------------------------------------------------------------- algorithmic work per launch

def algorithmic(scan, K1):
    """Algorithmic HBM bytes (or FLOPs) of one launch of each kernel:
    every input read once and every output written once."""
    N = scan.nt * scan.n ** 3
    M = scan.nt * scan.views * scan.nv * scan.nu
    return {
        # forward projection: volume in, sinogram out (+ Lambda, + measurement)
        "joseph_fwd": ("hbm", 4.0 * (N + 2 * M)),
        # adjoint: sinogram in, volume out (+ p in for the CG operator)
        "joseph_adj": ("hbm", 4.0 * (M + 2 * N)),
        "transpose": ("hbm", 8.0 * N),
        "transpose_pupdate": ("hbm", 16.0 * N),
        "cg_update": ("hbm", 4.0 * 6 * N),
        # one colour of the ICD sweep: its voxels read/written, all neighbours read
        "qggmrf_icd": ("hbm", 4.0 * (N + 3 * N / 16)),
        "mace_consensus": ("hbm", 4.0 * 3 * K1 * N),
    }


def roofline(prof, scan, K1, peaks, steps):
    alg = algorithmic(scan, K1)
    name = max(prof, key=lambda k: prof[k][1])
    launches, ms = prof[name]
    kind, work = alg.get(name, ("hbm", None))
    avg_s = ms / launches / 1e3
    if kind == "hbm":
        achieved = work / avg_s / 1e9 if work else None
        peak = peaks.get("hbm_gbs")
        unit = "GB/s"
    else:
        achieved = work / avg_s / 1e12 if work else None
        peak = peaks.get("bf16_tflops")
        unit = "TFLOP/s"
    return {"kernel": name, "bound": kind, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if (achieved and peak) else None, "traffic": None,
            "avg_launch_ms": ms / launches, "launches": launches,
            "share": ms / sum(v[1] for v in prof.values()),
            "peak_source": "measured (MEASURED_PEAKS.json)" if peaks.get("measured") else "fallback"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["measured"] = True
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "measured": False}


# ---------------------------------------------------------------- oracle CPU baseline

def cpu_baseline(scan, settings, learned: bool):
    """Times the FP64 oracle on bounded samples of the workload and composes the
    time of one MACE iteration from the measured unit costs:
      data prox per frame = (n_cg + 1) * views * (one-view A + one-view A^T)
      q-GGMRF = n_sweeps * N * (ICD cost per voxel, on a 16-slice slab of 2 frames)
      CNN agents = 3 * nt * n slices * (one n x n slice through the oracle CNN)
      consensus = N * (numpy cost per voxel on one frame)."""
    import oracle
    from paper_2008_01567_gb300 import synth
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    ell = synth.ellipsoids(99, 6, scan)
    one = synth.Scan(n=scan.n, nt=1, nu=scan.nu, nv=scan.nv, views=1, mode=scan.mode)
    x3 = oracle.ellipsoid_volume(ell[:1], one, ss=1)[0]
    ang = np.array([0.3])
    t0 = time.perf_counter()
    yv = oracle.project(x3, one, ang)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.backproject(yv, one, ang)
    t_adj = time.perf_counter() - t0
    slab = (2, 16, scan.n, scan.n)
    v = synth.uniform(98, slab)
    t0 = time.perf_counter()
    oracle.prox_qggmrf(v, v, settings["sigma"], 2.0, 1.2, 1.0, 0.1, 0.5, 1)
    t_vox = (time.perf_counter() - t0) / v.size
    Ns = scan.n ** 3
    Xs = [synth.uniform(97 + i, (1, scan.n, scan.n, scan.n)) for i in range(4 if learned else 2)]
    t0 = time.perf_counter()
    oracle.mace_iteration(Xs, Xs, [lambda w, x: x] * len(Xs), [1.0 / len(Xs)] * len(Xs), 0.5)
    t_cons = (time.perf_counter() - t0) / Ns
    n_cg = settings["n_cg"]
    T = scan.nt * (n_cg + 1) * scan.views * (t_fwd + t_adj) + scan.nt * Ns * t_cons
    sample = (f"one view of one {scan.n}^3 frame through A and A^T; one ICD sweep of a 2x16x{scan.n}x{scan.n} slab; "
              f"one consensus pass over one frame")
    if learned:
        convs, bns = synth.cnn_weights(7)
        layers = oracle.fold_bn(convs, bns, [(np.zeros(64), np.ones(64))] * 8)
        xs = synth.uniform(96, (1, 5, scan.n, scan.n))
        t0 = time.perf_counter()
        oracle.cnn_forward(xs, layers)
        t_slice = time.perf_counter() - t0
        T += 3 * scan.nt * scan.n * t_slice
        sample += f"; one {scan.n}x{scan.n} slice through the 10-layer CNN"
    else:
        T += settings["n_sweeps"] * scan.nt * Ns * t_vox
    return {"value": 1.0 / T, "unit": "MACE iters/s", "cores": cores, "kind": "oracle",
            "sample": sample + " (FP64 oracle; iteration time composed from these unit costs)",
            "ms_per_iter": T * 1e3}


# ---------------------------------------------------------------- main

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    scan = workload(args.workload)

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        for _ in range(args.warmup):
            cpu_baseline(scan, PLAIN, learned=False)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(cpu_baseline(scan, PLAIN, learned=False))
        wall = time.perf_counter() - t0
        v = statistics.mean(x["value"] for x in vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MACE iters/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"plain q-GGMRF MACE {scan.n}^3x{scan.nt}, det {scan.nu}x{scan.nv}, "
                                       f"{scan.views} views/frame {scan.mode}", "prior": "qggmrf"},
                "cpu_baseline": {k: vals[-1][k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": "MACE iters/s"},
                "e2e": {"value": v, "unit": "MACE iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": wall}
        print(json.dumps(line))
        return

    import torch
    dist = world > 1
    if dist:
        torch.distributed.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2008_01567_gb300 import build, msf
    build.build()
    peaks = load_peaks()

    prob = make_problem(scan, 20200804 + 17 * rank)
    P = prob["P"]
    N = scan.nt * scan.n ** 3
    shape = (2, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    s = PLAIN
    mrf = msf.msf_mrf(2.0, s["q"], s["T"], s["sx"], s["bt"])
    m = msf.Mace(P, W, X, prob["y"], prob["lam"], msf.MSF_PRIOR_QGGMRF, mrf=mrf)

    def step():
        msf.msf_mace_step(m, s["rho"], s["sigma"], s["mu"], s["n_cg"], s["n_sweeps"], want_residual=False)

    for _ in range(args.warmup):
        step()
    clocks = Clocks(local)
    msf.msf_profile_reset()
    msf.msf_profile_enable(True)
    clocks.start()
    ms = timed(step, args.steps, 0, dist)
    ck = clocks.stop()
    msf.msf_profile_enable(False)
    prof = msf.msf_profile_read()
    res = msf.msf_mace_step(m, s["rho"], s["sigma"], s["mu"], s["n_cg"], s["n_sweeps"])
    launches = sum(v[0] for v in prof.values())
    value = world * args.steps / (ms / 1e3)
    nrmse = (torch.linalg.vector_norm(X[0] - prob["x_true"]) / torch.linalg.vector_norm(prob["x_true"])).item()

    # projector throughput: one launch each, algorithmic bytes
    yb = torch.empty_like(prob["y"])
    xb = torch.empty_like(prob["x_true"])
    msf.msf_profile_reset()
    msf.msf_profile_enable(True)
    for _ in range(3):
        msf.msf_project(P, prob["x_true"], yb)
        msf.msf_backproject(P, prob["y"], xb)
    torch.cuda.synchronize()
    msf.msf_profile_enable(False)
    pp = msf.msf_profile_read()
    M = yb.numel()
    fwd_ms = pp["joseph_fwd"][1] / pp["joseph_fwd"][0]
    adj_ms = pp["joseph_adj"][1] / pp["joseph_adj"][0]
    tr_ms = pp["transpose"][1] / pp["transpose"][0]
    projector = {"fwd_ms": fwd_ms, "adj_ms": adj_ms, "transpose_ms": tr_ms,
                 "fwd_GBps_alg": 4.0 * (N + M) / (fwd_ms / 1e3) / 1e9,
                 "adj_GBps_alg": 4.0 * (N + M) / (adj_ms / 1e3) / 1e9,
                 "fwd_Gsteps_per_s": N / scan.n * scan.views * scan.nu * scan.nv / scan.n ** 2 / (fwd_ms / 1e3) / 1e9}

    e2e = None
    if not args.no_e2e:
        ch = prob["counts_h"]
        cd = prob["counts"]

        def e2e_step():
            cd.copy_(ch, non_blocking=True)
            msf.msf_weights(cd, prob["y"], prob["lam"], I0, I0)
            msf.msf_mace_step(m, s["rho"], s["sigma"], s["mu"], s["n_cg"], s["n_sweeps"], want_residual=True)

        e2e_ms = timed(e2e_step, args.steps, 1, dist)
        e2e = {"value": world * args.steps / (e2e_ms / 1e3), "unit": "MACE iters/s",
               "h2d_bytes_per_step": ch.numel() * 4, "d2h_bytes_per_step": 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(scan, s, learned=False)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MACE iters/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded moving-ellipsoid phantom, Poisson 1e4)",
                "config": {"workload": f"plain q-GGMRF MACE {scan.n}^3x{scan.nt}, det {scan.nu}x{scan.nv}, "
                                       f"{scan.views} views/frame {scan.mode}",
                           "prior": "qggmrf", "rho": s["rho"], "sigma": s["sigma"], "mu": s["mu"], "n_cg": s["n_cg"],
                           "n_sweeps": s["n_sweeps"], "l2": "inputs larger than L2 (3.6 GB per 4D volume)"},
                "roofline": roofline(prof, scan, 2, peaks, args.steps),
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": ck,
                "plain": {"iters_per_s": value, "nrmse": nrmse, "residual": res},
                "projector": projector,
                "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}}
        print(json.dumps(line))
    if dist:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
