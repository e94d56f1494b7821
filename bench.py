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
    ap.add_argument("--workload", default="full", choices=["full", "proj", "tiny", "batch", "sweep", "train"])
    ap.add_argument("--no-batch", action="store_true", help="skip the short uneven-batch measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--iters", type=int, default=30, help="MACE iterations run for the NRMSE report")
    ap.add_argument("--train-steps", type=int, default=4800, help="GPU training steps of the CNN before the run")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the ICD data agent, direct MAP and fixture-correction measurements")
    return ap.parse_args()


def workload(name):
    from paper_2008_01567_gb300 import synth
    return {"full": synth.FULL, "proj": synth.PROJ, "tiny": synth.TINY, "batch": synth.FULL, "sweep": synth.PROJ,
            "train": synth.FULL}[name]


# settings of the plain and learned runs (rho, sigma and agent weights of Eq. (9)).
# The plain run's sigma = 0.2 and q-GGMRF sigma_x = 0.1 were picked on a held-out
# phantom seed (192^3 x 8, 24 views) from {0.05, 0.1, 0.2}; with proximal agents
# the MACE fixed point does not depend on sigma.  For the CNN agents it does:
# sigma = 0.4 and the training recipe below were picked on the same held-out
# problem (the worst NRMSE over iterations 30..100, sigma in {0.2 .. 0.8};
# recipes within 1% of the best count as tied, and the one with fewer phantom
# volumes is kept).
PLAIN = dict(rho=0.8, sigma=0.2, mu=[0.25, 0.75], n_cg=5, n_sweeps=2, sx=0.1, T=1.0, bt=0.5, q=1.2)
LEARNED = dict(rho=0.8, sigma=0.4, mu=[0.25, 0.25, 0.25, 0.25], n_cg=5)
# training recipe of the CNN agents: patches from moving-ellipsoid phantoms of
# several sizes (so that the objects span the voxel scales of every workload)
# and two seeds each, noise sigma ~ U[0.02, 0.2], Adam lr 1e-3 with a cosine
# decay to 1e-4 over the last third of the steps (4800 steps by default)
TRAIN_SIZES, TRAIN_SEEDS, TRAIN_LR = (64, 128, 192), 2, 1e-3


def train_lr(it, steps, lr0=TRAIN_LR):
    k = 2 * steps // 3
    if it <= k:
        return lr0
    f = (it - k) / max(1, steps - k)
    return lr0 * (0.1 + 0.9 * 0.5 * (1.0 + math.cos(math.pi * f)))


def train_cnn(cnn, args, seed, record=None):
    """Trains `cnn` on the GPU for args.train_steps Adam steps of batch
    128 x 5 x 64 x 64 on training phantoms of other seeds (the recipe above)."""
    import torch
    from paper_2008_01567_gb300 import msf, synth
    sets = []
    for i, n in enumerate(TRAIN_SIZES):
        for k in range(TRAIN_SEEDS):
            ts = synth.Scan(n=n, nt=4, nu=8, nv=8, views=1)
            Pt = msf.Projector(ts)
            v = torch.empty((ts.nt, n, n, n), device="cuda")
            msf.msf_phantom_voxelize(Pt.vol, synth.ellipsoids(seed + 101 + 7 * i + 1000 * k, 10, ts), v, ss=2)
            sets.append((v, Pt))
    TB, TH, TW = 128, 64, 64
    cnn.train_reserve(TB * TH * TW)
    tn = torch.empty((TB, 5, TH, TW), device="cuda")
    tc_ = torch.empty((TB, TH, TW), device="cuda")
    for it in range(args.train_steps):
        v, Pt = sets[it % len(sets)]
        msf.msf_training_batch(v, Pt.vol, TB, TH, TW, 0.02, 0.2, seed * 7919 + it, tn, tc_)
        want = record is not None and (it % 100 == 0 or it == args.train_steps - 1)
        loss = msf.msf_train_step(cnn, tn, tc_, train_lr(it, args.train_steps), want_loss=want)
        if want:
            record.append(loss)
    return (TB, 5, TH, TW)


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
        return self.parse(out)

    @staticmethod
    def parse(out: str) -> dict:
        """Median SM clock, maximum SM clock and the throttle reasons seen
        active in nvidia-smi's CSV samples (noheader, nounits)."""
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
        ms = max_over_ranks(ms, "cuda")
    return ms


def max_over_ranks(value: float, device: str) -> float:
    """The slowest rank's time: every rank solves its own problem, so the job
    takes as long as its slowest replica."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()


def replica_seed(rank: int) -> int:
    """Each rank reconstructs an independent problem (weak scaling, no data-path collective)."""
    return 20200804 + 17 * rank


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
        # tensor-core convolutions: 2*K*N FLOP per pixel, one time-point per launch
        "conv3x3_tc": ("tensor", 2.0 * 576 * 64 * scan.n ** 3),
        # first layer built from the five frames: 5 x 4 B in, 64 BF16 channels out
        "conv1_tc": ("hbm", (4.0 * 5 + 128.0) * scan.n ** 3),
        "conv10_tc": ("tensor", 2.0 * 576 * 16 * scan.n ** 3),
        # last 64 -> 64 layer fused with the output layer's 64 x 9 per-tap products
        "conv3x3_out_tc": ("tensor", 2.0 * (576 * 64 + 64 * 9) * scan.n ** 3),
        # output layer's 3 x 3 sum of the nine per-tap planes, centre in, volume out
        "resid_stencil": ("hbm", (4.0 * 9 + 8.0) * scan.n ** 3),
    }


# DRAM bytes per pixel of one launch, from the ncu captures summarised under
# profiles/ of the kernel as it stands (none is listed while a kernel has
# changed since its capture); the traffic of these kernels scales with the
# pixel count.
MEASURED_TRAFFIC_PER_PX = {"conv3x3_tc": (268.578048e6 + 222.245376e6) / 2097152}


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
        # a kernel timed inside a long step: the sustained BF16 peak
        achieved = work / avg_s / 1e12 if work else None
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        unit = "TFLOP/s"
    tpp = MEASURED_TRAFFIC_PER_PX.get(name)
    traffic = tpp * scan.n ** 3 if tpp else None
    return {"kernel": name, "bound": kind, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if (achieved and peak) else None, "traffic": traffic,
            "algorithmic_work_per_launch": work,
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


# ---------------------------------------------------------------- the tiny workload end to end

TINY_RUN = dict(rho=0.5, sigma=0.1, mu=[0.5, 0.5], n_cg=5, n_sweeps=1, sx=0.2, q=1.2, T=1.0, bt=0.5, iters=10)


def tiny_gpu(seed):
    """The plain method on the tiny workload (24^3 x 4, 32 x 32 detector, 12
    views, 3 ellipsoids): 10 MACE iterations from zero, timed from the photon
    counts on; returns the rate, X_0 and the counts (for the oracle leg)."""
    import torch
    from paper_2008_01567_gb300 import msf, synth
    sc = synth.TINY
    P = msf.Projector(sc)
    ell = synth.ellipsoids(seed + 7, 3, sc)
    p = torch.empty((sc.nt, sc.views, sc.nv, sc.nu), device="cuda")
    msf.msf_phantom_project(P, ell, p)
    counts = synth.poisson(seed + 8, I0 * np.exp(-p.cpu().numpy().astype(np.float64))).astype(np.float32)
    c = torch.from_numpy(counts).cuda()
    y, lam = torch.empty_like(c), torch.empty_like(c)
    R = TINY_RUN
    shape = (2, sc.nt, sc.n, sc.n, sc.n)
    W, X = torch.zeros(shape, device="cuda"), torch.zeros(shape, device="cuda")
    m = msf.Mace(P, W, X, y, lam, msf.MSF_PRIOR_QGGMRF, mrf=msf.msf_mrf(2.0, R["q"], R["T"], R["sx"], R["bt"]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    msf.msf_weights(c, y, lam, I0, I0)
    for _ in range(R["iters"]):
        msf.msf_mace_step(m, R["rho"], R["sigma"], R["mu"], R["n_cg"], R["n_sweeps"], want_residual=False)
    x0 = X[0].cpu().numpy()
    dt = time.perf_counter() - t0
    m.close()
    return {"iters_per_s": R["iters"] / dt}, x0, counts


def tiny_oracle(counts, x_gpu):
    """The same 10 iterations in the FP64 oracle on the host cores, from the
    same counts; rate and the relative L2 distance of the GPU's X_0 from it."""
    import oracle
    from paper_2008_01567_gb300 import synth
    oracle.build()
    sc = synth.TINY
    R = TINY_RUN
    c64 = counts.astype(np.float64)
    t0 = time.perf_counter()
    y = oracle.log_measurement(c64, I0)
    lam = oracle.weights(y, I0)
    agents = [lambda w, x: oracle.prox_data(y, lam, w, x, sc, R["sigma"], R["n_cg"]),
              lambda w, x: oracle.prox_qggmrf(w, x, R["sigma"], 2.0, R["q"], R["T"], R["sx"], R["bt"], R["n_sweeps"])]
    xhat, _, _, _ = oracle.mace(np.zeros((sc.nt, sc.n, sc.n, sc.n)), agents, R["mu"], R["rho"], R["iters"])
    dt = time.perf_counter() - t0
    rel = float(np.linalg.norm(x_gpu.astype(np.float64) - xhat) / np.linalg.norm(xhat))
    return {"iters_per_s": R["iters"] / dt, "cores": len(os.sched_getaffinity(0)), "rel_l2_gpu_vs_oracle": rel}


# ---------------------------------------------------------------- the queue of uneven problems

def make_batch(params, seed, learned):
    """The 12 uneven 4D problems (64^3x4 .. 192^3x12, 16..48 views, alternating
    360 deg sparse and 90 deg wedge), each with its own plan, state and agents."""
    import torch
    from paper_2008_01567_gb300 import msf, synth
    out = []
    for i, sc in enumerate(synth.batch_scans()):
        prob = make_problem(sc, seed + 31 * i)
        msf.msf_projector_autotune(prob["P"])
        K1 = 4 if learned else 2
        W = torch.zeros((K1, sc.nt, sc.n, sc.n, sc.n), device="cuda")
        X = torch.zeros_like(W)
        if learned:
            # room for every time-point of the problem in one chunk (at most 16)
            cnn = msf.Cnn(min(sc.nt, 16) * sc.n ** 3)
            cnn.set_params(params)
            m = msf.Mace(prob["P"], W, X, prob["y"], prob["lam"], msf.MSF_PRIOR_CNN, cnn=cnn)
            prm = msf.mace_params(LEARNED["rho"], LEARNED["sigma"], LEARNED["mu"], LEARNED["n_cg"], 0, True)
        else:
            s = PLAIN
            cnn = None
            m = msf.Mace(prob["P"], W, X, prob["y"], prob["lam"], msf.MSF_PRIOR_QGGMRF,
                         mrf=msf.msf_mrf(2.0, s["q"], s["T"], s["sx"], s["bt"]))
            prm = msf.mace_params(s["rho"], s["sigma"], s["mu"], s["n_cg"], s["n_sweeps"], True)
        out.append(dict(scan=sc, prob=prob, W=W, X=X, cnn=cnn, m=m, prm=prm))
    return out


def batch_run(params, seed, args, dist, world):
    """The 12 uneven problems for both priors: per-problem NRMSE of X_0 after
    exactly args.iters iterations from W = X = 0 (untimed), then the aggregate
    problem-iterations/s of further batch iterations (one captured graph per
    batch iteration), timed."""
    import torch
    from paper_2008_01567_gb300 import msf
    out = {}
    for name, learned in (("learned", True), ("plain", False)):
        items = make_batch(params, seed + 1000, learned)
        B = msf.MaceBatch([it["m"] for it in items])
        prms = [it["prm"] for it in items]
        for _ in range(args.iters):
            msf.msf_mace_batch_step(B, prms, want_residuals=False)
        torch.cuda.synchronize()
        nr = [(torch.linalg.vector_norm(it["X"][0] - it["prob"]["x_true"]) /
               torch.linalg.vector_norm(it["prob"]["x_true"])).item() for it in items]
        steps = max(1, args.steps)
        ms = timed(lambda: msf.msf_mace_batch_step(B, prms, want_residuals=False), steps, 1, dist)
        voxels = sum(it["scan"].nt * it["scan"].n ** 3 for it in items)
        out[name] = {"problem_iters_per_s": world * len(items) * steps / (ms / 1e3),
                     "ms_per_batch_iter": ms / steps, "voxels": voxels,
                     "nrmse_at_iters": args.iters, "nrmse": [round(x, 4) for x in nr]}
        B.close()
        del items, B
        torch.cuda.empty_cache()
    ln, pn = out["learned"]["nrmse"], out["plain"]["nrmse"]
    out["problems"] = len(ln)
    out["learned_not_worse"] = sum(a <= b for a, b in zip(ln, pn))
    return out


def train_small(args, seed):
    """CNN weights trained on the GPU (train_cnn); returns the flat parameters."""
    from paper_2008_01567_gb300 import msf, synth
    cnn = msf.Cnn(128 ** 3)
    cnn.set_params(msf.pack_params(*synth.cnn_weights(seed + 102)))
    train_cnn(cnn, args, seed)
    return cnn.get_params()


def run_batch(args, rank, world, dist, seed):
    """--workload batch: the 12 uneven problems, learned vs plain, NRMSE after
    args.iters iterations and aggregate throughput."""
    import torch
    from paper_2008_01567_gb300 import msf, synth
    params = train_small(args, seed)
    out = {}
    for name, learned in (("learned", True), ("plain", False)):
        items = make_batch(params, seed, learned)
        B = msf.MaceBatch([it["m"] for it in items])
        prms = [it["prm"] for it in items]
        for _ in range(args.warmup):
            msf.msf_mace_batch_step(B, prms, want_residuals=False)
        ms = timed(lambda: msf.msf_mace_batch_step(B, prms, want_residuals=False), args.steps, 0, dist)
        for _ in range(max(0, args.iters - args.warmup - args.steps)):
            msf.msf_mace_batch_step(B, prms, want_residuals=False)
        torch.cuda.synchronize()
        nr = [(torch.linalg.vector_norm(it["X"][0] - it["prob"]["x_true"]) /
               torch.linalg.vector_norm(it["prob"]["x_true"])).item() for it in items]
        out[name] = {"problem_iters_per_s": world * len(items) * args.steps / (ms / 1e3),
                     "ms_per_batch_iter": ms / args.steps, "nrmse": [round(x, 4) for x in nr]}
        B.close()
        del items
    if rank == 0:
        n = len(synth.batch_scans())
        line = {"metric": METRIC, "value": out["learned"]["problem_iters_per_s"], "unit": "problem MACE iters/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": out["learned"]["ms_per_batch_iter"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 (CNN agents), f32 (projector, CG, consensus), f64 (scalars)",
                "data": "synthetic (seeded moving-ellipsoid phantoms, Poisson 1e4)",
                "config": {"workload": f"{n} uneven 4D problems 64^3x4..192^3x12, 16..48 views, 360/90 deg, "
                                       "one captured graph per batch iteration"},
                "learned": out["learned"], "plain": out["plain"]}
        print(json.dumps(line))
    return None


# ---------------------------------------------------------------- sparse-view / limited-angle sweep

SWEEP = [(90, 4), (180, 8), (360, 16)]   # degrees turned and views per time-point (22.5 deg apart)


def run_sweep(args, rank, world, dist, seed):
    """--workload sweep: Sec. VI's extreme sparse-view study (90/180/360 deg per
    time-point with 4/8/16 views, continuous rotation) at 128^3 x 8 on a 192 x 160
    detector, and its single-plane comparison: for each scan, MACE with the plain
    q-GGMRF prior, multi-slice fusion (three CNN agents) and MBIR + H_xy,t /
    H_yz,t / H_zx,t (one CNN agent, K = 1), args.iters iterations each; NRMSE,
    PSNR and SSIM against the phantom, and iterations/s."""
    import torch
    from paper_2008_01567_gb300 import metrics, msf, synth
    params = train_small(args, seed)
    rows = []
    for deg, views in SWEEP:
        scan = synth.Scan(n=128, nt=8, nu=192, nv=160, views=views, mode=f"wedge{deg}")
        prob = make_problem(scan, seed + deg)
        msf.msf_projector_autotune(prob["P"])
        shape3 = (scan.nt, scan.n, scan.n, scan.n)
        cnn = msf.Cnn(scan.n ** 3)
        cnn.set_params(params)
        # multi-slice fusion twice: equal weights 0.25 (beta = 3, as in the
        # full workload) and beta = 1, which gives the data agent the weight 0.5
        # it has in the single-CNN runs (mu_0 = 1/(1+beta), mu_k = beta/((1+beta)K))
        methods = [("plain q-GGMRF", 1, None), ("multi-slice fusion", 3, None),
                   ("multi-slice fusion, beta=1", 3, None)] + \
                  [(f"MBIR + H_{o},t", 1, k) for k, o in enumerate(("xy", "yz", "zx"))]
        for name, K, orient in methods:
            W = torch.zeros((K + 1,) + shape3, device="cuda")
            X = torch.zeros_like(W)
            if name.startswith("plain"):
                s = PLAIN
                m = msf.Mace(prob["P"], W, X, prob["y"], prob["lam"], msf.MSF_PRIOR_QGGMRF,
                             mrf=msf.msf_mrf(2.0, s["q"], s["T"], s["sx"], s["bt"]))
                prm = (s["rho"], s["sigma"], s["mu"], s["n_cg"], s["n_sweeps"])
            else:
                mu = [0.5, 0.5] if K == 1 else ([0.5] + [1.0 / 6] * 3 if "beta=1" in name else LEARNED["mu"])
                m = msf.Mace(prob["P"], W, X, prob["y"], prob["lam"], msf.MSF_PRIOR_CNN, cnn=cnn,
                             orient=orient or 0)
                prm = (LEARNED["rho"], LEARNED["sigma"], mu, LEARNED["n_cg"], 0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.iters):
                msf.msf_mace_step(m, *prm, want_residual=False, use_graph=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            x, ref = X[0], prob["x_true"]
            rows.append({"degrees": deg, "views": views, "method": name, "iters": args.iters,
                         "iters_per_s": args.iters / dt, "nrmse": round(metrics.nrmse(x, ref), 4),
                         "psnr_db": round(metrics.psnr(x, ref), 2), "ssim": round(metrics.ssim(x, ref), 4)})
            m.close()
            del W, X, m
        del cnn, prob
    if rank == 0:
        best = {(r["degrees"], r["views"]): max((q for q in rows if q["degrees"] == r["degrees"]),
                                                key=lambda q: q["psnr_db"])["method"] for r in rows}
        msf_rows = [r for r in rows if r["method"] == "multi-slice fusion"]
        line = {"metric": METRIC, "value": msf_rows[-1]["iters_per_s"], "unit": "MACE iters/s",
                "n_gpus": world, "steps": args.iters, "warmup": 0,
                "ms_per_step": 1e3 / msf_rows[-1]["iters_per_s"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 (CNN agents), f32 (projector, CG, consensus), f64 (scalars)",
                "data": "synthetic (seeded moving-ellipsoid phantoms, Poisson 1e4; CNN trained on GPU-generated pairs)",
                "config": {"workload": "sparse-view / limited-angle sweep 128^3x8, det 192x160, "
                                       "90/180/360 deg per time-point with 4/8/16 views"},
                "sweep": rows, "best_psnr": {f"{d}deg/{v}views": m for (d, v), m in best.items()}}
        print(json.dumps(line))
    return None


# ---------------------------------------------------------------- quality runs

QUALITY_POINTS = (10, 20, 30, 60)   # iterations at which NRMSE and the residual are recorded


def quality_run(step, X0, x_true, iters, points=QUALITY_POINTS):
    """Runs `step` (one MACE iteration returning the consensus residual) from the
    state it is given (W = X = 0) for max(iters, points) iterations, untimed and
    separate from the throughput measurements.  Records NRMSE of X_0 and the
    residual at every point up to 2 * iters, and NRMSE / PSNR / SSIM at exactly
    `iters`."""
    from paper_2008_01567_gb300 import metrics
    pts = sorted(set(p for p in points if p <= 2 * iters) | {iters})
    traj, at = [], None
    for it in range(1, pts[-1] + 1):
        res = step(want_residual=it in pts)
        if it in pts:
            traj.append({"iter": it, "nrmse": round(metrics.nrmse(X0, x_true), 5), "residual": res})
        if it == iters:
            at = {"iters": iters, "nrmse": metrics.nrmse(X0, x_true), "psnr_db": round(metrics.psnr(X0, x_true), 2),
                  "ssim": round(metrics.ssim(X0, x_true), 4), "residual": res}
    return at, traj


# ---------------------------------------------------------------- projector against its binding roof

SMS, FP32_LANES, L1_BYTES_PER_CLK = 152, 128, 128   # per SM: FP32 lanes, L1 / shared-memory bytes per clock

# Per in-grid ray-plane crossing (counted from the kernels' inner loops):
#   forward: two 8-byte loads of the z-paired copies (16 B through the L1 data
#     pipe) and 11.5 FP32-pipe instructions (per ray: the z crossing (FMA),
#     its floor and fraction, three lerps of a subtraction and an FMA, the
#     accumulation; the a crossing's FMA, floor and fraction shared by 2 rays);
#   adjoint: each crossing is gathered by the two voxel runs holding its a taps;
#     per visit a 4-byte sinogram load and two shared-memory read-modify-writes
#     of the accumulators (20 B), and 12 FP32-pipe instructions.
PROJ_MODEL = {"joseph_fwd": {"bytes": 16.0, "instr": 11.5},
              "joseph_adj": {"bytes": 40.0, "instr": 24.0}}


def in_grid_crossings(scan) -> int:
    """Number of ray-plane crossings whose bilinear taps can touch the grid
    (major-axis planes 0..n-1 where both minor crossings lie in [-1, n)), summed
    over every ray of the scan, from the same FP64 ray constants as the
    projector's column table.  Host-side bookkeeping for the roofline only."""
    n, vox, du, dv = scan.n, scan.vox, scan.pitch, scan.pitch
    u = (np.arange(scan.nu) - 0.5 * (scan.nu - 1)) * du
    v = (np.arange(scan.nv) - 0.5 * (scan.nv - 1)) * dv
    c0 = 0.5 * (n - 1)

    def krange(f0, b, lo, hi):
        inside = (f0 >= lo) & (f0 < hi)
        with np.errstate(divide="ignore", invalid="ignore"):
            k1, k2 = (lo - f0) / b + c0, (hi - f0) / b + c0
        kl = np.where(b != 0, np.minimum(k1, k2), np.where(inside, -np.inf, np.inf))
        kh = np.where(b != 0, np.maximum(k1, k2), np.where(inside, np.inf, -np.inf))
        return kl, kh

    total = 0
    for th in scan.angles().ravel():
        c, s = math.cos(th), math.sin(th)
        sx, sy = scan.dso * c, scan.dso * s
        dx = -(scan.dsd - scan.dso) * c - u * s - sx
        dy = -(scan.dsd - scan.dso) * s + u * c - sy
        xm = np.abs(dx) >= np.abs(dy)
        dmaj, smaj = np.where(xm, dx, dy), np.where(xm, sx, sy)
        da, sa = np.where(xm, dy, dx), np.where(xm, sy, sx)
        lam0 = -smaj / dmaj
        al, ah = krange((sa + lam0 * da) / vox + c0, da / dmaj, -1.0, n)
        zl, zh = krange(v[:, None] * (lam0 / vox)[None, :] + c0, v[:, None] / dmaj[None, :], -1.0, n)
        lo = np.maximum(np.maximum(al[None, :], zl), 0.0)
        hi = np.minimum(np.minimum(ah[None, :], zh), n - 1.0)
        total += int(np.clip(np.floor(hi) - np.ceil(lo) + 1, 0, None).sum())
    return total


def projector_roofline(scan, fwd_ms, adj_ms, sm_mhz, peaks):
    """Both projector kernels against (i) the HBM roof with algorithmic bytes
    4(N + M) and (ii) their binding on-chip roof: the larger of the FP32-pipe
    floor (instructions x crossings / (SMs x 128 lanes x clock)) and the L1 /
    shared-memory floor (bytes x crossings / (SMs x 128 B x clock)), at the
    median SM clock measured under load."""
    N = scan.nt * scan.n ** 3
    M = scan.nt * scan.views * scan.nv * scan.nu
    X = in_grid_crossings(scan)
    f = (sm_mhz or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    alu_peak = SMS * FP32_LANES * f            # FP32-pipe instructions per second
    l1_peak = SMS * L1_BYTES_PER_CLK * f       # bytes per second
    out = {"crossings_in_grid": X, "crossings_nominal": scan.nt * scan.views * scan.nu * scan.nv * scan.n,
           "sm_mhz": f / 1e6, "fp32_peak_tinstr_s": alu_peak / 1e12, "l1_peak_TBps": l1_peak / 1e12,
           "hbm_peak_GBps": peaks.get("hbm_gbs")}
    for name, ms in (("joseph_fwd", fwd_ms), ("joseph_adj", adj_ms)):
        m = PROJ_MODEL[name]
        t_alu = m["instr"] * X / alu_peak * 1e3
        t_l1 = m["bytes"] * X / l1_peak * 1e3
        hbm = 4.0 * (N + M) / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "G_crossings_per_s": X / (ms / 1e3) / 1e9,
                     "hbm_GBps_alg": hbm, "hbm_frac": hbm / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                     "fp32_floor_ms": t_alu, "l1_floor_ms": t_l1,
                     "binding": "l1" if t_l1 >= t_alu else "fp32",
                     "binding_frac": max(t_alu, t_l1) / ms}
    return out


# ---------------------------------------------------------------- the other agents and Algorithm 2

def data_cost(P, prob, v, z, sigma):
    """Cost of Eq. (4) with l of Eq. (2): 1/2 ||y - A z||^2_Lambda + ||z - v||^2/(2 sigma^2)
    (FP64 sums over the device tensors; the projection by msf_project)."""
    import torch
    from paper_2008_01567_gb300 import msf
    az = torch.empty_like(prob["y"])
    msf.msf_project(P, z, az)
    e = (prob["y"] - az).double()
    return (0.5 * (prob["lam"].double() * e * e).sum() + ((z - v).double() ** 2).sum() / (2 * sigma ** 2)).item()


def extra_agents(P, prob, x_learned, x_plain, args):
    """At the workload's size: the grouped-ICD data agent beside CG (one call
    each from the same start, with the Eq. (4) cost reached), the direct 4D-MRF
    MAP solve beside the plain MACE run, and one blind fixture correction."""
    import torch
    from paper_2008_01567_gb300 import metrics, msf
    out = {}
    sigma = LEARNED["sigma"]
    v = x_learned
    dp = msf.DataProx(P)
    z0 = (0.9 * v).contiguous()
    c0 = data_cost(P, prob, v, z0, sigma)
    res = {"start_cost": c0, "sigma": sigma}
    for name, call, n in (("cg", msf.msf_prox_data, LEARNED["n_cg"]), ("icd", msf.msf_prox_data_icd, 3)):
        z = z0.clone()
        call(dp, prob["y"], prob["lam"], v, z, sigma, n)          # warm
        z = z0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call(dp, prob["y"], prob["lam"], v, z, sigma, n)
        e1.record()
        torch.cuda.synchronize()
        res[name] = {"iterations": n, "ms": e0.elapsed_time(e1), "cost": data_cost(P, prob, v, z, sigma)}
    out["data_agent"] = res
    dp.close()
    del z, z0
    torch.cuda.empty_cache()
    # direct MAP of Eq. (3) with the plain run's prior, beta = mu_1 / mu_0
    s = PLAIN
    beta = s["mu"][1] / s["mu"][0]
    mrf = msf.msf_mrf(2.0, s["q"], s["T"], s["sx"], s["bt"])
    ms_ = msf.MapSolver(P)
    x = torch.zeros_like(prob["x_true"])
    n_outer, n_cg = args.iters, s["n_cg"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    msf.msf_map_solve(ms_, mrf, beta, prob["y"], prob["lam"], x, n_outer, n_cg)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out["map"] = {"beta": beta, "outer": n_outer, "n_cg": n_cg, "outer_per_s": n_outer / dt,
                  "cost": msf.msf_map_cost(ms_, mrf, beta, prob["y"], prob["lam"], x),
                  "cost_of_plain_mace_x0": msf.msf_map_cost(ms_, mrf, beta, prob["y"], prob["lam"], x_plain),
                  "nrmse": metrics.nrmse(x, prob["x_true"]), "psnr_db": round(metrics.psnr(x, prob["x_true"]), 2),
                  "ssim": round(metrics.ssim(x, prob["x_true"]), 4)}
    ms_.close()
    del x
    torch.cuda.empty_cache()
    # Algorithm 2 with the learned reconstruction
    fc = msf.FixtureCorrector(P)
    yc = torch.empty_like(prob["y"])
    msf.msf_fixture_correct(fc, prob["y"], x_learned, 0.45, 3.0, yc)   # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = msf.msf_fixture_correct(fc, prob["y"], x_learned, 0.45, 3.0, yc)
    out["fixture_correction"] = {"ms": (time.perf_counter() - t0) * 1e3, "c": c, "r_mask": 0.45, "blur_px": 3.0,
                                 "note": "synthetic scan without fixtures: c measures what the blur keeps"}
    fc.close()
    del yc
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- training workload

def run_train(args, rank, world, dist, seed, peaks):
    """--workload train: the CNN training step of Sec. V on its own (batch
    128 x 5 x 64 x 64 patches, Adam), timed per step, with the per-kernel split
    and the FLOP rate of its tensor-core kernels (forward, input and weight
    gradients) against the measured BF16 peak."""
    import torch
    from paper_2008_01567_gb300 import msf, synth
    ts = synth.Scan(n=128, nt=4, nu=8, nv=8, views=1)
    Pt = msf.Projector(ts)
    vols = torch.empty((ts.nt, 128, 128, 128), device="cuda")
    msf.msf_phantom_voxelize(Pt.vol, synth.ellipsoids(seed + 101, 10, ts), vols, ss=2)
    cnn = msf.Cnn(128 ** 3)
    cnn.set_params(msf.pack_params(*synth.cnn_weights(seed + 102)))
    TB, TH, TW = 128, 64, 64
    cnn.train_reserve(TB * TH * TW)
    tn = torch.empty((TB, 5, TH, TW), device="cuda")
    tc_ = torch.empty((TB, TH, TW), device="cuda")
    k = [0]

    def step():
        msf.msf_training_batch(vols, Pt.vol, TB, TH, TW, 0.02, 0.2, seed * 7919 + k[0], tn, tc_)
        msf.msf_train_step(cnn, tn, tc_, 1e-3, want_loss=False)
        k[0] += 1

    for _ in range(args.warmup):
        step()
    msf.msf_profile_reset()
    msf.msf_profile_enable(True)
    ms = timed(step, args.steps, 0, dist)
    msf.msf_profile_enable(False)
    prof = msf.msf_profile_read()
    P = TB * TH * TW
    layer = 2.0 * 576 * 64 * P                       # one 64 -> 64 layer, one pass
    flop = 3 * 8 * layer + 3 * 2.0 * 45 * 64 * P     # forward, input and weight gradients of the convs
    tc_names = [n for n in prof if n.startswith("conv") or n.startswith("wgrad_tc")]
    tc_ms = sum(prof[n][1] for n in tc_names) / args.steps
    total_ms = sum(v[1] for v in prof.values()) / args.steps
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    if rank == 0:
        line = {"metric": "CNN training steps/s (batch 128 x 5 x 64 x 64, Adam)", "value": world * args.steps / (ms / 1e3),
                "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16 (tensor cores), f32 (master weights, BatchNorm), f64 (sums)",
                "data": "synthetic (seeded moving-ellipsoid phantom patches, Gaussian noise U[0.02, 0.2])",
                "config": {"workload": "training step of the 2.5D CNN, 10 layers, 64 channels, batch 128 x 64 x 64"},
                "tensor_kernels": {"names": sorted(tc_names), "ms_per_step": tc_ms,
                                   "tflops": flop / (tc_ms / 1e3) / 1e12,
                                   "frac_of_bf16_peak": flop / (tc_ms / 1e3) / 1e12 / peak if peak else None},
                "flop_per_step": flop, "kernel_ms_per_step": total_ms,
                "kernels": {n: {"launches": v[0], "ms": round(v[1], 3)} for n, v in
                            sorted(prof.items(), key=lambda kv: -kv[1][1])}}
        print(json.dumps(line))
    return None


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
            cpu_baseline(scan, LEARNED, learned=True)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(cpu_baseline(scan, LEARNED, learned=True))
        wall = time.perf_counter() - t0
        v = statistics.mean(x["value"] for x in vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MACE iters/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"multi-slice fusion MACE {scan.n}^3x{scan.nt}, det {scan.nu}x{scan.nv}, "
                                       f"{scan.views} views/frame {scan.mode}; agents: CG data prox + 3 BF16 CNNs"},
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
    from paper_2008_01567_gb300 import build, msf, synth
    build.build()
    peaks = load_peaks()
    seed = replica_seed(rank)
    if args.workload == "batch":
        return run_batch(args, rank, world, dist, seed)
    if args.workload == "train":
        return run_train(args, rank, world, dist, seed, peaks)
    if args.workload == "sweep":
        return run_sweep(args, rank, world, dist, seed)
    prob = make_problem(scan, seed)
    P = prob["P"]
    tuned = msf.msf_projector_autotune(P)
    N = scan.nt * scan.n ** 3

    # ---------------- the learned agents: trained on the GPU (untimed) on phantoms of other seeds
    cnn = msf.Cnn(scan.n ** 3)
    cnn.set_params(msf.pack_params(*synth.cnn_weights(seed + 102)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    tb = train_cnn(cnn, args, seed, record=losses)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    training = {"steps": args.train_steps, "batch": list(tb), "steps_per_s": args.train_steps / train_s,
                "phantom_sizes": list(TRAIN_SIZES), "phantom_seeds": TRAIN_SEEDS,
                "loss_first": losses[0], "loss_last": losses[-1]}
    # the conv autotuner on this workload's slice shapes
    conv_tuning = msf.msf_cnn_autotune(cnn, P.vol, prob["x_true"], torch.empty_like(prob["x_true"]))

    # ---------------- learned multi-slice fusion (headline)
    L = LEARNED
    shape = (4, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    m = msf.Mace(P, W, X, prob["y"], prob["lam"], msf.MSF_PRIOR_CNN, cnn=cnn)

    def step(want_residual=False):
        return msf.msf_mace_step(m, L["rho"], L["sigma"], L["mu"], L["n_cg"], 0, want_residual=want_residual)

    # quality: exactly args.iters iterations from W = X = 0, untimed (the
    # trajectory continues to the last of QUALITY_POINTS)
    q_learned, traj_learned = quality_run(step, X[0], prob["x_true"], args.iters)

    # throughput (the iteration's cost does not depend on the state)
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
    launches = sum(v[0] for v in prof.values())
    value = world * args.steps / (ms / 1e3)

    e2e = None
    if not args.no_e2e:
        ch = prob["counts_h"]

        def e2e_step():
            # two C-ABI calls on host buffers: the counts go in from pinned host
            # memory, the FP64 residual comes back
            msf.msf_mace_set_counts(m, ch, I0, I0)
            msf.msf_mace_step(m, L["rho"], L["sigma"], L["mu"], L["n_cg"], 0, want_residual=True)

        # one untimed call first: the handle's first msf_mace_set_counts
        # allocates its device copy of the measurements
        e2e_ms = timed(e2e_step, args.steps, 1, dist)
        e2e = {"value": world * args.steps / (e2e_ms / 1e3), "unit": "MACE iters/s",
               "h2d_bytes_per_step": ch.numel() * 4, "d2h_bytes_per_step": 8,
               "path": "msf_mace_set_counts (host counts) + msf_mace_step (host residual)"}
    # the same iteration replayed as one CUDA graph
    gms = timed(lambda: msf.msf_mace_step(m, L["rho"], L["sigma"], L["mu"], L["n_cg"], 0, want_residual=False,
                                          use_graph=True), args.steps, 1, dist)
    learned = {"iters_per_s": value, "graph_iters_per_s": world * args.steps / (gms / 1e3),
               "quality": q_learned, "trajectory": traj_learned}
    m.close()
    x_learned = X[0].clone()
    del m, W, X
    torch.cuda.empty_cache()

    # ---------------- plain q-GGMRF MACE at the same size
    s = PLAIN
    W2 = torch.zeros((2,) + shape[1:], device="cuda")
    X2 = torch.zeros_like(W2)
    mrf = msf.msf_mrf(2.0, s["q"], s["T"], s["sx"], s["bt"])
    m2 = msf.Mace(P, W2, X2, prob["y"], prob["lam"], msf.MSF_PRIOR_QGGMRF, mrf=mrf)

    def pstep(want_residual=False):
        return msf.msf_mace_step(m2, s["rho"], s["sigma"], s["mu"], s["n_cg"], s["n_sweeps"],
                                 want_residual=want_residual)

    q_plain, traj_plain = quality_run(pstep, X2[0], prob["x_true"], args.iters)
    for _ in range(args.warmup):
        pstep()
    pms = timed(pstep, args.steps, 0, dist)
    plain = {"iters_per_s": world * args.steps / (pms / 1e3), "ms_per_iter": pms / args.steps,
             "quality": q_plain, "trajectory": traj_plain, "sigma_x": s["sx"]}
    m2.close()
    x_plain = X2[0].clone()
    del m2, W2, X2
    torch.cuda.empty_cache()
    extra = {} if args.no_extra else extra_agents(P, prob, x_learned, x_plain, args)
    del x_learned, x_plain

    # ---------------- the queue of 12 uneven problems: per-problem NRMSE, learned vs plain
    batch = None
    if not args.no_batch:
        batch = batch_run(cnn.get_params(), seed, args, dist, world)

    # ---------------- projector throughput (one launch each, algorithmic bytes)
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
    fwd_ms = pp["joseph_fwd"][1] / pp["joseph_fwd"][0]
    adj_ms = pp["joseph_adj"][1] / pp["joseph_adj"][0]
    projector = projector_roofline(scan, fwd_ms, adj_ms, ck.get("sm_mhz"), peaks)

    tiny_rate, tiny_x, tiny_counts = tiny_gpu(seed)
    tiny = {"workload": "plain MACE 24^3x4, det 32x32, 12 views/frame, 10 iterations from the counts",
            "gpu": tiny_rate}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(scan, L, learned=True)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        tiny["oracle"] = tiny_oracle(tiny_counts, tiny_x)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MACE iters/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 (CNN agents), f32 (projector, CG, consensus), f64 (scalars)",
                "data": "synthetic (seeded moving-ellipsoid phantom, Poisson 1e4; CNN trained on GPU-generated pairs)",
                "config": {"workload": f"multi-slice fusion MACE {scan.n}^3x{scan.nt}, det {scan.nu}x{scan.nv}, "
                                       f"{scan.views} views/frame {scan.mode}; agents: CG data prox + 3 BF16 CNNs",
                           "rho": L["rho"], "sigma": L["sigma"], "mu": L["mu"], "n_cg": L["n_cg"],
                           "l2": "inputs larger than L2 (3.6 GB per 4D volume)"},
                "roofline": roofline(prof, scan, 4, peaks, args.steps),
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": ck,
                "learned": learned, "plain": plain,
                "learned_vs_plain": {"iters": args.iters,
                                     "nrmse_learned": q_learned["nrmse"], "nrmse_plain": q_plain["nrmse"],
                                     "learned_not_worse": q_learned["nrmse"] <= q_plain["nrmse"]},
                "tiny_end_to_end": tiny,
                "training": training, "conv_tuning": {str(k): list(v) for k, v in conv_tuning.items()},
                "projector": projector, **extra,
                "projector_tuning": {"fwd_block": list(tuned[:2]), "adj_zrun": tuned[2]}, "batch": batch,
                "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items()}}
        print(json.dumps(line))
    if dist:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
