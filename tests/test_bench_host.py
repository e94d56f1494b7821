"""Host-side helpers of bench.py that run without a GPU."""
import bench

SAMPLE = """0, 2017, 2070, 1210.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 2010, 2070, 1300.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, [N/A], 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active
garbage line
0, 1980, 2070, 1350.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active
"""


def test_clock_samples_parse():
    r = bench.Clocks.parse(SAMPLE)
    assert r["samples"] == 3                       # the [N/A] and malformed lines are skipped
    assert r["sm_mhz"] == 2010 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_samples_empty():
    r = bench.Clocks.parse("")
    assert r["sm_mhz"] is None and r["reasons"] == [] and r["samples"] == 0


def test_replica_seeds_differ():
    assert len({bench.replica_seed(r) for r in range(8)}) == 8


def test_in_grid_crossings_brute_force():
    """The vectorised crossing count of the projector roofline against a
    plane-by-plane enumeration of every ray on a small scan (both protocols)."""
    import math

    import numpy as np

    from paper_2008_01567_gb300 import synth
    for mode in ("sparse360", "wedge90"):
        sc = synth.Scan(n=12, nt=2, nu=15, nv=11, views=3, mode=mode)
        n, c0 = sc.n, 0.5 * (sc.n - 1)
        brute = 0
        for th in sc.angles().ravel():
            c, s = math.cos(th), math.sin(th)
            for iu in range(sc.nu):
                u = (iu - 0.5 * (sc.nu - 1)) * sc.pitch
                sx, sy = sc.dso * c, sc.dso * s
                dx = -(sc.dsd - sc.dso) * c - u * s - sx
                dy = -(sc.dsd - sc.dso) * s + u * c - sy
                xm = abs(dx) >= abs(dy)
                dmaj, smaj = (dx, sx) if xm else (dy, sy)
                da, sa = (dy, sy) if xm else (dx, sx)
                for iv in range(sc.nv):
                    v = (iv - 0.5 * (sc.nv - 1)) * sc.pitch
                    for k in range(n):
                        lam = ((k - c0) * sc.vox - smaj) / dmaj
                        fa = (sa + lam * da) / sc.vox + c0
                        fz = lam * v / sc.vox + c0
                        brute += (-1.0 <= fa < n) and (-1.0 <= fz < n)
        got = bench.in_grid_crossings(sc)
        # interval end points are rounded differently from the per-plane test:
        # allow a crossing exactly on a boundary to fall either way
        assert abs(got - brute) <= max(2, brute // 1000), (mode, got, brute)
        assert 0 < got < sc.nt * sc.views * sc.nu * sc.nv * n


def test_training_lr_schedule():
    # constant for the first two thirds, then a cosine decay to a tenth
    steps = 4800
    lrs = [bench.train_lr(i, steps) for i in range(steps)]
    assert lrs[0] == lrs[2 * steps // 3] == bench.TRAIN_LR
    assert all(a >= b for a, b in zip(lrs, lrs[1:]))
    assert abs(bench.train_lr(steps, steps) - 0.1 * bench.TRAIN_LR) < 1e-12
    assert min(lrs) > 0.1 * bench.TRAIN_LR - 1e-12


def test_quality_points_follow_the_iteration_count():
    # the trajectory stops at twice the quality iteration count
    calls = []

    class Fake:
        def __call__(self, want_residual=False):
            calls.append(want_residual)
            return 0.5 if want_residual else None

    import torch
    x = torch.zeros(4)
    ref = torch.ones(4)
    import paper_2008_01567_gb300.metrics as metrics
    orig = (metrics.psnr, metrics.ssim)
    metrics.psnr = lambda a, b: 0.0
    metrics.ssim = lambda a, b: 0.0
    try:
        at, traj = bench.quality_run(Fake(), x, ref, 30)
        assert [t["iter"] for t in traj] == [10, 20, 30, 60] and at["iters"] == 30 and len(calls) == 60
        calls.clear()
        at, traj = bench.quality_run(Fake(), x, ref, 2)
        assert [t["iter"] for t in traj] == [2] and len(calls) == 2
    finally:
        metrics.psnr, metrics.ssim = orig


def test_roofline_reports_the_dominant_kernel():
    # the kernel with the largest total time is the one reported; its rate is
    # the per-launch algorithmic work over the average launch, its traffic the
    # captured bytes per pixel scaled to the launch's pixel count
    from paper_2008_01567_gb300 import synth
    scan = synth.FULL
    prof = {"joseph_adj": (6, 250.0), "conv3x3_tc": (100, 320.0), "conv1_tc": (10, 20.0)}
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "measured": True}
    r = bench.roofline(prof, scan, 4, peaks, 1)
    px = scan.n ** 3                                     # one time-point of one agent per launch
    assert r["kernel"] == "conv3x3_tc" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["avg_launch_ms"] - 3.2) < 1e-12 and r["launches"] == 100
    flops = 9 * 64 * 64 * 2 * px                         # 3x3 taps x 64 in x 64 out, multiply-add
    assert abs(r["achieved"] - flops / 3.2e-3 / 1e12) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 1700.0) < 1e-12
    assert abs(r["traffic"] - bench.MEASURED_TRAFFIC_PER_PX["conv3x3_tc"] * px) < 1.0
    assert 13.0e9 < r["traffic"] < 14.5e9                 # below the 256 B/px of one read and one write
    assert abs(r["share"] - 320.0 / 590.0) < 1e-12
    assert r["peak_source"].startswith("measured")


def test_projector_roofline_binds_on_the_larger_floor():
    from paper_2008_01567_gb300 import synth
    scan = synth.Scan(n=16, nt=2, nu=24, nv=20, views=4)
    peaks = {"hbm_gbs": 6800.0}
    r = bench.projector_roofline(scan, 0.01, 0.02, 2000.0, peaks)
    X = r["crossings_in_grid"]
    assert 0 < X <= r["crossings_nominal"]
    for name, ms in (("joseph_fwd", 0.01), ("joseph_adj", 0.02)):
        k = r[name]
        floors = (k["fp32_floor_ms"], k["l1_floor_ms"])
        assert k["binding"] == ("l1" if floors[1] >= floors[0] else "fp32")
        assert abs(k["binding_frac"] - max(floors) / ms) < 1e-12
        assert abs(k["G_crossings_per_s"] - X / (ms / 1e3) / 1e9) < 1e-9
    # the adjoint's model moves more bytes and instructions per crossing than the forward's
    assert r["joseph_adj"]["l1_floor_ms"] > r["joseph_fwd"]["l1_floor_ms"]
    assert r["joseph_adj"]["fp32_floor_ms"] > r["joseph_fwd"]["fp32_floor_ms"]
