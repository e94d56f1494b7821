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
