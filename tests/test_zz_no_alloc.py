"""The allocation-free forward projection (msf_project_static) through the C
ABI, against the plan-based msf_project and against the FP64 oracle.

Some callers cannot let a library allocate device memory: applications that
own the GPU's memory budget through their own pool or allocator, or that must
avoid cudaMalloc's device-wide synchronisation.  msf_project_static serves them
from a fixed static device array.  It performs the forward's FP32 operations in
the forward's order, so it must equal msf_project bit for bit, and like every
projection it must lie within 1e-5 (relative L2 per view) of the FP64 oracle.
This file is collected last so that a run stopping at the first failure has
already run every other test; it passes both alone in a fresh process and after
the rest of the suite."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2008_01567_gb300 import synth
from tests._problems import f32, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5   # the projector tolerance of the other parity tests

# A geometry whose plane check fails only on an interior column: at this view
# the columns switch from x-major to y-major at column 3, and only that column's
# voxel planes reach past the source (found by an FP64 search over geometries).
INTERIOR_FAIL = dict(n=8, nu=9, nv=4, du=0.35, dso=0.8724234700294715, dsd=1.5866013190278845,
                     theta=0.5672320068981571)


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_2008_01567_gb300 import build, msf
    build.build()
    assert torch.cuda.is_available()
    return msf


def _case(M, scan, seed):
    import torch
    P = M.Projector(scan)
    x = torch.empty((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    M.msf_phantom_voxelize(P.vol, synth.ellipsoids(seed, 3, scan), x, ss=2)
    ref = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    M.msf_project(P, x, ref)
    return x, ref


def test_static_projection_equals_plan_projection_twice(M):
    import torch
    a = synth.Scan(n=40, nt=2, nu=45, nv=37, views=5)
    b = dataclasses.replace(synth.PROJ_WEDGE, nt=2)
    xa, ra = _case(M, a, 61)
    xb, rb = _case(M, b, 62)
    # two calls in a row on one geometry, then another geometry, then back:
    # each call rebuilds the shared static table
    for scan, x, ref in ((a, xa, ra), (a, xa, ra), (b, xb, rb), (a, xa, ra)):
        y = torch.full((scan.nt, scan.views, scan.nv, scan.nu), -1.0, device="cuda")
        M.msf_project_static(scan, x, y)
        torch.cuda.synchronize()
        assert torch.equal(y, ref), (scan, (y - ref).abs().max().item())


@pytest.mark.parametrize("mode", ["sparse360", "wedge90"])
def test_static_projection_matches_oracle_per_view(M, mode):
    import torch
    scan = synth.Scan(n=40, nt=2, nu=45, nv=37, views=5, mode=mode)
    x4 = f32(oracle.ellipsoid_volume(synth.ellipsoids(63, 3, scan), scan, ss=2))
    y = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    M.msf_project_static(scan, torch.from_numpy(x4.astype(np.float32)).cuda(), y)
    got = y.cpu().numpy().astype(np.float64)
    ref = oracle.project4d(x4, scan)
    for t in range(scan.nt):
        for j in range(scan.views):
            assert rel_l2(got[t, j], ref[t, j]) <= TOL, (mode, t, j)


def test_static_projection_rejects_what_the_plan_rejects(M):
    import ctypes
    import torch
    g = INTERIOR_FAIL
    ang = np.array([g["theta"]], dtype=np.float64)
    geom = M.msf_geom(g["nu"], g["nv"], 1, g["du"], g["du"], g["dso"], g["dsd"],
                      ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    vol = M.msf_vol(g["n"], g["n"], g["n"], 1, 1.0 / g["n"])
    h = ctypes.c_void_p()
    assert M.lib().msf_projector_create(ctypes.byref(geom), ctypes.byref(vol), ctypes.byref(h)) == 1
    x = torch.zeros((1, g["n"], g["n"], g["n"]), device="cuda")
    y = torch.zeros((1, 1, g["nv"], g["nu"]), device="cuda")
    st = M.lib().msf_project_static(ctypes.byref(geom), ctypes.byref(vol), x.data_ptr(), y.data_ptr(), None)
    assert st == 1 and b"column 3" in M.lib().msf_last_error()


def test_static_projection_rejects_oversize_scans(M):
    import torch
    big = synth.Scan(n=8, nt=16, nu=2048, nv=8, views=24)   # 786432 view-columns > 250000
    x = torch.zeros((big.nt, 8, 8, 8), device="cuda")
    y = torch.zeros((big.nt, big.views, big.nv, big.nu), device="cuda")
    with pytest.raises(M.MsfError) as e:
        M.msf_project_static(big, x, y)
    assert e.value.status == 1 and "static table" in str(e.value)
