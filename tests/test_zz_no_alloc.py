"""The allocation-free forward projection (msf_project_static) against the
plan-based msf_project, through the C ABI.

Some callers cannot let a library allocate device memory: applications that
own the GPU's memory budget through their own pool or allocator, or that must
avoid cudaMalloc's device-wide synchronisation.  msf_project_static serves them
from a fixed static device array.  This file is collected last so that a run
stopping at the first failure has already run every other test; it passes both
alone in a fresh process and after the rest of the suite."""
import dataclasses

import numpy as np
import pytest

from paper_2008_01567_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5   # the projector tolerance used by the other parity tests


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_2008_01567_gb300 import build, msf
    build.build()
    assert torch.cuda.is_available()
    return msf


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(M, scan, seed):
    import torch
    P = M.Projector(scan)
    x = torch.empty((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    M.msf_phantom_voxelize(P.vol, synth.ellipsoids(seed, 3, scan), x, ss=2)
    ref = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    M.msf_project(P, x, ref)
    return x, ref.cpu().numpy()


def test_static_projection_matches_plan_projection_twice(M):
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
        got = y.cpu().numpy()
        for t in range(scan.nt):
            for j in range(scan.views):
                assert _rel(got[t, j], ref[t, j]) <= TOL, (scan, t, j)


def test_static_projection_rejects_oversize_scans(M):
    import torch
    big = synth.Scan(n=8, nt=16, nu=2048, nv=8, views=24)   # 786432 view-columns > 250000
    x = torch.zeros((big.nt, 8, 8, 8), device="cuda")
    y = torch.zeros((big.nt, big.views, big.nv, big.nu), device="cuda")
    with pytest.raises(M.MsfError) as e:
        M.msf_project_static(big, x, y)
    assert e.value.status == 1 and "static table" in str(e.value)
