"""Orchestration on the GPU, through the C ABI: a MACE iteration replayed as a
CUDA graph, a batch of uneven problems in one captured graph, and the projector
autotuner.  All three reorganise launches without changing any kernel's
arithmetic or summation order, so they must reproduce the eager path bit for bit."""
import dataclasses

import numpy as np
import pytest

from paper_2008_01567_gb300 import synth
from tests._problems import I0

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_2008_01567_gb300 import build, msf
    build.build()
    assert torch.cuda.is_available()
    return msf


def _problem(M, scan, seed, prior, cnn_params=None):
    """Everything one MACE problem owns: plan, data, state, agents."""
    import torch
    P = M.Projector(scan)
    ell = synth.ellipsoids(seed, 3, scan)
    p = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    M.msf_phantom_project(P, ell, p)
    counts = torch.from_numpy(synth.poisson(seed + 1, I0 * np.exp(-p.cpu().numpy().astype(np.float64)))
                              .astype(np.float32)).cuda()
    y, lam = torch.empty_like(counts), torch.empty_like(counts)
    M.msf_weights(counts, y, lam, I0, I0)
    K1 = 4 if prior == M.MSF_PRIOR_CNN else 2
    W = torch.zeros((K1, scan.nt, scan.n, scan.n, scan.n), device="cuda")
    X = torch.zeros_like(W)
    cnn = None
    if prior == M.MSF_PRIOR_CNN:
        cnn = M.Cnn(scan.n ** 3)
        cnn.set_params(cnn_params)
        m = M.Mace(P, W, X, y, lam, prior, cnn=cnn)
    else:
        m = M.Mace(P, W, X, y, lam, prior, mrf=M.msf_mrf(2.0, 1.2, 1.0, 0.1, 0.5))
    return dict(P=P, W=W, X=X, y=y, lam=lam, cnn=cnn, m=m, K1=K1)


def _params(M, K1, rho=0.8, graph=False):
    mu = [0.25] * 4 if K1 == 4 else [0.25, 0.75]
    return M.mace_params(rho, 0.2, mu, 3, 1, graph)


def test_graph_step_matches_eager(M):
    import torch
    flat = M.pack_params(*synth.cnn_weights(91))
    scan = synth.Scan(n=20, nt=5, nu=28, nv=24, views=8)
    a = _problem(M, scan, 92, M.MSF_PRIOR_CNN, flat)
    b = _problem(M, scan, 92, M.MSF_PRIOR_CNN, flat)
    for it in range(4):
        rho = 0.8 if it < 2 else 0.6          # a parameter change forces a new capture
        ra = M.msf_mace_step(a["m"], rho, 0.2, [0.25] * 4, 3)
        rb = M.msf_mace_step(b["m"], rho, 0.2, [0.25] * 4, 3, use_graph=True)
        assert ra == rb
    torch.cuda.synchronize()
    assert torch.equal(a["W"], b["W"]) and torch.equal(a["X"], b["X"])


def test_graph_is_recaptured_after_a_tuning_change(M):
    # the CG's partial sums follow the gather's z-run, so a graph that kept the
    # old launch shapes would drift from the eager steps in the last bits
    import torch
    flat = M.pack_params(*synth.cnn_weights(96))
    scan = synth.Scan(n=20, nt=5, nu=28, nv=24, views=8)
    a = _problem(M, scan, 97, M.MSF_PRIOR_CNN, flat)
    b = _problem(M, scan, 97, M.MSF_PRIOR_CNN, flat)
    for it in range(4):
        if it == 2:
            for q in (a, b):
                M.msf_projector_set_tuning(q["P"], 16, 8, 8)
        ra = M.msf_mace_step(a["m"], 0.8, 0.2, [0.25] * 4, 3)
        rb = M.msf_mace_step(b["m"], 0.8, 0.2, [0.25] * 4, 3, use_graph=True)
        assert ra == rb, it
    torch.cuda.synchronize()
    assert torch.equal(a["W"], b["W"]) and torch.equal(a["X"], b["X"])


def test_batch_of_uneven_problems_matches_individual_steps(M):
    import torch
    flat = M.pack_params(*synth.cnn_weights(93))
    scans = [synth.Scan(n=16, nt=4, nu=24, nv=24, views=6),
             synth.Scan(n=24, nt=5, nu=36, nv=28, views=9, mode="wedge90"),
             synth.Scan(n=32, nt=6, nu=44, nv=36, views=12)]
    priors = [M.MSF_PRIOR_CNN, M.MSF_PRIOR_QGGMRF, M.MSF_PRIOR_CNN]
    solo = [_problem(M, s, 94 + i, p, flat) for i, (s, p) in enumerate(zip(scans, priors))]
    batch = [_problem(M, s, 94 + i, p, flat) for i, (s, p) in enumerate(zip(scans, priors))]
    B = M.MaceBatch([q["m"] for q in batch])
    for it in range(3):
        res_solo = [M.msf_mace_step(q["m"], 0.8, 0.2, [0.25] * 4 if q["K1"] == 4 else [0.25, 0.75], 3, 1)
                    for q in solo]
        res_b = M.msf_mace_batch_step(B, [_params(M, q["K1"], graph=True) for q in batch])
        assert res_solo == res_b
    torch.cuda.synchronize()
    for q, r in zip(solo, batch):
        assert torch.equal(q["W"], r["W"]) and torch.equal(q["X"], r["X"])
    # eager batch (no graph) gives the same answer too
    res_e = M.msf_mace_batch_step(B, [_params(M, q["K1"], graph=False) for q in batch])
    res_s = [M.msf_mace_step(q["m"], 0.8, 0.2, [0.25] * 4 if q["K1"] == 4 else [0.25, 0.75], 3, 1) for q in solo]
    assert res_e == res_s


def test_batch_rejects_shared_workspaces(M):
    flat = M.pack_params(*synth.cnn_weights(95))
    scan = synth.Scan(n=16, nt=4, nu=24, nv=24, views=6)
    a = _problem(M, scan, 96, M.MSF_PRIOR_QGGMRF)
    with pytest.raises(M.MsfError):
        M.MaceBatch([a["m"], a["m"]])


def test_autotune_keeps_results(M):
    import torch
    scan = dataclasses.replace(synth.PROJ, nt=2)
    P = M.Projector(scan)
    x = torch.empty((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    M.msf_phantom_voxelize(P.vol, synth.ellipsoids(97, 4, scan), x, ss=1)
    e = torch.rand((scan.nt, scan.views, scan.nv, scan.nu), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    y0, b0 = torch.empty_like(e), torch.empty_like(x)
    M.msf_project(P, x, y0)
    M.msf_backproject(P, e, b0)
    choice = M.msf_projector_autotune(P)
    assert choice[0] * choice[1] == 128 and choice[2] in (8, 16, 32)
    y1, b1 = torch.empty_like(e), torch.empty_like(x)
    M.msf_project(P, x, y1)
    M.msf_backproject(P, e, b1)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1) and torch.equal(b0, b1)


def test_every_launch_shape_gives_the_same_results(M):
    # the forward's ray blocks and the adjoint's z-run lengths only reorganise
    # the launch: each ray keeps its arithmetic and each voxel its summation
    # order, so all twelve configurations agree bit for bit (a ragged volume, so
    # that runs and blocks end inside the grid)
    import torch
    scan = synth.Scan(n=44, nt=3, nu=61, nv=47, views=7)
    P = M.Projector(scan)
    x = torch.empty((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    M.msf_phantom_voxelize(P.vol, synth.ellipsoids(98, 4, scan), x, ss=1)
    e = torch.rand((scan.nt, scan.views, scan.nv, scan.nu), device="cuda",
                   generator=torch.Generator("cuda").manual_seed(2))
    ref_y = ref_b = None
    for cols, rows in ((32, 4), (64, 2), (16, 8)):
        for zrun in (8, 16, 32, 64):
            M.msf_projector_set_tuning(P, cols, rows, zrun)
            y, b = torch.empty_like(e), torch.empty_like(x)
            M.msf_project(P, x, y)
            M.msf_backproject(P, e, b)
            torch.cuda.synchronize()
            if ref_y is None:
                ref_y, ref_b = y, b
            assert torch.equal(y, ref_y) and torch.equal(b, ref_b), (cols, rows, zrun)
    with pytest.raises(M.MsfError):
        M.msf_projector_set_tuning(P, 128, 1, 16)
    with pytest.raises(M.MsfError):
        M.msf_projector_set_tuning(P, 32, 4, 12)


def test_autotuner_offers_long_gather_runs_only_for_deep_grids(M):
    # 64-voxel gather runs halve the adjoint's block count; a small plan's grid
    # is only a few waves deep, so its autotuner must not pick them (in a batch
    # of concurrent problems they measured slower although they won alone)
    scan = synth.Scan(n=64, nt=4, nu=96, nv=96, views=16)
    P = M.Projector(scan)
    cols, rows, zrun = M.msf_projector_autotune(P)
    assert zrun in (8, 16, 32), zrun
    assert (cols, rows) in ((32, 4), (64, 2), (16, 8))


def test_denoise_batch_equals_single_problems(M):
    # uneven problems through the multi-problem persistent launches: (16^3 x 4),
    # (24 x 32 x 40 x 6) and (32^3 x 3) run together; an odd height (21^3) and a
    # handle too small for one chunk run on their own inside the same call
    import torch
    flat = M.pack_params(*synth.cnn_weights(97))
    shapes = [(4, 16, 16, 16), (6, 24, 32, 40), (3, 21, 21, 21), (3, 32, 32, 32), (5, 16, 16, 16)]
    small = [False, False, False, False, True]
    cnns, vols, xs = [], [], []
    for i, (sh, sm) in enumerate(zip(shapes, small)):
        nt, nz, ny, nx = sh
        c = M.Cnn(nz * ny * nx * (1 if sm else nt))
        c.set_params(flat)
        cnns.append(c)
        vols.append(M.msf_vol(nx, ny, nz, nt, 1.0))
        xs.append(torch.rand(sh, device="cuda", generator=torch.Generator("cuda").manual_seed(100 + i)))
    for o in range(3):
        outs = [torch.full_like(x, -5.0) for x in xs]
        M.msf_denoise_batch(cnns, o, vols, xs, outs)
        for c, v, x, out in zip(cnns, vols, xs, outs):
            ref = torch.empty_like(x)
            M.msf_denoise(c, o, v, x, ref)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), o


def test_batch_with_shared_cnn_matches_individual_steps(M):
    # every problem runs the three CNN agents with the same parameters: the
    # batch takes the multi-problem path and must still equal the single steps
    import torch
    flat = M.pack_params(*synth.cnn_weights(98))
    scans = [synth.Scan(n=16, nt=4, nu=24, nv=24, views=6),
             synth.Scan(n=24, nt=5, nu=36, nv=28, views=9, mode="wedge90"),
             synth.Scan(n=32, nt=3, nu=44, nv=36, views=12)]

    def make(i, s):
        q = _problem(M, s, 99 + i, M.MSF_PRIOR_CNN, flat)
        q["m"].close()
        q["cnn"].close()
        q["cnn"] = M.Cnn(s.nt * s.n ** 3)        # room for every time-point
        q["cnn"].set_params(flat)
        q["m"] = M.Mace(q["P"], q["W"], q["X"], q["y"], q["lam"], M.MSF_PRIOR_CNN, cnn=q["cnn"])
        return q

    solo = [make(i, s) for i, s in enumerate(scans)]
    batch = [make(i, s) for i, s in enumerate(scans)]
    B = M.MaceBatch([q["m"] for q in batch])
    for it in range(3):
        graph = it > 0
        res_solo = [M.msf_mace_step(q["m"], 0.8, 0.2, [0.25] * 4, 3) for q in solo]
        res_b = M.msf_mace_batch_step(B, [_params(M, 4, graph=graph) for _ in batch])
        assert res_solo == res_b, it
    torch.cuda.synchronize()
    for q, r in zip(solo, batch):
        assert torch.equal(q["W"], r["W"]) and torch.equal(q["X"], r["X"])
