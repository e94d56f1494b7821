"""GPU parity of the proximal agents against the FP64 oracle, through the C ABI.

Tolerances, derived from the arithmetic:
  * CG data prox L~ (Eq. (13)): each CG iteration applies A and A^T, whose FP32
    error is bounded by the projector tolerance 1e-5; vectors are FP32 and the
    scalars FP64.  Over n_cg iterations the deviations add (CG on an SPD system
    with a fixed iteration count is a smooth map of its inputs), so the bound
    used is 2 * n_cg * 1e-5 relative L2.
  * q-GGMRF ICD: every update is a convex combination of v and 28 neighbours
    evaluated in FP32 (about 30 roundings of 6e-8); a sweep is a contraction, so
    the deviation stays below n_sweeps * 30 * 6e-8 ~ 2e-6 * n_sweeps; 1e-5 is
    used for up to 4 sweeps.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2008_01567_gb300 import synth
from tests._problems import I0, f32, measurement, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_2008_01567_gb300 import build, msf
    build.build()
    assert torch.cuda.is_available()
    return msf


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("scan,n_cg", [(synth.TINY, 5),
                                        (synth.Scan(n=40, nt=2, nu=45, nv=37, views=5, mode="wedge90"), 10)],
                         ids=["tiny", "ragged-wedge"])
def test_cg_prox_matches_oracle(M, scan, n_cg):
    x0, counts, y, lam = measurement(scan, 31)
    sigma = 0.1
    v = f32(x0 + synth.normal(32, x0.shape, 0.05))
    z0 = f32(0.5 * x0)
    P = M.Projector(scan)
    dp = M.DataProx(P)
    c = _t(counts)
    yg, lg = _t(np.zeros_like(counts)), _t(np.zeros_like(counts))
    M.msf_weights(c, yg, lg, I0, I0)
    z = _t(z0)
    M.msf_prox_data(dp, yg, lg, _t(v), z, sigma, n_cg)
    got = z.cpu().numpy()
    ref = oracle.prox_data(f32(y), f32(lam), v, z0, scan, sigma, n_cg)
    assert rel_l2(got, ref) <= 2 * n_cg * 1e-5
    # the prox moved the iterate: the comparison is not trivial
    assert rel_l2(z0, ref) > 1e-2


@pytest.mark.parametrize("scan", [synth.PROJ, synth.PROJ_WEDGE], ids=["sparse360", "wedge90"])
def test_cg_prox_projector_workload_frames(M, scan):
    # the projector workload (128^3 x 8, 192 x 160 detector, 32 views per
    # time-point, both protocols) with 10 CG iterations: the GPU solves all
    # eight frames in its production launch shapes (the CG partial sums and
    # z-runs at their full-size grids); the oracle solves the first and the
    # last frame on its own (the solves are independent per frame)
    n_cg, sigma = 10, 0.1
    x0, counts, y, lam = measurement(scan, 36)
    v = f32(x0 + synth.normal(37, x0.shape, 0.05))
    z0 = f32(0.5 * x0)
    P = M.Projector(scan)
    M.msf_projector_autotune(P)
    dp = M.DataProx(P)
    c = _t(counts)
    yg, lg = _t(np.zeros_like(counts)), _t(np.zeros_like(counts))
    M.msf_weights(c, yg, lg, I0, I0)
    z = _t(z0)
    M.msf_prox_data(dp, yg, lg, _t(v), z, sigma, n_cg)
    got = z.cpu().numpy()
    ang = scan.angles()
    yf, lf = f32(y), f32(lam)
    for t in (0, scan.nt - 1):
        ref = oracle.prox_data_frame(yf[t], lf[t], v[t], z0[t], scan, ang[t], sigma, n_cg)
        assert rel_l2(got[t], ref) <= 2 * n_cg * 1e-5, t
        assert rel_l2(z0[t], ref) > 1e-2


def test_cg_zero_iterations_is_identity(M):
    scan = synth.TINY
    P = M.Projector(scan)
    dp = M.DataProx(P)
    z0 = synth.uniform(33, (scan.nt, scan.n, scan.n, scan.n))
    z = _t(z0)
    s = _t(np.ones((scan.nt, scan.views, scan.nv, scan.nu)))
    M.msf_prox_data(dp, s, s, _t(z0), z, 0.1, 0)
    np.testing.assert_array_equal(z.cpu().numpy(), z0.astype(np.float32))


@pytest.mark.parametrize("q", [2.0, 1.2])
def test_qggmrf_matches_oracle(M, q):
    shape = (5, 21, 29, 37)   # [nt][nz][ny][nx], odd sizes: ragged colour grids
    v = f32(synth.uniform(34, shape, 0.0, 2.0))
    z0 = f32(synth.uniform(35, shape, 0.0, 2.0))
    sigma, T, sx, bt, n = 0.2, 1.0, 0.15, 0.5, 4
    vol = M.msf_vol(shape[3], shape[2], shape[1], shape[0], 1.0)
    mrf = M.msf_mrf(2.0, q, T, sx, bt)
    z = _t(z0)
    M.msf_prox_qggmrf(vol, mrf, _t(v), z, sigma, n)
    ref = oracle.prox_qggmrf(v, z0, sigma, 2.0, q, T, sx, bt, n)
    assert rel_l2(z.cpu().numpy(), ref) <= 1e-5
    assert rel_l2(z0, ref) > 1e-2


def test_qggmrf_single_voxel_and_frame(M):
    # no neighbours: H(v) = v
    vol = M.msf_vol(1, 1, 1, 1, 1.0)
    mrf = M.msf_mrf(2.0, 1.2, 1.0, 0.3, 0.5)
    z = _t(np.zeros((1, 1, 1, 1)))
    M.msf_prox_qggmrf(vol, mrf, _t(np.full((1, 1, 1, 1), 0.625)), z, 0.1, 3)
    assert z.item() == 0.625
