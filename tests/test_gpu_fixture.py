"""GPU parity of the blind fixture correction (Appendix A, Algorithm 2) against
the FP64 oracle, through the C ABI.

Tolerance, from the arithmetic: y^corr = y - c p where p is a normalised
Gaussian blur (FP32 sums of at most 2 * (2R + 1) terms, ~1e-6) of e = y - A x^m
(the projector's 1e-5 bound on A x^m), and c is an FP64 ratio of sums of those
terms; every quantity therefore carries the projector's 1e-5 relative error,
held here to 1e-5 relative L2 on the correction c p and to 1e-5 on c."""
import numpy as np
import pytest

import oracle
from paper_2008_01567_gb300 import synth
from tests._problems import f32, rel_l2

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


def _fixture_shadow(sc, amp=0.6):
    vv, uu = np.meshgrid(np.arange(sc.nv), np.arange(sc.nu), indexing="ij")
    f = np.zeros((sc.nt, sc.views, sc.nv, sc.nu))
    for t in range(sc.nt):
        for j in range(sc.views):
            f[t, j] = amp * np.exp(-((uu - 0.15 * sc.nu - 0.1 * sc.nu * j) ** 2) / (0.05 * sc.nu ** 2)
                                   - ((vv - 0.5 * sc.nv) ** 2) / (0.3 * sc.nv ** 2))
    return f


@pytest.mark.parametrize("scan,sigma_px", [(synth.Scan(n=24, nt=3, nu=33, nv=27, views=6), 2.0),
                                           (synth.Scan(n=40, nt=2, nu=45, nv=37, views=5, mode="wedge90"), 3.5)],
                         ids=["small", "ragged-wedge"])
def test_fixture_correction_matches_oracle(M, scan, sigma_px):
    import torch
    ell = synth.ellipsoids(91, 3, scan, axis_range=(0.08, 0.15))
    ell[:, :, 0:2] *= 0.5
    x = f32(oracle.ellipsoid_volume(ell, scan, ss=2))
    # a reconstruction with errors, and measurements with a fixture shadow
    xr = f32(x + synth.normal(92, x.shape, 0.02))
    y = f32(oracle.project4d(x, scan) + _fixture_shadow(scan) + synth.normal(93, (scan.nt, scan.views, scan.nv,
                                                                                  scan.nu), 0.01))
    P = M.Projector(scan)
    fc = M.FixtureCorrector(P)
    yc = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    for _ in range(2):          # twice in a row: the workspace is reused
        c = M.msf_fixture_correct(fc, _t(y), _t(xr), 0.4, sigma_px, yc)
        ref, c_ref = oracle.fixture_correct(y, xr, scan, 0.4, sigma_px)
        got = yc.cpu().numpy().astype(np.float64)
        assert c == pytest.approx(c_ref, rel=1e-5)
        assert rel_l2(y - got, y - ref) <= 1e-5
        assert c_ref > 0.5          # the shadow is found


def test_fixture_correction_argument_errors(M):
    import torch
    scan = synth.Scan(n=8, nt=1, nu=12, nv=10, views=2)
    P = M.Projector(scan)
    fc = M.FixtureCorrector(P)
    y = torch.zeros((1, 2, 10, 12), device="cuda")
    x = torch.zeros((1, 8, 8, 8), device="cuda")
    with pytest.raises(M.MsfError):
        M.msf_fixture_correct(fc, y, x, 0.4, 30.0, torch.zeros_like(y))    # blur radius beyond 64 taps
    with pytest.raises(M.MsfError):
        M.msf_fixture_correct(fc, y, x, -1.0, 2.0, torch.zeros_like(y))
