"""GPU parity of the direct MAP solve (the MBIR + 4D-MRF comparison of Sec. VI:
Eq. (3) with the 4D q-GGMRF prior, by majorise-minimise with CG) against the
FP64 oracle, through the C ABI.

Tolerance, from the arithmetic: every CG step applies A and A^T (FP32, 1e-5
each) and the surrogate Laplacian (FP32 sums of 28 terms, about 1e-6); the
scalars are FP64.  Over n_outer * (n_cg + 1) such steps the deviations add:
2 * n_outer * (n_cg + 1) * 1e-5 relative L2.  The cost is an FP64 sum of FP32
terms: 1e-5 relative."""
import numpy as np
import pytest

import oracle
from paper_2008_01567_gb300 import synth
from tests._problems import I0, f32, measurement, rel_l2

pytestmark = pytest.mark.gpu
PRIOR = dict(p=2.0, q=1.2, T=1.0, sx=0.2, bt=0.5)


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


def _problem(M, scan, seed):
    x0, counts, y, lam = measurement(scan, seed)
    P = M.Projector(scan)
    c = _t(counts)
    yg, lg = _t(np.zeros_like(counts)), _t(np.zeros_like(counts))
    M.msf_weights(c, yg, lg, I0, I0)
    return x0, f32(y), f32(lam), P, yg, lg


@pytest.mark.parametrize("scan", [synth.TINY, synth.Scan(n=21, nt=3, nu=29, nv=23, views=7, mode="wedge90")],
                         ids=["tiny", "odd-wedge"])
def test_map_solve_matches_oracle(M, scan):
    n_outer, n_cg, beta = 3, 4, 3.0
    x0, y, lam, P, yg, lg = _problem(M, scan, 51)
    pr = PRIOR
    mrf = M.msf_mrf(pr["p"], pr["q"], pr["T"], pr["sx"], pr["bt"])
    ms = M.MapSolver(P)
    xs = f32(0.5 * x0)
    x = _t(xs)
    M.msf_map_solve(ms, mrf, beta, yg, lg, x, n_outer, n_cg)
    got = x.cpu().numpy()
    ref = oracle.map_mm(y, lam, xs, scan, pr["p"], pr["q"], pr["T"], pr["sx"], pr["bt"], beta, n_outer, n_cg)
    assert rel_l2(got, ref) <= 2 * n_outer * (n_cg + 1) * 1e-5
    assert rel_l2(xs, ref) > 1e-2
    # the cost on the GPU against the oracle's, at the start and at the result
    for v in (xs, got.astype(np.float64)):
        c_gpu = M.msf_map_cost(ms, mrf, beta, yg, lg, _t(v))
        c_ref = oracle.map_cost(y, lam, f32(v), scan, pr["p"], pr["q"], pr["T"], pr["sx"], pr["bt"], beta)
        assert abs(c_gpu - c_ref) <= 1e-5 * abs(c_ref)


def test_map_cost_descends_on_gpu(M):
    scan = synth.TINY
    x0, y, lam, P, yg, lg = _problem(M, scan, 52)
    pr = PRIOR
    mrf = M.msf_mrf(pr["p"], pr["q"], pr["T"], pr["sx"], pr["bt"])
    ms = M.MapSolver(P)
    import torch
    x = torch.zeros((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    prev = M.msf_map_cost(ms, mrf, 3.0, yg, lg, x)
    for _ in range(8):
        M.msf_map_solve(ms, mrf, 3.0, yg, lg, x, 1, 5)
        c = M.msf_map_cost(ms, mrf, 3.0, yg, lg, x)
        assert c < prev
        prev = c


def test_map_argument_errors(M):
    scan = synth.TINY
    P = M.Projector(scan)
    ms = M.MapSolver(P)
    import torch
    x = torch.zeros((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    y = torch.zeros((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    with pytest.raises(M.MsfError) as e:
        M.msf_map_solve(ms, M.msf_mrf(1.5, 1.2, 1.0, 0.2, 0.5), 3.0, y, y, x, 1, 1)
    assert e.value.status == 1
    with pytest.raises(M.MsfError):
        M.msf_map_solve(ms, M.msf_mrf(2.0, 1.2, 1.0, 0.2, 0.5), -1.0, y, y, x, 1, 1)
