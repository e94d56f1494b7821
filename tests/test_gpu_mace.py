"""GPU parity of the MACE iteration (Sec. III, Algorithm 1) against the FP64
oracle on the tiny plain-method workload (24^3 x 4, 32x32 detector, 12 views
per frame interlaced over 360 deg, Poisson noise at 1e4 photons, rho 0.5,
CG data prox with 5 iterations, sigma 0.1, q-GGMRF p=2 q=1.2, 10 iterations).

Tolerance: the Mann iteration with rho in (0,1) is nonexpansive for proximal
agents, so per-iteration agent deviations (<= 1e-4 for 5 CG steps, see
test_gpu_prox) add up without amplification: 10 iterations -> 1e-3."""
import numpy as np
import pytest

import oracle
from paper_2008_01567_gb300 import synth
from tests._problems import I0, f32, measurement, rel_l2

pytestmark = pytest.mark.gpu

SX, BT, N_SWEEPS = 0.2, 0.5, 2


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


def test_plain_mace_matches_oracle(M):
    import torch
    scan = synth.TINY
    x0, counts, y, lam = measurement(scan, 41)
    sigma, rho, n_cg, iters = 0.1, 0.5, 5, 10
    mu = [0.5, 0.5]
    P = M.Projector(scan)
    c = _t(counts)
    yg = torch.empty_like(c)
    lg = torch.empty_like(c)
    M.msf_weights(c, yg, lg, I0, I0)
    shape = (2, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    mrf = M.msf_mrf(2.0, 1.2, 1.0, SX, BT)
    m = M.Mace(P, W, X, yg, lg, M.MSF_PRIOR_QGGMRF, mrf=mrf)
    res_gpu = [M.msf_mace_step(m, rho, sigma, mu, n_cg, N_SWEEPS) for _ in range(iters)]
    yf, lf = f32(y), f32(lam)
    agents = [lambda w, x: oracle.prox_data(yf, lf, w, x, scan, sigma, n_cg),
              lambda w, x: oracle.prox_qggmrf(w, x, sigma, 2.0, 1.2, 1.0, SX, BT, N_SWEEPS)]
    xhat, Wo, Xo, res = oracle.mace(np.zeros(shape[1:]), agents, mu, rho, iters)
    assert rel_l2(X[0].cpu().numpy(), xhat) <= 1e-3
    assert rel_l2(W.cpu().numpy(), np.stack(Wo)) <= 1e-3
    np.testing.assert_allclose(res_gpu, res, rtol=1e-3)
    # the reconstruction approaches the phantom
    assert rel_l2(X[0].cpu().numpy(), x0) < 0.6


def test_mace_argument_errors(M):
    import torch
    scan = synth.TINY
    P = M.Projector(scan)
    shape = (2, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    s = torch.ones((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    m = M.Mace(P, W, X, s, s, M.MSF_PRIOR_QGGMRF, mrf=M.msf_mrf(2.0, 1.2, 1.0, SX, BT))
    for rho, mu in ((1.0, [0.5, 0.5]), (0.5, [0.6, 0.5]), (0.0, [0.5, 0.5])):
        with pytest.raises(M.MsfError) as e:
            M.msf_mace_step(m, rho, 0.1, mu, 1, 1)
        assert e.value.status == 1
