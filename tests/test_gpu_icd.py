"""GPU parity of the grouped-ICD data agent L~ (Sec. III, Eq. (13) with the
cost of Eq. (4)) against the FP64 oracle, through the C ABI.

Tolerance, from the arithmetic: every group step gathers A^T Lambda e over the
group (one partial A^T) and projects the group's update (one A); both carry
the projector's FP32 error bound of 1e-5, and the step scalars are FP64.  Over
n_sweeps sweeps of eight groups the deviations add, so the bound used is
2 * 8 * n_sweeps * 1e-5 relative L2 (the CG agent's bound, per A/A^T pair)."""
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


def _setup(M, scan, seed):
    x0, counts, y, lam = measurement(scan, seed)
    P = M.Projector(scan)
    dp = M.DataProx(P)
    c = _t(counts)
    yg, lg = _t(np.zeros_like(counts)), _t(np.zeros_like(counts))
    M.msf_weights(c, yg, lg, I0, I0)
    return x0, f32(y), f32(lam), P, dp, yg, lg


RAGGED_WEDGE = synth.Scan(n=40, nt=2, nu=45, nv=37, views=5, mode="wedge90")
ODD = synth.Scan(n=21, nt=3, nu=29, nv=23, views=7)   # odd sizes: groups of unequal size


@pytest.mark.parametrize("scan,n_sweeps", [(synth.TINY, 3), (RAGGED_WEDGE, 3), (ODD, 2)],
                         ids=["tiny", "ragged-wedge", "odd"])
def test_icd_prox_matches_oracle(M, scan, n_sweeps):
    sigma = 0.1
    x0, y, lam, P, dp, yg, lg = _setup(M, scan, 41)
    v = f32(x0 + synth.normal(42, x0.shape, 0.05))
    z0 = f32(0.5 * x0)
    z = _t(z0)
    M.msf_prox_data_icd(dp, yg, lg, _t(v), z, sigma, n_sweeps)
    got = z.cpu().numpy()
    ref = oracle.prox_data_icd(y, lam, v, z0, scan, sigma, n_sweeps)
    assert rel_l2(got, ref) <= 2 * 8 * n_sweeps * 1e-5
    assert rel_l2(z0, ref) > 1e-2
    # and the GPU result lowers the cost of Eq. (4) in every frame
    ang = scan.angles()
    for t in range(scan.nt):
        c0 = oracle.data_cost(y[t], lam[t], v[t], z0[t], scan, ang[t], sigma)
        c1 = oracle.data_cost(y[t], lam[t], v[t], got[t].astype(np.float64), scan, ang[t], sigma)
        assert c1 < c0


def test_icd_zero_sweeps_is_identity(M):
    scan = synth.TINY
    P = M.Projector(scan)
    dp = M.DataProx(P)
    z0 = synth.uniform(43, (scan.nt, scan.n, scan.n, scan.n))
    z = _t(z0)
    s = _t(np.ones((scan.nt, scan.views, scan.nv, scan.nu)))
    M.msf_prox_data_icd(dp, s, s, _t(z0), z, 0.1, 0)
    np.testing.assert_array_equal(z.cpu().numpy(), z0.astype(np.float32))


def test_icd_repeatable_and_shares_workspace_with_cg(M):
    # the same call twice gives the same bits; a CG call in between (same
    # workspace) does not disturb it
    scan = synth.TINY
    x0, y, lam, P, dp, yg, lg = _setup(M, scan, 44)
    v = _t(x0)
    outs = []
    for k in range(2):
        z = _t(0.3 * x0)
        M.msf_prox_data_icd(dp, yg, lg, v, z, 0.1, 2)
        outs.append(z.cpu().numpy())
        z2 = _t(0.3 * x0)
        M.msf_prox_data(dp, yg, lg, v, z2, 0.1, 3)
    np.testing.assert_array_equal(outs[0], outs[1])


def test_mace_with_icd_data_agent_matches_oracle(M):
    # plain MACE (q-GGMRF prior) with the ICD data agent: Algorithm 1 with
    # L~ = 2 grouped-ICD sweeps, 4 iterations, against the oracle's loop
    import torch
    scan = synth.TINY
    x0, y, lam, P, dp, yg, lg = _setup(M, scan, 45)
    shape = (2, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    mrf = M.msf_mrf(2.0, 1.2, 1.0, 0.2, 0.5)
    m = M.Mace(P, W, X, yg, lg, M.MSF_PRIOR_QGGMRF, mrf=mrf)
    sigma, rho, n_icd, n_sw, mu, iters = 0.1, 0.5, 2, 1, [0.5, 0.5], 4
    for _ in range(iters):
        r = M.msf_mace_step(m, rho, sigma, mu, 0, n_sw, n_icd=n_icd)
    assert np.isfinite(r)
    agents = [lambda w, x: oracle.prox_data_icd(y, lam, w, x, scan, sigma, n_icd),
              lambda w, x: oracle.prox_qggmrf(w, x, sigma, 2.0, 1.2, 1.0, 0.2, 0.5, n_sw)]
    xhat, _, _, _ = oracle.mace(np.zeros(shape[1:]), agents, mu, rho, iters)
    assert rel_l2(X[0].cpu().numpy(), xhat) <= 1e-3


def test_mace_with_icd_graph_equals_eager(M):
    # the ICD data agent inside a captured MACE iteration: same bits as eager
    import torch
    scan = synth.TINY
    x0, y, lam, P1, dp, yg, lg = _setup(M, scan, 46)
    P2 = M.Projector(scan)
    shape = (2, scan.nt, scan.n, scan.n, scan.n)
    mrf = M.msf_mrf(2.0, 1.2, 1.0, 0.2, 0.5)
    Wa, Xa = torch.zeros(shape, device="cuda"), torch.zeros(shape, device="cuda")
    Wb, Xb = torch.zeros(shape, device="cuda"), torch.zeros(shape, device="cuda")
    ma = M.Mace(P1, Wa, Xa, yg, lg, M.MSF_PRIOR_QGGMRF, mrf=mrf)
    mb = M.Mace(P2, Wb, Xb, yg, lg, M.MSF_PRIOR_QGGMRF, mrf=mrf)
    for it in range(3):
        ra = M.msf_mace_step(ma, 0.5, 0.1, [0.5, 0.5], 0, 1, n_icd=2)
        rb = M.msf_mace_step(mb, 0.5, 0.1, [0.5, 0.5], 0, 1, n_icd=2, use_graph=True)
        assert ra == rb
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xb) and torch.equal(Wa, Wb)
