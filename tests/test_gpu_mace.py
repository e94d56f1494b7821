"""GPU parity of the MACE iteration (Sec. III, Algorithm 1) against the FP64
oracle.  Plain method on the tiny plain-method workload (24^3 x 4, 32x32 detector, 12 views
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


@pytest.mark.parametrize("mode", ["sparse360", "wedge90"])
def test_plain_mace_matches_oracle(M, mode):
    # sparse-view (views interlaced over 360 deg) and limited-angle (each
    # time-point a 90-deg wedge of a continuous rotation) scans of Sec. VI
    import dataclasses
    import torch
    scan = dataclasses.replace(synth.TINY, mode=mode)
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


def _cnn_net(seed):
    rng = np.random.default_rng(seed)
    convs, bns = synth.cnn_weights(seed)
    convs = [(w, rng.normal(0, 0.02, b.shape)) for w, b in convs]
    bns = [(g, rng.normal(0, 0.05, g.shape)) for g, _ in bns]
    stats = [(rng.normal(0, 0.05, 64), rng.uniform(0.5, 2.0, 64)) for _ in bns]
    return convs, bns, stats


def test_learned_mace_matches_oracle(M):
    # Multi-slice fusion: the data agent plus H_xy,t, H_yz,t, H_zx,t sharing one
    # network (Eq. (14)), equal weights 0.25, rho 0.8.  Per-iteration deviation:
    # CG <= 1e-4 and the BF16 CNN agents <= 1e-2 of their residual R (test_gpu_cnn),
    # R being ~10% of the state here; 3 iterations -> bound 1e-2.
    import torch
    scan = synth.TINY
    x0, counts, y, lam = measurement(scan, 43)
    sigma, rho, n_cg, iters = 0.1, 0.8, 5, 3
    mu = [0.25] * 4
    convs, bns, stats = _cnn_net(44)
    cnn = M.Cnn(scan.n ** 3)
    flat = M.pack_params(convs, bns, stats)
    cnn.set_params(flat)
    cv, bv, sv = M.unpack_params(flat)
    layers = oracle.fold_bn(cv, bv, sv)
    P = M.Projector(scan)
    c = _t(counts)
    yg, lg = torch.empty_like(c), torch.empty_like(c)
    M.msf_weights(c, yg, lg, I0, I0)
    shape = (4, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    m = M.Mace(P, W, X, yg, lg, M.MSF_PRIOR_CNN, cnn=cnn)
    res_gpu = [M.msf_mace_step(m, rho, sigma, mu, n_cg) for _ in range(iters)]
    yf, lf = f32(y), f32(lam)
    agents = [lambda w, x: oracle.prox_data(yf, lf, w, x, scan, sigma, n_cg)]
    for o in oracle.ORIENTS:
        agents.append(lambda w, x, o=o: oracle.denoise(w, layers, o, emulate_bf16=True))
    xhat, Wo, Xo, res = oracle.mace(np.zeros(shape[1:]), agents, mu, rho, iters)
    assert rel_l2(X[0].cpu().numpy(), xhat) <= 1e-2
    assert rel_l2(W.cpu().numpy(), np.stack(Wo)) <= 1e-2
    np.testing.assert_allclose(res_gpu, res, rtol=2e-2)


@pytest.mark.parametrize("orient", [0, 2])
def test_single_cnn_pnp_matches_oracle(M, orient):
    # The "MBIR + H" comparison of Sec. VI: the data agent and one CNN prior of
    # one orientation (K = 1), weights 0.5 / 0.5 (beta = 1).  Same bound as the
    # three-agent case.
    import torch
    scan = synth.TINY
    x0, counts, y, lam = measurement(scan, 45)
    sigma, rho, n_cg, iters = 0.1, 0.8, 5, 3
    mu = [0.5, 0.5]
    convs, bns, stats = _cnn_net(46)
    cnn = M.Cnn(scan.n ** 3)
    flat = M.pack_params(convs, bns, stats)
    cnn.set_params(flat)
    layers = oracle.fold_bn(*M.unpack_params(flat))
    P = M.Projector(scan)
    c = _t(counts)
    yg, lg = torch.empty_like(c), torch.empty_like(c)
    M.msf_weights(c, yg, lg, I0, I0)
    shape = (2, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    m = M.Mace(P, W, X, yg, lg, M.MSF_PRIOR_CNN, cnn=cnn, orient=orient)
    res_gpu = [M.msf_mace_step(m, rho, sigma, mu, n_cg) for _ in range(iters)]
    yf, lf = f32(y), f32(lam)
    o = oracle.ORIENTS[orient]
    agents = [lambda w, x: oracle.prox_data(yf, lf, w, x, scan, sigma, n_cg),
              lambda w, x: oracle.denoise(w, layers, o, emulate_bf16=True)]
    xhat, Wo, Xo, res = oracle.mace(np.zeros(shape[1:]), agents, mu, rho, iters)
    assert rel_l2(X[0].cpu().numpy(), xhat) <= 1e-2
    assert rel_l2(W.cpu().numpy(), np.stack(Wo)) <= 1e-2
    np.testing.assert_allclose(res_gpu, res, rtol=2e-2)


def test_single_cnn_agent_arguments(M):
    import torch
    scan = synth.TINY
    P = M.Projector(scan)
    cnn = M.Cnn(scan.n ** 3)
    y = torch.zeros((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    W = torch.zeros((2, scan.nt, scan.n, scan.n, scan.n), device="cuda")
    X = torch.zeros_like(W)
    with pytest.raises(M.MsfError):
        M.Mace(P, W, X, y, y, M.MSF_PRIOR_CNN, cnn=cnn, orient=3)
    W3 = torch.zeros((3, scan.nt, scan.n, scan.n, scan.n), device="cuda")
    with pytest.raises(M.MsfError):          # K = 2 is neither form
        M.Mace(P, W3, torch.zeros_like(W3), y, y, M.MSF_PRIOR_CNN, cnn=cnn)


def _train(M, cnn, vols, vol, steps, seed, B=32, H=48, W=48, lr=1e-3):
    import torch
    cnn.train_reserve(B * H * W)
    noisy = torch.empty((B, 5, H, W), device="cuda")
    clean = torch.empty((B, H, W), device="cuda")
    for it in range(steps):
        M.msf_training_batch(vols, vol, B, H, W, 0.02, 0.2, seed + it, noisy, clean)
        M.msf_train_step(cnn, noisy, clean, lr, want_loss=False)
    torch.cuda.synchronize()


def test_learned_prior_beats_plain_prior(M):
    # What the trained network gains over the method without it: on a sparse-view
    # 360 deg scan, multi-slice fusion with a CNN trained on the GPU (on other
    # phantoms) reaches a lower NRMSE than MACE with the 4D q-GGMRF prior whose
    # sigma_x is picked from a sweep for its best NRMSE on the same data.
    import torch
    scan = synth.Scan(n=64, nt=6, nu=96, nv=80, views=12)
    I0_ = I0
    P = M.Projector(scan)
    # training phantoms: other seeds, same family
    train_scan = synth.Scan(n=96, nt=6, nu=8, nv=8, views=1)
    Pt = M.Projector(train_scan)
    vols = torch.empty((6, 96, 96, 96), device="cuda")
    M.msf_phantom_voxelize(Pt.vol, synth.ellipsoids(81, 10, train_scan), vols, ss=2)
    cnn = M.Cnn(scan.n ** 3)
    cnn.set_params(M.pack_params(*synth.cnn_weights(82)))
    _train(M, cnn, vols, Pt.vol, 600, 5000)
    # the test problem
    ell = synth.ellipsoids(83, 6, scan)
    x_true = torch.empty((scan.nt, scan.n, scan.n, scan.n), device="cuda")
    M.msf_phantom_voxelize(P.vol, ell, x_true, ss=2)
    p = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
    M.msf_phantom_project(P, ell, p)
    counts = torch.from_numpy(synth.poisson(84, I0_ * np.exp(-p.cpu().numpy().astype(np.float64))).astype(np.float32)).cuda()
    yg, lg = torch.empty_like(counts), torch.empty_like(counts)
    M.msf_weights(counts, yg, lg, I0_, I0_)
    iters, sigma, rho, n_cg = 15, 0.1, 0.8, 5

    def nrmse(x):
        return (torch.linalg.vector_norm(x - x_true) / torch.linalg.vector_norm(x_true)).item()

    shape = (4, scan.nt, scan.n, scan.n, scan.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    m = M.Mace(P, W, X, yg, lg, M.MSF_PRIOR_CNN, cnn=cnn)
    for _ in range(iters):
        M.msf_mace_step(m, rho, sigma, [0.25] * 4, n_cg, want_residual=False)
    learned = nrmse(X[0])
    plain = {}
    for sx in (0.02, 0.05, 0.1, 0.2):
        W2 = torch.zeros((2,) + shape[1:], device="cuda")
        X2 = torch.zeros_like(W2)
        m2 = M.Mace(P, W2, X2, yg, lg, M.MSF_PRIOR_QGGMRF, mrf=M.msf_mrf(2.0, 1.2, 1.0, sx, 0.5))
        for _ in range(iters):
            M.msf_mace_step(m2, rho, sigma, [0.25, 0.75], n_cg, 2, want_residual=False)
        plain[sx] = nrmse(X2[0])
    print(f"NRMSE learned {learned:.4f}  plain {plain}")
    assert learned <= min(plain.values())


def test_counts_from_host_memory_give_the_same_steps(M):
    # msf_mace_set_counts (host counts -> y, Lambda inside the handle) against
    # the same counts conditioned by msf_weights on the device: identical steps
    import torch
    scan = synth.TINY
    x0, counts, y, lam = measurement(scan, 71)
    P1, P2 = M.Projector(scan), M.Projector(scan)
    c_dev = torch.from_numpy(counts.astype(np.float32)).cuda()
    yg, lg = torch.empty_like(c_dev), torch.empty_like(c_dev)
    M.msf_weights(c_dev, yg, lg, I0, I0)
    shape = (2, scan.nt, scan.n, scan.n, scan.n)
    Wa, Xa = torch.zeros(shape, device="cuda"), torch.zeros(shape, device="cuda")
    Wb, Xb = torch.zeros(shape, device="cuda"), torch.zeros(shape, device="cuda")
    mrf = M.msf_mrf(2.0, 1.2, 1.0, 0.2, 0.5)
    ma = M.Mace(P1, Wa, Xa, yg, lg, M.MSF_PRIOR_QGGMRF, mrf=mrf)
    zeros = torch.zeros_like(c_dev)                      # the handle's own data replaces these
    mb = M.Mace(P2, Wb, Xb, zeros, zeros, M.MSF_PRIOR_QGGMRF, mrf=mrf)
    h = torch.from_numpy(counts.astype(np.float32)).pin_memory()
    for it in range(3):
        M.msf_mace_set_counts(mb, h, I0, I0)
        ra = M.msf_mace_step(ma, 0.5, 0.1, [0.5, 0.5], 3, 1, use_graph=it > 0)
        rb = M.msf_mace_step(mb, 0.5, 0.1, [0.5, 0.5], 3, 1, use_graph=it > 0)
        assert ra == rb
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xb) and torch.equal(Wa, Wb)
