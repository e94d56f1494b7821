"""Failure detection without a GPU fault: a device-side wait that nothing
satisfies gives up after its limit and reports MSF_ERR_TIMEOUT; the context
stays usable.  Argument, numerical and out-of-memory errors are reported
before or after launches without touching the device state."""
import time

import numpy as np
import pytest

from paper_2008_01567_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    from paper_2008_01567_gb300 import build, msf
    build.build()
    assert torch.cuda.is_available()
    return msf


def test_bounded_wait_times_out_and_context_survives(M):
    import torch
    t0 = time.perf_counter()
    st = M.msf_selftest_wait(5_000_000)        # 5 ms limit
    dt = time.perf_counter() - t0
    assert st == 4                             # MSF_ERR_TIMEOUT
    assert dt < 5.0
    # the context still works: a projection runs and matches a fresh one
    scan = synth.Scan(n=16, nt=1, nu=20, nv=20, views=4)
    P = M.Projector(scan)
    x = torch.rand((1, 16, 16, 16), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    y1, y2 = torch.empty((1, 4, 20, 20), device="cuda"), torch.empty((1, 4, 20, 20), device="cuda")
    M.msf_project(P, x, y1)
    M.msf_project(P, x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2) and y1.abs().sum() > 0


def test_nonfinite_input_is_reported(M):
    import torch
    scan = synth.Scan(n=8, nt=1, nu=12, nv=12, views=3)
    P = M.Projector(scan)
    W = torch.zeros((2, 1, 8, 8, 8), device="cuda")
    X = torch.zeros_like(W)
    X[0, 0, 3, 3, 3] = float("nan")
    y = torch.ones((1, 3, 12, 12), device="cuda")
    m = M.Mace(P, W, X, y, y, M.MSF_PRIOR_QGGMRF, mrf=M.msf_mrf(2.0, 1.2, 1.0, 0.1, 0.5))
    with pytest.raises(M.MsfError) as e:
        M.msf_mace_step(m, 0.5, 0.1, [0.5, 0.5], 1, 1)
    assert e.value.status == 5                 # MSF_ERR_NUMERIC
    # and the next, clean problem runs
    W2 = torch.zeros_like(W)
    X2 = torch.zeros_like(W)
    m2 = M.Mace(P, W2, X2, y, y, M.MSF_PRIOR_QGGMRF, mrf=M.msf_mrf(2.0, 1.2, 1.0, 0.1, 0.5))
    assert np.isfinite(M.msf_mace_step(m2, 0.5, 0.1, [0.5, 0.5], 1, 1))


def test_out_of_memory_is_reported_and_recoverable(M):
    # allocations far beyond the device (2 x 128 TB of activations, ~1 TB of
    # training workspace) fail in cudaMalloc and come back as MSF_ERR_NOMEM;
    # the partial allocations are released and the context keeps working
    import torch
    with pytest.raises(M.MsfError) as e:
        M.Cnn(1 << 40)
    assert e.value.status == 3                 # MSF_ERR_NOMEM
    c = M.Cnn(4096)
    with pytest.raises(M.MsfError) as e:
        c.train_reserve(1 << 28)               # ~1 TB of training workspace
    assert e.value.status == 3
    with pytest.raises(M.MsfError) as e:
        c.train_reserve(1 << 40)               # past the 2^28-pixel limit
    assert e.value.status == 1                 # MSF_ERR_ARG
    c.train_reserve(1 << 12)
    convs, bns = synth.cnn_weights(3)
    c.set_params(M.pack_params(convs, bns))
    shape = (2, 4, 8, 8)
    x = torch.rand(shape, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    out = torch.empty_like(x)
    M.msf_denoise(c, 0, M.msf_vol(8, 8, 4, 2, 1.0), x, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()


def test_checkpoint_resume_is_bit_identical(M):
    # MACE state = (W, X) plus the CNN parameters: stopping after 2 iterations,
    # copying the state out to the host and resuming in fresh handles gives the
    # same result as running 4 iterations straight (the kernels are deterministic).
    import torch
    scan = synth.Scan(n=16, nt=4, nu=24, nv=24, views=6)
    flat = M.pack_params(*synth.cnn_weights(61))

    def setup():
        P = M.Projector(scan)
        ell = synth.ellipsoids(62, 3, scan)
        p = torch.empty((scan.nt, scan.views, scan.nv, scan.nu), device="cuda")
        M.msf_phantom_project(P, ell, p)
        counts = torch.from_numpy(synth.poisson(63, 1e4 * np.exp(-p.cpu().numpy().astype(np.float64)))
                                  .astype(np.float32)).cuda()
        y, lam = torch.empty_like(counts), torch.empty_like(counts)
        M.msf_weights(counts, y, lam, 1e4, 1e4)
        cnn = M.Cnn(scan.n ** 3)
        cnn.set_params(flat)
        W = torch.zeros((4, scan.nt, scan.n, scan.n, scan.n), device="cuda")
        X = torch.zeros_like(W)
        return P, y, lam, cnn, W, X

    P, y, lam, cnn, W, X = setup()
    m = M.Mace(P, W, X, y, lam, M.MSF_PRIOR_CNN, cnn=cnn)
    for _ in range(4):
        M.msf_mace_step(m, 0.8, 0.2, [0.25] * 4, 3)
    P2, y2, lam2, cnn2, W2, X2 = setup()
    m2 = M.Mace(P2, W2, X2, y2, lam2, M.MSF_PRIOR_CNN, cnn=cnn2)
    for _ in range(2):
        M.msf_mace_step(m2, 0.8, 0.2, [0.25] * 4, 3)
    ckpt = {"W": W2.cpu().numpy(), "X": X2.cpu().numpy(), "cnn": cnn2.get_params()}
    del m2, cnn2
    P3, y3, lam3, cnn3, W3, X3 = setup()
    cnn3.set_params(ckpt["cnn"])
    W3.copy_(torch.from_numpy(ckpt["W"]))
    X3.copy_(torch.from_numpy(ckpt["X"]))
    m3 = M.Mace(P3, W3, X3, y3, lam3, M.MSF_PRIOR_CNN, cnn=cnn3)
    for _ in range(2):
        M.msf_mace_step(m3, 0.8, 0.2, [0.25] * 4, 3)
    torch.cuda.synchronize()
    assert torch.equal(W, W3) and torch.equal(X, X3)
