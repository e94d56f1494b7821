"""GPU training step of the 2.5D CNN (Sec. V) against the FP64 oracle, through the C ABI.

Every forward and backward kernel is checked on its own: the training step
keeps its intermediate tensors (msf_cnn_train_trace / msf_cnn_train_tensor),
and the FP64 oracle is fed the GPU's own stored input of each kernel (the BF16
activation below it and the BF16 gradient above it), so no error carries from
one layer into the next.  Tolerances, from the arithmetic:
  * FP32 outputs of FP32-accumulated sums of exact BF16 x BF16 products (the
    pre-BatchNorm conv outputs, R, the weight gradients over all pixels):
    relative L2 <= 1e-5 (FP32 rounding, about 1e-6 here);
  * BF16 outputs (activations, inter-layer gradients): the GPU rounds to BF16
    (relative 2^-9 per element, about 2e-3 in relative L2 for uniform rounding
    errors); bound 4e-3 against the unrounded FP64 value;
  * BatchNorm statistics and the FP64-summed gamma / beta / bias gradients:
    1e-5.
The end-to-end loss is compared with the oracle's BF16-emulating mode at 1e-2."""
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


def _net(seed):
    rng = np.random.default_rng(seed)
    convs, bns = synth.cnn_weights(seed)
    convs = [(w, rng.normal(0, 0.05, b.shape)) for w, b in convs]
    bns = [(g * rng.uniform(0.7, 1.3, g.shape), rng.normal(0, 0.1, g.shape)) for g, _ in bns]
    return convs, bns


def _batch(seed, B, H, W):
    clean = synth.uniform(seed, (B, H, W), 0.0, 2.0)
    noisy = clean[:, None] + synth.normal(seed + 1, (B, 5, H, W), 0.1)
    return f32(noisy), f32(clean)


F32, BF16 = 1e-5, 4e-3


def test_every_training_kernel_matches_oracle(M):
    # B x H x W = 4 x 20 x 28: both image axes ragged against the 16 x 8 tiles
    convs, bns = _net(71)
    B, H, W = 4, 20, 28
    P = B * H * W
    noisy, clean = _batch(72, B, H, W)
    c = M.Cnn(4096)
    flat = M.pack_params(convs, bns)
    c.set_params(flat)
    c.train_reserve(P)
    c.train_trace(True)
    loss = M.msf_train_step(c, _t(noisy), _t(clean), 1e-3)
    g = c.get_grads().astype(np.float64)
    cv, bv, _ = M.unpack_params(flat)          # the FP32 parameters the GPU holds
    gcv, gbv, _ = M.unpack_params(g.astype(np.float32))
    T = c.train_tensor

    def nchw(t):                               # [P][64] -> [B][64][H][W]
        return t.reshape(B, H, W, -1).transpose(0, 3, 1, 2)

    bf = oracle.bf16
    x = bf(noisy)
    # ---- forward
    # layer 1 (5 -> 64, ReLU): conv of the BF16 input with BF16 weights
    z0 = oracle.conv3x3(x, bf(cv[0][0]), cv[0][1])
    assert rel_l2(nchw(T(c.TT_ACT, 1, P)), np.maximum(z0, 0.0)) <= BF16
    for l in range(1, 9):
        a_in = nchw(T(c.TT_ACT, l, P))
        z = nchw(T(c.TT_Z, l, P))
        assert rel_l2(z, oracle.conv3x3(a_in, bf(cv[l][0]), cv[l][1])) <= F32, ("conv", l)
        a, y, xhat, istd, mean, var = oracle.bn_relu_forward(z, *bv[l - 1])
        st = T(c.TT_BN, l, P)
        assert rel_l2(st[0], mean) <= F32 and rel_l2(st[1], istd) <= F32, ("bn stats", l)
        assert rel_l2(nchw(T(c.TT_ACT, l + 1, P)), a) <= BF16, ("bn+relu", l)
    a9 = nchw(T(c.TT_ACT, 9, P))
    R = T(c.TT_R, 0, P).reshape(B, H, W)
    assert rel_l2(R, oracle.conv3x3(a9, bf(cv[9][0]), cv[9][1])[:, 0]) <= F32
    dR = T(c.TT_DR, 0, P).reshape(B, H, W)
    assert rel_l2(dR, -2.0 * (noisy[:, 2] - R - clean) / P) <= F32
    # ---- backward, layer by layer from the GPU's own stored tensors
    # last layer (64 -> 1, FP32 weights in its input gradient)
    assert rel_l2(nchw(T(c.TT_DA, 9, P)), oracle.conv3x3_dgrad(dR[:, None], cv[9][0])) <= BF16
    assert rel_l2(gcv[9][0], oracle.conv3x3_wgrad(dR[:, None], a9)) <= F32
    assert gcv[9][1][0] == pytest.approx(dR.sum(), rel=F32)
    for l in range(8, 0, -1):
        a_in = nchw(T(c.TT_ACT, l, P))
        z = nchw(T(c.TT_Z, l, P))
        da_up = nchw(T(c.TT_DA, l + 1, P))
        dz = nchw(T(c.TT_DZ, l, P))
        _, y, xhat, istd, _, _ = oracle.bn_relu_forward(z, *bv[l - 1])
        dz_ref, dg, db = oracle.bn_relu_backward(da_up, y, xhat, istd, bv[l - 1][0])
        assert rel_l2(dz, dz_ref) <= BF16, ("bn backward", l)
        assert rel_l2(gbv[l - 1][0], dg) <= F32 and rel_l2(gbv[l - 1][1], db) <= F32, ("gamma/beta", l)
        assert rel_l2(gcv[l][0], oracle.conv3x3_wgrad(dz, a_in)) <= F32, ("wgrad", l)
        # the conv bias feeds BatchNorm: its gradient is the (near-zero) sum of dz
        np.testing.assert_allclose(gcv[l][1], dz.sum(axis=(0, 2, 3)), rtol=F32,
                                   atol=F32 * np.abs(dz).sum(axis=(0, 2, 3)).max())
        assert rel_l2(nchw(T(c.TT_DA, l, P)), oracle.conv3x3_dgrad(dz, bf(cv[l][0]))) <= BF16, ("dgrad", l)
    # first layer: ReLU backward is a mask (bit-exact), then its weight gradient
    dz0 = nchw(T(c.TT_DZ, 0, P))
    np.testing.assert_array_equal(dz0, nchw(T(c.TT_DA, 1, P)) * (nchw(T(c.TT_ACT, 1, P)) > 0))
    assert rel_l2(gcv[0][0], oracle.conv3x3_wgrad(dz0, x)) <= F32
    np.testing.assert_allclose(gcv[0][1], dz0.sum(axis=(0, 2, 3)), rtol=F32, atol=1e-12)
    # the loss against the BF16-emulating oracle end to end
    loss_o, _, _, _ = oracle.train_loss_grad(noisy, clean, cv, bv, emulate_bf16=True)
    assert loss == pytest.approx(loss_o, rel=1e-2)


def test_adam_three_steps_on_real_gradients(M):
    # three steps on three batches; the oracle applies its FP64 Adam to the
    # GPU's own gradients of each step from the same start; the running
    # statistics follow the GPU's batch statistics with momentum 0.1
    convs, bns = _net(77)
    B, H, W = 2, 16, 24
    P = B * H * W
    c = M.Cnn(4096)
    flat = M.pack_params(convs, bns)
    c.set_params(flat)
    c.train_reserve(P)
    theta = flat.astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    frozen = np.zeros(theta.size, bool)
    cv0, bv0, st0 = M.unpack_params(flat)
    o = flat.size - 4 * 64 * 8
    for l in range(8):
        frozen[o + 256 * l + 128:o + 256 * l + 256] = True   # running mean and variance
    stats = [(s[0].copy(), s[1].copy()) for s in st0]
    lr = 1e-3
    for step in range(1, 4):
        noisy, clean = _batch(80 + step, B, H, W)
        M.msf_train_step(c, _t(noisy), _t(clean), lr)
        g = c.get_grads().astype(np.float64)
        t2, m, v = oracle.adam_update(theta, g, m, v, step, lr)
        theta = np.where(frozen, theta, t2)
        for l in range(8):
            bn = c.train_tensor(c.TT_BN, l + 1, P)
            var = (1.0 / bn[1] ** 2 - 1e-5) * P / (P - 1)
            stats[l] = (0.9 * stats[l][0] + 0.1 * bn[0], 0.9 * stats[l][1] + 0.1 * var)
    got = c.get_params().astype(np.float64)
    upd = ~frozen
    assert rel_l2(got[upd] - flat[upd], theta[upd] - flat[upd]) <= 1e-5
    _, _, st = M.unpack_params(got.astype(np.float32))
    for l in range(8):
        assert rel_l2(st[l][0], stats[l][0]) <= 1e-5 and rel_l2(st[l][1], stats[l][1]) <= 1e-4, l


def test_adam_step_and_running_stats(M):
    convs, bns = _net(73)
    B, H, W = 2, 16, 32
    noisy, clean = _batch(74, B, H, W)
    c = M.Cnn(4096)
    flat = M.pack_params(convs, bns)
    c.set_params(flat)
    c.train_reserve(B * H * W)
    lr = 1e-3
    M.msf_train_step(c, _t(noisy), _t(clean), lr)
    g = c.get_grads().astype(np.float64)
    new = c.get_params().astype(np.float64)
    cv0, bv0, st0 = M.unpack_params(flat)
    cv1, bv1, st1 = M.unpack_params(new)
    # first Adam step: theta1 = theta0 - lr g / (|g| + eps)   (closed form)
    gcv, gbv, _ = M.unpack_params(g.astype(np.float32))
    for l in range(len(convs)):
        exp = cv0[l][0] - lr * gcv[l][0] / (np.abs(gcv[l][0]) + 1e-8)
        assert np.all(np.abs(cv1[l][0] - exp) <= 2e-7 + 1e-6 * np.abs(exp)), l
    # running statistics: momentum 0.1 towards the batch moments of the oracle
    _, cache = oracle.train_forward(noisy, cv0, bv0)
    P = B * H * W
    for l in range(len(bns)):
        mean, var = cache["stats"][l]
        em = 0.9 * st0[l][0] + 0.1 * mean
        ev = 0.9 * st0[l][1] + 0.1 * var * P / (P - 1)
        assert rel_l2(st1[l][0], em) <= 5e-2 and rel_l2(st1[l][1], ev) <= 5e-2, l


def test_training_batch_statistics(M):
    import torch
    vol = M.msf_vol(40, 36, 32, 2, 1.0)
    v = torch.rand((2, 32, 36, 40), device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    B, H, W = 256, 16, 16
    noisy = torch.empty((B, 5, H, W), device="cuda")
    clean = torch.empty((B, H, W), device="cuda")
    M.msf_training_batch(v, vol, B, H, W, 0.05, 0.15, 1234, noisy, clean)
    d = (noisy[:, 2] - clean).cpu().numpy().reshape(B, -1)
    s = d.std(axis=1)
    assert abs(d.mean()) < 0.01
    assert s.min() > 0.04 and s.max() < 0.17
    # the clean target is a slice of the volume: its values lie in [0, 1)
    cl = clean.cpu().numpy()
    assert cl.min() >= 0.0 and cl.max() < 1.0
    # a different seed gives different noise
    n2 = torch.empty_like(noisy)
    M.msf_training_batch(v, vol, B, H, W, 0.05, 0.15, 1235, n2, clean)
    assert not torch.equal(noisy, n2)


def test_training_learns_to_denoise(M):
    # The learned agent gains over the identity: after a short training run on
    # phantom patches its output is closer to the clean slice than its input.
    import torch
    scan = synth.Scan(n=96, nt=4, nu=8, nv=8, views=1)
    P = M.Projector(synth.Scan(n=96, nt=4, nu=8, nv=8, views=1))
    vols = torch.empty((4, 96, 96, 96), device="cuda")
    M.msf_phantom_voxelize(P.vol, synth.ellipsoids(75, 12, scan), vols, ss=2)
    c = M.Cnn(96 ** 3)
    convs, bns = synth.cnn_weights(76)
    c.set_params(M.pack_params(convs, bns))
    B, H, W = 32, 48, 48
    c.train_reserve(B * H * W)
    noisy = torch.empty((B, 5, H, W), device="cuda")
    clean = torch.empty((B, H, W), device="cuda")
    losses = []
    for it in range(300):
        M.msf_training_batch(vols, P.vol, B, H, W, 0.02, 0.2, 1000 + it, noisy, clean)
        losses.append(M.msf_train_step(c, noisy, clean, 1e-3))
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:20]), (losses[:5], losses[-5:])
    # held-out volume at sigma = 0.1: the denoiser must beat its input
    test = torch.empty((4, 96, 96, 96), device="cuda")
    M.msf_phantom_voxelize(P.vol, synth.ellipsoids(77, 12, scan), test, ss=2)
    noisy_v = test + 0.1 * torch.randn(test.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(9))
    out = torch.empty_like(test)
    M.msf_denoise(c, M.MSF_XY_T, P.vol, noisy_v, out)
    e_in = (torch.linalg.vector_norm(noisy_v - test) / torch.linalg.vector_norm(test)).item()
    e_out = (torch.linalg.vector_norm(out - test) / torch.linalg.vector_norm(test)).item()
    print(f"denoise NRMSE: input {e_in:.4f} output {e_out:.4f}")
    assert e_out < 0.7 * e_in


def test_train_argument_errors(M):
    import torch
    c = M.Cnn(4096)
    x = torch.zeros((2, 5, 16, 16), device="cuda")
    y = torch.zeros((2, 16, 16), device="cuda")
    with pytest.raises(M.MsfError) as e:
        M.msf_train_step(c, x, y, 1e-3)     # no workspace reserved
    assert e.value.status == 1
