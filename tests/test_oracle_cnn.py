"""Pins of the oracle's 2.5D CNN denoiser (Sec. IV) and its training step (Sec. V)
against library convolution, exact identities and central finite differences."""
import numpy as np
import pytest
from scipy import signal

from paper_2008_01567_gb300 import synth


def test_conv_matches_library_correlation(oracle):
    x = synth.normal(1, (2, 3, 7, 9))
    w = synth.normal(2, (4, 3, 3, 3))
    b = synth.normal(3, (4,))
    y = oracle.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[n, c], w[o, c], mode="same", boundary="fill")
                             for c in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=1e-12, atol=1e-12)


def test_delta_kernel_network_is_identity(oracle):
    # A net whose hidden convs pass channel 0 through (centre tap 1) and whose
    # last layer outputs 0 returns the centre frame: out = centre - R = centre.
    x = synth.uniform(4, (3, 5, 6, 8))
    layers = []
    w = np.zeros((4, 5, 3, 3)); w[0, 2, 1, 1] = 1.0
    layers.append((w, np.zeros(4)))
    w = np.zeros((4, 4, 3, 3)); w[0, 0, 1, 1] = 1.0
    layers.append((w, np.zeros(4)))
    layers.append((np.zeros((1, 4, 3, 3)), np.zeros(1)))
    out = oracle.cnn_forward(x, layers)
    np.testing.assert_array_equal(out, x[:, 2])
    # and with a last layer that copies channel 0, the residual cancels it
    w = np.zeros((1, 4, 3, 3)); w[0, 0, 1, 1] = 1.0
    layers[-1] = (w, np.zeros(1))
    np.testing.assert_allclose(oracle.cnn_forward(x, layers), 0.0, atol=1e-15)


def test_conv_gradients_are_adjoints(oracle):
    # <conv(x, w), dy> = <x, dgrad(dy, w)> = <w, wgrad(dy, x)>  (bilinearity).
    x = synth.normal(5, (2, 3, 6, 5))
    w = synth.normal(6, (4, 3, 3, 3))
    dy = synth.normal(7, (2, 4, 6, 5))
    lhs = np.vdot(oracle.conv3x3(x, w), dy)
    assert np.vdot(x, oracle.conv3x3_dgrad(dy, w)) == pytest.approx(lhs, rel=1e-12)
    assert np.vdot(w, oracle.conv3x3_wgrad(dy, x)) == pytest.approx(lhs, rel=1e-12)


def _tiny_net(seed):
    convs, bns = synth.cnn_weights(seed, channels=4, layers=4)
    rng = np.random.default_rng(seed + 1)
    convs = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in convs]
    bns = [(g + 0.2 * rng.standard_normal(g.shape), be + 0.1 * rng.standard_normal(be.shape)) for g, be in bns]
    return convs, bns


def test_training_gradients_match_finite_differences(oracle):
    convs, bns = _tiny_net(8)
    x = synth.uniform(9, (3, 5, 6, 6))
    clean = synth.uniform(10, (3, 6, 6))
    loss, gc, gb, _ = oracle.train_loss_grad(x, clean, convs, bns)

    def f(convs_, bns_):
        out, _ = oracle.train_forward(x, convs_, bns_)
        return float(np.mean((out - clean) ** 2))

    assert f(convs, bns) == pytest.approx(loss, rel=1e-14)
    rng = np.random.default_rng(11)
    h = 1e-6
    for l in range(len(convs)):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in convs[l][0].shape)
            cp = [(w.copy(), b) for w, b in convs]; cp[l][0][idx] += h
            cm = [(w.copy(), b) for w, b in convs]; cm[l][0][idx] -= h
            fd = (f(cp, bns) - f(cm, bns)) / (2 * h)
            assert gc[l][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        j = rng.integers(0, convs[l][1].shape[0])
        cp = [(w, b.copy()) for w, b in convs]; cp[l][1][j] += h
        cm = [(w, b.copy()) for w, b in convs]; cm[l][1][j] -= h
        fd = (f(cp, bns) - f(cm, bns)) / (2 * h)
        assert gc[l][1][j] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    for l in range(len(bns)):
        for k in range(2):
            j = rng.integers(0, bns[l][k].shape[0])
            bp = [(g.copy(), be.copy()) for g, be in bns]; bp[l][k][j] += h
            bm = [(g.copy(), be.copy()) for g, be in bns]; bm[l][k][j] -= h
            fd = (f(convs, bp) - f(convs, bm)) / (2 * h)
            assert gb[l][k][j] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_folded_bn_equals_batch_statistics_forward(oracle):
    convs, bns = _tiny_net(12)
    x = synth.uniform(13, (4, 5, 5, 7))
    out_train, cache = oracle.train_forward(x, convs, bns)
    folded = oracle.fold_bn(convs, bns, cache["stats"])
    np.testing.assert_allclose(oracle.cnn_forward(x, folded), out_train, rtol=1e-10, atol=1e-12)


def test_adam_first_step_closed_form(oracle):
    # After one step m^ = g and v^ = g^2, so theta1 = theta0 - lr g/(|g| + eps).
    g = np.array([0.3, -2.0, 1e-3])
    th = np.array([1.0, 2.0, 3.0])
    t1, m, v = oracle.adam_update(th, g, np.zeros(3), np.zeros(3), 1, 1e-3)
    np.testing.assert_allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding(oracle):
    # bfloat16 keeps 8 significant bits; ties go to even.
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -3.140625, 0.0])
    np.testing.assert_array_equal(oracle.bf16(a), [1.0, 1.0, 1.0 + 2 ** -6, 1.0, -3.140625, 0.0])


def test_orientations_and_window(oracle):
    v = synth.normal(14, (6, 3, 4, 5))
    for o in oracle.ORIENTS:
        s = oracle.orient_slices(v, o)
        np.testing.assert_array_equal(oracle.orient_volume(s, o), v)
    s = oracle.orient_slices(v, "yz")          # image (z, y) of slice x
    assert s.shape == (6, 5, 3, 4) and s[1, 2, 0, 3] == v[1, 0, 3, 2]
    s = oracle.orient_slices(v, "zx")          # image (x, z) of slice y
    assert s.shape == (6, 4, 5, 3) and s[1, 2, 4, 1] == v[1, 1, 2, 4]
    w = oracle.window5(oracle.orient_slices(v, "xy"))
    # frame 0: channels t = 0,0,0,1,2 ; frame 5: 3,4,5,5,5
    np.testing.assert_array_equal(w[0 * 3 + 1, :, 2, 2], v[[0, 0, 0, 1, 2], 1, 2, 2])
    np.testing.assert_array_equal(w[5 * 3 + 2, :, 1, 4], v[[3, 4, 5, 5, 5], 2, 1, 4])


def test_agents_share_one_model_across_planes(oracle):
    # H_yz,t on v equals H_xy,t on the volume whose (z', y', x') = (x, z, y).
    convs, bns = _tiny_net(15)
    x = synth.uniform(16, (3, 5, 4, 4))
    _, cache = oracle.train_forward(x, convs, bns)
    layers = oracle.fold_bn(convs, bns, cache["stats"])
    v = synth.uniform(17, (5, 4, 6, 3))
    a = oracle.denoise(v, layers, "yz")
    vp = v.transpose(0, 3, 1, 2)
    b = oracle.denoise(np.ascontiguousarray(vp), layers, "xy").transpose(0, 2, 3, 1)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13)


def test_bf16_emulation_modes(oracle):
    # (i) a net without hidden BatchNorm layers (conv -> ReLU -> conv) on
    # BF16-exact data with power-of-two weights keeps every forward value
    # representable, so the emulating forward equals the exact one; its
    # gradients pass through at most two roundings of 2^-9 each.
    convs = [(np.zeros((64, 5, 3, 3)), np.zeros(64)), (np.zeros((1, 64, 3, 3)), np.zeros(1))]
    convs[0][0][0, 2, 1, 1] = 0.5
    convs[1][0][0, 0, 1, 1] = 0.25
    x = oracle.bf16(synth.uniform(18, (2, 5, 6, 6)))
    clean = oracle.bf16(synth.uniform(19, (2, 6, 6)))
    l_e, g_e, _, _ = oracle.train_loss_grad(x, clean, convs, [], emulate_bf16=False)
    l_b, g_b, _, _ = oracle.train_loss_grad(x, clean, convs, [], emulate_bf16=True)
    assert l_b == l_e
    for (a, _), (b, _) in zip(g_e, g_b):
        # sums of products carrying two roundings each: norm-wise within 2^-7
        assert np.linalg.norm(b - a) <= 2 ** -7 * np.linalg.norm(a)
    # (ii) on a shallow, well-conditioned net the BF16 gradients stay within the
    # BF16 error of the exact ones
    convs, bns = synth.cnn_weights(20, channels=8, layers=3)
    x = synth.uniform(21, (3, 5, 8, 8))
    clean = synth.uniform(22, (3, 8, 8))
    _, g_e, gb_e, _ = oracle.train_loss_grad(x, clean, convs, bns)
    _, g_b, gb_b, _ = oracle.train_loss_grad(x, clean, convs, bns, emulate_bf16=True)
    for (a, _), (b, _) in zip(g_e, g_b):
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(a)


def test_bn_relu_backward_finite_differences(oracle):
    # the standalone BatchNorm + ReLU backward against central differences of
    # L = sum(c * a(z, gamma, beta)) for a random upstream gradient c
    rng = np.random.default_rng(81)
    z = rng.normal(0.3, 1.2, (3, 4, 5, 6))
    gamma, beta = rng.uniform(0.5, 1.5, 4), rng.normal(0, 0.3, 4)
    c = rng.normal(size=z.shape)

    def L(z_, g_, b_):
        return float(np.sum(c * oracle.bn_relu_forward(z_, g_, b_)[0]))

    a, y, xhat, istd, mean, var = oracle.bn_relu_forward(z, gamma, beta)
    dz, dg, db = oracle.bn_relu_backward(c, y, xhat, istd, gamma)
    h = 1e-6
    fz = np.zeros(z.size)
    for i in range(z.size):
        e = np.zeros(z.size); e[i] = h
        fz[i] = (L(z + e.reshape(z.shape), gamma, beta) - L(z - e.reshape(z.shape), gamma, beta)) / (2 * h)
    np.testing.assert_allclose(dz.ravel(), fz, rtol=1e-5, atol=1e-7)
    for k in range(4):
        e = np.zeros(4); e[k] = h
        assert dg[k] == pytest.approx((L(z, gamma + e, beta) - L(z, gamma - e, beta)) / (2 * h), rel=1e-6, abs=1e-8)
        assert db[k] == pytest.approx((L(z, gamma, beta + e) - L(z, gamma, beta - e)) / (2 * h), rel=1e-6, abs=1e-8)
    # biased variance, mean over (n, i, j)
    np.testing.assert_allclose(mean, z.mean(axis=(0, 2, 3)))
    np.testing.assert_allclose(istd, 1 / np.sqrt(z.var(axis=(0, 2, 3)) + 1e-5))
