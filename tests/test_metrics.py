"""Reporting metrics of Sec. VI (NRMSE, percentile-range PSNR, SSIM): the
oracle's direct definitions pinned by closed forms, and the library's tensor
versions checked against them.  Also the scan modes of the sparse-view /
limited-angle sweep (Sec. VI, 90/180/360 deg per time-point)."""
import math

import numpy as np
import pytest

import oracle
from paper_2008_01567_gb300 import metrics, synth


def _img(seed, shape=(15, 16)):
    return synth.uniform(seed, shape, 0.5, 2.0)


def test_ssim_identical_images_is_one():
    a = _img(1)
    np.testing.assert_allclose(oracle.ssim_map2d(a, a, 1.5), 1.0, rtol=0, atol=1e-12)


def test_ssim_map_has_one_entry_per_inner_window():
    a = _img(2, (13, 20))
    assert oracle.ssim_map2d(a, a, 1.0).shape == (3, 10)


def test_ssim_of_a_scaled_image_without_constants():
    # b = s a and C1 = C2 = 0 (L = 0): the luminance and the contrast-structure
    # terms are both 2 s / (1 + s^2) at every window, whatever the window
    a = _img(3)
    s = 1.7
    np.testing.assert_allclose(oracle.ssim_map2d(a, s * a, 0.0), (2 * s / (1 + s * s)) ** 2, rtol=1e-12)


def test_ssim_of_flat_images():
    # constant images: zero variances, so SSIM = (2 c d + C1) / (c^2 + d^2 + C1)
    c, d, L = 0.8, 1.3, 2.0
    got = oracle.ssim_map2d(np.full((12, 12), c), np.full((12, 12), d), L)
    C1 = (0.01 * L) ** 2
    np.testing.assert_allclose(got, (2 * c * d + C1) / (c * c + d * d + C1), rtol=1e-12)


def test_ssim_is_symmetric():
    a, b = _img(4), _img(5)
    np.testing.assert_allclose(oracle.ssim_map2d(a, b, 1.5), oracle.ssim_map2d(b, a, 1.5), rtol=1e-12)


def test_psnr_of_a_constant_offset():
    ref = synth.uniform(6, (2, 3, 8, 9), 0.0, 2.0)
    rng = np.percentile(ref, 99.9) - np.percentile(ref, 0.1)
    np.testing.assert_allclose(oracle.psnr(ref + 0.05, ref), 20 * math.log10(rng / 0.05), rtol=1e-12)


def test_library_metrics_match_oracle():
    torch = pytest.importorskip("torch")
    ref = synth.uniform(7, (2, 3, 14, 13), 0.0, 2.0)
    x = ref + 0.1 * synth.normal(8, ref.shape)
    tx, tr = torch.from_numpy(x), torch.from_numpy(ref)
    for q in (0.1, 50.0, 99.9):
        assert metrics.percentile(tr, q) == pytest.approx(float(np.percentile(ref, q)), rel=1e-12)
    assert metrics.nrmse(tx, tr) == pytest.approx(oracle.nrmse(x, ref), rel=1e-12)
    assert metrics.psnr(tx, tr) == pytest.approx(oracle.psnr(x, ref), rel=1e-12)
    assert metrics.ssim(tx, tr) == pytest.approx(oracle.ssim(x, ref), rel=1e-9)


def test_wedge_modes_turn_continuously():
    for deg in (90, 180, 360):
        sc = synth.Scan(n=8, nt=3, nu=8, nv=8, views=4 * deg // 90, mode=f"wedge{deg}")
        th = sc.angles()
        w = math.radians(deg)
        t = np.arange(3)[:, None]
        j = np.arange(sc.views)[None, :]
        np.testing.assert_allclose(th, w * (t + j / sc.views), rtol=0, atol=1e-15)
        # equal angular steps of 22.5 deg across the frame boundaries
        np.testing.assert_allclose(np.diff(th.reshape(-1)), math.radians(22.5), rtol=1e-12)
    with pytest.raises(ValueError):
        synth.Scan(n=8, nt=1, nu=8, nv=8, views=4, mode="wedge0").angles()
