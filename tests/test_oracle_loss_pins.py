"""Pins for the FP64 oracle of the training image loss (oracle/loss.py): each test checks it
against something other than itself (a library filter, closed forms, invariants, finite
differences).  CPU only."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import loss as ol

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("sigma", [0.3, 1.0, 2.0])
def test_blur_matches_scipy_gaussian_filter(sigma):
    # scipy truncates at int(3 sigma + 0.5) taps; these sigmas give the same radius as ceil(3 sigma)
    rng = np.random.default_rng(1)
    a = rng.random((23, 31))
    ref = ndi.gaussian_filter(a, sigma, mode="constant", cval=0.0, truncate=3.0)
    assert np.abs(ol.blur(a, sigma) - ref).max() < 1e-12


def test_blur_of_a_delta_is_the_outer_product_of_the_weights():
    a = np.zeros((21, 21))
    a[10, 10] = 1.0
    w = ol.gaussian_weights(1.7)
    r = (w.size - 1) // 2
    b = ol.blur(a, 1.7)
    assert abs(w.sum() - 1.0) < 1e-15 and np.allclose(w, w[::-1])
    assert np.allclose(b[10 - r:10 + r + 1, 10 - r:10 + r + 1], np.outer(w, w), atol=1e-15)


def test_dog_vanishes_on_a_linear_ramp_away_from_the_border():
    y, x = np.mgrid[0:60, 0:70].astype(np.float64)
    ramp = 0.3 + 0.01 * x - 0.004 * y
    d = ol.blur(ramp, 4.0) - ol.blur(ramp, 2.0)   # blurs keep affine functions where no padding enters
    assert np.abs(d[13:-13, 13:-13]).max() < 1e-12


def test_downsample_is_the_block_mean():
    rng = np.random.default_rng(2)
    gt = rng.random((3, 12, 17))
    small, f = ol.downsample_gray(gt, 0.2)
    assert f == 5 and small.shape == (3, 4)
    assert abs(small[1, 2] - gt[:, 5:10, 10:15].mean()) < 1e-15
    assert abs(small[2, 3] - gt[:, 10:12, 15:17].mean()) < 1e-15


def test_high_frequency_mask_follows_the_edges():
    # a plateau [100, 300) of ones in a zero image: the strongest band-pass responses sit on its two
    # edges and decay away from them (the image is zero at its border, so padding adds no edge)
    gt = np.zeros((3, 60, 400))
    gt[:, :, 100:300] = 1.0
    m, resp = ol.freq_mask(gt, omega=1.0, scale=1.0)
    cols = np.nonzero(m[30])[0]
    assert cols.size > 0
    assert np.all((np.abs(cols - 100) < 50) | (np.abs(cols - 300) < 50))
    assert m[30, 5] == 0 and m[30, 200] == 0 and m[30, 395] == 0
    # omega <= 1/2 takes the complement of the mirrored high-frequency mask
    m_low, _ = ol.freq_mask(gt, omega=0.0, scale=1.0)
    assert np.array_equal(m_low, 1 - m)


def test_ssim_of_constant_images_matches_the_closed_form():
    c1, c2 = 0.3, 0.7
    x = torch.full((3, 40, 40), c1, dtype=torch.float64)
    y = torch.full((3, 40, 40), c2, dtype=torch.float64)
    s = ol.ssim_map(x, y)
    want = (2 * c1 * c2 + ol.SSIM_C1) / (c1 * c1 + c2 * c2 + ol.SSIM_C1)  # variances are zero
    assert abs(float(s[0, 20, 20]) - want) < 1e-12


def test_identical_images_give_ssim_one_and_a_zero_ssim_gradient():
    rng = np.random.default_rng(3)
    gt = rng.random((3, 24, 20))
    L, g, parts = ol.image_loss(gt, gt, np.ones((24, 20)), lambda_ssim=1.0, lambda_omega=0.0)
    assert abs(parts["ssim"] - 1.0) < 1e-12 and abs(L) < 1e-12 and np.abs(g).max() < 1e-12


def test_l1_and_masked_l1_gradients_in_closed_form():
    rng = np.random.default_rng(4)
    gt = rng.random((3, 10, 12))
    img = gt + rng.choice([-1.0, 1.0], gt.shape) * (0.1 + rng.random(gt.shape))
    n = gt.size
    L, g, parts = ol.image_loss(img, gt, np.zeros((10, 12)), lambda_ssim=0.0, lambda_omega=0.0)
    assert np.allclose(g, np.sign(img - gt) / n, rtol=0, atol=1e-15)
    assert abs(L - np.abs(img - gt).mean()) < 1e-15
    mask = (rng.random((10, 12)) > 0.5).astype(np.uint8)
    L, g, parts = ol.image_loss(img, gt, mask, lambda_ssim=0.0, lambda_omega=1.0)
    assert np.allclose(g, np.sign(img - gt) * mask[None] / n, rtol=0, atol=1e-15)
    assert abs(parts["l_omega"] - np.abs((img - gt) * mask[None]).mean()) < 1e-15


def test_full_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    gt = rng.random((3, 14, 13))
    img = np.clip(gt + 0.2 * rng.standard_normal(gt.shape), 0.0, 1.0)
    mask, _ = ol.freq_mask(gt, 0.8, scale=0.5)
    L, g, _ = ol.image_loss(img, gt, mask)
    h = 1e-6
    for idx in [(0, 3, 4), (1, 7, 12), (2, 13, 0), (1, 0, 0), (0, 9, 6)]:
        a, b = img.copy(), img.copy()
        a[idx] += h
        b[idx] -= h
        fd = (ol.image_loss(a, gt, mask)[0] - ol.image_loss(b, gt, mask)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-7 + 1e-5 * abs(g[idx]), (idx, fd, g[idx])
