"""FP64 oracle of the training image loss (Sec. 4.3, Eq. mask, Eq. laplace, Eq. final) -- TEST
INFRASTRUCTURE ONLY, like the rest of this package.

    L = lambda_L1 L1 + lambda_ssim (1 - SSIM) + lambda_omega L_omega,
    lambda_L1 = 1 - lambda_ssim - lambda_omega            (Eq. final; lambda_ssim 0.2, lambda_omega 0.5)
    L_omega = mean |(I - I_gt) M_omega|                    (Eq. laplace)
    M_omega = 1(|DoG_omega(I_gt)| / max |DoG_omega(I_gt)| > 0.5)                  (Eq. mask)
    DoG_omega = G(., 0.2 + 20 omega) - G(., 0.1 + 10 omega), on the ground truth's channel mean
                downsampled by the image-frequency scale (App. Implementation Details, 0.2)
    for omega <= 1/2 the mask is 1 - M_(1 - omega) (Sec. 4.3, last paragraph)

Readings of the passages the paper leaves open (the kernels implement the same):
  * blur: separable, weights exp(-k^2 / (2 sigma^2)) for |k| <= ceil(3 sigma), normalised to sum 1,
    zero outside the image;
  * downsampling by scale s: factor f = max(1, round(1/s)); low-res pixel (i, j) is the mean of the
    full-resolution pixels [f i, f i + f) x [f j, f j + f) inside the image and over the 3 channels;
    the mask is upsampled by nearest neighbour (pixel (x, y) takes low-res (x // f, y // f));
  * "normalised response": |DoG| divided by its maximum over the image (0 if the maximum is 0);
  * L1, L_omega and SSIM are means over the 3 H W values; |x| has derivative sign(x) (0 at 0);
  * SSIM: 11 x 11 Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2, per channel.
The loss's gradient is taken by torch.autograd on the FP64 CPU expression of it.
"""
from __future__ import annotations

import math

import numpy as np

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
SSIM_SIGMA = 1.5
SSIM_RADIUS = 5


def gaussian_weights(sigma: float, radius: int | None = None) -> np.ndarray:
    """Normalised 1D Gaussian weights on [-radius, radius] (radius ceil(3 sigma) by default)."""
    r = int(math.ceil(3.0 * sigma)) if radius is None else int(radius)
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    return w / w.sum()


def blur(img: np.ndarray, sigma: float, radius: int | None = None) -> np.ndarray:
    """Separable Gaussian blur of a 2D array with zero padding (the same size out)."""
    w = gaussian_weights(sigma, radius)
    r = (w.size - 1) // 2
    a = np.asarray(img, np.float64)
    H, W = a.shape
    p = np.zeros((H, W + 2 * r))
    p[:, r:r + W] = a
    rows = sum(w[k] * p[:, k:k + W] for k in range(w.size))
    p = np.zeros((H + 2 * r, W))
    p[r:r + H, :] = rows
    return sum(w[k] * p[k:k + H, :] for k in range(w.size))


def downsample_gray(gt: np.ndarray, scale: float):
    """Channel mean of gt [3,H,W] box-averaged by the factor f = max(1, round(1/scale))."""
    f = max(1, int(round(1.0 / scale)))
    C, H, W = gt.shape
    h, w = (H + f - 1) // f, (W + f - 1) // f
    out = np.zeros((h, w))
    for i in range(h):
        for j in range(w):
            blk = gt[:, f * i:min(f * i + f, H), f * j:min(f * j + f, W)]
            out[i, j] = blk.mean()
    return out, f


def dog_response(gt: np.ndarray, omega: float, scale: float):
    """|DoG_omega| of the downsampled channel mean, normalised by its maximum; and the factor f."""
    small, f = downsample_gray(np.asarray(gt, np.float64), scale)
    s2 = 0.1 + 10.0 * omega
    d = np.abs(blur(small, 2.0 * s2) - blur(small, s2))
    m = d.max()
    return (d / m if m > 0 else d), f


def freq_mask(gt: np.ndarray, omega: float, scale: float = 0.2, threshold: float = 0.5):
    """M_omega [H,W] (uint8) and the normalised response at low resolution."""
    flip = omega <= 0.5
    resp, f = dog_response(gt, 1.0 - omega if flip else omega, scale)
    low = resp > threshold
    if flip:
        low = ~low
    H, W = gt.shape[1:]
    ys, xs = np.arange(H) // f, np.arange(W) // f
    return low[np.ix_(ys, xs)].astype(np.uint8), resp


def ssim_map(x, y):
    """Per-pixel SSIM of two [3,H,W] torch tensors (the 11 x 11 Gaussian window, zero padding)."""
    import torch
    import torch.nn.functional as F
    w = torch.tensor(gaussian_weights(SSIM_SIGMA, SSIM_RADIUS), dtype=torch.float64)
    k2 = (w[:, None] * w[None, :]).expand(3, 1, 2 * SSIM_RADIUS + 1, 2 * SSIM_RADIUS + 1).contiguous()

    def g(a):
        return F.conv2d(a[None], k2, padding=SSIM_RADIUS, groups=3)[0]

    mx, my = g(x), g(y)
    sxx, syy, sxy = g(x * x) - mx * mx, g(y * y) - my * my, g(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def image_loss(img, gt, mask, lambda_ssim: float = 0.2, lambda_omega: float = 0.5):
    """(L, dL/dimg [3,H,W], parts) in FP64 for the given mask [H,W] (Eq. final)."""
    import torch
    x = torch.tensor(np.asarray(img, np.float64), requires_grad=True)
    y = torch.tensor(np.asarray(gt, np.float64))
    m = torch.tensor(np.asarray(mask, np.float64))[None]
    l1 = (x - y).abs().mean()
    lw = ((x - y) * m).abs().mean()
    ssim = ssim_map(x, y).mean()
    lam_l1 = 1.0 - lambda_ssim - lambda_omega
    L = lam_l1 * l1 + lambda_ssim * (1.0 - ssim) + lambda_omega * lw
    (g,) = torch.autograd.grad(L, x)
    return float(L.detach()), g.numpy(), dict(l1=float(l1.detach()), ssim=float(ssim.detach()), l_omega=float(lw.detach()))
