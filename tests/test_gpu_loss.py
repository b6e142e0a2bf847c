"""The training image loss on the GPU (ges_freq_mask, ges_image_loss) against the FP64 oracle.

* the mask: bit-exact wherever the oracle's normalised response is not within 1e-4 of the
  threshold (there FP32 and FP64 may decide differently);
* the loss, given the oracle's mask on both sides (so that no input of the oracle comes from the
  GPU): the parts (L, L1, SSIM, L_omega) within 1e-5 relative; dL/dI within 1e-3 relative (L2)
  and within 1e-3 of the largest component everywhere.
Cases: a ragged image smaller than one tile row, a mid-size one, and a synthetic image of the
scene-scale view's size (1245 x 825) against a perturbed copy.
"""
import numpy as np
import pytest

from oracle import loss as ol
from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ges():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges as g, render
    return g, render.default_context(0)


def _dev(a, dtype=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype), device="cuda")


def _gpu_mask(ges_ctx, gt, omega, scale):
    g, ctx = ges_ctx
    C, H, W = gt.shape
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    g.ges_freq_mask(ctx.handle, _dev(gt), W, H, omega, mask, scale=scale)
    torch.cuda.synchronize()
    return mask.cpu().numpy()


def _gpu_loss(ges_ctx, img, gt, mask, lam_ssim=0.2, lam_w=0.5):
    g, ctx = ges_ctx
    C, H, W = img.shape
    ti = _dev(img)
    loss = torch.empty(4, device="cuda")
    grad = torch.empty_like(ti)
    g.ges_image_loss(ctx.handle, ti, _dev(gt), _dev(mask, np.uint8), W, H, loss, grad, lambda_ssim=lam_ssim,
                     lambda_omega=lam_w)
    torch.cuda.synchronize()
    return loss.cpu().numpy(), grad.cpu().numpy()


def _check_mask(ges_ctx, gt, omega, scale):
    """GPU mask against the oracle's where the decision is clear; returns the oracle's mask."""
    got = _gpu_mask(ges_ctx, gt, omega, scale)
    ref_mask, resp = ol.freq_mask(gt.astype(np.float64), omega, scale)
    f = max(1, int(round(1.0 / scale)))
    H, W = got.shape
    sure = (np.abs(resp - 0.5) > 1e-4)[np.ix_(np.arange(H) // f, np.arange(W) // f)]
    assert sure.mean() > 0.99
    assert np.array_equal(got[sure], ref_mask[sure])
    return ref_mask


def _check_loss(ges_ctx, img, gt, mask, lam_ssim=0.2, lam_w=0.5):
    loss, grad = _gpu_loss(ges_ctx, img, gt, mask, lam_ssim, lam_w)
    L, g, parts = ol.image_loss(img, gt, mask, lam_ssim, lam_w)
    want = np.array([L, parts["l1"], parts["ssim"], parts["l_omega"]])
    assert np.all(np.abs(loss - want) <= 1e-5 * np.maximum(np.abs(want), 1e-3)), (loss, want)
    err = np.linalg.norm(grad - g) / max(np.linalg.norm(g), 1e-30)
    assert err <= 1e-3, err
    assert np.abs(grad - g).max() <= 1e-3 * np.abs(g).max()


@pytest.mark.parametrize("omega", [0.0, 0.3, 0.8, 1.0])
@pytest.mark.parametrize("scale", [0.2, 1.0])
def test_small_ragged_image(ges, omega, scale):
    rng = np.random.default_rng(10)
    gt = rng.random((3, 37, 45)).astype(np.float32)
    gt[:, 10:25, 5:30] += 0.8  # a block with sharp edges
    img = np.clip(gt + 0.1 * rng.standard_normal(gt.shape), 0, 1.5).astype(np.float32)
    mask = _check_mask(ges, gt, omega, scale)
    _check_loss(ges, img, gt, mask)


def test_mid_size_image_all_weights(ges):
    rng = np.random.default_rng(11)
    y, x = np.mgrid[0:150, 0:230]
    gt = np.stack([np.sin(x / 7.0) * np.cos(y / 11.0), (x % 40 < 20).astype(float), y / 150.0]).astype(np.float32)
    img = (gt + 0.05 * rng.standard_normal(gt.shape)).astype(np.float32)
    mask = _check_mask(ges, gt, 0.6, 0.2)
    for lam in [(0.2, 0.5), (0.0, 0.0), (1.0, 0.0), (0.0, 1.0)]:
        _check_loss(ges, img, gt, mask, *lam)


def test_full_size_view(ges):
    gt = scenes.synthetic_image(1245, 825, seed=12)
    rng = np.random.default_rng(12)
    pred = (gt + 0.05 * rng.standard_normal(gt.shape)).astype(np.float32)
    mask = _check_mask(ges, gt, 0.7, 0.2)
    _check_loss(ges, pred, gt, mask)
