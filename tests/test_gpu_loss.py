"""The training image loss on the GPU (ges_freq_mask, ges_image_loss) against the FP64 oracle.

* the mask: bit-exact wherever the oracle's normalised response is not within 1e-4 of the
  threshold (there FP32 and FP64 may decide differently);
* the loss parts (L, L1, SSIM, L_omega): relative 1e-5;
* dL/dI: relative L2 error <= 1e-3 and max abs error <= 1e-3 of the largest component, with the
  GPU's own mask given to the oracle.
Cases: a ragged image smaller than one tile row, a mid-size one, and the full 1245 x 825 view of
the scene-scale workload (its rendered image against a perturbed copy).
"""
import numpy as np
import pytest

from oracle import loss as ol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ges():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges as g, render
    return g, render.default_context(0)


def _gpu(ges_ctx, img, gt, omega, scale, lam_ssim=0.2, lam_w=0.5):
    g, ctx = ges_ctx
    C, H, W = img.shape
    ti = torch.as_tensor(np.ascontiguousarray(img, np.float32), device="cuda")
    tg = torch.as_tensor(np.ascontiguousarray(gt, np.float32), device="cuda")
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    loss = torch.empty(4, device="cuda")
    grad = torch.empty_like(ti)
    g.ges_freq_mask(ctx.handle, tg, W, H, omega, mask, scale=scale)
    g.ges_image_loss(ctx.handle, ti, tg, mask, W, H, loss, grad, lambda_ssim=lam_ssim, lambda_omega=lam_w)
    torch.cuda.synchronize()
    return mask.cpu().numpy(), loss.cpu().numpy(), grad.cpu().numpy()


def _check(img, gt, omega, scale, got):
    mask, loss, grad = got
    ref_mask, resp = ol.freq_mask(gt.astype(np.float64), omega, scale)
    f = max(1, int(round(1.0 / scale)))
    H, W = mask.shape
    sure = (np.abs(resp - 0.5) > 1e-4)[np.ix_(np.arange(H) // f, np.arange(W) // f)]
    assert sure.mean() > 0.99
    assert np.array_equal(mask[sure], ref_mask[sure])
    L, g, parts = ol.image_loss(img, gt, mask)
    want = np.array([L, parts["l1"], parts["ssim"], parts["l_omega"]])
    assert np.all(np.abs(loss - want) <= 1e-5 * np.maximum(np.abs(want), 1e-3)), (loss, want)
    err = np.linalg.norm(grad - g) / np.linalg.norm(g)
    assert err <= 1e-3, err
    assert np.abs(grad - g).max() <= 1e-3 * np.abs(g).max()


@pytest.mark.parametrize("omega", [0.0, 0.3, 0.8, 1.0])
@pytest.mark.parametrize("scale", [0.2, 1.0])
def test_small_ragged_image(ges, omega, scale):
    rng = np.random.default_rng(10)
    gt = rng.random((3, 37, 45)).astype(np.float32)
    gt[:, 10:25, 5:30] += 0.8  # a block with sharp edges
    img = np.clip(gt + 0.1 * rng.standard_normal(gt.shape), 0, 1.5).astype(np.float32)
    _check(img, gt, omega, scale, _gpu(ges, img, gt, omega, scale))


def test_mid_size_image_all_weights(ges):
    rng = np.random.default_rng(11)
    y, x = np.mgrid[0:150, 0:230]
    gt = np.stack([np.sin(x / 7.0) * np.cos(y / 11.0), (x % 40 < 20).astype(float), y / 150.0]).astype(np.float32)
    img = (gt + 0.05 * rng.standard_normal(gt.shape)).astype(np.float32)
    for lam in [(0.2, 0.5), (0.0, 0.0), (1.0, 0.0), (0.0, 1.0)]:
        got = _gpu(ges, img, gt, 0.6, 0.2, *lam)
        mask, loss, grad = got
        L, g, parts = ol.image_loss(img, gt, mask, *lam)
        assert abs(loss[0] - L) <= 1e-5 * max(abs(L), 1e-3)
        assert np.linalg.norm(grad - g) / max(np.linalg.norm(g), 1e-30) <= 1e-3


def test_full_size_rendered_view(ges):
    from paper_2402_10128_gb300 import render, scenes
    sc, cams = scenes.scene_scale_workload()
    fr = render.Frame(sc.n, cams[0].width, cams[0].height)
    img, _, _ = fr.forward(render.scene_tensors(sc, "cuda"), sc.sh_degree, cams[0])
    torch.cuda.synchronize()
    gt = img.cpu().numpy()
    fr.close()
    rng = np.random.default_rng(12)
    pred = (gt + 0.05 * rng.standard_normal(gt.shape)).astype(np.float32)
    _check(pred, gt, 0.7, 0.2, _gpu(ges, pred, gt, 0.7, 0.2))
