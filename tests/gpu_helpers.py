"""Helpers for the GPU tests: run the CUDA path through the C-ABI and compare with the oracle."""
import numpy as np
import torch

from paper_2402_10128_gb300 import ges, render

NAMES = ["means", "scales", "quats", "betas", "opacities", "shs"]


def gpu_run(scene, cam, params=None, backward_grad=None, key_capacity=0, keys=True):
    """Forward (and optionally backward with upstream gradient ``backward_grad`` [3,H,W])."""
    t = render.scene_tensors(scene, "cuda")
    fr = render.Frame(max(1, scene.n), cam.width, cam.height, key_capacity=key_capacity)
    img, T, nc = fr.forward(t, scene.sh_degree, cam, params)
    out = dict(frame=fr)
    st, K = fr.status()
    out["status"], out["K"] = st, K
    if st != ges.GES_OK:
        return out
    torch.cuda.synchronize()
    out.update(img=img.cpu().numpy(), T=T.cpu().numpy(), nc=nc.cpu().numpy())
    if keys:
        out["keys"], out["vals"] = fr.keys()
        out["K_tiles"] = int(out["keys"].size)
    out["inspect"] = fr.inspect()
    if backward_grad is not None:
        g = torch.as_tensor(np.ascontiguousarray(backward_grad, np.float32), device="cuda")
        grads = fr.render_bwd(T, nc, g)
        torch.cuda.synchronize()
        out["grads"] = {k: v.cpu().double().numpy() for k, v in zip(NAMES, grads)}
        out["inspect"] = fr.inspect()
    return out


def grad_errors(got, ref):
    """Per-tensor relative L2 error."""
    out = {}
    for k in NAMES:
        a = np.asarray(got[k], np.float64).reshape(-1)
        b = np.asarray(ref[k], np.float64).reshape(-1)
        out[k] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    return out


GRAD_TOL = 1e-3
# rounding scale of an FP32 gradient element per unit of the sum of its per-pixel terms' magnitudes
# (the oracle's ``cond``): every fragment's alpha carries the MUFU exp2/log2 rounding (about 2^-22,
# times the exponent's size, up to log2(kappa/alpha_min) <= 8 at a splat's edge), and a pixel's
# transmittance and colour behind carry those of all its fragments, so each per-pixel term is good
# to a few 1e-6 and a sum of terms to that times the sum of their magnitudes
GRAD_TAU = 1e-5


def grad_failures(got, ref, names=NAMES, tol=GRAD_TOL, cond=None, tau=GRAD_TAU):
    """The gradient bar, per parameter tensor: relative L2 error <= tol, and element by element
    |g - g_ref| <= tol (|g_ref| + tol max|g_ref|) + tau cond, where cond (the oracle's per-element
    sum of the absolute per-pixel contributions) bounds the rounding of a sum whose terms cancel;
    without cond the last term is left out.  Returns one message per tensor that fails either
    bound, naming its worst element (index, both values, its share of the bound, and of the bound
    without the rounding term); an empty list means every tensor passes."""
    bad = []
    for k in names:
        a = np.asarray(got[k], np.float64).reshape(-1)
        b = np.asarray(ref[k], np.float64).reshape(-1)
        assert a.shape == b.shape, (k, a.shape, b.shape)
        if b.size == 0:
            continue
        l2 = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
        strict = tol * (np.abs(b) + tol * np.abs(b).max())
        c = np.zeros_like(b) if cond is None else np.asarray(cond[k], np.float64).reshape(-1)
        bound = strict + tau * c
        d = np.abs(a - b)
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(bound > 0, d / bound, np.where(d > 0, np.inf, 0.0))
            sratio = np.where(strict > 0, d / strict, np.where(d > 0, np.inf, 0.0))
        i = int(np.argmax(ratio))
        if l2 > tol or ratio[i] > 1.0:
            bad.append(f"{k}: rel L2 {l2:.3e}; worst element {i} got {a[i]:.9e} ref {b[i]:.9e} "
                       f"|diff| {d[i]:.3e} = {ratio[i]:.3f} x bound ({sratio[i]:.3f} x without the rounding term, "
                       f"terms' magnitude {c[i]:.3e}); {int((ratio > 1).sum())} of {b.size} over")
    return bad
