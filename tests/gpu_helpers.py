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
