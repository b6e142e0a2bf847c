"""FP64 oracle of the training-side updates (Sec. 4.4; App. B.2) -- TEST INFRASTRUCTURE ONLY,
like the rest of this package.

The paper keeps the optimisation and density control of Gaussian splatting (Kerbl et al. 2023)
and adds shape resets and shape pruning; App. B.2 lists the constants.  What is computed here:

Parameterisation (the optimizer's variables, one row per primitive):
    means  mu                                   identity
    scales s = exp(l)                           l: log-scales
    quats  q (unnormalised; the rasterizer normalises)
    betas  beta = b + 2                         b: the shifted shape (App. B.2: shifted by -2, b = 0 at init)
    opacities kappa = 1 / (1 + exp(-o))         o: logit
    SH coefficients                             identity
The rasterizer's gradients are with respect to the physical values; the step multiplies by the
activation's derivative (1, s, 1, 1, kappa (1 - kappa), 1).

Adam (Kingma & Ba 2015, with bias correction), per element:
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
    x <- x - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
    learning rates of App. B.2: position 1.6e-4 decayed log-linearly to 1.6e-6 over 30000 steps
    (delay multiplier 0.01), scaling 0.005, rotation 0.001, shape 0.001, opacity 0.05, SH DC 0.0025,
    higher SH 0.0025 / 20 (as in Gaussian splatting); b1 0.9, b2 0.999, eps 1e-15.

Densification statistics (per rendered view): a primitive that the view lists (touched > 0) adds
||(dL/du W/2, dL/dv H/2)|| (its screen-space mean gradient in NDC units) and counts 1.

Density control, with g = accum / max(count, 1) and thresholds of App. B.2:
    clone  g >= tau_g and max s <= percent_dense * extent: the row is copied (moments zero);
    split  g >= tau_g and max s > percent_dense * extent: two children mu + R(q)(s * xi_j),
           scales s / 1.6, the rest copied (moments zero); the parent is removed;
    prune  kappa < min_opacity, beta < min_beta (shape pruning), or (if set) max s > max_world * extent;
           applied to every row of the result (children with their own scales).
    The result lists kept originals, then clones, then first children, then second children, each
    in the original order.  Threshold comparisons are made on the optimizer's variables against
    thresholds mapped into them (log, logit, minus 2) in FP32, as the kernels do.
Resets: opacity kappa <- min(kappa, 0.01); shape beta <- 2 (b <- 0); the group's moments are zeroed.
"""
from __future__ import annotations

import math

import numpy as np

GROUPS = ("means", "scales", "quats", "betas", "opacities", "shs")

ADAM_DEFAULTS = dict(lr_means=1.6e-4, lr_scales=0.005, lr_quats=0.001, lr_betas=0.001, lr_opacities=0.05,
                     lr_sh_dc=0.0025, lr_sh_rest=0.0025 / 20.0, beta1=0.9, beta2=0.999, eps=1e-15)


def activate(raw: dict) -> dict:
    """Physical values of the optimizer's variables."""
    return dict(means=raw["means"].copy(), scales=np.exp(raw["scales"]), quats=raw["quats"].copy(),
                betas=raw["betas"] + 2.0, opacities=1.0 / (1.0 + np.exp(-raw["opacities"])),
                shs=raw["shs"].copy())


def raw_gradient(raw: dict, grads: dict) -> dict:
    """Chain rule from physical-value gradients to the optimizer's variables."""
    phys = activate(raw)
    k = phys["opacities"]
    return dict(means=grads["means"], scales=grads["scales"] * phys["scales"], quats=grads["quats"],
                betas=grads["betas"], opacities=grads["opacities"] * k * (1.0 - k), shs=grads["shs"])


def position_lr(step: int, lr_init: float = 1.6e-4, lr_final: float = 1.6e-6, delay_mult: float = 0.01,
                delay_steps: int = 0, max_steps: int = 30000) -> float:
    """Log-linear decay from lr_init to lr_final over max_steps; with delay_steps > 0 the rate is
    also scaled by delay_mult + (1 - delay_mult) sin(pi/2 min(step / delay_steps, 1))."""
    if step < 0 or (lr_init == 0.0 and lr_final == 0.0):
        return 0.0
    if delay_steps > 0:
        delay = delay_mult + (1.0 - delay_mult) * math.sin(0.5 * math.pi * min(max(step / delay_steps, 0.0), 1.0))
    else:
        delay = 1.0
    t = min(max(step / max_steps, 0.0), 1.0)
    return delay * math.exp(math.log(lr_init) * (1.0 - t) + math.log(lr_final) * t)


def adam_step(raw: dict, m: dict, v: dict, grads: dict, step: int, hp: dict | None = None, sh_dc: int = 3):
    """One Adam step (step >= 1) on every group; returns new (raw, m, v, phys).  The first sh_dc
    values of each SH row take lr_sh_dc, the rest lr_sh_rest."""
    h = dict(ADAM_DEFAULTS)
    if hp:
        h.update(hp)
    g = raw_gradient(raw, grads)
    b1, b2, eps = h["beta1"], h["beta2"], h["eps"]
    c1, c2 = 1.0 - b1 ** step, 1.0 - b2 ** step
    out_raw, out_m, out_v = {}, {}, {}
    for name in GROUPS:
        lr = h["lr_" + name] if name != "shs" else None
        if name == "shs":
            n = raw["shs"].shape[0]
            flat = np.full(raw["shs"].reshape(n, -1).shape, h["lr_sh_rest"])
            flat[:, :sh_dc] = h["lr_sh_dc"]
            lr = flat.reshape(raw["shs"].shape)
        mm = b1 * m[name] + (1.0 - b1) * g[name]
        vv = b2 * v[name] + (1.0 - b2) * g[name] ** 2
        out_raw[name] = raw[name] - lr * (mm / c1) / (np.sqrt(vv / c2) + eps)
        out_m[name], out_v[name] = mm, vv
    return out_raw, out_m, out_v, activate(out_raw)


def densify_stats(touched, inter, width: int, height: int, accum=None, count=None):
    """Add one view's screen-space gradient norms (inter[:, 0:2] = dL/du, dL/dv) for listed primitives."""
    n = inter.shape[0]
    accum = np.zeros(n) if accum is None else np.asarray(accum, np.float64).copy()
    count = np.zeros(n, np.int64) if count is None else np.asarray(count, np.int64).copy()
    vis = np.asarray(touched) > 0
    gx = inter[:, 0] * (0.5 * width)
    gy = inter[:, 1] * (0.5 * height)
    accum[vis] += np.sqrt(gx[vis] ** 2 + gy[vis] ** 2)
    count[vis] += 1
    return accum, count


def _quat_rot(q):
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def density_thresholds(grad_threshold=0.0003, percent_dense=0.01, extent=1.0, min_opacity=0.005,
                       min_beta=0.0, max_world=0.0):
    """The thresholds mapped into the optimizer's variables and rounded to FP32, as the host side of
    the kernels computes them: from the FP32 parameters, in FP64, then one rounding."""
    f = lambda x: float(np.float32(x))
    pd, ext, mo, mb, mw = (f(x) for x in (percent_dense, extent, min_opacity, min_beta, max_world))  # fp32 inputs
    return dict(grad=f(grad_threshold), log_small=f(math.log(pd * ext)),
                logit_opacity=f(math.log(mo / (1.0 - mo))) if mo > 0 else -math.inf,
                shifted_beta=f(mb - 2.0) if mb > 0 else -math.inf,
                log_big=f(math.log(mw * ext)) if mw > 0 else math.inf,
                log_split=f(math.log(1.6)))


def density_control(raw: dict, m: dict, v: dict, accum, count, xi, **thr_kw):
    """Clone, split and prune (rules above).  xi: [n, 2, 3] standard normals for the children.
    Returns (raw, m, v) of the result and the per-row decisions."""
    t = density_thresholds(**thr_kw)
    f32 = np.float32
    n = raw["means"].shape[0]
    # decisions in FP32 on the optimizer's variables, as the kernels take them
    cnt = np.maximum(np.asarray(count, np.int64), 1).astype(f32)
    g = np.asarray(accum, f32) / cnt
    sel = g >= f32(t["grad"])
    lmax = raw["scales"].astype(f32).max(1)
    small = lmax <= f32(t["log_small"])
    prune_common = (raw["opacities"].astype(f32) < f32(t["logit_opacity"])) | \
                   (raw["betas"].astype(f32) < f32(t["shifted_beta"]))
    big = lmax > f32(t["log_big"])
    lchild = (raw["scales"].astype(f32) - f32(t["log_split"])).astype(f32)
    big_child = lchild.max(1) > f32(t["log_big"])
    clone = sel & small & ~prune_common & ~big
    split = sel & ~small
    keep = ~split & ~prune_common & ~big
    child = split & ~prune_common & ~big_child

    R = _quat_rot(raw["quats"].astype(np.float64))
    s = np.exp(raw["scales"].astype(np.float64))
    out_raw, out_m, out_v = {}, {}, {}
    for name in GROUPS:
        a = raw[name]
        kids = [a[child].copy(), a[child].copy()]
        if name == "means":
            for j in range(2):
                off = np.einsum("nij,nj->ni", R[child], s[child] * xi[child, j])
                kids[j] = a[child] + off
        if name == "scales":
            kids = [a[child] - math.log(1.6)] * 2
        out_raw[name] = np.concatenate([a[keep], a[clone], kids[0], kids[1]])
        z = lambda k: np.zeros((int(k.sum()),) + a.shape[1:])
        out_m[name] = np.concatenate([m[name][keep], z(clone), z(child), z(child)])
        out_v[name] = np.concatenate([v[name][keep], z(clone), z(child), z(child)])
    return out_raw, out_m, out_v, dict(keep=keep, clone=clone, split=split, child=child)


def reset_opacity(raw: dict, m: dict, v: dict, max_opacity: float = 0.01):
    """kappa <- min(kappa, max_opacity) on the logit; the opacity moments are zeroed."""
    lim = math.log(max_opacity / (1.0 - max_opacity))
    r = dict(raw, opacities=np.minimum(raw["opacities"], lim))
    return r, dict(m, opacities=np.zeros_like(m["opacities"])), dict(v, opacities=np.zeros_like(v["opacities"]))


def reset_shape(raw: dict, m: dict, v: dict, beta: float = 2.0):
    """beta <- beta (b <- beta - 2); the shape moments are zeroed."""
    r = dict(raw, betas=np.full_like(raw["betas"], beta - 2.0))
    return r, dict(m, betas=np.zeros_like(m["betas"])), dict(v, betas=np.zeros_like(v["betas"]))
