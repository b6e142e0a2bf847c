"""Small seeded scenes and comparison helpers shared by the tests."""
import math

import numpy as np

from paper_2402_10128_gb300 import scenes

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def axis_camera(width=64, height=64, fov_x_deg=60.0, bg=(0.0, 0.0, 0.0)):
    """Camera at the world origin looking down +z (identity rotation)."""
    f = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    V = np.eye(4, dtype=np.float32)
    return scenes.Camera(width, height, float(np.float32(f)), float(np.float32(f)), 0.5 * width,
                         0.5 * height, V, np.zeros(3, np.float32), 0.2, bg)


def make_scene(means, scales, quats, betas, opac, rgb=None, shs=None, degree=0):
    n = len(means)
    if shs is None:
        rgb = np.asarray(rgb, np.float64).reshape(n, 3)
        shs = ((rgb - 0.5) / Y00).reshape(n, 1, 3)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return scenes.Scene(f(means), f(np.asarray(scales).reshape(n, 3)), f(np.asarray(quats).reshape(n, 4)),
                        f(np.asarray(betas).reshape(n)), f(np.asarray(opac).reshape(n)), f(shs), degree)


def random_small_scene(n, seed, beta_range=(0.7, 4.0), depth=(3.0, 6.0), spread=1.0,
                       scale_range=(0.05, 0.3), opac_range=(0.2, 0.9), degree=0):
    """n primitives in front of ``axis_camera``; used for FD and invariance checks."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(*depth, n)
    xy = rng.uniform(-spread, spread, (n, 2)) * z[:, None] * 0.35
    means = np.concatenate([xy, z[:, None]], 1)
    scales = np.exp(rng.uniform(math.log(scale_range[0]), math.log(scale_range[1]), (n, 3)))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    betas = rng.uniform(*beta_range, n)
    opac = rng.uniform(*opac_range, n)
    nb = (degree + 1) ** 2
    shs = np.zeros((n, nb, 3))
    shs[:, 0, :] = (rng.uniform(0.1, 0.9, (n, 3)) - 0.5) / Y00
    if nb > 1:
        shs[:, 1:, :] = rng.normal(0, 0.2, (n, nb - 1, 3))
    return make_scene(means, scales, q, betas, opac, shs=shs, degree=degree)


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------------ tile lists against FP64 geometry
def qmin_over_boxes(A, B, C, u, v, x0, x1, y0, y1):
    """Minimum of q(d) = A dx^2 + 2 B dx dy + C dy^2, d = (x - u, y - v), over each box
    [x0,x1] x [y0,y1] (arrays, FP64): 0 where the centre lies inside; otherwise the smallest of
    the four edges' minima, each the clamped stationary point of q along that edge (q is positive
    definite, so its minimum over a box without the centre lies on the boundary)."""
    best = np.full(np.broadcast(A, x0).shape, np.inf)
    for x in (x0, x1):
        dx = x - u
        dy = np.clip(-B * dx / C, y0 - v, y1 - v)
        best = np.minimum(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    for y in (y0, y1):
        dy = y - v
        dx = np.clip(-B * dy / A, x0 - u, x1 - u)
        best = np.minimum(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    inside = (x0 <= u) & (u <= x1) & (y0 <= v) & (v <= y1)
    return np.where(inside, 0.0, best)


def fp64_extents(scene, cam, params, oracle):
    """Per primitive, in FP64 and without the key path: visibility, 2D mean, conic, 2D covariance
    and q* = the value of q where kappa G reaches alpha_min (GEF falloff: (2 ln(kappa/alpha_min))^(2/beta);
    Gaussian form: 2 ln(kappa/alpha_min)).  Geometry from oracle.project (FP64); camera depth
    from the view matrix in FP64."""
    p = dict(oracle.DEFAULT_PARAMS, **(params or {}))
    proj = oracle.project(scene, cam, params)
    V = np.asarray(cam.viewmat, np.float64).reshape(4, 4)
    m = np.asarray(scene.means, np.float64)
    tz = m @ V[2, :3] + V[2, 3]
    kappa = np.asarray(scene.opacities, np.float64)
    beta = np.asarray(scene.betas, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        L = 2.0 * np.log(kappa / p["alpha_min"])
        qstar = L if p["mode"] == 1 else np.power(np.maximum(L, 0.0), 2.0 / beta)
    det = proj[:, 5] * proj[:, 7] - proj[:, 6] ** 2
    vis = (tz > cam.znear) & (kappa > p["alpha_min"]) & (det > 0)
    return dict(vis=vis, u=proj[:, 0], v=proj[:, 1], A=proj[:, 2], B=proj[:, 3], C=proj[:, 4],
                s00=proj[:, 5], s11=proj[:, 7], qstar=qstar, tz=tz,
                margin_rel=float(np.float32(p["margin_rel"])), margin_abs=float(p["margin_abs"]))


def check_tile_lists_fp64(scene, cam, params, keys, vals, oracle, prims=None, slack_px=2e-3, slack_q=1e-4):
    """Checks per-tile lists (key = tile << 32 | depth bits, value = primitive) against the extent
    ellipse {q <= q*} computed in FP64, independently of the key path's FP32 arithmetic:

    * complete: every tile whose box the ellipse meets with room to spare, min q < q* (1 - slack_q),
      is listed for that primitive (so no pixel with alpha >= alpha_min is left out);
    * tight: every listed tile meets the ellipse widened by the stated margins (q* (1 + margin_rel)^2,
      margin_abs px in x), with slack_px and slack_q for the FP32 key path's rounding.

    prims: restrict to these primitive ids (a sample).  Returns (number of (primitive, tile)
    candidates checked, list of failure descriptions)."""
    e = fp64_extents(scene, cam, params, oracle)
    tx_n = (cam.width + 15) // 16
    ty_n = (cam.height + 15) // 16
    n_tiles = tx_n * ty_n
    n = scene.n
    sel = np.arange(n) if prims is None else np.asarray(prims, np.int64)
    keys = np.asarray(keys, np.uint64)
    vals = np.asarray(vals, np.int64)
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    if prims is not None:
        m = np.isin(vals, sel)
        tiles, vals = tiles[m], vals[m]
    listed = vals * n_tiles + tiles
    fails = []
    if np.unique(listed).size != listed.size:
        fails.append("a (primitive, tile) pair is listed twice")
    # tight: listed tiles
    g = vals
    if not np.all(e["vis"][g]):
        bad = g[~e["vis"][g]]
        fails.append(f"{bad.size} entries of primitives that are not visible in FP64, e.g. {bad[:5]}")
    tx = tiles % tx_n
    ty = tiles // tx_n
    wx = e["margin_abs"] + slack_px
    q = qmin_over_boxes(e["A"][g], e["B"][g], e["C"][g], e["u"][g], e["v"][g],
                        16.0 * tx - wx, 16.0 * tx + 16 + wx, 16.0 * ty - slack_px, 16.0 * ty + 16 + slack_px)
    lim = e["qstar"][g] * (1 + e["margin_rel"]) ** 2 * (1 + slack_q)
    over = q > lim
    if over.any():
        i = int(np.argmax(q / lim))
        fails.append(f"{int(over.sum())} listed tiles miss the widened ellipse; worst primitive {g[i]} tile {tiles[i]}: "
                     f"min q {q[i]:.9g} > {lim[i]:.9g}")
    # complete: candidate tiles in the FP64 bounding box of {q <= q*}
    cand = sel[e["vis"][sel] & np.isfinite(e["qstar"][sel])]
    rx = np.sqrt(e["qstar"][cand] * e["s00"][cand])
    ry = np.sqrt(e["qstar"][cand] * e["s11"][cand])
    x0 = np.clip(np.floor((e["u"][cand] - rx) / 16), 0, tx_n).astype(np.int64)
    x1 = np.clip(np.floor((e["u"][cand] + rx) / 16) + 1, 0, tx_n).astype(np.int64)
    y0 = np.clip(np.floor((e["v"][cand] - ry) / 16), 0, ty_n).astype(np.int64)
    y1 = np.clip(np.floor((e["v"][cand] + ry) / 16) + 1, 0, ty_n).astype(np.int64)
    w = np.maximum(x1 - x0, 0)
    h = np.maximum(y1 - y0, 0)
    cnt = w * h
    total = int(cnt.sum())
    pid = np.repeat(cand, cnt)
    start = np.repeat(np.cumsum(cnt) - cnt, cnt)
    k = np.arange(total) - start
    ww = np.repeat(w, cnt)
    ctx = np.repeat(x0, cnt) + k % np.maximum(ww, 1)
    cty = np.repeat(y0, cnt) + k // np.maximum(ww, 1)
    q = qmin_over_boxes(e["A"][pid], e["B"][pid], e["C"][pid], e["u"][pid], e["v"][pid],
                        16.0 * ctx, 16.0 * ctx + 16, 16.0 * cty, 16.0 * cty + 16)
    need = q < e["qstar"][pid] * (1 - slack_q)
    have = np.isin(pid * n_tiles + cty * tx_n + ctx, listed)
    missing = need & ~have
    if missing.any():
        i = int(np.argmax(missing))
        fails.append(f"{int(missing.sum())} tiles the ellipse meets are not listed; e.g. primitive {pid[i]} tile "
                     f"{cty[i] * tx_n + ctx[i]}: min q {q[i]:.9g} < q* {e['qstar'][pid[i]]:.9g}")
    return total + g.size, fails


def check_depth_keys_fp64(scene, cam, depth_key, oracle, keys=None, vals=None):
    """The depth keys against the camera depth computed in FP64 from the view matrix and rounded
    once: each visible key's float lies within the rounding bound of the FP32 sum of four terms
    (3 ulp-sized errors of the terms' magnitude, plus one of the result); culled primitives hold
    0xFFFFFFFF.  With a sorted list (keys, vals), consecutive entries of a tile are in FP64 depth
    order up to the two keys' bounds, and equal keys keep ascending primitive index.  Returns a
    list of failure descriptions."""
    e = fp64_extents(scene, cam, None, oracle)
    V = np.asarray(cam.viewmat, np.float64).reshape(4, 4)
    m = np.asarray(scene.means, np.float64)
    mag = np.abs(m) @ np.abs(V[2, :3]) + abs(V[2, 3])
    bound = 4.0 * 2.0 ** -24 * mag
    fails = []
    dk = np.asarray(depth_key, np.uint32)
    live = dk != np.uint32(0xFFFFFFFF)
    d32 = dk.view(np.float32).astype(np.float64)
    err = np.abs(d32 - e["tz"])
    over = live & (err > bound)
    if over.any():
        i = int(np.argmax(np.where(live, err / bound, 0)))
        fails.append(f"{int(over.sum())} depth keys off the FP64 depth; worst {i}: {d32[i]!r} vs {e['tz'][i]!r}")
    if np.any(live & (e["tz"] <= cam.znear - bound)):
        fails.append("a primitive behind the near plane holds a depth key")
    if keys is not None:
        keys = np.asarray(keys, np.uint64)
        vals = np.asarray(vals, np.int64)
        tiles = keys >> np.uint64(32)
        same = tiles[1:] == tiles[:-1]
        a, b = vals[:-1][same], vals[1:][same]
        back = e["tz"][b] < e["tz"][a] - bound[a] - bound[b]
        if back.any():
            fails.append(f"{int(back.sum())} list neighbours out of FP64 depth order")
        eq = keys[1:][same] == keys[:-1][same]
        if np.any(b[eq] <= a[eq]):
            fails.append("equal keys not in ascending primitive order")
    return fails
