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
