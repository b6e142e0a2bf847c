"""Seeded synthetic scenes and cameras for the GEF rasterizer.

This module only draws inputs: primitive parameter arrays and pinhole cameras.
It holds none of the rasterizer's arithmetic and is the one module that both
the CUDA path's callers and the FP64 oracle's tests take their inputs from.

Every generator uses ``numpy.random.default_rng(seed)`` (PCG64), so a scene is
a pure function of its arguments.  Shapes follow the paper's primitive set
(Sec. 4.1): mean mu[N,3], scale s[N,3] (> 0), quaternion q[N,4] in (w,x,y,z)
order, shape beta[N] (> 0), opacity kappa[N] in (0,1), and spherical-harmonic
coefficients sh[N,(d+1)^2,3].

Workload recipes (sizes of the paper's scenes, Sec. 6.2 and Tab. comparisons; the
datasets themselves are not used):

* ``cube_scene``  -- means uniform in [-1,1]^3, scales log-uniform
  [0.01, 0.08] per axis, uniform random rotations, beta uniform [1,4],
  opacity sigmoid(N(0,1)), SH degree 0 with the DC term drawn so that the
  rendered base colour is uniform in [0,1] (2,000 primitives = the tiny
  128x128 case; 1.5M = the differentiation case).
* ``cluster_scene`` -- 90% of primitives from 64 anisotropic Gaussian
  clusters in a 20-unit box, 10% on a background shell of radius 12-15,
  scales log-uniform [0.002, 0.2], beta log-uniform [0.5, 8], SH degree 3
  with non-DC coefficients N(0, 0.2) (1.5M = the scene-scale case).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# 1 / Y_00: the real SH basis function of degree 0 is the constant 1/(2 sqrt(pi)).
# The DC coefficient that yields a base colour u is (u - 0.5) * 2 sqrt(pi).
_INV_Y00 = 2.0 * math.sqrt(math.pi)


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # [N,3] f32
    scales: np.ndarray     # [N,3] f32, > 0
    quats: np.ndarray      # [N,4] f32, (w,x,y,z), not necessarily unit
    betas: np.ndarray      # [N]   f32, > 0
    opacities: np.ndarray  # [N]   f32, in (0,1)
    shs: np.ndarray        # [N,(d+1)^2,3] f32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(),
                     self.quats[idx].copy(), self.betas[idx].copy(),
                     self.opacities[idx].copy(), self.shs[idx].copy(),
                     self.sh_degree)

    def arrays(self):
        return (self.means, self.scales, self.quats, self.betas,
                self.opacities, self.shs)


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray    # [4,4] f32 row-major world -> camera (OpenCV: +x right, +y down, +z forward)
    campos: np.ndarray     # [3] f32 camera centre in world space
    znear: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh_coeffs(rng, n, degree, dc_uniform=True, sigma=0.2):
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), np.float64)
    u = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = (u - 0.5) * _INV_Y00
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, sigma, (n, k - 1, 3))
    return sh


def _pack(means, scales, quats, betas, opac, shs, degree) -> Scene:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f(means), f(scales), f(quats), f(betas), f(opac), f(shs), degree)


def cube_scene(n: int, seed: int = 0, sh_degree: int = 0,
               beta_range=(1.0, 4.0), beta_log: bool = False,
               scale_range=(0.01, 0.08)) -> Scene:
    """Uniform-cube scene (the tiny-render distribution, any N)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    scales = np.exp(rng.uniform(math.log(scale_range[0]), math.log(scale_range[1]), (n, 3)))
    quats = _unit_quats(rng, n)
    if beta_log:
        betas = np.exp(rng.uniform(math.log(beta_range[0]), math.log(beta_range[1]), n))
    else:
        betas = rng.uniform(beta_range[0], beta_range[1], n)
    opac = _sigmoid(rng.standard_normal(n))
    shs = _sh_coeffs(rng, n, sh_degree)
    return _pack(means, scales, quats, betas, opac, shs, sh_degree)


def cluster_scene(n: int, seed: int = 1, sh_degree: int = 3, n_clusters: int = 64,
                  box: float = 10.0, shell=(12.0, 15.0), background_frac: float = 0.10,
                  beta_range=(0.5, 8.0), scale_range=(0.002, 0.2)) -> Scene:
    """Clustered scene (the scene-scale distribution)."""
    rng = np.random.default_rng(seed)
    n_bg = int(round(n * background_frac))
    n_fg = n - n_bg
    centres = rng.uniform(-box, box, (n_clusters, 3))
    rots = np.stack([np.linalg.qr(rng.standard_normal((3, 3)))[0] for _ in range(n_clusters)])
    stds = np.exp(rng.uniform(math.log(0.3), math.log(2.0), (n_clusters, 3)))
    cid = rng.integers(0, n_clusters, n_fg)
    local = rng.standard_normal((n_fg, 3)) * stds[cid]
    fg = centres[cid] + np.einsum("nij,nj->ni", rots[cid], local)
    d = rng.standard_normal((n_bg, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    bg = d * rng.uniform(shell[0], shell[1], (n_bg, 1))
    means = np.concatenate([fg, bg], 0)
    perm = rng.permutation(n)
    means = means[perm]
    scales = np.exp(rng.uniform(math.log(scale_range[0]), math.log(scale_range[1]), (n, 3)))
    quats = _unit_quats(rng, n)
    betas = np.exp(rng.uniform(math.log(beta_range[0]), math.log(beta_range[1]), n))
    opac = _sigmoid(rng.standard_normal(n))
    shs = _sh_coeffs(rng, n, sh_degree)
    return _pack(means, scales, quats, betas, opac, shs, sh_degree)


def look_at(eye, target, up, width, height, fov_x_deg, znear=0.2, bg=(0.0, 0.0, 0.0)) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; square pixels,
    principal point at the image centre (pixel (i,j) is sampled at (i+0.5, j+0.5))."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], 0)
    t = -R @ eye
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = t
    f = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(int(width), int(height), float(np.float32(f)), float(np.float32(f)),
                  0.5 * width, 0.5 * height, V.astype(np.float32), eye.astype(np.float32),
                  float(znear), tuple(float(b) for b in bg))


def tiny_camera(width=128, height=128, distance=4.0, fov_x_deg=60.0, bg=(0.0, 0.0, 0.0)) -> Camera:
    """Camera at (0,0,-distance) looking at the origin (the tiny-render camera)."""
    return look_at((0.0, 0.0, -distance), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0),
                   width, height, fov_x_deg, bg=bg)


def orbit_cameras(count=20, radius=25.0, elevation_deg=15.0, width=1245, height=825,
                  fov_x_deg=60.0) -> list:
    """``count`` cameras evenly spaced in azimuth on a circle around the origin."""
    cams = []
    el = math.radians(elevation_deg)
    for i in range(count):
        az = 2.0 * math.pi * i / count
        eye = (radius * math.cos(el) * math.cos(az), radius * math.cos(el) * math.sin(az),
               radius * math.sin(el))
        cams.append(look_at(eye, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), width, height, fov_x_deg))
    return cams


def random_sphere_cameras(count, seed, radius=(3.0, 5.0), sizes=((800, 800), (1245, 825), (1920, 1080)),
                          fov_x_deg=60.0) -> list:
    """Cameras at random directions, distance uniform in ``radius``, looking at the
    origin, resolution drawn uniformly from ``sizes`` (the serving mix)."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(count):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        r = rng.uniform(*radius)
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        up = (0.0, 0.0, 1.0) if abs(d[2]) < 0.9 else (0.0, 1.0, 0.0)
        cams.append(look_at(d * r, (0.0, 0.0, 0.0), up, w, h, fov_x_deg))
    return cams


# --- named workloads -------------------------------------------------------------

def tiny_workload(seed: int = 0):
    """2,000 primitives, SH degree 0, 128x128, one camera at distance 4 (fov 60)."""
    return cube_scene(2000, seed=seed), tiny_camera()


def scene_scale_workload(n: int = 1_500_000, seed: int = 1, n_cams: int = 20):
    """1.5M clustered primitives, SH degree 3, 20 orbit cameras at 1245x825."""
    return cluster_scene(n, seed=seed), orbit_cameras(n_cams)


def differentiation_workload(n: int = 1_500_000, seed: int = 2):
    """Cube distribution scaled to 1.5M primitives, SH0, 1245x825 (fwd+bwd case)."""
    return cube_scene(n, seed=seed), tiny_camera(1245, 825)


def stress_workload(n: int = 6_000_000, seed: int = 4):
    """6M cube primitives, beta log-uniform [0.3,16], SH3, 3840x2160."""
    return (cube_scene(n, seed=seed, sh_degree=3, beta_range=(0.3, 16.0), beta_log=True),
            tiny_camera(3840, 2160))


def stress_beta2_workload(n: int = 6_000_000, seed: int = 4):
    """The stress scene and view with every beta set to 2 (the Gaussian degenerate case)."""
    sc, cam = stress_workload(n, seed)
    sc.betas[:] = 2.0
    return sc, cam


def optimizer_workload(n: int, sh_degree: int = 3, seed: int = 7):
    """The optimizer's state for n primitives, drawn directly in its variables (means, log-scales,
    quaternions, shapes shifted by -2, opacity logits, SH) with Adam moments of a run in progress,
    upstream gradients w.r.t. the physical values, and densification statistics.

    Recipe: means U[-1,1]^3; log-scales U[ln 0.001, ln 0.3] (the largest of the three above
    0.01, the clone/split boundary at extent 1, for about 90% of rows); quaternions N(0,1); shifted
    shapes U[-1.7, 6] (beta in [0.3, 8]); opacity logits N(0, 2.5) (about 2% below kappa = 0.005);
    SH N(0, 0.3); first moments N(0, 1e-3), second moments N(0, 1e-3)^2; gradients N(0, 1e-3)
    (means 1e-4); gradient-norm sums of U{0..10} views at 2e-4 x U[0.5, 2.5] x Exp(1) per view, so
    that about 30% of the rows pass the 3e-4 densification threshold; split normals N(0,1) [n,2,3].
    All float32."""
    rng = np.random.default_rng(seed)
    f = np.float32
    nb = (sh_degree + 1) ** 2
    raw = dict(means=rng.uniform(-1, 1, (n, 3)), scales=rng.uniform(math.log(0.001), math.log(0.3), (n, 3)),
               quats=rng.normal(0, 1, (n, 4)), betas=rng.uniform(-1.7, 6.0, n), opacities=rng.normal(0, 2.5, n),
               shs=rng.normal(0, 0.3, (n, nb, 3)))
    shapes = {k: a.shape for k, a in raw.items()}
    m = {k: rng.normal(0, 1e-3, s) for k, s in shapes.items()}
    v = {k: rng.normal(0, 1e-3, s) ** 2 for k, s in shapes.items()}
    grads = {k: rng.normal(0, 1e-4 if k == "means" else 1e-3, s) for k, s in shapes.items()}
    count = rng.integers(0, 11, n)
    accum = rng.exponential(2e-4, n) * count * rng.uniform(0.5, 2.5, n)
    xi = rng.normal(0, 1, (n, 2, 3))
    cast = lambda d: {k: a.astype(f) for k, a in d.items()}
    return dict(raw=cast(raw), m=cast(m), v=cast(v), grads=cast(grads), accum=accum.astype(f),
                count=count.astype(np.int32), xi=xi.astype(f), sh_degree=sh_degree)


def synthetic_image(width: int, height: int, seed: int = 12):
    """A [3,H,W] float32 image with the mix of structure the training loss meets in a rendered view:
    a smooth field (a sum of 12 random low-frequency cosines per channel, amplitude 0.15 around 0.4),
    40 axis-aligned rectangles with sharp edges (values U[0,1]), and stripes of period 6 px in one
    band (fine detail).  Values clipped to [0, 1.2]."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:height, 0:width].astype(np.float64)
    img = np.full((3, height, width), 0.4)
    for c in range(3):
        for _ in range(12):
            fx, fy = rng.uniform(0, 6, 2) * 2 * math.pi
            img[c] += 0.15 / 12 * 4 * np.cos(fx * x / width + fy * y / height + rng.uniform(0, 2 * math.pi))
    for _ in range(40):
        x0, y0 = int(rng.integers(0, width)), int(rng.integers(0, height))
        w, h = int(rng.integers(4, max(5, width // 6))), int(rng.integers(4, max(5, height // 6)))
        img[:, y0:y0 + h, x0:x0 + w] = rng.uniform(0, 1, 3)[:, None, None]
    band = slice(height // 3, height // 3 + max(1, height // 10))
    img[:, band, :] += 0.2 * (np.sin(2 * math.pi * x[band] / 6.0) > 0)[None]
    return np.clip(img, 0.0, 1.2).astype(np.float32)


def mixture_init(model: str, n_components: int, runs: int, seed: int = 0):
    """Initial parameters [runs, rows, N] of 1D mixture fits, float64: weights U[0,1], means
    U[-1,1], scales U[0.05, 0.5], and for the GEF shapes U[1,3] (rows 0..3 in that order)."""
    rng = np.random.default_rng(seed)
    rows = [rng.uniform(0, 1, (runs, n_components)), rng.uniform(-1, 1, (runs, n_components)),
            rng.uniform(0.05, 0.5, (runs, n_components))]
    if model == "gef":
        rows.append(rng.uniform(1, 3, (runs, n_components)))
    return np.stack(rows, axis=1)
