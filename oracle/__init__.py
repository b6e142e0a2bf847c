"""FP64 CPU oracle for the GEF rasterizer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It never touches the CUDA library and the CUDA
library never touches it; they share only the seeded input generators.

The C++ source (``ges_oracle.cpp``) is compiled with g++ on first use (or by
``build()``) into ``oracle/_build/``.  ``-ffp-contract=off`` keeps the FP32 key
module's operation order exactly as written.

Conventions (same as the public C-ABI, restated here independently):
  * camera: pixel (i, j) is sampled at (i + 0.5, j + 0.5); OpenCV axes
    (+x right, +y down, +z forward); ``viewmat`` maps world to camera, row-major.
  * parameters are physical values: scale > 0, opacity in (0,1), beta > 0;
    quaternions (w,x,y,z), normalised inside.
  * images are planar [3, H, W].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ges_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libges_oracle.so")
_lock = threading.Lock()
_lib = None

# Default parameters of the method (rho from App. B.2; the compositing constants
# alpha clamp 0.99, skip below 1/255, stop below T = 1e-4; 0.3 px dilation; tangent
# clamp 1.3).  flag_tol_* mark pixels whose result sits on a threshold.
DEFAULT_PARAMS = dict(rho=0.1, mode=0, dilation=0.3, alpha_max=0.99, alpha_min=1.0 / 255.0,
                      t_min=1e-4, margin_rel=1e-3, margin_abs=1e-2, clamp_fov=1.3,
                      flag_tol_alpha=1e-4, flag_tol_t=1e-4, phi_mode=0)

MODE_GEF = 0
MODE_PAPER_APPROX = 1

# scale modification (Sec. 4.2): phi_bar_rho (Eq. approx); the exact Gamma ratio (Eq. probablity)
# normalised to phi_n = 2 Gamma(3/beta)/Gamma(1/beta) on the scale vector; phi_n on the variance
PHI_APPROX = 0
PHI_EXACT = 1
PHI_EXACT_VARIANCE = 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, i32, f64, f32 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float
    lib.ora_key_exp2.restype = f32
    lib.ora_key_exp2.argtypes = [f32]
    lib.ora_key_log2.restype = f32
    lib.ora_key_log2.argtypes = [f32]
    lib.ora_phi_bar.argtypes = [i64, P, f64, P]
    lib.ora_phi_exact.argtypes = [i64, P, P]
    lib.ora_phi_mod.argtypes = [i64, P, P, P, P]
    lib.ora_digamma.restype = f64
    lib.ora_digamma.argtypes = [f64]
    lib.ora_key_lgamma.restype = f32
    lib.ora_key_lgamma.argtypes = [f32]
    lib.ora_key_phi.restype = f32
    lib.ora_key_phi.argtypes = [f32, f32, i32]
    lib.ora_sh_basis.argtypes = [i32, i64, P, P]
    lib.ora_keys.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P, P, P]
    lib.ora_sorted_keys.argtypes = [i64, P, P, P, P, P, P, P, P, P]
    lib.ora_project.argtypes = [i64, P, P, P, P, P, P, i32, P, P, P]
    lib.ora_render.argtypes = [i64, P, P, P, P, P, P, i32, P, P, i64, P, P, P, P, P, i32, i32]
    lib.ora_render.restype = i32
    lib.ora_backward.argtypes = [i64, P, P, P, P, P, P, i32, P, P, i64, P, P,
                                 P, P, P, P, P, P, P, i32, P]
    lib.ora_backward.restype = i32
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def cam_array(cam) -> np.ndarray:
    """Flatten a camera (``scenes.Camera``-like) into the oracle's 29-double block."""
    c = np.zeros(29, np.float64)
    c[0], c[1] = cam.width, cam.height
    c[2:6] = [np.float32(cam.fx), np.float32(cam.fy), np.float32(cam.cx), np.float32(cam.cy)]
    c[6:22] = np.asarray(cam.viewmat, np.float32).reshape(16)
    c[22:25] = np.asarray(cam.campos, np.float32).reshape(3)
    c[25] = np.float32(cam.znear)
    c[26:29] = np.asarray(cam.bg, np.float32).reshape(3)
    return c


def par_array(params=None) -> np.ndarray:
    p = dict(DEFAULT_PARAMS)
    if params:
        p.update(params)
    keys = ["rho", "mode", "dilation", "alpha_max", "alpha_min", "t_min", "margin_rel",
            "margin_abs", "clamp_fov", "flag_tol_alpha", "flag_tol_t", "phi_mode"]
    out = np.zeros(16, np.float64)
    for i, k in enumerate(keys):
        v = p[k]
        # the kernels receive these as float32; the oracle uses the same values
        out[i] = v if k in ("mode", "flag_tol_alpha", "flag_tol_t", "phi_mode") else float(np.float32(v))
    return out


def _scene64(scene):
    n = scene.means.shape[0]
    nb = (scene.sh_degree + 1) ** 2
    return (n, _d(scene.means, (n, 3)), _d(scene.scales, (n, 3)), _d(scene.quats, (n, 4)),
            _d(scene.betas, (n,)), _d(scene.opacities, (n,)), _d(scene.shs, (n, nb, 3)))


def key_exp2(x: float) -> float:
    return float(_load().ora_key_exp2(float(x)))


def key_log2(x: float) -> float:
    return float(_load().ora_key_log2(float(x)))


def phi_bar(beta, rho=0.1):
    b = _d(np.atleast_1d(beta))
    out = np.empty_like(b)
    _load().ora_phi_bar(b.size, _p(b), float(rho), _p(out))
    return out


def phi_exact(beta):
    b = _d(np.atleast_1d(beta))
    out = np.empty_like(b)
    _load().ora_phi_exact(b.size, _p(b), _p(out))
    return out


def phi_mod(beta, params=None):
    """(phi, dphi/dbeta) of the projection's scale modification in FP64 (params' phi_mode, rho)."""
    b = _d(np.atleast_1d(beta))
    phi, dphi = np.empty_like(b), np.empty_like(b)
    _load().ora_phi_mod(b.size, _p(b), _p(par_array(params)), _p(phi), _p(dphi))
    return phi, dphi


def digamma(x: float) -> float:
    return float(_load().ora_digamma(float(x)))


def key_lgamma(x: float) -> float:
    """The key path's FP32 ln Gamma."""
    return float(_load().ora_key_lgamma(float(x)))


def key_phi(beta: float, rho: float = 0.1, phi_mode: int = 0) -> float:
    """The key path's FP32 scale modification."""
    return float(_load().ora_key_phi(float(beta), float(rho), int(phi_mode)))


def sh_basis(degree: int, dirs):
    d = _d(dirs).reshape(-1, 3)
    nb = (degree + 1) ** 2
    out = np.empty((d.shape[0], nb), np.float64)
    _load().ora_sh_basis(int(degree), d.shape[0], _p(d), _p(out))
    return out


def keys(scene, cam, params=None):
    """FP32 key module.  Returns dict with depth_key u32[n], rect i32[n,4] (bounding box of the
    extent in tiles: x0,y0,x1,y1, end-exclusive), touched u32[n] (tiles the extent meets: the sum
    of its row spans), mean2d f32[n,2], cov2d f32[n,3], qstar f32[n]."""
    n, m, s, q, b, o, _ = _scene64(scene)
    dk = np.empty(n, np.uint32)
    rect = np.empty((n, 4), np.int32)
    tt = np.empty(n, np.uint32)
    m2 = np.empty((n, 2), np.float32)
    c2 = np.empty((n, 3), np.float32)
    qs = np.empty(n, np.float32)
    _load().ora_keys(n, _p(m), _p(s), _p(q), _p(b), _p(o), _p(cam_array(cam)), _p(par_array(params)),
                     _p(dk), _p(rect), _p(tt), _p(m2), _p(c2), _p(qs))
    return dict(depth_key=dk, rect=rect, touched=tt, mean2d=m2, cov2d=c2, qstar=qs)


def sorted_keys(scene, cam, params=None, key_info=None):
    """Stable-sorted (key, value) list: key = tile << 32 | depth_key, value = primitive index,
    one entry per tile of each primitive's row spans."""
    k = key_info if key_info is not None else keys(scene, cam, params)
    K = int(k["touched"].astype(np.uint64).sum())
    n, m, s, q, b, o, _ = _scene64(scene)
    kk = np.empty(K, np.uint64)
    vv = np.empty(K, np.uint32)
    _load().ora_sorted_keys(n, _p(m), _p(s), _p(q), _p(b), _p(o), _p(cam_array(cam)), _p(par_array(params)),
                            _p(kk), _p(vv))
    return kk, vv


def tile_ranges(sorted_keys_arr, n_tiles):
    """[start, end) per tile from a sorted key list."""
    tiles = (sorted_keys_arr >> np.uint64(32)).astype(np.int64)
    t = np.arange(n_tiles)
    start = np.searchsorted(tiles, t, side="left")
    end = np.searchsorted(tiles, t, side="right")
    return np.stack([start, end], 1).astype(np.uint32)


def project(scene, cam, params=None):
    """FP64 projection per primitive: [n,12] = mx, my, conic a,b,c, cov2d s00,s01,s11, rgb(3), visible."""
    n, m, s, q, b, o, sh = _scene64(scene)
    out = np.empty((n, 12), np.float64)
    _load().ora_project(n, _p(m), _p(s), _p(q), _p(b), _p(o), _p(sh), int(scene.sh_degree),
                        _p(cam_array(cam)), _p(par_array(params)), _p(out))
    return out


def render(scene, cam, params=None, pixels=None, tiled=False, nthreads=0):
    """Brute-force (or tiled) FP64 render.

    pixels: None for the full frame, else an int64 array of linear ids y*W+x.
    Returns dict(img [3,H,W] or [3,npix], T, ncontrib, flags)."""
    n, m, s, q, b, o, sh = _scene64(scene)
    W, H = cam.width, cam.height
    if pixels is None:
        npix = W * H
        pix = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pix.size
    img = np.empty((3, npix), np.float64)
    T = np.empty(npix, np.float64)
    nc = np.empty(npix, np.int32)
    fl = np.empty(npix, np.uint8)
    _load().ora_render(n, _p(m), _p(s), _p(q), _p(b), _p(o), _p(sh), int(scene.sh_degree),
                       _p(cam_array(cam)), _p(par_array(params)), npix, _p(pix), _p(img), _p(T),
                       _p(nc), _p(fl), int(bool(tiled)), int(nthreads))
    if pixels is None:
        return dict(img=img.reshape(3, H, W), T=T.reshape(H, W), ncontrib=nc.reshape(H, W),
                    flags=fl.reshape(H, W))
    return dict(img=img, T=T, ncontrib=nc, flags=fl)


def backward(scene, cam, dL_dimg, params=None, pixels=None, nthreads=0, cond=False):
    """Analytic FP64 gradient of sum(dL_dimg * img).  dL_dimg is [3,H,W] (full frame) or
    [3,npix] over ``pixels``.  Returns dict of float64 gradients and ``inter`` [n,10]
    (mx, my, conic a, b, c, kappa, hb, r, g, b).  With cond=True also ``cond``: for every
    gradient (the same keys and shapes, "inter" included) the scale of its rounding error, the sum
    over pixels of the absolute per-pixel contributions, carried to the parameters through the
    absolute values of each primitive's Jacobian."""
    n, m, s, q, b, o, sh = _scene64(scene)
    W, H = cam.width, cam.height
    if pixels is None:
        npix = W * H
        pix = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pix.size
    g = _d(dL_dimg).reshape(3, npix)
    nb = (scene.sh_degree + 1) ** 2
    out = dict(means=np.empty((n, 3)), scales=np.empty((n, 3)), quats=np.empty((n, 4)),
               betas=np.empty(n), opacities=np.empty(n), shs=np.empty((n, nb, 3)),
               inter=np.empty((n, 10)))
    cbuf = np.empty((n, 22 + 3 * nb)) if cond else None
    _load().ora_backward(n, _p(m), _p(s), _p(q), _p(b), _p(o), _p(sh), int(scene.sh_degree),
                         _p(cam_array(cam)), _p(par_array(params)), npix, _p(pix), _p(g),
                         _p(out["means"]), _p(out["scales"]), _p(out["quats"]), _p(out["betas"]),
                         _p(out["opacities"]), _p(out["shs"]), _p(out["inter"]), int(nthreads),
                         _p(cbuf) if cond else None)
    if cond:
        out["cond"] = dict(inter=cbuf[:, 0:10], means=cbuf[:, 10:13], scales=cbuf[:, 13:16], quats=cbuf[:, 16:20],
                           betas=cbuf[:, 20], opacities=cbuf[:, 21], shs=cbuf[:, 22:].reshape(n, nb, 3))
    return out
