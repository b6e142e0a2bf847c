"""Python binding of libges (include/ges.h).

Argument marshalling only: every step of the rasterizer runs in the CUDA
library.  The functions carry the C names (``ges_preprocess`` ...) and raise
``GesError`` on a non-OK status.  Importing this module loads
``_build/libges.so`` and raises if it has not been built -- there is no
fallback path.

Device arrays are passed as ``torch.Tensor`` (contiguous, on the library's
device) or raw integer addresses; host arrays as numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libges.so")

GES_OK = 0
GES_ERR_INVALID_ARG = 1
GES_ERR_OOM = 2
GES_ERR_CUDA = 3
GES_ERR_CAPACITY = 4
GES_ERR_NOT_READY = 5
GES_ERR_TIMEOUT = 6
GES_ERR_BUSY = 7
GES_ERR_DEVICE_WAIT = 8
STATUS_NAMES = {0: "GES_OK", 1: "GES_ERR_INVALID_ARG", 2: "GES_ERR_OOM", 3: "GES_ERR_CUDA", 4: "GES_ERR_CAPACITY",
                5: "GES_ERR_NOT_READY", 6: "GES_ERR_TIMEOUT", 7: "GES_ERR_BUSY", 8: "GES_ERR_DEVICE_WAIT"}

GES_FALLOFF_GEF = 0
GES_FALLOFF_PAPER_APPROX = 1
GES_PHI_APPROX = 0
GES_PHI_EXACT = 1
GES_PHI_EXACT_VARIANCE = 2

# every symbol declared in include/ges.h
EXPORTED = ["ges_last_error", "ges_params_default", "ges_ctx_create", "ges_ctx_destroy", "ges_frame_create",
            "ges_frame_destroy", "ges_preprocess", "ges_bin_sort", "ges_render_fwd", "ges_render_bwd",
            "ges_frame_status", "ges_frame_keys", "ges_frame_inspect", "ges_frame_count_work",
            "ges_kernel_launches", "ges_trace_enable", "ges_trace_read", "ges_freq_mask", "ges_image_loss",
            "ges_render_fwd_noalloc",
            "ges_adam_params_default", "ges_density_params_default", "ges_position_lr", "ges_adam_step",
            "ges_activate", "ges_densify_stats", "ges_density_control", "ges_reset_opacity", "ges_reset_shape",
            "ges_fit1d_params_default", "ges_signal1d", "ges_fit1d",
            "ges_serve_create", "ges_serve_add_scene",
            "ges_serve_submit", "ges_serve_poll", "ges_serve_destroy"]


class GesError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ges_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("viewmat", ctypes.c_float * 16), ("campos", ctypes.c_float * 3), ("znear", ctypes.c_float),
                ("bg", ctypes.c_float * 3)]


class ges_params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_float), ("falloff", ctypes.c_int32), ("dilation", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("alpha_min", ctypes.c_float), ("t_min", ctypes.c_float),
                ("extent_margin_rel", ctypes.c_float), ("extent_margin_abs", ctypes.c_float),
                ("clamp_fov", ctypes.c_float), ("segment_tiles", ctypes.c_int32), ("phi_mode", ctypes.c_int32)]


class ges_scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("means", ctypes.c_void_p),
                ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p), ("betas", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("shs", ctypes.c_void_p)]


class ges_grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("betas", ctypes.c_void_p), ("opacities", ctypes.c_void_p), ("shs", ctypes.c_void_p)]


class ges_train_set(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("param", ctypes.c_void_p * 6),
                ("m", ctypes.c_void_p * 6), ("v", ctypes.c_void_p * 6)]


class ges_scene_out(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("betas", ctypes.c_void_p), ("opacities", ctypes.c_void_p), ("shs", ctypes.c_void_p)]


class ges_adam_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 6), ("lr_sh_rest", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class ges_density_params(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("percent_dense", ctypes.c_float),
                ("scene_extent", ctypes.c_float), ("min_opacity", ctypes.c_float), ("min_beta", ctypes.c_float),
                ("max_world_size", ctypes.c_float)]


class ges_fit1d_params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("n_components", ctypes.c_int32), ("positive_weights", ctypes.c_int32),
                ("epochs", ctypes.c_int32), ("precision", ctypes.c_int32), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double),
                ("nu", ctypes.c_double), ("mix_eps", ctypes.c_double)]


GES_MIX_GAUSSIAN, GES_MIX_DOG, GES_MIX_LOG, GES_MIX_GEF = 0, 1, 2, 3
MIX_MODELS = {"gaussian": 0, "dog": 1, "log": 2, "gef": 3}
SIGNAL_KINDS = {"square": 0, "triangle": 1, "parabolic": 2, "half_sinusoid": 3, "exponential": 4, "gaussian": 5}


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libges is not built ({_LIB_PATH} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "ges_last_error": ([], ctypes.c_char_p),
        "ges_params_default": ([P], i32),
        "ges_ctx_create": ([ctypes.c_int, ctypes.c_size_t, P], i32),
        "ges_ctx_destroy": ([P], None),
        "ges_frame_create": ([P, i64, i32, i32, i64, P], i32),
        "ges_frame_destroy": ([P], None),
        "ges_preprocess": ([P, P, P, P, P], i32),
        "ges_bin_sort": ([P, P], i32),
        "ges_render_fwd": ([P, P, P, P, P], i32),
        "ges_render_bwd": ([P, P, P, P, P, P, P], i32),
        "ges_frame_status": ([P, P, P], i32),
        "ges_frame_keys": ([P, P, P, P, i64, P], i32),
        "ges_frame_inspect": ([P, P, P, P, P, P, P], i32),
        "ges_frame_count_work": ([P, P, P, P, P, P], i32),
        "ges_kernel_launches": ([], u64),
        "ges_trace_enable": ([P, ctypes.c_int], i32),
        "ges_trace_read": ([P, i32, P, P, P, P], i32),
        "ges_freq_mask": ([P, P, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P], i32),
        "ges_image_loss": ([P, P, P, P, i32, i32, ctypes.c_float, ctypes.c_float, P, P, P], i32),
        "ges_render_fwd_noalloc": ([P, P, P, P, P, P, P], i32),
        "ges_adam_params_default": ([P], i32),
        "ges_density_params_default": ([P], i32),
        "ges_position_lr": ([i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, i64, i64, P], i32),
        "ges_adam_step": ([P, P, P, P, P, i64, P], i32),
        "ges_activate": ([P, P, P, P], i32),
        "ges_densify_stats": ([P, P, P, P], i32),
        "ges_density_control": ([P, P, P, P, P, P, P, P, P], i32),
        "ges_reset_opacity": ([P, P, ctypes.c_float, P], i32),
        "ges_reset_shape": ([P, P, ctypes.c_float, P], i32),
        "ges_fit1d_params_default": ([P], i32),
        "ges_signal1d": ([P, i32, ctypes.c_double, i32, ctypes.c_double, ctypes.c_double, i32, P, P, P], i32),
        "ges_fit1d": ([P, P, i32, i32, P, P, i64, P, P, P, P, P], i32),
        "ges_serve_create": ([P, P, i32, P], i32),
        "ges_serve_add_scene": ([P, P, P], i32),
        "ges_serve_submit": ([P, i32, P, P, P], i32),
        "ges_serve_poll": ([P, u64, i64, P], i32),
        "ges_serve_destroy": ([P], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()
LIB_PATH = _LIB_PATH


def last_error() -> str:
    return _lib.ges_last_error().decode()


def _check(status):
    if status != GES_OK:
        raise GesError(status, last_error())
    return status


def _addr(t):
    """Device/host address of a tensor, numpy array, int or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "arrays must be contiguous"
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ struct builders
def params_default() -> ges_params:
    p = ges_params()
    _check(_lib.ges_params_default(ctypes.byref(p)))
    return p


def make_params(**kw) -> ges_params:
    p = params_default()
    alias = {"mode": "falloff", "margin_rel": "extent_margin_rel", "margin_abs": "extent_margin_abs"}
    for k, v in kw.items():
        setattr(p, alias.get(k, k), v)
    return p


def make_camera(cam) -> ges_camera:
    """From any object with width, height, fx, fy, cx, cy, viewmat (4x4), campos, znear, bg."""
    c = ges_camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    vm = np.asarray(cam.viewmat, np.float32).reshape(16)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    cp = np.asarray(cam.campos, np.float32).reshape(3)
    bg = np.asarray(cam.bg, np.float32).reshape(3)
    for i in range(3):
        c.campos[i] = float(cp[i])
        c.bg[i] = float(bg[i])
    c.znear = float(cam.znear)
    return c


def make_scene(means, scales, quats, betas, opacities, shs, sh_degree) -> ges_scene:
    s = ges_scene()
    s.n = int(means.shape[0])
    s.sh_degree = int(sh_degree)
    s.means, s.scales, s.quats = _addr(means), _addr(scales), _addr(quats)
    s.betas, s.opacities, s.shs = _addr(betas), _addr(opacities), _addr(shs)
    return s


def make_grads(means, scales, quats, betas, opacities, shs) -> ges_grads:
    g = ges_grads()
    g.means, g.scales, g.quats = _addr(means), _addr(scales), _addr(quats)
    g.betas, g.opacities, g.shs = _addr(betas), _addr(opacities), _addr(shs)
    return g


# ------------------------------------------------------------------ C entry points
def ges_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(_lib.ges_ctx_create(int(device), int(hbm_budget_bytes), ctypes.byref(h)))
    return h.value


def ges_ctx_destroy(ctx: int) -> None:
    _lib.ges_ctx_destroy(ctx)


def ges_frame_create(ctx: int, n_capacity: int, width: int, height: int, key_capacity: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(_lib.ges_frame_create(ctx, int(n_capacity), int(width), int(height), int(key_capacity), ctypes.byref(h)))
    return h.value


def ges_frame_destroy(frame: int) -> None:
    _lib.ges_frame_destroy(frame)


def ges_preprocess(frame: int, scene: ges_scene, cam: ges_camera, params: ges_params, stream=None) -> None:
    _check(_lib.ges_preprocess(frame, ctypes.byref(scene), ctypes.byref(cam), ctypes.byref(params), _stream(stream)))


def ges_bin_sort(frame: int, stream=None) -> None:
    _check(_lib.ges_bin_sort(frame, _stream(stream)))


def ges_render_fwd(frame: int, img, final_T, n_contrib, stream=None) -> None:
    _check(_lib.ges_render_fwd(frame, _addr(img), _addr(final_T), _addr(n_contrib), _stream(stream)))


def ges_render_bwd(frame: int, scene: ges_scene, final_T, n_contrib, dL_dimg, grads: ges_grads, stream=None) -> None:
    _check(_lib.ges_render_bwd(frame, ctypes.byref(scene), _addr(final_T), _addr(n_contrib), _addr(dL_dimg),
                               ctypes.byref(grads), _stream(stream)))


def ges_frame_status(frame: int, stream=None):
    """Returns (status, K) without raising on GES_ERR_CAPACITY."""
    k = ctypes.c_int64(0)
    st = _lib.ges_frame_status(frame, _stream(stream), ctypes.byref(k))
    if st not in (GES_OK, GES_ERR_CAPACITY):
        _check(st)
    return st, int(k.value)


def ges_frame_keys(frame: int, stream=None):
    """Per-tile sorted 64-bit keys (tile << 32 | depth bits) and values (primitive index) of the
    last ges_bin_sort, expanded from its segment lists (host numpy arrays)."""
    n = ges_frame_tile_entries(frame, stream)
    keys = np.empty(n, np.uint64)
    vals = np.empty(n, np.uint32)
    k = ctypes.c_int64(0)
    _check(_lib.ges_frame_keys(frame, _stream(stream), _addr(keys) if n else None, _addr(vals) if n else None,
                               n, ctypes.byref(k)))
    return keys, vals


def ges_frame_tile_entries(frame: int, stream=None) -> int:
    """Number of (tile, primitive) entries of the last ges_bin_sort (its segment lists expanded)."""
    k = ctypes.c_int64(0)
    _check(_lib.ges_frame_keys(frame, _stream(stream), None, None, 0, ctypes.byref(k)))
    return int(k.value)


def ges_frame_inspect(frame: int, n: int, n_tiles: int, stream=None):
    out = dict(depth_key=np.empty(n, np.uint32), rect=np.empty((n, 4), np.int32),
               record=np.empty((n, 12), np.float32), ranges=np.empty((n_tiles, 2), np.uint32),
               grad2d=np.empty((n, 12), np.float32))
    _check(_lib.ges_frame_inspect(frame, _stream(stream), _addr(out["depth_key"]), _addr(out["rect"]),
                                  _addr(out["record"]), _addr(out["ranges"]), _addr(out["grad2d"])))
    return out


def ges_frame_count_work(frame: int, stream=None):
    """(evaluated, in_extent, composited, K) of the last binned frame (synchronises)."""
    a, b, c, k = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib.ges_frame_count_work(frame, _stream(stream), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                     ctypes.byref(k)))
    return int(a.value), int(b.value), int(c.value), int(k.value)


def ges_kernel_launches() -> int:
    return int(_lib.ges_kernel_launches())


def ges_freq_mask(ctx: int, gt, width: int, height: int, omega: float, mask, scale: float = 0.2,
                  threshold: float = 0.5, stream=None) -> None:
    """Frequency-modulated mask M_omega of gt [3,H,W] into mask [H,W] uint8 (device tensors)."""
    _check(_lib.ges_freq_mask(ctx, _addr(gt), width, height, omega, scale, threshold, _addr(mask), _stream(stream)))


def ges_image_loss(ctx: int, img, gt, mask, width: int, height: int, loss, dL_dimg, lambda_ssim: float = 0.2,
                   lambda_omega: float = 0.5, stream=None) -> None:
    """loss[4] = (L, L1, SSIM, L_omega) and dL_dimg [3,H,W] (device tensors)."""
    _check(_lib.ges_image_loss(ctx, _addr(img), _addr(gt), _addr(mask), width, height, lambda_ssim, lambda_omega,
                               _addr(loss), _addr(dL_dimg), _stream(stream)))


# ------------------------------------------------------------------ training-side updates
TRAIN_GROUPS = ("means", "scales", "quats", "betas", "opacities", "shs")


def make_train_set(n: int, sh_degree: int, params, m, v) -> ges_train_set:
    """From three sequences of six device tensors (the optimizer's variables and their moments, in
    the group order of TRAIN_GROUPS)."""
    t = ges_train_set()
    t.n, t.sh_degree = int(n), int(sh_degree)
    for g in range(6):
        t.param[g], t.m[g], t.v[g] = _addr(params[g]), _addr(m[g]), _addr(v[g])
    return t


def make_scene_out(means, scales, quats, betas, opacities, shs) -> ges_scene_out:
    o = ges_scene_out()
    o.means, o.scales, o.quats = _addr(means), _addr(scales), _addr(quats)
    o.betas, o.opacities, o.shs = _addr(betas), _addr(opacities), _addr(shs)
    return o


def adam_params_default() -> ges_adam_params:
    p = ges_adam_params()
    _check(_lib.ges_adam_params_default(ctypes.byref(p)))
    return p


def density_params_default(**kw) -> ges_density_params:
    p = ges_density_params()
    _check(_lib.ges_density_params_default(ctypes.byref(p)))
    for k, val in kw.items():
        setattr(p, k, val)
    return p


def ges_position_lr(step: int, lr_init: float = 1.6e-4, lr_final: float = 1.6e-6, delay_mult: float = 0.01,
                    delay_steps: int = 0, max_steps: int = 30000) -> float:
    out = ctypes.c_float()
    _check(_lib.ges_position_lr(step, lr_init, lr_final, delay_mult, delay_steps, max_steps, ctypes.byref(out)))
    return out.value


def ges_adam_step(ctx: int, tset: ges_train_set, grads: ges_grads, phys: ges_scene_out, hp: ges_adam_params,
                  step: int, stream=None) -> None:
    _check(_lib.ges_adam_step(ctx, ctypes.byref(tset), ctypes.byref(grads), ctypes.byref(phys), ctypes.byref(hp),
                              step, _stream(stream)))


def ges_activate(ctx: int, tset: ges_train_set, phys: ges_scene_out, stream=None) -> None:
    _check(_lib.ges_activate(ctx, ctypes.byref(tset), ctypes.byref(phys), _stream(stream)))


def ges_densify_stats(frame: int, grad_accum, count, stream=None) -> None:
    _check(_lib.ges_densify_stats(frame, _addr(grad_accum), _addr(count), _stream(stream)))


def ges_density_control(ctx: int, tin: ges_train_set, grad_accum, count, xi, dp: ges_density_params,
                        tout: ges_train_set, stream=None) -> int:
    """Rows written to tout (raises GesError with status GES_ERR_CAPACITY if tout is too small)."""
    n_out = ctypes.c_int64(0)
    st = _lib.ges_density_control(ctx, ctypes.byref(tin), _addr(grad_accum), _addr(count), _addr(xi),
                                  ctypes.byref(dp), ctypes.byref(tout), ctypes.byref(n_out), _stream(stream))
    if st != GES_OK:
        err = GesError(st, last_error())
        err.n_out = n_out.value
        raise err
    return n_out.value


def ges_reset_opacity(ctx: int, tset: ges_train_set, max_opacity: float = 0.01, stream=None) -> None:
    _check(_lib.ges_reset_opacity(ctx, ctypes.byref(tset), max_opacity, _stream(stream)))


def ges_reset_shape(ctx: int, tset: ges_train_set, beta: float = 2.0, stream=None) -> None:
    _check(_lib.ges_reset_shape(ctx, ctypes.byref(tset), beta, _stream(stream)))


# ------------------------------------------------------------------ 1D mixture fitting
def fit1d_params_default(**kw) -> ges_fit1d_params:
    p = ges_fit1d_params()
    _check(_lib.ges_fit1d_params_default(ctypes.byref(p)))
    for k, val in kw.items():
        setattr(p, k, val)
    return p


def ges_signal1d(ctx: int, kind, x, y, width: float = 1.0, x0: float = -1.0, x1: float = 1.0, stream=None) -> None:
    """x = linspace(x0, x1, len(x)) and y = the signal (device tensors, float32 or float64)."""
    import torch
    k = SIGNAL_KINDS[kind] if isinstance(kind, str) else int(kind)
    prec = 64 if x.dtype == torch.float64 else 32
    _check(_lib.ges_signal1d(ctx, k, width, x.numel(), x0, x1, prec, _addr(x), _addr(y), _stream(stream)))


def ges_fit1d(ctx: int, p: ges_fit1d_params, x, y, params, final_loss, loss_hist=None, grad=None, y_stride=None,
              stream=None) -> None:
    """params [runs, rows, N] (in: initial, out: final); y [runs, S] or [S] (shared)."""
    runs = params.shape[0]
    stride = y_stride if y_stride is not None else (x.numel() if y.dim() == 2 else 0)
    _check(_lib.ges_fit1d(ctx, ctypes.byref(p), runs, x.numel(), _addr(x), _addr(y), stride, _addr(params),
                          _addr(loss_hist), _addr(final_loss), _addr(grad), _stream(stream)))


def ges_trace_enable(ctx: int, on: bool) -> None:
    _check(_lib.ges_trace_enable(ctx, int(bool(on))))


def ges_trace_read(ctx: int, capacity: int = 32):
    """{name: (launches, total device ms)} of the launches traced since the last read (synchronises)."""
    names = ctypes.create_string_buffer(32 * capacity)
    launches = np.zeros(capacity, np.int64)
    total = np.zeros(capacity, np.float64)
    n = ctypes.c_int32(0)
    _check(_lib.ges_trace_read(ctx, capacity, names, _addr(launches), _addr(total), ctypes.byref(n)))
    out = {}
    for k in range(min(n.value, capacity)):
        name = names.raw[32 * k:32 * k + 32].split(b"\0", 1)[0].decode()
        out[name] = (int(launches[k]), float(total[k]))
    return out


def ges_render_fwd_noalloc(scene: ges_scene, cam: ges_camera, params: ges_params, img, final_T, n_contrib,
                           stream=None) -> None:
    """Forward render that allocates no device memory (bounded sizes; see include/ges.h)."""
    _check(_lib.ges_render_fwd_noalloc(ctypes.byref(scene), ctypes.byref(cam), ctypes.byref(params), _addr(img),
                                       _addr(final_T), _addr(n_contrib), _stream(stream)))


def ges_serve_create(ctx: int, params: ges_params, max_slots: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.ges_serve_create(ctx, ctypes.byref(params), int(max_slots), ctypes.byref(h)))
    return h.value


def ges_serve_add_scene(srv: int, host_scene: ges_scene) -> int:
    sid = ctypes.c_int32(-1)
    _check(_lib.ges_serve_add_scene(srv, ctypes.byref(host_scene), ctypes.byref(sid)))
    return int(sid.value)


def ges_serve_submit(srv: int, scene_id: int, cam: ges_camera, out_img: np.ndarray) -> int:
    t = ctypes.c_uint64(0)
    _check(_lib.ges_serve_submit(srv, int(scene_id), ctypes.byref(cam), _addr(out_img), ctypes.byref(t)))
    return int(t.value)


def ges_serve_poll(srv: int, ticket: int, timeout_us: int = 0):
    """Returns (status, latency_ms); status is GES_OK, GES_ERR_NOT_READY or GES_ERR_TIMEOUT."""
    lat = ctypes.c_float(0.0)
    st = _lib.ges_serve_poll(srv, int(ticket), int(timeout_us), ctypes.byref(lat))
    if st not in (GES_OK, GES_ERR_NOT_READY, GES_ERR_TIMEOUT):
        _check(st)
    return st, float(lat.value)


def ges_serve_destroy(srv: int) -> None:
    _check(_lib.ges_serve_destroy(srv))
