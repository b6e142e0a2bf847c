"""Torch-facing layer over libges: device contexts, frame workspaces and the
``torch.autograd.Function`` whose backward is the library's hand-written one.

PyTorch only supplies device memory and the current CUDA stream; all rasterizer
arithmetic runs in libges (see include/ges.h).
"""
from __future__ import annotations

import math
import threading

import numpy as np
import torch

from . import ges

_ctx_lock = threading.Lock()
_contexts = {}


class Context:
    """A libges context on one CUDA device (optionally bounded to an HBM budget)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = int(device)
        self.handle = ges.ges_ctx_create(self.device, hbm_budget_bytes)

    def close(self):
        if getattr(self, "handle", None):
            ges.ges_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_context(device: int = 0) -> Context:
    with _ctx_lock:
        if device not in _contexts:
            _contexts[device] = Context(device)
        return _contexts[device]


def scene_tensors(scene, device="cuda") -> tuple:
    """(means, scales, quats, betas, opacities, shs) as contiguous fp32 device tensors."""
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
    return tuple(f(a) for a in scene.arrays())


class Frame:
    """Workspace for one rendered view (library-owned device buffers)."""

    def __init__(self, n_capacity: int, width: int, height: int, key_capacity: int = 0, ctx: Context | None = None):
        self.ctx = ctx or default_context(torch.cuda.current_device())
        self.width, self.height = int(width), int(height)
        self.n_capacity = int(n_capacity)
        self.tiles_x = math.ceil(width / 16)
        self.tiles_y = math.ceil(height / 16)
        self.n_tiles = self.tiles_x * self.tiles_y
        self.handle = ges.ges_frame_create(self.ctx.handle, max(1, n_capacity), width, height, key_capacity)
        self.n = 0
        self.busy = False

    def close(self):
        if getattr(self, "handle", None):
            ges.ges_frame_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- pipeline steps (same names as the C entry points)
    def preprocess(self, tensors, sh_degree, cam, params=None, stream=None):
        self._scene = ges.make_scene(*tensors, sh_degree)
        self._tensors = tensors
        self.n = int(tensors[0].shape[0])
        self._cam = cam if isinstance(cam, ges.ges_camera) else ges.make_camera(cam)
        self._params = params if isinstance(params, ges.ges_params) else ges.make_params(**(params or {}))
        ges.ges_preprocess(self.handle, self._scene, self._cam, self._params, stream)

    def bin_sort(self, stream=None):
        ges.ges_bin_sort(self.handle, stream)

    def render_fwd(self, img=None, final_T=None, n_contrib=None, stream=None):
        dev = self._tensors[0].device
        H, W = self.height, self.width
        img = img if img is not None else torch.empty((3, H, W), dtype=torch.float32, device=dev)
        final_T = final_T if final_T is not None else torch.empty((H, W), dtype=torch.float32, device=dev)
        n_contrib = n_contrib if n_contrib is not None else torch.empty((H, W), dtype=torch.int32, device=dev)
        ges.ges_render_fwd(self.handle, img, final_T, n_contrib, stream)
        return img, final_T, n_contrib

    def render_bwd(self, final_T, n_contrib, dL_dimg, grads=None, stream=None):
        t = self._tensors
        grads = grads if grads is not None else tuple(torch.empty_like(a) for a in t)
        ges.ges_render_bwd(self.handle, self._scene, final_T, n_contrib, dL_dimg.contiguous(), ges.make_grads(*grads),
                           stream)
        return grads

    def forward(self, tensors, sh_degree, cam, params=None, stream=None):
        self.preprocess(tensors, sh_degree, cam, params, stream)
        self.bin_sort(stream)
        return self.render_fwd(stream=stream)

    def status(self, stream=None):
        return ges.ges_frame_status(self.handle, stream)

    def keys(self, stream=None):
        return ges.ges_frame_keys(self.handle, stream)

    def inspect(self, stream=None):
        return ges.ges_frame_inspect(self.handle, self.n, self.n_tiles, stream)


class GESRasterize(torch.autograd.Function):
    """img = rasterize(means, scales, quats, betas, opacities, shs); backward = ges_render_bwd.

    The frame holds the sorted lists of this forward until backward has run; do not reuse
    it for another forward in between."""

    @staticmethod
    def forward(ctx, means, scales, quats, betas, opacities, shs, frame, sh_degree, cam, params):
        tensors = tuple(a.detach().contiguous() for a in (means, scales, quats, betas, opacities, shs))
        img, final_T, n_contrib = frame.forward(tensors, sh_degree, cam, params)
        ctx.frame = frame
        ctx.save_for_backward(final_T, n_contrib)
        ctx.mark_non_differentiable(final_T, n_contrib)
        frame.busy = True
        return img, final_T, n_contrib

    @staticmethod
    def backward(ctx, g_img, g_T=None, g_nc=None):
        final_T, n_contrib = ctx.saved_tensors
        grads = ctx.frame.render_bwd(final_T, n_contrib, g_img.contiguous())
        ctx.frame.busy = False
        return (*grads, None, None, None, None)


_frame_cache = {}


def rasterize(means, scales, quats, betas, opacities, shs, sh_degree, cam, params=None, frame=None):
    """Differentiable render of one view.  Returns (img [3,H,W], final_T [H,W], n_contrib [H,W])."""
    if frame is None:
        key = (means.device.index, int(means.shape[0]), int(cam.width), int(cam.height))
        frame = _frame_cache.get(key)
        if frame is None or frame.busy:
            frame = Frame(int(means.shape[0]), cam.width, cam.height)
            _frame_cache[key] = frame
    return GESRasterize.apply(means, scales, quats, betas, opacities, shs, frame, sh_degree, cam, params)
