"""GB300-native dense RGBD plane fitting (Papadakis & Willis, "Real-Time Surface
Fitting to RGBD Sensor Data").

Thin PyTorch binding over the C ABI of ``libsurffit.so`` (``include/surffit.h``):
PyTorch supplies device memory and streams; every step of the fit runs in the
library's CUDA kernels.  There is no CPU fallback: on a machine without the
built library or without a GPU, the calls raise.

Example::

    import torch
    from paper_2103_06644_gb300 import SurfaceFitter

    fit = SurfaceFitter((fx, fy, cx, cy), W, H, 7)           # 7 x 7 windows, disparity form
    depth = torch.as_tensor(z_metres, device="cuda")         # [H, W] or [N, H, W] float32, 0 = missing
    normals, offsets, curvature = fit.fit(depth)             # NaN where a window has no fit
    counts = fit.fit(depth, counts=True)[3]                  # valid pixels per window
    n_host, d_host, k_host = fit.fit_host(z_numpy)           # the same from host memory
    n, d, k = fit.fit_differentiable(depth.requires_grad_()) # backward to the depth (implicit fits)

``SurfaceFitter(..., method="standard" | "explicit_disparity" | "explicit_standard",
depth_type="u16" | "disparity_u16")`` selects the fit and the depth encoding;
``set_precision``, ``set_constraint``, ``set_delta_table``, ``set_disparity_model`` and
``set_tiles`` adjust a context; ``quadtree`` segments frames into planes;
``SurfaceFitBatch`` fits frames of mixed sizes and windows in one persistent pass.
"""
from __future__ import annotations

import ctypes
from typing import Sequence, Tuple, Union

import numpy as np

from . import _native
from ._native import SurfFitError

__all__ = ["SurfaceFitter", "SurfaceFitBatch", "SurfFitError", "METHODS", "DEPTH_TYPES", "channel_counts",
           "version"]

METHODS = {"disparity": 0, "standard": 1, "explicit_disparity": 2, "explicit_standard": 3}
DEPTH_TYPES = {"f32": 0, "u16": 1, "disparity_u16": 2}


def version() -> str:
    return _native.lib().sf_version().decode()


def channel_counts(method: str) -> Tuple[int, int]:
    """(depth-dependent channels, mask-only channels) of the method's window sums."""
    d = ctypes.c_int()
    m = ctypes.c_int()
    _native.check(_native.lib().sf_channel_counts(METHODS[method], ctypes.byref(d), ctypes.byref(m)))
    return d.value, m.value


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class SurfaceFitter:
    """One camera, image size and window: the library context of ``sf_create``.

    ``intrinsics`` is (fx, fy, cx, cy) or (fx, fy, cx, cy, dx, dy) as in Eq. 1.
    """

    def __init__(self, intrinsics: Sequence[float], W: int, H: int, window: int, method: str = "disparity",
                 depth_type: str = "f32", depth_scale: float = 1e-3, min_valid: int = 3,
                 require_center: bool = True):
        it = tuple(float(v) for v in intrinsics)
        if len(it) == 4:
            it = it + (0.0, 0.0)
        if len(it) != 6:
            raise ValueError("intrinsics must have 4 or 6 entries")
        self.W, self.H, self.window = int(W), int(H), int(window)
        self.method, self.depth_type = method, depth_type
        self.depth_scale = float(depth_scale)
        L = _native.lib()
        h = ctypes.c_void_p()
        _native.check(L.sf_create(ctypes.byref(_native.Intrinsics(*it)), self.W, self.H, self.window, ctypes.byref(h)))
        self._h = h
        self.set_params(method, depth_type, depth_scale, min_valid, require_center)

    def set_params(self, method: str, depth_type: str = "f32", depth_scale: float = 1e-3, min_valid: int = 3,
                   require_center: bool = True) -> None:
        _native.check(_native.lib().sf_set_params(self._h, METHODS[method], DEPTH_TYPES[depth_type],
                                                  float(depth_scale), int(min_valid), int(bool(require_center))))
        self.method, self.depth_type, self.depth_scale = method, depth_type, float(depth_scale)

    def set_tiles(self, hseg: int = 0, vband: int = 0) -> None:
        """Tile shape: hseg in {8, 16, 32, 64, 128} columns per row-pass thread, vband rows per band
        (0 = automatic for either)."""
        _native.check(_native.lib().sf_set_tiles(self._h, int(hseg), int(vband)))

    def set_delta_table(self, ddx=None, ddy=None) -> None:
        """Per-pixel ray adjustments [H, W] in pixels (``sf_set_delta_table``); None, None removes them."""
        if ddx is None and ddy is None:
            _native.check(_native.lib().sf_set_delta_table(self._h, None, None))
            return
        a = np.ascontiguousarray(ddx, dtype=np.float32)
        b = np.ascontiguousarray(ddy, dtype=np.float32)
        if a.shape != (self.H, self.W) or b.shape != (self.H, self.W):
            raise ValueError("delta tables must be [H, W] = [%d, %d]" % (self.H, self.W))
        _native.check(_native.lib().sf_set_delta_table(self._h, a.ctypes.data, b.ctypes.data))

    def set_disparity_model(self, alpha: float, beta: float = 0.0) -> None:
        """Sensor model of ``disparity_u16`` input: 1/Z = alpha * D + beta (1/metres)."""
        _native.check(_native.lib().sf_set_disparity_model(self._h, float(alpha), float(beta)))

    def set_constraint(self, unit4: bool) -> None:
        """|(a,b,c)| = 1 (default, False) or the literal |(a,b,c,d)| = 1 of Eq. 4 (True) for the implicit fits."""
        _native.check(_native.lib().sf_set_constraint(self._h, 1 if unit4 else 0))

    def set_precision(self, mode: int, tau: float = 1e-3) -> None:
        """0: float32 solve; 1: + double-float refinement where gamma < tau; 2: refinement everywhere."""
        _native.check(_native.lib().sf_set_precision(self._h, int(mode), float(tau)))

    def precision_stats(self) -> Tuple[int, int]:
        """(windows queued for refinement, windows re-summed from the depth) in the last fit pass."""
        q, r = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
        _native.check(_native.lib().sf_precision_stats(self._h, ctypes.byref(q), ctypes.byref(r)))
        return int(q.value), int(r.value)

    def graph_replays(self) -> int:
        """How many fit calls of this context replayed its captured CUDA graph."""
        n = ctypes.c_longlong(0)
        _native.check(_native.lib().sf_graph_replays(self._h, ctypes.byref(n)))
        return int(n.value)

    # -- device API -------------------------------------------------------------
    def _check_depth(self, depth):
        import torch

        want = torch.float32 if self.depth_type == "f32" else torch.uint16  # u16 and disparity_u16
        if depth.dtype != want and not (want == torch.uint16 and depth.dtype == torch.int16):
            raise TypeError("depth must be %s for depth_type %s" % (want, self.depth_type))
        if not depth.is_cuda or not depth.is_contiguous():
            raise ValueError("depth must be a contiguous CUDA tensor")
        if depth.shape[-2:] != (self.H, self.W):
            raise ValueError("depth shape %s does not match %dx%d" % (tuple(depth.shape), self.H, self.W))

    def fit(self, depth, out=None, counts: bool = False, stream=None):
        """Fit every pixel of [H, W] or [N, H, W] depth; returns (normals, offsets, curvature[, counts])."""
        import torch

        self._check_depth(depth)
        batched = depth.dim() == 3
        n = depth.shape[0] if batched else 1
        shape = (n, self.H, self.W) if batched else (self.H, self.W)
        dev = depth.device
        if out is None:
            normals = torch.empty(shape + (3,), dtype=torch.float32, device=dev)
            offsets = torch.empty(shape, dtype=torch.float32, device=dev)
            curv = torch.empty(shape, dtype=torch.float32, device=dev)
        else:
            normals, offsets, curv = out
        cnt = torch.empty(shape, dtype=torch.int32, device=dev) if counts else None
        _native.check(_native.lib().sf_fit_ex(self._h, n, depth.data_ptr(), normals.data_ptr(), offsets.data_ptr(),
                                              curv.data_ptr(), cnt.data_ptr() if cnt is not None else None,
                                              _stream_handle(stream)))
        return (normals, offsets, curv, cnt) if counts else (normals, offsets, curv)

    def backward(self, depth, g_normals, g_offsets, g_curvature, stream=None, after_fit: bool = False):
        """dL/dZ [.., H, W] for L = sum(g_normals . n + g_offsets d + g_curvature kappa) (``sf_fit_backward_ex``).

        ``after_fit=True`` promises that ``depth`` is unchanged since this fitter last fitted it: the
        backward then reuses that fit's row pass when the library finds it still in place."""
        import torch

        self._check_depth(depth)
        n = depth.shape[0] if depth.dim() == 3 else 1
        gn = torch.nan_to_num(g_normals.float()).contiguous()
        gd = torch.nan_to_num(g_offsets.float()).contiguous()
        gk = torch.nan_to_num(g_curvature.float()).contiguous()
        g = torch.empty(depth.shape, dtype=torch.float32, device=depth.device)
        flags = 1 if after_fit else 0  # SF_BACKWARD_AFTER_FIT
        _native.check(_native.lib().sf_fit_backward_ex(self._h, n, depth.data_ptr(), gn.data_ptr(), gd.data_ptr(),
                                                       gk.data_ptr(), g.data_ptr(), flags, _stream_handle(stream)))
        return g

    def backward_reuses(self) -> int:
        """How many backward calls of this fitter reused the last fit's row pass."""
        n = ctypes.c_longlong(0)
        _native.check(_native.lib().sf_backward_reuses(self._h, ctypes.byref(n)))
        return int(n.value)

    def fit_differentiable(self, depth):
        """(normals, offsets, curvature) with a backward to the float32 depth (torch.autograd)."""
        return _FitFunction.apply(depth, self)

    # -- planar segmentation (Section III) -------------------------------------------
    QUAD_FIT, QUAD_SPLIT, QUAD_HIGH_ERROR, QUAD_INVALID = 0, 1, 2, 3

    def quadtree(self, depth, tile: int = 64, max_level: int = 3, tau: float = 1e-2, min_frac: float = 0.5,
                 capacity: int = 0, out=None, to_host: bool = True, stream=None):
        """Tile-subdivision plane segmentation of [H, W] or [N, H, W] depth (``sf_quadtree``).

        Returns every evaluated node as a numpy record array (fields of ``sf_quad_node``) sorted by
        frame, level, y0, x0.  ``min_frac`` is the minimum valid fraction of a node (rounded to
        per mille); ``capacity`` 0 sizes the node buffer for the largest possible tree.  With
        ``to_host=False`` nothing is copied or synchronised: the device buffers (nodes as bytes,
        count) are returned, and ``out`` may pass them back in for reuse.
        """
        import torch

        self._check_depth(depth)
        n = depth.shape[0] if depth.dim() == 3 else 1
        tiles = -(-self.W // tile) * -(-self.H // tile)
        if capacity <= 0:
            capacity = min(tiles * n * sum(4 ** l for l in range(max_level + 1)), 4 * self.W * self.H * n)
        if out is None:
            buf = torch.empty(capacity * 56, dtype=torch.uint8, device=depth.device)
            cnt = torch.zeros(1, dtype=torch.int32, device=depth.device)
        else:
            buf, cnt = out
            capacity = buf.numel() // 56
        prm = _native.QuadParams(int(tile), int(max_level), float(tau), int(round(1000 * float(min_frac))))
        _native.check(_native.lib().sf_quadtree(self._h, n, depth.data_ptr(), ctypes.byref(prm), buf.data_ptr(),
                                                int(capacity), cnt.data_ptr(), _stream_handle(stream)))
        if not to_host:
            return buf, cnt
        total = int(cnt.item())
        if total > capacity:
            raise SurfFitError("quadtree produced %d nodes, capacity %d" % (total, capacity))
        rec = buf[:total * 56].cpu().numpy().view(np.dtype(_native.QUAD_NODE_DTYPE))
        return np.sort(rec, order=["frame", "level", "y0", "x0"])

    # -- host API (copies inside the library call) --------------------------------
    def fit_host(self, depth: np.ndarray, counts: bool = False, out=None):
        """Fit host depth [H, W] or [N, H, W] through ``sf_fit_host``; returns numpy arrays.

        ``out`` = (normals, offsets, curvature[, counts]) reuses caller-owned
        C-contiguous arrays (float32; int32 counts) instead of allocating.
        """
        want = np.float32 if self.depth_type == "f32" else np.uint16
        d = np.ascontiguousarray(depth, dtype=want)
        batched = d.ndim == 3
        n = d.shape[0] if batched else 1
        shape = (n, self.H, self.W) if batched else (self.H, self.W)
        if out is None:
            normals = np.empty(shape + (3,), np.float32)
            offsets = np.empty(shape, np.float32)
            curv = np.empty(shape, np.float32)
            cnt = np.empty(shape, np.int32) if counts else None
        else:
            normals, offsets, curv = out[:3]
            cnt = out[3] if counts else None
            want_shapes = [(normals, shape + (3,), np.float32), (offsets, shape, np.float32), (curv, shape, np.float32)]
            if counts:
                want_shapes.append((cnt, shape, np.int32))
            for a, shp, dt in want_shapes:
                if a.shape != shp or a.dtype != dt or not a.flags.c_contiguous:
                    raise ValueError("out arrays must be C-contiguous %s of shape %s" % (np.dtype(dt).name, shp))
        _native.check(_native.lib().sf_fit_host(self._h, n, d.ctypes.data, normals.ctypes.data, offsets.ctypes.data,
                                                curv.ctypes.data, cnt.ctypes.data if cnt is not None else None, None))
        return (normals, offsets, curv, cnt) if counts else (normals, offsets, curv)

    # -- profiling (CUDA events around the library's own launches) ---------------
    STAGES = ("range", "hpass", "vpass_solve", "fp64_resolve")

    def profile(self, on: bool = True) -> None:
        _native.check(_native.lib().sf_profile_enable(self._h, int(bool(on))))

    def profile_read(self):
        """{stage: (total ms, launches)} since profiling was enabled; clears the record."""
        n = len(self.STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int * n)()
        _native.check(_native.lib().sf_profile_read(self._h, n, ms, cnt))
        return {s: (ms[i], cnt[i]) for i, s in enumerate(self.STAGES)}

    def close(self) -> None:
        if getattr(self, "_h", None):
            _native.lib().sf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class SurfaceFitBatch:
    """Frames of mixed sizes and windows fitted as one pass (``sf_batch_*``).

    ``frames``: list of dicts with keys W, H, window, intrinsics (4 or 6
    values), depth (CUDA tensor [H, W]) and optionally hseg, vband (tile
    shape).  Output tensors are allocated here and stay bound to the batch
    (``outputs[i] = (normals, offsets, curvature)``); refill the depth tensors
    in place and call ``run()`` again.
    """

    def __init__(self, frames, method: str = "disparity", depth_type: str = "f32", depth_scale: float = 1e-3,
                 min_valid: int = 3, require_center: bool = True, use_graph: bool = True):
        import torch

        self.frames = frames
        self.outputs = []
        arr = (_native.BatchFrame * len(frames))()
        for i, fr in enumerate(frames):
            W, H, k = int(fr["W"]), int(fr["H"]), int(fr["window"])
            it = tuple(float(v) for v in fr["intrinsics"])
            it = it + (0.0, 0.0) if len(it) == 4 else it
            d = fr["depth"]
            if not d.is_cuda or not d.is_contiguous() or tuple(d.shape) != (H, W):
                raise ValueError("frame %d: depth must be a contiguous CUDA tensor of shape (H, W)" % i)
            dev = d.device
            out = (torch.empty((H, W, 3), device=dev), torch.empty((H, W), device=dev), torch.empty((H, W), device=dev))
            self.outputs.append(out)
            arr[i] = _native.BatchFrame(W, H, k, _native.Intrinsics(*it), d.data_ptr(), out[0].data_ptr(),
                                        out[1].data_ptr(), out[2].data_ptr(), int(fr.get("hseg", 0)),
                                        int(fr.get("vband", 0)))
        h = ctypes.c_void_p()
        _native.check(_native.lib().sf_batch_create(arr, len(frames), METHODS[method], DEPTH_TYPES[depth_type],
                                                    float(depth_scale), int(min_valid), int(bool(require_center)),
                                                    int(bool(use_graph)), ctypes.byref(h)))
        self._h = h
        px = ctypes.c_longlong()
        nl = ctypes.c_int()
        _native.check(_native.lib().sf_batch_info(self._h, ctypes.byref(px), ctypes.byref(nl)))
        self.pixels, self.launches = int(px.value), int(nl.value)

    def run(self, stream=None) -> None:
        _native.check(_native.lib().sf_batch_run(self._h, _stream_handle(stream)))

    def check(self) -> None:
        """Wait for the last pass; raise SurfFitError (SF_ERR_TIMEOUT) if one of its waits gave up."""
        _native.check(_native.lib().sf_batch_check(self._h))

    def set_wait_limit(self, polls: int) -> None:
        """Polls per wait of the following passes (0: every wait that has something to wait for gives up)."""
        _native.check(_native.lib().sf_batch_set_wait_limit(self._h, int(polls)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            _native.lib().sf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_function():
    import torch

    class FitFunction(torch.autograd.Function):
        """Autograd wrapper: forward = sf_fit_ex, backward = sf_fit_backward (both in the CUDA library)."""

        @staticmethod
        def forward(ctx, depth, fitter):
            normals, offsets, curv = fitter.fit(depth)
            ctx.save_for_backward(depth)
            ctx.fitter = fitter
            return normals, offsets, curv

        @staticmethod
        def backward(ctx, g_normals, g_offsets, g_curv):
            (depth,) = ctx.saved_tensors
            shape = depth.shape
            if g_normals is None:
                g_normals = torch.zeros(shape + (3,), device=depth.device)
            if g_offsets is None:
                g_offsets = torch.zeros(shape, device=depth.device)
            if g_curv is None:
                g_curv = torch.zeros(shape, device=depth.device)
            # autograd refuses saved tensors modified in place, so the depth is the one fitted
            return ctx.fitter.backward(depth, g_normals, g_offsets, g_curv, after_fit=True), None

    return FitFunction


class _Lazy:
    fn = None


class _FitFunctionProxy:
    @staticmethod
    def apply(depth, fitter):
        if _Lazy.fn is None:
            _Lazy.fn = _make_function()
        return _Lazy.fn.apply(depth, fitter)


_FitFunction = _FitFunctionProxy
