"""FP64 CPU oracle for dense RGBD plane fitting -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and shares no code with it.

``fit`` runs the plain C oracle (``surffit_oracle.c``): direct per-window FP64
sums of the scatter-matrix monomials (Eq. 6 for the standard fit, Eq. 14 for
the disparity form, Eq. 9 / Eq. 16 for the explicit fits), the Schur
complement that eliminates the offset, and a cyclic Jacobi eigen-solve.
``twin`` holds a pure-NumPy restatement for tiny images that uses LAPACK's
``eigh`` instead of Jacobi, so each can pin the other.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "surffit_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsurffit_oracle.so")
_lib = None

METHODS = {"disparity": 0, "standard": 1, "explicit_disparity": 2, "explicit_standard": 3}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.sfo_fit.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, dp, dp, dp, ip, dp, dp, ctypes.c_int]
        lib.sfo_fit.restype = ctypes.c_int
        lib.sfo_fit_delta.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, ip, dp, dp, ctypes.c_int]
        lib.sfo_fit_delta.restype = ctypes.c_int
        lib.sfo_backward.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, dp, dp, dp, dp, ctypes.c_int]
        lib.sfo_backward.restype = ctypes.c_int
        lib.sfo_eig_sym.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.sfo_eig_sym.restype = ctypes.c_int
        lib.sfo_num_threads.argtypes = []
        lib.sfo_num_threads.restype = ctypes.c_int
        lib.sfo_fit_rect.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip]
        lib.sfo_fit_rect.restype = ctypes.c_int
        lib.sfo_fit_at.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, ip, dp, dp, ctypes.c_int]
        lib.sfo_fit_at.restype = ctypes.c_int
        lib.sfo_fit_at_delta.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, ip,
                                         dp, dp, ctypes.c_int]
        lib.sfo_fit_at_delta.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def depth_to_f64(depth: np.ndarray, depth_scale: float = 1e-3) -> np.ndarray:
    """Depth in metres as FP64: float32 converts exactly; uint16 is raw * scale (0 = missing)."""
    if depth.dtype == np.uint16:
        Z = depth.astype(np.float64) * float(depth_scale)
        Z[depth == 0] = 0.0
        return Z
    return np.ascontiguousarray(depth, dtype=np.float64)


def depth_from_disparity(D: np.ndarray, alpha: float, beta: float) -> np.ndarray:
    """FP64 depth (metres, 0 = missing) of raw disparity D under the sensor model 1/Z = alpha D + beta
    (the disparity input of the paper's conclusion); D == 0 or 1/Z <= 0 is missing."""
    D = np.asarray(D).astype(np.float64)
    w = alpha * D + beta
    ok = (D != 0) & (w > 0)
    Z = np.zeros(D.shape)
    Z[ok] = 1.0 / w[ok]
    return Z


def fit(depth: np.ndarray, intr: Sequence[float], k: int, method: str = "disparity", *, unit4: bool = False,
        min_valid: int = 3, require_center: bool = True, depth_scale: float = 1e-3, want_lambda: bool = False,
        want_moments: bool = False, threads: int = 0, delta=None) -> Dict[str, np.ndarray]:
    """Run the FP64 oracle on one [H, W] depth image.

    Returns a dict with ``normals`` [H,W,3], ``offsets`` [H,W], ``curvature``
    [H,W] (FP64, NaN where the validity rule fails), ``counts`` [H,W] int32
    and optionally ``lam`` [H,W,3] (eigenvalues of R, ascending) and
    ``moments`` [H,W,10] (A11 A12 A13 A22 A23 A33 g1 g2 g3 s).
    ``delta`` = (ddx, ddy), per-pixel adjustments [H, W] in pixels added to
    the intrinsics' (dx, dy) in the rays of Eq. 1 / Eq. 10, or None.
    """
    lib = _load()
    Z = np.ascontiguousarray(depth_to_f64(depth, depth_scale))
    H, W = Z.shape
    it = np.ascontiguousarray(np.asarray(intr, dtype=np.float64))
    assert it.shape == (6,)
    normals = np.empty((H, W, 3))
    offsets = np.empty((H, W))
    curv = np.empty((H, W))
    counts = np.empty((H, W), dtype=np.int32)
    lam = np.empty((H, W, 3)) if want_lambda else None
    mom = np.empty((H, W, 10)) if want_moments else None
    if delta is None:
        ddx = ddy = None
    else:
        ddx, ddy = (np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in delta)
        if ddx.shape != (H, W) or ddy.shape != (H, W):
            raise ValueError("delta tables must be [H, W]")
    rc = lib.sfo_fit_delta(_dp(Z), W, H, _dp(it), _dp(ddx) if ddx is not None else None,
                           _dp(ddy) if ddy is not None else None, int(k), METHODS[method], int(unit4),
                           int(min_valid), int(require_center), _dp(normals), _dp(offsets), _dp(curv),
                           counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           _dp(lam) if lam is not None else None, _dp(mom) if mom is not None else None,
                           int(threads))
    if rc != 0:
        raise ValueError("oracle rejected its arguments (rc=%d)" % rc)
    out = {"normals": normals, "offsets": offsets, "curvature": curv, "counts": counts}
    if lam is not None:
        out["lam"] = lam
    if mom is not None:
        out["moments"] = mom
    return out


def fit_at(depth: np.ndarray, intr: Sequence[float], k: int, xy: np.ndarray, method: str = "disparity", *,
           unit4: bool = False, min_valid: int = 3, require_center: bool = True, depth_scale: float = 1e-3,
           threads: int = 0, delta=None) -> Dict[str, np.ndarray]:
    """``fit`` evaluated at the pixels xy [N, 2] (x, y) only: the same dict with a leading N axis
    (lam and moments always included); ``delta`` as for ``fit``."""
    lib = _load()
    Z = np.ascontiguousarray(depth_to_f64(depth, depth_scale))
    H, W = Z.shape
    it = np.ascontiguousarray(np.asarray(intr, dtype=np.float64))
    pts = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    n = pts.shape[0]
    normals, offsets, curv = np.empty((n, 3)), np.empty(n), np.empty(n)
    counts = np.empty(n, dtype=np.int32)
    lam, mom = np.empty((n, 3)), np.empty((n, 10))
    ip = ctypes.POINTER(ctypes.c_int32)
    if delta is None:
        ddx = ddy = None
    else:
        ddx, ddy = (np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in delta)
        if ddx.shape != (H, W) or ddy.shape != (H, W):
            raise ValueError("delta tables must be [H, W]")
    rc = lib.sfo_fit_at_delta(_dp(Z), W, H, _dp(it), _dp(ddx) if ddx is not None else None,
                              _dp(ddy) if ddy is not None else None, int(k), METHODS[method], int(unit4),
                              int(min_valid), int(require_center), n, pts.ctypes.data_as(ip), _dp(normals),
                              _dp(offsets), _dp(curv), counts.ctypes.data_as(ip), _dp(lam), _dp(mom), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected its arguments (rc=%d)" % rc)
    return {"normals": normals, "offsets": offsets, "curvature": curv, "counts": counts, "lam": lam, "moments": mom}


def backward(depth: np.ndarray, intr: Sequence[float], k: int, g_normals: np.ndarray, g_offsets: np.ndarray,
             g_curv: np.ndarray, method: str = "disparity", *, min_valid: int = 3, require_center: bool = True,
             depth_scale: float = 1e-3, threads: int = 0) -> np.ndarray:
    """FP64 analytic gradient of sum(g_n . n + g_d * d + g_k * kappa) with respect to depth [H, W]."""
    lib = _load()
    Z = np.ascontiguousarray(depth_to_f64(depth, depth_scale))
    H, W = Z.shape
    it = np.ascontiguousarray(np.asarray(intr, dtype=np.float64))
    gn = np.ascontiguousarray(np.nan_to_num(g_normals.astype(np.float64)))
    gd = np.ascontiguousarray(np.nan_to_num(g_offsets.astype(np.float64)))
    gk = np.ascontiguousarray(np.nan_to_num(g_curv.astype(np.float64)))
    out = np.empty((H, W))
    rc = lib.sfo_backward(_dp(Z), W, H, _dp(it), int(k), METHODS[method], int(min_valid), int(require_center),
                          _dp(gn), _dp(gd), _dp(gk), _dp(out), int(threads))
    if rc != 0:
        raise ValueError("oracle backward rejected its arguments (rc=%d)" % rc)
    return out


def eig_sym(m: np.ndarray):
    """The oracle's Jacobi eigen-decomposition of one symmetric matrix: (lam ascending, vecs rows)."""
    lib = _load()
    n = m.shape[0]
    a = np.ascontiguousarray(m, dtype=np.float64)
    lam = np.empty(n)
    vec = np.empty((n, n))
    lib.sfo_eig_sym(n, _dp(a), _dp(lam), _dp(vec))
    return lam, vec


def num_threads() -> int:
    return int(_load().sfo_num_threads())


def fit_rect(Z: np.ndarray, intr: Sequence[float], x0: int, y0: int, w: int, h: int, method: str = "disparity",
             min_valid: int = 3) -> Dict[str, object]:
    """The fit of the pixels [x0, x0 + w) x [y0, y0 + h) of an FP64 depth image (metres).

    Returns ``ok``, ``count``, ``normal``, ``offset``, ``curvature`` (mean squared residual for the
    explicit fits), ``lam`` (eigenvalues of R) and ``residual`` (the minimised residual sum: lambda0
    of R for the implicit fits, the residual sum of squares for the explicit ones).
    """
    lib = _load()
    H, W = Z.shape
    it = np.ascontiguousarray(np.asarray(intr, dtype=np.float64))
    out = np.empty(9)
    cnt = np.zeros(1, np.int32)
    rc = lib.sfo_fit_rect(_dp(Z), W, H, _dp(it), int(x0), int(y0), int(w), int(h), METHODS[method],
                          int(min_valid), _dp(out), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc < 0:
        raise ValueError("oracle rejected the rectangle")
    return {"ok": rc == 1, "count": int(cnt[0]), "normal": out[0:3].copy(), "offset": float(out[3]),
            "curvature": float(out[4]), "lam": out[5:8].copy(), "residual": float(out[8])}


# Node status of the planar segmentation (Section III): a plane that fits, a
# tile split into four, a tile whose fit error stays above the threshold at
# the deepest level, and a tile with too few valid pixels.
QUAD_FIT, QUAD_SPLIT, QUAD_HIGH_ERROR, QUAD_INVALID = 0, 1, 2, 3


def quadtree(depth: np.ndarray, intr: Sequence[float], method: str = "disparity", *, tile: int = 64,
             max_level: int = 3, tau: float = 1e-3, min_valid_permille: int = 500, min_valid: int = 3,
             depth_scale: float = 1e-3) -> list:
    """Planar segmentation by tile subdivision (Section III, planar segmentation application).

    The image is cut into tile x tile squares from the top-left corner (clipped at the right and
    bottom borders).  A node with fewer than max(min_valid, ceil(permille * area / 1000)) valid
    pixels, or whose valid pixels are collinear in the image, is INVALID.  Otherwise its plane is fitted over all its valid pixels, and its error is the
    root mean square of the residual the method minimises, e = sqrt(residual / n) (for the implicit
    fits lambda0 of R: the algebraic distance over depth for the disparity form, the point-to-plane
    distance in metres for the standard form).  If e > tau the node splits into four children of
    half its width and height (left/top halves floor(w/2), floor(h/2)) while level < max_level and
    w, h >= 2; otherwise it is a FIT leaf (e <= tau) or a HIGH_ERROR leaf.

    Returns every evaluated node in breadth-first order as dicts with x0, y0, w, h, level, status,
    count, normal, offset, curvature, rms, lam (eigenvalues of R, NaN for explicit fits).
    """
    Z = np.ascontiguousarray(depth_to_f64(depth, depth_scale))
    H, W = Z.shape
    level_nodes = [(x0, y0, min(tile, W - x0), min(tile, H - y0)) for y0 in range(0, H, tile)
                   for x0 in range(0, W, tile)]
    out = []
    for level in range(max_level + 1):
        nxt = []
        for (x0, y0, w, h) in level_nodes:
            need = max(min_valid, (min_valid_permille * w * h + 999) // 1000)
            r = fit_rect(Z, intr, x0, y0, w, h, method, min_valid=need)
            node = {"x0": x0, "y0": y0, "w": w, "h": h, "level": level, "count": r["count"],
                    "normal": r["normal"], "offset": r["offset"], "curvature": r["curvature"], "rms": np.nan,
                    "lam": r["lam"]}
            if not r["ok"]:
                node["status"] = QUAD_INVALID
            else:
                node["rms"] = float(np.sqrt(max(r["residual"], 0.0) / r["count"]))
                if node["rms"] > tau and level < max_level and w >= 2 and h >= 2:
                    node["status"] = QUAD_SPLIT
                    w1, h1 = w // 2, h // 2
                    nxt += [(x0, y0, w1, h1), (x0 + w1, y0, w - w1, h1), (x0, y0 + h1, w1, h - h1),
                            (x0 + w1, y0 + h1, w - w1, h - h1)]
                else:
                    node["status"] = QUAD_FIT if node["rms"] <= tau else QUAD_HIGH_ERROR
            out.append(node)
        level_nodes = nxt
    return out
