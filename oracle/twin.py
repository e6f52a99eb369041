"""Pure-NumPy restatement of the FP64 oracle for tiny images -- TEST INFRASTRUCTURE ONLY.

It recomputes the same quantities as ``surffit_oracle.c`` through a different
route so that the two can pin each other:

* window sums come from 2D integral images (``numpy.cumsum``, Section II.C)
  instead of direct loops;
* the scatter matrix is built as M^T M from explicit monomial rows (Eq. 6 /
  Eq. 14) for each window;
* the eigen-solve is LAPACK's ``numpy.linalg.eigh`` instead of Jacobi.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np


def integral_image(v: np.ndarray) -> np.ndarray:
    """Summed-area table with a zero row/column in front: S[y+1, x+1] = sum v[:y+1, :x+1]."""
    S = np.zeros((v.shape[0] + 1, v.shape[1] + 1) + v.shape[2:], dtype=v.dtype)
    S[1:, 1:] = np.cumsum(np.cumsum(v, axis=0), axis=1)
    return S


def box_sums(v: np.ndarray, r: int) -> np.ndarray:
    """Window sums over [x-r, x+r] x [y-r, y+r], clipped at the borders, via four taps of the SAT."""
    H, W = v.shape[:2]
    S = integral_image(v)
    y0 = np.clip(np.arange(H) - r, 0, H)
    y1 = np.clip(np.arange(H) + r + 1, 0, H)
    x0 = np.clip(np.arange(W) - r, 0, W)
    x1 = np.clip(np.arange(W) + r + 1, 0, W)
    return (S[y1][:, x1] - S[y0][:, x1] - S[y1][:, x0] + S[y0][:, x0])


def monomials(Z: np.ndarray, intr: Sequence[float], method: str):
    """Per-pixel monomial rows [u1, u2, u3, t] and validity: the rows of M in Eq. 6 / Eq. 14."""
    fx, fy, cx, cy, dx, dy = intr
    H, W = Z.shape
    tx = (np.arange(W) + dx - cx) / fx
    ty = (np.arange(H) + dy - cy) / fy
    TX = np.broadcast_to(tx[None, :], (H, W))
    TY = np.broadcast_to(ty[:, None], (H, W))
    valid = np.isfinite(Z) & (Z > 0)
    Zs = np.where(valid, Z, 1.0)
    if method == "disparity":
        rows = np.stack([TX, TY, np.ones_like(TX), 1.0 / Zs], axis=-1)
    elif method == "standard":
        rows = np.stack([Zs * TX, Zs * TY, Zs, np.ones_like(TX)], axis=-1)
    else:
        raise ValueError(method)
    rows = np.where(valid[..., None], rows, 0.0)
    return rows, valid


def scatter_sums(Z: np.ndarray, intr: Sequence[float], k: int, method: str):
    """4x4 scatter matrix M^T M of every window [H, W, 4, 4] and the counts, from integral images."""
    rows, valid = monomials(Z, intr, method)
    outer = rows[..., :, None] * rows[..., None, :]
    r = (k - 1) // 2
    S = box_sums(outer, r)
    n = box_sums(valid.astype(np.int64), r)
    return S, n, valid


def fit_np(Z: np.ndarray, intr: Sequence[float], k: int, method: str = "disparity", min_valid: int = 3,
           require_center: bool = True) -> Dict[str, np.ndarray]:
    """Implicit fit (|(a,b,c)| = 1) of every window, using eigh on the Schur complement."""
    S, n, valid = scatter_sums(Z, intr, k, method)
    H, W = Z.shape
    normals = np.full((H, W, 3), np.nan)
    offsets = np.full((H, W), np.nan)
    curv = np.full((H, W), np.nan)
    lam = np.full((H, W, 3), np.nan)
    for y in range(H):
        for x in range(W):
            ok = n[y, x] >= min_valid and n[y, x] > 0 and (valid[y, x] or not require_center)
            if not ok:
                continue
            M = S[y, x]
            A, g, s = M[:3, :3], M[:3, 3], M[3, 3]
            R = A - np.outer(g, g) / s
            l, V = np.linalg.eigh(R)
            v = V[:, 0]
            d = -v @ g / s
            if d < 0 or (d == 0 and v[2] > 0):
                v, d = -v, -d
            normals[y, x] = v
            offsets[y, x] = d
            tr = l.sum()
            curv[y, x] = l[0] / tr if tr != 0 else 0.0
            lam[y, x] = l
    return {"normals": normals, "offsets": offsets, "curvature": curv, "counts": n.astype(np.int32), "lam": lam}


def weighted_covariance(Z: np.ndarray, intr: Sequence[float], k: int, method: str, y: int, x: int) -> np.ndarray:
    """Two-pass covariance of the window's 3D points, weights 1/Z^2 (disparity) or 1 (standard).

    For the disparity form, sum (n.m + d/Z)^2 = sum (1/Z^2) (n.P + d)^2, so its
    Schur complement equals this weighted covariance; for the standard form it
    is the plain covariance (times n).
    """
    fx, fy, cx, cy, dx, dy = intr
    H, W = Z.shape
    r = (k - 1) // 2
    pts, wts = [], []
    for yy in range(max(0, y - r), min(H, y + r + 1)):
        for xx in range(max(0, x - r), min(W, x + r + 1)):
            z = Z[yy, xx]
            if not (np.isfinite(z) and z > 0):
                continue
            m = np.array([(xx + dx - cx) / fx, (yy + dy - cy) / fy, 1.0])
            pts.append(z * m)
            wts.append(1.0 / (z * z) if method == "disparity" else 1.0)
    P = np.array(pts)
    w = np.array(wts)
    mu = (w[:, None] * P).sum(0) / w.sum()
    D = P - mu
    return (w[:, None, None] * D[:, :, None] * D[:, None, :]).sum(0)
