"""Seeded synthetic depth scenes for the plane-fitting hot path.

This module only makes inputs.  It holds none of the fitting arithmetic, so the
FP64 oracle and the CUDA path can both be fed from it without sharing code.

The paper's own workload (Section III, first paragraph) is a virtual 640x480
depth camera: a ray through the centre of every pixel is intersected with a 3D
plane and the hit is perturbed with Gaussian noise along the measurement
direction.  The generators below follow that recipe and extend it to
piecewise-planar scenes (Voronoi cells, each its own plane), an optional
sphere, missing pixels (i.i.d. or discs) and disparity quantisation, so that
the window statistics look like Kinect-style frames.

Camera convention (Eq. 1 and Eq. 10): pixel (x, y), x the column and y the
row, both 0-based integers at the pixel centre; the ray through it is
m = [(x + dx - cx)/fx, (y + dy - cy)/fy, 1] and the 3D point at depth Z is Z*m.

Every random draw comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 20170101

# Kinect depth-noise slope of Eq. 2 (sigma_Z = 1.425e-3 * Z^2).
KINECT_SIGMA_COEF = 1.425e-3


@dataclasses.dataclass(frozen=True)
class Intrinsics:
    """Pinhole intrinsics of Eq. 1: focal lengths, principal point, offsets."""

    fx: float
    fy: float
    cx: float
    cy: float
    dx: float = 0.0
    dy: float = 0.0

    def as_tuple(self) -> Tuple[float, float, float, float, float, float]:
        return (self.fx, self.fy, self.cx, self.cy, self.dx, self.dy)

    @staticmethod
    def scaled(W: int, H: int, f640: float = 525.0) -> "Intrinsics":
        """Intrinsics scaled with the image width: f = f640 * W / 640, centre at the middle."""
        f = f640 * W / 640.0
        return Intrinsics(f, f, (W - 1) / 2.0, (H - 1) / 2.0)


@dataclasses.dataclass
class Plane:
    """Plane n.P + d = 0 with unit n and d > 0 (the camera sits on the d > 0 side)."""

    n: np.ndarray
    d: float


def rays(intr: Intrinsics, W: int, H: int) -> Tuple[np.ndarray, np.ndarray]:
    """Ray tangents tan(theta_x)[W] and tan(theta_y)[H] of Eq. 10 (FP64)."""
    tx = (np.arange(W, dtype=np.float64) + intr.dx - intr.cx) / intr.fx
    ty = (np.arange(H, dtype=np.float64) + intr.dy - intr.cy) / intr.fy
    return tx, ty


def delta_table(seed: int, intr: Intrinsics, W: int, H: int, amp: float = 1.5) -> Tuple[np.ndarray, np.ndarray]:
    """Per-pixel ray adjustments (ddx, ddy) [H, W] in pixels, float32: a radial field (a stand-in for
    lens distortion, up to `amp` px at the corners) plus a seeded ripple, inside +-16 px."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (np.arange(W, dtype=np.float64) - intr.cx)[None, :]
    y = (np.arange(H, dtype=np.float64) - intr.cy)[:, None]
    rho2 = (x / max(W / 2.0, 1.0)) ** 2 + (y / max(H / 2.0, 1.0)) ** 2
    k1 = amp * 0.5 * rng.uniform(0.5, 1.0)
    ddx = k1 * rho2 * x / max(W / 2.0, 1.0)
    ddy = k1 * rho2 * y / max(H / 2.0, 1.0)
    ph = rng.uniform(0, 2 * np.pi, 2)
    ddx = ddx + 0.2 * amp * np.sin(0.05 * y + 0.03 * x + ph[0])
    ddy = ddy + 0.2 * amp * np.cos(0.04 * x - 0.02 * y + ph[1])
    c = lambda a: np.clip(a, -15.99, 15.99).astype(np.float32)
    return c(ddx), c(ddy)


def plane_depth_delta(plane: "Plane", intr: Intrinsics, ddx: np.ndarray, ddy: np.ndarray) -> np.ndarray:
    """plane_depth with per-pixel rays (x + dx + ddx - cx)/fx, (y + dy + ddy - cy)/fy."""
    H, W = ddx.shape
    tx = (np.arange(W, dtype=np.float64)[None, :] + intr.dx + ddx - intr.cx) / intr.fx
    ty = (np.arange(H, dtype=np.float64)[:, None] + intr.dy + ddy - intr.cy) / intr.fy
    denom = plane.n[0] * tx + plane.n[1] * ty + plane.n[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        Z = -plane.d / denom
    Z[~(denom < 0)] = np.inf
    return Z


def _random_normal_toward_camera(rng: np.random.Generator, max_tilt_deg: float) -> np.ndarray:
    """Unit normal tilted from -Z by U[0, max_tilt] at a uniform azimuth."""
    tilt = math.radians(rng.uniform(0.0, max_tilt_deg))
    az = rng.uniform(0.0, 2.0 * math.pi)
    return np.array([math.sin(tilt) * math.cos(az), math.sin(tilt) * math.sin(az), -math.cos(tilt)])


def plane_through(point: np.ndarray, n: np.ndarray) -> Plane:
    """Plane with normal n through a 3D point, oriented so that d > 0."""
    n = n / np.linalg.norm(n)
    d = -float(n @ point)
    if d < 0:
        n, d = -n, -d
    return Plane(n, d)


def plane_depth(plane: Plane, intr: Intrinsics, W: int, H: int) -> np.ndarray:
    """Exact depth of the ray/plane intersection at every pixel, FP64 [H, W].

    With n.(Z m) + d = 0, Z = -d / (n.m).  Rays that miss the plane (n.m >= 0)
    get +inf.
    """
    tx, ty = rays(intr, W, H)
    denom = plane.n[0] * tx[None, :] + plane.n[1] * ty[:, None] + plane.n[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        Z = np.where(denom < 0, -plane.d / denom, np.inf)
    return Z


def sphere_depth(center: np.ndarray, radius: float, intr: Intrinsics, W: int, H: int) -> np.ndarray:
    """Depth of the nearest hit of each pixel ray with a sphere, +inf on a miss."""
    tx, ty = rays(intr, W, H)
    mx = np.broadcast_to(tx[None, :], (H, W))
    my = np.broadcast_to(ty[:, None], (H, W))
    # |Z m - c|^2 = r^2  ->  Z^2 |m|^2 - 2 Z m.c + |c|^2 - r^2 = 0
    a = mx * mx + my * my + 1.0
    b = -2.0 * (mx * center[0] + my * center[1] + center[2])
    c = float(center @ center) - radius * radius
    disc = b * b - 4 * a * c
    with np.errstate(invalid="ignore"):
        z = (-b - np.sqrt(disc)) / (2 * a)
    return np.where((disc >= 0) & (z > 0), z, np.inf)


def voronoi_planes(
    rng: np.random.Generator,
    intr: Intrinsics,
    W: int,
    H: int,
    n_planes: int,
    z_lo: float,
    z_hi: float,
    max_tilt_deg: float = 60.0,
) -> Tuple[np.ndarray, np.ndarray, List[Plane]]:
    """Piecewise-planar depth: Voronoi cells of random seed pixels, one plane each.

    Returns (Z [H,W] FP64 with +inf where missing, labels [H,W] int32, planes).
    Depth outside [z_lo, z_hi] becomes missing (+inf).
    """
    sx = rng.integers(0, W, size=n_planes)
    sy = rng.integers(0, H, size=n_planes)
    tx, ty = rays(intr, W, H)
    planes: List[Plane] = []
    for j in range(n_planes):
        z0 = rng.uniform(z_lo, z_hi)
        p0 = z0 * np.array([tx[sx[j]], ty[sy[j]], 1.0])
        planes.append(plane_through(p0, _random_normal_toward_camera(rng, max_tilt_deg)))
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = (xx[None] - sx[:, None, None]) ** 2 + (yy[None] - sy[:, None, None]) ** 2
    labels = np.argmin(d2, axis=0).astype(np.int32)
    Z = np.full((H, W), np.inf)
    for j, pl in enumerate(planes):
        Zj = plane_depth(pl, intr, W, H)
        sel = labels == j
        Z[sel] = Zj[sel]
    Z[(Z < z_lo) | (Z > z_hi)] = np.inf
    return Z, labels, planes


def add_depth_noise(rng: np.random.Generator, Z: np.ndarray, coef: float) -> np.ndarray:
    """Gaussian noise along the ray, sigma_Z = coef * Z^2 (Eq. 2); the pixel stays fixed."""
    finite = np.isfinite(Z)
    out = Z.copy()
    out[finite] = Z[finite] + rng.standard_normal(int(finite.sum())) * coef * Z[finite] ** 2
    return out


def drop_iid(rng: np.random.Generator, Z: np.ndarray, frac: float) -> np.ndarray:
    """Mark exactly round(frac*N) pixels missing, chosen by a seeded permutation."""
    out = Z.copy()
    n = int(round(frac * Z.size))
    if n:
        idx = rng.permutation(Z.size)[:n]
        out.reshape(-1)[idx] = np.inf
    return out


def drop_blobs(rng: np.random.Generator, Z: np.ndarray, frac: float, r_lo: float = 3.0, r_hi: float = 30.0) -> np.ndarray:
    """Mark discs of radius U[r_lo, r_hi] missing until at least frac of the pixels are."""
    H, W = Z.shape
    out = Z.copy()
    miss = ~np.isfinite(out)
    target = frac * Z.size
    yy, xx = np.mgrid[0:H, 0:W]
    guard = 0
    while miss.sum() < target and guard < 100000:
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        rad = rng.uniform(r_lo, r_hi)
        x0, x1 = max(0, int(cx - rad) - 1), min(W, int(cx + rad) + 2)
        y0, y1 = max(0, int(cy - rad) - 1), min(H, int(cy + rad) + 2)
        sub = (xx[y0:y1, x0:x1] - cx) ** 2 + (yy[y0:y1, x0:x1] - cy) ** 2 <= rad * rad
        miss[y0:y1, x0:x1] |= sub
        guard += 1
    out[miss] = np.inf
    return out


def quantize_disparity_mm(Z: np.ndarray, f: float, baseline: float = 0.075, subpix: float = 8.0) -> np.ndarray:
    """Structured-light style quantisation, stored as uint16 millimetres (0 = missing).

    D = f*B/Z is rounded to 1/subpix of a pixel, turned back into depth and
    rounded to whole millimetres.
    """
    out = np.zeros(Z.shape, dtype=np.uint16)
    fin = np.isfinite(Z) & (Z > 0)
    D = f * baseline / Z[fin]
    Dq = np.round(D * subpix) / subpix
    ok = Dq > 0
    Zq = np.zeros_like(D)
    Zq[ok] = f * baseline / Dq[ok]
    mm = np.clip(np.round(Zq * 1000.0), 0, 65535).astype(np.uint16)
    out[fin] = mm
    return out


def to_f32_metres(Z: np.ndarray) -> np.ndarray:
    """FP32 depth in metres with 0 marking missing pixels."""
    out = np.where(np.isfinite(Z) & (Z > 0), Z, 0.0).astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# Frame recipes for the workloads.
# ---------------------------------------------------------------------------

def single_plane_frame(seed: int, intr: Intrinsics, W: int, H: int, z_lo=0.8, z_hi=4.0,
                       noise_coef: float = 0.0, max_tilt_deg: float = 60.0) -> Tuple[np.ndarray, Plane]:
    """One plane filling the view (the paper's experiment), optional noise. Returns (Z f64, plane)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z0 = rng.uniform(z_lo, z_hi)
    tx, ty = rays(intr, W, H)
    p0 = z0 * np.array([tx[W // 2], ty[H // 2], 1.0])
    pl = plane_through(p0, _random_normal_toward_camera(rng, max_tilt_deg))
    Z = plane_depth(pl, intr, W, H)
    if noise_coef > 0:
        Z = add_depth_noise(rng, Z, noise_coef)
    return Z, pl


def kinect_frame(seed: int, intr: Intrinsics, W: int, H: int, n_planes: int = 3, z_lo: float = 0.8,
                 z_hi: float = 4.0, noise_coef: float = 0.0012, missing_iid: float = 0.05) -> np.ndarray:
    """Voronoi planes + noise + i.i.d. missing pixels, FP32 metres (0 = missing)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z, _, _ = voronoi_planes(rng, intr, W, H, n_planes, z_lo, z_hi)
    Z = add_depth_noise(rng, Z, noise_coef)
    Z = drop_iid(rng, Z, missing_iid)
    return to_f32_metres(Z)


def structured_light_frame(seed: int, intr: Intrinsics, W: int, H: int, planes_lo: int = 4, planes_hi: int = 8,
                           z_lo: float = 0.5, z_hi: float = 6.0, miss_lo: float = 0.03,
                           miss_hi: float = 0.10) -> np.ndarray:
    """Voronoi planes + one sphere, disparity-quantised, blob holes; uint16 millimetres."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = int(rng.integers(planes_lo, planes_hi + 1))
    Z, _, _ = voronoi_planes(rng, intr, W, H, k, z_lo, z_hi)
    tx, ty = rays(intr, W, H)
    px, py = int(rng.integers(0, W)), int(rng.integers(0, H))
    zc = rng.uniform(1.0, 4.0)
    c = zc * np.array([tx[px], ty[py], 1.0])
    Zs = sphere_depth(c, rng.uniform(0.2, 0.5), intr, W, H)
    Z = np.minimum(Z, Zs)
    Z = quantize_disparity_mm(Z, intr.fx)
    Zf = Z.astype(np.float64) / 1000.0
    Zf[Z == 0] = np.inf
    Zf = drop_blobs(rng, Zf, rng.uniform(miss_lo, miss_hi))
    out = np.where(np.isfinite(Zf), np.round(Zf * 1000.0), 0).astype(np.uint16)
    return out


def wide_range_frame(seed: int, intr: Intrinsics, W: int, H: int, n_planes: int = 6, z_lo: float = 0.3,
                     z_hi: float = 10.0, noise_coef: float = 0.0015, missing_iid: float = 0.05) -> np.ndarray:
    """Depths spanning 0.3-10 m (precision stress), FP32 metres."""
    return kinect_frame(seed, intr, W, H, n_planes, z_lo, z_hi, noise_coef, missing_iid)


def mixed_frame(seed: int, W: int, H: int, miss_hi: float = 0.15) -> Tuple[np.ndarray, Intrinsics]:
    """Mixed-batch frame: intrinsics scaled with the resolution, 0-15% blob holes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    intr = Intrinsics.scaled(W, H)
    n_planes = int(rng.integers(3, 9))
    Z, _, _ = voronoi_planes(rng, intr, W, H, n_planes, 0.5, 6.0)
    Z = add_depth_noise(rng, Z, 0.0012)
    Z = drop_blobs(rng, Z, rng.uniform(0.0, miss_hi), 3.0, 30.0 * W / 640.0)
    return to_f32_metres(Z), intr


def mixed_batch_spec(n_frames: int = 64, seed: int = BASE_SEED,
                     resolutions: Sequence[Tuple[int, int]] = ((320, 240), (640, 480), (1280, 720), (1920, 1080)),
                     windows: Sequence[int] = (5, 7, 11, 21)) -> List[Tuple[int, int, int]]:
    """(W, H, k) for each frame of the mixed batch, drawn uniformly from the sets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_frames):
        W, H = resolutions[int(rng.integers(0, len(resolutions)))]
        k = int(windows[int(rng.integers(0, len(windows)))])
        out.append((W, H, k))
    return out


def target_normals(seed: int, H: int, W: int) -> np.ndarray:
    """Seeded unit target normals [H, W, 3] with n_z < 0 (for the differentiable loss)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((H, W, 3))
    v[..., 2] = -np.abs(v[..., 2]) - 0.5
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


# Time-of-flight camera of the paper's segmentation experiment (Section III):
# 512 x 424 depth frames; intrinsics of that sensor class.
SEG_W, SEG_H = 512, 424
SEG_INTRINSICS = Intrinsics(365.0, 365.0, 255.5, 211.5)


def segmentation_frame(seed: int, intr: Intrinsics = SEG_INTRINSICS, W: int = SEG_W, H: int = SEG_H,
                       planes_lo: int = 6, planes_hi: int = 10, z_lo: float = 0.5, z_hi: float = 4.5,
                       noise_coef: float = KINECT_SIGMA_COEF, miss_lo: float = 0.02,
                       miss_hi: float = 0.08) -> np.ndarray:
    """A room-like piecewise-planar frame for the planar segmentation: 6-10 Voronoi planes at
    0.5-4.5 m, noise 1.425e-3 Z^2 (Eq. 2), 2-8 % blob holes; float32 metres (0 = missing)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = int(rng.integers(planes_lo, planes_hi + 1))
    Z, _, _ = voronoi_planes(rng, intr, W, H, k, z_lo, z_hi)
    Z = add_depth_noise(rng, Z, noise_coef)
    Z = drop_blobs(rng, Z, rng.uniform(miss_lo, miss_hi))
    return to_f32_metres(Z)


def two_plane_frame(intr: Intrinsics, W: int, H: int, split_x: int, n_left, d_left, n_right,
                    d_right) -> np.ndarray:
    """Noise-free depth of two planes n.P + d = 0 meeting at column split_x (FP64 metres)."""
    left = plane_depth(Plane(np.asarray(n_left, float), float(d_left)), intr, W, H)
    right = plane_depth(Plane(np.asarray(n_right, float), float(d_right)), intr, W, H)
    Z = np.where(np.arange(W)[None, :] < split_x, left, right)
    return Z


# Raw disparity sensors (1/Z = alpha D + beta).  Stereo: D in 1/8 px of a pair
# of baseline 0.075 m, alpha = 1 / (8 f B), beta = 0.  A structured-light
# sensor of the Kinect class reports an 11-bit code with a negative alpha.
KINECT_RAW_ALPHA, KINECT_RAW_BETA = -0.0030711, 3.3309


def disparity_frame(seed: int, intr: Intrinsics, W: int, H: int, alpha: float, beta: float,
                    planes_lo: int = 4, planes_hi: int = 8, z_lo: float = 0.5, z_hi: float = 6.0,
                    noise_coef: float = KINECT_SIGMA_COEF, miss_lo: float = 0.02,
                    miss_hi: float = 0.08, d_max: int = 65535) -> np.ndarray:
    """Voronoi planes + Eq. 2 noise + blob holes as a raw disparity image: D = round((1/Z - beta) / alpha),
    uint16, 0 where missing or outside [1, d_max]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = int(rng.integers(planes_lo, planes_hi + 1))
    Z, _, _ = voronoi_planes(rng, intr, W, H, k, z_lo, z_hi)
    Z = add_depth_noise(rng, Z, noise_coef)
    Z = drop_blobs(rng, Z, rng.uniform(miss_lo, miss_hi))
    ok = np.isfinite(Z) & (Z > 0)
    D = np.zeros(Z.shape)
    D[ok] = np.round((1.0 / Z[ok] - beta) / alpha)
    D[(D < 1) | (D > d_max)] = 0
    return D.astype(np.uint16)
