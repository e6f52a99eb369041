"""Pins for the FP64 oracle: closed forms, brute force, LAPACK and identities.

Each test checks the oracle against something other than itself, so that a
dropped term, a wrong sign, a transposed operand or a wrong index in
``oracle/surffit_oracle.c`` fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import twin
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _angle(a, b):
    """Angle between unit vectors, accurate near 0 (atan2 of |a x b| and a.b)."""
    a, b = np.broadcast_arrays(a, b)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def _random_intr(rng, W, H):
    f = rng.uniform(300, 1500)
    return scenes.Intrinsics(f * rng.uniform(0.9, 1.1), f, (W - 1) / 2 + rng.uniform(-5, 5),
                             (H - 1) / 2 + rng.uniform(-5, 5), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5))


# ---------------------------------------------------------------------------
# Closed form: noise-free planar depth is fitted exactly (Eq. 3 and Eq. 12).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["disparity", "standard"])
@pytest.mark.parametrize("k", [3, 5, 7])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_noise_free_plane_is_recovered(method, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    W, H = 24, 18
    intr = _random_intr(rng, W, H)
    Z, pl = scenes.single_plane_frame(seed, intr, W, H)
    o = oracle.fit(Z, intr.as_tuple(), k, method, want_lambda=True)
    ok = np.isfinite(o["offsets"])
    assert ok.all()
    ang = _angle(o["normals"], pl.n[None, None, :])
    assert np.nanmax(ang) < 1e-8
    assert np.max(np.abs(o["offsets"] - pl.d)) < 1e-8 * pl.d
    assert np.max(o["curvature"]) < 1e-9
    assert np.max(np.abs(o["lam"][..., 0]) / o["lam"][..., 2]) < 1e-9


@pytest.mark.parametrize("method", ["explicit_disparity", "explicit_standard"])
def test_noise_free_plane_explicit(method):
    intr = scenes.Intrinsics(525, 525, 11.5, 8.5)
    Z, pl = scenes.single_plane_frame(7, intr, 24, 18, max_tilt_deg=50)
    o = oracle.fit(Z, intr.as_tuple(), 5, method)
    assert np.nanmax(_angle(o["normals"], pl.n[None, None, :])) < 1e-8
    assert np.max(np.abs(o["offsets"] - pl.d)) < 1e-8 * pl.d
    assert np.max(np.abs(o["curvature"])) < 1e-12 * max(1.0, np.max(Z) ** 2)


def test_noise_free_plane_unit4_literal_constraint():
    intr = scenes.Intrinsics(525, 525, 11.5, 8.5)
    Z, pl = scenes.single_plane_frame(3, intr, 24, 18)
    for method in ("disparity", "standard"):
        o = oracle.fit(Z, intr.as_tuple(), 5, method, unit4=True)
        assert np.nanmax(_angle(o["normals"], pl.n[None, None, :])) < 1e-7
        assert np.max(np.abs(o["offsets"] - pl.d)) < 1e-7 * pl.d


def test_rgbd_plane_equals_xyz_plane():
    """Eq. 12 is Eq. 3 divided by Z: both fits give the same (n, d) on a plane."""
    intr = scenes.Intrinsics(600, 610, 15.3, 11.1, 0.25, -0.25)
    Z, pl = scenes.single_plane_frame(11, intr, 32, 24)
    a = oracle.fit(Z, intr.as_tuple(), 7, "disparity")
    b = oracle.fit(Z, intr.as_tuple(), 7, "standard")
    assert np.max(_angle(a["normals"], b["normals"])) < 1e-8
    assert np.max(np.abs(a["offsets"] - b["offsets"])) < 1e-8


# ---------------------------------------------------------------------------
# Brute force and integral images: window sums and counts.
# ---------------------------------------------------------------------------
def _tiny_depth(seed, W, H, frac_missing=0.2):
    rng = np.random.Generator(np.random.PCG64(seed))
    Z = rng.uniform(0.5, 4.0, size=(H, W))
    Z[rng.random((H, W)) < frac_missing] = 0.0
    Z[0, 0] = np.nan
    Z[-1, -1] = -1.0
    return Z


@pytest.mark.parametrize("W,H,k", [(8, 6, 3), (16, 12, 5), (16, 12, 3), (7, 9, 5)])
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_window_moments_match_integral_images(W, H, k, method):
    Z = _tiny_depth(W * 100 + H, W, H)
    intr = (500.0, 510.0, (W - 1) / 2, (H - 1) / 2, 0.1, -0.2)
    o = oracle.fit(Z, intr, k, method, want_moments=True, min_valid=1, require_center=False)
    S, n, _ = twin.scatter_sums(Z, intr, k, method)
    mo = o["moments"]
    ref = np.stack([S[..., 0, 0], S[..., 0, 1], S[..., 0, 2], S[..., 1, 1], S[..., 1, 2], S[..., 2, 2],
                    S[..., 0, 3], S[..., 1, 3], S[..., 2, 3], S[..., 3, 3]], axis=-1)
    scale = np.maximum(np.abs(ref), 1e-300)
    assert np.max(np.abs(mo - ref) / np.maximum(scale, np.max(np.abs(ref)) * 1e-3)) < 1e-12
    assert np.array_equal(o["counts"], n.astype(np.int32))


def test_counts_brute_force_and_validity_rule():
    W, H, k = 13, 11, 5
    Z = _tiny_depth(5, W, H, 0.4)
    intr = (300.0, 300.0, 6.0, 5.0, 0.0, 0.0)
    r = k // 2
    for min_valid, center in [(3, True), (1, False), (10, True), (25, False)]:
        o = oracle.fit(Z, intr, k, "disparity", min_valid=min_valid, require_center=center)
        for y in range(H):
            for x in range(W):
                n = 0
                for yy in range(y - r, y + r + 1):
                    for xx in range(x - r, x + r + 1):
                        if 0 <= yy < H and 0 <= xx < W and np.isfinite(Z[yy, xx]) and Z[yy, xx] > 0:
                            n += 1
                assert o["counts"][y, x] == n
                c_ok = np.isfinite(Z[y, x]) and Z[y, x] > 0
                valid = n >= min_valid and (c_ok or not center)
                assert np.isfinite(o["offsets"][y, x]) == valid
                assert np.all(np.isfinite(o["normals"][y, x]) == valid)


# ---------------------------------------------------------------------------
# LAPACK: the Jacobi eigen-solver and the whole fit against numpy.linalg.eigh.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 4])
def test_jacobi_matches_lapack(n):
    rng = np.random.Generator(np.random.PCG64(42 + n))
    for _ in range(200):
        B = rng.standard_normal((n, n)) * rng.uniform(1e-6, 1e3)
        M = B @ B.T
        if rng.random() < 0.3:  # near-singular, like a planar window
            u = rng.standard_normal(n)
            M = M - (M @ u)[:, None] * (M @ u)[None, :] / (u @ M @ u) * (1 - 1e-9)
            M = 0.5 * (M + M.T)
        lam, vec = oracle.eig_sym(M)
        ref_l, ref_v = np.linalg.eigh(M)
        scale = np.max(np.abs(ref_l))
        assert np.max(np.abs(lam - ref_l)) <= 1e-12 * scale
        for i in range(n):
            gap = min([abs(ref_l[i] - ref_l[j]) for j in range(n) if j != i]) / scale
            if gap > 1e-6:
                c = abs(vec[i] @ ref_v[:, i])
                assert abs(1 - c) < 1e-12 / gap ** 2 + 1e-13
        # residual check independent of LAPACK
        for i in range(n):
            assert np.linalg.norm(M @ vec[i] - lam[i] * vec[i]) <= 1e-12 * scale


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_fit_matches_numpy_twin(method):
    intr = scenes.Intrinsics(525, 525, 15.5, 11.5)
    Z = scenes.kinect_frame(3, intr, 32, 24, n_planes=3, missing_iid=0.1).astype(np.float64)
    a = oracle.fit(Z, intr.as_tuple(), 5, method, want_lambda=True)
    b = twin.fit_np(Z, intr.as_tuple(), 5, method)
    assert np.array_equal(np.isfinite(a["offsets"]), np.isfinite(b["offsets"]))
    assert np.array_equal(a["counts"], b["counts"])
    ok = np.isfinite(a["offsets"])
    lam = a["lam"]
    gap = (lam[..., 1] - lam[..., 0]) / lam[..., 2]
    good = ok & (gap > 1e-4)
    assert good.sum() > 0.8 * ok.sum()
    assert np.max(_angle(a["normals"][good], b["normals"][good])) < 1e-9 / 1e-4
    assert np.max(np.abs(a["offsets"][good] - b["offsets"][good]) / np.abs(b["offsets"][good])) < 1e-6
    # The twin's FP64 summed-area tables accumulate over the whole image, so
    # their absolute error (~1e-16 of the image total) is amplified by the
    # Schur-complement cancellation (|A| / |R| ~ (f/r)^2 ~ 1e4): ~1e-8 relative.
    assert np.max(np.abs(a["curvature"][ok] - b["curvature"][ok])) < 1e-7
    assert np.max(np.abs(lam[ok] - b["lam"][ok]) / lam[ok][..., 2:3]) < 1e-7


# ---------------------------------------------------------------------------
# Identities: the Schur complement equals a two-pass (weighted) covariance.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_schur_complement_is_weighted_covariance(method):
    intr = (525.0, 525.0, 7.5, 5.5, 0.0, 0.0)
    Z = _tiny_depth(17, 16, 12, 0.15)
    o = oracle.fit(Z, intr, 5, method, want_moments=True, want_lambda=True)
    for (y, x) in [(5, 7), (0, 0), (11, 15), (6, 1), (3, 12)]:
        if not np.isfinite(o["offsets"][y, x]):
            continue
        mo = o["moments"][y, x]
        A = np.array([[mo[0], mo[1], mo[2]], [mo[1], mo[3], mo[4]], [mo[2], mo[4], mo[5]]])
        g, s = mo[6:9], mo[9]
        R = A - np.outer(g, g) / s
        C = twin.weighted_covariance(Z, intr, 5, method, y, x)
        assert np.max(np.abs(R - C)) < 1e-9 * np.max(np.abs(C))
        l = np.linalg.eigvalsh(C)
        assert np.allclose(o["lam"][y, x], l, rtol=1e-7, atol=1e-12 * l[-1])


def test_disparity_calibration_block_has_closed_form():
    """Full windows: A = sum m m^T depends only on the intrinsics (Section II.A)."""
    W, H, k = 20, 16, 5
    intr = (480.0, 470.0, 9.2, 7.7, 0.3, -0.1)
    r = k // 2
    rng = np.random.Generator(np.random.PCG64(3))
    Z1 = rng.uniform(0.5, 5.0, (H, W))
    Z2 = rng.uniform(0.5, 5.0, (H, W))
    m1 = oracle.fit(Z1, intr, k, "disparity", want_moments=True)["moments"]
    m2 = oracle.fit(Z2, intr, k, "disparity", want_moments=True)["moments"]
    fx, fy, cx, cy, dx, dy = intr
    u = np.arange(-r, r + 1)
    for (y, x) in [(5, 5), (8, 10), (r, r)]:
        tx = (x + u + dx - cx) / fx
        ty = (y + u + dy - cy) / fy
        A11 = k * np.sum(tx ** 2)
        A12 = np.sum(tx) * np.sum(ty)
        A13 = k * np.sum(tx)
        A22 = k * np.sum(ty ** 2)
        A23 = k * np.sum(ty)
        A33 = k * k
        ref = np.array([A11, A12, A13, A22, A23, A33])
        assert np.allclose(m1[y, x, :6], ref, rtol=1e-13, atol=1e-13)
        assert np.array_equal(m1[y, x, :6], m2[y, x, :6])


# ---------------------------------------------------------------------------
# Invariants on noisy Kinect-like data.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_invariants_on_noisy_frame(method):
    intr = scenes.Intrinsics(525, 525, 31.5, 23.5)
    Z = scenes.kinect_frame(9, intr, 64, 48)
    o = oracle.fit(Z, intr.as_tuple(), 7, method)
    ok = np.isfinite(o["offsets"])
    assert ok.mean() > 0.8
    nn = np.linalg.norm(o["normals"][ok], axis=-1)
    assert np.max(np.abs(nn - 1)) < 1e-12
    assert np.all(o["offsets"][ok] > 0)
    kap = o["curvature"][ok]
    assert np.all(kap >= -1e-15) and np.all(kap <= 1.0 / 3.0 + 1e-12)
    assert np.all(np.isnan(o["curvature"][~ok]))


def test_noise_statistics_sanity_band():
    """Residual of a single noisy plane: lambda0 ~ sum of squared residuals (Eq. 2 noise)."""
    intr = scenes.Intrinsics(525, 525, 63.5, 47.5)
    Z0, pl = scenes.single_plane_frame(5, intr, 128, 96, z_lo=1.5, z_hi=1.5, max_tilt_deg=0.0)
    coef = 1e-3
    rng = np.random.Generator(np.random.PCG64(77))
    Z = Z0 + rng.standard_normal(Z0.shape) * coef * Z0 ** 2
    o = oracle.fit(Z, intr.as_tuple(), 9, "standard", want_lambda=True)
    # fronto-parallel plane: residual along z, sigma = coef * Z^2
    expected = 81 * (coef * 1.5 ** 2) ** 2
    mean_l0 = np.nanmean(o["lam"][..., 0])
    assert 0.7 * expected < mean_l0 < 1.1 * expected


def test_missing_and_degenerate_inputs():
    intr = (525.0, 525.0, 3.5, 2.5, 0.0, 0.0)
    Z = np.zeros((6, 8))
    o = oracle.fit(Z, intr, 3, "disparity")
    assert np.all(np.isnan(o["offsets"])) and np.all(o["counts"] == 0)
    Z = np.full((6, 8), 2.0)
    o = oracle.fit(Z, intr, 1, "disparity")  # one point per window: below min_valid
    assert np.all(np.isnan(o["offsets"]))
    o = oracle.fit(Z, intr, 15, "standard")  # window larger than the image
    assert np.all(o["counts"] == 48)
    assert np.allclose(o["normals"][..., 2], -1.0)
    assert np.allclose(o["offsets"], 2.0)
    with pytest.raises(ValueError):
        oracle.fit(Z, intr, 4, "disparity")


def test_uint16_depth_conversion():
    raw = np.array([[0, 1000, 2000], [65535, 1, 500]], dtype=np.uint16)
    Z = oracle.depth_to_f64(raw, 1e-3)
    assert Z[0, 0] == 0.0 and Z[0, 1] == 1.0 and Z[1, 0] == 65.535 and Z[1, 1] == 1e-3


# ---------------------------------------------------------------------------
# Backward: analytic FP64 adjoint against central finite differences.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_backward_matches_finite_differences(method):
    intr = scenes.Intrinsics(525, 525, 7.5, 5.5)
    Z = scenes.kinect_frame(21, intr, 16, 12, n_planes=2, missing_iid=0.05).astype(np.float64)
    k = 5
    rng = np.random.Generator(np.random.PCG64(5))
    gn = rng.standard_normal((12, 16, 3))
    gd = rng.standard_normal((12, 16))
    gk = rng.standard_normal((12, 16)) * 10

    o0 = oracle.fit(Z, intr.as_tuple(), k, method, want_lambda=True)
    ok = np.isfinite(o0["offsets"])

    def loss(Zp):
        o = oracle.fit(Zp, intr.as_tuple(), k, method)
        assert np.array_equal(np.isfinite(o["offsets"]), ok)
        return (np.nansum(o["normals"] * gn) + np.nansum(o["offsets"] * gd) + np.nansum(o["curvature"] * gk))

    g = oracle.backward(Z, intr.as_tuple(), k, np.where(ok[..., None], gn, 0), np.where(ok, gd, 0),
                        np.where(ok, gk, 0), method)
    lam = o0["lam"]
    gap = np.where(ok, (lam[..., 1] - lam[..., 0]) / lam[..., 2], 1.0)
    checked = 0
    for y in range(12):
        for x in range(16):
            if not (np.isfinite(Z[y, x]) and Z[y, x] > 0):
                assert g[y, x] == 0.0
                continue
            # skip pixels whose windows contain near-degenerate fits (gradient ill-conditioned)
            y0, y1, x0, x1 = max(0, y - 2), min(12, y + 3), max(0, x - 2), min(16, x + 3)
            if np.min(gap[y0:y1, x0:x1]) < 1e-3:
                continue
            # Central differences, h = 1e-6 Z: the loss is computed from raw
            # FP64 moments whose Schur complement cancels ~4 digits, so the FD
            # carries ~1e-5 relative error from rounding plus truncation.
            h = 1e-6 * Z[y, x]
            Zp = Z.copy(); Zp[y, x] += h
            Zm = Z.copy(); Zm[y, x] -= h
            fd = (loss(Zp) - loss(Zm)) / (2 * h)
            assert abs(fd - g[y, x]) <= 5e-5 * max(1.0, abs(fd)), (y, x, fd, g[y, x])
            checked += 1
    assert checked > 50


# ---------------------------------------------------------------------------
# Paper numbers: cost-model channel counts (Section II.D / II.E).
# ---------------------------------------------------------------------------
def test_paper_cost_model_counts():
    with open(os.path.join(GOLDEN, "paper_cost_model.json")) as f:
        g = json.load(f)
    # Eq. 6: 9 depth-dependent unique entries; each integral image costs C + 4
    assert g["implicit_standard_depth_channels"] * 5 - 1 == g["implicit_standard_ops_per_pixel"]
    assert g["implicit_disparity_depth_channels"] * 5 == g["implicit_disparity_ops_per_pixel"]
    assert round(g["implicit_standard_ops_per_pixel"] / g["implicit_disparity_ops_per_pixel"], 1) == g["implicit_ratio"]
    assert round(g["explicit_standard_ops_per_pixel"] / g["explicit_disparity_ops_per_pixel"], 1) == g["explicit_ratio"]
    assert g["explicit_disparity_depth_channels"] * 5 == g["explicit_disparity_ops_per_pixel"]
    # Eq. 2: sigma_Z coefficient is half the disparity slope magnitude
    assert abs(g["kinect_sigma_coefficient"] - abs(g["kinect_disparity_slope"]) / 2) < 1e-12
    # The depth-dependent entries of Eq. 14 counted from the monomials: m=[tx,ty,1,1/Z]
    dep = [(i, j) for i in range(4) for j in range(i + 1) if i == 3 or j == 3]
    assert len(dep) == g["implicit_disparity_depth_channels"]
    # Eq. 6 with m=[X,Y,Z,1]: every unique entry except the 1*1 one depends on Z
    assert 10 - 1 == g["implicit_standard_depth_channels"]


# ---------------------------------------------------------------------------
# Explicit fits: rank-deficient (collinear) windows have no fit.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["explicit_disparity", "explicit_standard"])
def test_explicit_fit_undefined_on_collinear_windows(method):
    intr = (525.0, 525.0, 10.0, 0.0, 0.0, 0.0)
    Z = np.linspace(1.0, 2.0, 20)[None, :].repeat(1, 0)  # a single image row: every window collinear
    o = oracle.fit(Z, intr, 5, method)
    assert np.all(np.isnan(o["offsets"]))
    Z2 = np.full((6, 6), 2.0)
    Z2[::2, :] = 0.0  # rows 1, 3, 5 valid: 3x3 windows centred on them see one row only
    o = oracle.fit(Z2, intr, 3, method)
    assert np.all(np.isnan(o["offsets"][1::2, :]))
    o = oracle.fit(Z2, intr, 5, method, require_center=False)
    assert np.isfinite(o["offsets"][2, 2])  # two valid rows: not collinear


@pytest.mark.parametrize("method", ["explicit_disparity", "explicit_standard"])
def test_explicit_fit_is_least_squares(method):
    """Explicit fits against numpy lstsq on the design matrix of Eq. 9 / Eq. 16 (random noisy window)."""
    rng = np.random.Generator(np.random.PCG64(4))
    W, H, k = 9, 9, 7
    intr = (400.0, 410.0, 4.2, 3.9, 0.1, 0.0)
    Z = 2.0 + 0.3 * rng.random((H, W))
    Z[rng.random((H, W)) < 0.15] = 0
    Z[4, 4] = 2.1
    o = oracle.fit(Z, intr, k, method)
    fx, fy, cx, cy, dx, dy = intr
    y0 = x0 = 4
    rows, tgt = [], []
    for y in range(y0 - 3, y0 + 4):
        for x in range(x0 - 3, x0 + 4):
            z = Z[y, x]
            if z <= 0:
                continue
            tx, ty = (x + dx - cx) / fx, (y + dy - cy) / fy
            if method == "explicit_disparity":
                rows.append([tx, ty, 1.0]); tgt.append(1.0 / z)
            else:
                rows.append([z * tx, z * ty, 1.0]); tgt.append(z)
    M, b = np.array(rows), np.array(tgt)
    a, *_ = np.linalg.lstsq(M, b, rcond=None)
    res = np.sum((M @ a - b) ** 2) / len(b)
    if method == "explicit_disparity":
        v, d = a.copy(), -1.0
    else:
        v, d = np.array([a[0], a[1], -1.0]), a[2]
    nrm = np.linalg.norm(v)
    v, d = v / nrm, d / nrm
    if d < 0:
        v, d = -v, -d
    assert np.allclose(o["normals"][y0, x0], v, atol=1e-10)
    assert abs(o["offsets"][y0, x0] - d) < 1e-10 * abs(d)
    assert abs(o["curvature"][y0, x0] - res) < 1e-9 * max(res, 1e-12) + 1e-18


@pytest.mark.parametrize("method", ["disparity", "standard", "explicit_disparity", "explicit_standard"])
def test_fit_at_equals_fit_at_those_pixels(method):
    """The sampled form used at full workload sizes returns what the whole-frame fit returns there."""
    W, H, k = 97, 61, 9
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 77, intr, W, H)
    full = oracle.fit(depth, intr.as_tuple(), k, method, want_lambda=True, want_moments=True)
    rng = np.random.Generator(np.random.PCG64(5))
    xy = np.concatenate([[[0, 0], [W - 1, H - 1], [W - 1, 0], [0, H - 1]],
                         np.stack([rng.integers(0, W, 200), rng.integers(0, H, 200)], -1)])
    pts = oracle.fit_at(depth, intr.as_tuple(), k, xy, method)
    for key in ("normals", "offsets", "curvature", "counts", "lam", "moments"):
        a = np.nan_to_num(full[key][xy[:, 1], xy[:, 0]], nan=7.0)
        assert np.array_equal(a, np.nan_to_num(pts[key], nan=7.0)), key
    with pytest.raises(ValueError):
        oracle.fit_at(depth, intr.as_tuple(), k, [[W, 0]], method)
    table = scenes.delta_table(4, intr, W, H)
    full = oracle.fit(depth, intr.as_tuple(), k, method, want_lambda=True, want_moments=True, delta=table)
    pts = oracle.fit_at(depth, intr.as_tuple(), k, xy, method, delta=table)
    for key in ("normals", "offsets", "curvature", "counts", "lam", "moments"):
        a = np.nan_to_num(full[key][xy[:, 1], xy[:, 0]], nan=7.0)
        assert np.array_equal(a, np.nan_to_num(pts[key], nan=7.0)), key


def test_constant_delta_table_equals_constant_delta():
    """A per-pixel table holding one value c everywhere is the constant adjustment dx = c, dy = c
    of Eq. 1 (bit for bit: the same rays)."""
    W, H, k = 40, 30, 7
    base = scenes.Intrinsics(300.0, 310.0, 19.2, 14.7)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 33, base, W, H)
    c = (0.375, -0.625)
    shifted = scenes.Intrinsics(base.fx, base.fy, base.cx, base.cy, c[0], c[1])
    for method in ("disparity", "standard", "explicit_disparity"):
        a = oracle.fit(depth, shifted.as_tuple(), k, method, want_lambda=True)
        b = oracle.fit(depth, base.as_tuple(), k, method, want_lambda=True,
                       delta=(np.full((H, W), c[0]), np.full((H, W), c[1])))
        for key in ("normals", "offsets", "curvature", "counts"):
            assert np.array_equal(np.nan_to_num(a[key], nan=7.0), np.nan_to_num(b[key], nan=7.0)), (method, key)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_noise_free_plane_with_per_pixel_rays(method):
    """Depth rendered through per-pixel rays (a radial field + ripple of up to ~2 px) is fitted exactly
    when the fit uses the same rays, and visibly wrongly when it ignores them (closed form, Eq. 12)."""
    W, H, k = 48, 36, 7
    intr = scenes.Intrinsics(200.0, 205.0, 23.5, 17.5)
    ddx, ddy = scenes.delta_table(5, intr, W, H, amp=2.0)
    assert np.abs(ddx).max() > 0.5 and np.abs(ddy).max() > 0.5
    pl = scenes.plane_through(np.array([0.1, -0.05, 1.7]), np.array([0.3, -0.2, -1.0]))
    Z = scenes.plane_depth_delta(pl, intr, ddx, ddy)
    assert np.isfinite(Z).all()
    o = oracle.fit(Z, intr.as_tuple(), k, method, delta=(ddx, ddy))
    assert np.isfinite(o["offsets"]).all()
    assert np.nanmax(_angle(o["normals"], pl.n[None, None, :])) < 1e-8
    assert np.max(np.abs(o["offsets"] - pl.d)) < 1e-8 * pl.d
    plain = oracle.fit(Z, intr.as_tuple(), k, method)
    assert np.nanmax(_angle(plain["normals"], pl.n[None, None, :])) > 1e-3


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_unit4_and_curvature_match_lapack_on_noisy_windows(method):
    """On noisy data, the literal |(a,b,c,d)| = 1 fit is the smallest eigenvector of the 4x4 scatter of
    the window's monomials (Eq. 4-6 / Eq. 14), and the default fit's curvature is lambda0 / trace of the
    Schur complement: both recomputed here by brute force over the window and LAPACK (numpy eigh)."""
    W, H, k = 30, 24, 7
    intr = scenes.Intrinsics(90.0, 92.0, 14.7, 11.2, 0.1, -0.2)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 177, intr, W, H, noise_coef=0.004)
    Z = oracle.depth_to_f64(depth, 1e-3)
    o4 = oracle.fit(depth, intr.as_tuple(), k, method, unit4=True, want_lambda=True)
    o3 = oracle.fit(depth, intr.as_tuple(), k, method, want_lambda=True)
    r = k // 2
    rng = np.random.Generator(np.random.PCG64(3))
    checked = 0
    for _ in range(60):
        px, py = int(rng.integers(0, W)), int(rng.integers(0, H))
        us = []
        for y in range(py - r, py + r + 1):
            for x in range(px - r, px + r + 1):
                if 0 <= x < W and 0 <= y < H and np.isfinite(Z[y, x]) and Z[y, x] > 0:
                    tx = (x + intr.dx - intr.cx) / intr.fx
                    ty = (y + intr.dy - intr.cy) / intr.fy
                    z = Z[y, x]
                    us.append([tx, ty, 1.0, 1.0 / z] if method == "disparity" else [z * tx, z * ty, z, 1.0])
        if not np.isfinite(o4["offsets"][py, px]):
            continue
        U = np.array(us)
        M = U.T @ U
        lam, vec = np.linalg.eigh(M)
        if (lam[1] - lam[0]) < 1e-6 * lam[3]:
            continue  # the 4x4 eigenvector is ill-posed here
        a = vec[:, 0]
        nn = np.linalg.norm(a[:3])
        n, d = a[:3] / nn, a[3] / nn
        if d < 0:
            n, d = -n, -d
        assert _angle(o4["normals"][py, px], n) < 1e-8
        assert abs(o4["offsets"][py, px] - d) < 1e-8 * max(abs(d), 1e-3)
        assert abs(o4["curvature"][py, px] - lam[0] / lam.sum()) < 1e-9
        # default constraint: curvature = lambda0 / trace of the Schur complement
        A, g, s = M[:3, :3], M[:3, 3], M[3, 3]
        l3 = np.linalg.eigvalsh(A - np.outer(g, g) / s)
        assert abs(o3["curvature"][py, px] - l3[0] / l3.sum()) < 1e-9
        checked += 1
    assert checked > 30


def test_depth_from_disparity_model():
    """The raw-disparity model 1/Z = alpha D + beta, either sign of alpha, any beta: D == 0 or
    1/Z <= 0 is missing."""
    D = np.array([[0, 1, 7, 300], [1000, 65535, 2, 5]], dtype=np.uint16)
    a = 1.0 / (8.0 * 575.0 * 0.075)
    Z = oracle.depth_from_disparity(D, a, 0.0)
    ok = D > 0
    assert np.all(Z[~ok] == 0.0)
    assert np.allclose(Z[ok], 1.0 / (a * D[ok].astype(np.float64)), rtol=1e-15, atol=0)
    b = 0.3717 * a  # not a multiple of any power-of-two fraction of alpha
    Zb = oracle.depth_from_disparity(D, a, b)
    assert np.allclose(1.0 / Zb[ok], a * D[ok] + b, rtol=1e-14, atol=0)
    # a structured-light style model with negative alpha: larger raw values are farther
    ka, kb = scenes.KINECT_RAW_ALPHA, scenes.KINECT_RAW_BETA
    Dk = np.array([[0, 400, 800, 1084, 1085, 2047]], dtype=np.uint16)
    Zk = oracle.depth_from_disparity(Dk, ka, kb)
    w = ka * Dk.astype(np.float64) + kb
    valid = (Dk > 0) & (w > 0)
    assert np.all(Zk[Dk == 0] == 0.0)
    assert np.allclose(1.0 / Zk[valid], w[valid], rtol=1e-14, atol=0)
    assert np.all(np.diff(Zk[valid]) > 0)  # farther with the raw code
    assert np.all(Zk[(Dk > 0) & (w <= 0)] == 0.0)  # behind the camera: missing
