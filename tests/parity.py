"""Shared comparison helpers for the GPU parity tests (test infrastructure)."""
import numpy as np

# Tolerances for the floating-point outputs: normal angle 1e-3 rad; offset
# 1e-4 relative, measured against the distance |mu| of the window's (weighted)
# centroid from the camera: |d - d_ref| <= 1e-4 |mu|, and for head-on windows
# (|d_ref| >= 0.1 |mu|) also |d - d_ref| <= 1e-4 |d_ref|.  Since d = -n . mu,
# |d| <= |mu| and an error dn in the normal moves d by up to |dn| |mu|: for
# windows seen edge-on (d -> 0) a relative error in d itself is unbounded for
# any finite-precision normal, while |dd| / |mu| stays well-defined; for
# head-on windows the two coincide.
# Where the fitted plane passes the camera centre closer than the offset
# tolerance (|d| <= 1e-4 |mu|) the orientation rule (d >= 0) has nothing to
# decide at that tolerance, so normals and offsets are compared up to sign.
# They apply to windows that are not near-degenerate: the eigenvector of a
# 3x3 problem moves by |dR| / (lambda1 - lambda0) under a perturbation dR, so
# where the eigen-gap gamma = (lambda1 - lambda0) / lambda2 is tiny the normal
# is ill-posed and only its validity (unit, facing the camera, minimising the
# fit residual) is checked.
ANGLE_TOL = 1e-3
OFFSET_TOL = 1e-4
GAP_MIN = 1e-3
# curvature is lambda0 / trace in [0, 1/3]: absolute tolerance
CURV_TOL = 1e-5


def angle(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def schur(moments):
    mo = moments
    A = np.stack([np.stack([mo[..., 0], mo[..., 1], mo[..., 2]], -1),
                  np.stack([mo[..., 1], mo[..., 3], mo[..., 4]], -1),
                  np.stack([mo[..., 2], mo[..., 4], mo[..., 5]], -1)], -2)
    g = mo[..., 6:9]
    s = mo[..., 9]
    return A - g[..., :, None] * g[..., None, :] / s[..., None, None]


def compare(gpu, ref, *, angle_tol=ANGLE_TOL, offset_tol=OFFSET_TOL, gap_min=GAP_MIN, curv_tol=CURV_TOL,
            check_degenerate=True, label=""):
    """Check GPU outputs (normals, offsets, curvature, counts) against the oracle dict.

    Returns a dict of statistics.  Counts and the validity mask must match
    bit for bit; floats must meet the tolerances on non-degenerate windows;
    degenerate windows must still hold a unit normal facing the camera that
    minimises the fit residual to FP32 precision.
    """
    n, d, c, cnt = [np.asarray(v) for v in gpu]
    assert np.array_equal(cnt, ref["counts"]), "%s: counts differ at %d pixels" % (label, (cnt != ref["counts"]).sum())
    ok = np.isfinite(ref["offsets"])
    assert np.array_equal(np.isfinite(d), ok), "%s: validity mask differs at %d pixels" % (
        label, (np.isfinite(d) != ok).sum())
    assert np.array_equal(np.isfinite(n).all(-1), ok) and np.array_equal(np.isfinite(c), ok)
    stats = {"valid": int(ok.sum()), "pixels": int(ok.size)}
    if not ok.any():
        return stats
    lam = ref["lam"]
    l2 = np.where(ok, lam[..., 2], 1.0)
    gap = np.where(ok, (lam[..., 1] - lam[..., 0]) / l2, 0.0)
    # lambda1 at FP64 rounding level: rank <= 1 (collinear points), degenerate
    gap = np.where(np.abs(lam[..., 1]) <= 1e-9 * np.abs(l2), 0.0, gap)
    good = ok & (gap >= gap_min)
    mo = ref["moments"]
    mu = np.linalg.norm(mo[..., 6:9] / np.where(ok[..., None], mo[..., 9:10], 1.0), axis=-1)
    # a plane through the camera centre to within the offset tolerance has no
    # orientation at that tolerance (d ~ 0 decides it): compare up to sign
    sign_free = np.abs(np.where(ok, ref["offsets"], 1.0)) <= offset_tol * np.where(ok, mu, 1.0)
    ang = angle(n[good], ref["normals"][good])
    flipped = angle(-n[good], ref["normals"][good])
    ang = np.where(sign_free[good], np.minimum(ang, flipped), ang)
    err_d = np.abs(np.where(sign_free[good], np.abs(d[good]), d[good]).astype(np.float64) -
                   np.where(sign_free[good], np.abs(ref["offsets"][good]), ref["offsets"][good])) / mu[good]
    rel = err_d
    cerr = np.abs(c[good].astype(np.float64) - ref["curvature"][good])
    stats.update(good=int(good.sum()), max_angle=float(ang.max(initial=0)), max_offset_rel=float(rel.max(initial=0)),
                 max_curv=float(cerr.max(initial=0)), degenerate=int((ok & ~good).sum()))
    assert stats["max_angle"] <= angle_tol, "%s: normal angle %g > %g" % (label, stats["max_angle"], angle_tol)
    assert stats["max_offset_rel"] <= offset_tol, "%s: offset %g > %g" % (label, stats["max_offset_rel"], offset_tol)
    assert stats["max_curv"] <= curv_tol, "%s: curvature %g > %g" % (label, stats["max_curv"], curv_tol)
    # every valid pixel: unit normal, camera on the positive side
    nn = np.linalg.norm(n[ok].astype(np.float64), axis=-1)
    assert np.max(np.abs(nn - 1)) < 1e-5, "%s: normals not unit" % label
    # orientation rule: d >= 0 (d == 0 only for planes through the camera centre,
    # e.g. the degenerate fits of collinear windows)
    assert np.all(d[ok] >= 0), "%s: offsets negative" % label
    headon = good & (np.abs(np.where(ok, ref["offsets"], 0)) >= 0.1 * mu)
    stats["max_offset_rel_headon"] = float((np.abs(d[headon].astype(np.float64) - ref["offsets"][headon]) /
                                            np.abs(ref["offsets"][headon])).max(initial=0))
    assert stats["max_offset_rel_headon"] <= offset_tol, "%s: head-on offset %g > %g" % (
        label, stats["max_offset_rel_headon"], offset_tol)
    if check_degenerate and (ok & ~good).any():
        bad = ok & ~good
        R = schur(ref["moments"][bad])
        v = n[bad].astype(np.float64)
        rq = np.einsum("pi,pij,pj->p", v, R, v)
        excess = (rq - lam[bad][:, 0]) / lam[bad][:, 2]
        stats["degenerate_max_excess"] = float(excess.max())
        assert excess.max() < 1e-3, "%s: degenerate windows not minimised (%g)" % (label, excess.max())
    return stats


# Explicit fits (Section I.D, Section II.B) are linear least squares: their
# slopes move by about cond(C) * eps under rounding, C the centred 2x2
# covariance of the regressors ((tx, ty) for Eq. 15-16, (X, Y) for Eq. 7-9),
# so the tolerances apply where 1/cond(C) >= COND_MIN.  The third output, the
# mean squared residual, is compared against the variance of the target: it is
# the difference of that variance and the explained part, so its float32 error
# is about eps * cond(C) of the variance (up to ~1e-4 at COND_MIN).
COND_MIN = 1e-3
RESID_TOL = 1e-4


def explicit_design(moments):
    """(1/cond of the centred regressor covariance, n) from the oracle's moments."""
    mo = moments
    n = mo[..., 5]
    c11 = mo[..., 0] - mo[..., 2] ** 2 / n
    c12 = mo[..., 1] - mo[..., 2] * mo[..., 4] / n
    c22 = mo[..., 3] - mo[..., 4] ** 2 / n
    tr = c11 + c22
    disc = np.sqrt(np.maximum((c11 - c22) ** 2 + 4 * c12 ** 2, 0.0))
    lmax, lmin = (tr + disc) / 2, (tr - disc) / 2
    return np.where(lmax > 0, lmin / np.where(lmax > 0, lmax, 1.0), 0.0), n


def compare_explicit(gpu, ref, method, *, angle_tol=ANGLE_TOL, offset_tol=OFFSET_TOL, cond_min=COND_MIN,
                     resid_tol=RESID_TOL, label=""):
    """Check an explicit fit (method explicit_disparity / explicit_standard) against the oracle dict."""
    n, d, c, cnt = [np.asarray(v) for v in gpu]
    assert np.array_equal(cnt, ref["counts"]), "%s: counts differ at %d pixels" % (label, (cnt != ref["counts"]).sum())
    ok = np.isfinite(ref["offsets"])
    assert np.array_equal(np.isfinite(d), ok), "%s: validity mask differs at %d pixels" % (
        label, (np.isfinite(d) != ok).sum())
    assert np.array_equal(np.isfinite(n).all(-1), ok) and np.array_equal(np.isfinite(c), ok)
    stats = {"valid": int(ok.sum()), "pixels": int(ok.size)}
    if not ok.any():
        return stats
    mo = np.where(ok[..., None], ref["moments"], 1.0)
    rc, cnt_f = explicit_design(mo)
    good = ok & (rc >= cond_min)
    # centroid of the window's points: the scale of the offset
    if method == "explicit_disparity":   # A = sum m m^T (rays), g = sum m / Z
        mu = np.linalg.norm(np.stack([mo[..., 2], mo[..., 4], cnt_f], -1), axis=-1) / mo[..., 8]
    else:                                # A = sum [X, Y, 1][X, Y, 1]^T, g = sum Z [X, Y, 1]
        mu = np.linalg.norm(np.stack([mo[..., 2], mo[..., 4], mo[..., 8]], -1), axis=-1) / cnt_f
    var_b = np.maximum(mo[..., 9] / cnt_f - (mo[..., 8] / cnt_f) ** 2, 0.0)
    ang = angle(n[good], ref["normals"][good])
    rel = np.abs(d[good].astype(np.float64) - ref["offsets"][good]) / mu[good]
    # a window of equal targets has variance 0 and residual 0; the oracle's
    # uncentred residual then carries FP64 rounding of the mean square
    denom = np.maximum(var_b, 1e-9 * mo[..., 9] / cnt_f)
    cerr = np.abs(c[good].astype(np.float64) - ref["curvature"][good]) / denom[good]
    stats.update(good=int(good.sum()), max_angle=float(ang.max(initial=0)), max_offset_rel=float(rel.max(initial=0)),
                 max_resid_rel=float(cerr.max(initial=0)), ill_conditioned=int((ok & ~good).sum()),
                 rc_at_max_resid=float(rc[good][np.argmax(cerr)]) if cerr.size else 0.0)
    assert stats["max_angle"] <= angle_tol, "%s: normal angle %g > %g" % (label, stats["max_angle"], angle_tol)
    assert stats["max_offset_rel"] <= offset_tol, "%s: offset %g > %g" % (label, stats["max_offset_rel"], offset_tol)
    assert stats["max_resid_rel"] <= resid_tol, "%s: residual %g > %g" % (label, stats["max_resid_rel"], resid_tol)
    nn = np.linalg.norm(n[ok].astype(np.float64), axis=-1)
    assert np.max(np.abs(nn - 1)) < 1e-5, "%s: normals not unit" % label
    assert np.all(d[ok] >= 0), "%s: offsets negative" % label
    assert np.all(c[ok] >= 0), "%s: residual negative" % label
    return stats
