"""The GPU parity comparator itself (tests/parity.py), on CPU: outputs copied from the oracle pass,
and each planted mistake of the kind a kernel could make (a rotated normal, an offset off, a flipped
orientation, a count off by one, a lost or extra fit, a curvature off) is caught."""
import numpy as np
import pytest

import oracle
import scenes
from parity import compare


@pytest.fixture(scope="module")
def frame():
    W, H, k = 64, 48, 7
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 210, intr, W, H)
    ref = oracle.fit(depth, intr.as_tuple(), k, "disparity", want_lambda=True, want_moments=True)
    gpu = (ref["normals"].astype(np.float32), ref["offsets"].astype(np.float32),
           ref["curvature"].astype(np.float32), ref["counts"].copy())
    ok = np.isfinite(ref["offsets"])
    lam = ref["lam"]
    gap = np.where(ok, (lam[..., 1] - lam[..., 0]) / np.where(ok, lam[..., 2], 1.0), 0.0)
    mu = np.linalg.norm(ref["moments"][..., 6:9] / np.where(ok[..., None], ref["moments"][..., 9:10], 1.0), axis=-1)
    # a well-posed, head-on window to plant the mistakes in
    cand = np.argwhere(ok & (gap > 0.05) & (np.abs(np.where(ok, ref["offsets"], 0)) > 0.5 * mu))
    y, x = cand[len(cand) // 2]
    return ref, gpu, (y, x), mu[y, x]


def _copy(gpu):
    return tuple(a.copy() for a in gpu)


def test_exact_copy_passes(frame):
    ref, gpu, _, _ = frame
    s = compare(gpu, ref, label="copy")
    assert s["good"] > 0.5 * s["valid"]


def _rotate(n, ang):
    # rotate the unit vector n by ang about an axis perpendicular to it
    a = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    return n * np.cos(ang) + np.cross(a, n) * np.sin(ang)


@pytest.mark.parametrize("what", ["normal 2e-3 rad", "offset 3e-4 |mu|", "flipped orientation", "count + 1",
                                  "lost fit", "extra fit", "curvature + 3e-5",
                                  "offset 1.5e-4 |mu| beside a normal off by 1e-4 rad",
                                  "head-on offset 1.2e-4 relative"])
def test_planted_mistake_is_caught(frame, what):
    ref, gpu, (y, x), mu = frame
    n, d, c, cnt = _copy(gpu)
    if what == "normal 2e-3 rad":
        n[y, x] = _rotate(ref["normals"][y, x], 2e-3)
    elif what == "offset 3e-4 |mu|":
        d[y, x] += 3e-4 * mu
    elif what == "flipped orientation":
        n[y, x] = -n[y, x]
        d[y, x] = -d[y, x]
    elif what == "offset 1.5e-4 |mu| beside a normal off by 1e-4 rad":
        # the offset's own error may not hide behind the normal's
        n[y, x] = _rotate(ref["normals"][y, x], 1e-4)
        d[y, x] += 1.5e-4 * mu
    elif what == "head-on offset 1.2e-4 relative":
        d[y, x] *= 1.0 + 1.2e-4
    elif what == "count + 1":
        cnt[y, x] += 1
    elif what == "lost fit":
        n[y, x] = np.nan
        d[y, x] = np.nan
        c[y, x] = np.nan
    elif what == "extra fit":
        yy, xx = np.argwhere(~np.isfinite(ref["offsets"]))[0]
        n[yy, xx] = (0.0, 0.0, -1.0)
        d[yy, xx] = 1.0
        c[yy, xx] = 0.0
    else:
        c[y, x] += 3e-5
    with pytest.raises(AssertionError):
        compare((n, d, c, cnt), ref, label=what)


def test_mistakes_below_the_tolerances_pass(frame):
    ref, gpu, (y, x), mu = frame
    n, d, c, cnt = _copy(gpu)
    n[y, x] = _rotate(ref["normals"][y, x], 5e-4)
    d[y, x] += 5e-5 * mu
    c[y, x] += 5e-6
    compare((n, d, c, cnt), ref, label="within tolerance")


@pytest.mark.parametrize("method", ["explicit_disparity", "explicit_standard"])
@pytest.mark.parametrize("what", [None, "normal 2e-3 rad", "residual x 1.01", "count - 1", "lost fit"])
def test_explicit_comparator(method, what):
    from parity import compare_explicit, explicit_design

    W, H, k = 48, 40, 7
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 211, intr, W, H)
    ref = oracle.fit(depth, intr.as_tuple(), k, method, want_lambda=True, want_moments=True)
    n, d, c, cnt = (ref["normals"].astype(np.float32), ref["offsets"].astype(np.float32),
                    ref["curvature"].astype(np.float32), ref["counts"].copy())
    ok = np.isfinite(ref["offsets"])
    rc, _ = explicit_design(np.where(ok[..., None], ref["moments"], 1.0))
    y, x = np.argwhere(ok & (rc > 0.1) & (ref["curvature"] > 0))[0]
    if what == "normal 2e-3 rad":
        n[y, x] = _rotate(ref["normals"][y, x], 2e-3)
    elif what == "residual x 1.01":
        c[y, x] *= 1.01
    elif what == "count - 1":
        cnt[y, x] -= 1
    elif what == "lost fit":
        n[y, x] = np.nan
        d[y, x] = np.nan
        c[y, x] = np.nan
    if what is None:
        compare_explicit((n, d, c, cnt), ref, method, label="copy")
    else:
        with pytest.raises(AssertionError):
            compare_explicit((n, d, c, cnt), ref, method, label=what)
