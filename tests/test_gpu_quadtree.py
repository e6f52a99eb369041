"""GPU planar segmentation (sf_quadtree) against the oracle's quadtree.

The tree is integer structure: which nodes exist, their status and valid
counts must match the oracle exactly.  A split decision compares the node's
RMS error with tau; the GPU solves every node in FP64 from exact integer
sums of 24-bit (20-bit standard) fixed-point depth, so its RMS agrees with
the oracle's to ~1e-5 relative.  Each test therefore takes a tau from a
short list such that no evaluated node's RMS lies within 1e-3 of it
(relative), which makes the comparison exact rather than lucky.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import scenes

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitter, SurfFitError  # noqa: E402

MARGIN = 1e-3
TAUS = {"disparity": [6e-3, 8e-3, 1e-2, 1.3e-2, 1.7e-2], "standard": [1e-2, 1.3e-2, 1.7e-2, 2.2e-2, 3e-2],
        "explicit_disparity": [3e-3, 4e-3, 5e-3, 6.5e-3, 8e-3], "explicit_standard": [1.5e-2, 2e-2, 2.6e-2, 3.4e-2]}


def _angle(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def _pick_tau(frames, intr, method, **kw):
    for tau in TAUS[method]:
        trees = [oracle.quadtree(f, intr, method, tau=tau, **kw) for f in frames]
        rms = np.array([n["rms"] for t in trees for n in t if np.isfinite(n["rms"])])
        if rms.size == 0 or np.min(np.abs(rms / tau - 1.0)) >= MARGIN:
            return tau, trees
    pytest.fail("no tau with a decision margin of %g" % MARGIN)


def _centroid_distance(depth, intr, n):
    """|mu|: distance of the centroid of the node's valid 3D points from the camera."""
    fx, fy, cx, cy, dx, dy = intr
    Z = oracle.depth_to_f64(depth)[n["y0"]:n["y0"] + n["h"], n["x0"]:n["x0"] + n["w"]]
    tx = (np.arange(n["x0"], n["x0"] + n["w"]) + dx - cx) / fx
    ty = (np.arange(n["y0"], n["y0"] + n["h"]) + dy - cy) / fy
    v = Z > 0
    P = np.stack([Z * tx[None, :], Z * ty[:, None], Z], -1)[v]
    return float(np.linalg.norm(P.mean(0)))


def _compare(gpu, trees, label, frames, intr):
    for f, tree in enumerate(trees):
        g = gpu[gpu["frame"] == f]
        ref = {(n["level"], n["y0"], n["x0"]): n for n in tree}
        got = {(int(r["level"]), int(r["y0"]), int(r["x0"])): r for r in g}
        assert set(got) == set(ref), "%s frame %d: node sets differ (%d vs %d)" % (label, f, len(got), len(ref))
        for key, n in ref.items():
            r = got[key]
            assert (int(r["w"]), int(r["h"]), int(r["status"]), int(r["count"])) == (
                n["w"], n["h"], n["status"], n["count"]), (label, key)
            if n["status"] == oracle.QUAD_INVALID:
                assert np.isnan(r["rms"])
                continue
            # the per-pixel readings: normals within 1e-3 rad where the eigen-gap is >= 1e-3
            lam = n["lam"]
            well_posed = not np.isfinite(lam[2]) or (lam[1] - lam[0]) >= 1e-3 * lam[2]
            if well_posed:
                ang = _angle(r["normal"].astype(np.float64), n["normal"])
                assert ang < 1e-3, (label, key)
                # offsets relative to |mu|; a normal off by ang moves d by up to ang |mu| (the
                # fixed-point input alone turns small noisy nodes by ~1e-4 rad)
                mu = _centroid_distance(frames[f], intr, n)
                assert abs(float(r["offset"]) - n["offset"]) <= (1e-4 + ang) * mu, (label, key)
            # the GPU's sums are exact: a flat tile of equal depths has rms 0 there and ~1e-7 in the
            # oracle's FP64 Schur complement
            assert abs(float(r["rms"]) - n["rms"]) <= 1e-3 * n["rms"] + 1e-6, (label, key)


@pytest.mark.parametrize("method", ["disparity", "standard", "explicit_disparity", "explicit_standard"])
def test_segmentation_512x424(method):
    intr = scenes.SEG_INTRINSICS
    depth = scenes.segmentation_frame(scenes.BASE_SEED + 900)
    tau, trees = _pick_tau([depth], intr.as_tuple(), method, tile=64, max_level=3)
    f = SurfaceFitter(intr.as_tuple(), scenes.SEG_W, scenes.SEG_H, 5, method=method)
    gpu = f.quadtree(torch.from_numpy(depth).cuda(), tile=64, max_level=3, tau=tau)
    f.close()
    _compare(gpu, trees, "%s tau=%g" % (method, tau), [depth], intr.as_tuple())
    st = np.bincount(gpu["status"], minlength=4)
    assert st[oracle.QUAD_FIT] > 50 and st[oracle.QUAD_SPLIT] > 5, st


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_batch_ragged_size(method):
    W, H = 200, 150
    intr = scenes.Intrinsics.scaled(W, H, f640=365.0)
    frames = [scenes.segmentation_frame(scenes.BASE_SEED + 910 + i, intr, W, H) for i in range(3)]
    tau, trees = _pick_tau(frames, intr.as_tuple(), method, tile=48, max_level=4, min_valid_permille=300)
    f = SurfaceFitter(intr.as_tuple(), W, H, 3, method=method)
    gpu = f.quadtree(torch.from_numpy(np.stack(frames)).cuda(), tile=48, max_level=4, tau=tau, min_frac=0.3)
    f.close()
    _compare(gpu, trees, "batch %s" % method, frames, intr.as_tuple())


def test_uint16_input():
    W, H = 320, 180
    intr = scenes.Intrinsics(920.0 / 4, 920.0 / 4, 159.5, 89.5)
    depth = scenes.structured_light_frame(scenes.BASE_SEED + 920, intr, W, H)
    tau, trees = _pick_tau([depth], intr.as_tuple(), "disparity", tile=32, max_level=2)
    f = SurfaceFitter(intr.as_tuple(), W, H, 5, method="disparity", depth_type="u16")
    t = torch.from_numpy(depth.view(np.int16)).cuda().view(torch.uint16)
    gpu = f.quadtree(t, tile=32, max_level=2, tau=tau)
    f.close()
    _compare(gpu, trees, "u16", [depth], intr.as_tuple())


def test_all_missing_and_arguments():
    W, H = 100, 70
    intr = scenes.Intrinsics.scaled(W, H)
    f = SurfaceFitter(intr.as_tuple(), W, H, 3)
    gpu = f.quadtree(torch.zeros((H, W), device="cuda"), tile=32, max_level=2, tau=1e-2)
    assert len(gpu) == 4 * 3 and np.all(gpu["status"] == oracle.QUAD_INVALID) and np.all(gpu["count"] == 0)
    d = torch.ones((H, W), device="cuda")
    for kw in [dict(tile=65), dict(tile=1), dict(max_level=7), dict(tau=0.0), dict(min_frac=1.5)]:
        with pytest.raises(SurfFitError):
            f.quadtree(d, **kw)
    f.close()
