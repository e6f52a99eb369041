"""Pins of the oracle's planar segmentation (Section III, tile subdivision).

Checked against what the geometry fixes, not against the oracle itself:
noise-free planes are recovered exactly and never split; a tile straddling
two planes splits and its pure children recover either plane; the leaves
partition the image; the reported error is the definition written out (the
RMS of the residual at the fitted plane); the rectangle fit equals the
per-pixel window fit on the same pixels; the valid-count rule is an integer
rule.
"""
import numpy as np
import pytest

import oracle
import scenes

INTR = scenes.Intrinsics(300.0, 310.0, 63.7, 47.2, 0.25, -0.5)
W, H = 128, 96


def _leaves(nodes):
    return [n for n in nodes if n["status"] != oracle.QUAD_SPLIT]


def _angle(a, b):
    return float(np.arctan2(np.linalg.norm(np.cross(a, b)), np.dot(a, b)))


@pytest.mark.parametrize("method", ["disparity", "standard", "explicit_disparity", "explicit_standard"])
def test_noise_free_plane_is_one_fit_per_root(method):
    Z, pl = scenes.single_plane_frame(11, INTR, W, H)
    # the FP64 Schur complement of an exact plane keeps lambda0 at rounding level (rms ~1e-8)
    nodes = oracle.quadtree(Z, INTR.as_tuple(), method, tile=32, max_level=3, tau=1e-6)
    assert len(nodes) == (W // 32) * (H // 32)
    for n in nodes:
        assert n["status"] == oracle.QUAD_FIT and n["level"] == 0
        assert _angle(n["normal"], pl.n) < 1e-9
        assert abs(n["offset"] - pl.d) < 1e-9 * pl.d
        assert n["rms"] < 1e-6


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_two_planes_split_only_across_the_seam(method):
    n1 = np.array([0.3, -0.2, -1.0]); n1 /= np.linalg.norm(n1)
    n2 = np.array([-0.4, 0.1, -1.0]); n2 /= np.linalg.norm(n2)
    split = 70  # inside the third 32-pixel root column
    Z = scenes.two_plane_frame(INTR, W, H, split, n1, 2.0, n2, 2.2)
    nodes = oracle.quadtree(Z, INTR.as_tuple(), method, tile=32, max_level=3, tau=1e-6)
    for n in _leaves(nodes):
        crosses = n["x0"] < split < n["x0"] + n["w"]
        if crosses:
            assert n["level"] == 3 and n["status"] == oracle.QUAD_HIGH_ERROR
        else:
            assert n["status"] == oracle.QUAD_FIT
            ref = n1 if n["x0"] + n["w"] <= split else n2
            assert _angle(n["normal"], ref) < 1e-8
    roots = [n for n in nodes if n["level"] == 0]
    assert sorted(n["x0"] for n in roots if n["status"] == oracle.QUAD_SPLIT) == [64, 64, 64]


@pytest.mark.parametrize("method", ["disparity", "standard", "explicit_disparity"])
def test_leaves_partition_the_image(method):
    intr = scenes.Intrinsics.scaled(150, 101)
    depth = scenes.kinect_frame(21, intr, 150, 101, n_planes=5, missing_iid=0.1)
    nodes = oracle.quadtree(depth, intr.as_tuple(), method, tile=40, max_level=3, tau=3e-3 if method != "standard" else 6e-3)
    cover = np.zeros((101, 150), np.int32)
    for n in _leaves(nodes):
        cover[n["y0"]:n["y0"] + n["h"], n["x0"]:n["x0"] + n["w"]] += 1
    assert np.all(cover == 1)
    # children of a split node tile it exactly
    by = {(n["level"], n["x0"], n["y0"]): n for n in nodes}
    for n in nodes:
        if n["status"] == oracle.QUAD_SPLIT:
            kids = [k for k in nodes if k["level"] == n["level"] + 1 and n["x0"] <= k["x0"] < n["x0"] + n["w"]
                    and n["y0"] <= k["y0"] < n["y0"] + n["h"]]
            assert len(kids) == 4 and sum(k["w"] * k["h"] for k in kids) == n["w"] * n["h"]
    assert len(by) == len(nodes)


@pytest.mark.parametrize("method", ["disparity", "standard", "explicit_disparity", "explicit_standard"])
def test_rms_is_the_residual_at_the_fitted_plane(method):
    intr = scenes.Intrinsics.scaled(64, 48)
    depth = scenes.kinect_frame(31, intr, 64, 48, n_planes=2, missing_iid=0.2).astype(np.float64)
    r = oracle.fit_rect(depth, intr.as_tuple(), 5, 7, 40, 30, method)
    assert r["ok"]
    Z = depth[7:37, 5:45]
    v = Z > 0
    tx = (np.arange(5, 45) + intr.dx - intr.cx) / intr.fx
    ty = (np.arange(7, 37) + intr.dy - intr.cy) / intr.fy
    P = np.stack([Z * tx[None, :], Z * ty[:, None], Z], -1)[v]
    n, d = r["normal"], r["offset"]
    dist = P @ n + d
    if method == "disparity":
        e = dist / P[:, 2]            # (n.P + d) / Z
    elif method == "standard":
        e = dist
    elif method == "explicit_disparity":
        e = dist / P[:, 2] / d        # 1/Z - (a tx + b ty + c): the plane is (a, b, c).m - 1/Z scaled by |d|
    else:
        e = dist / n[2]               # Z - (a X + b Y + c)
    rms = np.sqrt(np.mean(e ** 2))
    assert np.sqrt(max(r["residual"], 0.0) / r["count"]) == pytest.approx(rms, rel=1e-9)
    assert r["count"] == int(v.sum())


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_rect_fit_equals_window_fit(method):
    intr = scenes.Intrinsics.scaled(48, 40)
    depth = scenes.kinect_frame(41, intr, 48, 40, missing_iid=0.1)
    Z = oracle.depth_to_f64(depth)
    ref = oracle.fit(depth, intr.as_tuple(), 7, method, require_center=False)
    for (px, py) in [(10, 10), (20, 15), (30, 30)]:
        r = oracle.fit_rect(Z, intr.as_tuple(), px - 3, py - 3, 7, 7, method)
        assert r["count"] == ref["counts"][py, px]
        assert _angle(r["normal"], ref["normals"][py, px]) < 1e-12
        assert r["offset"] == pytest.approx(ref["offsets"][py, px], rel=1e-12)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_collinear_node_is_invalid(method):
    """One row of pixels: every depth lies in the plane of its camera rays, so there is no surface."""
    Z, _ = scenes.single_plane_frame(13, INTR, 16, 16)
    r = oracle.fit_rect(Z, INTR.as_tuple(), 0, 5, 16, 1, method)
    assert not r["ok"] and r["count"] == 16
    Zd = Z.copy()
    Zd[6:, :] = 0.0
    Zd[:5, :] = 0.0
    nodes = oracle.quadtree(Zd, INTR.as_tuple(), method, tile=16, max_level=1, tau=1.0, min_valid_permille=0)
    assert nodes[0]["status"] == oracle.QUAD_INVALID


def test_valid_count_rule_is_integer():
    Z, _ = scenes.single_plane_frame(12, INTR, 16, 16)
    area = 16 * 16
    need = (500 * area + 999) // 1000  # 128
    for missing, status in [(area - need, oracle.QUAD_FIT), (area - need + 1, oracle.QUAD_INVALID)]:
        Zm = Z.copy().reshape(-1)
        Zm[:missing] = 0.0
        nodes = oracle.quadtree(Zm.reshape(16, 16), INTR.as_tuple(), "disparity", tile=16, max_level=2,
                                tau=1.0, min_valid_permille=500)
        assert len(nodes) == 1 and nodes[0]["status"] == status
