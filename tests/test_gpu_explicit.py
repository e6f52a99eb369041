"""GPU parity of the explicit fits (Eq. 15-16 in RGBD space, Eq. 7-9 in
Euclidean space) against the FP64 oracle.

They share the window sums of the implicit fits; only the per-pixel solve
differs (a 2x2 centred regression).  Counts and validity masks, including
the rule that a window whose valid pixels are collinear in the image has no
explicit fit, must match bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import scenes
from parity import angle, compare_explicit

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitter  # noqa: E402

EXPLICIT = ["explicit_disparity", "explicit_standard"]


def run_gpu(depth, intr, k, method, depth_type="f32", precision=0, **kw):
    H, W = depth.shape[-2:]
    f = SurfaceFitter(intr, W, H, k, method=method, depth_type=depth_type, **kw)
    if precision:
        f.set_precision(precision)
    t = torch.from_numpy(depth.view(np.int16) if depth.dtype == np.uint16 else depth).cuda()
    if depth.dtype == np.uint16:
        t = t.view(torch.uint16)
    n, d, c, cnt = f.fit(t, counts=True)
    torch.cuda.synchronize()
    out = (n.cpu().numpy(), d.cpu().numpy(), c.cpu().numpy(), cnt.cpu().numpy())
    f.close()
    return out


def run_ref(depth, intr, k, method, **kw):
    return oracle.fit(depth, intr, k, method, want_moments=True, **kw)


@pytest.mark.parametrize("method", EXPLICIT)
def test_kinect_640x480_k7(method):
    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    depth = scenes.kinect_frame(scenes.BASE_SEED, intr, 640, 480)
    s = compare_explicit(run_gpu(depth, intr.as_tuple(), 7, method), run_ref(depth, intr.as_tuple(), 7, method),
                         method, label="640x480 " + method)
    assert s["good"] > 0.99 * s["valid"]
    print(method, s)


@pytest.mark.parametrize("W,H", [(1, 40), (40, 1), (37, 23), (130, 257)])
@pytest.mark.parametrize("k", [1, 3, 7, 31])
@pytest.mark.parametrize("method", EXPLICIT)
def test_ragged_sizes_and_windows(W, H, k, method):
    """Single rows and columns have collinear windows only: every output is NaN."""
    intr = scenes.Intrinsics.scaled(W, H) if W > 1 else scenes.Intrinsics(525.0, 525.0, 0.0, (H - 1) / 2)
    depth = scenes.kinect_frame(1000 + W * 7 + H, intr, W, H)
    s = compare_explicit(run_gpu(depth, intr.as_tuple(), k, method), run_ref(depth, intr.as_tuple(), k, method),
                         method, label="%dx%d k=%d %s" % (W, H, k, method))
    if W == 1 or H == 1 or k == 1:
        assert s["valid"] == 0


@pytest.mark.parametrize("method", EXPLICIT)
def test_sparse_windows_collinear_rule(method):
    """40% i.i.d. missing pixels, 3x3 windows, min_valid 2: many windows keep
    two or three pixels, some of them collinear."""
    W, H = 96, 64
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(77, intr, W, H, missing_iid=0.4)
    gpu = run_gpu(depth, intr.as_tuple(), 3, method, min_valid=2, require_center=False)
    ref = run_ref(depth, intr.as_tuple(), 3, method, min_valid=2, require_center=False)
    s = compare_explicit(gpu, ref, method, label="sparse " + method)
    collinear = (ref["counts"] >= 2) & ~np.isfinite(ref["offsets"])
    assert collinear.sum() > 20, "the scene should contain collinear windows"
    print(method, s, int(collinear.sum()))


@pytest.mark.parametrize("k", [5, 15])
@pytest.mark.parametrize("method", EXPLICIT)
def test_uint16_structured_light(k, method):
    W, H = 320, 180
    intr = scenes.Intrinsics(920.0 / 4, 920.0 / 4, 159.5, 89.5)
    depth = scenes.structured_light_frame(scenes.BASE_SEED + 1, intr, W, H)
    compare_explicit(run_gpu(depth, intr.as_tuple(), k, method, depth_type="u16"),
                     run_ref(depth, intr.as_tuple(), k, method), method, label="u16 k=%d %s" % (k, method))


@pytest.mark.parametrize("method", EXPLICIT)
def test_wide_depth_range_k31(method):
    W, H = 480, 270
    intr = scenes.Intrinsics.scaled(W, H, f640=525.0)
    depth = scenes.wide_range_frame(scenes.BASE_SEED + 2, intr, W, H)
    s = compare_explicit(run_gpu(depth, intr.as_tuple(), 31, method), run_ref(depth, intr.as_tuple(), 31, method),
                         method, label="wide k=31 " + method)
    print(method, s)


@pytest.mark.parametrize("method", EXPLICIT)
def test_fp64_mode_every_window(method):
    """Precision mode 2 solves the regression in FP64 from the same exact sums:
    every valid window (ill-conditioned ones included) within 1e-6 rad, the
    offset within 1e-6 and the residual within 1e-5 of the variance (float32
    outputs, fixed-point inputs)."""
    W, H = 200, 150
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(91, intr, W, H)
    s = compare_explicit(run_gpu(depth, intr.as_tuple(), 7, method, precision=2),
                         run_ref(depth, intr.as_tuple(), 7, method), method, angle_tol=1e-6, offset_tol=1e-6,
                         cond_min=0.0, resid_tol=1e-5, label="fp64 " + method)
    print(method, s)


@pytest.mark.parametrize("method", EXPLICIT)
def test_noise_free_plane(method):
    """A plane seen without noise is fitted exactly by both explicit forms."""
    W, H = 160, 120
    intr = scenes.Intrinsics(300.0, 310.0, 80.2, 59.7, 0.3, -0.2)
    Z, pl = scenes.single_plane_frame(5, intr, W, H)
    depth = scenes.to_f32_metres(Z)
    n, d, c, cnt = run_gpu(depth, intr.as_tuple(), 5, method)
    assert np.max(angle(n, pl.n[None, None, :])) < 2e-4
    assert np.max(np.abs(d - pl.d)) < 1e-4 * pl.d
