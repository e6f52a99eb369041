"""Precision fallback (sf_set_precision): refinement of near-degenerate windows.

Mode 1 queues every window whose float32 eigen-gap is below tau and refines
its normal in double-float from the same exact integer moments, re-summing
the depth where the fixed-point rounding could move the normal; mode 2 does so
for every window.  With the fallback the tolerances hold down to the
degeneracy cut gamma = 1e-6 (mode 0 needs gamma >= 1e-3).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import scenes
from parity import compare

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitter  # noqa: E402


def _gpu(depth, intr, k, method, mode, tau=1e-3):
    H, W = depth.shape
    f = SurfaceFitter(intr, W, H, k, method=method)
    f.set_precision(mode, tau)
    out = f.fit(torch.from_numpy(depth).cuda(), counts=True)
    torch.cuda.synchronize()
    f.close()
    return tuple(t.cpu().numpy() for t in out)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_fallback_extends_tolerance_to_small_gaps(method, mode):
    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    depth = scenes.kinect_frame(scenes.BASE_SEED, intr, 640, 480)
    ref = oracle.fit(depth, intr.as_tuple(), 7, method, want_lambda=True, want_moments=True)
    s = compare(_gpu(depth, intr.as_tuple(), 7, method, mode), ref, gap_min=1e-6, angle_tol=1e-4,
                label="%s mode %d" % (method, mode))
    print(method, mode, s)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_fallback_benchmark_frame_1080p_k31(method):
    """The first 1920x1080 frame of the benchmark batch, k = 31, mode 1: every window with gamma >= 1e-6."""
    W, H = 1920, 1080
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.wide_range_frame(scenes.BASE_SEED + 300, intr, W, H)
    ref = oracle.fit(depth, intr.as_tuple(), 31, method, want_lambda=True, want_moments=True)
    s = compare(_gpu(depth, intr.as_tuple(), 31, method, 1), ref, gap_min=1e-6, label="1080p k=31 %s" % method)
    print(method, s)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_fallback_wide_range_k31(method):
    W, H = 480, 270
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.wide_range_frame(scenes.BASE_SEED + 2, intr, W, H)
    ref = oracle.fit(depth, intr.as_tuple(), 31, method, want_lambda=True, want_moments=True)
    compare(_gpu(depth, intr.as_tuple(), 31, method, 1), ref, gap_min=1e-6, label="wide k=31 %s" % method)


def test_mode1_leaves_well_conditioned_windows_untouched():
    intr = scenes.Intrinsics(525.0, 525.0, 159.5, 119.5)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 9, intr, 320, 240)
    a = _gpu(depth, intr.as_tuple(), 7, "disparity", 0)
    b = _gpu(depth, intr.as_tuple(), 7, "disparity", 1, 1e-3)
    ref = oracle.fit(depth, intr.as_tuple(), 7, "disparity", want_lambda=True)
    lam = ref["lam"]
    ok = np.isfinite(ref["offsets"])
    gap = np.where(ok, (lam[..., 1] - lam[..., 0]) / np.where(ok, lam[..., 2], 1), 0)
    far = ok & (gap > 5e-2)
    assert np.array_equal(a[0][far], b[0][far]) and np.array_equal(a[1][far], b[1][far])
    assert np.array_equal(a[3], b[3])


def test_precision_argument_checks():
    f = SurfaceFitter((525.0, 525.0, 31.5, 23.5), 64, 48, 5)
    with pytest.raises(Exception):
        f.set_precision(3)
    with pytest.raises(Exception):
        f.set_precision(1, 0.0)
    f.close()
