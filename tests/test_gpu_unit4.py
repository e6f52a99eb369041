"""GPU fits under the literal constraint of Eq. 4, |(a, b, c, d)| = 1
(sf_set_constraint), against the oracle's 4x4 Jacobi solution (unit4=True).

Counts and masks bit-exact; the normal within 1e-3 rad and the offset within
1e-4 |mu| where the 4x4 problem is well posed.  The float32 solve reaches
lambda by an iteration of 3x3 solves on R_lambda, whose two smallest
eigenvalues can cluster (a line-like R_lambda); its 3x3 solves take the
isolated eigenvalue first.  The float32 mode is judged at 4x4 eigen-gaps
gamma = (lambda1 - lambda0) / lambda2 >= 1e-2, the FP64 modes at 1e-3 and
mode 1 (whose FP64 re-solve covers every window below tau) at 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import scenes
from parity import angle, compare

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitter, SurfFitError  # noqa: E402


def _gpu(depth, intr, k, method, precision=0):
    H, W = depth.shape
    f = SurfaceFitter(intr, W, H, k, method=method)
    f.set_constraint(True)
    if precision:
        f.set_precision(precision)
    out = f.fit(torch.from_numpy(depth).cuda(), counts=True)
    torch.cuda.synchronize()
    f.close()
    return tuple(t.cpu().numpy() for t in out)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_unit4_640x480_k7(method):
    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    depth = scenes.kinect_frame(scenes.BASE_SEED, intr, 640, 480)
    ref = oracle.fit(depth, intr.as_tuple(), 7, method, unit4=True, want_lambda=True, want_moments=True)
    s = compare(_gpu(depth, intr.as_tuple(), 7, method), ref, gap_min=1e-2, check_degenerate=False,
                label="unit4 " + method)
    assert s["good"] > 0.85 * s["valid"]
    print(method, s)
    for mode, gmin in ((1, 1e-5), (2, 1e-3)):
        compare(_gpu(depth, intr.as_tuple(), 7, method, mode), ref, gap_min=gmin, check_degenerate=False,
                label="unit4 %s mode %d" % (method, mode))


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_unit4_wide_range_k31_fp64(method):
    W, H = 480, 270
    intr = scenes.Intrinsics.scaled(W, H, f640=525.0)
    depth = scenes.wide_range_frame(scenes.BASE_SEED + 2, intr, W, H)
    ref = oracle.fit(depth, intr.as_tuple(), 31, method, unit4=True, want_lambda=True, want_moments=True)
    for precision, gmin in ((0, 1e-2), (2, 1e-3)):
        compare(_gpu(depth, intr.as_tuple(), 31, method, precision), ref, gap_min=gmin, check_degenerate=False,
                label="unit4 k31 %s mode %d" % (method, precision))


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_unit4_noise_free_plane_is_exact(method):
    """On a noise-free plane both constraints give the plane itself."""
    W, H = 160, 120
    intr = scenes.Intrinsics(300.0, 310.0, 80.2, 59.7, 0.3, -0.2)
    Z, pl = scenes.single_plane_frame(5, intr, W, H)
    n, d, c, cnt = _gpu(scenes.to_f32_metres(Z), intr.as_tuple(), 5, method)
    assert np.max(angle(n, pl.n[None, None, :])) < 2e-4
    assert np.max(np.abs(d - pl.d)) < 1e-4 * pl.d


def test_unit4_unsupported_combinations():
    W, H = 64, 48
    intr = scenes.Intrinsics.scaled(W, H)
    d = torch.ones((H, W), device="cuda")
    f = SurfaceFitter(intr.as_tuple(), W, H, 5, method="explicit_disparity")
    f.set_constraint(True)
    with pytest.raises(SurfFitError):
        f.fit(d)
    f.set_params("disparity")
    with pytest.raises(SurfFitError):
        f.backward(d, torch.zeros((H, W, 3), device="cuda"), torch.zeros((H, W), device="cuda"),
                   torch.zeros((H, W), device="cuda"))
    with pytest.raises(SurfFitError):
        f.quadtree(d)
    f.close()
