"""GPU fits with a per-pixel table of ray adjustments (sf_set_delta_table) against the oracle's
per-pixel rays (Eq. 1 / Eq. 10 with one adjustment per pixel).

The tables are continuous float32 fields; the library stores them to 1/2^18 pixel and the oracle uses
them as given, so the library's rounding of the rays is part of what is judged: counts and masks
bit-exact, floats within the tolerances of tests/parity.py.
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


def _fit(depth, intr, k, table, depth_type="f32", constraint=False, counts=True, mode=0, stats=None):
    H, W = depth.shape
    f = SurfaceFitter(intr, W, H, k, depth_type=depth_type)
    if constraint:
        f.set_constraint(True)
    if mode:
        f.set_precision(mode)
    if table is not None:
        f.set_delta_table(*table)
    t = torch.from_numpy(depth.view(np.int16) if depth.dtype == np.uint16 else depth).cuda()
    if depth.dtype == np.uint16:
        t = t.view(torch.uint16)
    out = f.fit(t, counts=counts)
    torch.cuda.synchronize()
    if stats is not None:
        stats.extend(f.precision_stats())
    f.close()
    return tuple(x.cpu().numpy() for x in out)


@pytest.mark.parametrize("W,H,k", [(320, 240, 7), (200, 150, 15), (480, 270, 31), (37, 23, 5)])
def test_delta_table_matches_oracle(W, H, k):
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 120 + k, intr, W, H)
    table = scenes.delta_table(scenes.BASE_SEED + 7, intr, W, H, amp=1.5)
    ref = oracle.fit(depth, intr.as_tuple(), k, "disparity", want_lambda=True, want_moments=True, delta=table)
    s = compare(_fit(depth, intr.as_tuple(), k, table), ref, label="delta table %dx%d k=%d" % (W, H, k))
    assert s["good"] > 0.8 * s["valid"]


@pytest.mark.parametrize("W,H,k", [(320, 240, 7), (480, 270, 31)])
@pytest.mark.parametrize("mode", [1, 2])
def test_delta_table_precision_modes(W, H, k, mode):
    """Precision modes with a table: the queued windows (mode 1) or all of them (mode 2) are solved again
    in FP64 from the unrounded depth, so the tolerances hold down to a relative gap of 1e-6."""
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 120 + k, intr, W, H)
    table = scenes.delta_table(scenes.BASE_SEED + 7, intr, W, H, amp=1.5)
    ref = oracle.fit(depth, intr.as_tuple(), k, "disparity", want_lambda=True, want_moments=True, delta=table)
    st = []
    got = _fit(depth, intr.as_tuple(), k, table, mode=mode, stats=st)
    s = compare(got, ref, gap_min=1e-6, label="delta table %dx%d k=%d mode %d" % (W, H, k, mode))
    queued = st[0]
    if mode == 2:
        assert queued == s["valid"]
    else:  # the small window has line-like windows to queue; the large one may have none
        assert queued < s["valid"] and (queued > 0 or k > 7)


@pytest.mark.parametrize("mode", [1, 2])
def test_delta_table_uint16(mode):
    """Millimetre depth through per-pixel rays.  Repeated depth values round alike, so the float32 solve's
    head-on offsets can stray just past the tolerance; the precision modes re-solve from the raw values."""
    W, H, k = 320, 180, 9
    intr = scenes.Intrinsics(230.0, 230.0, 159.5, 89.5)
    u = scenes.structured_light_frame(scenes.BASE_SEED + 131, intr, W, H)
    table = scenes.delta_table(scenes.BASE_SEED + 8, intr, W, H, amp=2.0)
    ref = oracle.fit(u, intr.as_tuple(), k, "disparity", want_lambda=True, want_moments=True, delta=table)
    compare(_fit(u, intr.as_tuple(), k, table, depth_type="u16", mode=mode), ref,
            gap_min=1e-6 if mode == 2 else 1e-3, label="delta table u16 mode %d" % mode)


@pytest.mark.parametrize("mode", [0, 2])
def test_delta_table_unit4(mode):
    W, H, k = 320, 180, 9
    intr = scenes.Intrinsics(230.0, 230.0, 159.5, 89.5)
    table = scenes.delta_table(scenes.BASE_SEED + 8, intr, W, H, amp=2.0)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 132, intr, W, H)
    ref4 = oracle.fit(depth, intr.as_tuple(), k, "disparity", unit4=True, want_lambda=True, want_moments=True,
                      delta=table)
    compare(_fit(depth, intr.as_tuple(), k, table, constraint=True, mode=mode), ref4,
            gap_min=1e-2 if mode == 0 else 1e-6, check_degenerate=False, label="delta table unit4 mode %d" % mode)


def test_noise_free_plane_through_per_pixel_rays():
    """Depth rendered through per-pixel rays: with the table the plane comes back exactly; without it
    (the rays the depth was not rendered with) it does not."""
    W, H, k = 160, 120, 9
    intr = scenes.Intrinsics(150.0, 152.0, 79.5, 59.5)
    table = scenes.delta_table(3, intr, W, H, amp=2.5)
    pl = scenes.plane_through(np.array([0.2, -0.1, 1.6]), np.array([0.35, -0.25, -1.0]))
    Z = scenes.to_f32_metres(scenes.plane_depth_delta(pl, intr, *table))
    n, d, c, cnt = _fit(Z, intr.as_tuple(), k, table)
    assert np.isfinite(d).all()
    assert np.max(angle(n, pl.n[None, None, :])) < 2e-4
    assert np.max(np.abs(d - pl.d)) < 1e-4 * pl.d
    n0, d0, _, _ = _fit(Z, intr.as_tuple(), k, None)
    assert np.max(angle(n0, pl.n[None, None, :])) > 1e-3


def test_zero_table_and_removal():
    """A zero table gives the plain fit (within tolerance of the same oracle); removing the table
    restores the plain path bit for bit."""
    W, H, k = 200, 150, 11
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 140, intr, W, H)
    ref = oracle.fit(depth, intr.as_tuple(), k, "disparity", want_lambda=True, want_moments=True)
    zero = (np.zeros((H, W), np.float32), np.zeros((H, W), np.float32))
    compare(_fit(depth, intr.as_tuple(), k, zero), ref, label="zero table")
    f = SurfaceFitter(intr.as_tuple(), W, H, k)
    t = torch.from_numpy(depth).cuda()
    plain = [x.clone() for x in f.fit(t, counts=True)]
    f.set_delta_table(*scenes.delta_table(9, intr, W, H))
    f.fit(t)
    f.set_delta_table(None, None)
    again = f.fit(t, counts=True)
    torch.cuda.synchronize()
    for a, b in zip(plain, again):
        assert torch.equal(torch.nan_to_num(a.float(), nan=7.0), torch.nan_to_num(b.float(), nan=7.0))
    f.close()


def test_delta_table_arguments_and_unsupported_paths():
    W, H = 64, 48
    intr = scenes.Intrinsics.scaled(W, H)
    d = torch.ones((H, W), device="cuda")
    ok = (np.zeros((H, W), np.float32), np.zeros((H, W), np.float32))
    f = SurfaceFitter(intr.as_tuple(), W, H, 5)
    for bad in [np.full((H, W), 16.0, np.float32), np.full((H, W), np.nan, np.float32)]:
        with pytest.raises(SurfFitError):
            f.set_delta_table(bad, ok[1])
    with pytest.raises(SurfFitError):  # both tables or neither
        from paper_2103_06644_gb300 import _native
        _native.check(_native.lib().sf_set_delta_table(f._h, ok[0].ctypes.data, None))
    f.set_delta_table(*ok)
    for method in ("standard", "explicit_disparity", "explicit_standard"):
        g = SurfaceFitter(intr.as_tuple(), W, H, 5, method=method)
        g.set_delta_table(*ok)
        with pytest.raises(SurfFitError):
            g.fit(d)
        g.close()
    f.set_precision(1)
    f.fit(d)
    f.set_precision(0)
    f.fit(d)
    with pytest.raises(SurfFitError):
        f.backward(d, torch.zeros((H, W, 3), device="cuda"), torch.zeros((H, W), device="cuda"),
                   torch.zeros((H, W), device="cuda"))
    with pytest.raises(SurfFitError):
        f.quadtree(d[None], tile=16, max_level=1, tau=1e-2)
    torch.cuda.synchronize()
    f.close()
