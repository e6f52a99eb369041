"""GPU backward (sf_fit_backward) against the FP64 oracle's analytic adjoint.

The oracle's adjoint is itself pinned to central finite differences of the
oracle forward on the CPU (tests/test_oracle.py).  Pixels whose gradient
involves a near-degenerate window (gamma < 1e-2 anywhere in their k x k
neighbourhood) are excluded: there the eigenvector derivative scales with
1 / (lambda1 - lambda0) and the gradient is ill-posed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import scenes

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitter  # noqa: E402

GAP_MIN = 1e-2
REL_TOL = 2e-3  # of the largest gradient magnitude in the frame
# and per pixel: |g - g_ref| <= PIX_REL |g_ref| + PIX_FLOOR max |g_ref|
PIX_REL = 1e-3
PIX_FLOOR = 1e-5


def _check_per_pixel(g, ref, sel, label=""):
    scale = np.abs(ref[sel]).max()
    bound = PIX_REL * np.abs(ref[sel]) + PIX_FLOOR * scale
    excess = np.abs(g[sel] - ref[sel]) / bound
    assert excess.max() <= 1.0, "%s: per-pixel gradient error %g of its bound (%d pixels over)" % (
        label, excess.max(), int((excess > 1).sum()))
    return float(excess.max())


def _box_min(a, r):
    H, W = a.shape
    out = np.full_like(a, np.inf)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            sh = np.full_like(a, np.inf)
            ys, yd = (slice(max(0, dy), H + min(0, dy)), slice(max(0, -dy), H + min(0, -dy)))
            xs, xd = (slice(max(0, dx), W + min(0, dx)), slice(max(0, -dx), W + min(0, -dx)))
            sh[yd, xd] = a[ys, xs]
            out = np.minimum(out, sh)
    return out


def _compare(depth, intr, k, method, gn, gd, gk, min_frac=0.5):
    H, W = depth.shape
    ref_fwd = oracle.fit(depth, intr, k, method, want_lambda=True)
    ok = np.isfinite(ref_fwd["offsets"])
    gn = np.where(ok[..., None], gn, 0.0)
    gd = np.where(ok, gd, 0.0)
    gk = np.where(ok, gk, 0.0)
    ref = oracle.backward(depth, intr, k, gn, gd, gk, method)
    f = SurfaceFitter(intr, W, H, k, method=method)
    g = f.backward(torch.from_numpy(depth).cuda(), torch.from_numpy(gn.astype(np.float32)).cuda(),
                   torch.from_numpy(gd.astype(np.float32)).cuda(), torch.from_numpy(gk.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    f.close()
    lam = ref_fwd["lam"]
    gap = np.where(ok, (lam[..., 1] - lam[..., 0]) / np.where(ok, lam[..., 2], 1.0), np.inf)
    good = _box_min(gap, k // 2) >= GAP_MIN
    valid = depth > 0
    assert np.all(g[~valid] == 0.0)
    sel = good & valid
    scale = np.abs(ref[sel]).max()
    err = np.abs(g[sel] - ref[sel]).max() / scale
    assert sel.mean() > min_frac
    assert err < REL_TOL, err
    _check_per_pixel(g, ref, sel, "%s k=%d" % (method, k))
    return err, sel.mean()


@pytest.mark.parametrize("method", ["disparity", "standard"])
@pytest.mark.parametrize("k", [5, 9, 31])
def test_backward_matches_oracle_adjoint(method, k):
    W, H = (96, 72) if k < 31 else (200, 150)
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 60 + k, intr, W, H, n_planes=2)
    rng = np.random.Generator(np.random.PCG64(7))
    err, frac = _compare(depth, intr.as_tuple(), k, method, rng.standard_normal((H, W, 3)),
                         rng.standard_normal((H, W)), rng.standard_normal((H, W)) * 10)
    print(method, k, err, frac)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_backward_normal_and_curvature_loss_640x480_k9(method):
    """Loss = sum over valid pixels of |n - n*|^2 + 0.1 kappa, seeded targets n* (n*_z < 0)."""
    W, H, k = 640, 480, 9
    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 500, intr, W, H)
    ref_fwd = oracle.fit(depth, intr.as_tuple(), k, method)
    tgt = scenes.target_normals(scenes.BASE_SEED + 501, H, W)
    gn = 2.0 * (np.nan_to_num(ref_fwd["normals"]) - tgt)
    err, frac = _compare(depth, intr.as_tuple(), k, method, gn, np.zeros((H, W)), np.full((H, W), 0.1))
    print(method, err, frac)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_backward_640x480_k31(method):
    """The largest window: every pixel sums 961 windows' contributions (box sums of the adjoint
    channels), against the oracle's direct sum over the same windows."""
    W, H, k = 640, 480, 31
    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 510, intr, W, H)
    rng = np.random.Generator(np.random.PCG64(31))
    err, frac = _compare(depth, intr.as_tuple(), k, method, rng.standard_normal((H, W, 3)),
                         rng.standard_normal((H, W)), rng.standard_normal((H, W)) * 10, min_frac=0.3)
    print(method, err, frac)


def test_autograd_function_matches_direct_backward():
    W, H, k = 128, 96, 9
    intr = scenes.Intrinsics.scaled(W, H)
    frames = np.stack([scenes.kinect_frame(70 + i, intr, W, H) for i in range(2)])
    f = SurfaceFitter(intr.as_tuple(), W, H, k)
    d = torch.from_numpy(frames).cuda().requires_grad_(True)
    n, off, cu = f.fit_differentiable(d)
    tgt = torch.from_numpy(np.stack([scenes.target_normals(80 + i, H, W) for i in range(2)]).astype(np.float32)).cuda()
    valid = torch.isfinite(off)
    diff = torch.where(valid[..., None], n - tgt, torch.zeros_like(n))
    loss = (diff ** 2).sum() + 0.1 * torch.where(valid, cu, torch.zeros_like(cu)).sum()
    loss.backward()
    # the autograd backward follows the fit of the same (unmodified) tensor: it reuses the fit's row pass
    assert f.backward_reuses() == 1
    gn = torch.where(valid[..., None], 2 * (n.detach() - tgt), torch.zeros_like(n))
    gk = torch.where(valid, torch.full_like(cu, 0.1), torch.zeros_like(cu))
    direct = f.backward(d.detach(), gn, torch.zeros_like(off), gk)
    torch.cuda.synchronize()
    assert torch.allclose(d.grad, direct, rtol=1e-5, atol=1e-6 * direct.abs().max().item())
    f.close()


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_backward_after_fit_reuses_the_row_pass(method):
    """SF_BACKWARD_AFTER_FIT: a backward that follows the fit of the same frames takes that fit's quantum and
    row sums instead of computing them again, and gives the same gradient bit for bit; where the scratch no
    longer holds those frames (another fit, changed settings) the library runs the row pass itself."""
    W, H, k = 200, 150, 9
    intr = scenes.Intrinsics.scaled(W, H)
    d = torch.from_numpy(np.stack([scenes.kinect_frame(scenes.BASE_SEED + 210 + i, intr, W, H)
                                   for i in range(3)])).cuda()
    other = torch.from_numpy(np.stack([scenes.kinect_frame(scenes.BASE_SEED + 220 + i, intr, W, H)
                                       for i in range(3)])).cuda()
    rng = np.random.Generator(np.random.PCG64(23))
    gn = torch.from_numpy(rng.standard_normal((3, H, W, 3)).astype(np.float32)).cuda()
    gd = torch.from_numpy(rng.standard_normal((3, H, W)).astype(np.float32)).cuda()
    gk = torch.from_numpy(rng.standard_normal((3, H, W)).astype(np.float32)).cuda()
    f = SurfaceFitter(intr.as_tuple(), W, H, k, method=method)
    ref = f.backward(d, gn, gd, gk).clone()           # no promise: the row pass runs
    f.fit(d)
    got = f.backward(d, gn, gd, gk, after_fit=True)   # reuses the fit's row pass
    torch.cuda.synchronize()
    assert f.backward_reuses() == 1 and torch.equal(got, ref)
    f.fit(d)
    f.fit(other)                                      # the scratch now holds other frames
    got = f.backward(d, gn, gd, gk, after_fit=True)
    torch.cuda.synchronize()
    assert f.backward_reuses() == 1 and torch.equal(got, ref)
    got = f.backward(d, gn, gd, gk, after_fit=True)   # the previous backward left d's row pass in place
    torch.cuda.synchronize()
    assert f.backward_reuses() == 2 and torch.equal(got, ref)
    f.fit(d)
    f.set_params(method, min_valid=3)                 # a settings call: the context's generation moves on
    got = f.backward(d, gn, gd, gk, after_fit=True)
    torch.cuda.synchronize()
    assert f.backward_reuses() == 2 and torch.equal(got, ref)
    f.close()


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_backward_uint16_frame_batch(method):
    """uint16 millimetre frames fitted and differentiated as one batch of 3: each frame's dL/dZ (metres)
    matches the oracle's adjoint of that frame alone."""
    W, H, k = 160, 120, 7
    intr = scenes.Intrinsics(115.0, 115.0, 79.5, 59.5)
    frames = [scenes.structured_light_frame(scenes.BASE_SEED + 170 + i, intr, W, H) for i in range(3)]
    rng = np.random.Generator(np.random.PCG64(17))
    gns, gds, gks, refs, goods = [], [], [], [], []
    for u in frames:
        fwd = oracle.fit(u, intr.as_tuple(), k, method, want_lambda=True)
        ok = np.isfinite(fwd["offsets"])
        gn = np.where(ok[..., None], rng.standard_normal((H, W, 3)), 0.0)
        gd = np.where(ok, rng.standard_normal((H, W)), 0.0)
        gk = np.where(ok, rng.standard_normal((H, W)) * 10, 0.0)
        refs.append(oracle.backward(u, intr.as_tuple(), k, gn, gd, gk, method))
        lam = fwd["lam"]
        gap = np.where(ok, (lam[..., 1] - lam[..., 0]) / np.where(ok, lam[..., 2], 1.0), np.inf)
        goods.append((_box_min(gap, k // 2) >= GAP_MIN) & (u > 0))
        gns.append(gn); gds.append(gd); gks.append(gk)
    f = SurfaceFitter(intr.as_tuple(), W, H, k, method=method, depth_type="u16")
    t = torch.from_numpy(np.stack(frames).view(np.int16)).cuda().view(torch.uint16)
    as_t = lambda a: torch.from_numpy(np.stack(a).astype(np.float32)).cuda()
    g = f.backward(t, as_t(gns), as_t(gds), as_t(gks))
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    f.close()
    for i, (ref, sel) in enumerate(zip(refs, goods)):
        assert np.all(g[i][frames[i] == 0] == 0.0)
        assert sel.mean() > 0.4
        err = np.abs(g[i][sel] - ref[sel]).max() / np.abs(ref[sel]).max()
        assert err < REL_TOL, (i, err)
        _check_per_pixel(g[i], ref, sel, "frame %d" % i)
