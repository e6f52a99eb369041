"""GPU parity at full workload sizes, in the launch configurations the benchmark times.

A window sees only its k x k neighbourhood, so the FP64 oracle can check a
full-size frame pixel by pixel (``oracle.fit_at``) without fitting all of it.
Each frame is checked at its four corners, at pixels along every border
(ragged windows, frame seams of a stacked batch) and at seeded interior
pixels; counts and validity bit for bit, floats with the tolerances of
tests/parity.py.

Workloads (synthetic, seeded as in the benchmark):
- 8 x 1920x1080 + 2 x 4096x3072 float32 frames, 0.3-10 m, k = 31, each
  resolution fitted as one stacked batch (both forms) in precision mode 1
  (tau = 1e-3), judged on every sampled window with gamma >= 1e-6;
- 30 x 1280x720 uint16 structured-light frames, k in {5, 9, 15} (both forms);
- the 64-frame mixed batch (320x240 .. 1920x1080, k in {5, 7, 11, 21}) with
  autotuned tiles, replayed from a CUDA graph;
- a per-pixel ray table on 1080p and 4K frames of the benchmark, k = 31.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import scenes
from parity import compare

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitBatch, SurfaceFitter, autotune  # noqa: E402


def sample_xy(seed, W, H, k, n_interior=1500, n_edge=48):
    """Corners, pixels within k of each border, and uniform interior pixels: [N, 2] (x, y)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = k // 2
    pts = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1)]
    band = min(k, W), min(k, H)
    for _ in range(n_edge):
        pts.append((int(rng.integers(0, W)), int(rng.integers(0, band[1]))))
        pts.append((int(rng.integers(0, W)), H - 1 - int(rng.integers(0, band[1]))))
        pts.append((int(rng.integers(0, band[0])), int(rng.integers(0, H))))
        pts.append((W - 1 - int(rng.integers(0, band[0])), int(rng.integers(0, H))))
    x = rng.integers(r, max(W - r, r + 1), n_interior)
    y = rng.integers(r, max(H - r, r + 1), n_interior)
    pts += list(zip(x.tolist(), y.tolist()))
    return np.unique(np.clip(np.array(pts, dtype=np.int64), 0, [W - 1, H - 1]), axis=0)


def at(t, xy):
    """Sampled outputs of one frame's [H, W(, 3)] result tensor."""
    a = t.cpu().numpy()
    return a[xy[:, 1], xy[:, 0]]


def check_frame(outs, counts, depth, intr, k, method, xy, label, **kw):
    ref = oracle.fit_at(depth, intr, k, xy, method)
    gpu = tuple(at(t, xy) for t in outs) + (at(counts, xy),)
    return compare(gpu, ref, label=label, **kw)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_wide_range_1080p_and_4k_k31(method):
    """The benchmark's batch: 8 x 1920x1080 and 2 x 4096x3072, k = 31, fitted per resolution in the
    benchmark's precision mode (1, tau = 1e-3)."""
    K = 31
    for (W, H, n, seed0) in [(1920, 1080, 8, scenes.BASE_SEED + 300), (4096, 3072, 2, scenes.BASE_SEED + 400)]:
        intr = scenes.Intrinsics.scaled(W, H)
        frames = [scenes.wide_range_frame(seed0 + i, intr, W, H) for i in range(n)]
        d = torch.from_numpy(np.stack(frames)).cuda()
        f = SurfaceFitter(intr.as_tuple(), W, H, K, method=method)
        f.set_precision(1, 1e-3)
        out = (torch.empty((n, H, W, 3), device="cuda"), torch.empty((n, H, W), device="cuda"),
               torch.empty((n, H, W), device="cuda"))
        f.fit(d, out=out)
        withc = f.fit(d, counts=True)
        torch.cuda.synchronize()
        for a, b in zip(out, withc[:3]):  # asking for counts changes no other output
            assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
        for i in range(n):
            xy = sample_xy(seed0 + 50 + i, W, H, K)
            s = check_frame(tuple(t[i] for t in out), withc[3][i], frames[i], intr.as_tuple(), K, method, xy,
                            "%dx%d frame %d %s" % (W, H, i, method), gap_min=1e-6)
            assert s["good"] > 0.8 * s["valid"], s
        f.close()
        del d, out, withc


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_structured_light_30x720p_u16(method):
    """30 uint16 millimetre frames at 1280x720, fx = fy = 920, windows 5, 9 and 15."""
    W, H = 1280, 720
    intr = scenes.Intrinsics(920.0, 920.0, 639.5, 359.5)
    frames = [scenes.structured_light_frame(scenes.BASE_SEED + 500 + i, intr, W, H) for i in range(30)]
    d = torch.from_numpy(np.stack(frames).view(np.int16)).cuda().view(torch.uint16)
    for k in (5, 9, 15):
        f = SurfaceFitter(intr.as_tuple(), W, H, k, method=method, depth_type="u16")
        n, o, c, cnt = f.fit(d, counts=True)
        torch.cuda.synchronize()
        for i in range(0, 30, 3):
            xy = sample_xy(scenes.BASE_SEED + 550 + i, W, H, k, n_interior=600, n_edge=16)
            check_frame((n[i], o[i], c[i]), cnt[i], frames[i], intr.as_tuple(), k, method, xy,
                        "u16 frame %d k=%d %s" % (i, k, method))
        f.close()


def test_mixed_batch_64_frames_graph():
    """The 64-frame mixed batch with autotuned tiles, one persistent launch per pass from a CUDA graph."""
    spec = scenes.mixed_batch_spec(64)
    frames, host = [], []
    for i, (W, H, k) in enumerate(spec):
        depth, intr = scenes.mixed_frame(scenes.BASE_SEED + 800 + i, W, H)
        host.append((depth, intr))
        frames.append(dict(W=W, H=H, window=k, intrinsics=intr.as_tuple(), depth=torch.from_numpy(depth).cuda()))
    b = SurfaceFitBatch(autotune.tune(frames), use_graph=True)
    b.run()
    b.run()
    torch.cuda.synchronize()
    for i, ((W, H, k), (depth, intr), out) in enumerate(zip(spec, host, b.outputs)):
        f = SurfaceFitter(intr.as_tuple(), W, H, k)
        cnt = f.fit(frames[i]["depth"], counts=True)[3]
        torch.cuda.synchronize()
        xy = sample_xy(scenes.BASE_SEED + 900 + i, W, H, k, n_interior=300, n_edge=8)
        check_frame(out, cnt, depth, intr.as_tuple(), k, "disparity", xy, "mixed frame %d %dx%d k=%d" % (i, W, H, k))
        f.close()
    b.close()


def test_delta_table_1080p_and_4k_k31():
    """The per-pixel ray table at the benchmark's sizes: 2 x 1920x1080 and 1 x 4096x3072, k = 31,
    disparity form, each resolution fitted as one stacked batch."""
    K = 31
    for (W, H, n, seed0) in [(1920, 1080, 2, scenes.BASE_SEED + 300), (4096, 3072, 1, scenes.BASE_SEED + 400)]:
        intr = scenes.Intrinsics.scaled(W, H)
        frames = [scenes.wide_range_frame(seed0 + i, intr, W, H) for i in range(n)]
        table = scenes.delta_table(scenes.BASE_SEED + 600, intr, W, H)
        f = SurfaceFitter(intr.as_tuple(), W, H, K)
        f.set_delta_table(*table)
        nrm, off, cur, cnt = f.fit(torch.from_numpy(np.stack(frames)).cuda(), counts=True)
        torch.cuda.synchronize()
        for i in range(n):
            xy = sample_xy(seed0 + 70 + i, W, H, K, n_interior=800, n_edge=24)
            ref = oracle.fit_at(frames[i], intr.as_tuple(), K, xy, "disparity", delta=table)
            gpu = (at(nrm[i], xy), at(off[i], xy), at(cur[i], xy), at(cnt[i], xy))
            s = compare(gpu, ref, label="delta table %dx%d frame %d" % (W, H, i))
            assert s["good"] > 0.8 * s["valid"], s
        f.close()
