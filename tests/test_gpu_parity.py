"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Counts and validity masks must match bit for bit; normals within 1e-3 rad and
offsets within 1e-4 relative on non-degenerate windows (tests/parity.py).
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

from paper_2103_06644_gb300 import SurfaceFitter  # noqa: E402


def run_gpu(depth, intr, k, method, depth_type="f32", depth_scale=1e-3, **kw):
    H, W = depth.shape[-2:]
    f = SurfaceFitter(intr, W, H, k, method=method, depth_type=depth_type, depth_scale=depth_scale, **kw)
    t = torch.from_numpy(depth.view(np.int16) if depth.dtype == np.uint16 else depth).cuda()
    if depth.dtype == np.uint16:
        t = t.view(torch.uint16)
    n, d, c, cnt = f.fit(t, counts=True)
    torch.cuda.synchronize()
    out = (n.cpu().numpy(), d.cpu().numpy(), c.cpu().numpy(), cnt.cpu().numpy())
    f.close()
    return out


def run_ref(depth, intr, k, method, depth_scale=1e-3, **kw):
    return oracle.fit(depth, intr, k, method, want_lambda=True, want_moments=True, depth_scale=depth_scale, **kw)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_kinect_640x480_k7(method):
    """One 640x480 float32 frame: 3 planes at 0.8-4 m, sigma 0.0012 Z^2, 5% missing, 7x7."""
    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    depth = scenes.kinect_frame(scenes.BASE_SEED, intr, 640, 480)
    s = compare(run_gpu(depth, intr.as_tuple(), 7, method), run_ref(depth, intr.as_tuple(), 7, method),
                label="640x480 " + method)
    assert s["good"] > 0.9 * s["valid"]
    print(method, s)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 40), (40, 1), (37, 23), (200, 150), (130, 257)])
@pytest.mark.parametrize("k", [1, 3, 7, 15, 31])
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_ragged_sizes_and_windows(W, H, k, method):
    intr = scenes.Intrinsics.scaled(W, H) if W > 1 else scenes.Intrinsics(525.0, 525.0, 0.0, (H - 1) / 2)
    depth = scenes.kinect_frame(1000 + W * 7 + H, intr, W, H)
    compare(run_gpu(depth, intr.as_tuple(), k, method), run_ref(depth, intr.as_tuple(), k, method),
            label="%dx%d k=%d %s" % (W, H, k, method))


@pytest.mark.parametrize("k", [5, 9, 15])
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_uint16_structured_light(k, method):
    """uint16 millimetres, 4-8 planes + sphere, disparity-quantised, blob holes."""
    W, H = 320, 180
    intr = scenes.Intrinsics(920.0 / 4, 920.0 / 4, 159.5, 89.5)
    depth = scenes.structured_light_frame(scenes.BASE_SEED + 1, intr, W, H)
    compare(run_gpu(depth, intr.as_tuple(), k, method, depth_type="u16"),
            run_ref(depth, intr.as_tuple(), k, method), label="u16 k=%d %s" % (k, method))


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_wide_depth_range_k31(method):
    """Depths 0.3-10 m, sigma 0.0015 Z^2, 31x31 windows."""
    W, H = 480, 270
    intr = scenes.Intrinsics.scaled(W, H, f640=525.0)
    depth = scenes.wide_range_frame(scenes.BASE_SEED + 2, intr, W, H)
    s = compare(run_gpu(depth, intr.as_tuple(), 31, method), run_ref(depth, intr.as_tuple(), 31, method),
                label="wide k=31 " + method)
    print(method, s)


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_noise_free_plane(method):
    W, H = 160, 120
    intr = scenes.Intrinsics(300.0, 310.0, 80.2, 59.7, 0.3, -0.2)
    Z, pl = scenes.single_plane_frame(5, intr, W, H)
    depth = scenes.to_f32_metres(Z)
    n, d, c, cnt = run_gpu(depth, intr.as_tuple(), 5, method)
    from parity import angle
    assert np.max(angle(n, pl.n[None, None, :])) < 2e-4
    assert np.max(np.abs(d - pl.d)) < 1e-4 * pl.d
    assert np.max(c) < 1e-5


def test_all_missing_and_flags():
    W, H = 70, 50
    intr = (525.0, 525.0, 34.5, 24.5, 0.0, 0.0)
    depth = np.zeros((H, W), np.float32)
    n, d, c, cnt = run_gpu(depth, intr, 5, "disparity")
    assert np.all(np.isnan(d)) and np.all(cnt == 0)
    depth = scenes.kinect_frame(3, scenes.Intrinsics.scaled(W, H), W, H, missing_iid=0.3)
    for mv, rc in [(1, False), (10, True), (25, False)]:
        compare(run_gpu(depth, intr, 5, "disparity", min_valid=mv, require_center=rc),
                run_ref(depth, intr, 5, "disparity", min_valid=mv, require_center=rc), label="flags")


def test_batched_frames_match_single():
    W, H, k = 200, 120, 9
    intr = scenes.Intrinsics.scaled(W, H)
    frames = np.stack([scenes.kinect_frame(50 + i, intr, W, H) for i in range(5)])
    f = SurfaceFitter(intr.as_tuple(), W, H, k)
    nb, db, cb = f.fit(torch.from_numpy(frames).cuda())
    for i in range(5):
        n1, d1, c1 = f.fit(torch.from_numpy(frames[i]).cuda())
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(nb[i], 7.0), torch.nan_to_num(n1, 7.0))
        assert torch.equal(torch.nan_to_num(db[i], 7.0), torch.nan_to_num(d1, 7.0))
    f.close()


@pytest.mark.parametrize("nfr", [1, 3, 5, 8])
@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_host_api_matches_device(nfr, method):
    """sf_fit_host (chunked over two streams, pageable buffers) == sf_fit_ex, bit for bit."""
    W, H, k = 128, 96, 7
    intr = scenes.Intrinsics.scaled(W, H)
    frames = np.stack([scenes.kinect_frame(80 + i, intr, W, H) for i in range(nfr)])
    f = SurfaceFitter(intr.as_tuple(), W, H, k, method=method)
    for counts in (True, False):
        host = f.fit_host(frames, counts=counts)
        dev = f.fit(torch.from_numpy(frames).cuda(), counts=counts)
        torch.cuda.synchronize()
        for h, d in zip(host, dev):
            assert np.array_equal(np.nan_to_num(h, nan=7.0), np.nan_to_num(d.cpu().numpy(), nan=7.0))
    # caller-owned result arrays
    outs = (np.empty(frames.shape + (3,), np.float32), np.empty(frames.shape, np.float32),
            np.empty(frames.shape, np.float32))
    r = f.fit_host(frames, out=outs)
    assert r[0] is outs[0] and np.array_equal(np.nan_to_num(outs[1], nan=7.0), np.nan_to_num(host[1], nan=7.0))
    with pytest.raises(ValueError):
        f.fit_host(frames, out=(outs[0][..., :2], outs[1], outs[2]))
    # a host call between device calls on the same context (shared scratch)
    d0 = f.fit(torch.from_numpy(frames).cuda())
    h1 = f.fit_host(frames[::-1].copy())
    d2 = f.fit(torch.from_numpy(frames).cuda())
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(d0[1], 7.0), torch.nan_to_num(d2[1], 7.0))
    assert np.array_equal(np.nan_to_num(h1[1][::-1], nan=7.0), np.nan_to_num(d2[1].cpu().numpy(), nan=7.0))
    f.close()


@pytest.mark.parametrize("depth_type", ["f32", "u16"])
def test_unaligned_frame_bases(depth_type):
    """Frames whose base is not 16-byte aligned (odd pixel counts, sliced batches) are read correctly,
    and a buffer not aligned to its element size is rejected before any work."""
    from paper_2103_06644_gb300 import SurfFitError, _native

    W, H, k = 37, 23, 7  # 851 px: every frame of a stacked batch starts at a different 16-byte phase
    intr = scenes.Intrinsics.scaled(W, H)
    frames = []
    for i in range(5):
        z = scenes.kinect_frame(scenes.BASE_SEED + 60 + i, intr, W, H)
        frames.append(np.where(z > 0, np.round(z * 1000.0), 0).astype(np.uint16) if depth_type == "u16" else z)
    stack = np.stack(frames)
    t = torch.from_numpy(stack.view(np.int16) if depth_type == "u16" else stack).cuda()
    if depth_type == "u16":
        t = t.view(torch.uint16)
    f = SurfaceFitter(intr.as_tuple(), W, H, k, depth_type=depth_type)
    out = f.fit(t[1:], counts=True)  # the slice starts 851 elements in
    torch.cuda.synchronize()
    for i in range(4):
        ref = oracle.fit(frames[i + 1], intr.as_tuple(), k, "disparity", want_lambda=True, want_moments=True)
        compare(tuple(o[i].cpu().numpy() for o in out), ref, label="frame %d of a sliced batch" % (i + 1))
    n, d, c = (torch.empty((H, W, 3), device="cuda"), torch.empty((H, W), device="cuda"),
               torch.empty((H, W), device="cuda"))
    with pytest.raises(SurfFitError):
        _native.check(_native.lib().sf_fit_ex(f._h, 1, t.data_ptr() + 1, n.data_ptr(), n.data_ptr(), n.data_ptr(),
                                              None, None))
    with pytest.raises(SurfFitError):
        _native.check(_native.lib().sf_fit_ex(f._h, 1, t.data_ptr(), n.data_ptr() + 2, d.data_ptr(), c.data_ptr(),
                                              None, None))
    f.close()


@pytest.mark.parametrize("method", ["disparity", "explicit_disparity"])
def test_row_sums_beyond_32_bits(method):
    """A near surface (0.3 m) beside missing pixels: the row sums of w j reach ~2^33 at k = 31, so their
    high part (packed with the mask moments) is nonzero; results must still match the oracle."""
    W, H, k = 160, 96, 31
    intr = scenes.Intrinsics.scaled(W, H)
    rng = np.random.Generator(np.random.PCG64(scenes.BASE_SEED + 71))
    x = np.arange(W)[None, :]
    y = np.arange(H)[:, None]
    depth = (0.3 + 0.0004 * x + 0.0003 * y + rng.normal(0.0, 2e-5, (H, W))).astype(np.float32)
    depth[:, W // 2:] = 0.0                       # missing right half
    depth[H // 3: H // 3 + 4, :] = 9.5            # a far strip sets the quantum's dynamic range
    depth[H // 3: H // 3 + 4, W // 2:] = 0.0
    ref = oracle.fit(depth, intr.as_tuple(), k, method, want_lambda=True, want_moments=True)
    # the largest |row sum of w j| in fixed-point units (26 bits at k = 31): beyond int32
    wq = np.where(depth > 0, 1.0 / np.where(depth > 0, depth, 1.0), 0.0)
    wq = wq / wq.max() * 2.0 ** 26
    r = k // 2
    j = np.arange(-r, r + 1)
    rows = np.array([[np.dot(wq[yy, xx - r: xx + r + 1], j) for xx in range(r, W - r)] for yy in range(0, H, 8)])
    assert np.abs(rows).max() > 2.0 ** 32
    gpu = run_gpu(depth, intr.as_tuple(), k, method)
    if method == "disparity":
        compare(gpu, ref, label="near surface beside missing pixels")
    else:
        from parity import compare_explicit
        compare_explicit(gpu, ref, method, label="near surface beside missing pixels (explicit)")


@pytest.mark.parametrize("method", ["disparity", "standard", "explicit_disparity", "explicit_standard"])
def test_tile_shapes_do_not_change_results(method):
    """Every horizontal segment width (8, 16, 32, 64, 128 columns per thread: one kernel each; the
    automatic choice for these small frames is 8) and vertical band height gives bit-identical results:
    the window sums are exact integers whatever the tiling."""
    W, H, k = 300, 170, 15
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 91, intr, W, H)
    t = torch.from_numpy(np.stack([depth, depth[::-1].copy()])).cuda()
    f = SurfaceFitter(intr.as_tuple(), W, H, k, method=method)
    base = [x.clone() for x in f.fit(t, counts=True)]
    for hseg, vband in [(32, 0), (16, 0), (8, 3), (64, 0), (128, 0), (32, 2), (32, 8), (64, 4), (64, 48),
                        (128, 1024)]:
        f.set_tiles(hseg, vband)
        out = f.fit(t, counts=True)
        torch.cuda.synchronize()
        for a, b in zip(base, out):
            assert torch.equal(torch.nan_to_num(a.float(), nan=7.0), torch.nan_to_num(b.float(), nan=7.0)), \
                (method, hseg, vband)
    f.close()
    ref = oracle.fit(depth, intr.as_tuple(), k, method, want_lambda=True, want_moments=True)
    gpu = tuple(x[0].cpu().numpy() for x in base)
    if method.startswith("explicit"):
        from parity import compare_explicit
        compare_explicit(gpu, ref, method, label="tiles " + method)
    else:
        compare(gpu, ref, label="tiles " + method)


def test_repeated_calls_replay_a_graph():
    """A call that repeats the previous one (same buffers, same configuration) is captured in a CUDA graph
    and replayed: the results stay bit-identical to a fresh context's, a refilled input is read, and a
    setting changed between calls takes effect."""
    W, H, k = 160, 120, 7
    intr = scenes.Intrinsics.scaled(W, H)
    d0 = scenes.kinect_frame(scenes.BASE_SEED + 190, intr, W, H)
    d1 = scenes.kinect_frame(scenes.BASE_SEED + 191, intr, W, H)
    t = torch.from_numpy(d0).cuda()
    out = (torch.empty((H, W, 3), device="cuda"), torch.empty((H, W), device="cuda"),
           torch.empty((H, W), device="cuda"))
    f = SurfaceFitter(intr.as_tuple(), W, H, k)
    fresh = SurfaceFitter(intr.as_tuple(), W, H, k)
    ref0 = [x.clone() for x in fresh.fit(t)]
    for _ in range(4):
        f.fit(t, out=out)
        torch.cuda.synchronize()
        for a, b in zip(out, ref0):
            assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    # the first call launches its kernels; the second repeats it, is captured and runs as the graph;
    # the third and fourth replay that graph
    assert f.graph_replays() == 3
    t.copy_(torch.from_numpy(d1))
    f.fit(t, out=out)
    ref1 = fresh.fit(t)
    torch.cuda.synchronize()
    for a, b in zip(out, ref1):
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    f.set_params("disparity", min_valid=40)
    fresh.set_params("disparity", min_valid=40)
    f.fit(t, out=out)
    f.fit(t, out=out)
    ref2 = fresh.fit(t)
    torch.cuda.synchronize()
    for a, b in zip(out, ref2):
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    assert torch.isnan(out[1]).sum() > torch.isnan(ref1[1]).sum()
    f.close()
    fresh.close()


def test_more_frames_than_one_pass():
    """A call of 70 frames runs as two passes (at most 64 frames each); every frame matches its own fit
    bit for bit, including the first frame of the second pass."""
    W, H, k = 40, 30, 5
    intr = scenes.Intrinsics.scaled(W, H)
    frames = np.stack([scenes.kinect_frame(scenes.BASE_SEED + 300 + i, intr, W, H) for i in range(70)])
    f = SurfaceFitter(intr.as_tuple(), W, H, k)
    t = torch.from_numpy(frames).cuda()
    nb, db, cb, kb = f.fit(t, counts=True)
    for i in (0, 37, 63, 64, 69):
        n1, d1, c1, k1 = f.fit(t[i], counts=True)
        torch.cuda.synchronize()
        for a, b in zip((nb[i], db[i], cb[i], kb[i]), (n1, d1, c1, k1)):
            assert torch.equal(torch.nan_to_num(a.float(), nan=7.0), torch.nan_to_num(b.float(), nan=7.0)), i
    f.close()


def test_concurrent_contexts_on_two_streams():
    """Two host threads, each with its own context and stream, fitting different frames at the same time
    (the library releases no global state between them): every result equals the same fit run alone."""
    import threading

    cfgs = [(320, 240, 7, "disparity", scenes.BASE_SEED + 250), (200, 150, 15, "standard", scenes.BASE_SEED + 251)]
    jobs = []
    for W, H, k, method, seed in cfgs:
        intr = scenes.Intrinsics.scaled(W, H)
        t = torch.from_numpy(np.stack([scenes.kinect_frame(seed + i, intr, W, H) for i in range(3)])).cuda()
        f = SurfaceFitter(intr.as_tuple(), W, H, k, method=method)
        ref = [x.clone() for x in f.fit(t, counts=True)]
        torch.cuda.synchronize()
        jobs.append((f, t, ref, torch.cuda.Stream()))
    errors = []

    def work(f, t, ref, stream):
        try:
            with torch.cuda.stream(stream):
                for _ in range(20):
                    out = f.fit(t, counts=True, stream=stream)
                    stream.synchronize()
                    for a, b in zip(out, ref):
                        if not torch.equal(torch.nan_to_num(a.float(), nan=7.0), torch.nan_to_num(b.float(), nan=7.0)):
                            errors.append("mismatch")
                            return
        except Exception as exc:  # pragma: no cover - reported below
            errors.append(repr(exc))

    threads = [threading.Thread(target=work, args=job) for job in jobs]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert errors == []
    for f, _, _, _ in jobs:
        f.close()
