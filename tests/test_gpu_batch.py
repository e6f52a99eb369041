"""Mixed-resolution batches (sf_batch_*): one persistent launch per pass over a
table of work items (quantum chunks, horizontal tiles, column bands), replayed
from a CUDA graph.

The window sums are exact integers, so a frame's results cannot depend on the
batch it runs in, on its tile shape or on the order in which CTAs claim work:
batch outputs must equal the single-frame fits bit for bit.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import scenes
from parity import compare

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitBatch, SurfaceFitter, SurfFitError  # noqa: E402

SPEC = [(200, 150, 5), (97, 61, 21), (320, 240, 7), (640, 480, 11), (320, 240, 21), (160, 120, 5), (640, 480, 5),
        (131, 257, 7)]


def _frames(seed0=900):
    out = []
    for i, (W, H, k) in enumerate(SPEC):
        depth, intr = scenes.mixed_frame(seed0 + i, W, H)
        out.append(dict(W=W, H=H, window=k, intrinsics=intr.as_tuple(), depth=torch.from_numpy(depth).cuda(),
                        np_depth=depth, intr=intr))
    return out


def _same(a, b):
    return torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))


@pytest.mark.parametrize("method", ["disparity", "standard"])
def test_batch_equals_single_frame_fits(method):
    frames = _frames()
    b = SurfaceFitBatch([{k: v for k, v in f.items() if k not in ("np_depth", "intr")} for f in frames],
                        method=method)
    b.run()
    torch.cuda.synchronize()
    for f, out in zip(frames, b.outputs):
        s = SurfaceFitter(f["intrinsics"], f["W"], f["H"], f["window"], method=method)
        ref = s.fit(f["depth"])
        torch.cuda.synchronize()
        for x, y in zip(out, ref):
            assert _same(x, y)
        s.close()
    # one frame against the FP64 oracle
    f = frames[3]
    r = oracle.fit(f["np_depth"], f["intrinsics"], f["window"], method, want_lambda=True, want_moments=True)
    cnt = SurfaceFitter(f["intrinsics"], f["W"], f["H"], f["window"], method=method).fit(f["depth"], counts=True)[3]
    compare(tuple(t.cpu().numpy() for t in b.outputs[3]) + (cnt.cpu().numpy(),), r, label="batch frame 3")
    b.close()


def test_tiles_and_graph_do_not_change_results():
    frames = [{k: v for k, v in f.items() if k not in ("np_depth", "intr")} for f in _frames(950)]
    a = SurfaceFitBatch(frames, use_graph=False)
    a.run()
    tiled = [dict(f, hseg=[32, 64, 128][i % 3], vband=[8, 32, 64, 256, 1024][i % 5]) for i, f in enumerate(frames)]
    b = SurfaceFitBatch(tiled, use_graph=True)
    b.run()
    b.run()
    torch.cuda.synchronize()
    for oa, ob in zip(a.outputs, b.outputs):
        for x, y in zip(oa, ob):
            assert _same(x, y)
    # refill one input in place: the replayed graph reads the new depth
    new = torch.from_numpy(scenes.mixed_frame(999, frames[2]["W"], frames[2]["H"])[0]).cuda()
    frames[2]["depth"].copy_(new)
    b.run()
    torch.cuda.synchronize()
    s = SurfaceFitter(frames[2]["intrinsics"], frames[2]["W"], frames[2]["H"], frames[2]["window"])
    for x, y in zip(b.outputs[2], s.fit(new)):
        assert _same(x, y)
    a.close()
    b.close()
    s.close()


def test_uint16_batch():
    frames = []
    for i, (W, H, k) in enumerate([(320, 180, 5), (160, 90, 9), (320, 180, 15)]):
        intr = scenes.Intrinsics(230.0 * W / 320, 230.0 * W / 320, (W - 1) / 2, (H - 1) / 2)
        u = scenes.structured_light_frame(1200 + i, intr, W, H)
        frames.append(dict(W=W, H=H, window=k, intrinsics=intr.as_tuple(),
                           depth=torch.from_numpy(u.view(np.int16)).cuda().view(torch.uint16)))
    b = SurfaceFitBatch(frames, depth_type="u16")
    b.run()
    torch.cuda.synchronize()
    for f, out in zip(frames, b.outputs):
        s = SurfaceFitter(f["intrinsics"], f["W"], f["H"], f["window"], depth_type="u16")
        for x, y in zip(out, s.fit(f["depth"])):
            assert _same(x, y)
        s.close()
    b.close()


def test_autotuner_returns_valid_shapes(tmp_path):
    os.environ["SF_TILE_CACHE"] = str(tmp_path / "tiles.json")
    from paper_2103_06644_gb300 import autotune
    frames = [{k: v for k, v in f.items() if k not in ("np_depth", "intr")} for f in _frames(970)[:3]]
    tuned = autotune.tune(frames)
    assert all(t["hseg"] in autotune.HSEGS and t["vband"] in autotune.VBANDS for t in tuned)
    assert os.path.exists(str(tmp_path / "tiles.json"))
    again = autotune.tune(frames)  # from the cache
    assert [(t["hseg"], t["vband"]) for t in again] == [(t["hseg"], t["vband"]) for t in tuned]


@pytest.mark.parametrize("use_graph", [False, True])
def test_one_launch_and_bounded_waits(use_graph):
    """One kernel launch per pass.  With a poll limit of 0 every tile and band that has something to wait
    for gives up at once: the pass ends, sf_batch_check reports SF_ERR_TIMEOUT, and with the limit restored
    the same batch runs again and matches the single-frame fits bit for bit."""
    frames = [{k: v for k, v in f.items() if k not in ("np_depth", "intr")} for f in _frames(980)]
    b = SurfaceFitBatch(frames, use_graph=use_graph)
    assert b.launches == 1
    b.run()
    b.check()
    b.set_wait_limit(0)
    for o in b.outputs:
        o[1].fill_(123.0)
    b.run()
    with pytest.raises(SurfFitError) as exc:
        b.check()
    assert exc.value.status == 5  # SF_ERR_TIMEOUT
    assert any(bool((o[1] == 123.0).any()) for o in b.outputs)  # skipped bands left their outputs unwritten
    b.set_wait_limit(1 << 22)
    b.run()
    b.check()
    torch.cuda.synchronize()
    for f, out in zip(frames, b.outputs):
        s = SurfaceFitter(f["intrinsics"], f["W"], f["H"], f["window"])
        for x, y in zip(out, s.fit(f["depth"])):
            assert _same(x, y)
        s.close()
    b.close()
