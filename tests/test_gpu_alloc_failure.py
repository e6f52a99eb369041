"""Allocation failures: every device allocation of the library can be made to fail from the host
(sf_debug_fail_allocs, a fake of the failing cudaMalloc), so each SF_ERR_ALLOC path runs without
exhausting the device.  Each must return SF_ERR_ALLOC, free whatever it had allocated (the library's
count of live device allocations, sf_debug_live_allocs, comes back), and leave the context or batch
usable."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

import scenes

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_06644_gb300 import SurfaceFitBatch, SurfaceFitter, SurfFitError, _native  # noqa: E402

ALLOC = 3  # SF_ERR_ALLOC


def _fail_after(n):
    _native.check(_native.lib().sf_debug_fail_allocs(n))


def _live():
    n = ctypes.c_longlong()
    _native.check(_native.lib().sf_debug_live_allocs(ctypes.byref(n)))
    return n.value


@pytest.fixture(autouse=True)
def _restore():
    yield
    _fail_after(-1)


def test_context_creation_fails_cleanly_at_every_allocation():
    W, H = 640, 480
    intr = scenes.Intrinsics.scaled(W, H)
    base = _live()
    failures = 0
    for rounds in range(3):
        for n in range(0, 40):
            _fail_after(n)
            try:
                f = SurfaceFitter(intr.as_tuple(), W, H, 7)
            except SurfFitError as e:
                assert e.status == ALLOC, str(e)
                assert _live() == base  # every partial allocation freed
                failures += 1
                continue
            _fail_after(-1)
            f.close()
            break
        else:
            pytest.fail("context creation never succeeded")
    _fail_after(-1)
    assert failures >= 3 * 3  # several allocations, each failed in turn
    assert _live() == base


def test_scratch_failures_leave_the_context_usable():
    W, H, k = 320, 240, 7
    intr = scenes.Intrinsics.scaled(W, H)
    depth = scenes.kinect_frame(scenes.BASE_SEED + 210, intr, W, H)
    d = torch.from_numpy(depth).cuda()
    f = SurfaceFitter(intr.as_tuple(), W, H, k)
    ref = [x.clone() for x in f.fit(d)]
    start = _live()
    d4 = torch.stack([d] * 4)
    calls = [
        ("fit of more frames (scratch grows)", lambda: f.fit(d4)),
        ("precision queue", lambda: (f.set_precision(1), f.fit(d))),
        ("backward", lambda: f.backward(d, torch.zeros((H, W, 3), device="cuda"), torch.zeros((H, W), device="cuda"),
                                        torch.zeros((H, W), device="cuda"))),
        ("quadtree", lambda: f.quadtree(d[None], tile=32, max_level=2, tau=1e-2)),
        ("host staging", lambda: f.fit_host(depth)),
    ]
    for name, call in calls:
        before = _live()
        _fail_after(0)
        with pytest.raises(SurfFitError) as exc:
            call()
        assert exc.value.status == ALLOC, name
        assert _live() <= before, name  # nothing half-allocated kept (old scratch may have been released)
        _fail_after(-1)
        f.set_precision(0)
        got = f.fit(d)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0)), name
    f.close()
    assert _live() <= start - 1  # the context's own allocations are gone too


def test_batch_creation_fails_cleanly():
    frames = []
    for i, (W, H, k) in enumerate([(200, 150, 5), (320, 240, 7)]):
        depth, intr = scenes.mixed_frame(1300 + i, W, H)
        frames.append(dict(W=W, H=H, window=k, intrinsics=intr.as_tuple(), depth=torch.from_numpy(depth).cuda()))
    base = _live()
    for n in range(0, 10):
        _fail_after(n)
        try:
            b = SurfaceFitBatch(frames)
        except SurfFitError as e:
            assert e.status == ALLOC, str(e)
            assert _live() == base
            continue
        _fail_after(-1)
        b.run()
        b.check()
        b.close()
        break
    else:
        pytest.fail("batch creation never succeeded")
    _fail_after(-1)
    assert _live() == base
