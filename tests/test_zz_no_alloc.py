"""sf_fit_static: the fit without a context and without device allocation.

Callers that cannot allocate device memory when they need a fit (graph
capture in progress, allocation-free real-time loops, hosts whose allocator
owns the GPU memory) use this entry point; its scratch is a fixed device
array inside the library.  The test calls it through the C ABI on a run of
frames (disparity and standard forms, float32 and uint16 depth, then the
first case again on a new frame) -- no call may see an earlier call's
leftovers -- and checks each result against sf_fit_ex on the same frame bit
for bit: both run the same kernels on exact window sums.  It needs no other
test to have run first.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import scenes

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def lib():
    from paper_2103_06644_gb300 import _native, build
    build.build()
    return _native


def _static_fit(nat, intr, depth, k, method, dt=0, scale=1e-3):
    H, W = depth.shape
    n = torch.full((H, W, 3), 7.0, device="cuda")
    d = torch.full((H, W), 7.0, device="cuda")
    c = torch.full((H, W), 7.0, device="cuda")
    st = nat.lib().sf_fit_static(ctypes.byref(nat.Intrinsics(*intr)), W, H, k, method, dt, scale, 3, 1,
                                 depth.data_ptr(), n.data_ptr(), d.data_ptr(), c.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0, nat.lib().sf_last_error().decode()
    return n, d, c


def _context_fit(nat, intr, depth, k, method, dt=0, scale=1e-3):
    H, W = depth.shape
    h = ctypes.c_void_p()
    assert nat.lib().sf_create(ctypes.byref(nat.Intrinsics(*intr)), W, H, k, ctypes.byref(h)) == 0
    assert nat.lib().sf_set_params(h, method, dt, scale, 3, 1) == 0
    n = torch.empty((H, W, 3), device="cuda")
    d = torch.empty((H, W), device="cuda")
    c = torch.empty((H, W), device="cuda")
    assert nat.lib().sf_fit_ex(h, 1, depth.data_ptr(), n.data_ptr(), d.data_ptr(), c.data_ptr(), None,
                               torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    nat.lib().sf_destroy(h)
    return n, d, c


def _same(a, b):
    for x, y in zip(a, b):
        assert torch.equal(torch.nan_to_num(x, nan=7.0), torch.nan_to_num(y, nan=7.0))
    assert torch.isfinite(b[1]).float().mean().item() > 0.5


def _depth(seed, intr, W, H, dt):
    if dt == 0:
        return torch.from_numpy(scenes.kinect_frame(seed, intr, W, H)).cuda()
    u = scenes.structured_light_frame(seed, intr, W, H)  # uint16 millimetres
    return torch.from_numpy(u.view(np.int16)).cuda().view(torch.uint16)


def test_static_calls_match_context_fit_bit_for_bit(lib):
    # (W, H, k, method, depth type, seed); the last repeats the first on a new frame
    cases = [(640, 480, 7, 0, 0, scenes.BASE_SEED + 11), (320, 240, 15, 1, 0, scenes.BASE_SEED + 12),
             (320, 240, 9, 1, 1, scenes.BASE_SEED + 13), (640, 480, 7, 0, 0, scenes.BASE_SEED + 14)]
    results = []
    for (W, H, k, method, dt, seed) in cases:
        intr = scenes.Intrinsics.scaled(W, H)
        depth = _depth(seed, intr, W, H, dt)
        results.append((intr, depth, k, method, dt, _static_fit(lib, intr.as_tuple(), depth, k, method, dt)))
    torch.cuda.synchronize()
    for intr, depth, k, method, dt, got in results:
        _same(got, _context_fit(lib, intr.as_tuple(), depth, k, method, dt))
    # the two frames of the repeated case differ, and so do their fits
    assert not torch.equal(torch.nan_to_num(results[0][5][1], nan=7.0), torch.nan_to_num(results[3][5][1], nan=7.0))


def test_oversize_frame_is_rejected(lib):
    W, H = 4096, 3072
    intr = scenes.Intrinsics.scaled(W, H)
    depth = torch.zeros((H, W), device="cuda")
    out = torch.zeros((H, W, 3), device="cuda")
    one = torch.zeros((H, W), device="cuda")
    st = lib.lib().sf_fit_static(ctypes.byref(lib.Intrinsics(*intr.as_tuple())), W, H, 31, 0, 0, 1e-3, 3, 1,
                                 depth.data_ptr(), out.data_ptr(), one.data_ptr(), one.data_ptr(), None)
    assert st == 1
    assert "static array" in lib.lib().sf_last_error().decode()
    assert torch.count_nonzero(out).item() == 0
