"""sf_fit_static: the fit without a context and without device allocation.

Callers that cannot allocate device memory when they need a fit (graph
capture in progress, allocation-free real-time loops, hosts whose allocator
owns the GPU memory) use this entry point; its scratch is a fixed device
array inside the library.  The test calls it through the C ABI twice in a
row on different frames -- the second call must not see the first call's
leftovers -- and checks each result against sf_fit_ex on the same frame
with the parity tolerances of the other GPU tests.  It needs no other test
to have run first.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import scenes
from parity import ANGLE_TOL, CURV_TOL, OFFSET_TOL, angle

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


def _context_fit(nat, intr, depth, k, method):
    H, W = depth.shape
    h = ctypes.c_void_p()
    assert nat.lib().sf_create(ctypes.byref(nat.Intrinsics(*intr)), W, H, k, ctypes.byref(h)) == 0
    assert nat.lib().sf_set_params(h, method, 0, 1e-3, 3, 1) == 0
    n = torch.empty((H, W, 3), device="cuda")
    d = torch.empty((H, W), device="cuda")
    c = torch.empty((H, W), device="cuda")
    assert nat.lib().sf_fit_ex(h, 1, depth.data_ptr(), n.data_ptr(), d.data_ptr(), c.data_ptr(), None,
                               torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    nat.lib().sf_destroy(h)
    return n, d, c


def _close(a, b, mu):
    na, da, ca = [t.cpu().numpy() for t in a]
    nb, db, cb = [t.cpu().numpy() for t in b]
    ok = np.isfinite(db)
    assert np.array_equal(np.isfinite(da), ok)
    assert ok.mean() > 0.5
    assert angle(na[ok], nb[ok]).max() <= ANGLE_TOL
    assert (np.abs(da[ok] - db[ok]) / mu[ok]).max() <= OFFSET_TOL
    assert np.abs(ca[ok] - cb[ok]).max() <= CURV_TOL


def test_two_static_calls_match_context_fit(lib):
    cases = [(640, 480, 7, 0, scenes.BASE_SEED + 11), (320, 240, 15, 1, scenes.BASE_SEED + 12)]
    results = []
    for (W, H, k, method, seed) in cases:
        intr = scenes.Intrinsics.scaled(W, H)
        depth = torch.from_numpy(scenes.kinect_frame(seed, intr, W, H)).cuda()
        results.append((intr, depth, k, method, _static_fit(lib, intr.as_tuple(), depth, k, method)))
    torch.cuda.synchronize()
    for intr, depth, k, method, got in results:
        ref = _context_fit(lib, intr.as_tuple(), depth, k, method)
        z = depth.cpu().numpy()
        mu = np.where(z > 0, z, 1.0).astype(np.float64)  # window distance scale: the depth
        _close(got, ref, mu)


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
