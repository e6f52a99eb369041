"""Raw disparity input (SF_DEPTH_DISPARITY_U16, sf_set_disparity_model) against
the oracle fed the depth that the input's sensor model defines.

The oracle takes the model 1/Z = alpha D + beta exactly (oracle.depth_from_disparity,
FP64).  The library sums the integers sign(alpha) 128 D + B with
B + f = 128 beta / |alpha| and adds the fraction f to the mean disparity, so its
own representation of the model is judged: no reciprocal, no range pass for the
disparity form.
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

from paper_2103_06644_gb300 import SurfaceFitter, SurfFitError  # noqa: E402

INTR = scenes.Intrinsics(580.0, 580.0, 319.5, 239.5)
STEREO = (1.0 / (8 * 580.0 * 0.075), 0.0)
# a stereo pair with a calibrated disparity offset: beta not a multiple of |alpha| / 128
STEREO_OFFSET = (1.0 / (8 * 580.0 * 0.075), 0.0123)
KINECT = (scenes.KINECT_RAW_ALPHA, scenes.KINECT_RAW_BETA)


def _frame(model, seed):
    if model is KINECT:
        return scenes.disparity_frame(seed, INTR, 640, 480, *model, z_lo=0.6, z_hi=4.0, d_max=2047)
    return scenes.disparity_frame(seed, INTR, 640, 480, *model)


def _gpu(D, model, k, method):
    f = SurfaceFitter(INTR.as_tuple(), 640, 480, k, method=method, depth_type="disparity_u16")
    f.set_disparity_model(*model)
    if method == "standard":
        # depth quantised in disparity steps (a few distinct depths per window, steps of ~0.1 m at
        # 6 m) makes the standard form's float32 solve ill-conditioned (~1e-5 / gamma rad, whatever
        # the input type); these tests check the decoding of the input, so that form runs its FP64
        # solve (the disparity form stays in float32)
        f.set_precision(2)
    t = torch.from_numpy(D.view(np.int16)).cuda().view(torch.uint16)
    out = f.fit(t, counts=True)
    torch.cuda.synchronize()
    f.close()
    return tuple(x.cpu().numpy() for x in out)


@pytest.mark.parametrize("method", ["disparity", "standard", "explicit_disparity"])
@pytest.mark.parametrize("k", [5, 9])
@pytest.mark.parametrize("model", [STEREO, STEREO_OFFSET, KINECT], ids=["stereo", "stereo_offset", "kinect"])
def test_disparity_input_matches_oracle(model, k, method):
    D = _frame(model, 4000 + k)
    Z = oracle.depth_from_disparity(D, *model)
    ref = oracle.fit(Z, INTR.as_tuple(), k, method, want_lambda=True, want_moments=True)
    gpu = _gpu(D, model, k, method)
    if method.startswith("explicit"):
        from parity import compare_explicit
        compare_explicit(gpu, ref, method, label="disparity input %s k=%d" % (method, k))
    else:
        s = compare(gpu, ref, label="disparity input %s k=%d" % (method, k))
        assert s["good"] > 0.8 * s["valid"]


def test_disparity_form_equals_depth_input_on_the_same_depth():
    """The same frame as disparity and as the float32 depth it defines: same windows, same fits."""
    D = _frame(STEREO, 4100)
    Z = oracle.depth_from_disparity(D, *STEREO).astype(np.float32)
    nd, dd, cd, kd = _gpu(D, STEREO, 7, "disparity")
    f = SurfaceFitter(INTR.as_tuple(), 640, 480, 7)
    nz, dz, cz, kz = (x.cpu().numpy() for x in f.fit(torch.from_numpy(Z).cuda(), counts=True))
    f.close()
    assert np.array_equal(kd, kz) and np.array_equal(np.isfinite(dd), np.isfinite(dz))


def test_quadtree_on_disparity_input():
    D = _frame(STEREO, 4200)
    Z = oracle.depth_from_disparity(D, *STEREO)
    tree = oracle.quadtree(Z, INTR.as_tuple(), "disparity", tile=64, max_level=2, tau=2e-2)
    rms = np.array([n["rms"] for n in tree if np.isfinite(n["rms"])])
    assert np.min(np.abs(rms / 2e-2 - 1)) >= 1e-3
    f = SurfaceFitter(INTR.as_tuple(), 640, 480, 5, depth_type="disparity_u16")
    f.set_disparity_model(*STEREO)
    gpu = f.quadtree(torch.from_numpy(D.view(np.int16)).cuda().view(torch.uint16), tile=64, max_level=2, tau=2e-2)
    f.close()
    ref = {(n["level"], n["y0"], n["x0"]): (n["status"], n["count"]) for n in tree}
    got = {(int(r["level"]), int(r["y0"]), int(r["x0"])): (int(r["status"]), int(r["count"])) for r in gpu}
    assert got == ref


def test_disparity_model_arguments_and_unsupported_paths():
    f = SurfaceFitter(INTR.as_tuple(), 64, 48, 5, depth_type="disparity_u16")
    for bad in [(0.0, 0.0), (float("inf"), 0.0), (1e-3, 1e6)]:
        with pytest.raises(SurfFitError):
            f.set_disparity_model(*bad)
    f.set_disparity_model(*STEREO)
    t = torch.ones((48, 64), dtype=torch.int16, device="cuda").view(torch.uint16)
    with pytest.raises(SurfFitError):
        f.backward(t, torch.zeros((48, 64, 3), device="cuda"), torch.zeros((48, 64), device="cuda"),
                   torch.zeros((48, 64), device="cuda"))
    f.close()
