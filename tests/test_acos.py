"""The float32 arccos of the per-pixel solve's trigonometric eigenvalue estimate (the closed-form
roots of the 3x3 characteristic polynomial behind Eq. 4-5).

It has the Abramowitz & Stegun 4.4.45 form acos(x) = sqrt(1 - x) P(x) on [0, 1] (pi - acos(-x) below
0) with a degree-6 P.  The CPU test reads P's coefficients from the kernel source and checks the
stated bound of the form in exact arithmetic (FP64 evaluation, error below 9e-8 on a fine grid); the
GPU test runs the device function itself against CUDA's acosf (torch.acos) and against FP64 arccos,
with the float32 bound 1.5e-6.
"""
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2103_06644_gb300", "csrc", "sf_solve.cuh")


def _coefficients():
    src = open(SRC).read()
    body = src[src.index("float acos_fast(float x)"):]
    body = body[:body.index("}")]
    co = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    assert len(co) == 7, co
    return co


def test_polynomial_bound_in_exact_arithmetic():
    co = _coefficients()
    x = np.linspace(0.0, 1.0, 1_000_001)
    p = np.zeros_like(x)
    for c in co:
        p = p * x + c
    err = np.abs(np.sqrt(1.0 - x) * p - np.arccos(x))
    assert err.max() < 9e-8
    # the end points: acos(1) = 0 exactly, acos(0) = pi/2 to float32 rounding of the constant term
    assert abs(co[-1] - np.pi / 2) < 1e-7


@pytest.mark.gpu
def test_device_acos_against_acosf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2103_06644_gb300 import _native

    x = torch.linspace(-1.0, 1.0, 2_000_001, dtype=torch.float32, device="cuda")
    x = torch.cat([x, torch.tensor([-1.0, -0.0, 0.0, 1.0, 1e-30, -1e-30, 0.9999999, -0.9999999], device="cuda")])
    y = torch.empty_like(x)
    _native.check(_native.lib().sf_eval_acos(x.data_ptr(), y.data_ptr(), x.numel(), None))
    ref32 = torch.acos(x)
    torch.cuda.synchronize()
    exact = np.arccos(x.cpu().numpy().astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    assert np.abs(got - exact).max() < 1.5e-6
    assert np.abs(got - ref32.cpu().numpy().astype(np.float64)).max() < 1.5e-6
    assert got[-8] == pytest.approx(np.pi, abs=1e-6) and got[-5] == 0.0
    # monotone non-increasing up to float32 rounding
    assert np.all(np.diff(got[:2_000_001]) <= 2e-7)
