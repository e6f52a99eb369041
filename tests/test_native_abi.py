"""The C ABI library loads, exports every declared entry point, and rejects bad
arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2103_06644_gb300 import build as sfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sfbuild.build()
    from paper_2103_06644_gb300 import _native
    return _native.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sf_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "sf_create" in names and "sf_fit" in names and "sf_destroy" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_declarations():
    from paper_2103_06644_gb300 import _native
    assert set(declared_functions()) <= set(_native.SIGNATURES)


def test_host_argument_checks(lib):
    from paper_2103_06644_gb300 import _native
    K = _native.Intrinsics(525, 525, 319.5, 239.5, 0, 0)
    h = ctypes.c_void_p()
    for W, H, k in [(0, 10, 3), (10, -1, 3), (64, 48, 4), (64, 48, 33), (64, 48, 0)]:
        assert lib.sf_create(ctypes.byref(K), W, H, k, ctypes.byref(h)) == 1
        assert lib.sf_last_error()
    bad = _native.Intrinsics(0, 525, 1, 1, 0, 0)
    assert lib.sf_create(ctypes.byref(bad), 64, 48, 3, ctypes.byref(h)) == 1
    assert lib.sf_create(None, 64, 48, 3, ctypes.byref(h)) == 1
    assert lib.sf_destroy(None) == 0
    assert lib.sf_fit(None, None, None, None, None, None) == 1
    assert lib.sf_set_params(None, 0, 0, 1e-3, 3, 1) == 1
    assert lib.sf_set_delta_table(None, None, None) == 1


def test_channel_counts_follow_the_paper(lib):
    """Section II.D: the RGBD scatter matrix has 4 depth-dependent entries, the standard one 9."""
    import json
    from paper_2103_06644_gb300 import channel_counts
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_cost_model.json")))
    assert channel_counts("disparity")[0] == g["implicit_disparity_depth_channels"]
    assert channel_counts("standard")[0] == g["implicit_standard_depth_channels"]
    assert channel_counts("explicit_disparity")[0] == g["explicit_disparity_depth_channels"]
    d = ctypes.c_int(); m = ctypes.c_int()
    assert lib.sf_channel_counts(9, ctypes.byref(d), ctypes.byref(m)) == 1


def test_no_cuda_device_reports_error_not_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_06644_gb300 import _native
    K = _native.Intrinsics(525, 525, 31.5, 23.5, 0, 0)
    h = ctypes.c_void_p()
    st = lib.sf_create(ctypes.byref(K), 64, 48, 5, ctypes.byref(h))
    assert st in (3, 4)
    assert not h.value
