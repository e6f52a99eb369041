"""The oracle's pins catch plausible mistakes: each case below plants one mistake in a copy of the
C oracle (a dropped term, a wrong index, a flipped sign, a swapped operand, a skipped check),
builds it, and requires at least one of the pins of tests/test_oracle.py to fail against it.
CPU only; the real oracle library is untouched."""
import os
import subprocess

import pytest

import oracle
import test_oracle as pins

# (name, exact text of the correct source, the mistake)
MUTANTS = [
    ("dropped Schur term", "if (!unit4) {\n            for (int i = 0; i < 3; ++i)\n                for (int j = 0; j < 3; ++j) R[i][j] = A[i][j] - g[i] * g[j] / s;",
     "if (!unit4) {\n            for (int i = 0; i < 3; ++i)\n                for (int j = 0; j < 3; ++j) R[i][j] = A[i][j];"),
    ("cx for cy in the row ray", "const double ty0 = (y + dy - cy) / fy;", "const double ty0 = (y + dy - cx) / fy;"),
    ("orientation sign", "if (*d < 0) flip = 1;", "if (*d > 0) flip = 1;"),
    ("curvature from lambda1", "third = tr != 0.0 ? l[0] / tr : 0.0;\n        } else {",
     "third = tr != 0.0 ? l[1] / tr : 0.0;\n        } else {"),
    ("disparity weight Z for 1/Z", "wgt = 1.0 / z; b = wgt;", "wgt = z; b = wgt;"),
    ("offset sign", "d = -(nrm[0] * g[0] + nrm[1] * g[1] + nrm[2] * g[2]) / s;",
     "d = (nrm[0] * g[0] + nrm[1] * g[1] + nrm[2] * g[2]) / s;"),
    ("missing pixels counted", "if (!valid_depth(z)) continue;", "if (z != z) continue;"),
    ("swapped monomials in the standard form", "u[0] = z * tx; u[1] = z * ty; u[2] = z;",
     "u[0] = z * ty; u[1] = z * tx; u[2] = z;"),
    ("explicit standard target sign", "else { v[0] = x[0]; v[1] = x[1]; v[2] = -1.0; d = x[2]; }",
     "else { v[0] = x[0]; v[1] = x[1]; v[2] = 1.0; d = x[2]; }"),
    ("4x4 scatter without the offset row", "R[i][3] = R[3][i] = g[i];", "R[i][3] = R[3][i] = 0.0;"),
    ("window one row short", "return box_sums(Z, W, H, intr, ddx, ddy, method, px - r, px + r, py - r, py + r,",
     "return box_sums(Z, W, H, intr, ddx, ddy, method, px - r, px + r, py - r, py + r - 1,"),
    ("per-pixel x adjustment ignored", "const double tx = ddx ? (x + dx + ddx[q] - cx) / fx",
     "const double tx = ddx ? (x + dx - cx) / fx"),
]

# the pins, with their parameters: any failing one catches the mistake
PINS = [
    (pins.test_noise_free_plane_is_recovered, ("disparity", 5, 1)),
    (pins.test_noise_free_plane_is_recovered, ("standard", 5, 2)),
    (pins.test_noise_free_plane_explicit, ("explicit_disparity",)),
    (pins.test_noise_free_plane_explicit, ("explicit_standard",)),
    (pins.test_noise_free_plane_unit4_literal_constraint, ()),
    (pins.test_rgbd_plane_equals_xyz_plane, ()),
    (pins.test_counts_brute_force_and_validity_rule, ()),
    (pins.test_fit_matches_numpy_twin, ("disparity",)),
    (pins.test_fit_matches_numpy_twin, ("standard",)),
    (pins.test_schur_complement_is_weighted_covariance, ("disparity",)),
    (pins.test_invariants_on_noisy_frame, ("standard",)),
    (pins.test_explicit_fit_is_least_squares, ("explicit_standard",)),
    (pins.test_unit4_and_curvature_match_lapack_on_noisy_windows, ("disparity",)),
    (pins.test_noise_free_plane_with_per_pixel_rays, ("disparity",)),
]


@pytest.fixture
def mutant_oracle(tmp_path, monkeypatch):
    """Returns a function that builds and installs a mutated oracle library."""
    src = open(oracle._SRC).read()

    def install(old, new):
        assert src.count(old) == 1, old
        path = tmp_path / "mutant.c"
        path.write_text(src.replace(old, new))
        lib = tmp_path / ("mutant%d.so" % len(os.listdir(tmp_path)))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", str(lib), str(path), "-lm"])
        monkeypatch.setattr(oracle, "_SRC", str(path))
        monkeypatch.setattr(oracle, "_LIB_PATH", str(lib))
        monkeypatch.setattr(oracle, "_lib", None)

    yield install
    oracle._lib = None  # the next user reloads the real library


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(mutant_oracle, name, old, new):
    mutant_oracle(old, new)
    failed = []
    for fn, args in PINS:
        try:
            fn(*args)
        except Exception as exc:  # an assertion, or the mistake breaking the call itself
            failed.append((fn.__name__, type(exc).__name__))
    assert failed, "no pin caught the planted mistake: %s" % name


def test_pins_pass_on_the_unmodified_oracle(mutant_oracle):
    """The control: the same pins, run against a rebuilt copy of the unmodified source, all pass."""
    mutant_oracle("if (*d < 0) flip = 1;", "if (*d < 0) flip = 1;")
    for fn, args in PINS:
        fn(*args)
