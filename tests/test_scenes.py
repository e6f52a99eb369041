"""Checks of the seeded input generators (they hold no fitting arithmetic)."""
import numpy as np

import scenes


def test_plane_depth_lies_on_plane():
    intr = scenes.Intrinsics(525, 525, 31.5, 23.5, 0.2, -0.1)
    Z, pl = scenes.single_plane_frame(4, intr, 64, 48)
    tx, ty = scenes.rays(intr, 64, 48)
    P = np.stack([Z * tx[None, :], Z * ty[:, None], Z], axis=-1)
    assert np.max(np.abs(P @ pl.n + pl.d)) < 1e-12
    assert pl.d > 0 and abs(np.linalg.norm(pl.n) - 1) < 1e-15


def test_seeded_and_missing_fraction_exact():
    intr = scenes.Intrinsics.scaled(160, 120)
    a = scenes.kinect_frame(3, intr, 160, 120, missing_iid=0.05)
    b = scenes.kinect_frame(3, intr, 160, 120, missing_iid=0.05)
    assert np.array_equal(a, b)
    c = scenes.kinect_frame(4, intr, 160, 120, missing_iid=0.05)
    assert not np.array_equal(a, c)
    assert a.dtype == np.float32


def test_noise_model_of_eq2():
    intr = scenes.Intrinsics(525, 525, 127.5, 95.5)
    Z0, _ = scenes.single_plane_frame(8, intr, 256, 192, z_lo=2.0, z_hi=2.0, max_tilt_deg=0)
    rng = np.random.Generator(np.random.PCG64(1))
    Zn = scenes.add_depth_noise(rng, Z0, scenes.KINECT_SIGMA_COEF)
    s = np.std(Zn - Z0)
    assert abs(s / (scenes.KINECT_SIGMA_COEF * 4.0) - 1) < 0.02


def test_uint16_structured_light_frame():
    intr = scenes.Intrinsics(920, 920, 127.5, 71.5)
    u = scenes.structured_light_frame(2, intr, 256, 144)
    assert u.dtype == np.uint16
    miss = (u == 0).mean()
    assert 0.02 < miss < 0.6
    z = u[u > 0] / 1000.0
    assert z.min() >= 0.45 and z.max() <= 6.1


def test_mixed_batch_spec_draws_from_sets():
    spec = scenes.mixed_batch_spec(64)
    assert len(spec) == 64
    assert {s[:2] for s in spec} <= {(320, 240), (640, 480), (1280, 720), (1920, 1080)}
    assert {s[2] for s in spec} <= {5, 7, 11, 21}
