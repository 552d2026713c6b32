"""The synthetic inputs against the recipe they are stated to follow (CPU):
camera intrinsics per configuration, seeded determinism, per-frame motion
bounds, the depth noise models, the 5 % edge dropout, and the dynamic
configuration's movers (count, speed, pixel coverage)."""
import math

import numpy as np
import pytest

from synth import make_sequence
from synth.scenes import CAM_HD, CAM_QVGA, CAM_TINY, CAM_VGA, apply_noise


def test_cameras_of_the_configurations():
    assert (CAM_TINY.width, CAM_TINY.height, CAM_TINY.fx, CAM_TINY.fy, CAM_TINY.cx, CAM_TINY.cy) == \
        (160, 120, 130.0, 130.0, 80.0, 60.0)
    assert (CAM_VGA.width, CAM_VGA.height, CAM_VGA.fx, CAM_VGA.cx, CAM_VGA.cy) == (640, 480, 525.0, 319.5, 239.5)
    # the other resolutions keep the 640x480 horizontal field of view
    for cam in (CAM_HD, CAM_QVGA):
        assert math.isclose(cam.width / cam.fx, CAM_VGA.width / CAM_VGA.fx)
        assert (cam.cx, cam.cy) == ((cam.width - 1) / 2, (cam.height - 1) / 2)
    for cfg, cam in (("tiny", CAM_TINY), ("static", CAM_VGA), ("dynamic", CAM_VGA), ("precision", CAM_HD)):
        assert make_sequence(cfg, 0, n_frames=2).camera == cam


def test_frames_are_seeded_and_independent_of_access_order():
    a = make_sequence("tiny", 3)
    b = make_sequence("tiny", 3)
    d2, rgb2, T2, s2 = a.frame(2)
    b.frame(5)
    e2, c2, U2, t2 = b.frame(2)
    np.testing.assert_array_equal(d2, e2)
    np.testing.assert_array_equal(rgb2, c2)
    np.testing.assert_array_equal(T2, U2)
    assert d2.dtype == np.uint16 and rgb2.dtype == np.uint8 and rgb2.shape == (120, 160, 3)
    assert not np.array_equal(d2, make_sequence("tiny", 4).frame(2)[0])


@pytest.mark.parametrize("cfg", ["tiny", "static", "precision"])
def test_per_frame_motion_is_bounded(cfg):
    seq = make_sequence(cfg, 1)
    P = np.array(seq.poses)
    dt = np.linalg.norm(np.diff(P[:, :3, 3], axis=0), axis=1)
    rel = np.einsum("kji,kjl->kil", P[:-1, :3, :3], P[1:, :3, :3])  # R_k^T R_k+1
    ang = np.degrees(np.arccos(np.clip((np.trace(rel, axis1=1, axis2=2) - 1) / 2, -1, 1)))
    assert dt.max() <= 0.02 and ang.max() <= 1.0
    assert dt.max() > 0.005  # the camera does move
    for T in P:  # proper rotations
        np.testing.assert_allclose(T[:3, :3] @ T[:3, :3].T, np.eye(3), atol=1e-12)
        assert np.linalg.det(T[:3, :3]) > 0


@pytest.mark.parametrize("model,z,sigma", [("kinect", 2.0, 0.0012 + 0.0019 * 1.6 ** 2),
                                           ("kinect", 1.0, 0.0012 + 0.0019 * 0.6 ** 2),
                                           ("quadratic", 2.0, 0.0015 * 4.0)])
def test_depth_noise_models(model, z, sigma):
    rng = np.random.default_rng(0)
    raw = apply_noise(np.full((480, 640), z), rng, model)
    err = raw.astype(np.float64) / 1000.0 - z
    expect = math.sqrt(sigma ** 2 + 1e-6 / 12.0)  # plus the millimetre quantisation
    assert abs(err.mean()) < 3e-4
    assert abs(err.std() / expect - 1.0) < 0.02


def test_edge_dropout_rate_and_location():
    # a depth image with a 5 cm-plus step every 8 columns: a wide edge band
    z = np.where((np.arange(640) // 8) % 2 == 0, 1.5, 1.7)[None, :].repeat(480, axis=0)
    z[:, :3] = np.inf  # a few misses
    rng = np.random.default_rng(1)
    raw = apply_noise(z, rng, "none", dropout=0.05)
    clean = apply_noise(z, np.random.default_rng(1), "none")
    valid = clean > 0
    dropped = valid & (raw == 0)
    assert abs(dropped.sum() / valid.sum() - 0.05) < 0.005
    # only pixels within 2 px of a step drop
    cols = np.where(dropped.any(axis=0))[0]
    steps = np.where(np.diff(np.where(np.isfinite(z[0]), z[0], 1e6)) != 0)[0]
    assert all(np.min(np.abs(c - steps - 0.5)) <= 2.5 for c in cols)


def test_dynamic_configuration_movers():
    seq = make_sequence("dynamic", 0, n_frames=16)
    assert 2 <= seq.n_movers <= 4
    movers = [p for p in seq.scene.prims if p.dynamic]
    assert len(movers) == seq.n_movers
    assert all(0.2 <= np.linalg.norm(p.velocity) <= 1.0 for p in movers)
    cov = [1.0 - seq.frame(i)[3].mean() for i in (0, 15)]
    assert 0.10 <= np.mean(cov) <= 0.40
    assert make_sequence("static", 0, n_frames=2).n_movers == 0
