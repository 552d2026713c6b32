"""Virtual depth (Sec. III-E, second option): the CUDA path against the FP64
oracle, bit-exact on the same temporary model.

The oracle integrates n consecutive frames at their ground-truth poses; its
snapshot (SDF rounded to float32, or to FP16 storage) is imported into both
sides, and both fill the zero pixels of a frame by casting rays from a pose.
Every filled value must be identical (the decisions along a ray are exact on
the GPU: FP32 with an error bound, FP64 in the oracle's order near it).
"""
import numpy as np
import pytest

from synth import make_sequence
from synth.scenes import CAM_VGA

from . import test_gpu_parity as P
from .test_gpu_precision import fp16_snapshot

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_WINDOW = 10  # frames of the temporary model (the paper's n)


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02082_gb300 import build as B
    B.build()
    import paper_1905_02082_gb300.refusion as R
    R.load()
    return R


@pytest.fixture(scope="module")
def O():
    from oracle import oracle as O
    O.build()
    return O


def _window_snapshot(O, seq, voxel, n=N_WINDOW):
    orc = O.OracleVolume(voxel_size=voxel, trunc=P.TAU)
    cam = seq.camera
    for i in range(n):
        d, rgb, T, _ = seq.frame(i)
        orc.integrate(P.orc_frame(O, d, rgb, cam), T)
    return P.to_f32_snapshot(orc.export())


def _holes(depth, seed, frac=0.3):
    """The frame's depth with a random fraction of pixels and a rectangle set
    to zero (the invalid measurements to fill)."""
    rng = np.random.default_rng(seed)
    d = depth.copy()
    d[rng.random(d.shape) < frac] = 0
    h, w = d.shape
    d[h // 4:h // 2, w // 3:w // 2] = 0
    return d


def _both(R, O, snap, cam, voxel, depth, rgb, T, far_raw=0, rows=None, storage=0):
    orc = O.OracleVolume(voxel_size=voxel, trunc=P.TAU)
    orc.import_(snap)
    vol = P.gpu_volume(R, cam, voxel, n_buckets=1 << 16, max_blocks=200000, storage=storage)
    vol.import_(snap)
    g = vol.virtual_depth(P.dev_frame(R, vol, depth, rgb, cam), T, far_raw=far_raw)
    vol.sync()
    o = orc.virtual_depth(P.orc_frame(O, depth, rgb, cam), T, far_raw=None if far_raw == 0 else far_raw, rows=rows)
    return g.cpu().numpy(), o, vol


def test_virtual_depth_bit_exact_tiny(R, O):
    seq = make_sequence("tiny", 4)
    cam = seq.camera
    snap = _window_snapshot(O, seq, 0.02)
    filled = 0
    for i, seed in ((0, 1), (4, 2), (9, 3)):
        d, rgb, T, _ = seq.frame(i)
        holes = _holes(d, seed)
        for Tq in (T, O.se3_exp(np.array([0.01, -0.02, 0.015, 0.01, -0.005, 0.008])) @ T):
            g, o, vol = _both(R, O, snap, cam, 0.02, holes, rgb, Tq)
            np.testing.assert_array_equal(g, o)
            np.testing.assert_array_equal(g[holes > 0], holes[holes > 0])
            filled += int(((holes == 0) & (g != 5000)).sum())
            vol.close()
    assert filled > 10000  # most holes found a surface


def test_virtual_depth_bit_exact_fp16_storage(R, O):
    seq = make_sequence("tiny", 5)
    cam = seq.camera
    snap = fp16_snapshot(_window_snapshot(O, seq, 0.02))
    d, rgb, T, _ = seq.frame(5)
    holes = _holes(d, 7)
    g, o, vol = _both(R, O, snap, cam, 0.02, holes, rgb, T, storage=R.STORAGE_FP16)
    np.testing.assert_array_equal(g, o)
    vol.close()


def test_virtual_depth_full_size_sampled_rows(R, O):
    """640x480 static room, 1 cm voxels, the temporary model of frames 0-9;
    frame 5's depth with 30 % holes, cast from its pose.  The oracle fills 12
    sampled rows (and returns 0 elsewhere); those rows must match exactly."""
    seq = make_sequence("static", 8, n_frames=N_WINDOW)
    cam = seq.camera
    snap = _window_snapshot(O, seq, 0.01)
    d, rgb, T, _ = seq.frame(5)
    holes = _holes(d, 11)
    rows = list(range(3, cam.height, 40))
    orc = O.OracleVolume(voxel_size=0.01, trunc=P.TAU)
    orc.import_(snap)
    vol = P.gpu_volume(R, cam, 0.01, n_buckets=1 << 18, max_blocks=200000)
    vol.import_(snap)
    g = vol.virtual_depth(P.dev_frame(R, vol, holes, rgb, cam), T)
    vol.sync()
    g = g.cpu().numpy()
    n_holes = 0
    for r in rows:
        o = orc.virtual_depth(P.orc_frame(O, holes, rgb, cam), T, rows=(r, r + 1))
        np.testing.assert_array_equal(g[r], o[r], err_msg=f"row {r}")
        n_holes += int((holes[r] == 0).sum())
    assert n_holes > 1000
    # filled holes sit near the true surface (the rendered depth before the holes)
    sel = (holes == 0) & (d > 0) & (g != 5000)
    assert np.median(np.abs(g[sel].astype(np.int64) - d[sel].astype(np.int64))) < 15
    vol.close()


def test_virtual_depth_rules_and_in_place(R, O):
    """An empty model fills every hole with the far value (d_max or the one
    given); the fill may write into the input buffer itself."""
    cam = CAM_VGA
    vol = P.gpu_volume(R, cam, 0.01, n_buckets=1 << 12, max_blocks=1000)
    rng = np.random.default_rng(2)
    depth = np.where(rng.random((cam.height, cam.width)) < 0.4, 0, 1234).astype(np.uint16)
    rgb = np.zeros((cam.height, cam.width, 3), np.uint8)
    fr = P.dev_frame(R, vol, depth, rgb, cam)
    out = vol.virtual_depth(fr, np.eye(4)).cpu().numpy()
    assert np.all(out[depth == 0] == 5000) and np.all(out[depth > 0] == 1234)
    out = vol.virtual_depth(fr, np.eye(4), far_raw=7777).cpu().numpy()
    assert np.all(out[depth == 0] == 7777)
    d_in = fr._keep[0]
    vol.virtual_depth(fr, np.eye(4), far_raw=4321, out=d_in)  # in place
    vol.sync()
    got = d_in.cpu().numpy()
    assert np.all(got[depth == 0] == 4321) and np.all(got[depth > 0] == 1234)
    with pytest.raises(R.RFError):
        vol.virtual_depth(fr, np.eye(4), far_raw=70000)
    vol.close()
