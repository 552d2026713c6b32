"""Bounded failure paths of the library, each made to happen without any GPU
fault: a flood fill capped below the sweeps it needs, a frustum candidate list
too small for the frame, a pose beyond the hash key range, a mesh buffer too
small for the surface, and grid-wide waits that run out (fault injection
through rf_set_wait_limits: the flood fill's barrier and the registration's
arrival count each wait for one arrival more than there are CTAs, which
never comes; each wait gives up after a short, bounded number of polls, and
the kernel returns).  Also the restart of the registration's tag sequence.
Every error is read back through rf_sync_status (or the call's return code),
and the volume keeps working afterwards.
"""
import ctypes as C
import time

import numpy as np
import pytest

from synth import make_sequence
from synth.scenes import CAM_QVGA, Prim

from ._scenes import ROOM, look_at, render_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOT_CONVERGED, BUFFER_TOO_SMALL, OUT_OF_RANGE, CAPACITY = 5, 6, 7, 8
TARGET = np.array([2.0, 2.0, 0.6])


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02082_gb300 import build as B
    B.build()
    import paper_1905_02082_gb300.refusion as R
    R.load()
    return R


def _dev(R, vol, d, rgb, cam):
    dt = torch.from_numpy(d.astype(np.int32)).cuda().to(torch.uint16).contiguous()
    ct = torch.from_numpy(np.ascontiguousarray(rgb)).cuda().contiguous()
    fr = vol.frame(dt, ct, R.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy))
    fr._keep = (dt, ct)
    return fr


def _room_volume(R, cam=CAM_QVGA, **kw):
    vol = R.Volume(n_buckets=1 << 16, max_blocks=120000, max_width=cam.width, max_height=cam.height,
                   voxel_size=0.02, trunc=0.1, **kw)
    for i in range(3):
        T = look_at([0.4 + 0.03 * i, 0.3, 1.3], TARGET)
        d, rgb, _ = render_frame([ROOM], cam, T)
        vol.integrate(_dev(R, vol, d, rgb, cam), T)
    vol.sync()
    return vol


BOX = Prim("box", {"center": np.array([1.3, 1.1, 0.45]), "half": np.array([0.2, 0.2, 0.45]), "yaw": 0.3},
           (0.9, 0.2, 0.2), (4.0, 4.0, 4.0, 0.0, 0.0, 0.0, 5.0, 0.0), dynamic=True)


def _expect_status(R, vol, status):
    with pytest.raises(R.RFError) as e:
        vol.sync()
    assert e.value.status == status, str(e.value)
    vol.sync()  # the status word was cleared


def test_flood_fill_sweep_cap_reports_not_converged(R):
    cam = CAM_QVGA
    T = look_at([0.45, 0.32, 1.31], TARGET)
    d, rgb, dyn = render_frame([ROOM, BOX], cam, T)
    ref = _room_volume(R)
    capped = _room_volume(R, max_ff_sweeps=1)
    fr_ref, fr_cap = _dev(R, ref, d, rgb, cam), _dev(R, capped, d, rgb, cam)
    m_ref = ref.compute_mask(fr_ref, T)
    ref.sync()  # the uncapped fill converges
    assert m_ref.cpu().numpy()[dyn].mean() > 0.5
    capped.compute_mask(fr_cap, T)
    _expect_status(R, capped, NOT_CONVERGED)
    # a frame with nothing to fill converges within the cap: the volume still works
    d2, rgb2, _ = render_frame([ROOM], cam, T)
    m2 = capped.compute_mask(_dev(R, capped, d2, rgb2, cam), T)
    capped.sync()
    assert m2.cpu().numpy().sum() < 0.02 * m2.numel()
    ref.close()
    capped.close()


def test_candidate_overflow_reports_capacity(R):
    seq = make_sequence("tiny", 0, n_frames=1)
    cam = seq.camera
    d, rgb, T, _ = seq.frame(0)
    vol = R.Volume(n_buckets=1 << 14, max_blocks=20000, max_width=cam.width, max_height=cam.height,
                   voxel_size=0.02, max_candidates=10)
    vol.integrate(_dev(R, vol, d, rgb, cam), T)
    _expect_status(R, vol, CAPACITY)
    empty = np.zeros_like(d)  # no valid pixel: no candidates at all
    vol.integrate(_dev(R, vol, empty, rgb, cam), T)
    vol.sync()
    vol.close()


def test_pose_beyond_the_key_range_reports_out_of_range(R):
    seq = make_sequence("tiny", 0, n_frames=1)
    cam = seq.camera
    d, rgb, T, _ = seq.frame(0)
    vol = R.Volume(n_buckets=1 << 14, max_blocks=20000, max_width=cam.width, max_height=cam.height,
                   voxel_size=0.02)
    far = T.copy()
    far[0, 3] += 8192 * 8 * 0.02 + 10.0  # more than 8,191 blocks along x
    vol.integrate(_dev(R, vol, d, rgb, cam), far)
    _expect_status(R, vol, OUT_OF_RANGE)
    vol.integrate(_dev(R, vol, d, rgb, cam), T)
    vol.sync()
    assert vol.stats().n_blocks > 0
    vol.close()


def test_mesh_buffer_too_small(R):
    seq = make_sequence("tiny", 0, n_frames=1)
    cam = seq.camera
    d, rgb, T, _ = seq.frame(0)
    vol = R.Volume(n_buckets=1 << 14, max_blocks=20000, max_width=cam.width, max_height=cam.height,
                   voxel_size=0.02)
    vol.integrate(_dev(R, vol, d, rgb, cam), T)
    vol.sync()
    lib = R.load()
    n = C.c_int64()
    assert lib.rf_extract_mesh(vol.h, None, None, 0, C.byref(n), None) == 0
    need = n.value
    assert need > 10
    verts = torch.empty(4, 3, 3, dtype=torch.float32, device="cuda")
    cols = torch.empty(4, 3, 3, dtype=torch.uint8, device="cuda")
    st = lib.rf_extract_mesh(vol.h, verts.data_ptr(), cols.data_ptr(), 4, C.byref(n), None)
    assert st == BUFFER_TOO_SMALL and n.value == need
    assert b"buffer holds 4" in lib.rf_last_error(vol.h)
    tris, _ = vol.extract_mesh()  # a large enough buffer succeeds
    assert tris.shape[0] == need
    vol.close()


@pytest.mark.parametrize("stage", ["registration", "flood fill"])
def test_grid_wide_waits_run_out_and_are_reported(R, stage):
    """Fault injection on the bounded grid-wide waits (the flood fill's
    barrier and the registration's arrival count each expect one arrival
    more than there are CTAs): every CTA's wait runs out after 2^14 polls (no
    sleeps below 4,096 polls and 64 ns after), the kernel returns, the status
    reads RF_ERR_NOT_CONVERGED, and with the injection removed the same call
    succeeds and gives the normal result."""
    cam = CAM_QVGA
    T = look_at([0.45, 0.32, 1.31], TARGET)
    d, rgb, _ = render_frame([ROOM, BOX], cam, T)
    vol = _room_volume(R)
    fr = _dev(R, vol, d, rgb, cam)

    def run():
        if stage == "registration":
            out, _ = vol.track(fr, T)
            return out
        return vol.compute_mask(fr, T)

    good = run()
    vol.sync()
    vol.set_wait_limits(spin_limit=1 << 14, extra_arrivals=1)
    t0 = time.perf_counter()
    run()
    with pytest.raises(R.RFError) as e:
        vol.sync()
    elapsed = time.perf_counter() - t0
    assert e.value.status == NOT_CONVERGED and "grid-wide wait" in str(e.value)
    assert elapsed < 2.0
    vol.set_wait_limits(0, 0)
    again = run()
    vol.sync()
    np.testing.assert_array_equal(again.cpu().numpy(), good.cpu().numpy())
    vol.close()


def test_registration_tag_sequence_restarts(R):
    """The registration's tags restart at 0 (the partial-sum buffer cleared)
    before they would reach 2^31; a registration right at the limit, the one
    after the restart and one from an arbitrary base all give the pose of a
    registration from the initial base, bit for bit, without an error."""
    cam = CAM_QVGA
    T = look_at([0.45, 0.32, 1.31], TARGET)
    d, rgb, _ = render_frame([ROOM, BOX], cam, T)
    vol = _room_volume(R)
    fr = _dev(R, vol, d, rgb, cam)
    ref, _ = vol.track(fr, T)
    vol.sync()
    span = 3 + 10 + 5 + 5  # 3 + the default iteration caps
    limit = (1 << 31) - 1 - span
    with pytest.raises(R.RFError):
        vol.set_registration_tag_base(limit + 1)
    for base in (limit, None, 12345):
        if base is not None:
            vol.set_registration_tag_base(base)
        out, _ = vol.track(fr, T)
        vol.sync()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    vol.close()
