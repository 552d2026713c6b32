"""The allocation-free mask entry point (rf_compute_mask_noalloc).

It serves callers that cannot call cudaMalloc at the time they need a mask
(an application whose own allocator or fixed budget owns all device memory,
or a frame loop that cannot afford cudaMalloc's implicit synchronisation).
Its scratch is a static device array shared by all calls, so this checks
that it reproduces rf_compute_mask exactly on two calls in a row with
different inputs (the second call must not see the first call's leftovers),
that oversize frames are refused, and (with two GPUs) that a current device
other than the volume's is refused.

This file is collected last on purpose: it must pass alone in a fresh process
and after every other test.
"""
import numpy as np
import pytest

from synth.scenes import CAM_QVGA, Prim

from ._scenes import ROOM, look_at, render_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_noalloc_mask_matches_compute_mask_twice(R):
    cam = CAM_QVGA
    vol = R.Volume(n_buckets=1 << 16, max_blocks=120000, max_width=cam.width, max_height=cam.height,
                   voxel_size=0.02, trunc=0.1)
    target = np.array([2.0, 2.0, 0.6])
    for i in range(4):  # static room model from a few views
        T = look_at([0.4 + 0.03 * i, 0.3, 1.3], target)
        d, rgb, _ = render_frame([ROOM], cam, T)
        vol.integrate(_dev(R, vol, d, rgb, cam), T)
    vol.sync()
    boxes = [Prim("box", {"center": np.array([1.3, 1.1, 0.45]), "half": np.array([0.15, 0.15, 0.45]), "yaw": 0.3},
                  (0.9, 0.2, 0.2), (4.0, 4.0, 4.0, 0.0, 0.0, 0.0, 5.0, 0.0), dynamic=True),
             Prim("box", {"center": np.array([1.0, 1.5, 0.3]), "half": np.array([0.25, 0.1, 0.3]), "yaw": 1.1},
                  (0.2, 0.8, 0.2), (3.0, 5.0, 4.0, 0.0, 0.0, 0.0, 5.0, 0.0), dynamic=True)]
    poses = [look_at([0.45, 0.32, 1.31], target), look_at([0.5, 0.25, 1.28], target + np.array([0.1, 0.0, 0.0]))]
    for call in range(2):  # two calls in a row, different frames and poses
        T = poses[call]
        d, rgb, dyn = render_frame([ROOM, boxes[call]], cam, T, noise="quadratic", seed=call)
        fr = _dev(R, vol, d, rgb, cam)
        Td = torch.as_tensor(T, device="cuda").contiguous()
        ref = torch.empty(cam.height, cam.width, dtype=torch.uint8, device="cuda")
        out = torch.full((cam.height, cam.width), 7, dtype=torch.uint8, device="cuda")
        R.rf_compute_mask(vol.h, fr, Td, ref)
        R.rf_compute_mask_noalloc(vol.h, fr, Td, out)
        vol.sync()
        ref_h, out_h = ref.cpu().numpy(), out.cpu().numpy()
        np.testing.assert_array_equal(out_h, ref_h)  # masks are exact: bit-for-bit equality
        assert ref_h[dyn].mean() > 0.5 and ref_h.sum() < ref_h.size  # a real, non-trivial mask
    vol.close()


def test_noalloc_mask_rejects_frames_beyond_the_static_limit(R):
    vol = R.Volume(n_buckets=1 << 10, max_blocks=1000, max_width=1920, max_height=1080, voxel_size=0.02)
    d = torch.zeros(1080, 1920, dtype=torch.uint16, device="cuda")
    rgb = torch.zeros(1080, 1920, 3, dtype=torch.uint8, device="cuda")
    fr = vol.frame(d, rgb, R.Intrinsics(1400.0, 1400.0, 959.5, 539.5))
    T = torch.eye(4, dtype=torch.float64, device="cuda")
    out = torch.empty(1080, 1920, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RFError) as e:
        R.rf_compute_mask_noalloc(vol.h, fr, T, out)
    assert e.value.status == 1 and "static scratch limit" in str(e.value)
    vol.close()


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2, reason="needs two GPUs")
def test_noalloc_mask_refuses_a_current_device_other_than_the_volumes(R):
    torch.cuda.set_device(0)
    vol = R.Volume(n_buckets=1 << 10, max_blocks=1000, max_width=64, max_height=48, voxel_size=0.02)
    d = torch.zeros(48, 64, dtype=torch.uint16, device="cuda:0")
    rgb = torch.zeros(48, 64, 3, dtype=torch.uint8, device="cuda:0")
    fr = vol.frame(d, rgb, R.Intrinsics(50.0, 50.0, 31.5, 23.5))
    T = torch.eye(4, dtype=torch.float64, device="cuda:0")
    out = torch.empty(48, 64, dtype=torch.uint8, device="cuda:0")
    try:
        torch.cuda.set_device(1)
        with pytest.raises(R.RFError) as e:
            R.rf_compute_mask_noalloc(vol.h, fr, T, out)
        assert e.value.status == 1 and "volume's device" in str(e.value)
    finally:
        torch.cuda.set_device(0)
    vol.close()
