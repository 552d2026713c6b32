"""Launch shapes (rf_launch_config) change the work distribution only: the
volume after a sequence and the filled virtual depth are the same for any
grid, and out-of-range shapes are refused."""
import numpy as np
import pytest

from synth import make_sequence

from . import test_gpu_parity as P

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


def test_launch_shapes_do_not_change_results(R):
    seq = make_sequence("tiny", 6)
    cam = seq.camera
    outs = []
    for cfg in ((16, 8, 2, 8, 16), (1, 1, 1, 1, 1), (48, 32, 8, 32, 0)):
        vol = P.gpu_volume(R, cam, 0.02, tune=False)
        vol.set_launch_config(R.rf_launch_config(*cfg))
        got = vol.launch_config()
        assert (got.integrate_ctas_per_sm, got.cull_ctas_per_sm, got.fixup_ctas_per_sm,
                got.raycast_ctas_per_sm, got.batch_group) == cfg
        T = None
        poses = []
        for i in range(len(seq)):
            d, rgb, Tg, _ = seq.frame(i)
            Tn, _ = vol.process(P.dev_frame(R, vol, d, rgb, cam), Tg if T is None else T)
            vol.sync()
            T = Tn.cpu().numpy()
            poses.append(T)
        d, rgb, Tg, _ = seq.frame(3)
        holes = d.copy()
        holes[::3, ::2] = 0
        filled = vol.virtual_depth(P.dev_frame(R, vol, holes, rgb, cam), Tg).cpu().numpy()
        outs.append((np.array(poses), vol.export(), filled))
        with pytest.raises(R.RFError):
            vol.set_launch_config(R.rf_launch_config(0, 8, 2, 8, 0))
        vol.close()
    for poses, snap, filled in outs[1:]:
        np.testing.assert_array_equal(poses, outs[0][0])
        np.testing.assert_array_equal(filled, outs[0][2])
        for k in ("coords", "F", "W", "rgb", "wc"):
            np.testing.assert_array_equal(snap[k], outs[0][1][k])


def test_profiling_times_whole_frames_and_standalone_integration(R):
    """rf_set_profiling: the whole-frame call (a captured graph) and a
    standalone integration (no capture) both record their device times, and
    profiling changes no result."""
    seq = make_sequence("tiny", 6, n_frames=4)
    cam = seq.camera
    plain, prof = P.gpu_volume(R, cam, 0.02, tune=False), P.gpu_volume(R, cam, 0.02, tune=False)
    prof.set_profiling(True)
    T = {id(plain): None, id(prof): None}
    for i in range(3):
        d, rgb, Tg, _ = seq.frame(i)
        for vol in (plain, prof):
            Tn, _ = vol.process(P.dev_frame(R, vol, d, rgb, cam), Tg if T[id(vol)] is None else T[id(vol)])
            vol.sync()
            T[id(vol)] = Tn.cpu().numpy()
        np.testing.assert_array_equal(T[id(plain)], T[id(prof)])
    p = prof.profile()
    assert p.frame_ms > 0 and p.track_ms[0] > 0 and p.integrate_kernel_ms > 0
    d, rgb, Tg, _ = seq.frame(3)
    for vol in (plain, prof):
        vol.integrate(P.dev_frame(R, vol, d, rgb, cam), Tg)
        vol.sync()
    assert prof.profile().integrate_kernel_ms > 0
    a, b = plain.export(), prof.export()
    for k in ("coords", "F", "W", "rgb", "wc"):
        np.testing.assert_array_equal(a[k], b[k])
    plain.close()
    prof.close()
