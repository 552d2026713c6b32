"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars (per the method's exact-decision design):
  * allocated-block set, SDF weights, colours, colour weights, dynamic masks:
    bit-exact;
  * TSDF values: within 1e-4 tau;
  * poses: within 1e-4 m and 1e-4 rad.
Mask and tracking parity run both sides on the same volume snapshot (made by
the oracle, its SDF rounded to float32, imported into both), since
free-running volumes differ in their last float bits.
"""
import math

import numpy as np
import pytest

from synth import make_sequence
from synth.scenes import CAM_QVGA, CAM_TINY, CAM_VGA, Camera, Prim

from ._scenes import ROOM, corner_pose, render_frame, rot_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU = 0.1
POSE_TOL = 1e-4


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


def dev_frame(R, vol, depth, rgb, cam):
    d = torch.from_numpy(depth.astype(np.int32)).cuda().to(torch.uint16).contiguous()
    c = torch.from_numpy(np.ascontiguousarray(rgb)).cuda().contiguous()
    fr = vol.frame(d, c, R.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy))
    fr._keep = (d, c)
    return fr


def orc_frame(O, depth, rgb, cam):
    return O.FrameData(depth, rgb, cam.fx, cam.fy, cam.cx, cam.cy)


def gpu_volume(R, cam, voxel, n_buckets=1 << 14, max_blocks=60000, **kw):
    return R.Volume(n_buckets=n_buckets, max_blocks=max_blocks, max_width=cam.width, max_height=cam.height,
                    voxel_size=voxel, trunc=kw.pop("trunc", TAU), **kw)


def to_f32_snapshot(snap):
    s = dict(snap)
    s["F"] = snap["F"].astype(np.float32)
    return s


def assert_volumes_match(gs, os_, tau=TAU, f_tol=1e-4):
    """Block sets, weights and colours exact; SDF within f_tol * tau."""
    gk = {tuple(c): i for i, c in enumerate(gs["coords"])}
    ok = {tuple(c): i for i, c in enumerate(os_["coords"])}
    assert set(gk) == set(ok), (len(set(gk) - set(ok)), len(set(ok) - set(gk)))
    order = np.array([gk[tuple(c)] for c in os_["coords"]], dtype=np.int64)
    np.testing.assert_array_equal(gs["W"][order], os_["W"])
    np.testing.assert_array_equal(gs["wc"][order], os_["wc"])
    np.testing.assert_array_equal(gs["rgb"][order], os_["rgb"])
    obs = os_["W"] > 0
    err = np.abs(gs["F"][order].astype(np.float64) - os_["F"])[obs]
    assert err.max() <= f_tol * tau, err.max()
    return err.max() if err.size else 0.0


def pose_diff(Ta, Tb):
    return float(np.linalg.norm(Ta[:3, 3] - Tb[:3, 3])), rot_err(Ta[:3, :3], Tb[:3, :3])


# ---------------------------------------------------------------------------
# integration (Sec. III-A, III-D)
# ---------------------------------------------------------------------------

def test_integration_lockstep_tiny_sequence(R, O):
    seq = make_sequence("tiny", 0)
    cam = seq.camera
    vol = gpu_volume(R, cam, 0.02)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    for i in range(len(seq)):
        d, rgb, T, _ = seq.frame(i)
        vol.integrate(dev_frame(R, vol, d, rgb, cam), T)
        vol.sync()
        orc.integrate(orc_frame(O, d, rgb, cam), T)
        if i in (0, 4, len(seq) - 1):
            assert_volumes_match(vol.export(), orc.export())


def test_integration_with_mask_and_ragged_frame(R, O):
    """161x97 frame (ragged against every tile size), odd intrinsics, a random
    mask and invalid pixels."""
    cam = Camera(161, 97, 131.5, 129.0, 80.5, 47.0)
    T = corner_pose(1)
    d, rgb, _ = render_frame([ROOM], cam, T, noise="quadratic", seed=3)
    rng = np.random.default_rng(1)
    d[rng.random(d.shape) < 0.05] = 0
    mask = (rng.random(d.shape) < 0.2).astype(np.uint8)
    vol = gpu_volume(R, cam, 0.02)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    m_dev = torch.from_numpy(mask).cuda()
    for rep in range(2):
        vol.integrate(dev_frame(R, vol, d, rgb, cam), T, mask=m_dev)
        vol.sync()
        orc.integrate(orc_frame(O, d, rgb, cam), T, mask)
    assert_volumes_match(vol.export(), orc.export())


def test_integration_frames_of_changing_size(R, O):
    """One volume sized for 640x480 integrates frames of 161x97, 640x480 and
    320x240 in turn (the frustum search's tile count and its last-CTA ticket
    change from call to call); every result equals the oracle's."""
    cams = (Camera(161, 97, 131.5, 129.0, 80.5, 47.0), CAM_VGA, CAM_QVGA)
    vol = R.Volume(n_buckets=1 << 14, max_blocks=60000, max_width=640, max_height=480, voxel_size=0.02, trunc=TAU)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    for k, cam in enumerate(cams * 2):
        T = corner_pose(k % 3)
        d, rgb, _ = render_frame([ROOM], cam, T, noise="quadratic", seed=10 + k)
        vol.integrate(dev_frame(R, vol, d, rgb, cam), T)
        vol.sync()
        orc.integrate(orc_frame(O, d, rgb, cam), T)
        if k in (0, 2, 5):
            assert_volumes_match(vol.export(), orc.export())
    vol.close()


def test_integration_empty_and_invalid_frames(R, O):
    cam = CAM_TINY
    vol = gpu_volume(R, cam, 0.02)
    zero = np.zeros((cam.height, cam.width), np.uint16)
    rgb = np.zeros((cam.height, cam.width, 3), np.uint8)
    vol.integrate(dev_frame(R, vol, zero, rgb, cam), np.eye(4))
    vol.sync()
    assert vol.stats().n_blocks == 0
    # every pixel beyond d_max (invalid): nothing either
    far = np.full((cam.height, cam.width), 9000, np.uint16)
    vol.integrate(dev_frame(R, vol, far, rgb, cam), np.eye(4))
    vol.sync()
    assert vol.stats().n_blocks == 0


def test_integration_full_size_static_frame(R, O):
    """640x480, 1 cm voxels, two frames of the static room at ground truth:
    exact block set and weights, TSDF within 1e-4 tau."""
    seq = make_sequence("static", 0, n_frames=2)
    cam = seq.camera
    vol = gpu_volume(R, cam, 0.01, n_buckets=1 << 20, max_blocks=200000)
    orc = O.OracleVolume(voxel_size=0.01, trunc=TAU)
    for i in range(2):
        d, rgb, T, _ = seq.frame(i)
        vol.integrate(dev_frame(R, vol, d, rgb, cam), T)
        vol.sync()
        orc.integrate(orc_frame(O, d, rgb, cam), T)
    assert_volumes_match(vol.export(), orc.export())


# ---------------------------------------------------------------------------
# registration (Sec. III-B)
# ---------------------------------------------------------------------------

def _corner_snapshot(O, n=5):
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    for i in range(n):
        T = corner_pose(i)
        d, rgb, _ = render_frame([ROOM], CAM_TINY, T)
        orc.integrate(orc_frame(O, d, rgb, CAM_TINY), T)
    return to_f32_snapshot(orc.export())


def test_tracking_parity_corner_perturbations(R, O):
    snap = _corner_snapshot(O)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    orc.import_(snap)
    vol = gpu_volume(R, CAM_TINY, 0.02)
    vol.import_(snap)
    Tg = corner_pose(2.5)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, Tg)
    fr = dev_frame(R, vol, d, rgb, CAM_TINY)
    of = orc_frame(O, d, rgb, CAM_TINY)
    rng = np.random.default_rng(7)
    for _ in range(4):
        xi = rng.normal(size=6)
        xi[:3] *= 0.02 / np.linalg.norm(xi[:3])
        xi[3:] *= math.radians(1.0) / np.linalg.norm(xi[3:])
        T0 = O.se3_exp(xi) @ Tg
        Tgpu, info = vol.track(fr, T0)
        vol.sync()
        Tgpu = Tgpu.cpu().numpy()
        Torc, oinfo = orc.track(of, T0)
        dt, dr = pose_diff(Tgpu, Torc)
        assert dt < POSE_TOL and dr < POSE_TOL, (dt, dr)
        gi = R.Volume.info_of(info)
        assert gi.final_valid > 0.5 * oinfo.final_valid
        assert np.linalg.norm(Tgpu[:3, 3] - Tg[:3, 3]) < 1e-3  # the perturbation is recovered


def test_tracking_parity_sequence_frame_with_mask(R, O):
    seq = make_sequence("tiny", 2)
    cam = seq.camera
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    for i in range(6):
        d, rgb, T, _ = seq.frame(i)
        orc.integrate(orc_frame(O, d, rgb, cam), T)
    snap = to_f32_snapshot(orc.export())
    o2 = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    o2.import_(snap)
    vol = gpu_volume(R, cam, 0.02)
    vol.import_(snap)
    d, rgb, T7, _ = seq.frame(7)
    _, _, T6, _ = seq.frame(6)
    mask = np.zeros(d.shape, np.uint8)
    mask[30:70, 40:90] = 1
    Tgpu, _ = vol.track(dev_frame(R, vol, d, rgb, cam), T6, mask=torch.from_numpy(mask).cuda())
    vol.sync()
    Torc, _ = o2.track(orc_frame(O, d, rgb, cam), T6, mask)
    dt, dr = pose_diff(Tgpu.cpu().numpy(), Torc)
    assert dt < POSE_TOL and dr < POSE_TOL, (dt, dr)


def test_tracking_empty_volume_keeps_pose(R, O):
    vol = gpu_volume(R, CAM_TINY, 0.02)
    T = corner_pose(0)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, T)
    Tg, info = vol.track(dev_frame(R, vol, d, rgb, CAM_TINY), T)
    vol.sync()
    np.testing.assert_array_equal(Tg.cpu().numpy(), T)
    assert R.Volume.info_of(info).final_valid == 0


# ---------------------------------------------------------------------------
# dynamic mask (Sec. III-C): bit-exact on a shared snapshot
# ---------------------------------------------------------------------------

BOX = Prim("box", {"center": np.array([1.3, 1.1, 0.45]), "half": np.array([0.15, 0.15, 0.45]), "yaw": 0.3},
           (0.9, 0.2, 0.2), (4.0, 4.0, 4.0, 0.0, 0.0, 0.0, 5.0, 0.0), dynamic=True)


@pytest.mark.parametrize("gamma", [0.5, 0.0, 1.0, 0.05])
def test_mask_bit_exact(R, O, gamma):
    snap = _corner_snapshot(O)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU, gamma=gamma)
    orc.import_(snap)
    vol = gpu_volume(R, CAM_TINY, 0.02, gamma=gamma)
    vol.import_(snap)
    Tg = corner_pose(2.5)
    d, rgb, dyn = render_frame([ROOM, BOX], CAM_TINY, Tg, noise="quadratic", seed=5)
    for T in (Tg, O.se3_exp(np.array([0.01, -0.004, 0.006, 0.002, 0.0, -0.003])) @ Tg):
        m_gpu = vol.compute_mask(dev_frame(R, vol, d, rgb, CAM_TINY), T)
        vol.sync()
        m_orc = orc.compute_mask(orc_frame(O, d, rgb, CAM_TINY), T)
        np.testing.assert_array_equal(m_gpu.cpu().numpy(), m_orc)
    if gamma == 1.0:
        assert m_orc.sum() == 0
    if gamma == 0.5:
        assert m_orc[dyn].mean() > 0.8


def test_mask_bit_exact_full_size_dynamic(R, O):
    """640x480 dynamic room: the oracle integrates 3 frames at ground truth,
    both sides compute the mask of frame 3 at its ground-truth pose."""
    seq = make_sequence("dynamic", 0, n_frames=4)
    cam = seq.camera
    orc = O.OracleVolume(voxel_size=0.01, trunc=TAU)
    for i in range(3):
        d, rgb, T, _ = seq.frame(i)
        orc.integrate(orc_frame(O, d, rgb, cam), T)
    snap = to_f32_snapshot(orc.export())
    o2 = O.OracleVolume(voxel_size=0.01, trunc=TAU)
    o2.import_(snap)
    vol = gpu_volume(R, cam, 0.01, n_buckets=1 << 20, max_blocks=200000)
    vol.import_(snap)
    d, rgb, T, static = seq.frame(3)
    m_gpu = vol.compute_mask(dev_frame(R, vol, d, rgb, cam), T)
    vol.sync()
    m_orc = o2.compute_mask(orc_frame(O, d, rgb, cam), T)
    np.testing.assert_array_equal(m_gpu.cpu().numpy(), m_orc)


# ---------------------------------------------------------------------------
# whole frame and determinism
# ---------------------------------------------------------------------------

def test_process_frame_tracks_oracle(R, O):
    """Free-running whole-frame loop on the tiny sequence: each side on its
    own volume (they differ in their last float bits), poses within 1e-4 m
    and 1e-4 rad of the oracle's every frame (measured: a few 1e-6), masks
    matching to 1e-3 of the pixels (measured: identical)."""
    seq = make_sequence("tiny", 3)
    cam = seq.camera
    vol = gpu_volume(R, cam, 0.02)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    Tg_prev = To_prev = None
    m_out = torch.empty(cam.height, cam.width, dtype=torch.uint8, device="cuda")
    for i in range(6):
        d, rgb, Tgt, _ = seq.frame(i)
        Tg, _ = vol.process(dev_frame(R, vol, d, rgb, cam), Tgt if Tg_prev is None else Tg_prev, mask_out=m_out)
        vol.sync()
        Tg = Tg.cpu().numpy()
        To, mo, _ = orc.process_frame(orc_frame(O, d, rgb, cam), Tgt if To_prev is None else To_prev)
        dt, dr = pose_diff(Tg, To)
        print(f"frame {i}: free-running pose difference {dt:.2e} m {dr:.2e} rad, "
              f"mask mismatch {np.mean(m_out.cpu().numpy() != mo):.2e}")
        assert dt < POSE_TOL and dr < POSE_TOL, (i, dt, dr)
        assert np.mean(m_out.cpu().numpy() != mo) < 1e-3
        Tg_prev, To_prev = Tg, To


def test_process_frame_tracks_oracle_full_size(R, O):
    """Free-running whole-frame loop on 5 frames of the 640x480 static room
    (1 cm voxels), each side on its own volume: poses within 1e-4 m and
    1e-4 rad of the oracle's (measured: up to 4e-5 m, 2e-5 rad) and within
    a few millimetres of the ground truth."""
    seq = make_sequence("static", 21, n_frames=5)
    cam = seq.camera
    vol = gpu_volume(R, cam, 0.01, n_buckets=1 << 18, max_blocks=200000)
    orc = O.OracleVolume(voxel_size=0.01, trunc=TAU)
    Tg_prev = To_prev = None
    for i in range(5):
        d, rgb, Tgt, _ = seq.frame(i)
        Tg, _ = vol.process(dev_frame(R, vol, d, rgb, cam), Tgt if Tg_prev is None else Tg_prev)
        vol.sync()
        Tg = Tg.cpu().numpy()
        To, _, _ = orc.process_frame(orc_frame(O, d, rgb, cam), Tgt if To_prev is None else To_prev)
        dt, dr = pose_diff(Tg, To)
        gt, gr = pose_diff(Tg, Tgt)
        print(f"frame {i}: GPU vs oracle {dt:.2e} m {dr:.2e} rad; GPU vs ground truth {gt:.2e} m {gr:.2e} rad")
        assert dt < POSE_TOL and dr < POSE_TOL, (i, dt, dr)
        assert gt < 5e-3, (i, gt)
        Tg_prev, To_prev = Tg, To


def test_process_frame_is_deterministic_and_host_path_agrees(R, O):
    seq = make_sequence("tiny", 4, n_frames=4)
    cam = seq.camera
    K = R.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy)
    outs = []
    for mode in ("device", "device", "host"):
        vol = gpu_volume(R, cam, 0.02)
        T = None
        poses = []
        for i in range(4):
            d, rgb, Tgt, _ = seq.frame(i)
            Tin = Tgt if T is None else T
            if mode == "host":
                T, _ = vol.process_host(d, rgb, K, Tin)
            else:
                Tt, _ = vol.process(dev_frame(R, vol, d, rgb, cam), Tin)
                vol.sync()
                T = Tt.cpu().numpy()
            poses.append(T)
        outs.append((np.array(poses), vol.export()))
        vol.close()
    for k in (1, 2):
        np.testing.assert_array_equal(outs[0][0], outs[k][0])
        for key in ("coords", "F", "W", "rgb", "wc"):
            np.testing.assert_array_equal(outs[0][1][key], outs[k][1][key])


# ---------------------------------------------------------------------------
# mesh, snapshots and error paths
# ---------------------------------------------------------------------------

def test_mesh_matches_oracle(R, O):
    snap = _corner_snapshot(O, n=2)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    orc.import_(snap)
    vol = gpu_volume(R, CAM_TINY, 0.02)
    vol.import_(snap)
    vg, cg = vol.extract_mesh()
    vo, co = orc.extract_mesh()
    assert len(vg) == len(vo) > 100
    vg = vg.cpu().numpy().astype(np.float64)
    cg = cg.cpu().numpy()
    from scipy.spatial import cKDTree
    key_o = vo.reshape(len(vo), 9)
    key_g = vg.reshape(len(vg), 9)
    dist, idx = cKDTree(key_o).query(key_g)
    assert dist.max() < 1e-5
    assert len(np.unique(idx)) == len(idx)  # a one-to-one matching of triangles
    assert np.abs(cg.astype(int) - co[idx].astype(int)).max() <= 1


def test_export_import_roundtrip(R, O):
    snap = _corner_snapshot(O, n=2)
    vol = gpu_volume(R, CAM_TINY, 0.02)
    vol.import_(snap)
    back = vol.export()
    for k in ("coords", "W", "rgb", "wc"):
        np.testing.assert_array_equal(back[k], snap[k])
    np.testing.assert_array_equal(back["F"][snap["W"] > 0], snap["F"][snap["W"] > 0])


def test_pool_and_hash_exhaustion_are_reported(R, O):
    seq = make_sequence("tiny", 0, n_frames=1)
    cam = seq.camera
    d, rgb, T, _ = seq.frame(0)
    vol = gpu_volume(R, cam, 0.02, n_buckets=1 << 10, max_blocks=100)
    vol.integrate(dev_frame(R, vol, d, rgb, cam), T)
    with pytest.raises(R.RFError) as e:
        vol.sync()
    assert e.value.status == 4  # RF_ERR_POOL_FULL
    vol.sync()  # the status word was cleared
    vol2 = gpu_volume(R, cam, 0.02, n_buckets=1, max_blocks=20000)
    vol2.integrate(dev_frame(R, vol2, d, rgb, cam), T)
    with pytest.raises(R.RFError) as e:
        vol2.sync()
    assert e.value.status == 3  # RF_ERR_HASH_FULL


def test_invalid_arguments(R):
    vol = gpu_volume(R, CAM_TINY, 0.02)
    big = torch.zeros(CAM_TINY.height + 1, CAM_TINY.width, dtype=torch.uint16, device="cuda")
    rgb = torch.zeros(CAM_TINY.height + 1, CAM_TINY.width, 3, dtype=torch.uint8, device="cuda")
    fr = vol.frame(big, rgb, R.Intrinsics(130, 130, 80, 60))
    with pytest.raises(R.RFError) as e:
        vol.integrate(fr, np.eye(4))
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# batches of streams (one launch covers several uneven streams)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("batch_group", [0, 2])
def test_batch_is_bit_identical_to_single_streams(R, O, batch_group):
    """Three streams of different resolution, intrinsics and voxel size: the
    batched path gives exactly the poses, masks and volumes of the streams
    processed alone (partial sums over fixed pixel chunks), whether their
    registrations share one launch or run in groups of two; and (one launch)
    every frame of every stream matches the oracle run in lockstep: poses
    within 1e-4 m / 1e-4 rad, masks to 1e-3 of the pixels, final volumes with
    exact blocks, weights and colours and the SDF within 1e-4 tau."""
    from synth.scenes import CAM_QVGA
    specs = [("tiny", 0, None, 0.02), ("dynamic", 1, CAM_QVGA, 0.03), ("static", 2, None, 0.01)]
    seqs = [make_sequence(c, sd, n_frames=4, camera=cam) for c, sd, cam, _ in specs]
    outs = {}
    for mode in ("single", "batch"):
        vols = [gpu_volume(R, s.camera, vx, n_buckets=1 << 18, max_blocks=150000) for s, (_, _, _, vx) in
                zip(seqs, specs)]
        if mode == "batch":
            cfg = vols[0].launch_config()
            cfg.batch_group = batch_group
            vols[0].set_launch_config(cfg)
        batch = R.Batch(vols) if mode == "batch" else None
        T = [None] * len(seqs)
        poses, masks = [], []
        for i in range(4):
            frames, tin, tout, mk = [], [], [], []
            for k, s in enumerate(seqs):
                d, rgb, Tgt, _ = s.frame(i)
                frames.append(dev_frame(R, vols[k], d, rgb, s.camera))
                tin.append(torch.as_tensor(Tgt if T[k] is None else T[k], device="cuda").contiguous())
                tout.append(torch.empty(4, 4, dtype=torch.float64, device="cuda"))
                mk.append(torch.empty(s.camera.height, s.camera.width, dtype=torch.uint8, device="cuda"))
            if batch is not None:
                batch.process(frames, tin, tout, mk)
            else:
                for k in range(len(seqs)):
                    R.rf_process_frame(vols[k].h, frames[k], tin[k], tout[k], mk[k], None)
            for v in vols:
                v.sync()
            T = [t.cpu().numpy() for t in tout]
            poses.append(np.array(T))
            masks.append([m.cpu().numpy() for m in mk])
        outs[mode] = (np.array(poses), masks, [v.export() for v in vols])
        if batch is not None:
            batch.close()
        for v in vols:
            v.close()
    np.testing.assert_array_equal(outs["single"][0], outs["batch"][0])
    for ma, mb in zip(outs["single"][1], outs["batch"][1]):
        for a, b in zip(ma, mb):
            np.testing.assert_array_equal(a, b)
    for sa, sb in zip(outs["single"][2], outs["batch"][2]):
        for key in ("coords", "F", "W", "rgb", "wc"):
            np.testing.assert_array_equal(sa[key], sb[key])
    if batch_group == 0:
        poses, masks, snaps = outs["batch"]
        for k, (s, (_, _, _, vx)) in enumerate(zip(seqs, specs)):
            check_against_oracle(O, s, [poses[i][k] for i in range(4)], [masks[i][k] for i in range(4)],
                                 snaps[k], vx)


def check_against_oracle(O, seq, poses, masks, snap, voxel, fp16=False):
    """The frames of one stream as served (poses, masks, final volume) against
    the oracle in lockstep (tests/_oracle_lockstep.py; poses gated after the
    oracle's convergence, check_rows)."""
    from ._oracle_lockstep import assert_volume_matches, check_rows, replay
    n = len(poses)
    frames = [seq.frame(i)[:2] for i in range(n)]
    T_in = [seq.frame(0)[2]] + [poses[i - 1] for i in range(1, n)]
    orc, rows = replay(O, frames, seq.camera, T_in, poses, [None] + list(masks[1:]), voxel, TAU, fp16)
    check_rows(rows, POSE_TOL)
    f_tol = (2.0 ** -11 + 1e-5) * TAU if fp16 else 1e-4 * TAU
    return rows, assert_volume_matches(snap, orc.export(), TAU, f_tol)


@pytest.mark.gpu
def test_batch_streams_join_sit_out_and_evict(R):
    """Streams that join a running batch (first frame), sit calls out (no
    frame) and are evicted to the host and re-imported give exactly the poses,
    masks and volumes of the same frames processed alone, one stream after the
    other, with rf_process_frame."""
    from synth.scenes import CAM_QVGA
    specs = [("static", 3, None, 0.02), ("dynamic", 4, CAM_QVGA, 0.03), ("tiny", 5, None, 0.02)]
    seqs = [make_sequence(c, sd, n_frames=5, camera=cam) for c, sd, cam, _ in specs]
    # per step: which frame each stream gets (None: sits out); stream 2 is
    # exported after step 1 and imported back before step 4
    plan = [(0, None, 0), (1, 0, 1), (2, 1, None), (3, None, None), (4, 2, 2), (None, 3, 3)]
    evict_after, restore_before = 1, 4

    def frame_of(k, i):
        d, rgb, Tgt, _ = seqs[k].frame(i)
        return d, rgb, Tgt

    # alone
    alone = []
    for k, s in enumerate(seqs):
        v = gpu_volume(R, s.camera, specs[k][3], n_buckets=1 << 18, max_blocks=150000)
        T, poses, masks = None, [], []
        for i in sorted({p[k] for p in plan if p[k] is not None}):
            d, rgb, Tgt = frame_of(k, i)
            fr = dev_frame(R, v, d, rgb, s.camera)
            tin = torch.as_tensor(Tgt if T is None else T, device="cuda").contiguous()
            tout = torch.empty(4, 4, dtype=torch.float64, device="cuda")
            mk = torch.empty(s.camera.height, s.camera.width, dtype=torch.uint8, device="cuda")
            R.rf_process_frame(v.h, fr, tin, tout, mk, None)
            v.sync()
            T = tout.cpu().numpy()
            poses.append(T)
            masks.append(mk.cpu().numpy())
        alone.append((poses, masks, v.export()))
        v.close()

    # mixed
    vols = [gpu_volume(R, s.camera, specs[k][3], n_buckets=1 << 18, max_blocks=150000) for k, s in enumerate(seqs)]
    batch = R.Batch(vols)
    T = [None] * 3
    mixed = [([], []) for _ in seqs]
    saved = None
    for step, p in enumerate(plan):
        if step == restore_before:
            vols[2].import_(saved)
        frames, tin, tout, mk = [], [], [], []
        for k, s in enumerate(seqs):
            cam = s.camera
            if p[k] is None:
                frames.append(R.idle_frame(cam.height, cam.width, cam.fx, cam.fy, cam.cx, cam.cy))
                start = T[k] if T[k] is not None else np.eye(4)
            else:
                d, rgb, Tgt = frame_of(k, p[k])
                frames.append(dev_frame(R, vols[k], d, rgb, cam))
                start = Tgt if T[k] is None else T[k]
            tin.append(torch.as_tensor(start, device="cuda").contiguous())
            tout.append(torch.full((4, 4), float("nan"), dtype=torch.float64, device="cuda"))
            mk.append(torch.full((cam.height, cam.width), 7, dtype=torch.uint8, device="cuda"))
        batch.process(frames, tin, tout, mk)
        for v in vols:
            v.sync()
        for k in range(3):
            out = tout[k].cpu().numpy()
            if p[k] is None:
                np.testing.assert_array_equal(out, tin[k].cpu().numpy())
                assert (mk[k].cpu().numpy() == 7).all(), "a stream that sat out had its mask written"
            else:
                T[k] = out
                mixed[k][0].append(out)
                mixed[k][1].append(mk[k].cpu().numpy())
        if step == evict_after:
            saved = vols[2].export()
            vols[2].reset()
    snaps = [v.export() for v in vols]
    batch.close()
    for v in vols:
        v.close()
    for k in range(3):
        np.testing.assert_array_equal(np.array(alone[k][0]), np.array(mixed[k][0]))
        for a, b in zip(alone[k][1], mixed[k][1]):
            np.testing.assert_array_equal(a, b)
        for key in ("coords", "F", "W", "rgb", "wc"):
            np.testing.assert_array_equal(alone[k][2][key], snaps[k][key])
