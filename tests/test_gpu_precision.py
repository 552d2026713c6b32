"""The precision form (compact FP16 storage, RF_STORAGE_FP16) against the FP64
oracle, with the error of each result stated.

Stored values: F as FP16 of F/tau, W and Wc as uint8, colour RGB8, intensity
as round(254 I).  Per-pixel maths and reductions are FP32, the LM solve FP64,
as in the FP32 storage form.

Stated errors (asserted here):
  * allocated blocks, weights W and Wc, colours: bit-exact (no decision reads
    a stored SDF value);
  * TSDF after n updates of a voxel: |F - F_oracle| <= (n + 1)/2 * 2^-12 tau
    (+ 1e-5 tau of FP32 arithmetic).  Each update stores FP16(F/tau), an error
    of at most half a unit in the last place, 2^-12 for |F/tau| < 1; the
    running average scales the carried error by W/(W+1), so by induction the
    error after n updates is at most (n + 1)/2 half-units;
  * dynamic mask: bit-exact on the same stored values (the oracle imports the
    FP16-rounded snapshot);
  * poses on the same stored values: within 1e-4 m and 1e-4 rad of the oracle
    (the intensity quantisation to 1/254 is the only model difference).
A batch in FP16 storage gives exactly the results of its streams alone.
"""
import math

import numpy as np
import pytest

from synth import make_sequence
from synth.scenes import CAM_HD, CAM_QVGA, CAM_TINY, CAM_VGA

from . import test_gpu_parity as P
from ._scenes import ROOM, corner_pose, render_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU = P.TAU
HALF_UNIT = 2.0 ** -12
R_FP32, R_FP16 = 0, 1  # rf_params.storage (RF_STORAGE_FP32, RF_STORAGE_FP16)


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


def fp16_volume(R, cam, voxel, **kw):
    return P.gpu_volume(R, cam, voxel, storage=R.STORAGE_FP16, **kw)


def fp16_snapshot(snap, tau=TAU):
    """The values FP16 storage holds for a float snapshot: float32(float16(F /
    tau)) * tau in float32, observed voxels only."""
    s = dict(snap)
    t = np.float32(tau)
    F = snap["F"].astype(np.float32)
    h = (F / t).astype(np.float16)
    s["F"] = np.where(snap["W"] > 0, h.astype(np.float32) * t, np.float32(0.0)).astype(np.float32)
    return s


def test_fp16_export_import_roundtrip(R):
    seq = make_sequence("tiny", 1)
    cam = seq.camera
    vol = fp16_volume(R, cam, 0.02)
    for i in range(4):
        d, rgb, T, _ = seq.frame(i)
        vol.integrate(P.dev_frame(R, vol, d, rgb, cam), T)
    vol.sync()
    snap = vol.export()
    assert len(snap["coords"]) > 100
    # exported values are representable: rounding them again changes nothing
    np.testing.assert_array_equal(fp16_snapshot(snap)["F"], snap["F"])
    v2 = fp16_volume(R, cam, 0.02)
    v2.import_(snap)
    s2 = v2.export()
    for k in ("coords", "F", "W", "rgb", "wc"):
        np.testing.assert_array_equal(snap[k], s2[k])


def test_fp16_footprint_has_no_weight_array(R):
    p16 = R.params(storage=R.STORAGE_FP16)
    p32 = R.params()
    a = R.rf_volume_footprint(p16, 1 << 12, 1001, 160, 120) - R.rf_volume_footprint(p16, 1 << 12, 1000, 160, 120)
    b = R.rf_volume_footprint(p32, 1 << 12, 1001, 160, 120) - R.rf_volume_footprint(p32, 1 << 12, 1000, 160, 120)
    assert (a, b) == (512 * 8 + 48, 512 * 9 + 48)
    vol = fp16_volume(R, CAM_TINY, 0.02, n_buckets=1 << 12, max_blocks=1000)
    assert vol.stats().device_bytes == R.rf_volume_footprint(vol.params, 1 << 12, 1000, 160, 120)


def test_fp16_integration_error_bound(R, O):
    """Same frames and poses on both sides: exact blocks, weights and colours;
    the SDF within the rounding bound of the number of updates."""
    seq = make_sequence("tiny", 0)
    cam = seq.camera
    vol = fp16_volume(R, cam, 0.02)
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    worst = 0.0
    for i in range(len(seq)):
        d, rgb, T, _ = seq.frame(i)
        vol.integrate(P.dev_frame(R, vol, d, rgb, cam), T)
        vol.sync()
        orc.integrate(P.orc_frame(O, d, rgb, cam), T)
        if i in (0, 3, len(seq) - 1):
            gs, os_ = vol.export(), orc.export()
            gk = {tuple(c): k for k, c in enumerate(gs["coords"])}
            assert set(gk) == {tuple(c) for c in os_["coords"]}
            order = np.array([gk[tuple(c)] for c in os_["coords"]], dtype=np.int64)
            for key in ("W", "wc", "rgb"):
                np.testing.assert_array_equal(gs[key][order], os_[key])
            obs = os_["W"] > 0
            err = np.abs(gs["F"][order].astype(np.float64) - os_["F"])[obs]
            bound = ((os_["W"][obs].astype(np.float64) + 1.0) / 2.0 * HALF_UNIT + 1e-5) * TAU
            assert np.all(err <= bound), float((err - bound).max())
            worst = max(worst, float(err.max() / TAU))
    print(f"FP16 storage: max |F - F_oracle| = {worst:.3e} tau")


@pytest.mark.parametrize("gamma", [0.5, 0.05])
def test_fp16_mask_bit_exact(R, O, gamma):
    snap = fp16_snapshot(P._corner_snapshot(O))
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU, gamma=gamma)
    orc.import_(snap)
    vol = fp16_volume(R, CAM_TINY, 0.02, gamma=gamma)
    vol.import_(snap)
    np.testing.assert_array_equal(vol.export()["F"], snap["F"])
    Tg = corner_pose(2.5)
    d, rgb, _ = render_frame([ROOM, P.BOX], CAM_TINY, Tg, noise="quadratic", seed=5)
    for T in (Tg, O.se3_exp(np.array([0.01, -0.004, 0.006, 0.002, 0.0, -0.003])) @ Tg):
        m_gpu = vol.compute_mask(P.dev_frame(R, vol, d, rgb, CAM_TINY), T)
        vol.sync()
        m_orc = orc.compute_mask(P.orc_frame(O, d, rgb, CAM_TINY), T)
        np.testing.assert_array_equal(m_gpu.cpu().numpy(), m_orc)


def test_fp16_tracking_vs_oracle(R, O):
    snap = fp16_snapshot(P._corner_snapshot(O))
    orc = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    orc.import_(snap)
    vol = fp16_volume(R, CAM_TINY, 0.02)
    vol.import_(snap)
    Tg = corner_pose(2.5)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, Tg)
    fr = P.dev_frame(R, vol, d, rgb, CAM_TINY)
    of = P.orc_frame(O, d, rgb, CAM_TINY)
    rng = np.random.default_rng(7)
    worst = (0.0, 0.0)
    for _ in range(4):
        xi = rng.normal(size=6)
        xi[:3] *= 0.02 / np.linalg.norm(xi[:3])
        xi[3:] *= math.radians(1.0) / np.linalg.norm(xi[3:])
        T0 = O.se3_exp(xi) @ Tg
        Tgpu, _ = vol.track(fr, T0)
        vol.sync()
        Torc, _ = orc.track(of, T0)
        dt, dr = P.pose_diff(Tgpu.cpu().numpy(), Torc)
        worst = (max(worst[0], dt), max(worst[1], dr))
        assert dt < P.POSE_TOL and dr < P.POSE_TOL, (dt, dr)
    print(f"FP16 storage: pose vs oracle {worst[0]:.2e} m, {worst[1]:.2e} rad")


def _batch_vs_single(R, specs, n_frames, n_buckets, max_blocks, O=None, storage=R_FP16):
    """Each stream's poses, masks and final volume from one batch, and from
    rf_process_frame on the stream alone, must be identical; with O, every
    stream's frames must also match the oracle run in lockstep."""
    seqs = [make_sequence(c, sd, n_frames=n_frames, camera=cam) for c, sd, cam, _ in specs]
    outs = {}
    for mode in ("single", "batch"):
        vols = [(fp16_volume if storage == R_FP16 else P.gpu_volume)(R, s.camera, vx, n_buckets=n_buckets,
                                                                      max_blocks=max_blocks)
                for s, (_, _, _, vx) in zip(seqs, specs)]
        batch = R.Batch(vols) if mode == "batch" else None
        T = [None] * len(seqs)
        poses, masks = [], []
        for i in range(n_frames):
            frames, tin, tout, mk = [], [], [], []
            for k, s in enumerate(seqs):
                d, rgb, Tgt, _ = s.frame(i)
                frames.append(P.dev_frame(R, vols[k], d, rgb, s.camera))
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
    if O is not None:
        poses, masks, snaps = outs["batch"]
        for k, (s, (_, _, _, vx)) in enumerate(zip(seqs, specs)):
            rows, ferr = P.check_against_oracle(O, s, [poses[i][k] for i in range(n_frames)],
                                                [masks[i][k] for i in range(n_frames)], snaps[k], vx,
                                                fp16=storage == R_FP16)
            print(f"stream {k} ({s.camera.width}x{s.camera.height}): worst pose vs oracle "
                  f"{max(r.dt for r in rows):.2e} m {max(r.dr for r in rows):.2e} rad, mask mismatch "
                  f"{max(r.mask for r in rows):.2e}, SDF {ferr:.2e} m, converged "
                  f"{sum(r.converged for r in rows[1:])} of {len(rows) - 1}")
    return outs


def test_fp16_batch_is_bit_identical_to_single_streams(R):
    _batch_vs_single(R, [("tiny", 0, None, 0.02), ("dynamic", 1, CAM_QVGA, 0.03)], 4, 1 << 16, 100000)


@pytest.mark.parametrize("storage", ["fp16", "fp32"])
def test_batch_full_size_serving_resolutions(R, O, storage):
    """The serving workload's three resolutions in one batch at full size:
    1280x720 at 2 cm, 640x480 with movers at 1 cm, 320x240 with movers at
    3 cm; three frames each, identical to each stream alone, and every frame
    of every stream against the oracle in lockstep (poses within 1e-4, masks
    to 1e-3, blocks, weights and colours exact, SDF within 1e-4 tau for FP32
    and one FP16 step of F / tau for FP16)."""
    outs = _batch_vs_single(R, [("precision", 0, CAM_HD, 0.02), ("dynamic", 1, CAM_VGA, 0.01),
                                ("dynamic", 2, CAM_QVGA, 0.03)], 3, 1 << 18, 200000, O=O,
                            storage=R_FP16 if storage == "fp16" else R_FP32)
    assert all(len(s["coords"]) > 100 for s in outs["batch"][2])  # ~770, ~7900, ~270 blocks


def test_fp16_and_fp32_volumes_do_not_share_a_batch(R):
    a = P.gpu_volume(R, CAM_TINY, 0.02)
    b = fp16_volume(R, CAM_TINY, 0.02)
    with pytest.raises(R.RFError):
        R.Batch([a, b])


def test_fp16_process_frame_follows_fp32(R):
    """The whole loop free-running on the dynamic 320x240 room: the FP16 form
    stays within 2 mm / 0.1 deg of the FP32 form over 8 frames (stated, the
    two differ by the storage rounding only)."""
    seq = make_sequence("dynamic", 3, n_frames=8, camera=CAM_QVGA)
    cam = seq.camera
    out = {}
    for storage in (R.STORAGE_FP32, R.STORAGE_FP16):
        vol = P.gpu_volume(R, cam, 0.02, n_buckets=1 << 16, max_blocks=100000, storage=storage)
        T = None
        poses = []
        for i in range(len(seq)):
            d, rgb, Tgt, _ = seq.frame(i)
            Tn, _ = vol.process(P.dev_frame(R, vol, d, rgb, cam), Tgt if T is None else T)
            vol.sync()
            T = Tn.cpu().numpy()
            poses.append(T)
        out[storage] = poses
    worst = max(P.pose_diff(a, b)[0] for a, b in zip(out[0], out[1]))
    worst_r = max(P.pose_diff(a, b)[1] for a, b in zip(out[0], out[1]))
    print(f"FP16 vs FP32 storage, free-running: {worst:.2e} m, {worst_r:.2e} rad")
    assert worst < 2e-3 and worst_r < math.radians(0.1)


def test_fp16_precision_form_full_size(R, O):
    """The precision form at its full sizes: 1280x720 (fx = fy = 1050), 0.5 cm
    voxels, tau = 5 cm, 2^22 buckets, FP16 storage.  (1) One frame integrated
    at ground truth on both sides: exact blocks, weights and colours, the SDF
    within one update's rounding bound.  (2) On the oracle's FP16-rounded
    snapshot: the mask of the next frame with a nearer fronto-parallel
    rectangle pasted in (an object the model does not hold), bit-exact and
    non-trivial; and registration from the previous frame's pose and from a
    perturbed one within 1e-4 m and 1e-4 rad of the oracle."""
    tau, voxel = 0.05, 0.005
    seq = make_sequence("precision", 0, n_frames=2)
    cam = seq.camera
    assert (cam.width, cam.height, cam.fx) == (1280, 720, 1050.0)
    d0, rgb0, T0, _ = seq.frame(0)
    d1, rgb1, T1, _ = seq.frame(1)
    orc = O.OracleVolume(voxel_size=voxel, trunc=tau)
    orc.integrate(P.orc_frame(O, d0, rgb0, cam), T0)
    os_ = orc.export()
    vol = fp16_volume(R, cam, voxel, trunc=tau, n_buckets=1 << 22, max_blocks=200000)
    vol.integrate(P.dev_frame(R, vol, d0, rgb0, cam), T0)
    vol.sync()
    gs = vol.export()
    gk = {tuple(c): k for k, c in enumerate(gs["coords"])}
    assert set(gk) == {tuple(c) for c in os_["coords"]} and len(gk) > 10000
    order = np.array([gk[tuple(c)] for c in os_["coords"]], dtype=np.int64)
    for key in ("W", "wc", "rgb"):
        np.testing.assert_array_equal(gs[key][order], os_[key])
    obs = os_["W"] > 0
    err = np.abs(gs["F"][order].astype(np.float64) - os_["F"])[obs]
    assert err.max() <= (HALF_UNIT + 1e-5) * tau, err.max() / tau
    vol.close()

    snap = fp16_snapshot(P.to_f32_snapshot(os_), tau=tau)
    o2 = O.OracleVolume(voxel_size=voxel, trunc=tau)
    o2.import_(snap)
    v2 = fp16_volume(R, cam, voxel, trunc=tau, n_buckets=1 << 22, max_blocks=200000)
    v2.import_(snap)
    d_obj = d1.copy()
    d_obj[240:480, 400:800] = 600  # a fronto-parallel rectangle at 0.6 m, nearer than the room
    m_gpu = v2.compute_mask(P.dev_frame(R, v2, d_obj, rgb1, cam), T1)
    v2.sync()
    m_orc = o2.compute_mask(P.orc_frame(O, d_obj, rgb1, cam), T1)
    np.testing.assert_array_equal(m_gpu.cpu().numpy(), m_orc)
    assert m_orc[240:480, 400:800].all() and 0.1 < m_orc.mean() < 0.11  # the rectangle and its dilation
    fr = P.dev_frame(R, v2, d1, rgb1, cam)
    of = P.orc_frame(O, d1, rgb1, cam)
    # from the previous frame's pose (a 7.7 mm / 0.78 deg step) and from a small perturbation
    for Ts in (T0, O.se3_exp(np.array([0.004, -0.003, 0.002, 0.003, -0.002, 0.004])) @ T1):
        Tgpu, _ = v2.track(fr, Ts)
        v2.sync()
        Torc, _ = o2.track(of, Ts)
        dt, dr = P.pose_diff(Tgpu.cpu().numpy(), Torc)
        assert dt < P.POSE_TOL and dr < P.POSE_TOL, (dt, dr)
    v2.close()
