"""The continuous-batching serving loop.

CPU: the arrival and clip helpers.  GPU: every stream's poses, masks and final
volume are bit-identical whether it is served alone (rf_process_frame, one
frame after the other) or in the mix: batched with other streams of other
resolutions and voxel sizes, joining and leaving at different times, sitting
batches out, and evicted to a host snapshot and restored in between; and the
served frames match the FP64 oracle run in lockstep beside them.
"""
import numpy as np
import pytest

from synth import make_sequence
from synth.scenes import CAM_QVGA, CAM_TINY


def test_pingpong_plays_the_clip_back_and_forth():
    from paper_1905_02082_gb300.serving import pingpong
    assert pingpong(4, 10) == [0, 1, 2, 3, 2, 1, 0, 1, 2, 3]
    assert pingpong(1, 3) == [0, 0, 0]
    assert pingpong(2, 5) == [0, 1, 0, 1, 0]


def test_poisson_arrivals_have_the_requested_rate():
    from paper_1905_02082_gb300.serving import poisson_arrivals
    a = poisson_arrivals(np.random.default_rng(3), 20000, 30.0)
    gaps = np.diff([0.0] + a)
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 30.0) < 0.03 / 30.0
    # exponential gaps: standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03


def _streams(R, torch):
    """Four streams: A tiny 2 cm, B QVGA 2 cm with movers, C and D tiny 3 cm.
    C pauses while D runs, so D (same volume shape) takes C's slot by
    eviction; C comes back into D's slot when D has finished."""
    from paper_1905_02082_gb300.serving import StreamSpec, pingpong
    plan = [("A", "tiny", CAM_TINY, 0.02, 11, 0.0, [0.03 * k for k in range(80)]),
            ("B", "dynamic", CAM_QVGA, 0.02, 12, 0.0, [0.035 * k for k in range(70)]),
            ("C", "tiny", CAM_TINY, 0.03, 13, 0.0, [0.03 * k for k in range(4)] + [2.0 + 0.03 * k for k in range(4)]),
            ("D", "tiny", CAM_TINY, 0.03, 14, 0.8, [0.03 * k for k in range(8)])]
    specs = []
    for name, cfg, cam, vx, seed, start, arr in plan:
        seq = make_sequence(cfg, seed, n_frames=4, camera=cam)
        clip = []
        for i in range(4):
            d, rgb, T, _ = seq.frame(i)
            clip.append((torch.from_numpy(np.ascontiguousarray(d, dtype=np.uint16)).pin_memory(),
                         torch.from_numpy(np.ascontiguousarray(rgb)).pin_memory()))
        specs.append(StreamSpec(name=name, width=cam.width, height=cam.height,
                                K=R.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy), voxel_size=vx, frames=clip,
                                order=pingpong(4, len(arr)), arrivals=arr, T0=seq.frame(0)[2], start=start,
                                n_buckets=1 << 14, max_blocks=20_000))
    return specs


def _alone(R, torch, spec):
    vol = R.Volume(spec.params(), n_buckets=spec.n_buckets, max_blocks=spec.max_blocks, max_width=spec.width,
                   max_height=spec.height)
    T = torch.as_tensor(np.asarray(spec.T0, np.float64), device="cuda").contiguous()
    Tn = torch.empty_like(T)
    poses, masks = [], []
    for k in range(len(spec.arrivals)):
        d, c = spec.frames[spec.order[k]]
        fr = R.make_frame(d.cuda(), c.cuda(), spec.K.fx, spec.K.fy, spec.K.cx, spec.K.cy)
        m = torch.empty(spec.height, spec.width, dtype=torch.uint8, device="cuda")
        R.rf_process_frame(vol.h, fr, T, Tn, m, None)
        vol.sync()
        T, Tn = Tn, T
        poses.append(T.cpu().numpy())
        masks.append(m.cpu().numpy())
    snap = vol.export()
    vol.close()
    return poses, masks, snap


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["batch", "per_stream"])
def test_serving_results_are_the_same_alone_and_in_the_mix(mode):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02082_gb300 import build as B
    B.build()
    import paper_1905_02082_gb300.refusion as R
    from paper_1905_02082_gb300.serving import ServingEngine, summarize

    specs = _streams(R, torch)
    budget = sum(s.footprint() for s in specs[:3])  # room for three volumes
    eng = ServingEngine(budget, mode=mode, evict_idle_s=0.1, keep_masks=True, export_final=True)
    res = eng.run(specs, time_limit=120.0)
    eng.close()
    assert len(res) == sum(len(s.arrivals) for s in specs)
    assert eng.stats["evictions"] >= 1 and eng.stats["restores"] >= 1, eng.stats
    assert eng.stats["peak_bytes"] <= budget
    summ = summarize(res)
    assert summ["latency_ms"]["p99"] >= summ["latency_ms"]["p50"] > 0
    for spec in specs:
        poses, masks, snap = _alone(R, torch, spec)
        mine = sorted((r for r in res if r.stream == spec.name), key=lambda r: r.index)
        assert [r.index for r in mine] == list(range(len(spec.arrivals)))
        for r, T, m in zip(mine, poses, masks):
            np.testing.assert_array_equal(r.pose, T, err_msg=f"{spec.name} frame {r.index}")
            np.testing.assert_array_equal(r.mask, m, err_msg=f"{spec.name} frame {r.index}")
        fin = eng.final[spec.name]
        for key in ("coords", "F", "W", "rgb", "wc"):
            np.testing.assert_array_equal(fin[key], snap[key], err_msg=f"{spec.name} {key}")
    if mode == "batch":
        _check_served_against_oracle(specs, res, eng.final)


def _check_served_against_oracle(specs, res, final):
    """The served frames against the FP64 oracle in lockstep (each frame
    registered from the pose the GPU started from, then integrated with the
    GPU's pose and mask): poses within 1e-4 m and 1e-4 rad where the oracle's
    registration converged (check_rows), masks to 1e-3 of the pixels; for
    the two streams that share a slot by eviction and restore
    (C and D) every frame and the final volume (blocks, weights, colours
    exact, SDF within 1e-4 tau); for A and B their first 10 frames."""
    from oracle import oracle as O
    from synth.scenes import Camera

    from ._oracle_lockstep import assert_volume_matches, check_rows, replay
    for spec in specs:
        mine = sorted((r for r in res if r.stream == spec.name), key=lambda r: r.index)
        n = len(mine) if spec.name in ("C", "D") else 10
        cam = Camera(spec.width, spec.height, spec.K.fx, spec.K.fy, spec.K.cx, spec.K.cy)
        frames = [tuple(t.numpy() for t in spec.frames[spec.order[k]]) for k in range(n)]
        T_in = [np.asarray(spec.T0, np.float64)] + [mine[k - 1].pose for k in range(1, n)]
        orc, rows = replay(O, frames, cam, T_in, [r.pose for r in mine[:n]], [None] + [r.mask for r in mine[1:n]],
                           spec.voxel_size, spec.trunc)
        print(spec.name, [(round(r.dt, 7), r.converged) for r in rows])
        check_rows(rows)
        if spec.name in ("C", "D"):
            assert_volume_matches(final[spec.name], orc.export(), spec.trunc, 1e-4 * spec.trunc)
