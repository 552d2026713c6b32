"""The serving engine's scheduling on the host, with a stand-in for the CUDA
library (no GPU): admission against the memory budget, slot reuse, eviction
of an idle stream to a host snapshot and its restore, per-stream frame
order, and the lone-frame path.  The stand-in volume records the frames it
integrates; its pose moves by one unit per tracked frame."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1905_02082_gb300.serving as SV  # noqa: E402


class FakeVolume:
    def __init__(self, lib, params, n_buckets, max_blocks, max_width, max_height):
        self.lib = lib
        self.h = self
        self.model = []  # (stream, clip frame) integrated, in order
        self.bytes = lib.rf_volume_footprint(params, n_buckets, max_blocks, max_width, max_height)
        lib.live += self.bytes
        lib.peak = max(lib.peak, lib.live)
        self.closed = False

    def close(self):
        if not self.closed:
            self.lib.live -= self.bytes
            self.closed = True

    def reset(self):
        self.model = []

    def export(self):
        return list(self.model)

    def import_(self, snap):
        self.model = list(snap)


class FakeLib:
    STORAGE_FP32 = 0
    Intrinsics = SV.R.Intrinsics

    def __init__(self):
        self.live = 0
        self.peak = 0
        self.batch_calls = 0
        self.single_calls = 0

    def params(self, **kw):
        return dict(kw)

    def rf_volume_footprint(self, params, n_buckets, max_blocks, w, h):
        return n_buckets * 32 + max_blocks * 4656 + w * h * 30

    def Volume(self, params, n_buckets, max_blocks, max_width, max_height):
        return FakeVolume(self, params, n_buckets, max_blocks, max_width, max_height)

    def make_frame(self, d, c, fx, fy, cx, cy):
        return types.SimpleNamespace(depth=d, rgb=c, height=d.shape[0], width=d.shape[1])

    def idle_frame(self, h, w, fx, fy, cx, cy):
        return types.SimpleNamespace(depth=None, rgb=None, height=h, width=w)

    def _one(self, vol, fr, tin, tout):
        tout.copy_(tin)
        if vol.model:  # tracked: the pose moves; a first frame keeps T_init
            tout[0, 3] += 1.0
        vol.model.append((int(fr.depth[0, 0]), int(fr.depth[0, 1])))

    def rf_process_frame(self, h, fr, tin, tout, mask, info, stream):
        self.single_calls += 1
        self._one(h, fr, tin, tout)

    def Batch(self, vols):
        lib = self

        class _B:
            def process(self, frames, tin, tout, masks, stream):
                lib.batch_calls += 1
                for v, fr, a, b in zip(vols, frames, tin, tout):
                    if fr.depth is None:
                        b.copy_(a)
                    else:
                        lib._one(v, fr, a, b)

            def close(self):
                pass

        return _B()


def _spec(name, sid, arrivals, start=0.0, clip=3):
    frames = []
    for i in range(clip):
        d = torch.zeros(4, 4, dtype=torch.int32)
        d[0, 0], d[0, 1] = sid, i
        frames.append((d, torch.zeros(4, 4, 3, dtype=torch.uint8)))
    return SV.StreamSpec(name=name, width=4, height=4, K=SV.R.Intrinsics(1.0, 1.0, 2.0, 2.0), voxel_size=0.01,
                         frames=frames, order=SV.pingpong(clip, len(arrivals)), arrivals=arrivals,
                         T0=np.eye(4), start=start, n_buckets=1 << 10, max_blocks=1000)


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(SV, "R", lib)
    return lib


@pytest.mark.parametrize("mode", ["batch", "per_stream"])
def test_admission_eviction_restore_and_order(fake, mode):
    # A streams throughout; B pauses in the middle; C arrives while A and B
    # hold the only two slots the budget allows, so the idle B is evicted to a
    # snapshot, C takes its slot, and B comes back when C has finished.
    a = _spec("A", 1, [0.004 * k for k in range(100)])
    b = _spec("B", 2, [0.004 * k for k in range(10)] + [0.35 + 0.004 * k for k in range(10)])
    c = _spec("C", 3, [0.004 * k for k in range(15)], start=0.1)
    budget = 2 * a.footprint()
    eng = SV.ServingEngine(budget, mode=mode, evict_idle_s=0.02, export_final=True, device="cpu")
    res = eng.run([a, b, c], time_limit=30.0)
    assert fake.peak <= budget
    assert eng.stats["slots_created"] == 2  # C and the restored B reuse slots of the same shape
    assert eng.stats["evictions"] >= 1 and eng.stats["restores"] >= 1
    for spec, sid in ((a, 1), (b, 2), (c, 3)):
        mine = sorted((r for r in res if r.stream == spec.name), key=lambda r: r.index)
        assert [r.index for r in mine] == list(range(len(spec.arrivals)))  # every frame, in order
        assert all(r.done >= r.arrival for r in mine)
        # the volume saw exactly this stream's frames, in arrival order
        assert eng.final[spec.name] == [(sid, spec.order[k]) for k in range(len(spec.arrivals))]
        # one unit of motion per tracked frame (the first is integrated at T0)
        assert mine[-1].pose[0, 3] == len(spec.arrivals) - 1
    eng.close()
    assert fake.live == 0


def test_lone_ready_frames_skip_the_batch(fake):
    # frames of two streams that never coincide: every step has one ready frame
    a = _spec("A", 1, [0.040 * k for k in range(10)])
    b = _spec("B", 2, [0.020 + 0.040 * k for k in range(10)])
    eng = SV.ServingEngine(1 << 40, mode="batch", device="cpu")
    eng.run([a, b], time_limit=30.0)
    # (a late wake-up can find both ready once in a while; then they share a batch)
    assert fake.single_calls >= 10 and fake.single_calls + 2 * fake.batch_calls >= 20
    eng.close()


def test_a_stream_larger_than_the_budget_is_refused(fake):
    a = _spec("A", 1, [0.0, 0.001])
    eng = SV.ServingEngine(a.footprint() - 1, device="cpu")
    with pytest.raises(ValueError):
        eng.run([a], time_limit=5.0)
