"""Continuous-batching serving loop: many camera streams on one GPU.

Every admitted stream owns a slot: a device-resident volume (hash table,
voxel pool, staging) plus its pose, kept on the device between frames.
Frames arrive on each stream's own clock.  Each iteration of the loop runs
ONE rf_batch_process over all slots: streams with an arrived frame process it
(each registration as cooperative launches over groups of streams, the mask
stages as one launch each over all streams, integrations concurrently); the other slots sit the call out, which costs
them nothing but an empty pass and keeps the captured graph the same, so
frames that arrive while a batch is on the GPU simply join the next one.

Admission charges rf_volume_footprint against a device-memory budget.  A
stream that finishes frees its slot, which the next stream with the same
volume shape reuses (rf_volume_reset, no re-allocation, no new graph); slots
of other shapes are destroyed when memory is needed.  When a waiting stream
cannot be placed, the stream that has been idle longest is evicted: its
volume goes to a host snapshot (rf_volume_export) and comes back, into any
slot of its shape, by rf_volume_import when its next frame arrives.  A
stream's results do not depend on its slot, its batch mates or evictions
(registration sums over fixed pixel chunks; snapshots are exact).

Frames are read by the batch's staging kernel directly from page-locked host
memory (the host link of the GPU), so a frame's host-to-device transfer is
part of the batch.

mode="per_stream" serves the same arrivals with one rf_process_frame call per
frame (the plain per-stream path) for comparison.  In batch mode a lone ready
frame also goes through rf_process_frame (single_when_alone): the result is
the same, and the idle slots are not replayed with it.

Latency of a frame = host clock when its batch (or call) has completed minus
its arrival time.  This module is host-side scheduling only: every step of
the per-frame path runs in the CUDA library.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import refusion as R


@dataclass
class StreamSpec:
    """One camera stream.

    frames: clip of (depth uint16 [H,W], rgb uint8 [H,W,3]) page-locked CPU
    tensors; order[k]: clip frame delivered at arrival k; arrivals[k]: its
    arrival time in seconds after `start`.  T0: pose of the first delivered
    frame (the stream's world frame)."""
    name: str
    width: int
    height: int
    K: R.Intrinsics
    voxel_size: float
    frames: Sequence[Tuple[object, object]]
    order: Sequence[int]
    arrivals: Sequence[float]
    T0: np.ndarray
    start: float = 0.0
    trunc: float = 0.1
    n_buckets: int = 1 << 18
    max_blocks: int = 100_000
    storage: int = R.STORAGE_FP32

    def key(self):
        return (self.width, self.height, self.voxel_size, self.trunc, self.n_buckets, self.max_blocks, self.storage)

    def params(self):
        return R.params(voxel_size=self.voxel_size, trunc=self.trunc, storage=self.storage)

    def footprint(self) -> int:
        return R.rf_volume_footprint(self.params(), self.n_buckets, self.max_blocks, self.width, self.height)


@dataclass
class FrameResult:
    stream: str
    index: int      # arrival index within the stream
    frame: int      # clip frame
    arrival: float  # seconds since the run started
    done: float
    pose: np.ndarray
    mask: Optional[np.ndarray] = None
    batch: int = 0  # frames processed in the same batch

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _Slot:
    def __init__(self, vol, key, nbytes, spec: StreamSpec, dev):
        import torch
        self.vol = vol
        self.key = key
        self.bytes = nbytes
        self.width, self.height, self.K = spec.width, spec.height, spec.K
        self.owner: Optional["_Stream"] = None
        self.dirty = False
        self.t_idle = torch.eye(4, dtype=torch.float64, device=dev)
        self.t_idle_out = torch.empty(4, 4, dtype=torch.float64, device=dev)


class _Stream:
    def __init__(self, spec: StreamSpec, dev):
        import torch
        self.spec = spec
        self.next = 0
        self.pose = torch.as_tensor(np.asarray(spec.T0, np.float64), device=dev).contiguous()
        self.out = torch.empty(4, 4, dtype=torch.float64, device=dev)
        self.slot: Optional[_Slot] = None
        self.snapshot = None
        self.last_done = 0.0
        self.final = None

    def arrival(self, k: int) -> float:
        return self.spec.start + self.spec.arrivals[k]

    @property
    def done(self) -> bool:
        return self.next >= len(self.spec.arrivals)


class ServingEngine:
    """Serves StreamSpecs on the current CUDA device (see the module text)."""

    def __init__(self, budget_bytes: int, mode: str = "batch", max_slots: Optional[int] = None,
                 evict_idle_s: float = 0.25, keep_masks: bool = False, export_final: bool = False,
                 single_when_alone: bool = True, device=None):
        import torch
        assert mode in ("batch", "per_stream")
        self.torch = torch
        self.mode = mode
        self.budget = int(budget_bytes)
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.dev.type == "cuda":
            sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
            self.max_slots = min(max_slots or sms, sms)  # a batch holds at most one stream per SM
            self.cuda_stream = torch.cuda.Stream(self.dev)
        else:  # host-only runs (the scheduling logic with a stand-in library)
            self.max_slots = max_slots or 152
            self.cuda_stream = None
        self.evict_idle_s = evict_idle_s
        self.keep_masks = keep_masks
        self.export_final = export_final
        # a lone ready frame goes through rf_process_frame (same result, no
        # idle slots replayed with it)
        self.single_when_alone = single_when_alone
        self.slots: List[_Slot] = []
        self.batch: Optional[R.Batch] = None
        self.used = 0
        self.results: List[FrameResult] = []
        self.batch_ms: List[float] = []  # host time of each batch call, synchronised
        self.stats = {"slots_created": 0, "slots_destroyed": 0, "slot_reuses": 0, "evictions": 0, "restores": 0,
                      "batches": 0, "peak_bytes": 0}

    # -- slots ---------------------------------------------------------------
    def _rebuild(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        if self.slots and self.mode == "batch":
            self.batch = R.Batch([s.vol for s in self.slots])

    def _create(self, spec: StreamSpec, nbytes: int) -> _Slot:
        vol = R.Volume(spec.params(), n_buckets=spec.n_buckets, max_blocks=spec.max_blocks, max_width=spec.width,
                       max_height=spec.height)
        slot = _Slot(vol, spec.key(), nbytes, spec, self.dev)
        self.slots.append(slot)
        self.used += nbytes
        self.stats["slots_created"] += 1
        self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.used)
        return slot

    def _destroy(self, slot: _Slot):
        self.slots.remove(slot)
        slot.vol.close()
        self.used -= slot.bytes
        self.stats["slots_destroyed"] += 1

    def _evict(self, st: _Stream):
        st.snapshot = st.slot.vol.export()
        st.slot.owner = None
        st.slot = None
        self.stats["evictions"] += 1

    def _place(self, st: _Stream, now: float, streams: List[_Stream]) -> bool:
        """Gives `st` a slot; False if memory does not allow it yet."""
        spec = st.spec
        key = spec.key()
        changed = False
        slot = next((s for s in self.slots if s.owner is None and s.key == key), None)
        if slot is None:
            need = spec.footprint()
            if need > self.budget:
                raise ValueError(f"stream {spec.name}: volume of {need} B exceeds the budget of {self.budget} B")
            # free slots of other shapes go first, then idle streams are evicted
            for s in [s for s in self.slots if s.owner is None]:
                if self.used + need <= self.budget and len(self.slots) < self.max_slots:
                    break
                self._destroy(s)
                changed = True
            idle = sorted((o for o in streams if o.slot is not None and o is not st and not o.done
                           and o.arrival(o.next) > now and now - o.last_done >= self.evict_idle_s),
                          key=lambda o: -o.arrival(o.next))
            for o in idle:
                if self.used + need <= self.budget and len(self.slots) < self.max_slots:
                    break
                s = o.slot
                self._evict(o)
                if s.key == key:
                    slot = s
                    break
                self._destroy(s)
                changed = True
            if slot is None:
                if self.used + need > self.budget or len(self.slots) >= self.max_slots:
                    if changed:
                        self._rebuild()
                    return False
                slot = self._create(spec, need)
                changed = True
        else:
            self.stats["slot_reuses"] += 1
        if changed:
            self._rebuild()
        if st.snapshot is not None:
            slot.vol.import_(st.snapshot)
            st.snapshot = None
            self.stats["restores"] += 1
        elif slot.dirty:
            slot.vol.reset()
        slot.dirty = True
        slot.owner = st
        slot.K = spec.K
        st.slot = slot
        return True

    def _release(self, st: _Stream):
        if self.export_final:
            st.final = st.slot.vol.export()
        st.slot.owner = None
        st.slot = None

    def _sync(self):
        if self.cuda_stream is not None:
            self.cuda_stream.synchronize()

    # -- one iteration -----------------------------------------------------
    def _ready(self, st: _Stream, now: float) -> bool:
        return st.slot is not None and not st.done and st.arrival(st.next) <= now

    def _finish(self, st: _Stream, done: float, mask, nbatch: int):
        spec = st.spec
        st.pose, st.out = st.out, st.pose
        k = st.next
        self.results.append(FrameResult(spec.name, k, spec.order[k], st.arrival(k), done, st.pose.cpu().numpy(),
                                        mask.cpu().numpy() if mask is not None else None, nbatch))
        st.next += 1
        st.last_done = done

    def _mask_for(self, spec):
        if not self.keep_masks:
            return None
        return self.torch.empty(spec.height, spec.width, dtype=self.torch.uint8, device=self.dev)

    def _step_batch(self, now: float) -> int:
        if self.single_when_alone:
            alone = [slot.owner for slot in self.slots if slot.owner is not None and self._ready(slot.owner, now)]
            if len(alone) == 1:
                return self._step_per_stream(now, alone)
        frames, tin, tout, masks, ready = [], [], [], [], []
        for slot in self.slots:
            st = slot.owner
            if st is not None and self._ready(st, now):
                spec = st.spec
                d, c = spec.frames[spec.order[st.next]]
                frames.append(R.make_frame(d, c, spec.K.fx, spec.K.fy, spec.K.cx, spec.K.cy))
                tin.append(st.pose)
                tout.append(st.out)
                m = self._mask_for(spec)
                masks.append(m)
                ready.append((st, m))
            else:
                frames.append(R.idle_frame(slot.height, slot.width, slot.K.fx, slot.K.fy, slot.K.cx, slot.K.cy))
                tin.append(slot.t_idle)
                tout.append(slot.t_idle_out)
                masks.append(None)
        if not ready:
            return 0
        t_start = time.perf_counter()
        self.batch.process(frames, tin, tout, masks if self.keep_masks else None, self.cuda_stream)
        self._sync()
        done = time.perf_counter() - self.t0
        self.batch_ms.append(1000.0 * (time.perf_counter() - t_start))
        for st, m in ready:
            self._finish(st, done, m, len(ready))
        self.stats["batches"] += 1
        return len(ready)

    def _step_per_stream(self, now: float, streams: List[_Stream]) -> int:
        ready = sorted((st for st in streams if self._ready(st, now)), key=lambda s: s.arrival(s.next))
        for st in ready:
            spec = st.spec
            d, c = spec.frames[spec.order[st.next]]
            fr = R.make_frame(d, c, spec.K.fx, spec.K.fy, spec.K.cx, spec.K.cy)
            m = self._mask_for(spec)
            R.rf_process_frame(st.slot.vol.h, fr, st.pose, st.out, m, None, self.cuda_stream)
            self._sync()
            self._finish(st, time.perf_counter() - self.t0, m, 1)
        return len(ready)

    # -- the loop ----------------------------------------------------------
    def run(self, specs: List[StreamSpec], time_limit: float = 600.0) -> List[FrameResult]:
        """Serves the streams until every frame is done (garbage collection is
        paused meanwhile, so that its pauses do not enter the latencies)."""
        import gc
        enabled = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            return self._run(specs, time_limit)
        finally:
            if enabled:
                gc.enable()

    def _run(self, specs: List[StreamSpec], time_limit: float) -> List[FrameResult]:
        streams = [_Stream(s, self.dev) for s in specs]
        self.t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - self.t0
            if now > time_limit:
                raise TimeoutError("serving run exceeded its time limit")
            for st in streams:
                if st.slot is not None and st.done:
                    self._release(st)
            live = [st for st in streams if not st.done]
            if not live:
                break
            # admission, in order of the waiting streams' next arrival
            for st in sorted((st for st in live if st.slot is None and st.arrival(st.next) <= now),
                             key=lambda s: s.arrival(s.next)):
                if not self._place(st, now, streams):
                    break
            if self.mode == "batch":
                n = self._step_batch(now) if self.slots else 0
            else:
                n = self._step_per_stream(now, streams)
            if n == 0:
                nxt = min(st.arrival(st.next) for st in live)
                wait = nxt - (time.perf_counter() - self.t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        for st in streams:
            if st.slot is not None:
                self._release(st)
        self.final = {st.spec.name: st.final for st in streams}
        return self.results

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for s in list(self.slots):
            self._destroy(s)


def poisson_arrivals(rng: np.random.Generator, n: int, fps: float) -> List[float]:
    """n arrival times with exponential gaps of mean 1/fps (a Poisson process)."""
    return [float(x) for x in np.cumsum(rng.exponential(1.0 / fps, size=n))]


def pingpong(n_clip: int, n: int) -> List[int]:
    """Clip frames 0,1,..,n_clip-1,n_clip-2,..,1,0,1,.. (the camera moves back
    and forth along the clip's trajectory), n of them."""
    if n_clip == 1:
        return [0] * n
    period = 2 * (n_clip - 1)
    return [k % period if k % period < n_clip else period - k % period for k in range(n)]


def summarize(results: List[FrameResult]) -> Dict:
    if not results:
        return {"frames": 0}
    lat = np.array([r.latency for r in results]) * 1000.0
    t_first = min(r.arrival for r in results)
    t_last = max(r.done for r in results)
    sizes = np.array([r.batch for r in results])
    return {"frames": len(results), "frames_per_s": len(results) / (t_last - t_first),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max()), "mean": float(lat.mean())},
            "frames_per_batch_mean": float(sizes.mean())}
