"""Python binding of librefusion.so (the C ABI in include/refusion.h).

Argument marshalling only: every step of the per-frame path runs in the CUDA
library.  PyTorch supplies device memory and streams.  If the library is not
built, importing the binding fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librefusion.so")

RF_OK = 0
RF_ERR_INVALID_ARG = 1
STATUS_NAMES = {0: "RF_OK", 1: "RF_ERR_INVALID_ARG", 2: "RF_ERR_CUDA", 3: "RF_ERR_HASH_FULL", 4: "RF_ERR_POOL_FULL",
                5: "RF_ERR_NOT_CONVERGED", 6: "RF_ERR_BUFFER_TOO_SMALL", 7: "RF_ERR_OUT_OF_RANGE",
                8: "RF_ERR_CAPACITY"}


STORAGE_FP32, STORAGE_FP16 = 0, 1


class RFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class rf_params(C.Structure):
    _fields_ = [
        ("voxel_size", C.c_double), ("trunc", C.c_double), ("w_c", C.c_double), ("theta", C.c_double),
        ("gamma", C.c_double), ("depth_scale", C.c_double), ("d_min", C.c_double), ("d_max", C.c_double),
        ("z_near", C.c_double), ("w_max", C.c_int), ("lm_iters", C.c_int * 3), ("lm_strides", C.c_int * 3),
        ("lm_lambda0", C.c_double), ("lm_eps_trans", C.c_double), ("lm_eps_rot", C.c_double),
        ("lm_min_valid", C.c_int), ("max_ff_sweeps", C.c_int), ("max_candidates", C.c_int64),
        ("storage", C.c_int),
    ]


class rf_frame(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("depth", C.c_void_p), ("rgb", C.c_void_p)]


class rf_track_info(C.Structure):
    _fields_ = [("evals", C.c_int), ("level_evals", C.c_int * 3), ("converged", C.c_int * 3),
                ("final_cost", C.c_double), ("final_valid", C.c_int64)]


class rf_stats(C.Structure):
    _fields_ = [("n_blocks", C.c_int64), ("max_blocks", C.c_int64), ("n_buckets", C.c_int64), ("frames", C.c_int64),
                ("load_factor", C.c_double), ("device_bytes", C.c_int64)]


class rf_profile(C.Structure):
    _fields_ = [("frame_ms", C.c_float), ("track_ms", C.c_float * 2), ("mask_ms", C.c_float),
                ("integrate_ms", C.c_float), ("integrate_kernel_ms", C.c_float), ("candidates", C.c_int64),
                ("updated_voxels", C.c_int64), ("new_blocks", C.c_int64), ("guard_pixels", C.c_int64)]


class rf_launch_config(C.Structure):
    _fields_ = [("integrate_ctas_per_sm", C.c_int), ("cull_ctas_per_sm", C.c_int), ("fixup_ctas_per_sm", C.c_int),
                ("raycast_ctas_per_sm", C.c_int), ("batch_group", C.c_int)]


# (name, restype, argtypes) of every entry point of refusion.h
_vp, _i64, _int = C.c_void_p, C.c_int64, C.c_int
SIGNATURES = [
    ("rf_default_params", _int, [C.POINTER(rf_params)]),
    ("rf_create_volume", _int, [C.POINTER(rf_params), _i64, _i64, _int, _int, C.POINTER(_vp)]),
    ("rf_volume_footprint", _int, [C.POINTER(rf_params), _i64, _i64, _int, _int, C.POINTER(_i64)]),
    ("rf_destroy_volume", _int, [_vp]),
    ("rf_volume_reset", _int, [_vp]),
    ("rf_track_frame", _int, [_vp, C.POINTER(rf_frame), _vp, _vp, _vp, _vp, _vp]),
    ("rf_compute_mask", _int, [_vp, C.POINTER(rf_frame), _vp, _vp, _vp]),
    ("rf_compute_mask_noalloc", _int, [_vp, C.POINTER(rf_frame), _vp, _vp, _vp]),
    ("rf_integrate_frame", _int, [_vp, C.POINTER(rf_frame), _vp, _vp, _vp]),
    ("rf_virtual_depth", _int, [_vp, C.POINTER(rf_frame), _vp, _int, _vp, _vp]),
    ("rf_process_frame", _int, [_vp, C.POINTER(rf_frame), _vp, _vp, _vp, _vp, _vp]),
    ("rf_process_frame_host", _int, [_vp, _int, _int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("rf_extract_mesh", _int, [_vp, _vp, _vp, _i64, C.POINTER(_i64), _vp]),
    ("rf_volume_export", _int, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, C.POINTER(_i64)]),
    ("rf_volume_import", _int, [_vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    ("rf_volume_stats", _int, [_vp, C.POINTER(rf_stats)]),
    ("rf_get_launch_config", _int, [_vp, C.POINTER(rf_launch_config)]),
    ("rf_set_launch_config", _int, [_vp, C.POINTER(rf_launch_config)]),
    ("rf_set_wait_limits", _int, [_vp, _i64, _int]),
    ("rf_set_registration_tag_base", _int, [_vp, C.c_uint32]),
    ("rf_batch_create", _int, [_vp, _int, C.POINTER(_vp)]),
    ("rf_batch_destroy", _int, [_vp]),
    ("rf_batch_process", _int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("rf_batch_last_error", C.c_char_p, [_vp]),
    ("rf_set_profiling", _int, [_vp, _int]),
    ("rf_get_profile", _int, [_vp, _vp, C.POINTER(rf_profile)]),
    ("rf_sync_status", _int, [_vp, _vp]),
    ("rf_last_error", C.c_char_p, [_vp]),
    ("rf_status_string", C.c_char_p, [_int]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Loads librefusion.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librefusion.so not built at {path}: run paper_1905_02082_gb300.build.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, vol=None):
    if status != RF_OK:
        lib = load()
        msg = lib.rf_last_error(vol)
        raise RFError(status, msg.decode() if msg else "")


def _ptr(t) -> Optional[int]:
    """Raw data pointer of a torch tensor / numpy array / None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return t.ctypes.data
    return int(t)


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------------------
# thin same-name wrappers (pointers and sizes in, status checked)
# ---------------------------------------------------------------------------

def rf_default_params() -> rf_params:
    p = rf_params()
    _check(load().rf_default_params(C.byref(p)))
    return p


def rf_create_volume(params: rf_params, n_buckets: int, max_blocks: int, max_width: int, max_height: int):
    h = C.c_void_p()
    _check(load().rf_create_volume(C.byref(params), n_buckets, max_blocks, max_width, max_height, C.byref(h)))
    return h


def rf_volume_footprint(params: rf_params, n_buckets: int, max_blocks: int, max_width: int, max_height: int) -> int:
    out = C.c_int64()
    lib = load()
    st = lib.rf_volume_footprint(C.byref(params), n_buckets, max_blocks, max_width, max_height, C.byref(out))
    if st != RF_OK:
        raise RFError(st, lib.rf_last_error(None).decode())
    return out.value


def rf_destroy_volume(h):
    _check(load().rf_destroy_volume(h))


def make_frame(depth, rgb, fx, fy, cx, cy) -> rf_frame:
    """rf_frame over tensors depth [H,W] uint16 and rgb [H,W,3] uint8, on the
    device or in page-locked host memory."""
    H, W = int(depth.shape[0]), int(depth.shape[1])
    if depth.dim() != 2 or depth.element_size() != 2 or tuple(rgb.shape) != (H, W, 3) or rgb.element_size() != 1:
        raise ValueError("depth must be [H, W] 16-bit and rgb [H, W, 3] 8-bit")
    if not (depth.is_contiguous() and rgb.is_contiguous()):
        raise ValueError("depth and rgb must be contiguous")
    if not ((depth.is_cuda or depth.is_pinned()) and (rgb.is_cuda or rgb.is_pinned())):
        raise ValueError("depth and rgb must be device or page-locked host tensors")
    return rf_frame(H, W, float(fx), float(fy), float(cx), float(cy), depth.data_ptr(), rgb.data_ptr())


def idle_frame(height, width, fx, fy, cx, cy) -> rf_frame:
    """rf_frame without images: in rf_batch_process the stream sits the call out."""
    return rf_frame(int(height), int(width), float(fx), float(fy), float(cx), float(cy), None, None)


def rf_track_frame(h, frame: rf_frame, T_init, mask, T_out, info=None, stream=None):
    _check(load().rf_track_frame(h, C.byref(frame), _ptr(T_init), _ptr(mask), _ptr(T_out), _ptr(info),
                                 _stream(stream)), h)


def rf_compute_mask(h, frame: rf_frame, T, mask_out, stream=None):
    _check(load().rf_compute_mask(h, C.byref(frame), _ptr(T), _ptr(mask_out), _stream(stream)), h)


def rf_compute_mask_noalloc(h, frame: rf_frame, T, mask_out, stream=None):
    """rf_compute_mask with its scratch in a static device array (no allocation)."""
    _check(load().rf_compute_mask_noalloc(h, C.byref(frame), _ptr(T), _ptr(mask_out), _stream(stream)), h)


def rf_integrate_frame(h, frame: rf_frame, T, mask=None, stream=None):
    _check(load().rf_integrate_frame(h, C.byref(frame), _ptr(T), _ptr(mask), _stream(stream)), h)


def rf_virtual_depth(h, frame: rf_frame, T, far_raw, depth_out, stream=None):
    _check(load().rf_virtual_depth(h, C.byref(frame), _ptr(T), int(far_raw), _ptr(depth_out), _stream(stream)), h)


def rf_process_frame(h, frame: rf_frame, T_init, T_out, mask_out=None, info=None, stream=None):
    _check(load().rf_process_frame(h, C.byref(frame), _ptr(T_init), _ptr(T_out), _ptr(mask_out), _ptr(info),
                                   _stream(stream)), h)


def rf_process_frame_host(h, depth: np.ndarray, rgb: np.ndarray, intr, T_init: np.ndarray, T_out: np.ndarray,
                          mask: Optional[np.ndarray] = None, stream=None):
    intr = np.ascontiguousarray(intr, dtype=np.float64)
    H, W = depth.shape[0], depth.shape[1]
    if depth.dtype != np.uint16 or depth.ndim != 2 or rgb.dtype != np.uint8 or rgb.shape != (H, W, 3):
        raise ValueError("depth must be uint16 [H, W] and rgb uint8 [H, W, 3]")
    if T_init.dtype != np.float64 or T_init.size != 16 or T_out.dtype != np.float64 or T_out.size != 16:
        raise ValueError("poses must be float64 4x4")
    if mask is not None and (mask.dtype != np.uint8 or mask.shape != (H, W)):
        raise ValueError("mask must be uint8 [H, W]")
    if intr.size != 4:
        raise ValueError("intrinsics are fx, fy, cx, cy")
    _check(load().rf_process_frame_host(h, depth.shape[0], depth.shape[1], _ptr(intr), _ptr(depth), _ptr(rgb),
                                        _ptr(T_init), _ptr(T_out), _ptr(mask), _stream(stream)), h)


def rf_sync_status(h, stream=None):
    _check(load().rf_sync_status(h, _stream(stream)), h)


def rf_volume_stats(h) -> rf_stats:
    s = rf_stats()
    _check(load().rf_volume_stats(h, C.byref(s)), h)
    return s


# ---------------------------------------------------------------------------
# convenience object over one volume
# ---------------------------------------------------------------------------

@dataclass
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float


def params(**overrides) -> rf_params:
    """Default parameters (Tab. I plus readings) with keyword overrides."""
    p = rf_default_params()
    for k, v in overrides.items():
        if k in ("lm_iters", "lm_strides"):
            setattr(p, k, (C.c_int * 3)(*v))
        else:
            setattr(p, k, v)
    return p


TUNING_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning")


def tuning_path(device=None) -> str:
    """Launch-shape table of the autotuner for a device (name and SM count)."""
    import torch
    prop = torch.cuda.get_device_properties(device if device is not None else torch.cuda.current_device())
    name = "".join(ch if ch.isalnum() else "_" for ch in prop.name)
    return os.path.join(TUNING_DIR, f"{name}_{prop.multi_processor_count}sm.json")


_tuned = {}


def tuned_launch_config(device=None) -> Optional[rf_launch_config]:
    """The autotuned launch shapes of this device, or None without a table."""
    path = tuning_path(device)
    if path not in _tuned:
        cfg = None
        if os.path.exists(path):
            import json
            d = json.load(open(path))["launch"]
            defaults = {"integrate_ctas_per_sm": 16, "cull_ctas_per_sm": 8, "fixup_ctas_per_sm": 2,
                        "raycast_ctas_per_sm": 8, "batch_group": 16}
            cfg = rf_launch_config(**{k: int(d.get(k, defaults[k])) for k, _ in rf_launch_config._fields_})
        _tuned[path] = cfg
    return _tuned[path]


class Volume:
    """A device-resident voxel-hashed TSDF volume (one camera stream).  The
    autotuned launch shapes of the device are applied when a table exists
    (tune=False keeps the library defaults)."""

    def __init__(self, p: Optional[rf_params] = None, n_buckets: int = 1 << 20, max_blocks: int = 1 << 18,
                 max_width: int = 640, max_height: int = 480, tune: bool = True, **overrides):
        import torch
        self.torch = torch
        self.params = p if p is not None else params(**overrides)
        self.h = rf_create_volume(self.params, n_buckets, max_blocks, max_width, max_height)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        cfg = tuned_launch_config() if tune else None
        if cfg is not None:
            self.set_launch_config(cfg)

    def close(self):
        if getattr(self, "h", None):
            rf_destroy_volume(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers -----------------------------------------------------------
    def _pose(self, T):
        torch = self.torch
        if isinstance(T, torch.Tensor) and T.is_cuda and T.dtype == torch.float64 and T.is_contiguous():
            return T
        return torch.as_tensor(np.asarray(T, dtype=np.float64).reshape(4, 4), device=self.dev).contiguous()

    def frame(self, depth, rgb, K: Intrinsics) -> rf_frame:
        return make_frame(depth, rgb, K.fx, K.fy, K.cx, K.cy)

    # -- calls --------------------------------------------------------------
    def track(self, frame: rf_frame, T_init, mask=None, stream=None):
        torch = self.torch
        Tin = self._pose(T_init)
        Tout = torch.empty(4, 4, dtype=torch.float64, device=self.dev)
        info = torch.zeros(C.sizeof(rf_track_info), dtype=torch.uint8, device=self.dev)
        rf_track_frame(self.h, frame, Tin, mask, Tout, info, stream)
        return Tout, info

    def compute_mask(self, frame: rf_frame, T, out=None, stream=None):
        torch = self.torch
        if out is None:
            out = torch.empty(frame.height, frame.width, dtype=torch.uint8, device=self.dev)
        rf_compute_mask(self.h, frame, self._pose(T), out, stream)
        return out

    def integrate(self, frame: rf_frame, T, mask=None, stream=None):
        rf_integrate_frame(self.h, frame, self._pose(T), mask, stream)

    def virtual_depth(self, frame: rf_frame, T, far_raw: int = 0, out=None, stream=None):
        """Depth of `frame` with its zero pixels filled from this volume (used
        as the temporary model of Sec. III-E's second option)."""
        torch = self.torch
        if out is None:
            out = torch.empty(frame.height, frame.width, dtype=torch.uint16, device=self.dev)
        rf_virtual_depth(self.h, frame, self._pose(T), far_raw, out, stream)
        return out

    def process(self, frame: rf_frame, T_init, mask_out=None, stream=None):
        torch = self.torch
        Tout = torch.empty(4, 4, dtype=torch.float64, device=self.dev)
        info = torch.zeros(C.sizeof(rf_track_info), dtype=torch.uint8, device=self.dev)
        rf_process_frame(self.h, frame, self._pose(T_init), Tout, mask_out, info, stream)
        return Tout, info

    def process_host(self, depth: np.ndarray, rgb: np.ndarray, K: Intrinsics, T_init, want_mask=False,
                     stream=None):
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        Tin = np.ascontiguousarray(T_init, dtype=np.float64)
        Tout = np.zeros((4, 4))
        mask = np.zeros(depth.shape, np.uint8) if want_mask else None
        rf_process_frame_host(self.h, depth, rgb, [K.fx, K.fy, K.cx, K.cy], Tin, Tout, mask, stream)
        return Tout, mask

    def sync(self, stream=None):
        rf_sync_status(self.h, stream)

    def launch_config(self) -> rf_launch_config:
        out = rf_launch_config()
        _check(load().rf_get_launch_config(self.h, C.byref(out)), self.h)
        return out

    def set_launch_config(self, cfg: rf_launch_config):
        _check(load().rf_set_launch_config(self.h, C.byref(cfg)), self.h)

    def set_wait_limits(self, spin_limit: int = 0, extra_arrivals: int = 0):
        """Bound of every grid-wide wait (0: the default, about one second);
        extra_arrivals > 0 makes every wait run out (tests of the error path)."""
        _check(load().rf_set_wait_limits(self.h, int(spin_limit), int(extra_arrivals)), self.h)

    def set_registration_tag_base(self, base: int):
        """Next base of the registration's tag sequence (tests of its restart)."""
        _check(load().rf_set_registration_tag_base(self.h, int(base)), self.h)

    def set_profiling(self, enable: bool):
        _check(load().rf_set_profiling(self.h, 1 if enable else 0), self.h)

    def profile(self, stream=None) -> rf_profile:
        out = rf_profile()
        _check(load().rf_get_profile(self.h, _stream(stream), C.byref(out)), self.h)
        return out

    def stats(self) -> rf_stats:
        return rf_volume_stats(self.h)

    @staticmethod
    def info_of(info_tensor) -> rf_track_info:
        b = info_tensor.cpu().numpy().tobytes()
        return rf_track_info.from_buffer_copy(b)

    def export(self):
        lib = load()
        n = C.c_int64()
        _check(lib.rf_volume_export(self.h, 0, None, None, None, None, None, C.byref(n)), self.h)
        nb = n.value
        snap = dict(coords=np.zeros((nb, 3), np.int32), F=np.zeros((nb, 512), np.float32),
                    W=np.zeros((nb, 512), np.uint8), rgb=np.zeros((nb, 512, 3), np.uint8),
                    wc=np.zeros((nb, 512), np.uint8))
        if nb:
            _check(lib.rf_volume_export(self.h, nb, _ptr(snap["coords"]), _ptr(snap["F"]), _ptr(snap["W"]),
                                        _ptr(snap["rgb"]), _ptr(snap["wc"]), C.byref(n)), self.h)
        return snap

    def import_(self, snap):
        c = np.ascontiguousarray(snap["coords"], dtype=np.int32)
        F = np.ascontiguousarray(snap["F"], dtype=np.float32)
        W = np.ascontiguousarray(snap["W"], dtype=np.uint8)
        rgb = np.ascontiguousarray(snap["rgb"], dtype=np.uint8)
        wc = np.ascontiguousarray(snap["wc"], dtype=np.uint8)
        _check(load().rf_volume_import(self.h, len(c), _ptr(c), _ptr(F), _ptr(W), _ptr(rgb), _ptr(wc)), self.h)

    def reset(self):
        _check(load().rf_volume_reset(self.h), self.h)

    def extract_mesh(self, stream=None):
        torch = self.torch
        lib = load()
        n = C.c_int64()
        _check(lib.rf_extract_mesh(self.h, None, None, 0, C.byref(n), _stream(stream)), self.h)
        nt = n.value
        verts = torch.empty(max(nt, 1), 3, 3, dtype=torch.float32, device=self.dev)
        cols = torch.empty(max(nt, 1), 3, 3, dtype=torch.uint8, device=self.dev)
        if nt:
            _check(lib.rf_extract_mesh(self.h, verts.data_ptr(), cols.data_ptr(), nt, C.byref(n), _stream(stream)),
                   self.h)
        return verts[:nt], cols[:nt]


class Batch:
    """One frame for each of several volumes per call (rf_batch_process)."""

    def __init__(self, volumes):
        import torch
        self.torch = torch
        self.volumes = list(volumes)
        lib = load()
        arr = (C.c_void_p * len(self.volumes))(*[v.h.value for v in self.volumes])
        self._arr = arr
        h = C.c_void_p()
        st = lib.rf_batch_create(arr, len(self.volumes), C.byref(h))
        if st != RF_OK:
            raise RFError(st, lib.rf_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().rf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def process(self, frames, T_inits, T_outs, masks=None, stream=None):
        """frames: list of rf_frame; T_inits/T_outs: device float64 [4,4] tensors;
        masks: optional list of device uint8 [H,W] tensors (or None entries)."""
        n = len(self.volumes)
        if not getattr(self, "h", None) or any(not getattr(v, "h", None) for v in self.volumes):
            raise RFError(RF_ERR_INVALID_ARG, "batch or one of its volumes is closed")
        if not (len(frames) == len(T_inits) == len(T_outs) == n) or (masks is not None and len(masks) != n):
            raise RFError(RF_ERR_INVALID_ARG, f"a batch of {n} volumes takes {n} frames, poses and masks")
        fr = (rf_frame * n)(*frames)
        tin = (C.c_void_p * n)(*[t.data_ptr() for t in T_inits])
        tout = (C.c_void_p * n)(*[t.data_ptr() for t in T_outs])
        m = None
        if masks is not None:
            m = (C.c_void_p * n)(*[(x.data_ptr() if x is not None else None) for x in masks])
        lib = load()
        st = lib.rf_batch_process(self.h, fr, tin, tout, m, _stream(stream))
        if st != RF_OK:
            raise RFError(st, lib.rf_batch_last_error(self.h).decode())
