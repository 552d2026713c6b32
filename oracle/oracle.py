"""ctypes wrapper of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module.  It builds ``refusion_oracle.cpp`` with g++ (no
CUDA, no shared code with the GPU library) and exposes numpy-friendly calls.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "refusion_oracle.cpp")
_HDR = os.path.join(_HERE, "refusion_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "librefusion_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2, -ffp-contract=off keeps FP64 op order)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("voxel_size", C.c_double), ("trunc", C.c_double), ("w_c", C.c_double), ("theta", C.c_double),
        ("gamma", C.c_double), ("depth_scale", C.c_double), ("d_min", C.c_double), ("d_max", C.c_double),
        ("z_near", C.c_double), ("w_max", C.c_int), ("lm_iters", C.c_int * 3), ("lm_strides", C.c_int * 3),
        ("lm_lambda0", C.c_double), ("lm_eps_trans", C.c_double), ("lm_eps_rot", C.c_double),
        ("lm_min_valid", C.c_int),
    ]


class Frame(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("depth", C.c_void_p), ("rgb", C.c_void_p)]


class TrackInfo(C.Structure):
    _fields_ = [("evals", C.c_int), ("level_evals", C.c_int * 3), ("converged", C.c_int * 3),
                ("final_cost", C.c_double), ("final_valid", C.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp, dp, u8p, i32p = C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_void_p
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.POINTER(Params)]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_num_blocks.restype = C.c_int64
        lib.orc_num_blocks.argtypes = [vp]
        lib.orc_num_frames.restype = C.c_int
        lib.orc_num_frames.argtypes = [vp]
        lib.orc_integrate.restype = C.c_int64
        lib.orc_integrate.argtypes = [vp, C.POINTER(Frame), dp, u8p]
        lib.orc_track.argtypes = [vp, C.POINTER(Frame), dp, u8p, dp, C.POINTER(TrackInfo)]
        lib.orc_track_footprint.argtypes = [vp, C.POINTER(Frame), dp, u8p, dp, C.POINTER(TrackInfo),
                                            C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.orc_eval.argtypes = [vp, C.POINTER(Frame), dp, C.c_int, u8p, dp, dp, dp, C.POINTER(C.c_int64)]
        lib.orc_lookup.restype = C.c_int
        lib.orc_lookup.argtypes = [vp, dp, dp, dp, dp, dp, C.POINTER(C.c_int)]
        lib.orc_residual_seeds.argtypes = [vp, C.POINTER(Frame), dp, C.c_void_p, u8p]
        lib.orc_erode3.argtypes = [u8p, C.c_int, C.c_int, u8p]
        lib.orc_dilate3.argtypes = [u8p, C.c_int, C.c_int, u8p]
        lib.orc_floodfill.argtypes = [u8p, C.c_void_p, C.c_int, C.c_int, C.c_int64, u8p]
        lib.orc_compute_mask.argtypes = [vp, C.POINTER(Frame), dp, u8p]
        lib.orc_process_frame.argtypes = [vp, C.POINTER(Frame), dp, dp, u8p, C.POINTER(TrackInfo)]
        lib.orc_virtual_depth.argtypes = [vp, C.POINTER(Frame), dp, C.c_uint16, C.c_int, C.c_int,
                                          C.POINTER(C.c_uint16)]
        lib.orc_se3_exp.argtypes = [dp, dp]
        lib.orc_lm_solve.restype = C.c_int
        lib.orc_lm_solve.argtypes = [dp, dp, C.c_double, dp]
        lib.orc_export.argtypes = [vp, i32p, dp, u8p, u8p, u8p]
        lib.orc_import.restype = C.c_int
        lib.orc_import.argtypes = [vp, C.c_int64, i32p, dp, u8p, u8p, u8p]
        lib.orc_extract_mesh.restype = C.c_int64
        lib.orc_extract_mesh.argtypes = [vp, C.c_void_p, C.c_void_p, C.c_int64]
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


@dataclass
class OracleParams:
    """Defaults: Tab. I (voxel 0.01 m, tau 0.1 m, w_c 0.025, theta 0.007,
    gamma 0.5) plus the readings for what the paper leaves open."""
    voxel_size: float = 0.01
    trunc: float = 0.1
    w_c: float = 0.025
    theta: float = 0.007
    gamma: float = 0.5
    depth_scale: float = 1000.0
    d_min: float = 0.2
    d_max: float = 5.0
    z_near: float = 0.2
    w_max: int = 255
    lm_iters: Tuple[int, int, int] = (10, 5, 5)
    lm_strides: Tuple[int, int, int] = (4, 2, 1)
    lm_lambda0: float = 1e-4
    lm_eps_trans: float = 1e-6
    lm_eps_rot: float = 1e-6
    lm_min_valid: int = 10

    def to_c(self) -> Params:
        p = Params()
        for f in ("voxel_size", "trunc", "w_c", "theta", "gamma", "depth_scale", "d_min", "d_max", "z_near",
                  "w_max", "lm_lambda0", "lm_eps_trans", "lm_eps_rot", "lm_min_valid"):
            setattr(p, f, getattr(self, f))
        p.lm_iters = (C.c_int * 3)(*self.lm_iters)
        p.lm_strides = (C.c_int * 3)(*self.lm_strides)
        return p


class FrameData:
    """Host frame: uint16 depth [H,W] and uint8 rgb [H,W,3] with intrinsics."""

    def __init__(self, depth, rgb, fx, fy, cx, cy):
        self.depth = np.ascontiguousarray(depth, dtype=np.uint16)
        self.rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        assert self.rgb.shape == self.depth.shape + (3,)
        self.c = Frame(self.depth.shape[0], self.depth.shape[1], fx, fy, cx, cy,
                       self.depth.ctypes.data, self.rgb.ctypes.data)

    @property
    def shape(self):
        return self.depth.shape


def _T(T) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(4, 4))


class OracleVolume:
    """An FP64 voxel-hashed TSDF volume on the host."""

    def __init__(self, params: Optional[OracleParams] = None, **kw):
        self.lib = _load()
        self.params = params or OracleParams(**kw)
        self._cp = self.params.to_c()
        self.h = self.lib.orc_create(C.byref(self._cp))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    @property
    def num_blocks(self) -> int:
        return int(self.lib.orc_num_blocks(self.h))

    def integrate(self, f: FrameData, T, mask=None) -> int:
        T = _T(T)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        return int(self.lib.orc_integrate(self.h, C.byref(f.c), _dptr(T), _vptr(m)))

    def track(self, f: FrameData, T_init, mask=None):
        T = _T(T_init)
        out = np.zeros((4, 4))
        info = TrackInfo()
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self.lib.orc_track(self.h, C.byref(f.c), _dptr(T), _vptr(m), _dptr(out), C.byref(info))
        return out, info

    def track_footprint(self, f: FrameData, T_init, mask=None):
        """track(), plus the distinct blocks probed and voxels read by its
        model lookups: (T, info, n_blocks, n_voxels)."""
        T = _T(T_init)
        out = np.zeros((4, 4))
        info = TrackInfo()
        nb, nv = C.c_int64(), C.c_int64()
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self.lib.orc_track_footprint(self.h, C.byref(f.c), _dptr(T), _vptr(m), _dptr(out), C.byref(info),
                                     C.byref(nb), C.byref(nv))
        return out, info, nb.value, nv.value

    def eval(self, f: FrameData, T, stride=1, mask=None):
        T = _T(T)
        H = np.zeros(21)
        g = np.zeros(6)
        E = C.c_double()
        N = C.c_int64()
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self.lib.orc_eval(self.h, C.byref(f.c), _dptr(T), stride, _vptr(m), _dptr(H), _dptr(g), C.byref(E),
                          C.byref(N))
        return unpack_H(H), g, E.value, N.value

    def lookup(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        s = C.c_double()
        I = C.c_double()
        gs = np.zeros(3)
        gI = np.zeros(3)
        cok = C.c_int()
        ok = self.lib.orc_lookup(self.h, _dptr(p), C.byref(s), _dptr(gs), C.byref(I), _dptr(gI), C.byref(cok))
        return bool(ok), s.value, gs, I.value, gI, bool(cok.value)

    def residuals(self, f: FrameData, T):
        T = _T(T)
        r = np.zeros(f.shape, dtype=np.float64)
        seeds = np.zeros(f.shape, dtype=np.uint8)
        self.lib.orc_residual_seeds(self.h, C.byref(f.c), _dptr(T), _vptr(r), _vptr(seeds))
        return r, seeds

    def compute_mask(self, f: FrameData, T):
        T = _T(T)
        m = np.zeros(f.shape, dtype=np.uint8)
        self.lib.orc_compute_mask(self.h, C.byref(f.c), _dptr(T), _vptr(m))
        return m

    def virtual_depth(self, f: FrameData, T, far_raw: Optional[int] = None, rows=None):
        """Sec. III-E, second option: f's depth with its zero pixels filled by
        casting rays through this (temporary) model from pose T.  far_raw
        defaults to d_max in raw units.  rows = (r0, r1) limits the work to
        those rows (others are returned as 0)."""
        T = _T(T)
        if far_raw is None:
            far_raw = int(round(self.params.d_max * self.params.depth_scale))
        H, W = f.shape
        r0, r1 = rows if rows is not None else (0, H)
        out = np.zeros((H, W), dtype=np.uint16)
        self.lib.orc_virtual_depth(self.h, C.byref(f.c), _dptr(T), far_raw, r0, r1,
                                   out.ctypes.data_as(C.POINTER(C.c_uint16)))
        return out

    def process_frame(self, f: FrameData, T_init):
        T = _T(T_init)
        out = np.zeros((4, 4))
        m = np.zeros(f.shape, dtype=np.uint8)
        info = TrackInfo()
        self.lib.orc_process_frame(self.h, C.byref(f.c), _dptr(T), _dptr(out), _vptr(m), C.byref(info))
        return out, m, info

    def export(self):
        """Snapshot dict: coords int32 [n,3], F float64 [n,512], W/wc uint8 [n,512], rgb uint8 [n,512,3]."""
        n = self.num_blocks
        snap = dict(coords=np.zeros((n, 3), np.int32), F=np.zeros((n, 512)), W=np.zeros((n, 512), np.uint8),
                    rgb=np.zeros((n, 512, 3), np.uint8), wc=np.zeros((n, 512), np.uint8))
        self.lib.orc_export(self.h, _vptr(snap["coords"]), _dptr(snap["F"]), _vptr(snap["W"]), _vptr(snap["rgb"]),
                            _vptr(snap["wc"]))
        return snap

    def import_(self, snap):
        n = len(snap["coords"])
        c = np.ascontiguousarray(snap["coords"], dtype=np.int32)
        F = np.ascontiguousarray(snap["F"], dtype=np.float64)
        W = np.ascontiguousarray(snap["W"], dtype=np.uint8)
        rgb = np.ascontiguousarray(snap["rgb"], dtype=np.uint8)
        wc = np.ascontiguousarray(snap["wc"], dtype=np.uint8)
        self.lib.orc_import(self.h, n, _vptr(c), _dptr(F), _vptr(W), _vptr(rgb), _vptr(wc))

    def extract_mesh(self):
        n = int(self.lib.orc_extract_mesh(self.h, None, None, 0))
        verts = np.zeros((n * 3, 3))
        cols = np.zeros((n * 3, 3), np.uint8)
        if n:
            self.lib.orc_extract_mesh(self.h, _vptr(verts), _vptr(cols), n)
        return verts.reshape(n, 3, 3), cols.reshape(n, 3, 3)


def unpack_H(H21) -> np.ndarray:
    Hm = np.zeros((6, 6))
    n = 0
    for i in range(6):
        for j in range(i, 6):
            Hm[i, j] = Hm[j, i] = H21[n]
            n += 1
    return Hm


def pack_H(Hm) -> np.ndarray:
    return np.array([Hm[i, j] for i in range(6) for j in range(i, 6)])


def se3_exp(xi) -> np.ndarray:
    lib = _load()
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    T = np.zeros((4, 4))
    lib.orc_se3_exp(_dptr(xi), _dptr(T))
    return T


def lm_solve(Hm, g, lam):
    lib = _load()
    H21 = pack_H(np.asarray(Hm, dtype=np.float64))
    g = np.ascontiguousarray(g, dtype=np.float64)
    d = np.zeros(6)
    ok = lib.orc_lm_solve(_dptr(H21), _dptr(g), float(lam), _dptr(d))
    return bool(ok), d


def erode3(m):
    lib = _load()
    m = np.ascontiguousarray(m, dtype=np.uint8)
    out = np.zeros_like(m)
    lib.orc_erode3(_vptr(m), m.shape[0], m.shape[1], _vptr(out))
    return out


def dilate3(m):
    lib = _load()
    m = np.ascontiguousarray(m, dtype=np.uint8)
    out = np.zeros_like(m)
    lib.orc_dilate3(_vptr(m), m.shape[0], m.shape[1], _vptr(out))
    return out


def floodfill(MR, depth, theta_ppm: int):
    lib = _load()
    MR = np.ascontiguousarray(MR, dtype=np.uint8)
    depth = np.ascontiguousarray(depth, dtype=np.uint16)
    out = np.zeros_like(MR)
    lib.orc_floodfill(_vptr(MR), _vptr(depth), MR.shape[0], MR.shape[1], int(theta_ppm), _vptr(out))
    return out
