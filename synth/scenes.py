"""Analytic RGB-D scenes, trajectories and sensor noise.

World frame: z up, metres.  Camera frame: x right, y down, z forward (pinhole,
the camera model of ReFusion Sec. III-B, Eq. 1).  A pose ``T`` is a 4x4 float64
camera-to-world transform.

Every ray is cast in float64 against analytic primitives (room walls, boxes,
vertical cylinders, spheres and moving capsules).  The colour is a smooth
procedural albedo times Lambertian shading.  Depth is the camera-frame z of the
first hit, perturbed by a seeded noise model and quantised to integer
millimetres (uint16, 0 = invalid), like a Kinect-class sensor.

Recipes (all seeded with numpy's PCG64 through ``np.random.default_rng``):

* ``tiny``: 160x120, fx=fy=130, cx=80, cy=60, a 4x4x3 m room with 3 spheres of
  radius 0.2-0.5 m, 10 frames, noise N(0, (1.5 mm * z^2)^2).
* ``static``: 640x480, fx=fy=525, cx=319.5, cy=239.5, the room with about 6
  boxes, 3 cylinders and 4 spheres, Kinect-like axial noise
  0.0012 + 0.0019 (z - 0.4)^2 m and 5 % edge dropout.
* ``dynamic``: the static room plus 2-4 moving boxes/capsules at 0.2-1.0 m/s,
  resampled until they cover 10-40 % of the pixels of the first frames.
* ``precision``: 1280x720, fx=fy=1050, cx=639.5, cy=359.5.
* ``serving``: 320x240 / 640x480 / 1280x720 streams with 0-3 movers.

Edge dropout rule: pixels within 2 px of a depth discontinuity larger than
5 cm (in the noise-free depth) are zeroed i.i.d. with probability
``p = min(1, rate * N_valid / N_edge)``, so that ``rate`` of the valid pixels
drop when the edge band is large enough.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

ROOM_MIN = np.array([-2.0, -2.0, 0.0])
ROOM_MAX = np.array([2.0, 2.0, 3.0])
FPS = 30.0


@dataclass(frozen=True)
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def ray_dirs(self) -> np.ndarray:
        """Camera-frame ray directions with unit z, shape (H*W, 3), row-major."""
        u = np.arange(self.width, dtype=np.float64)
        v = np.arange(self.height, dtype=np.float64)
        uu, vv = np.meshgrid(u, v)
        d = np.empty((self.height * self.width, 3))
        d[:, 0] = ((uu - self.cx) / self.fx).ravel()
        d[:, 1] = ((vv - self.cy) / self.fy).ravel()
        d[:, 2] = 1.0
        return d


CAM_TINY = Camera(160, 120, 130.0, 130.0, 80.0, 60.0)
CAM_VGA = Camera(640, 480, 525.0, 525.0, 319.5, 239.5)
CAM_HD = Camera(1280, 720, 1050.0, 1050.0, 639.5, 359.5)
CAM_QVGA = Camera(320, 240, 262.5, 262.5, 159.5, 119.5)


# ----------------------------------------------------------------------------
# primitives: each returns (t, normal) for rays o + t d, t = camera depth when
# d has unit camera-z.  Misses give t = inf.
# ----------------------------------------------------------------------------

def _room_hit(o, d, bmin, bmax):
    with np.errstate(divide="ignore", invalid="ignore"):
        tb = np.where(d > 0, (bmax - o) / d, np.where(d < 0, (bmin - o) / d, np.inf))
    axis = np.argmin(tb, axis=1)
    t = tb[np.arange(len(d)), axis]
    n = np.zeros_like(d)
    sgn = np.sign(d[np.arange(len(d)), axis])
    n[np.arange(len(d)), axis] = -sgn
    return t, n


def _box_hit(o, d, center, half, yaw):
    c, s = math.cos(yaw), math.sin(yaw)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    ol = (o - center) @ Rz  # world -> box frame (R^T applied as row-vector @ R)
    dl = d @ Rz
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (-half - ol) / dl
        t2 = (half - ol) / dl
    tmin = np.minimum(t1, t2)
    tmax = np.maximum(t1, t2)
    # rays parallel to a slab: inside -> (-inf, inf), outside -> miss
    par = dl == 0
    inside = np.abs(ol) <= half
    tmin = np.where(par, np.where(inside, -np.inf, np.inf), tmin)
    tmax = np.where(par, np.where(inside, np.inf, -np.inf), tmax)
    tn = np.max(tmin, axis=1)
    tf = np.min(tmax, axis=1)
    hit = (tn <= tf) & (tn > 1e-6)
    t = np.where(hit, tn, np.inf)
    axis = np.argmax(tmin, axis=1)
    nl = np.zeros_like(d)
    idx = np.arange(len(d))
    nl[idx, axis] = -np.sign(dl[idx, axis])
    n = nl @ Rz.T
    return t, n


def _sphere_hit(o, d, center, r):
    oc = o - center
    a = np.einsum("ij,ij->i", d, d)
    b = 2.0 * np.einsum("ij,ij->i", oc, d)
    c = np.einsum("ij,ij->i", oc, oc) - r * r
    disc = b * b - 4 * a * c
    sq = np.sqrt(np.maximum(disc, 0.0))
    t = (-b - sq) / (2 * a)
    hit = (disc >= 0) & (t > 1e-6)
    t = np.where(hit, t, np.inf)
    p = o + d * np.where(hit, t, 0.0)[:, None]
    n = (p - center) / r
    return t, n


def _cylinder_hit(o, d, base, radius, height):
    """Vertical solid cylinder: axis along world z from base to base+height."""
    oc = o - base
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = 2 * (oc[:, 0] * d[:, 0] + oc[:, 1] * d[:, 1])
    c = oc[:, 0] ** 2 + oc[:, 1] ** 2 - radius ** 2
    disc = b * b - 4 * a * c
    with np.errstate(divide="ignore", invalid="ignore"):
        ts = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
    zs = oc[:, 2] + ts * d[:, 2]
    side = (disc >= 0) & (a > 0) & (ts > 1e-6) & (zs >= 0) & (zs <= height)
    t = np.where(side, ts, np.inf)
    n = np.zeros_like(d)
    ps = oc + d * np.where(side, ts, 0.0)[:, None]
    n[:, 0] = ps[:, 0] / radius
    n[:, 1] = ps[:, 1] / radius
    # caps
    for zc, nz in ((height, 1.0), (0.0, -1.0)):
        with np.errstate(divide="ignore", invalid="ignore"):
            tc = (zc - oc[:, 2]) / d[:, 2]
        pc = oc + d * np.where(np.isfinite(tc), tc, 0.0)[:, None]
        cap = np.isfinite(tc) & (tc > 1e-6) & (pc[:, 0] ** 2 + pc[:, 1] ** 2 <= radius ** 2) & (tc < t)
        t = np.where(cap, tc, t)
        n[cap] = np.array([0.0, 0.0, nz])
    return t, n


def _capsule_hit(o, d, a_pt, b_pt, r):
    """Capsule = cylinder of radius r around segment a-b plus two end spheres."""
    ab = b_pt - a_pt
    L = np.linalg.norm(ab)
    axis = ab / L
    # cylinder body in a local frame
    oc = o - a_pt
    dpar = d @ axis
    opar = oc @ axis
    dperp = d - np.outer(dpar, axis)
    operp = oc - np.outer(opar, axis)
    A = np.einsum("ij,ij->i", dperp, dperp)
    B = 2 * np.einsum("ij,ij->i", operp, dperp)
    C = np.einsum("ij,ij->i", operp, operp) - r * r
    disc = B * B - 4 * A * C
    with np.errstate(divide="ignore", invalid="ignore"):
        tcy = (-B - np.sqrt(np.maximum(disc, 0))) / (2 * A)
    s = opar + tcy * dpar
    body = (disc >= 0) & (A > 0) & (tcy > 1e-6) & (s >= 0) & (s <= L)
    t = np.where(body, tcy, np.inf)
    pb = oc + d * np.where(body, tcy, 0.0)[:, None]
    n = pb - np.outer(np.clip(pb @ axis, 0, L), axis)
    for cen in (a_pt, b_pt):
        ts, ns = _sphere_hit(o, d, cen, r)
        better = ts < t
        t = np.where(better, ts, t)
        n[better] = ns[better]
    nn = np.linalg.norm(n, axis=1, keepdims=True)
    n = n / np.where(nn > 0, nn, 1.0)
    return t, n


# ----------------------------------------------------------------------------
# scene description
# ----------------------------------------------------------------------------

@dataclass
class Prim:
    kind: str                    # room | box | sphere | cylinder | capsule | plane
    params: dict
    color: Tuple[float, float, float]
    tex: Tuple[float, ...]       # texture frequencies and phases
    dynamic: bool = False
    # for movers: position(t) offset = p0 + v * t, bounced inside the room
    velocity: Optional[np.ndarray] = None


@dataclass
class Scene:
    prims: List[Prim] = field(default_factory=list)
    light: np.ndarray = field(default_factory=lambda: np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8]))

    def at_time(self, t: float) -> List[Prim]:
        """Primitives with movers displaced to time t (seconds)."""
        out = []
        for p in self.prims:
            if p.velocity is None:
                out.append(p)
                continue
            q = dict(p.params)
            off = _bounce(p.params["anchor"], p.velocity, t, p.params["extent"])
            if p.kind == "box":
                q["center"] = p.params["center"] + off
            elif p.kind == "capsule":
                q["a"] = p.params["a"] + off
                q["b"] = p.params["b"] + off
            out.append(Prim(p.kind, q, p.color, p.tex, p.dynamic, None))
        return out


def _bounce(anchor, vel, t, extent):
    """Offset of a mover bouncing between [-extent, extent] around its anchor."""
    off = np.empty(3)
    for i in range(3):
        if extent[i] <= 0 or vel[i] == 0:
            off[i] = 0.0
            continue
        period = 4 * extent[i] / abs(vel[i])
        ph = (t % period) / period
        tri = 4 * ph if ph < 0.25 else (2 - 4 * ph if ph < 0.75 else 4 * ph - 4)
        off[i] = math.copysign(extent[i], vel[i]) * tri
    return off


def _hit(prim: Prim, o, d):
    k, p = prim.kind, prim.params
    if k == "room":
        return _room_hit(o, d, p["min"], p["max"])
    if k == "box":
        return _box_hit(o, d, p["center"], p["half"], p.get("yaw", 0.0))
    if k == "sphere":
        return _sphere_hit(o, d, p["center"], p["radius"])
    if k == "cylinder":
        return _cylinder_hit(o, d, p["base"], p["radius"], p["height"])
    if k == "capsule":
        return _capsule_hit(o, d, p["a"], p["b"], p["radius"])
    if k == "plane":  # infinite plane n.x = off
        n = np.asarray(p["normal"], dtype=np.float64)
        den = d @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (p["offset"] - o @ n) / den
        t = np.where((den != 0) & (t > 1e-6), t, np.inf)
        return t, np.broadcast_to(n, d.shape).copy()
    raise ValueError(k)


def _albedo(prim: Prim, pts):
    f = prim.tex
    s = (np.sin(f[0] * pts[:, 0] + f[3]) * np.sin(f[1] * pts[:, 1] + f[4])
         * np.sin(f[2] * pts[:, 2] + f[5]))
    g = 0.5 + 0.5 * np.sin(f[6] * (pts[:, 0] + pts[:, 1] + pts[:, 2]) + f[7])
    w = 0.55 + 0.3 * s + 0.15 * g
    return np.asarray(prim.color)[None, :] * w[:, None]


def render(scene_prims: List[Prim], cam: Camera, T: np.ndarray, light=None):
    """Cast one ray per pixel centre.

    Returns (depth_m float64 [H,W] with inf for misses, rgb uint8 [H,W,3],
    dynamic bool [H,W] = first hit is a moving primitive).
    """
    if light is None:
        light = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    R, t0 = T[:3, :3], T[:3, 3]
    dc = cam.ray_dirs()
    dw = dc @ R.T
    o = np.broadcast_to(t0, dw.shape)
    best = np.full(len(dw), np.inf)
    nrm = np.zeros_like(dw)
    owner = np.full(len(dw), -1, dtype=np.int64)
    for i, p in enumerate(scene_prims):
        ti, ni = _hit(p, o, dw)
        better = ti < best
        best = np.where(better, ti, best)
        nrm[better] = ni[better]
        owner[better] = i
    pts = o + dw * np.where(np.isfinite(best), best, 0.0)[:, None]
    # two-sided normals facing the camera
    flip = np.einsum("ij,ij->i", nrm, dw) > 0
    nrm[flip] *= -1
    shade = 0.35 + 0.65 * np.clip(nrm @ light, 0.0, 1.0)
    col = np.zeros_like(dw)
    dyn = np.zeros(len(dw), dtype=bool)
    for i, p in enumerate(scene_prims):
        sel = owner == i
        if np.any(sel):
            col[sel] = _albedo(p, pts[sel]) * shade[sel, None]
            dyn[sel] = p.dynamic
    rgb = np.clip(np.rint(col * 255.0), 0, 255).astype(np.uint8)
    H, W = cam.height, cam.width
    return best.reshape(H, W), rgb.reshape(H, W, 3), dyn.reshape(H, W)


# ----------------------------------------------------------------------------
# poses and trajectories
# ----------------------------------------------------------------------------

def pose_from_rpy(pos, yaw, pitch, roll=0.0) -> np.ndarray:
    """Camera-to-world pose.  yaw about world z, pitch down-positive, roll
    about the optical axis.  Camera looks along world +x at yaw = 0."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    fwd = np.array([cy_ * cp, sy_ * cp, -sp])
    right0 = np.array([sy_, -cy_, 0.0])
    down0 = np.cross(fwd, right0)
    cr, sr = math.cos(roll), math.sin(roll)
    right = cr * right0 + sr * down0
    down = -sr * right0 + cr * down0
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2] = right, down, fwd
    T[:3, 3] = pos
    return T


def look_at(pos, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2] = right, down, fwd
    T[:3, 3] = pos
    return T


def _trajectory(rng, n, max_step_m, max_step_deg, center=(0.0, 0.0, 1.4)):
    """Smooth sum-of-sinusoids trajectory, scaled so that every frame-to-frame
    step stays within (max_step_m, max_step_deg)."""
    k = np.arange(n, dtype=np.float64)
    comps = []
    for _ in range(6):  # x, y, z, yaw, pitch, roll
        amp = rng.uniform(0.3, 1.0, size=3)
        frq = rng.uniform(0.01, 0.05, size=3) * 2 * math.pi
        ph = rng.uniform(0, 2 * math.pi, size=3)
        comps.append((amp, frq, ph))

    def raw(kk):
        out = np.zeros((len(kk), 6))
        for j, (amp, frq, ph) in enumerate(comps):
            out[:, j] = sum(a * np.sin(f * kk + p) for a, f, p in zip(amp, frq, ph))
        return out

    r = raw(np.arange(max(n, 2), dtype=np.float64))
    r -= r[0]
    # base motion ranges (metres, radians) before step scaling
    scale = np.array([0.35, 0.35, 0.12, 0.9, 0.15, 0.05])
    r = r / (np.abs(r).max(axis=0) + 1e-12) * scale
    yaw0 = rng.uniform(-math.pi, math.pi)
    steps_t = np.linalg.norm(np.diff(r[:, :3], axis=0), axis=1)
    steps_r = np.degrees(np.abs(np.diff(r[:, 3:], axis=0)).sum(axis=1))
    f = 1.0
    if len(steps_t):
        f = min(1.0, 0.95 * max_step_m / max(steps_t.max(), 1e-12),
                0.95 * max_step_deg / max(steps_r.max(), 1e-12))
    r *= f
    poses = []
    for i in range(n):
        pos = np.asarray(center) + r[i, :3]
        poses.append(pose_from_rpy(pos, yaw0 + r[i, 3], 0.15 + r[i, 4], r[i, 5]))
    return poses


# ----------------------------------------------------------------------------
# noise
# ----------------------------------------------------------------------------

def _quantise_mm(z):
    raw = np.where(np.isfinite(z) & (z > 0), np.rint(z * 1000.0), 0.0)
    return np.clip(raw, 0, 65535).astype(np.uint16)


def _edge_band(z, jump=0.05, radius=2):
    zz = np.where(np.isfinite(z), z, 1e6)
    e = np.zeros(z.shape, dtype=bool)
    dx = np.abs(np.diff(zz, axis=1)) > jump
    dy = np.abs(np.diff(zz, axis=0)) > jump
    e[:, :-1] |= dx
    e[:, 1:] |= dx
    e[:-1, :] |= dy
    e[1:, :] |= dy
    out = e.copy()
    for _ in range(radius):
        g = out.copy()
        g[1:, :] |= out[:-1, :]
        g[:-1, :] |= out[1:, :]
        g[:, 1:] |= out[:, :-1]
        g[:, :-1] |= out[:, 1:]
        out = g
    return out


def apply_noise(z, rng, model: str, dropout: float = 0.0):
    """Noisy uint16 millimetre depth from clean depth z (metres, inf = miss)."""
    zf = np.where(np.isfinite(z), z, 0.0)
    if model == "none":
        zn = zf
    elif model == "quadratic":  # sigma = 1.5 mm * z^2
        zn = zf + rng.standard_normal(z.shape) * (0.0015 * zf * zf)
    elif model == "kinect":  # axial sigma = 0.0012 + 0.0019 (z - 0.4)^2
        zn = zf + rng.standard_normal(z.shape) * (0.0012 + 0.0019 * (zf - 0.4) ** 2)
    else:
        raise ValueError(model)
    zn = np.where(np.isfinite(z), zn, np.inf)
    raw = _quantise_mm(zn)
    if dropout > 0:
        band = _edge_band(z) & (raw > 0)
        nb = int(band.sum())
        if nb:
            p = min(1.0, dropout * int((raw > 0).sum()) / nb)
            drop = band & (rng.random(z.shape) < p)
            raw[drop] = 0
    return raw


# ----------------------------------------------------------------------------
# scene builders
# ----------------------------------------------------------------------------

def _rand_color(rng):
    return tuple(rng.uniform(0.25, 0.95, size=3))


def _rand_tex(rng):
    """Albedo pattern frequencies (rad/m) and phases: wavelengths of about
    9-40 cm, the scale of texture on indoor surfaces (a smoother albedo leaves
    the colour term of the registration almost nothing to hold on to)."""
    return tuple(np.concatenate([rng.uniform(16.0, 72.0, size=3), rng.uniform(0, 2 * math.pi, size=3),
                                 rng.uniform(24.0, 96.0, size=1), rng.uniform(0, 2 * math.pi, size=1)]))


def _ring_point(rng, rmin=1.0, rmax=1.7):
    a = rng.uniform(0, 2 * math.pi)
    r = rng.uniform(rmin, rmax)
    return np.array([r * math.cos(a), r * math.sin(a)])


def build_room(rng, n_boxes=0, n_cyl=0, n_spheres=3, sphere_r=(0.2, 0.5)) -> Scene:
    sc = Scene()
    sc.prims.append(Prim("room", {"min": ROOM_MIN, "max": ROOM_MAX}, _rand_color(rng), _rand_tex(rng)))
    for _ in range(n_boxes):
        xy = _ring_point(rng)
        half = rng.uniform([0.15, 0.15, 0.2], [0.4, 0.4, 0.6])
        sc.prims.append(Prim("box", {"center": np.array([xy[0], xy[1], half[2]]), "half": half,
                                     "yaw": rng.uniform(0, math.pi)}, _rand_color(rng), _rand_tex(rng)))
    for _ in range(n_cyl):
        xy = _ring_point(rng)
        sc.prims.append(Prim("cylinder", {"base": np.array([xy[0], xy[1], 0.0]), "radius": rng.uniform(0.1, 0.3),
                                          "height": rng.uniform(0.5, 2.0)}, _rand_color(rng), _rand_tex(rng)))
    for _ in range(n_spheres):
        xy = _ring_point(rng)
        r = rng.uniform(*sphere_r)
        sc.prims.append(Prim("sphere", {"center": np.array([xy[0], xy[1], rng.uniform(r, 2.5)]), "radius": r},
                             _rand_color(rng), _rand_tex(rng)))
    return sc


def add_movers(sc: Scene, rng, n_movers: int):
    for _ in range(n_movers):
        speed = rng.uniform(0.2, 1.0)
        ang = rng.uniform(0, 2 * math.pi)
        vel = np.array([speed * math.cos(ang), speed * math.sin(ang), 0.0])
        xy = _ring_point(rng, 0.8, 1.4)
        ext = np.array([0.5, 0.5, 0.0])
        if rng.random() < 0.5:
            half = rng.uniform([0.15, 0.15, 0.3], [0.35, 0.35, 0.8])
            c = np.array([xy[0], xy[1], half[2]])
            sc.prims.append(Prim("box", {"center": c, "half": half, "yaw": rng.uniform(0, math.pi),
                                         "anchor": c, "extent": ext}, _rand_color(rng), _rand_tex(rng),
                                 dynamic=True, velocity=vel))
        else:
            r = rng.uniform(0.15, 0.3)
            a = np.array([xy[0], xy[1], r])
            b = np.array([xy[0], xy[1], r + rng.uniform(0.6, 1.4)])
            sc.prims.append(Prim("capsule", {"a": a, "b": b, "radius": r, "anchor": a, "extent": ext},
                                 _rand_color(rng), _rand_tex(rng), dynamic=True, velocity=vel))


# ----------------------------------------------------------------------------
# sequences
# ----------------------------------------------------------------------------

CONFIGS = {
    "tiny": dict(camera=CAM_TINY, n_frames=10, voxel=0.02, trunc=0.1, n_buckets=2 ** 14,
                 noise="quadratic", dropout=0.0, boxes=0, cylinders=0, spheres=3, movers=(0, 0),
                 max_step_m=0.02, max_step_deg=1.0),
    "static": dict(camera=CAM_VGA, n_frames=300, voxel=0.01, trunc=0.1, n_buckets=2 ** 20,
                   noise="kinect", dropout=0.05, boxes=6, cylinders=3, spheres=4, movers=(0, 0),
                   max_step_m=0.02, max_step_deg=1.0),
    "dynamic": dict(camera=CAM_VGA, n_frames=600, voxel=0.01, trunc=0.1, n_buckets=2 ** 20,
                    noise="kinect", dropout=0.05, boxes=6, cylinders=3, spheres=4, movers=(2, 4),
                    max_step_m=0.02, max_step_deg=1.0),
    "precision": dict(camera=CAM_HD, n_frames=900, voxel=0.005, trunc=0.05, n_buckets=2 ** 22,
                      noise="kinect", dropout=0.05, boxes=6, cylinders=3, spheres=4, movers=(0, 0),
                      max_step_m=0.02, max_step_deg=1.0),
}


class Sequence:
    """A seeded RGB-D sequence; frames are rendered on demand (deterministic
    per (seed, index), independent of access order)."""

    def __init__(self, config: str, seed: int = 0, n_frames: Optional[int] = None,
                 camera: Optional[Camera] = None, noise: Optional[str] = None, movers: Optional[int] = None,
                 coverage_scale: int = 1):
        cfg = dict(CONFIGS[config])
        self.config = config
        self.seed = seed
        self.cfg = cfg
        self.camera = camera or cfg["camera"]
        self.n_frames = n_frames or cfg["n_frames"]
        self.noise = noise or cfg["noise"]
        rng = np.random.default_rng([seed, 1905_02082, sum(ord(ch) * 31 ** j for j, ch in enumerate(config)) & 0xFFFFFFFF])
        self.scene = build_room(rng, cfg["boxes"], cfg["cylinders"], cfg["spheres"])
        self.poses = _trajectory(rng, self.n_frames, cfg["max_step_m"], cfg["max_step_deg"])
        lo, hi = cfg["movers"]
        n_mov = movers if movers is not None else (int(rng.integers(lo, hi + 1)) if hi > 0 else 0)
        if n_mov > 0:
            base = list(self.scene.prims)
            for _attempt in range(20):
                self.scene.prims = list(base)
                add_movers(self.scene, rng, n_mov)
                cov = np.mean([self._render(i, coverage_scale)[2].mean() for i in (0, min(self.n_frames - 1, 15))])
                if 0.10 <= cov <= 0.40:
                    break
        self.n_movers = n_mov

    def _render(self, i, scale: int = 1):
        """Ray cast of frame i; scale > 1 renders a 1/scale-resolution image
        (used only to measure the movers' pixel coverage quickly)."""
        prims = self.scene.at_time(i / FPS)
        cam = self.camera
        if scale > 1:
            cam = Camera(cam.width // scale, cam.height // scale, cam.fx / scale, cam.fy / scale,
                         (cam.cx + 0.5) / scale - 0.5, (cam.cy + 0.5) / scale - 0.5)
        return render(prims, cam, self.poses[i], self.scene.light)

    def frame(self, i: int):
        """(depth uint16 [H,W] mm, rgb uint8 [H,W,3], T_gt 4x4, static_mask bool [H,W])."""
        z, rgb, dyn = self._render(i)
        rng = np.random.default_rng([self.seed, i, 77])
        depth = apply_noise(z, rng, self.noise, self.cfg["dropout"])
        return depth, rgb, self.poses[i].copy(), ~dyn

    def __len__(self):
        return self.n_frames


def make_sequence(config: str, seed: int = 0, **kw) -> Sequence:
    return Sequence(config, seed, **kw)
