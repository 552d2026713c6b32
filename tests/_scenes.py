"""Small analytic scenes shared by the tests (inputs only, no method arithmetic)."""
import numpy as np

from synth.scenes import (CAM_TINY, ROOM_MAX, ROOM_MIN, Camera, Prim, _quantise_mm, apply_noise, look_at,
                          render)

ROOM = Prim("room", {"min": ROOM_MIN, "max": ROOM_MAX}, (0.8, 0.7, 0.6), (3.0, 4.0, 5.0, 0.1, 0.2, 0.3, 6.0, 0.5))
SPHERE = Prim("sphere", {"center": np.array([1.2, 1.3, 0.9]), "radius": 0.35}, (0.3, 0.6, 0.9),
              (5.0, 6.0, 7.0, 0.4, 0.5, 0.6, 9.0, 0.2))

# Views into the room corner x = 2, y = 2, z = 0: three orthogonal planes, so
# every pose parameter is observable.
CORNER_TARGET = np.array([2.0, 2.0, 0.6])


def corner_pose(i=0.0):
    return look_at([0.4 + 0.02 * i, 0.3, 1.3], CORNER_TARGET + np.array([0.0, 0.0, 0.004 * i]))


def render_frame(prims, cam: Camera, T, noise="none", seed=0):
    z, rgb, dyn = render(prims, cam, T)
    if noise == "none":
        depth = _quantise_mm(z)
    else:
        depth = apply_noise(z, np.random.default_rng(seed), noise)
    return depth, rgb, dyn


def fronto_plane_frame(cam: Camera, depth_mm: int, rgb=(120, 80, 40)):
    depth = np.full((cam.height, cam.width), depth_mm, np.uint16)
    col = np.empty((cam.height, cam.width, 3), np.uint8)
    col[:] = rgb
    return depth, col


def rot_err(Ra, Rb):
    R = Ra @ Rb.T
    return float(np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)))


__all__ = ["CAM_TINY", "ROOM", "SPHERE", "corner_pose", "render_frame", "fronto_plane_frame", "rot_err",
           "look_at"]
