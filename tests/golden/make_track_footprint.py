"""Writes track_footprint_static.json: the algorithmic bytes of one
registration on the static 640x480 room (its 300-frame trajectory), counted
by the FP64 oracle (the only code this script calls besides the seeded input
generator).

A registration (Sec. III-B: LM over three pixel sub-samplings) must read, at
least once, every pixel's depth and colour (5 B; plus 1 B of mask for the
second registration of Sec. III-C) and, of the model, every distinct voxel its
trilinear lookups touch (8 B each in the FP32 storage form, 4 B in the FP16
form: the word a lookup gathers per corner) and one hash entry (8 B) per
distinct block it probes.  The oracle counts the distinct voxels and blocks
exactly while it runs the whole-frame loop of frames 1..N of the benchmark's
sequence (seed 1000, the first GPU rank's stream); frame 0 is integrated at
its ground-truth pose, as the loop does for a first frame.

    python tests/golden/make_track_footprint.py [n_frames]
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from synth import make_sequence  # noqa: E402

SEED, VOXEL, TAU = 1000, 0.01, 0.1


def main(n_frames: int = 4):
    seq = make_sequence("static", SEED)  # the configuration's 300-frame trajectory
    cam = seq.camera
    vol = O.OracleVolume(voxel_size=VOXEL, trunc=TAU)
    npix = cam.width * cam.height
    d, rgb, T, _ = seq.frame(0)
    vol.integrate(O.FrameData(d, rgb, cam.fx, cam.fy, cam.cx, cam.cy), T)
    rows = []
    for i in range(1, n_frames + 1):
        d, rgb, _, _ = seq.frame(i)
        f = O.FrameData(d, rgb, cam.fx, cam.fy, cam.cx, cam.cy)
        T1, i1, b1, v1 = vol.track_footprint(f, T)
        mask = vol.compute_mask(f, T1)
        T2, i2, b2, v2 = vol.track_footprint(f, T1, mask)
        vol.integrate(f, T2, mask)
        T = T2
        for reg, (nb, nv, inf, mask_bytes) in enumerate(((b1, v1, i1, 0), (b2, v2, i2, npix))):
            rows.append({"frame": i, "registration": reg + 1, "evals": inf.evals, "blocks_probed": nb,
                         "voxels_read": nv, "bytes_fp32": 5 * npix + mask_bytes + 8 * nv + 8 * nb,
                         "bytes_fp16": 5 * npix + mask_bytes + 4 * nv + 8 * nb})
    out = {"what": "distinct model voxels read and blocks probed by one registration (both registrations of "
                   "frames 1..N of the static 640x480 room, seed 1000, voxel 1 cm, tau 0.1 m), counted by the "
                   "FP64 oracle; bytes = 5 B per pixel (+1 B mask for the second) + voxel word per voxel + "
                   "8 B per block",
           "generator": "tests/golden/make_track_footprint.py",
           "rows": rows,
           "mean_bytes_fp32": float(np.mean([r["bytes_fp32"] for r in rows])),
           "mean_bytes_fp16": float(np.mean([r["bytes_fp16"] for r in rows]))}
    with open(os.path.join(HERE, "track_footprint_static.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps({k: out[k] for k in ("mean_bytes_fp32", "mean_bytes_fp16")}))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 4)
