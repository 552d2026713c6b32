"""The oracle run in lockstep beside frames the CUDA path has served.

For every frame of one stream the oracle (FP64, its own volume) registers
from the same starting pose the GPU started from, computes its mask at its
first-registration pose and registers again without the masked pixels, so
the GPU's pose and mask can be compared with the oracle's; it then integrates
the frame with the GPU's pose and mask, so that the two volumes see the same
updates and stay comparable (the lockstep protocol: free-running volumes
would differ in their last float bits).  A first frame is integrated at its
starting pose without tracking, as the loop does.  For the FP16 storage form
the oracle's SDF values are rounded to the same FP16 grid (F / tau to the
nearest half) after every integration, so that both track against the same
stored values.
"""
from typing import NamedTuple

import numpy as np


class Row(NamedTuple):
    dt: float          # |t_gpu - t_oracle|, metres
    dr: float          # rotation angle of R_gpu R_oracle^T, radians
    mask: float        # fraction of pixels whose mask differs
    converged: bool    # the oracle's last level stopped on its step-size test
    cost_gpu: float    # mean cost E / N of Eq. 4 at the GPU's pose (oracle model, full resolution)
    cost_oracle: float  # the same at the oracle's pose


def check_rows(rows, pose_tol=1e-4, mask_tol=1e-3, cost_rel=1e-2, far=5e-3):
    """Poses within pose_tol of the oracle's where the oracle's registration
    converged (LM stopped on its step-size test): a converged LM pose is
    compared after convergence (the damping path before it may differ).
    Where it ended on its iteration caps instead, both poses stop on the
    cost's noise floor: the GPU's pose must then be as good a solution (mean
    cost within cost_rel of the oracle's) and within `far` of it.  Masks
    within mask_tol of the pixels everywhere."""
    for i, r in enumerate(rows):
        assert r.mask < mask_tol, (i, r)
        if r.converged:
            assert r.dt < pose_tol and r.dr < pose_tol, (i, r)
        else:
            assert r.cost_gpu <= r.cost_oracle * (1.0 + cost_rel) + 1e-12, (i, r)
            assert r.dt < far and r.dr < far, (i, r)


def pose_diff(Ta, Tb):
    dt = float(np.linalg.norm(Ta[:3, 3] - Tb[:3, 3]))
    R = Ta[:3, :3] @ Tb[:3, :3].T
    dr = float(np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)))
    return dt, dr


def _round_fp16(O, orc, tau):
    snap = orc.export()
    obs = snap["W"] > 0
    F = snap["F"].copy()
    F[obs] = (F[obs] / tau).astype(np.float16).astype(np.float64) * tau
    snap["F"] = F
    orc.import_(snap)


def replay(O, frames, cam, T_in, T_out, masks, voxel, tau=0.1, fp16=False):
    """frames: (depth, rgb) per frame; T_in[k], T_out[k], masks[k]: what the
    GPU started from and returned for frame k (masks[k] may be None for a
    first frame).  Returns the oracle volume and a Row per frame."""
    orc = O.OracleVolume(voxel_size=voxel, trunc=tau)
    rows = []
    for k, (d, rgb) in enumerate(frames):
        f = O.FrameData(d, rgb, cam.fx, cam.fy, cam.cx, cam.cy)
        if orc.num_blocks == 0:  # first frame: integration at the starting pose
            orc.integrate(f, T_in[k])
            rows.append(Row(0.0, 0.0, 0.0, True, 0.0, 0.0))
        else:
            T1, _ = orc.track(f, T_in[k])
            mo = orc.compute_mask(f, T1)
            T2, info = orc.track(f, T1, mo)
            dt, dr = pose_diff(np.asarray(T_out[k]), T2)
            mm = float(np.mean(np.asarray(masks[k]) != mo)) if masks[k] is not None else 0.0
            # mean cost of Eq. 4 (full resolution, the oracle's mask) at the GPU's pose and at the oracle's
            _, _, Eg, Ng = orc.eval(f, np.asarray(T_out[k]), 1, mo)
            _, _, Eo, No = orc.eval(f, T2, 1, mo)
            rows.append(Row(dt, dr, mm, bool(info.converged[2]), Eg / max(Ng, 1), Eo / max(No, 1)))
            orc.integrate(f, T_out[k], None if masks[k] is None else np.asarray(masks[k]))
        if fp16:
            _round_fp16(O, orc, tau)
    return orc, rows


def assert_volume_matches(gpu_snap, orc_snap, tau, f_tol):
    """Block sets, SDF weights, colours and colour weights exact; SDF within
    f_tol (metres) on observed voxels."""
    gk = {tuple(c): i for i, c in enumerate(gpu_snap["coords"])}
    ok = {tuple(c): i for i, c in enumerate(orc_snap["coords"])}
    assert set(gk) == set(ok), (len(set(gk) - set(ok)), len(set(ok) - set(gk)))
    order = np.array([gk[tuple(c)] for c in orc_snap["coords"]], dtype=np.int64)
    np.testing.assert_array_equal(gpu_snap["W"][order], orc_snap["W"])
    np.testing.assert_array_equal(gpu_snap["wc"][order], orc_snap["wc"])
    np.testing.assert_array_equal(gpu_snap["rgb"][order], orc_snap["rgb"])
    obs = orc_snap["W"] > 0
    err = np.abs(gpu_snap["F"][order][obs].astype(np.float64) - orc_snap["F"][obs])
    assert err.max() <= f_tol, (float(err.max()), f_tol)
    return float(err.max())
