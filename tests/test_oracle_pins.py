"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: closed
forms of analytic scenes, library routines (scipy expm, numpy solve, scipy
morphology), brute force on tiny inputs, finite differences and invariants.
"""
import json
import math
import os
from collections import deque

import numpy as np
import pytest
import scipy.linalg
import scipy.ndimage as ndi

from synth.scenes import CAM_TINY, Camera, Prim, look_at

from ._scenes import ROOM, SPHERE, corner_pose, fronto_plane_frame, render_frame, rot_err

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers (inputs only)
# ---------------------------------------------------------------------------

def _frame(O, depth, rgb, cam):
    return O.FrameData(depth, rgb, cam.fx, cam.fy, cam.cx, cam.cy)


def _corner_volume(O, voxel=0.02, n=5, **kw):
    vol = O.OracleVolume(voxel_size=voxel, trunc=0.1, **kw)
    for i in range(n):
        T = corner_pose(i)
        d, rgb, _ = render_frame([ROOM], CAM_TINY, T)
        vol.integrate(_frame(O, d, rgb, CAM_TINY), T)
    return vol


def _hat(xi):
    r, p = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -p[2], p[1]], [p[2], 0, -p[0]], [-p[1], p[0], 0]]
    M[:3, 3] = r
    return M


def _snapshot_from_field(coords, field_fn, voxel, colour_fn=None):
    """Volume snapshot whose voxel k (world v k) carries field_fn(world pos)."""
    coords = np.asarray(coords, np.int32)
    n = len(coords)
    lz, ly, lx = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    local = np.stack([lx.ravel(), ly.ravel(), lz.ravel()], axis=1)  # index x + 8y + 64z
    k = coords[:, None, :].astype(np.int64) * 8 + local[None, :, :]
    pos = k * voxel
    F = field_fn(pos)
    snap = dict(coords=coords, F=F, W=np.ones((n, 512), np.uint8), rgb=np.zeros((n, 512, 3), np.uint8),
                wc=np.zeros((n, 512), np.uint8))
    if colour_fn is not None:
        c = colour_fn(k)
        snap["rgb"][:] = c[..., None].astype(np.uint8)
        snap["wc"][:] = 1
    return snap


def _blocks_covering(points, voxel, pad=1):
    b = np.floor(points / (8 * voxel)).astype(np.int64)
    lo, hi = b.min(axis=0) - pad, b.max(axis=0) + pad
    zz, yy, xx = np.meshgrid(*[np.arange(lo[i], hi[i] + 1) for i in (2, 1, 0)], indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def _backproject(depth, cam, T, stride=1, depth_scale=1000.0):
    vs, us = np.mgrid[0:cam.height:stride, 0:cam.width:stride]
    D = depth[vs, us].astype(np.float64) / depth_scale
    x = (us - cam.cx) / cam.fx * D
    y = (vs - cam.cy) / cam.fy * D
    pc = np.stack([x, y, D], axis=-1).reshape(-1, 3)
    valid = (depth[vs, us] > 0).ravel()
    return pc @ T[:3, :3].T + T[:3, 3], valid, (vs.ravel(), us.ravel())


# ---------------------------------------------------------------------------
# Tab. I defaults (golden fixture with citation)
# ---------------------------------------------------------------------------

def test_default_parameters_match_table_1(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "tab1_parameters.json")))
    p = oracle_mod.OracleParams()
    for k in ("voxel_size", "trunc", "w_c", "theta", "gamma"):
        assert getattr(p, k) == g[k], k


# ---------------------------------------------------------------------------
# se(3) exponential and the LM step (Sec. III-B)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-6, 1e-3, 0.3, 2.5])
def test_se3_exp_matches_matrix_exponential(oracle_mod, scale):
    rng = np.random.default_rng(int(scale * 1e9) % 1000)
    for _ in range(5):
        xi = rng.normal(size=6) * scale
        T = oracle_mod.se3_exp(xi)
        ref = scipy.linalg.expm(_hat(xi))
        np.testing.assert_allclose(T, ref, atol=1e-13, rtol=0)


def test_lm_solve_matches_numpy(oracle_mod):
    rng = np.random.default_rng(3)
    for lam in (0.0, 1e-4, 1.0, 100.0):
        A = rng.normal(size=(6, 6))
        H = A @ A.T + 0.1 * np.eye(6)
        g = rng.normal(size=6)
        ok, d = oracle_mod.lm_solve(H, g, lam)
        ref = np.linalg.solve(H + lam * np.diag(np.diag(H)), -g)
        assert ok
        np.testing.assert_allclose(d, ref, rtol=1e-10, atol=1e-12)
    ok, _ = oracle_mod.lm_solve(-np.eye(6), np.ones(6), 1e-4)
    assert not ok


# ---------------------------------------------------------------------------
# trilinear model lookup (Sec. III-B): affine fields are reproduced exactly
# ---------------------------------------------------------------------------

def test_trilinear_reproduces_affine_fields(oracle_mod):
    voxel = 0.02
    a, b = np.array([0.3, -0.7, 0.45]), 0.01
    coords = [(bx, by, bz) for bx in range(-1, 2) for by in range(-1, 2) for bz in range(-1, 2)]
    snap = _snapshot_from_field(coords, lambda p: p @ a + b, voxel,
                                colour_fn=lambda k: 100 + k[..., 0])  # R=G=B = 100 + kx
    vol = oracle_mod.OracleVolume(voxel_size=voxel)
    vol.import_(snap)
    rng = np.random.default_rng(0)
    for _ in range(200):
        p = rng.uniform(-0.1, 0.1, size=3)
        ok, s, gs, I, gI, cok = vol.lookup(p)
        assert ok and cok
        assert abs(s - (p @ a + b)) < 1e-14
        np.testing.assert_allclose(gs, a, atol=1e-12)
        assert abs(I - (100 + p[0] / voxel) / 255.0) < 1e-12
        np.testing.assert_allclose(gI, [1.0 / (255 * voxel), 0, 0], atol=1e-10)
    # at a lattice point the interpolant equals the stored value
    ok, s, *_ = vol.lookup(np.array([3, 4, 5]) * voxel)
    assert ok and abs(s - (np.array([3, 4, 5]) * voxel @ a + b)) < 1e-15
    # outside the allocated blocks the lookup is invalid
    ok, *_ = vol.lookup(np.array([1.0, 1.0, 1.0]))
    assert not ok


def test_lookup_needs_all_eight_corners_observed(oracle_mod):
    voxel = 0.02
    snap = _snapshot_from_field([(0, 0, 0)], lambda p: p[..., 0], voxel)
    snap["W"][0, 1 + 8 * 1 + 64 * 1] = 0  # voxel (1,1,1) never observed
    vol = oracle_mod.OracleVolume(voxel_size=voxel)
    vol.import_(snap)
    assert not vol.lookup(np.array([0.5, 0.5, 0.5]) * voxel)[0]   # cell (0,0,0) uses it
    assert vol.lookup(np.array([2.5, 2.5, 2.5]) * voxel)[0]


# ---------------------------------------------------------------------------
# Eq. 2-4: normal equations, Jacobians
# ---------------------------------------------------------------------------

def test_normal_equations_on_affine_field(oracle_mod):
    """SDF F(x) = n.x - d and intensity affine in x: trilinear is exact, so
    r_d = n.p - d, J_d = [n, p x n], r_c = I(p) - I_pix, J_c = [a, p x a]."""
    O = oracle_mod
    voxel, wc = 0.02, 0.025
    T = corner_pose(0)
    depth, rgb, _ = render_frame([ROOM], CAM_TINY, T)
    pts, valid, (vs, us) = _backproject(depth, CAM_TINY, T, stride=2)
    pts, vs, us = pts[valid], vs[valid], us[valid]
    nrm = np.array([0.6, 0.0, 0.8])
    d0 = 1.1
    coords = _blocks_covering(pts, voxel)
    kx0 = coords[:, 0].min() * 8
    snap = _snapshot_from_field(coords, lambda p: p @ nrm - d0, voxel, colour_fn=lambda k: (k[..., 0] - kx0) % 256)
    assert (coords[:, 0].max() * 8 + 8 - kx0) < 256  # colour ramp stays affine (no wrap)
    vol = O.OracleVolume(voxel_size=voxel, w_c=wc)
    vol.import_(snap)
    H, g, E, N = vol.eval(_frame(O, depth, rgb, CAM_TINY), T, stride=2)
    rd = pts @ nrm - d0
    Jd = np.concatenate([np.broadcast_to(nrm, pts.shape), np.cross(pts, nrm)], axis=1)
    a = np.array([1.0 / (255.0 * voxel), 0.0, 0.0])
    Imod = (pts[:, 0] / voxel - kx0) / 255.0
    Ipix = (rgb[vs, us] @ np.array([0.2126, 0.7152, 0.0722])) / 255.0
    rc = Imod - Ipix
    Jc = np.concatenate([np.broadcast_to(a, pts.shape), np.cross(pts, a)], axis=1)
    assert N == len(pts)
    np.testing.assert_allclose(E, np.sum(rd ** 2) + wc * np.sum(rc ** 2), rtol=1e-9)
    np.testing.assert_allclose(g, Jd.T @ rd + wc * Jc.T @ rc, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(H, Jd.T @ Jd + wc * Jc.T @ Jc, rtol=1e-9, atol=1e-9)


def test_gradient_matches_finite_differences(oracle_mod):
    O = oracle_mod
    vol = _corner_volume(O)
    Tg = corner_pose(2.5)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, Tg)
    f = _frame(O, d, rgb, CAM_TINY)
    T = O.se3_exp(np.array([0.01, -0.005, 0.004, 0.003, -0.004, 0.002])) @ Tg
    _, g, E, N = vol.eval(f, T, stride=1)
    h = 1e-7
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        _, _, Ep, Np = vol.eval(f, O.se3_exp(e) @ T, stride=1)
        _, _, Em, Nm = vol.eval(f, O.se3_exp(-e) @ T, stride=1)
        assert Np == N == Nm
        fd = (Ep - Em) / (2 * h)  # dE/dxi = 2 J^T r = 2 g
        assert abs(fd - 2 * g[i]) <= 2e-5 * max(1.0, abs(fd)), (i, fd, 2 * g[i])


def test_colour_weight_zero_is_point_to_implicit(oracle_mod):
    """w_c = 0 reduces Eq. 4 to the pure depth error of Eq. 2: equal to the
    same volume with every colour weight cleared."""
    O = oracle_mod
    vol = _corner_volume(O)
    snap = vol.export()
    v0 = O.OracleVolume(voxel_size=0.02, trunc=0.1, w_c=0.0)
    v0.import_(snap)
    snap2 = dict(snap)
    snap2["wc"] = np.zeros_like(snap["wc"])
    v1 = O.OracleVolume(voxel_size=0.02, trunc=0.1)
    v1.import_(snap2)
    T = corner_pose(1.5)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, T)
    f = _frame(O, d, rgb, CAM_TINY)
    a = v0.eval(f, T, 2)
    b = v1.eval(f, T, 2)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2] and a[3] == b[3]


# ---------------------------------------------------------------------------
# LM registration (Sec. III-B): recover a known perturbation
# ---------------------------------------------------------------------------

def test_tracking_recovers_known_perturbation(oracle_mod):
    O = oracle_mod
    vol = _corner_volume(O)
    Tg = corner_pose(2.5)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, Tg)
    f = _frame(O, d, rgb, CAM_TINY)
    T_star, _ = vol.track(f, Tg)  # minimiser reached from ground truth
    assert np.linalg.norm(T_star[:3, 3] - Tg[:3, 3]) < 1e-3
    assert rot_err(T_star[:3, :3], Tg[:3, :3]) < 1e-3
    rng = np.random.default_rng(7)
    for _ in range(3):
        xi = rng.normal(size=6)
        xi[:3] *= 0.02 / np.linalg.norm(xi[:3])           # 2 cm
        xi[3:] *= math.radians(1.0) / np.linalg.norm(xi[3:])  # 1 degree
        T0 = O.se3_exp(xi) @ Tg
        T, info = vol.track(f, T0)
        assert np.linalg.norm(T[:3, 3] - T_star[:3, 3]) < 1e-6
        assert rot_err(T[:3, :3], T_star[:3, :3]) < 1e-6
        assert info.evals >= 3


def test_tracking_from_minimiser_takes_zero_step(oracle_mod):
    """Single full-resolution level run to convergence, then restarted at its
    result: the first LM step is below the convergence threshold."""
    O = oracle_mod
    vol = _corner_volume(O, lm_iters=(0, 0, 40))
    Tg = corner_pose(2.5)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, Tg)
    f = _frame(O, d, rgb, CAM_TINY)
    T1, i1 = vol.track(f, Tg)
    assert i1.converged[2] == 1
    T2, i2 = vol.track(f, T1)
    assert i2.converged[2] == 1 and i2.level_evals[2] == 1
    np.testing.assert_array_equal(T2, T1)


def test_tracking_on_empty_volume_keeps_pose(oracle_mod):
    O = oracle_mod
    vol = O.OracleVolume(voxel_size=0.02)
    T = corner_pose(0)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, T)
    T1, info = vol.track(_frame(O, d, rgb, CAM_TINY), T)
    np.testing.assert_array_equal(T1, T)
    assert info.final_valid == 0


# ---------------------------------------------------------------------------
# integration (Sec. III-A, III-D): closed forms
# ---------------------------------------------------------------------------

def _plane_expectation(cam: Camera, D_mm, voxel, tau, z_near, d_max):
    """Voxels (k, F) a fronto-parallel plane at integer depth D updates when the
    camera sits at the world origin looking along +z (exact integers)."""
    v_um = round(voxel * 1e6)
    D_um = D_mm * 1000
    out = {}
    kz_lo = int(z_near * 1e6) // v_um + 1
    kz_hi = min(D_um + round(tau * 1e6), round(d_max * 1e6)) // v_um
    fx2, cx2 = round(2 * cam.fx), round(2 * cam.cx + 1)  # exact for half-integer intrinsics
    fy2, cy2 = round(2 * cam.fy), round(2 * cam.cy + 1)
    for kz in range(kz_lo, kz_hi + 1):
        z_um = kz * v_um
        if z_um <= z_near * 1e6:
            continue
        sdf_um = D_um - z_um
        if sdf_um < -tau * 1e6:
            continue
        Fv = tau if sdf_um > tau * 1e6 else sdf_um / 1e6
        span = int(kz * (max(cam.width, cam.height) + 2) / min(cam.fx, cam.fy)) + 2
        kx = np.arange(-span, span + 1)
        # u = floor(fx x / z + cx + 1/2) = floor((2 fx kx + (2 cx + 1) kz) / (2 kz))
        u = (fx2 * kx + cx2 * kz) // (2 * kz)
        v = (fy2 * kx + cy2 * kz) // (2 * kz)
        kxs = kx[(u >= 0) & (u < cam.width)]
        kys = kx[(v >= 0) & (v < cam.height)]
        for ky in kys:
            for kxx in kxs:
                out[(int(kxx), int(ky), kz)] = Fv
    return out


def _voxels_of(snap, voxel_filter=lambda W: W > 0):
    res = {}
    for b, (bx, by, bz) in enumerate(snap["coords"]):
        idx = np.nonzero(voxel_filter(snap["W"][b]))[0]
        for i in idx:
            k = (int(bx) * 8 + int(i % 8), int(by) * 8 + int((i // 8) % 8), int(bz) * 8 + int(i // 64))
            res[k] = (snap["F"][b, i], int(snap["W"][b, i]), tuple(snap["rgb"][b, i]), int(snap["wc"][b, i]))
    return res


def test_integration_fronto_parallel_plane_closed_form(oracle_mod):
    O = oracle_mod
    cam, voxel, tau = CAM_TINY, 0.02, 0.1
    depth, rgb = fronto_plane_frame(cam, 1503, (200, 100, 50))
    vol = O.OracleVolume(voxel_size=voxel, trunc=tau)
    f = _frame(O, depth, rgb, cam)
    expect = _plane_expectation(cam, 1503, voxel, tau, 0.2, 5.0)
    for rep in (1, 2, 3):
        vol.integrate(f, np.eye(4))
        got = _voxels_of(vol.export())
        assert set(got) == set(expect)
        for k, Fv in expect.items():
            F, W, col, wc = got[k]
            assert abs(F - Fv) <= 1e-15, (k, F, Fv)  # averaging identical observations
            assert W == rep
            band = abs(Fv) < tau or (k[2] * 20000 >= 1503000 - 100000)
            if band:
                assert col == (200, 100, 50) and wc == rep
            else:
                assert wc == 0
    # allocated blocks are exactly the blocks of the updated voxels
    blocks = {tuple(np.floor_divide(k, 8)) for k in expect}
    snap = vol.export()
    assert {tuple(c) for c in snap["coords"]} == blocks


def test_carving_closed_form(oracle_mod):
    """Free voxels average towards tau: F_N = (w0 s0 + N tau) / (w0 + N), then
    geometric approach to tau at the weight cap (Sec. III-D)."""
    O = oracle_mod
    cam, voxel, tau, wmax = Camera(32, 24, 26.0, 26.0, 16.0, 12.0), 0.02, 0.1, 12
    depth, rgb = fronto_plane_frame(cam, 2000)
    k = (2, 1, 50)  # z = 1.0 m: free space in front of the 2 m plane
    b = tuple(np.floor_divide(k, 8))
    snap = _snapshot_from_field([b], lambda p: np.zeros(p.shape[:-1]), voxel)
    li = (k[0] - b[0] * 8) + 8 * (k[1] - b[1] * 8) + 64 * (k[2] - b[2] * 8)
    s0, w0 = -0.04, 5
    snap["F"][0, li] = s0
    snap["W"][0, li] = w0
    vol = O.OracleVolume(voxel_size=voxel, trunc=tau, w_max=wmax)
    vol.import_(snap)
    f = _frame(O, depth, rgb, cam)
    F = s0
    for n in range(1, 20):
        vol.integrate(f, np.eye(4))
        sn = vol.export()
        bi = int(np.nonzero((sn["coords"] == np.array(b)).all(axis=1))[0][0])
        got = (sn["F"][bi, li], int(sn["W"][bi, li]))
        if w0 + n <= wmax:
            F = (w0 * s0 + n * tau) / (w0 + n)
            assert abs(got[0] - F) < 1e-15 and got[1] == w0 + n
        else:
            F = (wmax * F + tau) / (wmax + 1)
            assert abs(got[0] - F) < 1e-15 and got[1] == wmax
    Fc = (w0 * s0 + (wmax - w0) * tau) / wmax
    assert abs(got[0] - (tau + (Fc - tau) * (wmax / (wmax + 1.0)) ** (19 - (wmax - w0)))) < 1e-14


def test_integration_sphere_projective_sdf(oracle_mod):
    """Band voxels carry D(associated pixel) - z with D the analytic ray-sphere
    depth at that pixel centre (quantised to mm)."""
    O = oracle_mod
    cam, voxel, tau = CAM_TINY, 0.02, 0.1
    T = look_at([0.0, 0.0, 0.9], SPHERE.params["center"])
    depth, rgb, _ = render_frame([ROOM, SPHERE], cam, T)
    vol = O.OracleVolume(voxel_size=voxel, trunc=tau)
    vol.integrate(_frame(O, depth, rgb, cam), T)
    got = _voxels_of(vol.export())
    ks = np.array(list(got.keys()), dtype=np.float64)
    F = np.array([got[tuple(int(c) for c in k)][0] for k in ks])
    pw = ks * voxel
    pc = (pw - T[:3, 3]) @ T[:3, :3]  # world -> camera
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    safe = (np.abs(u + 0.5 - np.round(u + 0.5)) > 1e-6) & (np.abs(v + 0.5 - np.round(v + 0.5)) > 1e-6)
    ui = np.floor(u + 0.5).astype(int)
    vi = np.floor(v + 0.5).astype(int)
    assert np.all((ui >= 0) & (ui < cam.width) & (vi >= 0) & (vi < cam.height))
    D = depth[vi, ui] / 1000.0
    sdf = D - pc[:, 2]
    band = safe & (np.abs(sdf) < tau - 1e-6)
    free = safe & (sdf > tau + 1e-6)
    assert band.sum() > 1000 and free.sum() > 1000
    np.testing.assert_allclose(F[band], sdf[band], atol=1e-8)
    np.testing.assert_allclose(F[free], tau, atol=0)
    assert np.all(sdf[safe] >= -tau - 1e-6)  # nothing behind the band was updated
    # the sphere's own band: projective distance bounds the Euclidean one
    c, r = SPHERE.params["center"], SPHERE.params["radius"]
    e = np.linalg.norm(pw - c, axis=1) - r
    on_sphere = band & (np.abs(e) < 0.05) & (np.linalg.norm(pw - c, axis=1) < r + 0.06)
    assert on_sphere.sum() > 50
    assert np.mean(np.sign(F[on_sphere]) == np.sign(e[on_sphere])) > 0.9


def _llround(x):
    x = np.asarray(x, dtype=np.float64)
    return (np.sign(x) * np.floor(np.abs(x) + 0.5)).astype(np.int64)


def _dense_integrate(state, depth, rgb, cam, T, voxel, tau, mask=None, z_near=0.2, d_min=0.2, d_max=5.0,
                     wmax=255):
    """Dense-grid restatement of the per-voxel rule over every voxel of a fixed
    box (no hashing, no blocks, no frustum search)."""
    kx, ky, kz = state["k"]
    v_um = int(round(voxel * 1e6))
    A = _llround(T[:3, :3].T * 2.0 ** 30)
    t = _llround(T[:3, 3] * 1e6)
    d = [v_um * kx - t[0], v_um * ky - t[1], v_um * kz - t[2]]
    Cs = [A[i, 0] * d[0] + A[i, 1] * d[1] + A[i, 2] * d[2] for i in range(3)]
    Cx, Cy, Cz = (c >> 20 for c in Cs)
    zn, zf = int(round(z_near * 1e6)) * 1024, int(round(d_max * 1e6)) * 1024
    ok = (Cz > zn) & (Cz <= zf)
    Czs = np.where(ok, Cz, 1)
    fxq, fyq = int(round(cam.fx * 256)), int(round(cam.fy * 256))
    cxq, cyq = int(round((cam.cx + 0.5) * 256)), int(round((cam.cy + 0.5) * 256))
    u = (fxq * Cx + cxq * Czs) // (256 * Czs)
    v = (fyq * Cy + cyq * Czs) // (256 * Czs)
    ok &= (u >= 0) & (u < cam.width) & (v >= 0) & (v < cam.height)
    ui, vi = np.where(ok, u, 0), np.where(ok, v, 0)
    raw = depth[vi, ui].astype(np.int64)
    D_um = raw * 1000
    ok &= (raw > 0) & (D_um >= d_min * 1e6) & (D_um <= d_max * 1e6)
    if mask is not None:
        ok &= mask[vi, ui] == 0
    sdf = D_um * 1024 - Cz
    tt = int(round(tau * 1e6 * 1024))
    ok &= sdf >= -tt
    band = ok & (sdf <= tt)
    x = np.where(band, sdf / 1.024e9, tau)
    W = state["W"]
    F = state["F"]
    upd = ok
    F[upd] = np.where(W[upd] == 0, x[upd], (W[upd] * F[upd] + x[upd]) / (W[upd] + 1))
    W[upd] = np.minimum(W[upd] + 1, wmax)
    col = rgb[vi, ui].astype(np.int64)
    wc = state["Wc"]
    for ch in range(3):
        C = state["rgb"][..., ch]
        num = wc[band] * C[band] + col[..., ch][band]
        C[band] = (2 * num + wc[band] + 1) // (2 * (wc[band] + 1))
    wc[band] = np.minimum(wc[band] + 1, wmax)
    return int(upd.sum())


def test_hash_reproduces_dense_grid(oracle_mod):
    """Tiny room, 3 noisy frames at ground-truth poses: every voxel of the
    hashed volume equals the dense grid and no dense update lies outside the
    allocated blocks (allocation = support of the update)."""
    from synth import make_sequence
    O = oracle_mod
    seq = make_sequence("tiny", 1, n_frames=3)
    cam, voxel, tau = seq.camera, 0.02, 0.1
    lo = np.array([-120, -120, -20])
    hi = np.array([120, 120, 170])
    shape = tuple(hi - lo)
    kk = np.meshgrid(*[np.arange(lo[i], hi[i]) for i in range(3)], indexing="ij")
    state = dict(k=kk, F=np.zeros(shape), W=np.zeros(shape, np.int64), Wc=np.zeros(shape, np.int64),
                 rgb=np.zeros(shape + (3,), np.int64))
    vol = O.OracleVolume(voxel_size=voxel, trunc=tau)
    for i in range(3):
        d, rgb, T, _ = seq.frame(i)
        n_h = vol.integrate(_frame(O, d, rgb, cam), T)
        n_d = _dense_integrate(state, d, rgb, cam, T, voxel, tau)
        assert n_h == n_d
    snap = vol.export()
    kb = snap["coords"].astype(np.int64) * 8
    assert np.all(kb >= lo) and np.all(kb + 8 <= hi)
    in_blocks = np.zeros(shape, bool)
    for b, c in enumerate(kb):
        sl = tuple(slice(c[i] - lo[i], c[i] - lo[i] + 8) for i in range(3))
        in_blocks[sl] = True
        Fd = state["F"][sl].transpose(2, 1, 0).reshape(512)   # to x + 8y + 64z order
        Wd = state["W"][sl].transpose(2, 1, 0).reshape(512)
        Wcd = state["Wc"][sl].transpose(2, 1, 0).reshape(512)
        Cd = state["rgb"][sl].transpose(2, 1, 0, 3).reshape(512, 3)
        np.testing.assert_array_equal(snap["W"][b], Wd)
        np.testing.assert_array_equal(snap["wc"][b], Wcd)
        np.testing.assert_array_equal(snap["rgb"][b], Cd)
        np.testing.assert_allclose(snap["F"][b][Wd > 0], Fd[Wd > 0], atol=1e-15)
    assert not np.any((state["W"] > 0) & ~in_blocks)
    # every allocated block holds at least one updated voxel
    assert np.all(snap["W"].max(axis=1) > 0)


# ---------------------------------------------------------------------------
# dynamics detection (Sec. III-C)
# ---------------------------------------------------------------------------

def test_morphology_matches_scipy(oracle_mod):
    rng = np.random.default_rng(11)
    st = np.ones((3, 3), bool)
    for shape in [(1, 1), (2, 3), (7, 5), (31, 47)]:
        for p in (0.3, 0.7, 0.95):
            m = (rng.random(shape) < p).astype(np.uint8)
            e = oracle_mod.erode3(m)
            np.testing.assert_array_equal(e, ndi.binary_erosion(m, st, border_value=0).astype(np.uint8))
            dl = oracle_mod.dilate3(m)
            np.testing.assert_array_equal(dl, ndi.binary_dilation(m, st, border_value=0).astype(np.uint8))


def _fixpoint_fill(MR, depth, theta_ppm):
    """Reachability by repeated relaxation until nothing changes."""
    H, W = MR.shape
    M = MR.astype(bool).copy()
    D = depth.astype(np.int64)
    changed = True
    while changed:
        changed = False
        for y in range(H):
            for x in range(W):
                if not M[y, x]:
                    continue
                for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W and not M[yy, xx]:
                        if abs(D[y, x] - D[yy, xx]) * 1_000_000 < theta_ppm * D[y, x]:
                            M[yy, xx] = True
                            changed = True
    return M.astype(np.uint8)


def test_floodfill_matches_fixpoint(oracle_mod):
    rng = np.random.default_rng(5)
    for trial in range(30):
        H, W = rng.integers(1, 14, size=2)
        depth = rng.integers(900, 1100, size=(H, W)).astype(np.uint16)
        depth[rng.random((H, W)) < 0.1] = 0
        # smooth patches so that regions grow
        depth[: H // 2, : W // 2] = 1000 + rng.integers(0, 6, size=(H // 2, W // 2))
        MR = (rng.random((H, W)) < 0.08).astype(np.uint8) & (depth > 0)
        got = oracle_mod.floodfill(MR, depth, 7000)
        np.testing.assert_array_equal(got, _fixpoint_fill(MR, depth, 7000))


def test_floodfill_edge_is_directed(oracle_mod):
    """|D(p) - D(n)| < theta D(p) uses the source depth: 1000 -> 1007 fails
    (7 < 7 is false) while 1007 -> 1000 passes (7 < 7.049)."""
    depth = np.array([[1000, 1007]], np.uint16)
    assert oracle_mod.floodfill(np.array([[1, 0]], np.uint8), depth, 7000).tolist() == [[1, 0]]
    assert oracle_mod.floodfill(np.array([[0, 1]], np.uint8), depth, 7000).tolist() == [[1, 1]]
    # invalid (zero) depth never joins
    depth = np.array([[1000, 0, 1000]], np.uint16)
    assert oracle_mod.floodfill(np.array([[1, 0, 0]], np.uint8), depth, 7000).tolist() == [[1, 0, 0]]


def test_gamma_limits(oracle_mod):
    """gamma = 1 masks nothing and gamma = 0 masks every valid pixel with a
    nonzero residual (Eq. 5)."""
    O = oracle_mod
    snap = _corner_volume(O).export()
    T = O.se3_exp(np.array([0.03, 0.0, -0.02, 0.0, 0.01, 0.0])) @ corner_pose(2.5)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, corner_pose(2.5))
    f = _frame(O, d, rgb, CAM_TINY)
    snap32 = dict(snap)
    snap32["F"] = snap["F"].astype(np.float32).astype(np.float64)  # float32(tau) > tau in FP64
    for gamma, sn in ((1.0, snap), (1.0, snap32), (0.0, snap), (0.5, snap)):
        vol = O.OracleVolume(voxel_size=0.02, trunc=0.1, gamma=gamma)
        vol.import_(sn)
        r, seeds = vol.residuals(f, T)
        if gamma == 1.0:
            assert seeds.sum() == 0 and r.max() <= 0.1 ** 2
        elif gamma == 0.0:
            np.testing.assert_array_equal(seeds, (r > 0).astype(np.uint8))
            assert seeds.sum() > 0
        else:
            np.testing.assert_array_equal(seeds, (r > 0.5 * 0.1 * 0.1).astype(np.uint8))


def test_mask_pipeline_composition_and_new_object(oracle_mod):
    """compute_mask = dilate(floodfill(erode(seeds))), and an object that is
    absent from the model (Sec. III-C) ends up masked."""
    O = oracle_mod
    snap = _corner_volume(O).export()
    vol = O.OracleVolume(voxel_size=0.02, trunc=0.1)
    vol.import_(snap)
    T = corner_pose(2.5)
    box = Prim("box", {"center": np.array([1.3, 1.1, 0.45]), "half": np.array([0.15, 0.15, 0.45]), "yaw": 0.3},
               (0.9, 0.2, 0.2), (4.0, 4.0, 4.0, 0.0, 0.0, 0.0, 5.0, 0.0), dynamic=True)
    d, rgb, dyn = render_frame([ROOM, box], CAM_TINY, T)
    f = _frame(O, d, rgb, CAM_TINY)
    _, seeds = vol.residuals(f, T)
    ref = O.dilate3(O.floodfill(O.erode3(seeds), d, 7000))
    got = vol.compute_mask(f, T)
    np.testing.assert_array_equal(got, ref)
    assert dyn.sum() > 500
    assert got[dyn].mean() > 0.9          # the new object is masked
    assert got[~dyn].mean() < 0.1         # the static room is not


# ---------------------------------------------------------------------------
# whole frame, snapshots, mesh
# ---------------------------------------------------------------------------

def test_first_frame_integrates_at_initial_pose(oracle_mod):
    O = oracle_mod
    T = corner_pose(0)
    d, rgb, _ = render_frame([ROOM], CAM_TINY, T)
    f = _frame(O, d, rgb, CAM_TINY)
    a = O.OracleVolume(voxel_size=0.02)
    Tout, mask, _ = a.process_frame(f, T)
    np.testing.assert_array_equal(Tout, T)
    assert mask.sum() == 0
    b = O.OracleVolume(voxel_size=0.02)
    b.integrate(f, T)
    sa, sb = a.export(), b.export()
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k])


def test_export_import_roundtrip(oracle_mod):
    O = oracle_mod
    s1 = _corner_volume(O, n=2).export()
    v = O.OracleVolume(voxel_size=0.02)
    v.import_(s1)
    s2 = v.export()
    for k in s1:
        np.testing.assert_array_equal(s1[k], s2[k])


def test_mesh_of_plane_lies_on_plane(oracle_mod):
    voxel, z0 = 0.02, 0.0537
    coords = [(bx, by, 0) for bx in range(2) for by in range(2)]
    snap = _snapshot_from_field(coords, lambda p: p[..., 2] - z0, voxel)
    vol = oracle_mod.OracleVolume(voxel_size=voxel)
    vol.import_(snap)
    tris, cols = vol.extract_mesh()
    assert len(tris) > 0
    np.testing.assert_allclose(tris[..., 2], z0, atol=1e-12)
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert np.all(n[:, 2] > 0)  # normals point to positive SDF (free space)
    area = 0.5 * np.linalg.norm(n, axis=1).sum()
    side = (2 * 8 - 1) * voxel  # cells with all 8 corners inside the 16x16 voxel patch
    assert abs(area - side * side) < 1e-9


def test_mesh_of_sphere_is_close_and_outward(oracle_mod):
    voxel, c, r = 0.02, np.array([0.1613, 0.1587, 0.1601]), 0.0973  # off-lattice: no exact-zero corners
    coords = [(bx, by, bz) for bx in range(3) for by in range(3) for bz in range(3)]
    snap = _snapshot_from_field(coords, lambda p: np.linalg.norm(p - c, axis=-1) - r, voxel)
    vol = oracle_mod.OracleVolume(voxel_size=voxel)
    vol.import_(snap)
    tris, _ = vol.extract_mesh()
    dist = np.linalg.norm(tris - c, axis=-1)
    assert np.abs(dist - r).max() < voxel * voxel / r
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    big = np.linalg.norm(n, axis=1) > 1e-10   # zero-area triangles at exact-zero corners carry no normal
    assert big.sum() > 0.9 * len(tris)
    assert np.all(np.einsum("ij,ij->i", n[big], tris[big].mean(axis=1) - c) > 0)


# ---------------------------------------------------------------------------
# virtual depth (Sec. III-E, second option)
# ---------------------------------------------------------------------------

def test_virtual_depth_of_a_fronto_parallel_plane_is_exact(oracle_mod):
    """The projective TSDF of a fronto-parallel plane is affine in the band, so
    the linear interpolation of the crossing recovers the plane depth exactly:
    from the integrating pose, from a pose 10 cm closer, and from a pose moved
    sideways (interior pixels whose rays stay in the observed region)."""
    O = oracle_mod
    cam = CAM_TINY
    vol = O.OracleVolume(voxel_size=0.02, trunc=0.1)
    depth, rgb = fronto_plane_frame(cam, 1503, (200, 100, 50))
    vol.integrate(_frame(O, depth, rgb, cam), np.eye(4))
    zero = np.zeros_like(depth)
    f0 = _frame(O, zero, rgb, cam)
    m = 12
    out = vol.virtual_depth(f0, np.eye(4))
    assert np.all(out[m:-m, m:-m] == 1503)
    T = np.eye(4)
    T[2, 3] = 0.1
    assert np.all(vol.virtual_depth(f0, T)[m:-m, m:-m] == 1403)
    T = np.eye(4)
    T[0, 3] = 0.05
    assert np.all(vol.virtual_depth(f0, T)[m:-m, m:-m] == 1503)


def test_virtual_depth_fill_rules(oracle_mod):
    """Non-zero pixels are copied unchanged (even outside the valid range);
    zero pixels without a crossing get the far value (d_max by default)."""
    O = oracle_mod
    cam = CAM_TINY
    vol = O.OracleVolume(voxel_size=0.02, trunc=0.1)
    rng = np.random.default_rng(4)
    depth = np.where(rng.random((cam.height, cam.width)) < 0.5, 0, rng.integers(1, 9000, (cam.height, cam.width)))
    depth = depth.astype(np.uint16)
    rgb = np.zeros((cam.height, cam.width, 3), np.uint8)
    f = _frame(O, depth, rgb, cam)
    out = vol.virtual_depth(f, np.eye(4))  # empty model: no crossing anywhere
    np.testing.assert_array_equal(out[depth > 0], depth[depth > 0])
    assert np.all(out[depth == 0] == 5000)
    assert np.all(vol.virtual_depth(f, np.eye(4), far_raw=65535)[depth == 0] == 65535)
    # a plane model fills exactly the zero pixels
    plane, prgb = fronto_plane_frame(cam, 2000)
    vol.integrate(_frame(O, plane, prgb, cam), np.eye(4))
    out = vol.virtual_depth(f, np.eye(4))
    np.testing.assert_array_equal(out[depth > 0], depth[depth > 0])
    inner = np.zeros_like(depth, dtype=bool)
    inner[12:-12, 12:-12] = True
    assert np.all(out[(depth == 0) & inner] == 2000)


def test_virtual_depth_of_a_sphere_matches_the_ray_intersection(oracle_mod):
    """Integrated from one view and cast from the same view, the crossing lies
    on the analytic sphere where the surface faces the camera (cos > 0.9),
    within the error of the projective TSDF: a stored value takes the depth of
    the voxel's nearest pixel, up to half a pixel off its ray, i.e. up to
    0.5 z/fx tan(theta) of depth slope, plus 0.5 mm of depth quantisation."""
    O = oracle_mod
    cam = CAM_TINY
    T = look_at([1.2, 0.2, 0.9], SPHERE.params["center"])
    d, rgb, _ = render_frame([SPHERE], cam, T)
    vol = O.OracleVolume(voxel_size=0.02, trunc=0.1)
    vol.integrate(_frame(O, d, rgb, cam), T)
    out = vol.virtual_depth(_frame(O, np.zeros_like(d), rgb, cam), T)
    # analytic depth along each pixel ray (camera z), and the facing angle
    c = np.linalg.inv(T)[:3, :3] @ SPHERE.params["center"] + np.linalg.inv(T)[:3, 3]
    r = SPHERE.params["radius"]
    u, v = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    dirs = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones_like(u, dtype=float)], -1)
    a = (dirs * dirs).sum(-1)
    b = -2 * (dirs * c).sum(-1)
    disc = b * b - 4 * a * (c @ c - r * r)
    hit = disc > 0
    z = np.where(hit, (-b - np.sqrt(np.where(hit, disc, 0))) / (2 * a), 0.0)
    p = dirs * z[..., None]
    n = (p - c) / r
    facing = np.where(hit, -(n * dirs).sum(-1) / np.sqrt(a), 0.0)
    sel = hit & (facing > 0.9) & (d > 0)
    assert sel.sum() > 500
    err = np.abs(out[sel].astype(np.float64) - z[sel] * 1000.0)
    tan = np.sqrt(np.clip(1.0 - facing[sel] ** 2, 0.0, None)) / facing[sel]
    bound = 0.5 + 1000.0 * 0.5 * z[sel] / cam.fx * tan + 0.5  # + rounding of the result
    assert np.all(err <= bound), float((err - bound).max())


# ---------------------------------------------------------------------------
# closed-form pins of the mask residual, the colour average and tracking
# ---------------------------------------------------------------------------

# A camera whose pixels back-project onto the voxel lattice: with fx = fy =
# 128, principal point (80, 60), voxel 8 mm and a depth of 1.024 m, pixel
# (u, v) lands on lattice point (u - 80, v - 60, 128) exactly.
LATTICE_CAM = Camera(160, 120, 128.0, 128.0, 80.0, 60.0)
LATTICE_VOXEL = 0.008
LATTICE_DEPTH_MM = 1024


def _lattice_texture(kx, ky):
    """Integer grey level of lattice column (kx, ky): a smooth texture with
    gradients along x and y (values 28..228)."""
    return np.rint(128.0 + 50.0 * np.sin(2 * np.pi * kx / 37.0) + 50.0 * np.sin(2 * np.pi * ky / 29.0 + 1.0))


def _lattice_plane_snapshot(z_margin=0.2):
    """Model of the plane z = 1.024 m seen by LATTICE_CAM at the identity pose:
    F(p) = 1.024 - p_z (affine, positive in front), voxel colour the grey
    texture of its (kx, ky) column."""
    v = LATTICE_VOXEL
    zc = LATTICE_DEPTH_MM / 1000.0
    reach = (LATTICE_CAM.width / 2 + 2) / LATTICE_CAM.fx * (zc + z_margin)
    bx = np.arange(int(np.floor(-reach / (8 * v))) - 1, int(np.floor(reach / (8 * v))) + 2)
    by = np.arange(int(np.floor(-reach * 0.75 / (8 * v))) - 1, int(np.floor(reach * 0.75 / (8 * v))) + 2)
    bz = np.arange(int(np.floor((zc - z_margin) / (8 * v))), int(np.floor((zc + z_margin) / (8 * v))) + 1)
    zz, yy, xx = np.meshgrid(bz, by, bx, indexing="ij")
    coords = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    return _snapshot_from_field(coords, lambda p: zc - p[..., 2], v,
                                colour_fn=lambda k: _lattice_texture(k[..., 0], k[..., 1]))


def _lattice_frame(depth_mm):
    cam = LATTICE_CAM
    vs, us = np.mgrid[0:cam.height, 0:cam.width]
    depth = np.full((cam.height, cam.width), depth_mm, np.uint16)
    g = _lattice_texture(us - 80, vs - 60).astype(np.uint8)
    return depth, np.repeat(g[..., None], 3, axis=2)


def test_mask_residual_is_the_squared_sdf_of_an_offset_plane(oracle_mod):
    """Eq. 2's underbraced term r_i = V_SDF(T x_i)^2 against a closed form: a
    frame of the plane moved by delta along the view gives V_SDF = -delta at
    every pixel (the model is affine, so trilinear lookup is exact), hence
    r_i = delta^2, and tau^2 once |delta| > tau (the TSDF is truncated at tau,
    Sec. III-A).  Eq. 5 seeds r_i > gamma tau^2 = 0.005 at gamma = 0.5,
    tau = 0.1: the decision flips between |delta| = 60 mm and 80 mm.  Seeding
    on |V_SDF| instead of its square would seed at 60 mm already."""
    O = oracle_mod
    vol = O.OracleVolume(voxel_size=LATTICE_VOXEL, trunc=0.1, gamma=0.5)
    vol.import_(_lattice_plane_snapshot())
    for delta_mm, seeded in ((-150, True), (-80, True), (-60, False), (0, False), (60, False), (80, True),
                             (150, True)):
        depth, rgb = _lattice_frame(LATTICE_DEPTH_MM + delta_mm)
        r, seeds = vol.residuals(_frame(O, depth, rgb, LATTICE_CAM), np.eye(4))
        delta = delta_mm / 1000.0
        expect = min(delta * delta, 0.1 * 0.1)
        assert np.all(r >= 0.0)  # every pixel has a valid model lookup
        np.testing.assert_allclose(r, expect, rtol=0, atol=1e-12)
        assert seeds.all() if seeded else not seeds.any(), delta_mm


def test_colour_running_average_rounds_half_up(oracle_mod):
    """Colour running average (Sec. III-A; reading: RGB8 stored rounded half
    up at every update, own weight Wc), hand-computed per channel:
      (100, 50, 7) then (101, 53, 8): 100.5 -> 101, 51.5 -> 52, 7.5 -> 8
      (truncation would give 100, 51, 7; round-half-even 100, 52, 8);
      (100, 50, 7) twice then (101, 52, 9): 301/3 -> 100, 152/3 -> 51, 23/3 -> 8."""
    O = oracle_mod
    cam, voxel, tau = CAM_TINY, 0.02, 0.1
    for colours, expect in ((((100, 50, 7), (101, 53, 8)), (101, 52, 8)),
                            (((100, 50, 7), (100, 50, 7), (101, 52, 9)), (100, 51, 8))):
        vol = O.OracleVolume(voxel_size=voxel, trunc=tau)
        for c in colours:
            depth, rgb = fronto_plane_frame(cam, 1503, c)
            vol.integrate(_frame(O, depth, rgb, cam), np.eye(4))
        got = _voxels_of(vol.export(), voxel_filter=lambda W: W > 0)
        band = [v for v in got.values() if v[3] > 0]
        assert len(band) > 1000
        for F, W, col, wc in band:
            assert col == expect and wc == len(colours), (col, expect, wc)


def test_tracking_recovers_an_exact_minimiser(oracle_mod):
    """A scene where the ground truth is an exact minimiser of Eq. 4: the
    plane z = 1.024 m (affine TSDF model) with a grey texture on the voxel
    lattice, seen by a camera whose pixels back-project onto lattice points,
    so every depth and colour residual is zero at the true pose (the identity)
    and the plane's normal plus the texture's two gradient directions observe
    all six pose parameters.  From 2 cm / 1 degree perturbations LM must
    return the ground truth to 1e-8 (convergence thresholds tightened so that
    the levels run to machine precision)."""
    O = oracle_mod
    vol = O.OracleVolume(voxel_size=LATTICE_VOXEL, trunc=0.2, lm_iters=(10, 10, 30), lm_eps_trans=1e-13,
                         lm_eps_rot=1e-13)
    vol.import_(_lattice_plane_snapshot())
    depth, rgb = _lattice_frame(LATTICE_DEPTH_MM)
    f = _frame(O, depth, rgb, LATTICE_CAM)
    H, g, E, N = vol.eval(f, np.eye(4), stride=1)
    assert N == LATTICE_CAM.width * LATTICE_CAM.height and E < 1e-20  # zero residuals at the truth
    assert np.linalg.eigvalsh(H).min() > 1e-6 * np.linalg.eigvalsh(H).max()  # no unobserved direction
    rng = np.random.default_rng(11)
    for _ in range(3):
        xi = rng.normal(size=6)
        xi[:3] *= 0.02 / np.linalg.norm(xi[:3])
        xi[3:] *= math.radians(1.0) / np.linalg.norm(xi[3:])
        T, info = vol.track(f, O.se3_exp(xi))
        assert np.linalg.norm(T[:3, 3]) < 1e-8, T[:3, 3]
        assert rot_err(T[:3, :3], np.eye(3)) < 1e-8
        assert info.evals >= 4


def test_tracking_footprint_fixture_matches_the_oracle(oracle_mod):
    """The stored registration footprint (tests/golden/track_footprint_static.json,
    written by make_track_footprint.py from the oracle alone) is what the
    oracle counts now, on the first frame's two registrations; counting does
    not change the registration's result."""
    O = oracle_mod
    from synth import make_sequence
    g = json.load(open(os.path.join(GOLDEN, "track_footprint_static.json")))
    seq = make_sequence("static", 1000)
    cam = seq.camera
    vol = O.OracleVolume(voxel_size=0.01, trunc=0.1)
    d, rgb, T, _ = seq.frame(0)
    vol.integrate(_frame(O, d, rgb, cam), T)
    d, rgb, _, _ = seq.frame(1)
    f = _frame(O, d, rgb, cam)
    T1, _, b1, v1 = vol.track_footprint(f, T)
    T1_plain, _ = vol.track(f, T)
    np.testing.assert_array_equal(T1, T1_plain)
    mask = vol.compute_mask(f, T1)
    _, _, b2, v2 = vol.track_footprint(f, T1, mask)
    rows = [r for r in g["rows"] if r["frame"] == 1]
    assert [(r["blocks_probed"], r["voxels_read"]) for r in rows] == [(b1, v1), (b2, v2)]
    assert 0 < b1 < vol.num_blocks and 0 < v1 < 512 * b1


def test_model_intensity_uses_the_papers_luminance_weights(oracle_mod):
    """V_I of a model whose voxels all carry one colour (R, G, B) is the
    intensity of Sec. III-B, (w_R R + w_G G + w_B B) / 255, with the weights
    printed there (tests/golden/intensity_weights.json); the gradient is zero."""
    O = oracle_mod
    w = json.load(open(os.path.join(GOLDEN, "intensity_weights.json")))["weights"]
    coords = [(bx, by, bz) for bx in range(2) for by in range(2) for bz in range(2)]
    snap = _snapshot_from_field(coords, lambda p: p[..., 2] - 0.05, 0.02)
    for rgb in ((255, 0, 0), (0, 255, 0), (0, 0, 255), (200, 100, 50)):
        snap["rgb"][:] = rgb
        snap["wc"][:] = 1
        vol = O.OracleVolume(voxel_size=0.02)
        vol.import_(snap)
        ok, s, gs, I, gI, cok = vol.lookup(np.array([0.1234, 0.1711, 0.0931]))
        assert ok and cok
        assert abs(I - np.dot(w, rgb) / 255.0) < 1e-14, (rgb, I)
        np.testing.assert_allclose(gI, 0.0, atol=1e-12)
