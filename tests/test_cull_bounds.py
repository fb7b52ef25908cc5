"""The conservative culls of stage 1 against the oracle's exact snapping.

The cull kernels drop a (triangle, pair) -- or a whole group of triangles of
one pair -- when a bbox estimated in FP32 with rcp.approx, widened by an
error bound, holds no pixel centre.  That is only sound if every exact
snapped vertex (the oracle's projection: fixed-order FP32 transform, IEEE
division, 1/256-pixel snap) lies inside the widened estimate.  These tests
restate the host constants (margin terms, window, near-plane limit, row
rounding bounds) and the kernels' FP32 arithmetic in numpy, sample vertices
and small vertex groups under the bench cameras and random instance
transforms, and check that the exact positions never leave the widened
ranges: the worst excursion must stay below the margin.  rcp.approx is
modelled with a relative error of 2^-20 either way, the error the margins
are derived for (8 times the documented bound of the instruction).
"""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import oracle as orc

U = 2.0 ** -24
RHO = 2.0 ** -20
F32 = np.float32


def _f32(x):
    return np.asarray(x, np.float64).astype(F32)


def _fma(a, b, c):
    """a * b + c with one rounding to FP32 (the product of two FP32 values is
    exact in FP64)."""
    return _f32(np.asarray(a, F32).astype(np.float64) * np.asarray(b, F32).astype(np.float64)
                + np.asarray(c, F32).astype(np.float64))


def _rcp(x, s):
    """rcp.approx modelled as the exact reciprocal off by RHO = 2^-20
    relative, the error the host's margins assume, in direction s."""
    return _f32(1.0 / np.asarray(x, F32).astype(np.float64) * (1.0 + s * RHO))


def _constants(mv, lo, hi, cp, W, H):
    """The per-pair constants of the host: FMA rows for X'w, Y'w and w (X' =
    X - 1/2), the margin terms ka..kd, wsafe, the window and the rows'
    rounding bounds; None where the host turns the test off."""
    fx, fy, near = (float(v) for v in cp)
    hw, hh = W / 2.0, H / 2.0
    amax = np.maximum(np.abs(lo), np.abs(hi))
    M = np.asarray(mv, np.float64).reshape(3, 4)
    Sr = np.abs(M[:, 3]) + np.abs(M[:, :3]) @ amax
    ax, bx, ay, by = hw * fx, hw - 0.5, hh * fy, hh - 0.5
    wr = -M[2]
    rows = (_f32(ax * M[0] + bx * wr), _f32(ay * M[1] + by * wr), _f32(wr))
    ws = near * (1 + 1e-3) + 8 * U * Sr[2]
    F = 1.01 * (1 + 4 * U * Sr[2] / ws) / (1 - RHO)
    kax = 9.002 * ax * Sr[0] + 4.001 * bx * Sr[2] + 4.001 * hw * Sr[2] + 7.002 * Sr[2]
    kay = 9.002 * ay * Sr[1] + 4.001 * by * Sr[2] + 4.001 * hh * Sr[2] + 7.002 * Sr[2]
    ka, kb = F * U * max(kax, kay), F * U * 7.002 * Sr[2]
    kc = 1.01 * (RHO + 7.01 * U)
    kd = 1.01 * (5.01 * U * (max(hw, hh) + 1) + RHO + 7.01 * U) + 1.0 / 512
    win = 100.0 * min(hw, hh)
    room = 20.0 * min(hw, hh) - kc * win - kd
    if not room > 0:
        return None
    ws = max(ws, 1.01 * (1 + RHO) * (ka + kb * win) / room)
    k = _f32(np.array([ka, kb, kc, kd]) * (1 + 1e-6))
    sl = _f32(np.array([(ax * Sr[0] + bx * Sr[2]), (ay * Sr[1] + by * Sr[2]), Sr[2]]) * 2.0 ** -19 * (1 + 1e-6))
    return rows, k, F32(ws * (1 + 1e-6)), F32(win), sl


def _row(r, x, y, z):
    return _fma(r[0], x, _fma(r[1], y, _fma(r[2], z, r[3])))


def _setups():
    """(model-view, camera params, W, H, mesh bounds, label): the billion
    frame's tiles, close-up poses of the unique heightfield, and far, rotated
    and scaled instances as in the many-mesh workload."""
    rng = np.random.default_rng(7)
    lo, hi = np.array([0.0, -0.25, 0.0]), np.array([1.0, 0.25, 1.0])
    out = []
    cam = S.camera_billion(3840, 2160, 8)
    for tx, tz in ((0, 0), (3, 5), (7, 7)):
        model = np.eye(4, dtype=np.float32)
        model[0, 3], model[2, 3] = tx, tz
        out.append((cam, model, lo, hi, f"billion tile {tx},{tz}"))
    for k in (0, 3, 6):
        out.append((S.camera_unique_pose(k, 1920, 1080), np.eye(4, dtype=np.float32), lo, hi, f"unique pose {k}"))
    # extremes: a tiny near plane with the mesh far away, and a huge instance seen from afar
    # (large row magnitudes, so wsafe is raised well above near)
    cam = S.Camera(S.look_at((0.5, 0.3, -0.2), (0.5, 0.0, 0.6)), S.perspective(70.0, 16 / 9, 1e-3, 100.0), 1920, 1080)
    far = np.eye(4, dtype=np.float32)
    far[:3, 3] = (0.0, 0.0, 40.0)
    out.append((cam, far, lo, hi, "tiny near, far mesh"))
    big = np.eye(4)
    big[:3, :3] = S.scenes._random_rotation(rng) * 1000.0
    big[:3, 3] = (-300.0, -10.0, -300.0)
    centre = big[:3, :3] @ np.array([0.5, 0.0, 0.5]) + big[:3, 3]
    out.append((S.Camera(S.look_at(tuple(centre + np.array([0.0, 700.0, -1200.0])), tuple(centre)),
                         S.perspective(60.0, 16 / 9, 0.05, 5000.0), 3840, 2160),
                big.astype(np.float32), lo, hi, "instance of scale 1000"))
    for k, (W, H) in enumerate(((640, 360), (3840, 2160), (1920, 1080))):
        ang = rng.uniform(0, 2 * np.pi)
        eye = (140 * math.cos(ang), 70.0, 140 * math.sin(ang))
        cam = S.Camera(S.look_at(eye, (0, 0, 0)), S.perspective(60.0, W / H, 0.05, 2000.0), W, H)
        model = np.eye(4)
        model[:3, :3] = S.scenes._random_rotation(rng) * rng.uniform(0.1, 10.0)
        model[:3, 3] = (rng.uniform(-100, 100), 0.0, rng.uniform(-100, 100))
        out.append((cam, model.astype(np.float32), lo, hi, f"instance {k} {W}x{H}"))
    return out


SETUPS = _setups()


def _exact(mv, cp, cam, pts):
    _, XY, _, inside = orc.project(mv, cp, cam.W, cam.H, pts.reshape(-1, 3))
    Xe = XY[:, 0].astype(np.float64) / 256.0 - 0.5
    Ye = XY[:, 1].astype(np.float64) / 256.0 - 0.5
    return Xe.reshape(pts.shape[:-1]), Ye.reshape(pts.shape[:-1]), inside.reshape(pts.shape[:-1])


def _vertex_margin_worst(setup, kscale=1.0, n=60000):
    """Largest ratio of the exact snapped vertex's distance from its estimate
    to the margin m (scaled by kscale) over sampled mesh points where the
    test applies, and the number of such samples (both rcp directions)."""
    cam, model, lo, hi, _ = setup
    cp = orc.camera_params(np.asarray(cam.proj, np.float32))
    mv = orc.model_view(np.asarray(cam.view, np.float32), model)
    c = _constants(mv, lo, hi, cp, cam.W, cam.H)
    assert c is not None
    rows, k, ws, win, _ = c
    pts = np.random.default_rng(11).uniform(lo, hi, size=(n, 3)).astype(F32)
    Xe, Ye, inside = _exact(mv, cp, cam, pts)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    xw, yw, w = _row(rows[0], x, y, z), _row(rows[1], x, y, z), _row(rows[2], x, y, z)
    worst, applied = 0.0, 0
    for s in (-1, 1):
        r = _rcp(w, s)
        X, Y = _f32(xw * r), _f32(yw * r)
        a = np.maximum(np.abs(X), np.abs(Y))
        m = _fma(r, _fma(k[1], a, k[0]), _fma(k[2], a, k[3])).astype(np.float64) * kscale
        ok = (w > ws) & (a < win)
        # the premise of the bound: every tested vertex is snapped unclipped,
        # which the host secures by keeping the margin below 20 min(W/2, H/2)
        assert inside[ok].all(), "a tested vertex lies outside the guard band in the exact path"
        assert (m[ok] < 20.0 * min(cam.W, cam.H) / 2.0).all()
        err = np.maximum(np.abs(X - Xe), np.abs(Y - Ye))
        applied += int(ok.sum())
        if ok.any():
            worst = max(worst, float((err[ok] / m[ok]).max()))
    return worst, applied


@pytest.mark.parametrize("setup", SETUPS, ids=[s[-1] for s in SETUPS])
def test_triangle_margin_holds_exact_snapped_vertices(setup):
    """Per vertex: the estimate X'~ = (X'w) * rcp(w) from the FMA rows and the
    exact snapped X' differ by less than m = max(1/w)(ka + kb a) + kc a + kd
    wherever the test applies (w > wsafe, |X'|, |Y'| < window)."""
    worst, applied = _vertex_margin_worst(setup)
    assert applied > 0
    assert worst < 1.0, f"an exact snapped vertex lies {worst:.3f} margins from its estimate"


def test_a_margin_a_quarter_too_small_is_caught():
    """The check is sharp: with the margin constants scaled by 1/4 some exact
    snapped vertex falls outside its widened estimate."""
    worst = max(_vertex_margin_worst(s, kscale=0.25, n=20000)[0] for s in SETUPS)
    assert worst > 1.0


@pytest.mark.parametrize("setup", SETUPS, ids=[s[-1] for s in SETUPS])
def test_group_margin_holds_exact_snapped_vertices(setup):
    """Per group of vertices: the instanced cull's range X0 +- max|d| / min w
    (the box's projected centre, the affine residual d = X'w - X0 w over the
    box, rows widened by their rounding bound), widened by the doubled
    margin, holds the exact snapped X' of every vertex of the group."""
    cam, model, lo, hi, _ = setup
    cp = orc.camera_params(np.asarray(cam.proj, np.float32))
    mv = orc.model_view(np.asarray(cam.view, np.float32), model)
    c = _constants(mv, lo, hi, cp, cam.W, cam.H)
    assert c is not None
    (rx, ry, rw), k, ws, win, sl = c
    rng = np.random.default_rng(13)
    nbox, npts = 3000, 24
    size = (10.0 ** rng.uniform(-4, -1.5, size=(nbox, 1, 1))) * rng.uniform(0.1, 1.0, size=(nbox, 1, 3))
    centre = rng.uniform(lo, hi, size=(nbox, 1, 3))
    pts = np.clip(centre + rng.uniform(-1, 1, size=(nbox, npts, 3)) * size, lo, hi).astype(F32)
    Xe, Ye, inside = _exact(mv, cp, cam, pts)
    blo, bhi = pts.min(axis=1), pts.max(axis=1)
    gc = _f32(_f32(blo + bhi) * F32(0.5))
    ge = np.maximum(_f32(bhi - gc), _f32(gc - blo))
    cx = _row(rx, gc[:, 0], gc[:, 1], gc[:, 2])
    cy = _row(ry, gc[:, 0], gc[:, 1], gc[:, 2])
    cw = _row(rw, gc[:, 0], gc[:, 1], gc[:, 2])
    arw = np.abs(rw)
    ew = _fma(arw[0], ge[:, 0], _fma(arw[1], ge[:, 1], _fma(arw[2], ge[:, 2], sl[2])))
    wl = _f32(cw - ew)

    def half(Z0, r, cz, s_):
        acc = _fma(np.abs(Z0), sl[2], _f32(np.abs(_fma(-Z0, cw, cz)) + s_))
        for j in (2, 1, 0):
            acc = _fma(np.abs(_fma(-Z0, rw[j], r[j])), ge[:, j], acc)
        return acc

    worst, applied = 0.0, 0
    for s in (-1, 1):
        r0 = _rcp(cw, s)
        X0, Y0 = _f32(cx * r0), _f32(cy * r0)
        dx, dy = half(X0, rx, cx, sl[0]), half(Y0, ry, cy, sl[1])
        rh = _f32(_rcp(wl, s) * F32(1.0000039))
        hx, hy = _f32(dx * rh), _f32(dy * rh)
        a = np.maximum(_f32(np.abs(X0) + hx), _f32(np.abs(Y0) + hy))
        m = (_f32(F32(2.0) * _fma(rh, _fma(k[1], a, k[0]), _fma(k[2], a, k[3])))
             + _f32(F32(2.0) * _f32(hx + hy) * F32(4.0e-6))).astype(np.float64)
        ok = (wl > ws) & (a < win)
        assert inside[ok].all(), "a tested group holds a vertex outside the guard band in the exact path"
        exc = np.maximum.reduce([(X0 - hx)[:, None] - Xe, Xe - (X0 + hx)[:, None],
                                 (Y0 - hy)[:, None] - Ye, Ye - (Y0 + hy)[:, None]]).max(axis=1)
        exc = np.maximum(exc, 0.0)
        applied += int(ok.sum())
        if ok.any():
            worst = max(worst, float((exc[ok] / m[ok]).max()))
    assert applied > 0
    assert worst < 1.0, f"an exact snapped vertex lies {worst:.3f} margins outside its group's range"


@pytest.mark.parametrize("setup", SETUPS, ids=[s[-1] for s in SETUPS])
def test_near_plane_bound_holds_exact_depths(setup):
    """The near-plane cull of stage 1: a vertex whose estimated w (the w row,
    the exact path's coefficients negated, evaluated by FMA) lies below
    nlo = near - 8 u S_z has an exact w (the oracle's fixed-order FP32
    transform) below near, so a triangle with all three vertices there is
    dropped by the exact path's clipping as well.  Checked on random points
    of the mesh bounds and on points placed within a few margins of the near
    plane (solved for the coordinate with the largest w coefficient)."""
    cam, model, lo, hi, _ = setup
    cp = orc.camera_params(np.asarray(cam.proj, np.float32))
    mv = orc.model_view(np.asarray(cam.view, np.float32), model)
    M = np.asarray(mv, np.float64).reshape(3, 4)
    amax = np.maximum(np.abs(lo), np.abs(hi))
    Sz = abs(M[2, 3]) + np.abs(M[2, :3]) @ amax
    near = float(cp[2])
    nl = near - 8 * U * Sz
    nlo = np.float32(nl)
    if float(nlo) > nl:
        nlo = np.nextafter(nlo, np.float32(-np.inf))
    rw = _f32(-M[2])                                   # exact: negation of FP32 coefficients
    rng = np.random.default_rng(17)
    pts = rng.uniform(lo, hi, size=(40000, 3))
    # points on the near plane: w = -(m . p + m3) = near (1 + t), solved for the axis j
    j = int(np.argmax(np.abs(M[2, :3]) * (hi - lo)))
    span = max(1e-5, 3 * 8 * U * Sz / near)          # a few times the margin, relative to near
    t = rng.uniform(-span, span, size=40000)
    q = rng.uniform(lo, hi, size=(40000, 3))
    rest = M[2, 3] + sum(M[2, a] * q[:, a] for a in range(3) if a != j)
    if abs(M[2, j]) > 0:
        q[:, j] = (-near * (1 + t) - rest) / M[2, j]
    q = q[((q >= lo) & (q <= hi)).all(1)]
    pts = np.concatenate([pts, q]).astype(F32)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    w_est = _row(rw, x, y, z)
    clipv, _, _, _ = orc.project(mv, cp, cam.W, cam.H, pts)
    w_exact = clipv[:, 2]
    below = w_est < nlo
    assert (w_exact[below] < np.float32(near)).all()
    if len(q) > 100:
        # the boundary is exercised: points within 1e-5 of the plane on both sides of nlo
        close = np.abs(w_exact.astype(np.float64) - near) < 2 * span * near
        assert (below & close).any() and (~below & close).any()
