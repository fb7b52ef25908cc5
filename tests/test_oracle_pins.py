"""Pins of the oracle against things other than itself.

Each test checks the oracle (oracle/curast_oracle.c) against an independent
fact: float64 geometry, an exact brute force with a differently formulated
tie-break, closed-form pixel counts, tilings, invariants of closed meshes,
triangle order and duplicate instances, and finite differences for the
adjoint.  A dropped term, a flipped sign, a transposed operand or a wrong
index anywhere in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import synthetic as S
from synthetic.scenes import Camera, Instance, Mesh, Scene

rng0 = np.random.default_rng(1234)


def mesh_np(pos, idx, rgba8=None):
    return Mesh(pos=torch.tensor(np.asarray(pos, np.float32)), idx=torch.tensor(np.asarray(idx, np.int32)),
                rgba8=None if rgba8 is None else torch.tensor(np.asarray(rgba8, np.uint8)))


def ident():
    return np.eye(4, dtype=np.float32)


def f32bits(x):
    return int(np.array([x], np.float32).view(np.uint32)[0])


# ----------------------------------------------------------------- camera ---
def test_camera_params_follow_projection_vector(oracle_lib):
    O = oracle_lib
    for fovy, aspect, near, far in [(60, 1.0, 1e-3, 1000.0), (45, 16 / 9, 0.1, 50.0), (90, 0.5, 2.0, None)]:
        p = S.perspective(fovy, aspect, near, far)
        fx, fy, n = O.camera_params(p)
        f = 1.0 / math.tan(math.radians(fovy) / 2)
        assert fx == pytest.approx(f / aspect, rel=1e-6)
        assert fy == pytest.approx(f, rel=1e-6)
        assert n == pytest.approx(near, rel=2e-3)
    bad = S.perspective(60, 1.0, 0.1, 10.0)
    bad[0, 2] = 0.1          # off-centre projection is not the projection vector of Eq. 2
    with pytest.raises(ValueError):
        O.camera_params(bad)


def test_model_view_is_the_matrix_product(oracle_lib):
    O = oracle_lib
    for _ in range(20):
        v = np.eye(4)
        m = np.eye(4)
        v[:3, :] = rng0.normal(size=(3, 4))
        m[:3, :] = rng0.normal(size=(3, 4)) * 3
        v, m = v.astype(np.float32), m.astype(np.float32)
        ref = (v.astype(np.float64) @ m.astype(np.float64))[:3]
        got = O.model_view(v, m)
        np.testing.assert_allclose(got, ref, rtol=1.2e-7, atol=1e-6 * np.abs(ref).max())


def _view64(mv, pts):
    M = np.asarray(mv, np.float64).reshape(3, 4)
    return pts.astype(np.float64) @ M[:, :3].T + M[:, 3]


def test_projection_matches_float64_geometry(oracle_lib):
    """Snapped positions sit within half a subpixel (plus FP32 error) of
    X = (fx vx / d + 1) W/2 in float64, y up, and only vertices in front of
    the near plane and inside the guard band are flagged inside."""
    O = oracle_lib
    W, H = 640, 360
    view = S.look_at((0.3, 1.2, 2.0), (0.0, 0.0, -1.0))
    proj = S.perspective(70, W / H, 0.05, 100.0)
    cp = O.camera_params(proj)
    mv = O.model_view(view, ident())
    pts = rng0.uniform(-3, 3, size=(4000, 3)).astype(np.float32)
    clipv, XY, iz, inside = O.project(mv, cp, W, H, pts)
    v = _view64(mv, pts.astype(np.float32))
    d = -v[:, 2]
    front = d >= cp[2] * (1 + 1e-6)
    sx = cp[0] * v[:, 0] / d
    sy = cp[1] * v[:, 1] / d
    guard = (np.abs(sx) < 128 * (1 - 1e-6)) & (np.abs(sy) < 128 * (1 - 1e-6))
    ok = front & guard
    assert inside[ok].all()
    assert not inside[d < cp[2] * (1 - 1e-6)].any()
    X = (sx + 1) * W / 2
    Y = (sy + 1) * H / 2
    # forward error bound of the FP32 evaluation: each view coordinate is off
    # by at most 6u * sum|terms|, amplified by 1/d through the division
    u = 2.0 ** -24
    M = np.asarray(mv, np.float64)
    sab = np.abs(pts.astype(np.float64)) @ np.abs(M[:, :3]).T + np.abs(M[:, 3])
    for S_, s_, WH, f, axis in ((X, sx, W, cp[0], 0), (Y, sy, H, cp[1], 1)):
        bound = (WH / 2) * (f * 6 * u * sab[:, axis] + np.abs(s_) * 6 * u * sab[:, 2]) / d
        tol = 1 / 512 + bound + 8 * u * (np.abs(S_) + WH)
        err = np.abs(XY[ok, axis] / 256.0 - S_[ok])
        assert (err <= tol[ok]).all()
    rel_d = 6 * u * sab[ok, 2] / d[ok] + 2 * u
    assert (np.abs(iz[ok] * d[ok] - 1.0) <= rel_d).all()
    # a point above the optical axis lands in the upper half (row 0 = bottom)
    up = ok & (v[:, 1] > 0.05 * d)
    assert (XY[up, 1] > 256 * H // 2).all()


# --------------------------------------------------------------- coverage ---
SH = 40   # perturbation exponent: sample moved by (2^-20, -2^-40) subpixel units


def brute_force_mask(tri, W, H):
    """Exact brute force of one triangle's samples, written independently of
    the fill rule: a pixel centre P belongs to the (CCW-ordered) triangle iff
    the slightly moved point P + (e, -e^2), e = 2^-20 subpixel units, lies
    strictly inside all three edges.  Integer arithmetic scaled by 2^40."""
    (x0, y0), (x1, y1), (x2, y2) = tri
    A = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
    if A == 0:
        return np.zeros((H, W), bool)
    if A < 0:
        (x1, y1), (x2, y2) = (x2, y2), (x1, y1)
    V = [(x0 << SH, y0 << SH), (x1 << SH, y1 << SH), (x2 << SH, y2 << SH)]
    out = np.zeros((H, W), bool)
    for y in range(H):
        py = ((256 * y + 128) << SH) - 1
        for x in range(W):
            px = ((256 * x + 128) << SH) + (1 << 20)
            inside = True
            for k in range(3):
                ax, ay = V[k]
                bx, by = V[(k + 1) % 3]
                if (bx - ax) * (py - ay) - (by - ay) * (px - ax) <= 0:
                    inside = False
                    break
            out[y, x] = inside
    return out


def _random_fixed_triangles(n, W, H, rng):
    tris = []
    for i in range(n):
        kind = i % 4
        if kind == 0:      # anywhere, subpixel positions
            t = rng.integers(-300, 256 * W + 300, size=(3, 2))
        elif kind == 1:    # vertices exactly on pixel centres
            t = rng.integers(0, W, size=(3, 2)) * 256 + 128
        elif kind == 2:    # axis-aligned edges through centres
            a = rng.integers(0, W, size=2) * 256 + 128
            w, h = rng.integers(1, 8, size=2) * 256
            t = np.array([a, a + [w, 0], a + [0, h]])
        else:              # small, around one pixel centre
            c = rng.integers(1, W - 1, size=2) * 256 + 128
            t = c + rng.integers(-300, 300, size=(3, 2))
        tris.append([(int(t[k, 0]), int(t[k, 1])) for k in range(3)])
    return tris


def test_coverage_matches_brute_force(oracle_lib):
    O = oracle_lib
    W = H = 20
    rng = np.random.default_rng(7)
    tris = _random_fixed_triangles(160, W, H, rng)
    for t in tris:
        XY = np.array(t, np.int32).reshape(1, 6)
        got = O.raster_fixed(XY, np.ones((1, 3), np.float32), W, H, mode=1, cull_back=False)
        np.testing.assert_array_equal(got.astype(bool), brute_force_mask(t, W, H), err_msg=str(t))


def test_tiling_covers_every_pixel_exactly_once(oracle_lib):
    """A triangulation of the viewport rectangle (random vertices, some on
    pixel centres, some on centre lines) covers each sample exactly once."""
    from scipy.spatial import Delaunay
    O = oracle_lib
    W, H = 48, 32
    rng = np.random.default_rng(11)
    pts = [(0, 0), (256 * W, 0), (0, 256 * H), (256 * W, 256 * H)]
    pts += [tuple(p) for p in rng.integers(1, [256 * W, 256 * H], size=(60, 2))]
    pts += [tuple(p) for p in rng.integers(0, [W, H], size=(40, 2)) * 256 + 128]
    pts += [(int(x) * 256 + 128, int(y)) for x, y in rng.integers(0, [W, 256 * H], size=(20, 2))]
    pts = np.array(sorted(set(pts)), np.int64)
    tri = Delaunay(pts.astype(np.float64)).simplices
    XY = pts[tri].reshape(-1, 6)
    a = (XY[:, 2] - XY[:, 0]) * (XY[:, 5] - XY[:, 1]) - (XY[:, 4] - XY[:, 0]) * (XY[:, 3] - XY[:, 1])
    XY[a < 0] = XY[a < 0][:, [0, 1, 4, 5, 2, 3]]        # orient CCW
    cnt = O.raster_fixed(XY.astype(np.int32), np.ones((len(XY), 3), np.float32), W, H, mode=1)
    assert (cnt == 1).all()


@pytest.mark.parametrize("a", list(range(1, 13)) + [31, 64])
def test_closed_form_counts(oracle_lib, a):
    """Right isosceles triangle with legs a through pixel centres covers
    a(a-1)/2 samples; the square of side a through centres covers a^2."""
    O = oracle_lib
    W = H = a + 4
    c = 2 * 256 + 128            # the pixel centre (2, 2)
    L = 256 * a
    tri = np.array([[c, c, c + L, c, c, c + L]], np.int32)
    n = O.raster_fixed(tri, np.ones((1, 3), np.float32), W, H, mode=1)
    assert int(n.sum()) == a * (a - 1) // 2
    sq = np.array([[c, c, c + L, c, c + L, c + L], [c, c, c + L, c + L, c, c + L]], np.int32)
    n = O.raster_fixed(sq, np.ones((2, 3), np.float32), W, H, mode=1)
    assert int(n.sum()) == a * a and n.max() == 1


def test_full_viewport_quad_covers_w_times_h(oracle_lib):
    O = oracle_lib
    W, H = 37, 23
    q = np.array([[0, 0, 256 * W, 0, 0, 256 * H], [256 * W, 0, 256 * W, 256 * H, 0, 256 * H]], np.int32)
    cnt = O.raster_fixed(q, np.ones((2, 3), np.float32), W, H, mode=1)
    assert (cnt == 1).all() and int(cnt.sum()) == W * H


def _golden_rows(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


def test_visibility_word_golden(oracle_lib):
    """Words of fragments at exactly known depths match the hand-derived
    values of tests/golden/visibility_word.txt (28 depth bits over 36 id
    bits, Section 4.1), and the closer fragment wins in either order."""
    O = oracle_lib
    tri = np.array([[0, 0, 2048, 0, 0, 2048]], np.int32)     # covers every centre of 4x4
    rows = _golden_rows("visibility_word.txt")
    assert len(rows) == 6
    for iz, tid, word in rows:
        vis = O.raster_fixed(tri, np.full((1, 3), float(iz), np.float32), 4, 4, id0=int(tid))
        assert (vis == np.uint64(int(word, 16))).all(), (iz, tid, hex(int(vis[0, 0])))
    # depth 1 (iz 1) beats depth 2 (iz 0.5) whichever of the two comes first
    two = np.concatenate([tri, tri])
    for izs, want in (([0.5, 1.0], 0x7F00000000000001), ([1.0, 0.5], 0x7F00000000000000)):
        iz = np.array([[izs[0]] * 3, [izs[1]] * 3], np.float32)
        vis = O.raster_fixed(two, iz, 4, 4, id0=0)
        assert (vis == np.uint64(want)).all(), hex(int(vis[0, 0]))


# -------------------------------------------------------------- end to end ---
def _cam(view, proj, W, H):
    return Camera(np.asarray(view, np.float32), np.asarray(proj, np.float32), W, H)


def test_camera_facing_plane_depth(oracle_lib):
    """A quad at view depth D filling the frustum: every pixel covered once,
    every depth within one 28-bit step of bits(D) >> 3."""
    O = oracle_lib
    W, H = 64, 48
    for D in (0.37, 3.0, 250.0):
        h = 4 * D
        pos = [[-h, -h, -D], [h, -h, -D], [-h, h, -D], [h, h, -D]]
        sc = Scene([mesh_np(pos, [[0, 1, 2], [1, 3, 2]])], [Instance(0, ident())])
        cam = _cam(np.eye(4), S.perspective(60, W / H, 0.01, 1000.0), W, H)
        osc = O.OracleScene(sc)
        assert (O.render(osc, cam, mode=1) == 1).all()
        d28, ids = O.decode(O.render(osc, cam))
        ref = f32bits(D) >> 3
        assert np.abs(d28.astype(np.int64) - ref).max() <= 1
        assert set(np.unique(ids)) <= {0, 1}


def _convex_mesh(rng, n=40, r=1.0):
    from scipy.spatial import ConvexHull
    p = rng.normal(size=(n, 3))
    p = r * p / np.linalg.norm(p, axis=1, keepdims=True) * rng.uniform(0.7, 1.0, size=(n, 1))
    hull = ConvexHull(p)
    tri = hull.simplices.copy()
    cen = p.mean(0)
    for k, t in enumerate(tri):
        nrm = np.cross(p[t[1]] - p[t[0]], p[t[2]] - p[t[0]])
        if np.dot(nrm, p[t[0]] - cen) < 0:
            tri[k] = t[[0, 2, 1]]
    return p.astype(np.float32), tri.astype(np.int32)


def test_closed_convex_mesh_is_watertight(oracle_lib):
    """Without backface culling every sample inside the silhouette of a
    closed convex mesh is covered exactly twice (front and back layer); with
    culling exactly once, on the same samples."""
    O = oracle_lib
    rng = np.random.default_rng(5)
    W, H = 96, 80
    for trial in range(4):
        pos, tri = _convex_mesh(rng)
        sc = Scene([mesh_np(pos, tri)], [Instance(0, ident())])
        eye = rng.normal(size=3)
        eye = 3.5 * eye / np.linalg.norm(eye)
        cam = _cam(S.look_at(eye, (0, 0, 0)), S.perspective(50, W / H, 0.1, 100.0), W, H)
        osc = O.OracleScene(sc)
        both = O.render(osc, cam, mode=1, cull_back=False)
        front = O.render(osc, cam, mode=1, cull_back=True)
        assert set(np.unique(both)) <= {0, 2}
        assert set(np.unique(front)) <= {0, 1}
        np.testing.assert_array_equal(both == 2, front == 1)
        assert (front == 1).sum() > 500


def test_result_independent_of_triangle_order(oracle_lib):
    O = oracle_lib
    hf = S.heightfield_mesh(24, seed=3)
    cam = _cam(S.look_at((0.5, 0.6, -0.4), (0.5, 0.05, 0.5)), S.perspective(60, 1.0, 1e-3, 10.0), 96, 96)
    osc = O.OracleScene(Scene([hf], [Instance(0, ident())]))
    d1, i1 = O.decode(O.render(osc, cam))
    perm = np.random.default_rng(2).permutation(hf.T)
    hp = Mesh(pos=hf.pos, idx=hf.idx[torch.tensor(perm)])
    d2, i2 = O.decode(O.render(O.OracleScene(Scene([hp], [Instance(0, ident())])), cam))
    np.testing.assert_array_equal(d1, d2)
    cov = d1 != (O.EMPTY >> np.uint64(36))
    mapped = perm[i2[cov].astype(np.int64)]
    differ = mapped != i1[cov].astype(np.int64)
    assert differ.mean() < 1e-3       # only exact depth ties may pick another id


def test_duplicate_instance_changes_nothing(oracle_lib):
    O = oracle_lib
    hf = S.heightfield_mesh(16, seed=9)
    cam = _cam(S.look_at((0.5, 0.7, -0.3), (0.5, 0.0, 0.5)), S.perspective(60, 1.0, 1e-3, 10.0), 64, 64)
    one = O.render(O.OracleScene(Scene([hf], [Instance(0, ident())])), cam)
    two = O.render(O.OracleScene(Scene([hf], [Instance(0, ident()), Instance(0, ident())])), cam)
    np.testing.assert_array_equal(one, two)


def _plane_hit(cam, fx, fy, ypl, W, H):
    """float64 ray cast of every pixel centre against the plane y = ypl."""
    V = np.asarray(cam.view, np.float64)
    Rinv = V[:3, :3].T
    eye = -Rinv @ V[:3, 3]
    x = (2 * np.arange(W) + 1) / W - 1
    y = (2 * np.arange(H) + 1) / H - 1
    rv = np.stack(np.broadcast_arrays(x[None, :] / fx, y[:, None] / fy, -np.ones((H, W))), -1)
    rw = rv @ Rinv.T
    t = (ypl - eye[1]) / rw[..., 1]
    return t, eye + t[..., None] * rw   # view depth d = t (ray has unit -z component)


def test_near_clipped_fan_matches_ray_cast(oracle_lib):
    """A large fan on the plane y = -0.3 whose centre lies behind the camera
    (near plane crosses most triangles): every sample whose float64 ray hit
    lies clearly inside the fan and in front of the near plane is covered
    exactly once, no sample twice, rays that miss the plane cover nothing,
    and depths agree with the float64 hit distance."""
    O = oracle_lib
    W, H = 160, 120
    R, ypl, k = 40.0, -0.3, 12
    ang = np.arange(k) * 2 * np.pi / k
    ctr = np.array([0.0, ypl, 2.0])
    pos = np.vstack([ctr, np.stack([R * np.cos(ang), np.full(k, ypl), R * np.sin(ang)], 1) + [0, 0, 2.0]])
    tri = np.array([[0, 1 + (i + 1) % k, 1 + i] for i in range(k)])
    sc = Scene([mesh_np(pos, tri)], [Instance(0, ident())])
    proj = S.perspective(75, W / H, 0.02, 100.0)
    cam = _cam(S.look_at((0, 0, 0), (0, -0.25, -1)), proj, W, H)
    osc = O.OracleScene(sc)
    fx, fy, nr = O.camera_params(proj)
    cnt = O.render(osc, cam, mode=1, cull_back=True)
    assert cnt.max() == 1
    t, hit = _plane_hit(cam, fx, fy, ypl, W, H)
    rr = np.hypot(hit[..., 0] - 0.0, hit[..., 2] - 2.0)
    inner = R * math.cos(math.pi / k)
    clear = (t > nr * 1.01) & (rr < inner * 0.99)
    miss = ~(t > 0)
    assert clear.sum() > 0.3 * W * H and miss.sum() > 0.1 * W * H
    assert (cnt[clear] == 1).all()
    assert (cnt[miss] == 0).all()
    d28, _ = O.decode(O.render(osc, cam))
    depth = (d28[clear].astype(np.uint32) << np.uint32(3)).view(np.float32).astype(np.float64)
    # 1/d is affine in screen space on a plane; snapping the vertices by at
    # most 1/512 px moves it by at most a few subpixels times its gradient
    inv = 1.0 / t
    g = np.hypot(np.nanmax(np.abs(np.diff(inv[clear.any(1)], axis=1))),
                 np.nanmax(np.abs(np.diff(inv[:, clear.any(0)], axis=0))))
    tol = t[clear] ** 2 * g * 3.0 / 256.0 + 4e-6 * t[clear]
    assert (np.abs(depth - t[clear]) <= tol).all()


def test_clip_polygon_properties(oracle_lib):
    """Clipped polygons lie inside every plane, inside the input triangle
    (barycentric weights in [0, 1]) and keep its orientation; unclipped
    triangles come back unchanged; triangles beyond one plane vanish."""
    O = oracle_lib
    rng = np.random.default_rng(3)
    nearv = np.float32(0.05)
    for _ in range(300):
        tri = np.stack([rng.uniform(-400, 400, 3), rng.uniform(-400, 400, 3), rng.uniform(-1, 3, 3)], 1)
        tri = tri.astype(np.float32)
        poly = O.clip(tri, nearv)
        w = tri[:, 2].astype(np.float64)
        x = tri[:, 0].astype(np.float64)
        y = tri[:, 1].astype(np.float64)
        inside = (w >= nearv) & (np.abs(x) <= 128 * w) & (np.abs(y) <= 128 * w)
        if inside.all():
            np.testing.assert_array_equal(poly, tri)
            continue
        if (w < nearv).all() or (x > 128 * w).all() or (x < -128 * w).all():
            assert len(poly) == 0
        if len(poly) == 0:
            continue
        assert 3 <= len(poly) <= 8
        P = poly.astype(np.float64)
        tol = 1e-4 * (np.abs(tri).max() + 1)
        assert (P[:, 2] >= nearv * (1 - 1e-6)).all()
        assert (np.abs(P[:, 0]) <= 128 * P[:, 2] + tol).all()
        assert (np.abs(P[:, 1]) <= 128 * P[:, 2] + tol).all()
        T = tri.astype(np.float64)
        bary, *_ = np.linalg.lstsq(T.T, P.T, rcond=None)
        well = abs(np.linalg.det(T)) > 1e-3 * np.abs(T).max() ** 3
        if well:
            assert (bary > -1e-3).all() and (bary < 1 + 1e-3).all()


def test_near_plane_cut_lies_on_the_plane(oracle_lib):
    """The point where an edge meets the near plane w = near has w = near
    exactly (Section 4.2 clips against the near plane; the intersection is a
    point of the plane).  x and y come from the FP32 interpolation and carry
    its rounding, but w is fixed by the geometry: every vertex the near cut
    creates must hold w == near bit for bit.  Triangles are kept well inside
    the guard band, so the near plane is the only cut."""
    O = oracle_lib
    rng = np.random.default_rng(29)
    nearv = np.float32(0.05)
    created = 0
    for _ in range(400):
        w = rng.uniform(-1.0, 2.0, 3)
        if (w >= nearv).all() or (w < nearv).all():
            continue
        xy = rng.uniform(-0.1, 0.1, (3, 2))
        tri = np.concatenate([xy, w[:, None]], 1).astype(np.float32)
        poly = O.clip(tri, nearv)
        assert len(poly) in (3, 4)
        for v in poly:
            if any(np.array_equal(v, t) for t in tri):
                continue
            created += 1
            assert v[2] == nearv, f"near cut at w = {v[2]!r}, not {nearv!r}"
    assert created > 200


def test_shared_edges_clip_watertight(oracle_lib):
    """Random triangle pairs sharing an edge that crosses the near plane and
    the guard band never double-cover a sample."""
    O = oracle_lib
    rng = np.random.default_rng(17)
    W, H = 64, 48
    proj = S.perspective(90, W / H, 0.5, 100.0)
    cam = _cam(np.eye(4), proj, W, H)
    for _ in range(60):
        a = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(-4, -0.6)])
        b = np.array([rng.uniform(-300, 300), rng.uniform(-300, 300), rng.uniform(-0.4, 2)])
        c = a + rng.normal(size=3) * [3, 3, 0.5]
        d = b + rng.normal(size=3) * [3, 3, 0.5]
        pos = np.stack([a, b, c, d])
        sc = Scene([mesh_np(pos, [[0, 1, 2], [1, 0, 3]])], [Instance(0, ident())])
        cnt = O.render(O.OracleScene(sc), cam, mode=1, cull_back=False)
        # c and d on opposite sides of ab -> each sample at most once
        n1 = np.cross(b - a, c - a)
        n2 = np.cross(b - a, d - a)
        if np.dot(n1, n2) < 0:
            assert cnt.max() <= 1


# ---------------------------------------------------------------- resolve ---
def test_resolve_barycentrics_match_linear_solve(oracle_lib):
    O = oracle_lib
    sc = S.scene_small(n=32, W=96, H=96)
    cam = sc.cameras[0]
    osc = O.OracleScene(sc)
    vis = O.render(osc, cam)
    _, bary = O.interpolate(osc, cam, vis, 0, np.zeros((sc.meshes[0].V, 1), np.float32))
    fx, fy, _ = O.camera_params(cam.proj)
    mv = O.model_view(cam.view, ident())
    _, ids = O.decode(vis)
    ys, xs = np.nonzero((vis != O.EMPTY) & (ids < sc.meshes[0].T))
    idx = sc.meshes[0].idx.numpy()
    pos = sc.meshes[0].pos.numpy()
    errs = []
    for y, x in zip(ys[::7], xs[::7]):
        t = int(ids[y, x])
        v = _view64(mv, pos[idx[t]])
        r = np.array([((2 * x + 1) / 96 - 1) / fx, ((2 * y + 1) / 96 - 1) / fy, -1.0])
        Msys = np.stack([v[1] - v[0], v[2] - v[0], -r], 1)
        u, w, _ = np.linalg.solve(Msys, -v[0])
        errs.append(np.abs(bary[y, x] - [1 - u - w, u, w]).max())
    assert len(errs) > 50 and max(errs) < 2e-3 and np.median(errs) < 1e-5


def test_resolve_constant_colour_and_background(oracle_lib):
    O = oracle_lib
    hf = S.heightfield_mesh(12, seed=4)
    col = np.tile(np.array([[200, 17, 99, 255]], np.uint8), (hf.V, 1))
    sc = Scene([Mesh(hf.pos, hf.idx, torch.tensor(col))], [Instance(0, ident())])
    cam = _cam(S.look_at((0.5, 1.5, -0.8), (0.5, 0.0, 0.5)), S.perspective(40, 1.0, 0.01, 10.0), 64, 64)
    osc = O.OracleScene(sc)
    vis = O.render(osc, cam)
    rgba, rgba8 = O.resolve(osc, cam, vis)
    cov = vis != O.EMPTY
    assert cov.sum() > 200 and (~cov).sum() > 200
    assert (rgba8[cov] == [200, 17, 99, 255]).all()
    assert (rgba8[~cov] == 0).all() and (rgba[~cov] == 0).all()
    np.testing.assert_allclose(rgba[cov], np.broadcast_to(np.array([200, 17, 99, 255]) / 255.0, rgba[cov].shape),
                               atol=1e-6)


def test_resolve_rgba8_clamps_extrapolated_colours(oracle_lib):
    """The resolve's barycentrics are not clamped (Section 4.4 extrapolates
    outside the triangle for mip levels): a buffer that names one small
    triangle at every pixel gives FP32 colours far outside [0, 1] away from
    it, and RGBA8 is rint(clamp(c, 0, 1) * 255) of those FP32 colours."""
    O = oracle_lib
    pos = [[-0.1, -0.1, -2.0], [0.1, -0.1, -2.0], [0.0, 0.1, -2.0]]
    col = [[255, 0, 128, 255], [0, 255, 0, 255], [0, 0, 255, 255]]
    sc = Scene([mesh_np(pos, [[0, 1, 2]], col)], [Instance(0, ident())])
    cam = _cam(np.eye(4), S.perspective(60, 1.0, 0.01, 10.0), 40, 40)
    osc = O.OracleScene(sc)
    vis = np.full((40, 40), np.uint64(1 << 36), np.uint64)             # triangle 0 everywhere
    rgba, rgba8 = O.resolve(osc, cam, vis)
    assert (rgba > 1.01).any() and (rgba < -0.01).any()
    want = np.rint(np.clip(rgba.astype(np.float64), 0.0, 1.0) * 255.0).astype(np.uint8)
    np.testing.assert_array_equal(rgba8, want)


def test_ids_follow_prefix_sum_with_empty_instances(oracle_lib):
    """Id = base[instance] + triangle; zero-triangle instances share their
    base with the successor and never capture a pixel in the resolve."""
    O = oracle_lib
    hf = S.heightfield_mesh(8, seed=2)
    empty = Mesh(pos=hf.pos, idx=torch.zeros((0, 3), dtype=torch.int32), rgba8=hf.rgba8)
    cam = _cam(S.look_at((0.5, 1.2, -0.6), (0.5, 0.0, 0.5)), S.perspective(50, 1.0, 0.01, 10.0), 48, 48)
    shift = np.eye(4, dtype=np.float32)
    shift[0, 3] = 0.2
    a = Scene([hf, empty], [Instance(1, ident()), Instance(0, ident()), Instance(1, ident()), Instance(0, shift)])
    b = Scene([hf], [Instance(0, ident()), Instance(0, shift)])
    oa, ob = O.OracleScene(a), O.OracleScene(b)
    np.testing.assert_array_equal(oa.bases(), [0, 0, 128, 128, 256])
    va, vb = O.render(oa, cam), O.render(ob, cam)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(O.resolve(oa, cam, va)[1], O.resolve(ob, cam, vb)[1])


def test_id_space_overflow_is_rejected(oracle_lib):
    O = oracle_lib
    hf = S.heightfield_mesh(2, seed=2)
    big = Scene([None, hf], [Instance(0, ident()), Instance(1, ident())])
    with pytest.raises(ValueError):
        O.OracleScene(big, tri_counts=[(1 << 36) - 4, 0]).bases()
    ok = O.OracleScene(big, tri_counts=[(1 << 36) - 1 - hf.T, 0]).bases()
    assert int(ok[-1]) == (1 << 36) - 1


# ------------------------------------------------------------- compression ---
def test_compression_golden_examples(oracle_lib):
    """The paper's worked examples (tests/golden/compression.txt): indices
    2500..3000 take 9 bits; 16 bits over 65 m resolve 1 mm."""
    O = oracle_lib
    rows = _golden_rows("compression.txt")
    kinds = {r[0] for r in rows}
    assert kinds == {"index", "position"}
    for r in rows:
        if r[0] == "index":
            assert O.index_bits(int(r[2]) - int(r[1])) == int(r[3])
        else:
            span, prec = float(r[1]), float(r[2])
            pos = np.array([[0, 0, 0], [span, 1, 1]], np.float32)
            f, dec, _ = O.compress_mesh(pos, np.array([0, 1, 1], np.uint32))
            assert float(f["step"][0]) <= prec
            np.testing.assert_allclose(dec, pos, rtol=0, atol=prec / 2 + 1e-5)


def test_index_packing_round_trip_and_bit_layout(oracle_lib):
    """Packing is exact for every width 0..32, and the stream holds index k's
    bits at k * bits, little-endian (checked against a bit-matrix layout);
    a span that is a power of two needs one bit more than log2(span)."""
    O = oracle_lib
    rng = np.random.default_rng(31)
    assert O.index_bits(512) == 10 and O.index_bits(511) == 9 and O.index_bits(0) == 0
    for bits in list(range(0, 33)):
        span = (1 << bits) - 1
        imin = int(rng.integers(0, 2**32 - span)) if bits < 32 else 0
        n = 97
        idx = (imin + rng.integers(0, span + 1, size=n, dtype=np.uint64)).astype(np.uint32)
        if bits > 0:
            idx[0], idx[1] = imin, imin + span
        assert O.index_bits(int(idx.max()) - int(idx.min())) == (bits if bits > 0 else 0)
        words = O.pack_indices(idx, imin, bits)
        np.testing.assert_array_equal(O.unpack_indices(words, n, imin, bits), idx)
        # independent layout: a bits-wide little-endian bit matrix, flattened
        v = (idx.astype(np.uint64) - imin)
        m = ((v[:, None] >> np.arange(bits, dtype=np.uint64)[None, :]) & 1).astype(np.uint8).reshape(-1)
        m = np.concatenate([m, np.zeros((-m.size) % 32 + 32, np.uint8)])
        ref = np.packbits(m.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").reshape(-1)
        np.testing.assert_array_equal(words[:ref.size], ref)


def test_position_quantization_error_and_ends(oracle_lib):
    """Decoded positions lie within half a step (plus FP32 rounding) of the
    originals; the minimum decodes exactly; a flat axis decodes to its value."""
    O = oracle_lib
    rng = np.random.default_rng(32)
    pos = np.stack([rng.uniform(-3.0, 5.0, 5000), rng.uniform(10.0, 10.5, 5000), np.full(5000, 2.25)], 1)
    pos = pos.astype(np.float32)
    f, dec, _ = O.compress_mesh(pos, np.arange(3, dtype=np.uint32))
    step = f["step"].astype(np.float64)
    err = np.abs(dec.astype(np.float64) - pos.astype(np.float64))
    tol = step / 2 + 4 * np.finfo(np.float32).eps * np.abs(pos).max(axis=0)
    assert (err <= tol).all()
    i = np.argmin(pos[:, 0])
    assert dec[i, 0] == pos[i, 0]
    assert (dec[:, 2] == np.float32(2.25)).all()


def test_positions_on_the_grid_survive_compression(oracle_lib):
    """Positions that are decoded grid points (fma(q, step, lo)) quantize back
    to the same q, so encoding them loses nothing."""
    O = oracle_lib
    rng = np.random.default_rng(33)
    lo = np.array([-2.5, 0.0, 7.0], np.float32)
    size = np.array([8.0, 0.75, 3.0], np.float64)
    step = (size / 65535.0).astype(np.float32)
    q = rng.integers(0, 65536, size=(4000, 3)).astype(np.uint16)
    q[0] = 0
    q[1] = 65535
    pos = O.dequantize_positions(q, lo, step)
    np.testing.assert_array_equal(O.quantize_positions(pos, lo, size), q)


# ---------------------------------------------------------- super sampling ---
def test_box_filter_identity_mean_and_half_coverage(oracle_lib):
    """ss = 1 is the plain resolve; the box filter is the mean of the ss x ss
    samples (float64 reference); a triangle edge between sample columns
    covers exactly half of every pixel's samples."""
    O = oracle_lib
    rng = np.random.default_rng(21)
    fine = rng.uniform(0, 1, size=(6, 10, 4)).astype(np.float32)
    r1, q1 = O.box_filter(fine, 1)
    np.testing.assert_array_equal(r1, fine)
    np.testing.assert_array_equal(q1, np.rint(fine * 255).astype(np.uint8))
    r2, _ = O.box_filter(fine, 2)
    ref = fine.astype(np.float64).reshape(3, 2, 5, 2, 4).mean(axis=(1, 3))
    np.testing.assert_allclose(r2, ref, rtol=0, atol=3e-7)
    # a camera-facing quad whose right edge runs between the two sample
    # columns of every pixel (ss = 2): colour / 2 in every covered pixel
    W, H, ss, D = 8, 6, 2, 2.0
    t = math.tan(math.radians(30.0))
    hx, hy = D * t * W / H, D * t                 # half extents of the view at depth D
    xr = -hx + 2 * hx * (2 * 3 + 1) / (ss * W)    # boundary between sample columns 6 and 7
    pos = [[-2 * hx, -2 * hy, -D], [xr, -2 * hy, -D], [-2 * hx, 2 * hy, -D], [xr, 2 * hy, -D]]
    col = np.full((4, 4), 200, np.uint8)
    sc = Scene([mesh_np(pos, [[0, 1, 2], [1, 3, 2]], col)], [Instance(0, ident())])
    cam = _cam(np.eye(4), S.perspective(60, W / H, 0.01, 100.0), ss * W, ss * H)
    osc = O.OracleScene(sc)
    vis = O.render(osc, cam)
    r, _ = O.resolve_ss(osc, cam, vis, ss)
    c = 200.0 / 255.0      # constant colour: barycentric interpolation is exact to a few ulps
    np.testing.assert_allclose(r[:, :3, :], c, rtol=0, atol=4e-7)
    np.testing.assert_allclose(r[:, 3, :], c / 2, rtol=0, atol=4e-7)
    np.testing.assert_array_equal(r[:, 4:, :], 0)


# --------------------------------------------------------------- adjoint ---
def _small_diff_scene():
    sc, col = S.scene_differentiable(n=20, W=72, H=64)
    return sc, col.numpy()


def test_forward64_matches_closed_form_and_fp32_oracle(oracle_lib):
    from oracle import adjoint as A
    O = oracle_lib
    sc, col = _small_diff_scene()
    cam = sc.cameras[0]
    osc = O.OracleScene(sc)
    vis = O.render(osc, cam)
    fx, fy, _ = O.camera_params(cam.proj)
    mv = O.model_view(cam.view, ident())
    m = sc.meshes[0]
    tri = A.pixel_triangles(vis, 0, m.T)
    out64, b64, cov = A.forward64(m.pos.numpy(), m.idx.numpy(), col, mv, fx, fy, cam.W, cam.H, tri)
    bcf = A.barycentrics_closed_form(m.pos.numpy(), m.idx.numpy(), mv, fx, fy, cam.W, cam.H, tri)
    assert cov.sum() > 1000
    np.testing.assert_allclose(b64, bcf, atol=1e-9)
    out32, _ = O.interpolate(osc, cam, vis, 0, col)
    np.testing.assert_allclose(out32.reshape(-1, 3), out64, atol=2e-4)


def test_adjoint_matches_central_differences(oracle_lib):
    from oracle import adjoint as A
    O = oracle_lib
    sc, col = _small_diff_scene()
    cam = sc.cameras[0]
    osc = O.OracleScene(sc)
    vis = O.render(osc, cam)
    fx, fy, _ = O.camera_params(cam.proj)
    mv = O.model_view(cam.view, ident())
    m = sc.meshes[0]
    pos = m.pos.numpy().astype(np.float64)
    idx = m.idx.numpy()
    tri = A.pixel_triangles(vis, 0, m.T)
    rng = np.random.default_rng(8)
    target = rng.uniform(0, 1, size=(cam.W * cam.H, 3))
    col64 = col.astype(np.float64)
    out, _, _ = A.forward64(pos, idx, col64, mv, fx, fy, cam.W, cam.H, tri)
    g = 2.0 * (out - target)
    dcol, dpos = A.adjoint64(pos, idx, col64, mv, fx, fy, cam.W, cam.H, tri, g)

    def L(p, c):
        return A.loss64(p, idx, c, mv, fx, fy, cam.W, cam.H, tri, target)

    used = np.unique(idx[tri[tri >= 0]])
    h = 1e-5       # float64 central differences: truncation ~(h/cell)^2, rounding ~1e-16 L/h
    for v in rng.choice(used, size=40, replace=False):
        for ax in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[v, ax] += h
            pm[v, ax] -= h
            fd = (L(pp, col64) - L(pm, col64)) / (2 * h)
            assert fd == pytest.approx(dpos[v, ax], rel=1e-5, abs=1e-7 * (np.abs(dpos).max() + 1))
            cp_, cm_ = col64.copy(), col64.copy()
            cp_[v, ax] += h
            cm_[v, ax] -= h
            fd = (L(pos, cp_) - L(pos, cm_)) / (2 * h)
            assert fd == pytest.approx(dcol[v, ax], rel=1e-6, abs=1e-9)


# ------------------------------------------- paper-mode stage 3 (R16) ---
def _ray_hits64(fx, fy, tri_view, W, H):
    """float64 barycentrics (b0, b1, b2) and hit distance t of every
    pixel-centre ray (ndx / fx, ndy / fy, -1) with a view-space triangle,
    from a direct 3x3 solve of v0 + b1 e1 + b2 e2 = t r."""
    v = np.asarray(tri_view, np.float64)
    x = (2 * np.arange(W) + 1) / W - 1
    y = (2 * np.arange(H) + 1) / H - 1
    r = np.stack(np.broadcast_arrays(x[None, :] / fx, y[:, None] / fy, -np.ones((H, W))), -1)
    e1, e2 = v[1] - v[0], v[2] - v[0]
    M = np.stack([np.broadcast_to(e1, (H, W, 3)), np.broadcast_to(e2, (H, W, 3)), -r], -1)
    sol = np.linalg.solve(M, np.broadcast_to(-v[0], (H, W, 3))[..., None])[..., 0]
    b1, b2, t = sol[..., 0], sol[..., 1], sol[..., 2]
    return 1 - b1 - b2, b1, b2, t


def test_paper_stage3_plane_depth_closed_form(oracle_lib):
    """The paper's ray-cast stage 3 on a quad at view depth D that fills the
    frustum (far beyond stage 1's and stage 2's limits): every depth within
    one 28-bit step of bits(D) >> 3, each triangle covering the pixels on its
    side of the diagonal.  The ray cast is not watertight: a pixel centre
    within rounding of the shared diagonal may be missed by both triangles,
    and only there may a pixel stay empty."""
    O = oracle_lib
    W, H = 64, 48
    for D in (0.37, 3.0, 250.0):
        h = 4 * D
        pos = [[-h, -h, -D], [h, -h, -D], [-h, h, -D], [h, h, -D]]
        sc = Scene([mesh_np(pos, [[0, 1, 2], [1, 3, 2]])], [Instance(0, ident())])
        proj = S.perspective(60, W / H, 0.01, 1000.0)
        cam = _cam(np.eye(4), proj, W, H)
        fx, fy, _ = O.camera_params(proj)
        vis = O.render_paper(O.OracleScene(sc), cam, s1_max=128, s2_max=1000)
        d28, ids = O.decode(vis)
        hit = vis != O.EMPTY
        assert hit.sum() >= W * H - max(W, H)
        assert np.abs(d28.astype(np.int64) - (f32bits(D) >> 3))[hit].max() <= 1
        # the diagonal from (h, -h) to (-h, h): side of each pixel's float64 hit
        t0 = _ray_hits64(fx, fy, np.asarray(pos)[[0, 1, 2]], W, H)
        t1 = _ray_hits64(fx, fy, np.asarray(pos)[[1, 3, 2]], W, H)
        m0 = np.minimum(np.minimum(t0[0], t0[1]), t0[2])
        m1 = np.minimum(np.minimum(t1[0], t1[1]), t1[2])
        assert (ids[hit & (m0 > 1e-5)] == 0).all() and (ids[hit & (m1 > 1e-5)] == 1).all()
        assert (np.maximum(m0, m1)[~hit] < 1e-5).all()


def _tri_scene(tri_view):
    return Scene([mesh_np(tri_view, [[0, 1, 2]])], [Instance(0, ident())])


@pytest.mark.parametrize("case", ["inside", "near-crossing"])
def test_paper_stage3_coverage_and_depth_match_float64_rays(oracle_lib, case):
    """A large front-facing triangle (inside the frustum, or crossing the
    near plane): pixels whose float64 ray hits clearly inside it and in front
    of the near plane are covered at depth t (relative 1e-5, 3e-5 at grazing
    incidence), pixels clearly outside are not; the same triangle wound the
    other way covers nothing."""
    O = oracle_lib
    W, H = 96, 64
    near = 0.05
    proj = S.perspective(70, W / H, near, 100.0)
    fx, fy, nv = O.camera_params(proj)
    if case == "inside":
        tri = [[-2.0, -1.5, -4.0], [2.5, -1.0, -6.0], [-0.5, 2.0, -3.0]]
    else:
        # a tilted ground plane just below the camera, two vertices behind
        # it: the near plane cuts it along a slanted screen line, so the
        # clipped polygon's bbox also holds pixels that see the plane closer
        # than the near plane
        tri = [[-3.0, -1.21, 1.0], [3.0, 1.19, 1.0], [0.0, -0.01, -8.0]]
    cam = _cam(np.eye(4), proj, W, H)
    b0, b1, b2, t = _ray_hits64(fx, fy, tri, W, H)
    vis = O.render_paper(O.OracleScene(_tri_scene(tri)), cam, s1_max=128, s2_max=256)
    bmin = np.minimum(np.minimum(b0, b1), b2)
    inside = (bmin > 1e-5) & (t > nv * (1 + 1e-5))
    outside = (bmin < -1e-5) | (t < nv * (1 - 1e-5))
    assert inside.sum() > 300
    if case == "near-crossing":
        assert ((bmin > 1e-5) & (t > 0) & (t < nv * (1 - 1e-5))).sum() > 100
    assert (vis[inside] != O.EMPTY).all()
    assert (vis[outside] == O.EMPTY).all()
    d = O.decode(vis)[0][inside].astype(np.int64)
    tb = np.array([f32bits(x) >> 3 for x in t[inside]], np.int64)
    # one 28-bit step is 2^-20 relative; the FP32 ray cast loses a few more
    # bits at grazing angles (the tilted ground): 32 steps is 3e-5 relative
    assert np.abs(d - tb).max() <= (11 if case == "inside" else 32)
    back = [tri[0], tri[2], tri[1]]
    vb = O.render_paper(O.OracleScene(_tri_scene(back)), cam, s1_max=128, s2_max=256)
    assert (vb == O.EMPTY).all()


def test_paper_stage3_routing_thresholds(oracle_lib):
    """Only triangles past stage 1 (more than s1_max centres) whose visible
    bbox holds more than s2_max pixel centres are ray cast: with s2_max at
    the bbox's count the result is the edge-function one bit for bit, one
    below it the depths come from the ray cast; a triangle within s1_max is
    never ray cast."""
    O = oracle_lib
    W, H = 80, 60
    proj = S.perspective(60, W / H, 0.05, 100.0)
    cam = _cam(np.eye(4), proj, W, H)
    fx, fy, nv = O.camera_params(proj)
    tri = np.array([[-1.1, -0.9, -3.0], [1.3, -0.6, -5.0], [-0.2, 1.2, -2.5]], np.float32)
    osc = O.OracleScene(_tri_scene(tri))
    _, XY, _, _ = O.project(np.eye(4, dtype=np.float32)[:3], np.array([fx, fy, nv], np.float32), W, H, tri)
    lo = np.maximum(-((128 - XY.min(0).astype(np.int64)) // 256), 0)
    hi = np.minimum((XY.max(0).astype(np.int64) - 128) // 256, [W - 1, H - 1])
    K = int((hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1))
    assert K > 128
    edge = O.render(osc, cam)
    np.testing.assert_array_equal(O.render_paper(osc, cam, s1_max=128, s2_max=K), edge)
    ray = O.render_paper(osc, cam, s1_max=128, s2_max=K - 1)
    assert (O.decode(ray)[0] != O.decode(edge)[0]).any()
    np.testing.assert_array_equal(O.render_paper(osc, cam, s1_max=K, s2_max=32), edge)
    # a long thin triangle (76 centres, within s1_max) still leaves stage 1 for its 64-pixel
    # extent, and with s2_max below its count it is ray cast
    W2, H2 = 200, 60
    proj2 = S.perspective(60, W2 / H2, 0.05, 100.0)
    cam2 = _cam(np.eye(4), proj2, W2, H2)
    fx2, fy2, nv2 = O.camera_params(proj2)
    thin = np.array([[-2.6, -0.05, -3.2], [2.5, -0.035, -3.8], [0.1, 0.01, -3.5]], np.float32)
    _, XY2, _, _ = O.project(np.eye(4, dtype=np.float32)[:3], np.array([fx2, fy2, nv2], np.float32), W2, H2, thin)
    lo2 = np.maximum(-((128 - XY2.min(0).astype(np.int64)) // 256), 0)
    hi2 = np.minimum((XY2.max(0).astype(np.int64) - 128) // 256, [W2 - 1, H2 - 1])
    assert int((hi2[0] - lo2[0] + 1) * (hi2[1] - lo2[1] + 1)) <= 128 and XY2[:, 0].max() - XY2[:, 0].min() >= 1 << 14
    osc2 = O.OracleScene(_tri_scene(thin))
    edge2 = O.render(osc2, cam2)
    assert (edge2 != O.EMPTY).sum() > 20
    assert (O.decode(O.render_paper(osc2, cam2, s1_max=128, s2_max=32))[0] != O.decode(edge2)[0]).any()


def test_snap_ties_round_to_even(oracle_lib):
    """R1 snaps with round-half-to-even: a vertex whose 256 X falls exactly
    on k + 1/2 goes to the even neighbour (camera with fx = fy = 1, depth 1
    and a 2 x 2 screen make 256 X = 256 (vx + 1) exact)."""
    O = oracle_lib
    cp = O.camera_params(S.perspective(90.0, 1.0, 0.01, 100.0))
    assert tuple(cp[:2]) == (1.0, 1.0)
    mv = np.eye(4, dtype=np.float32)[:3]
    k = np.arange(250, 262)
    for frac in (0.5, 0.25, 0.75):
        v = ((k + frac) / 256.0 - 1.0).astype(np.float32)
        assert np.array_equal((v.astype(np.float64) + 1.0) * 256.0, k + frac)      # the ties are exact
        pts = np.stack([v, v[::-1], -np.ones_like(v)], 1).astype(np.float32)
        _, XY, _, inside = O.project(mv, cp, 2, 2, pts)
        assert inside.all()
        np.testing.assert_array_equal(XY[:, 0], np.rint(k + frac))          # numpy rint: half to even
        np.testing.assert_array_equal(XY[:, 1], np.rint(k[::-1] + frac))


# ------------------------------------------------- textured resolve (R17) ---
def _coord_texture(L):
    """Mip chain of side 2^L (L <= 8) whose texel (column c, row r) of level l
    holds (c, r, l, 255): the resolved RGBA8 names the texel that was read."""
    out = []
    for l in range(L + 1):
        s = 1 << (L - l)
        r, c = np.meshgrid(np.arange(s), np.arange(s), indexing="ij")
        out.append(np.stack([c, r, np.full_like(c, l), np.full_like(c, 255)], axis=2).reshape(-1))
    return np.concatenate(out).astype(np.uint8)


def _plane_quad(a, b, D, u_span, v_span):
    """Camera-facing rectangle |x| <= a, |y| <= b at view depth D (camera at
    the origin looking down -z), front face towards the camera, texture
    coordinates u = (x + a) / (2a) * u_span, v = (y + b) / (2b) * v_span."""
    pos = np.array([[-a, -b, -D], [a, -b, -D], [-a, b, -D], [a, b, -D]], np.float64)
    uv = np.stack([(pos[:, 0] + a) / (2 * a) * u_span, (pos[:, 1] + b) / (2 * b) * v_span], 1)
    return pos, [[0, 1, 2], [2, 1, 3]], uv.astype(np.float32)


def test_mip_level_of_a_camera_facing_plane(oracle_lib):
    """Section 4.4: the four rays through the pixel and its right, top and
    top-right neighbours meet a camera-facing plane at D / (W fx) and
    D / (H fy) apart; with the texture repeated `span` times over the 2a x 2b
    rectangle the footprint is F = 2^L span max(D / (W fx a), D / (H fy b))
    level-0 texels, the same for every pixel, and the level is floor(log2 F)
    clamped to 0..L.  Depth and span are chosen with log2 F 0.6 above an
    integer (round would pick the next level), plus one case below a texel
    per pixel (level 0) and one beyond the coarsest level (clamped).  The sampled texel is the float64 floor(u s), floor(v s)
    of the pixel's own uv, s the level's side, away from texel boundaries."""
    O = oracle_lib
    W, H, L = 64, 48, 8
    proj = S.perspective(60.0, W / H, 0.01, 1000.0)
    cp = O.camera_params(proj.astype(np.float32)).astype(np.float64)
    fx, fy = cp[0], cp[1]
    a, b = 1.5, 0.5
    tex = _coord_texture(L)
    seen = set()
    c = 2 ** L * max(1 / (W * fx * a), 1 / (H * fy * b))     # F = c D span
    targets = [0.3] + [2 ** (k + 0.6) for k in range(L)] + [2 ** (L + 1.5)]
    for k, Ft in enumerate(targets):
        D = 0.8 * (1 + k % 3)
        span = Ft / (c * D)
        F = c * D * span
        want = 0 if F < 1 else min(int(math.floor(math.log2(F))), L)
        pos, idx, uv = _plane_quad(a, b, D, span, span)
        sc = Scene([mesh_np(pos, idx)], [Instance(0, ident())])
        cam = _cam(np.eye(4), proj, W, H)
        osc = O.OracleScene(sc)
        vis = O.render(osc, cam)
        cov = vis != O.EMPTY
        assert cov.sum() >= 1
        _, rgba8, lev = O.resolve_textured(osc, cam, vis, [(uv, tex, L)])
        assert (lev[cov] == want).all(), (D, want, np.unique(lev[cov]))
        assert (lev[~cov] == 255).all()
        seen.add(want)
        # the texel of the pixel's own uv, from a float64 ray-plane hit
        ys, xs = np.nonzero(cov)
        ndx, ndy = (2 * xs + 1) / W - 1, (2 * ys + 1) / H - 1
        px, py = D * ndx / fx, D * ndy / fy
        u, v = (px + a) / (2 * a) * span, (py + b) / (2 * b) * span
        side = 1 << (L - want)
        cu, cv = u * side, v * side
        clear = (np.abs(cu - np.round(cu)) > 1e-3) & (np.abs(cv - np.round(cv)) > 1e-3)
        got = rgba8[ys, xs]
        assert clear.sum() > 0.5 * len(xs)
        np.testing.assert_array_equal(got[clear, 0], np.clip(np.floor(cu[clear]), 0, side - 1))
        np.testing.assert_array_equal(got[clear, 1], np.clip(np.floor(cv[clear]), 0, side - 1))
        assert (got[:, 2] == want).all()
    assert seen == set(range(L + 1))


def test_mip_level_of_a_tilted_plane_matches_float64(oracle_lib):
    """A plane seen at a grazing angle (the footprint grows quickly towards
    the horizon and differs along x and y): per pixel, the four float64
    ray-plane hits give the uv samples, their bounding box the footprint and
    floor(log2 F) the level; the oracle's level must agree wherever log2 F
    is at least 1e-3 from an integer, and its texel wherever u s and v s are
    at least 1e-3 from a texel edge."""
    O = oracle_lib
    W, H, L = 96, 64, 8
    tex = _coord_texture(L)
    view = S.look_at((0.3, 0.35, 2.2), (0.55, 0.0, -0.4))
    proj = S.perspective(70.0, W / H, 0.01, 100.0)
    cam = _cam(view, proj, W, H)
    pos = np.array([[-2.0, 0.0, 3.0], [3.0, 0.0, 3.0], [-2.0, 0.0, -6.0], [3.0, 0.0, -6.0]])
    idx = [[0, 1, 2], [2, 1, 3]]
    # u along x over 5 units, v along -z over 9 units, rotated texture: u and v each mix x and z
    uvm = np.array([[0.15, -0.05], [0.02, 0.09]])
    uv = ((pos[:, [0, 2]] - [-2.0, 3.0]) @ uvm.T).astype(np.float32)
    sc = Scene([mesh_np(pos, idx)], [Instance(0, ident())])
    osc = O.OracleScene(sc)
    vis = O.render(osc, cam)
    cov = vis != O.EMPTY
    _, rgba8, lev = O.resolve_textured(osc, cam, vis, [(uv, tex, L)])
    cp = O.camera_params(np.asarray(proj, np.float32)).astype(np.float64)
    V = np.asarray(view, np.float64)
    Vi = np.linalg.inv(V)
    eye = Vi[:3, 3]
    ys, xs = np.nonzero(cov)

    def hit_uv(x, y):
        ndx, ndy = (2 * x + 1) / W - 1, (2 * y + 1) / H - 1
        d = Vi[:3, :3] @ np.stack([ndx / cp[0], ndy / cp[1], -np.ones_like(ndx)])
        t = -eye[1] / d[1]
        p = eye[:, None] + d * t
        return uvm @ (p[[0, 2]] - np.array([[-2.0], [3.0]]))

    s = [hit_uv(xs + (q & 1), ys + (q >> 1)) for q in range(4)]
    us, vs = np.stack([q[0] for q in s]), np.stack([q[1] for q in s])
    F = np.maximum(us.max(0) - us.min(0), vs.max(0) - vs.min(0)) * 2 ** L
    lg = np.log2(F)
    want = np.where(F < 1, 0, np.minimum(np.floor(lg), L)).astype(int)
    clear = np.abs(lg - np.round(lg)) > 1e-3
    assert clear.mean() > 0.95 and len(np.unique(want)) >= 4
    np.testing.assert_array_equal(lev[ys, xs][clear], want[clear])
    side = (1 << (L - lev[ys, xs].astype(int))).astype(np.float64)
    cu, cv = s[0][0] * side, s[0][1] * side
    ok = clear & (np.abs(cu - np.round(cu)) > 1e-3) & (np.abs(cv - np.round(cv)) > 1e-3)
    assert ok.mean() > 0.9
    got = rgba8[ys, xs].astype(int)
    np.testing.assert_array_equal(got[ok, 0], np.clip(np.floor(cu[ok]), 0, side[ok] - 1))
    np.testing.assert_array_equal(got[ok, 1], np.clip(np.floor(cv[ok]), 0, side[ok] - 1))


def test_textured_resolve_without_textures_is_the_plain_resolve(oracle_lib):
    """Meshes without a texture keep the vertex colours of the plain resolve
    (Section 4.4), and report no level."""
    O = oracle_lib
    sc = S.scene_small(n=32, W=80, H=60)
    cam = sc.cameras[0]
    osc = O.OracleScene(sc)
    vis = O.render(osc, cam)
    f, e8 = O.resolve(osc, cam, vis)
    g, g8, lev = O.resolve_textured(osc, cam, vis, [None] * len(sc.meshes))
    np.testing.assert_array_equal(g, f)
    np.testing.assert_array_equal(g8, e8)
    assert (lev == 255).all()
