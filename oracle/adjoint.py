"""FP64 oracle of the differentiable interpolation step (numpy).

TEST INFRASTRUCTURE ONLY (see oracle.py).

With the visibility buffer held fixed, every covered pixel p shows one
triangle (v0, v1, v2) of the mesh, in view space v_k = M p_k + t.  Following
Section 4.4 (shading in world/view space from the barycentrics of the pixel
ray and the triangle), the pixel ray through the pixel centre is
r = (ndx / fx, ndy / fy, -1) with ndx = (2x + 1) / W - 1, and the image is

    I(p) = sum_k b_k(p) c_k,     L = sum_p sum_ch (I - T)^2.

``forward64`` evaluates b with the same Moeller-Trumbore steps the FP32
oracle uses, in float64.  ``adjoint64`` is the exact derivative: with
D_k = r . (v_{k+1} x v_{k+2}) and S = D_0 + D_1 + D_2 the barycentrics are
b_k = D_k / S, so for g = dL/dI, gamma_k = g . c_k and gbar = sum_k b_k gamma_k

    dL/dc_k   = sum_p g(p) b_k(p)
    dL/dv_j   = (1/S) [ (gamma_{j-1} - gbar) (v_{j+1} x r) + (gamma_{j+1} - gbar) (r x v_{j-1}) ]
    dL/dpos   = M^T dL/dv          (accumulated per vertex)

Discontinuities of the visibility (edges, occlusion) are not differentiated.
"""
from __future__ import annotations

import numpy as np

ID_MASK = np.uint64((1 << 36) - 1)
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def pixel_triangles(vis: np.ndarray, base_id: int, T: int) -> np.ndarray:
    """Triangle index within the mesh per pixel (-1 where the pixel is empty
    or shows another instance), for a mesh instance whose ids start at base_id."""
    v = np.asarray(vis, np.uint64).reshape(-1)
    ids = (v & ID_MASK).astype(np.int64)
    t = ids - int(base_id)
    ok = (v != EMPTY) & (t >= 0) & (t < T)
    return np.where(ok, t, -1)


def _rays(W: int, H: int, fx: float, fy: float) -> np.ndarray:
    x = np.arange(W, dtype=np.float64)
    y = np.arange(H, dtype=np.float64)
    ndx = (2.0 * x + 1.0) / W - 1.0
    ndy = (2.0 * y + 1.0) / H - 1.0
    r = np.empty((H, W, 3))
    r[..., 0] = (ndx / fx)[None, :]
    r[..., 1] = (ndy / fy)[:, None]
    r[..., 2] = -1.0
    return r.reshape(-1, 3)


def _gather(pos, idx, mv, tri):
    M = np.asarray(mv, np.float64).reshape(3, 4)
    P = np.asarray(pos, np.float64)
    I = np.asarray(idx, np.int64).reshape(-1, 3)[tri]          # (n, 3)
    v = [P[I[:, k]] @ M[:, :3].T + M[:, 3] for k in range(3)]
    return I, v, M


def forward64(pos, idx, col, mv, fx, fy, W, H, tri):
    """I (H*W, C) in float64; b (n, 3) for the covered pixels; covered mask."""
    tri = np.asarray(tri).reshape(-1)
    cov = tri >= 0
    r = _rays(W, H, float(fx), float(fy))[cov]
    I, v, _ = _gather(pos, idx, mv, tri[cov])
    e1 = v[1] - v[0]
    e2 = v[2] - v[0]
    tv = -v[0]
    pv = np.cross(r, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    u = np.einsum("ij,ij->i", tv, pv) / det
    qv = np.cross(tv, e1)
    w = np.einsum("ij,ij->i", r, qv) / det
    b = np.stack([1.0 - u - w, u, w], axis=1)
    c = np.asarray(col, np.float64)
    out = np.zeros((W * H, c.shape[1]))
    out[cov] = sum(b[:, k:k + 1] * c[I[:, k]] for k in range(3))
    return out, b, cov


def barycentrics_closed_form(pos, idx, mv, fx, fy, W, H, tri):
    """b_k = D_k / S (the triple-product closed form), for pinning forward64."""
    tri = np.asarray(tri).reshape(-1)
    cov = tri >= 0
    r = _rays(W, H, float(fx), float(fy))[cov]
    _, v, _ = _gather(pos, idx, mv, tri[cov])
    D = np.stack([np.einsum("ij,ij->i", r, np.cross(v[(k + 1) % 3], v[(k + 2) % 3])) for k in range(3)], 1)
    return D / D.sum(1, keepdims=True)


def loss_at_pixels64(pos, idx, col, mv, fx, fy, W, H, pix, tri_pix, target_pix) -> float:
    """L restricted to the listed pixels (flat indices y*W+x showing triangle
    tri_pix): the same per-pixel formula as forward64, for local finite
    differences where a vertex moves only the pixels of its triangles."""
    pix = np.asarray(pix)
    x = (pix % W).astype(np.float64)
    y = (pix // W).astype(np.float64)
    r = np.stack([((2.0 * x + 1.0) / W - 1.0) / fx, ((2.0 * y + 1.0) / H - 1.0) / fy, -np.ones_like(x)], 1)
    I, v, _ = _gather(pos, idx, mv, np.asarray(tri_pix))
    e1, e2, tv = v[1] - v[0], v[2] - v[0], -v[0]
    pv = np.cross(r, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    u = np.einsum("ij,ij->i", tv, pv) / det
    w = np.einsum("ij,ij->i", r, np.cross(tv, e1)) / det
    c = np.asarray(col, np.float64)
    out = (1.0 - u - w)[:, None] * c[I[:, 0]] + u[:, None] * c[I[:, 1]] + w[:, None] * c[I[:, 2]]
    d = out - np.asarray(target_pix, np.float64)
    return float((d * d).sum())


def loss64(pos, idx, col, mv, fx, fy, W, H, tri, target) -> float:
    out, _, _ = forward64(pos, idx, col, mv, fx, fy, W, H, tri)
    d = out - np.asarray(target, np.float64).reshape(out.shape)
    return float((d * d).sum())


def adjoint64(pos, idx, col, mv, fx, fy, W, H, tri, grad_img):
    """Exact gradients (dL/dcol (V, C), dL/dpos (V, 3)) in float64 for the
    pixel gradient grad_img = dL/dI (H*W, C)."""
    tri = np.asarray(tri).reshape(-1)
    cov = tri >= 0
    r = _rays(W, H, float(fx), float(fy))[cov]
    I, v, M = _gather(pos, idx, mv, tri[cov])
    c = np.asarray(col, np.float64)
    g = np.asarray(grad_img, np.float64).reshape(W * H, -1)[cov]
    D = np.stack([np.einsum("ij,ij->i", r, np.cross(v[(k + 1) % 3], v[(k + 2) % 3])) for k in range(3)], 1)
    S = D.sum(1)
    b = D / S[:, None]
    gam = np.stack([np.einsum("ij,ij->i", g, c[I[:, k]]) for k in range(3)], 1)
    gbar = (b * gam).sum(1)
    V = np.asarray(pos).shape[0]
    dcol = np.zeros((V, c.shape[1]))
    dpos = np.zeros((V, 3))
    for k in range(3):
        np.add.at(dcol, I[:, k], g * b[:, k:k + 1])
    for j in range(3):
        jm, jp = (j + 2) % 3, (j + 1) % 3
        dv = ((gam[:, jm] - gbar)[:, None] * np.cross(v[jp], r)
              + (gam[:, jp] - gbar)[:, None] * np.cross(r, v[jm])) / S[:, None]
        np.add.at(dpos, I[:, j], dv @ M[:, :3])
    return dcol, dpos
