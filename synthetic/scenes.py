"""Seeded scene generators (heightfields, displaced spheres, instances, cameras).

The paper evaluates on photogrammetry scans (Sponza, Lantern, Komainu Kobe,
Venice, Zorah; Section 5, Table 1) that are not available here.  These
generators stand in for them with the same structure: dense, opaque, indexed
triangle meshes with uint32 indices, FP32 xyz positions, RGBA8 vertex colours,
and row-major vertex/triangle order (the locality a mesh optimizer produces).

Determinism across devices: all real arithmetic is float64 using only
+, -, *, / and floor (each a correctly rounded IEEE operation executed as its
own tensor op, so no fused multiply-add can occur), and the lattice hash uses
int64 arithmetic whose intermediate values stay below 2**62.  The same call on
CPU and GPU therefore yields bit-identical tensors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

_M32 = 0xFFFFFFFF


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclass
class Mesh:
    pos: torch.Tensor             # (V, 3) float32, xyz
    idx: torch.Tensor             # (T, 3) int32 holding uint32 vertex indices
    rgba8: Optional[torch.Tensor] = None   # (V, 4) uint8
    aabb: Optional[tuple] = None  # ((xmin, ymin, zmin), (xmax, ymax, zmax)) bound of pos

    @property
    def V(self) -> int:
        return int(self.pos.shape[0])

    @property
    def T(self) -> int:
        return int(self.idx.shape[0])


@dataclass
class Instance:
    mesh: int
    model: np.ndarray             # (4, 4) float32, row-major affine (last row 0 0 0 1)


@dataclass
class Camera:
    view: np.ndarray              # (4, 4) float32, row-major affine world->view
    proj: np.ndarray              # (4, 4) float32, row-major symmetric perspective
    W: int
    H: int


@dataclass
class Scene:
    meshes: List[Mesh]
    instances: List[Instance]
    cameras: List[Camera] = field(default_factory=list)

    @property
    def total_triangles(self) -> int:
        return sum(self.meshes[i.mesh].T for i in self.instances)


# ----------------------------------------------------------------------------
# value noise
# ----------------------------------------------------------------------------
def _hash32(x: torch.Tensor) -> torch.Tensor:
    """PCG-style 32-bit integer hash on int64 tensors holding values < 2**32."""
    x = (x * 747796405 + 2891336453) & _M32
    w = (((x >> ((x >> 28) + 4)) ^ x) * 277803737) & _M32
    return (w >> 22) ^ w


def _lattice(ix: torch.Tensor, iz: torch.Tensor, salt: int) -> torch.Tensor:
    """Hashed lattice value in [0, 1) (24-bit, exact in float64)."""
    h = _hash32(((iz + 4096) & _M32) ^ salt)
    h = _hash32(((ix + 4096) & _M32) ^ h)
    return (h & 0xFFFFFF).to(torch.float64) / 16777216.0


def _smooth(t: torch.Tensor) -> torch.Tensor:
    t2 = t * t
    a = 3.0 - (t * 2.0)
    return t2 * a


def value_noise(x: torch.Tensor, z: torch.Tensor, seed: int, octaves: int = 6,
                base_freq: int = 8, amplitude: float = 0.2) -> torch.Tensor:
    """Fractal value noise, float64.

    ``octaves`` octaves of smoothstep-bilinear hashed lattice noise; octave o
    has frequency base_freq * 2**o and weight 0.5**o; the weighted sum is
    normalised so that its range is [0, amplitude).
    """
    x = x.to(torch.float64)
    z = z.to(torch.float64)
    total = torch.zeros_like(x)
    wsum = 0.0
    seed_h = int(_hash32(torch.tensor([seed & _M32], dtype=torch.int64))[0])
    for o in range(octaves):
        f = float(base_freq * (2 ** o))
        px = x * f
        pz = z * f
        fx = torch.floor(px)
        fz = torch.floor(pz)
        tx = _smooth(px - fx)
        tz = _smooth(pz - fz)
        ix = fx.to(torch.int64)
        iz = fz.to(torch.int64)
        salt = (seed_h ^ (o * 0x9E3779B1)) & _M32
        v00 = _lattice(ix, iz, salt)
        v10 = _lattice(ix + 1, iz, salt)
        v01 = _lattice(ix, iz + 1, salt)
        v11 = _lattice(ix + 1, iz + 1, salt)
        top = v00 + (tx * (v10 - v00))
        bot = v01 + (tx * (v11 - v01))
        v = top + (tz * (bot - top))
        w = 0.5 ** o
        total = total + (v * w)
        wsum += w
    return total * (amplitude / wsum)


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
def _grid_indices(nu: int, nv: int, device) -> torch.Tensor:
    """Two triangles per cell, row-major; CCW when seen from the +y side.

    Vertex (i, j) sits at index j * (nu + 1) + i; cell (i, j) yields
    (v00, v01, v10) and (v10, v01, v11).
    """
    i = torch.arange(nu, device=device, dtype=torch.int64)
    j = torch.arange(nv, device=device, dtype=torch.int64)
    v00 = (j[:, None] * (nu + 1) + i[None, :]).reshape(-1)
    v10 = v00 + 1
    v01 = v00 + (nu + 1)
    v11 = v01 + 1
    tri = torch.stack([v00, v01, v10, v10, v01, v11], dim=1).reshape(-1, 3)
    return tri.to(torch.int32)


def _ramp_rgba8(h: torch.Tensor, amplitude: float) -> torch.Tensor:
    t = torch.clamp(h / amplitude, 0.0, 1.0)
    r = torch.round(t * 255.0)
    g = torch.round((1.0 - t) * 180.0 + 40.0)
    b = torch.round((1.0 - t) * 90.0 + t * 160.0)
    a = torch.full_like(r, 255.0)
    return torch.stack([r, g, b, a], dim=1).to(torch.uint8)


def heightfield_mesh(n: int, seed: int, device="cpu", amplitude: float = 0.2,
                     colours: bool = True) -> Mesh:
    """n x n cells over [0,1]^2 in xz with y = value noise height; grid spacing 1/n."""
    k = torch.arange(n + 1, device=device, dtype=torch.float64) / float(n)
    z = k[:, None].expand(n + 1, n + 1).reshape(-1)
    x = k[None, :].expand(n + 1, n + 1).reshape(-1)
    h = value_noise(x, z, seed, amplitude=amplitude)
    pos = torch.stack([x, h, z], dim=1).to(torch.float32)
    idx = _grid_indices(n, n, device)
    rgba = _ramp_rgba8(h, amplitude) if colours else None
    aabb = ((0.0, 0.0, 0.0), (1.0, amplitude, 1.0))
    return Mesh(pos=pos, idx=idx, rgba8=rgba, aabb=aabb)


def grid_uv(n: int, device="cpu") -> torch.Tensor:
    """Texture coordinates of a heightfield of n x n cells: vertex (i, j)
    (index j (n + 1) + i) gets (u, v) = (i / n, j / n), its x and z in the
    unit square, as (V, 2) float32."""
    k = torch.arange(n + 1, device=device, dtype=torch.float64) / float(n)
    v = k[:, None].expand(n + 1, n + 1).reshape(-1)
    u = k[None, :].expand(n + 1, n + 1).reshape(-1)
    return torch.stack([u, v], dim=1).to(torch.float32)


def texture_mip_chain(log2_size: int, seed: int, device="cpu") -> torch.Tensor:
    """A seeded square RGBA8 texture of side 2^log2_size with its full mip
    chain, flat: level l (side 2^(log2_size - l)) follows level l - 1, each
    row-major with row 0 at v = 0.  Level 0 holds hashed random RGB bytes
    (alpha 255) on 8 x 8 texel blocks modulated by a per-texel hash, so that
    every level differs; each coarser level is the 2 x 2 box average of the
    one before, (a + b + c + d + 2) >> 2 per channel."""
    side = 1 << log2_size
    j = torch.arange(side, device=device, dtype=torch.int64)
    jj, ii = j[:, None].expand(side, side), j[None, :].expand(side, side)
    blk = (jj >> 3) * 65536 + (ii >> 3)
    tex = []
    for ch, salt in enumerate((11, 23, 37)):
        coarse = _hash32(blk * 7 + salt + seed * 131) & 0xFF
        fine = _hash32((jj * side + ii) * 5 + salt * 3 + seed) & 0x3F
        tex.append(((coarse * 3 + fine * 4) >> 2).clamp(0, 255))
    tex.append(torch.full_like(tex[0], 255))
    lev = torch.stack(tex, dim=2)                      # (side, side, 4) int64
    out = [lev.reshape(-1)]
    while lev.shape[0] > 1:
        lev = (lev[0::2, 0::2] + lev[0::2, 1::2] + lev[1::2, 0::2] + lev[1::2, 1::2] + 2) >> 2
        out.append(lev.reshape(-1))
    return torch.cat(out).to(torch.uint8)


def sphere_mesh(n: int, seed: int, device="cpu", amplitude: float = 0.2) -> Mesh:
    """UV sphere of n latitude x 2n longitude cells with radius 1 + noise.

    Unlike the heightfields this uses sin/cos, whose last bit may differ
    between devices: build it once and hand the same tensors to every side.

    The seam column and the pole rows repeat identical positions so the
    surface is closed; triangles face outward (CCW from outside).  The
    pole cells yield zero-area triangles, as real scans often contain.
    """
    nl, nn = n, 2 * n
    lat = torch.arange(nl + 1, device=device, dtype=torch.float64) / float(nl)
    lon = torch.arange(nn + 1, device=device, dtype=torch.float64) / float(nn)
    v = lat[:, None].expand(nl + 1, nn + 1).reshape(-1)
    u = lon[None, :].expand(nl + 1, nn + 1).reshape(-1)
    u_wrapped = torch.where(u >= 1.0, torch.zeros_like(u), u)
    pole = (v <= 0.0) | (v >= 1.0)
    u_eval = torch.where(pole, torch.zeros_like(u), u_wrapped)
    r = 1.0 + value_noise(u_eval * 4.0, v * 2.0, seed, amplitude=amplitude)
    theta = v * math.pi
    phi = u_wrapped * (2.0 * math.pi)
    st = torch.sin(theta)
    x = r * st * torch.cos(phi)
    y = r * torch.cos(theta)
    z = r * st * torch.sin(phi)
    x = torch.where(pole, torch.zeros_like(x), x)
    z = torch.where(pole, torch.zeros_like(z), z)
    pos = torch.stack([x, y, z], dim=1).to(torch.float32)
    # grid rows run from the north pole (v=0, +y) southwards; with u growing
    # towards +z at phi=90deg, the (v00, v01, v10) order faces outward.
    idx = _grid_indices(nn, nl, device)
    idx = idx[:, [0, 2, 1]].contiguous()
    rgba = _ramp_rgba8(r - 1.0, amplitude)
    a = 1.0 + amplitude
    return Mesh(pos=pos, idx=idx, rgba8=rgba, aabb=((-a, -a, -a), (a, a, a)))


def ground_mesh(half: float = 100.0, y: float = -0.05, device="cpu") -> Mesh:
    """Two large CCW-from-above triangles spanning [-half, half]^2 at height y."""
    pos = torch.tensor([[-half, y, -half], [half, y, -half],
                        [-half, y, half], [half, y, half]], dtype=torch.float32, device=device)
    # (0: -x-z, 1: +x-z, 2: -x+z, 3: +x+z); CCW from +y: (0, 2, 1), (1, 2, 3)
    idx = torch.tensor([[0, 2, 1], [1, 2, 3]], dtype=torch.int32, device=device)
    rgba = torch.tensor([[90, 90, 96, 255]] * 4, dtype=torch.uint8, device=device)
    return Mesh(pos=pos, idx=idx, rgba8=rgba, aabb=((-half, y, -half), (half, y, half)))


# ----------------------------------------------------------------------------
# cameras and transforms
# ----------------------------------------------------------------------------
def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Right-handed world->view matrix (camera looks down -z), row-major float32."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, np.asarray(up, np.float64))
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[0, 3], m[1, 3], m[2, 3] = -s @ eye, -u @ eye, f @ eye
    return m.astype(np.float32)


def perspective(fovy_deg: float, aspect: float, near: float, far: Optional[float] = None) -> np.ndarray:
    """OpenGL-style symmetric perspective matrix, row-major float32 (far=None: infinite)."""
    f = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    p = np.zeros((4, 4))
    p[0, 0] = f / aspect
    p[1, 1] = f
    if far is None:
        p[2, 2], p[2, 3] = -1.0 + 1e-7, -2.0 * near
    else:
        p[2, 2] = (far + near) / (near - far)
        p[2, 3] = 2.0 * far * near / (near - far)
    p[3, 2] = -1.0
    return p.astype(np.float32)


def _translate(t) -> np.ndarray:
    m = np.eye(4, dtype=np.float64)
    m[:3, 3] = t
    return m


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
def scene_small(device="cpu", n: int = 256, W: int = 512, H: int = 512) -> Scene:
    """Heightfield of n x n cells (seed 1) plus two ground triangles at y=-0.05
    spanning +-100 that cross the near plane; 60 deg camera at (0.5, 0.8, -0.3)
    looking at (0.5, 0, 0.5) (45 deg pitch), near 1e-3."""
    hf = heightfield_mesh(n, seed=1, device=device)
    gr = ground_mesh(device=device)
    eye = (0.5, 0.8, -0.3)
    cam = Camera(look_at(eye, (0.5, 0.0, 0.5)), perspective(60.0, W / H, 1e-3, 1000.0), W, H)
    inst = [Instance(0, np.eye(4, dtype=np.float32)), Instance(1, np.eye(4, dtype=np.float32))]
    return Scene([hf, gr], inst, [cam])


def camera_unique_pose(k: int, W: int, H: int, seed_base: int = 100) -> Camera:
    """Pose k of the 100M-triangle heightfield: distance to a random target
    log-uniform in [0.01, 1.5], pitch in [30, 60] deg, yaw uniform."""
    rng = np.random.default_rng(seed_base + k)
    tx, tz = rng.uniform(0.2, 0.8, size=2)
    th = float(value_noise(torch.tensor([tx]), torch.tensor([tz]), seed_base)[0])
    dist = math.exp(rng.uniform(math.log(0.01), math.log(1.5)))
    pitch = math.radians(rng.uniform(30.0, 60.0))
    yaw = rng.uniform(0.0, 2.0 * math.pi)
    tgt = np.array([tx, th, tz])
    d = np.array([math.cos(pitch) * math.sin(yaw), math.sin(pitch), math.cos(pitch) * math.cos(yaw)])
    eye = tgt + dist * d
    near = max(1e-4, 1e-3 * dist)
    return Camera(look_at(eye, tgt), perspective(60.0, W / H, near, 100.0), W, H)


def scene_unique(device="cpu", n: int = 7072, seed: int = 100) -> Scene:
    """One heightfield of n x n cells (default ~100M triangles)."""
    hf = heightfield_mesh(n, seed=seed, device=device)
    return Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))], [])


def camera_billion(W: int = 3840, H: int = 2160, tiles: int = 8) -> Camera:
    """Overview of the tiles x tiles terrain from above its near edge; the
    frustum leaves out 18 of the 64 tiles (28%) of the 8 x 8 layout."""
    s = tiles / 8.0
    eye = (4.0 * s, 2.6 * s, 1.0 * s)
    tgt = (4.0 * s, 0.0, 4.0 * s)
    return Camera(look_at(eye, tgt), perspective(50.0, W / H, 1e-2, 100.0), W, H)


def scene_billion(device="cpu", tiles: int = 8, n: int = 4096, colours: bool = True,
                  only: Optional[List[int]] = None) -> Scene:
    """tiles x tiles heightfield tiles of n x n cells (seeds 200 + k), tile k =
    (i, j) translated to (i, 0, j).  ``only`` restricts which tiles get
    geometry (the others are empty placeholders with the right triangle count
    held in ``Mesh.idx`` shape only when generated); used to stream the oracle
    one tile at a time."""
    meshes, inst = [], []
    for k in range(tiles * tiles):
        i, j = k % tiles, k // tiles
        if only is None or k in only:
            meshes.append(heightfield_mesh(n, seed=200 + k, device=device, colours=colours))
        else:
            meshes.append(None)
        inst.append(Instance(k, _translate((float(i), 0.0, float(j))).astype(np.float32)))
    return Scene(meshes, inst, [])


def batched_mesh_specs(n_meshes: int = 256, tmin: float = 1e4, tmax: float = 2e7, seed: int = 300) -> list:
    """The meshes of the many-mesh workload without building them: per mesh
    (kind, n, seed, T) -- even ones heightfields of n x n cells (T = 2 n^2),
    odd ones spheres of n x 2n cells (T = 4 n^2) -- with T drawn
    log-uniform in [tmin, tmax]."""
    rng = np.random.default_rng(seed)
    tcount = np.exp(rng.uniform(math.log(tmin), math.log(tmax), size=n_meshes))
    out = []
    for m in range(n_meshes):
        if m % 2 == 0:
            n = max(2, int(round(math.sqrt(tcount[m] / 2.0))))
            out.append(("heightfield", n, seed + 1 + m, 2 * n * n))
        else:
            n = max(2, int(round(math.sqrt(tcount[m] / 4.0))))
            out.append(("sphere", n, seed + 1 + m, 4 * n * n))
    return out


def batched_mesh(spec, device="cpu") -> Mesh:
    kind, n, mseed, _ = spec
    return heightfield_mesh(n, seed=mseed, device=device) if kind == "heightfield" else \
        sphere_mesh(n, seed=mseed, device=device)


def scene_batched(device="cpu", n_meshes: int = 256, n_instances: int = 10000,
                  tmin: float = 1e4, tmax: float = 2e7, area: float = 200.0,
                  views=((3840, 2160), (3840, 2160), (1920, 1080), (1920, 1080)),
                  seed: int = 300, only=None) -> Scene:
    """Many meshes of log-uniform size, many rigid+uniform-scale instances,
    several views.  ``only`` restricts which meshes are built (the others are
    None placeholders; their triangle counts come from batched_mesh_specs)."""
    rng = np.random.default_rng(seed)
    rng.uniform(size=n_meshes)                       # the triangle counts (batched_mesh_specs)
    specs = batched_mesh_specs(n_meshes, tmin, tmax, seed)
    meshes = [batched_mesh(sp, device) if only is None or m in only else None for m, sp in enumerate(specs)]
    inst = []
    for k in range(n_instances):
        mesh = k if k < n_meshes else int(rng.integers(0, n_meshes))
        t = (rng.uniform(-area / 2, area / 2), 0.0, rng.uniform(-area / 2, area / 2))
        rot = _random_rotation(rng)
        sc = rng.uniform(0.1, 10.0)
        m4 = np.eye(4)
        m4[:3, :3] = rot * sc
        m4[:3, 3] = t
        inst.append(Instance(mesh, m4.astype(np.float32)))
    cams = []
    for v, (W, H) in enumerate(views):
        ang = 2.0 * math.pi * v / len(views) + 0.3
        eye = (0.7 * area * math.cos(ang), 0.35 * area, 0.7 * area * math.sin(ang))
        tgt = (0.1 * area * math.cos(ang + 1.0), 0.0, 0.1 * area * math.sin(ang + 1.0))
        cams.append(Camera(look_at(eye, tgt), perspective(60.0, W / H, 0.05, 2000.0), W, H))
    return Scene(meshes, inst, cams)


def scene_room(device="cpu", W: int = 300, H: int = 200) -> Scene:
    """The camera inside a closed 6 x 4 x 8 box whose 12 triangles face
    inwards: every face crosses the near plane or the guard band and covers a
    large part of the screen (a stage-3 workload).  Two cameras: W x H at 80
    degrees near the centre, and a square 100-degree view from a corner."""
    p = np.array([[x, y, z] for x in (-3, 3) for y in (-2, 2) for z in (-4, 4)], np.float32)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    idx = []
    for a, b, c, d in quads:          # wound to face the inside
        idx += [[a, c, b], [a, d, c]]
    col = np.tile(np.array([[200, 120, 40, 255]], np.uint8), (8, 1))
    m = Mesh(pos=torch.tensor(p, device=device), idx=torch.tensor(np.array(idx, np.int32), device=device),
             rgba8=torch.tensor(col, device=device))
    cams = [Camera(look_at((0.3, 0.1, 0.2), (1.0, -0.4, -2.0)), perspective(80, W / H, 0.05, 100.0), W, H),
            Camera(look_at((-2.5, 1.5, 3.5), (2.0, -1.0, -3.0)), perspective(100, 1.0, 0.01, 100.0), H, H)]
    return Scene([m], [Instance(0, np.eye(4, dtype=np.float32))], cams)


def scene_differentiable(device="cpu", n: int = 1448, W: int = 1024, H: int = 1024,
                         seed: int = 500) -> tuple:
    """Heightfield of n x n cells, FP32 RGB per-vertex colours from height.
    Returns (scene, colours (V,3) float32)."""
    hf = heightfield_mesh(n, seed=seed, device=device)
    h = hf.pos[:, 1].to(torch.float64)
    t = torch.clamp(h / 0.2, 0.0, 1.0)
    col = torch.stack([t, 1.0 - t, (t * 0.5) + 0.25], dim=1).to(torch.float32)
    cam = Camera(look_at((0.5, 1.1, -0.25), (0.5, 0.0, 0.55)), perspective(55.0, W / H, 1e-2, 100.0), W, H)
    return Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))], [cam]), col


def target_colour_noise(V: int, channels: int = 3, sigma: float = 0.05,
                        seed: int = 501) -> torch.Tensor:
    """N(0, sigma) per vertex and channel (float32, CPU): the perturbation of
    the vertex colours that renders the target image of the differentiable
    workload."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    return (torch.randn((V, channels), generator=g, dtype=torch.float64) * sigma).to(torch.float32)
