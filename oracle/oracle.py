"""ctypes front end of the C oracle (curast_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the product path never imports it.  It shares
nothing with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "curast_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
ID_MASK = np.uint64((1 << 36) - 1)


def lib_path() -> str:
    return os.path.join(_BUILD, f"liborc_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (contraction off, no fast math)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Mesh(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("V", C.c_uint64), ("idx", C.c_void_p), ("T", C.c_uint64),
                ("rgba8", C.c_void_p)]


class _Texture(C.Structure):
    _fields_ = [("uv", C.c_void_p), ("texels", C.c_void_p), ("log2_size", C.c_int32), ("pad", C.c_int32)]


class _Instance(C.Structure):
    _fields_ = [("mesh", C.c_uint32), ("pad", C.c_uint32), ("model", C.c_float * 16)]


class _Camera(C.Structure):
    _fields_ = [("view", C.c_float * 16), ("proj", C.c_float * 16), ("W", C.c_int32), ("H", C.c_int32)]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = C.CDLL(build())
            L.orc_render.restype = C.c_int
            L.orc_render.argtypes = [C.POINTER(_Mesh), C.c_int, C.POINTER(_Instance), C.c_int,
                                     C.POINTER(_Camera), C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
            L.orc_render_paper.restype = C.c_int
            L.orc_render_paper.argtypes = [C.POINTER(_Mesh), C.c_int, C.POINTER(_Instance), C.c_int,
                                           C.POINTER(_Camera), C.c_uint32, C.c_uint32, C.c_void_p]
            L.orc_resolve.argtypes = [C.POINTER(_Mesh), C.c_int, C.POINTER(_Instance), C.c_int,
                                      C.POINTER(_Camera), C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_resolve_textured.argtypes = [C.POINTER(_Mesh), C.c_int, C.POINTER(_Texture), C.POINTER(_Instance),
                                               C.c_int, C.POINTER(_Camera), C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.c_void_p]
            L.orc_interpolate.argtypes = [C.POINTER(_Mesh), C.c_int, C.POINTER(_Instance), C.c_int,
                                          C.POINTER(_Camera), C.c_void_p, C.c_uint32, C.c_void_p, C.c_int,
                                          C.c_void_p, C.c_void_p]
            L.orc_box_filter.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_index_bits.argtypes = [C.c_uint32]
            L.orc_index_bits.restype = C.c_int
            L.orc_pack_indices.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p]
            L.orc_unpack_indices.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p]
            L.orc_quantize_positions.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_dequantize_positions.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_camera_params.argtypes = [C.c_void_p, C.c_void_p]
            L.orc_model_view.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_clip.argtypes = [C.c_void_p, C.c_float, C.c_void_p]
            L.orc_raster_fixed.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_int,
                                           C.c_int, C.c_int, C.c_void_p]
            L.orc_project.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_uint64,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_bases.argtypes = [C.POINTER(_Mesh), C.c_int, C.POINTER(_Instance), C.c_int, C.c_void_p]
            _LIB = L
    return _LIB


def _np(t, dtype):
    """torch tensor or array -> contiguous CPU numpy array of dtype."""
    if t is None:
        return None
    if hasattr(t, "detach"):
        t = t.detach().cpu().numpy()
    return np.ascontiguousarray(t, dtype=dtype)


class OracleScene:
    """Holds numpy copies of a synthetic.Scene in the oracle's C layout.

    ``tri_counts`` stands in for meshes given as None (no geometry): they
    still count towards the id bases but cannot be rendered.
    """

    def __init__(self, scene, tri_counts=None):
        self._keep = []
        n = len(scene.meshes)
        self.meshes = (_Mesh * n)()
        for k, m in enumerate(scene.meshes):
            if m is None:
                self.meshes[k].pos = None
                self.meshes[k].V = 0
                self.meshes[k].idx = None
                self.meshes[k].T = int(tri_counts[k])
                self.meshes[k].rgba8 = None
                continue
            pos = _np(m.pos, np.float32)
            idx = _np(m.idx, np.int32).view(np.uint32)
            col = _np(m.rgba8, np.uint8)
            self._keep += [pos, idx, col]
            self.meshes[k].pos = pos.ctypes.data
            self.meshes[k].V = pos.shape[0]
            self.meshes[k].idx = idx.ctypes.data
            self.meshes[k].T = idx.shape[0]
            self.meshes[k].rgba8 = col.ctypes.data if col is not None else None
        ni = len(scene.instances)
        self.inst = (_Instance * ni)()
        for k, it in enumerate(scene.instances):
            self.inst[k].mesh = it.mesh
            self.inst[k].model[:] = [float(v) for v in np.asarray(it.model, np.float32).reshape(-1)]
        self.n_meshes, self.n_inst = n, ni

    def bases(self) -> np.ndarray:
        b = np.zeros(self.n_inst + 1, np.uint64)
        st = _lib().orc_bases(self.meshes, self.n_meshes, self.inst, self.n_inst, b.ctypes.data)
        if st != 0:
            raise ValueError(f"orc_bases failed: {st}")
        return b


def _cam(camera) -> _Camera:
    c = _Camera()
    c.view[:] = [float(v) for v in np.asarray(camera.view, np.float32).reshape(-1)]
    c.proj[:] = [float(v) for v in np.asarray(camera.proj, np.float32).reshape(-1)]
    c.W, c.H = int(camera.W), int(camera.H)
    return c


def render(osc: OracleScene, camera, first: int = 0, count=None, mode: int = 0,
           cull_back: bool = True, out=None) -> np.ndarray:
    """Visibility buffer (mode 0, uint64, all ones = empty) or coverage counts
    (mode 1) as an (H, W) array, row 0 = bottom."""
    if count is None:
        count = osc.n_inst - first
    if out is None:
        out = np.full((camera.H, camera.W), EMPTY if mode == 0 else 0, np.uint64)
    st = _lib().orc_render(osc.meshes, osc.n_meshes, osc.inst, osc.n_inst, C.byref(_cam(camera)),
                           first, count, mode, int(cull_back), out.ctypes.data)
    if st != 0:
        raise ValueError(f"orc_render failed: {st}")
    return out


def render_paper(osc: OracleScene, camera, s1_max: int = 128, s2_max: int = 4096) -> np.ndarray:
    """Visibility buffer with the paper's ray-cast stage 3: triangles whose
    visible bbox on reaching stage 2 holds more than s2_max pixel centres are
    covered by view-space pixel rays, every other one by edge functions."""
    out = np.full((camera.H, camera.W), EMPTY, np.uint64)
    st = _lib().orc_render_paper(osc.meshes, osc.n_meshes, osc.inst, osc.n_inst, C.byref(_cam(camera)),
                                 s1_max, s2_max, out.ctypes.data)
    if st != 0:
        raise ValueError(f"orc_render_paper failed: {st}")
    return out


def resolve(osc: OracleScene, camera, vis: np.ndarray):
    vis = np.ascontiguousarray(vis, np.uint64)
    rgba = np.zeros((camera.H, camera.W, 4), np.float32)
    rgba8 = np.zeros((camera.H, camera.W, 4), np.uint8)
    st = _lib().orc_resolve(osc.meshes, osc.n_meshes, osc.inst, osc.n_inst, C.byref(_cam(camera)),
                            vis.ctypes.data, rgba.ctypes.data, rgba8.ctypes.data)
    if st != 0:
        raise ValueError(f"orc_resolve failed: {st}")
    return rgba, rgba8


def resolve_textured(osc: OracleScene, camera, vis: np.ndarray, textures):
    """Resolve with textures and the 4-ray mip-level choice (Section 4.4).
    textures: one entry per mesh, None or (uv (V, 2) float32, flat RGBA8 mip
    chain, log2_size).  Returns (rgba float32 (H, W, 4), rgba8, level uint8
    (H, W), 255 where no texture was sampled)."""
    vis = np.ascontiguousarray(vis, np.uint64)
    tx = (_Texture * osc.n_meshes)()
    keep = []
    for k, t in enumerate(textures):
        if t is None:
            continue
        uv = _np(t[0], np.float32)
        tex = _np(t[1], np.uint8)
        keep += [uv, tex]
        tx[k].uv = uv.ctypes.data
        tx[k].texels = tex.ctypes.data
        tx[k].log2_size = int(t[2])
    rgba = np.zeros((camera.H, camera.W, 4), np.float32)
    rgba8 = np.zeros((camera.H, camera.W, 4), np.uint8)
    level = np.zeros((camera.H, camera.W), np.uint8)
    st = _lib().orc_resolve_textured(osc.meshes, osc.n_meshes, tx, osc.inst, osc.n_inst, C.byref(_cam(camera)),
                                     vis.ctypes.data, rgba.ctypes.data, rgba8.ctypes.data, level.ctypes.data)
    if st != 0:
        raise ValueError(f"orc_resolve_textured failed: {st}")
    return rgba, rgba8, level


# ------------------------------------------------------------ compression --
def index_bits(span: int) -> int:
    return int(_lib().orc_index_bits(span))


def pack_indices(idx, imin: int, bits: int) -> np.ndarray:
    idx = np.ascontiguousarray(idx, np.uint32).reshape(-1)
    words = np.zeros((idx.size * bits + 31) // 32 + 1, np.uint32)
    _lib().orc_pack_indices(idx.ctypes.data, idx.size, imin, bits, words.ctypes.data)
    return words


def unpack_indices(words, n: int, imin: int, bits: int) -> np.ndarray:
    words = np.ascontiguousarray(words, np.uint32)
    out = np.zeros(n, np.uint32)
    _lib().orc_unpack_indices(words.ctypes.data, n, imin, bits, out.ctypes.data)
    return out


def quantize_positions(pos, lo, size):
    pos = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
    lo = np.ascontiguousarray(lo, np.float32)
    size = np.ascontiguousarray(size, np.float64)
    q = np.zeros(pos.shape, np.uint16)
    _lib().orc_quantize_positions(pos.ctypes.data, pos.shape[0], lo.ctypes.data, size.ctypes.data, q.ctypes.data)
    return q


def dequantize_positions(q, lo, step):
    q = np.ascontiguousarray(q, np.uint16).reshape(-1, 3)
    lo = np.ascontiguousarray(lo, np.float32)
    step = np.ascontiguousarray(step, np.float32)
    out = np.zeros(q.shape, np.float32)
    _lib().orc_dequantize_positions(q.ctypes.data, q.shape[0], lo.ctypes.data, step.ctypes.data, out.ctypes.data)
    return out


def compress_mesh(pos, idx):
    """The Section 4.6 encoding of a mesh and the mesh it decodes to:
    returns (fields, decoded positions, decoded indices).  Bounds are the
    per-axis min / max of the positions; size and step as described at
    orc_quantize_positions."""
    pos = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
    idx = np.ascontiguousarray(idx, np.uint32).reshape(-1)
    lo = pos.min(axis=0).astype(np.float32)
    hi = pos.max(axis=0).astype(np.float32)
    size = hi.astype(np.float64) - lo.astype(np.float64)
    step = (size / 65535.0).astype(np.float32)
    imin = int(idx.min()) if idx.size else 0
    imax = int(idx.max()) if idx.size else 0
    bits = index_bits(imax - imin)
    q = quantize_positions(pos, lo, size)
    words = pack_indices(idx, imin, bits)
    fields = {"lo": lo, "step": step, "size": size, "imin": imin, "bits": bits, "q": q, "words": words}
    return fields, dequantize_positions(q, lo, step), unpack_indices(words, idx.size, imin, bits)


def box_filter(fine: np.ndarray, ss: int):
    """Box filter of an (ss H, ss W, 4) FP32 image to (H, W, 4) FP32 and RGBA8."""
    fine = np.ascontiguousarray(fine, np.float32)
    Hs, Ws = fine.shape[:2]
    H, W = Hs // ss, Ws // ss
    rgba = np.zeros((H, W, 4), np.float32)
    rgba8 = np.zeros((H, W, 4), np.uint8)
    st = _lib().orc_box_filter(fine.ctypes.data, W, H, ss, rgba.ctypes.data, rgba8.ctypes.data)
    if st != 0:
        raise ValueError(f"orc_box_filter failed: {st}")
    return rgba, rgba8


def resolve_ss(osc: OracleScene, camera_fine, vis_fine: np.ndarray, ss: int):
    """Super-sampled resolve: the resolve of the (ss W) x (ss H) render,
    box-filtered to W x H."""
    fine, _ = resolve(osc, camera_fine, vis_fine)
    return box_filter(fine, ss)


def interpolate(osc: OracleScene, camera, vis: np.ndarray, mesh: int, attr):
    vis = np.ascontiguousarray(vis, np.uint64)
    attr = _np(attr, np.float32)
    Cc = attr.shape[1]
    out = np.zeros((camera.H, camera.W, Cc), np.float32)
    bary = np.zeros((camera.H, camera.W, 3), np.float32)
    st = _lib().orc_interpolate(osc.meshes, osc.n_meshes, osc.inst, osc.n_inst, C.byref(_cam(camera)),
                                vis.ctypes.data, mesh, attr.ctypes.data, Cc, out.ctypes.data, bary.ctypes.data)
    if st != 0:
        raise ValueError(f"orc_interpolate failed: {st}")
    return out, bary


def camera_params(proj) -> np.ndarray:
    p = np.ascontiguousarray(proj, np.float32).reshape(16)
    out = np.zeros(3, np.float32)
    st = _lib().orc_camera_params(p.ctypes.data, out.ctypes.data)
    if st != 0:
        raise ValueError("not a symmetric perspective matrix")
    return out


def model_view(view, model) -> np.ndarray:
    v = np.ascontiguousarray(view, np.float32).reshape(16)
    m = np.ascontiguousarray(model, np.float32).reshape(16)
    out = np.zeros(12, np.float32)
    _lib().orc_model_view(v.ctypes.data, m.ctypes.data, out.ctypes.data)
    return out.reshape(3, 4)


def clip(tri_clip, nearv: float) -> np.ndarray:
    t = np.ascontiguousarray(tri_clip, np.float32).reshape(9)
    out = np.zeros(24, np.float32)
    n = _lib().orc_clip(t.ctypes.data, C.c_float(nearv), out.ctypes.data)
    return out[: 3 * n].reshape(n, 3)


def project(mv, cp, W: int, H: int, pos):
    pos = _np(pos, np.float32)
    n = pos.shape[0]
    mv = np.ascontiguousarray(mv, np.float32).reshape(12)
    cp = np.ascontiguousarray(cp, np.float32).reshape(3)
    clipv = np.zeros((n, 3), np.float32)
    XY = np.zeros((n, 2), np.int32)
    iz = np.zeros(n, np.float32)
    inside = np.zeros(n, np.int32)
    _lib().orc_project(mv.ctypes.data, cp.ctypes.data, W, H, pos.ctypes.data, n, clipv.ctypes.data,
                       XY.ctypes.data, iz.ctypes.data, inside.ctypes.data)
    return clipv, XY, iz, inside.astype(bool)


def raster_fixed(XY, iz, W: int, H: int, id0: int = 0, mode: int = 0, cull_back: bool = True) -> np.ndarray:
    XY = np.ascontiguousarray(XY, np.int32).reshape(-1, 6)
    iz = np.ascontiguousarray(iz, np.float32).reshape(-1, 3)
    out = np.full((H, W), EMPTY if mode == 0 else 0, np.uint64)
    _lib().orc_raster_fixed(XY.ctypes.data, iz.ctypes.data, XY.shape[0], id0, W, H, mode, int(cull_back),
                            out.ctypes.data)
    return out


def decode(vis: np.ndarray):
    """(depth28, id) fields of visibility words."""
    v = np.asarray(vis, np.uint64)
    return (v >> np.uint64(36)), (v & ID_MASK)
