"""ctypes binding of the C ABI in include/curast.h (argument marshalling only).

PyTorch provides device memory and streams; every step of the rasterizer
runs in the CUDA library.  There is no CPU fallback: without the built
library or without a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional, Sequence

import numpy as np
import torch

from .build import build_library, lib_path

OK = 0
STATUS_NAMES = {
    0: "CURAST_OK", -1: "CURAST_ERR_INVALID_ARG", -2: "CURAST_ERR_OUT_OF_MEMORY", -3: "CURAST_ERR_ID_SPACE_OVERFLOW",
    -4: "CURAST_ERR_INDEX_OUT_OF_RANGE", -5: "CURAST_ERR_DEVICE_TIMEOUT", -6: "CURAST_ERR_CUDA",
    -7: "CURAST_ERR_NOT_AFFINE", -8: "CURAST_ERR_BAD_CAMERA", -9: "CURAST_ERR_NOT_BUILT",
    -10: "CURAST_ERR_TOO_LARGE",
}
STATIC_MAX_INSTANCES = 32
EXPORTS = ["curast_create", "curast_destroy", "curast_status_string", "curast_get_config", "curast_set_config",
           "curast_upload_mesh", "curast_update_mesh", "curast_add_instance", "curast_clear_instances",
           "curast_clear", "curast_render", "curast_render_mesh", "curast_render_batch", "curast_resolve", "curast_resolve_ss", "curast_get_mesh_info",
           "curast_interpolate", "curast_interpolate_backward", "curast_sync", "curast_stage_times",
           "curast_autotune", "curast_last_frame", "curast_render_static", "curast_set_mesh_texture",
           "curast_resolve_textured"]


class CurastError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{what}: {name}" if what else name)


class View(C.Structure):
    _fields_ = [("view", C.c_float * 16), ("proj", C.c_float * 16), ("W", C.c_int32), ("H", C.c_int32),
                ("vis", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("stage1_max_pixels", C.c_uint32), ("stage2_max_pixels", C.c_uint32), ("tile_log2", C.c_uint32),
                ("stage1_tri_per_thread", C.c_uint32), ("pairs_per_segment", C.c_uint32),
                ("queue1_capacity", C.c_uint64), ("queue2_capacity", C.c_uint64), ("check_indices", C.c_uint32),
                ("collect_stats", C.c_uint32), ("stage1_bitmap_bytes", C.c_uint64),
                ("stage1_group_min_pairs", C.c_uint32), ("stage3_raycast", C.c_uint32),
                ("stage1_exact_all", C.c_uint32), ("stage1_vertex_reuse", C.c_uint32),
                ("stage3_tile_buffer", C.c_uint32), ("reserved", C.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("triangles_in", C.c_uint64), ("culled_clip", C.c_uint64), ("culled_backface", C.c_uint64),
                ("culled_tiny", C.c_uint64), ("stage1_rasterized", C.c_uint64), ("queued_stage2", C.c_uint64),
                ("stage2_rasterized", C.c_uint64), ("queued_stage3", C.c_uint64), ("queue1_overflow", C.c_uint64),
                ("queue2_overflow", C.c_uint64), ("exact_path", C.c_uint64), ("device_error", C.c_uint32),
                ("reserved", C.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class MeshInfo(C.Structure):
    _fields_ = [("V", C.c_uint64), ("T", C.c_uint64), ("compressed", C.c_uint32), ("index_bits", C.c_uint32),
                ("index_min", C.c_uint32), ("pad", C.c_uint32), ("pos_lo", C.c_float * 3), ("pos_step", C.c_float * 3),
                ("geometry_bytes", C.c_uint64), ("packed_indices", C.c_void_p), ("quantized_positions", C.c_void_p),
                ("grid_flags", C.c_void_p)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}
        d["pos_lo"] = list(self.pos_lo)
        d["pos_step"] = list(self.pos_step)
        return d


MESH_COMPRESSED = 1


class FrameInfo(C.Structure):
    _fields_ = [("pairs", C.c_uint64), ("segments", C.c_uint64), ("work_items", C.c_uint64),
                ("triangles", C.c_uint64), ("unique_triangles", C.c_uint64), ("unique_vertices", C.c_uint64),
                ("rounds", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LOCK = threading.Lock()
_LIB = None


def load(build: bool = False, path: Optional[str] = None) -> C.CDLL:
    """Loads the CUDA library; raises if it has not been built."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        p = path or lib_path()
        if build:
            p = build_library()
        if not os.path.exists(p):
            raise RuntimeError(f"the CUDA library {p} is not built; run __graft_entry__.build() first")
        L = C.CDLL(p)
        vp, i32, u32, u64 = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64
        fp = C.POINTER(C.c_float)
        sig = {
            "curast_create": [C.POINTER(vp), i32],
            "curast_destroy": [vp],
            "curast_get_config": [vp, C.POINTER(Config)],
            "curast_set_config": [vp, C.POINTER(Config)],
            "curast_upload_mesh": [vp, vp, u64, vp, u64, vp, u32, C.POINTER(u32)],
            "curast_get_mesh_info": [vp, u32, C.POINTER(MeshInfo)],
            "curast_update_mesh": [vp, u32, vp, vp, vp],
            "curast_add_instance": [vp, u32, fp, C.POINTER(u32)],
            "curast_clear_instances": [vp],
            "curast_clear": [vp, u64, vp],
            "curast_render": [vp, fp, fp, i32, i32, vp, vp],
            "curast_render_mesh": [vp, u32, fp, fp, i32, i32, vp, vp],
            "curast_render_batch": [vp, C.POINTER(View), i32, i32, vp],
            "curast_resolve": [vp, fp, fp, i32, i32, vp, vp, vp, vp],
            "curast_resolve_ss": [vp, fp, fp, i32, i32, i32, vp, vp, vp, vp],
            "curast_set_mesh_texture": [vp, u32, vp, vp, i32],
            "curast_resolve_textured": [vp, fp, fp, i32, i32, vp, vp, vp, vp, vp],
            "curast_interpolate": [vp, u32, vp, fp, fp, i32, i32, vp, vp, i32, vp, vp],
            "curast_interpolate_backward": [vp, u32, vp, fp, fp, i32, i32, vp, vp, i32, vp, vp, vp, vp],
            "curast_sync": [vp, vp, C.POINTER(Stats)],
            "curast_stage_times": [vp, fp],
            "curast_last_frame": [vp, C.POINTER(FrameInfo)],
            "curast_render_static": [vp, u64, vp, u64, fp, i32, fp, fp, i32, i32, vp, vp],
            "curast_autotune": [vp, C.POINTER(View), i32, vp, C.POINTER(Config)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = None if name == "curast_destroy" else C.c_int32
        L.curast_status_string.argtypes = [C.c_int32]
        L.curast_status_string.restype = C.c_char_p
        _LIB = L
        return L


def _check(st: int, what: str):
    if st != OK:
        raise CurastError(st, what)


def _mat(m) -> C.Array:
    a = np.ascontiguousarray(np.asarray(m.cpu() if hasattr(m, "cpu") else m, dtype=np.float32)).reshape(16)
    return (C.c_float * 16)(*[float(x) for x in a])


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, dtype, what: str, device):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA {dtype} tensor")
    if t.device != device:
        raise ValueError(f"{what} is on {t.device}, the renderer on {device}")


class Renderer:
    """One rasterizer context on one CUDA device.

    Meshes are borrowed: the tensors passed to upload_mesh are referenced
    until the renderer is closed.  Visibility buffers are (H, W) int64
    tensors holding the unsigned 64-bit words (row 0 = bottom)."""

    def __init__(self, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the rasterizer needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else int(device))
        self.L = load()
        h = C.c_void_p()
        _check(self.L.curast_create(C.byref(h), self.device.index), "curast_create")
        self._h = h
        self._keep = {}
        self._mesh_T = []
        self._n_inst = 0

    def close(self):
        if getattr(self, "_h", None):
            self.L.curast_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- config
    @property
    def config(self) -> Config:
        c = Config()
        _check(self.L.curast_get_config(self._h, C.byref(c)), "curast_get_config")
        return c

    def set_config(self, **kw) -> Config:
        known = {k for k, _ in Config._fields_}
        for k in kw:
            if k not in known:
                raise KeyError(f"unknown config field {k!r}")
        c = self.config
        for k, v in kw.items():
            setattr(c, k, v)
        _check(self.L.curast_set_config(self._h, C.byref(c)), "curast_set_config")
        return c

    # ---------------------------------------------------------------- scene
    def upload_mesh(self, pos: torch.Tensor, idx: torch.Tensor, rgba8: Optional[torch.Tensor] = None,
                    compressed: bool = False) -> int:
        """Registers a mesh; compressed=True keeps only the Section 4.6
        encoding (the context owns it; pos and idx may be freed after)."""
        _need(pos, torch.float32, "pos", self.device)
        if idx.dtype not in (torch.int32, torch.uint32):
            raise ValueError("idx must hold uint32 (int32 tensor)")
        _need(idx, idx.dtype, "idx", self.device)
        if rgba8 is not None:
            _need(rgba8, torch.uint8, "rgba8", self.device)
        mid = C.c_uint32()
        flags = MESH_COMPRESSED if compressed else 0
        _check(self.L.curast_upload_mesh(self._h, _ptr(pos), pos.shape[0], _ptr(idx), idx.shape[0], _ptr(rgba8), flags,
                                         C.byref(mid)), "curast_upload_mesh")
        self._keep[("mesh", mid.value)] = (None, None, rgba8) if compressed else (pos, idx, rgba8)
        self._mesh_T.append(int(idx.shape[0]))
        return mid.value

    def update_mesh(self, mesh: int, pos=None, idx=None, rgba8=None):
        old = list(self._keep[("mesh", mesh)])
        for k, t in enumerate((pos, idx, rgba8)):
            if t is not None:
                old[k] = t
        _check(self.L.curast_update_mesh(self._h, mesh, _ptr(pos), _ptr(idx), _ptr(rgba8)), "curast_update_mesh")
        self._keep[("mesh", mesh)] = tuple(old)

    def add_instance(self, mesh: int, model=None) -> int:
        iid = C.c_uint32()
        m = np.eye(4, dtype=np.float32) if model is None else model
        _check(self.L.curast_add_instance(self._h, mesh, _mat(m), C.byref(iid)), "curast_add_instance")
        self._n_inst += 1
        return iid.value

    def clear_instances(self):
        _check(self.L.curast_clear_instances(self._h), "curast_clear_instances")
        self._n_inst = 0

    # --------------------------------------------------------------- render
    def new_vis(self, W: int, H: int) -> torch.Tensor:
        return torch.empty((H, W), dtype=torch.int64, device=self.device)

    def render(self, view, proj, W: int, H: int, vis: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        vis = self.new_vis(W, H) if vis is None else vis
        _need(vis, torch.int64, "vis", self.device)
        if vis.numel() != W * H:
            raise ValueError("vis must hold W*H words")
        _check(self.L.curast_render(self._h, _mat(view), _mat(proj), W, H, _ptr(vis), _stream(stream)),
               "curast_render")
        return vis

    def render_mesh(self, mesh: int, view, proj, W: int, H: int, vis: torch.Tensor, stream=None) -> torch.Tensor:
        _need(vis, torch.int64, "vis", self.device)
        _check(self.L.curast_render_mesh(self._h, mesh, _mat(view), _mat(proj), W, H, _ptr(vis), _stream(stream)),
               "curast_render_mesh")
        return vis

    @staticmethod
    def _views(views) -> C.Array:
        arr = (View * len(views))()
        for k, (view, proj, W, H, vis) in enumerate(views):
            arr[k].view[:] = list(_mat(view))
            arr[k].proj[:] = list(_mat(proj))
            arr[k].W, arr[k].H = int(W), int(H)
            arr[k].vis = vis.data_ptr()
        return arr

    def render_batch(self, views: Sequence, use_graph: bool = True, stream=None) -> List[torch.Tensor]:
        """views: sequence of (view, proj, W, H, vis-or-None)."""
        full = []
        for v in views:
            view, proj, W, H = v[:4]
            vis = v[4] if len(v) > 4 and v[4] is not None else self.new_vis(W, H)
            _need(vis, torch.int64, "vis", self.device)
            full.append((view, proj, W, H, vis))
        arr = self._views(full)
        _check(self.L.curast_render_batch(self._h, arr, len(full), int(use_graph), _stream(stream)),
               "curast_render_batch")
        return [f[4] for f in full]

    def clear(self, vis: torch.Tensor, stream=None):
        _check(self.L.curast_clear(_ptr(vis), vis.numel(), _stream(stream)), "curast_clear")

    # -------------------------------------------------------------- resolve
    def resolve(self, view, proj, vis: torch.Tensor, want_f32: bool = True, want_rgba8: bool = True, stream=None):
        H, W = vis.shape
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device) if want_f32 else None
        u8 = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device) if want_rgba8 else None
        _check(self.L.curast_resolve(self._h, _mat(view), _mat(proj), W, H, _ptr(vis), _ptr(f32), _ptr(u8),
                                     _stream(stream)), "curast_resolve")
        return f32, u8

    def resolve_ss(self, view, proj, vis: torch.Tensor, ss: int, want_f32: bool = True, want_rgba8: bool = True,
                   stream=None):
        """Box-filtered resolve of a view rendered at ss times the output
        size per axis; returns the (H, W) output images."""
        Hs, Ws = vis.shape
        if Hs % ss or Ws % ss:
            raise ValueError("the super-sampled buffer must be ss times the output size")
        H, W = Hs // ss, Ws // ss
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device) if want_f32 else None
        u8 = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device) if want_rgba8 else None
        _check(self.L.curast_resolve_ss(self._h, _mat(view), _mat(proj), W, H, ss, _ptr(vis), _ptr(f32), _ptr(u8),
                                        _stream(stream)), "curast_resolve_ss")
        return f32, u8

    def set_mesh_texture(self, mesh: int, uv: Optional[torch.Tensor], texels: Optional[torch.Tensor],
                         log2_size: int = 0):
        """Per-vertex uv (V, 2) float32 and a flat RGBA8 mip chain of side
        2^log2_size for the textured resolve; texels=None removes it.  The
        tensors are kept referenced while registered."""
        if texels is None:
            _check(self.L.curast_set_mesh_texture(self._h, mesh, None, None, 0), "curast_set_mesh_texture")
            self._keep.pop(("tex", mesh), None)
            return
        _need(uv, torch.float32, "uv", self.device)
        _need(texels, torch.uint8, "texels", self.device)
        want = 4 * sum(4 ** (log2_size - l) for l in range(log2_size + 1))
        if texels.numel() != want:
            raise ValueError(f"a mip chain of side 2^{log2_size} holds {want} bytes, got {texels.numel()}")
        _check(self.L.curast_set_mesh_texture(self._h, mesh, _ptr(uv), _ptr(texels), log2_size),
               "curast_set_mesh_texture")
        self._keep[("tex", mesh)] = (uv, texels)

    def resolve_textured(self, view, proj, vis: torch.Tensor, want_f32: bool = True, want_rgba8: bool = True,
                         want_level: bool = True, stream=None):
        """Resolve with textures and the 4-ray mip-level choice; returns
        (rgba float32 (H, W, 4), rgba8 (H, W, 4), level uint8 (H, W)), each
        None when not wanted."""
        H, W = vis.shape
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device) if want_f32 else None
        u8 = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device) if want_rgba8 else None
        lev = torch.empty((H, W), dtype=torch.uint8, device=self.device) if want_level else None
        _check(self.L.curast_resolve_textured(self._h, _mat(view), _mat(proj), W, H, _ptr(vis), _ptr(f32), _ptr(u8),
                                              _ptr(lev), _stream(stream)), "curast_resolve_textured")
        return f32, u8, lev

    # ------------------------------------------------------- differentiable
    def interpolate(self, mesh: int, view, proj, vis: torch.Tensor, attr: torch.Tensor,
                    pos: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        H, W = vis.shape
        _need(attr, torch.float32, "attr", self.device)
        Cc = attr.shape[1]
        out = torch.empty((H, W, Cc), dtype=torch.float32, device=self.device)
        _check(self.L.curast_interpolate(self._h, mesh, _ptr(pos), _mat(view), _mat(proj), W, H, _ptr(vis),
                                         _ptr(attr), Cc, _ptr(out), _stream(stream)), "curast_interpolate")
        return out

    def interpolate_backward(self, mesh: int, view, proj, vis: torch.Tensor, attr: torch.Tensor,
                             grad_out: torch.Tensor, pos: Optional[torch.Tensor] = None, want_attr: bool = True,
                             want_pos: bool = True, stream=None):
        H, W = vis.shape
        Cc = attr.shape[1]
        grad_out = grad_out.contiguous()
        V = attr.shape[0]
        ga = torch.zeros((V, Cc), dtype=torch.float32, device=self.device) if want_attr else None
        gp = torch.zeros((V, 3), dtype=torch.float32, device=self.device) if want_pos else None
        _check(self.L.curast_interpolate_backward(self._h, mesh, _ptr(pos), _mat(view), _mat(proj), W, H, _ptr(vis),
                                                  _ptr(attr), Cc, _ptr(grad_out), _ptr(ga), _ptr(gp),
                                                  _stream(stream)), "curast_interpolate_backward")
        return ga, gp

    # ----------------------------------------------------------- sync & co
    def sync(self, stream=None) -> dict:
        st = Stats()
        _check(self.L.curast_sync(self._h, _stream(stream), C.byref(st)), "curast_sync")
        return st.as_dict()

    def mesh_info(self, mesh: int) -> dict:
        mi = MeshInfo()
        _check(self.L.curast_get_mesh_info(self._h, mesh, C.byref(mi)), "curast_get_mesh_info")
        return mi.as_dict()

    def last_frame(self) -> dict:
        fi = FrameInfo()
        _check(self.L.curast_last_frame(self._h, C.byref(fi)), "curast_last_frame")
        return fi.as_dict()

    def stage_times(self) -> List[float]:
        """Milliseconds of the last render: clear, stage-1 cull, stage-1
        exact, stage 2, stage 3."""
        out = (C.c_float * 5)()
        _check(self.L.curast_stage_times(self._h, out), "curast_stage_times")
        return list(out)

    def autotune(self, views: Sequence, stream=None) -> dict:
        full = [(v[0], v[1], v[2], v[3], v[4]) for v in views]
        arr = self._views(full)
        cfg = Config()
        _check(self.L.curast_autotune(self._h, arr, len(full), _stream(stream), C.byref(cfg)), "curast_autotune")
        return cfg.as_dict()


def render_static(pos: torch.Tensor, idx: torch.Tensor, models, view, proj, W: int, H: int,
                  vis: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Context-free render of up to 32 instances of one mesh that allocates no
    device memory in the library (curast_render_static): for callers that must
    not allocate, such as real-time loops or plug-ins whose host owns all
    device memory.  ``models`` is a sequence of 4x4 matrices or None (one
    identity instance).  All calls share one fixed scratch array, so calls
    must not overlap on the GPU; the first call on a device should happen
    before any stream capture.  pos, idx and vis must live on one device; the
    call runs with that device current."""
    L = load()
    dev = pos.device if isinstance(pos, torch.Tensor) else None
    if dev is None or dev.type != "cuda":
        raise ValueError("pos must be a contiguous CUDA float32 tensor")
    _need(pos, torch.float32, "pos", dev)
    if not isinstance(idx, torch.Tensor) or idx.dtype not in (torch.int32, torch.uint32):
        raise ValueError("idx must hold uint32 (int32 tensor)")
    _need(idx, idx.dtype, "idx", dev)
    if pos.dim() != 2 or pos.shape[1] != 3 or idx.dim() != 2 or idx.shape[1] != 3:
        raise ValueError("pos must be (V, 3) and idx (T, 3)")
    if vis is None:
        vis = torch.empty((H, W), dtype=torch.int64, device=dev)
    _need(vis, torch.int64, "vis", dev)
    if vis.numel() != W * H:
        raise ValueError("vis must hold W*H words")
    if models is None:
        mats, n = None, 1
    else:
        arr = np.ascontiguousarray(np.stack([np.asarray(m, np.float32).reshape(16) for m in models]), np.float32)
        n = arr.shape[0]
        mats = (C.c_float * (16 * n))(*[float(x) for x in arr.reshape(-1)])
    with torch.cuda.device(dev):
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        if st.device != dev:
            raise ValueError(f"the stream is on {st.device}, the buffers on {dev}")
        _check(L.curast_render_static(_ptr(pos), pos.shape[0], _ptr(idx), idx.shape[0], mats, n, _mat(view),
                                      _mat(proj), W, H, _ptr(vis), C.c_void_p(st.cuda_stream)),
               "curast_render_static")
    return vis


class InterpolateFn(torch.autograd.Function):
    """out = interpolate(attr) with the visibility buffer held fixed;
    differentiable with respect to the vertex attributes and positions.

    Call as InterpolateFn.apply(renderer, mesh, pos, attr, vis, view, proj)."""

    @staticmethod
    def forward(ctx, renderer: Renderer, mesh: int, pos: torch.Tensor, attr: torch.Tensor, vis: torch.Tensor,
                view, proj):
        pos_c = pos.detach().contiguous()
        attr_c = attr.detach().contiguous()
        out = renderer.interpolate(mesh, view, proj, vis, attr_c, pos=pos_c)
        ctx.save_for_backward(pos_c, attr_c, vis)
        ctx.renderer, ctx.mesh, ctx.view, ctx.proj = renderer, mesh, view, proj
        return out

    @staticmethod
    def backward(ctx, grad_out):
        pos, attr, vis = ctx.saved_tensors
        ga, gp = ctx.renderer.interpolate_backward(ctx.mesh, ctx.view, ctx.proj, vis, attr, grad_out, pos=pos,
                                                   want_attr=ctx.needs_input_grad[3],
                                                   want_pos=ctx.needs_input_grad[2])
        return None, None, gp, ga, None, None, None
