"""Textured resolve with the 4-ray mip-level choice (Section 4.4, reading R17):
the GPU's levels and RGBA8 colours equal the oracle's, FP32 colours within
1e-6, on the small workload, a grazing plane and close-up and distant poses
of a heightfield, with textured and untextured meshes side by side."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import oracle as orc
from synthetic.scenes import Camera, Instance, Mesh, Scene

from gpu_util import upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api as A
    return A


def _check(api, sc, textures, cams, min_levels=1):
    r = api.Renderer(0)
    keep = upload(r, sc)
    dev_tex = []
    for k, t in enumerate(textures):
        if t is None:
            continue
        uv, tex, L = t[0].cuda().contiguous(), t[1].cuda().contiguous(), t[2]
        dev_tex.append((uv, tex))
        r.set_mesh_texture(k, uv, tex, L)
    osc = orc.OracleScene(sc)
    seen = set()
    for cam in cams:
        vis = r.render(cam.view, cam.proj, cam.W, cam.H)
        f32, u8, lev = r.resolve_textured(cam.view, cam.proj, vis)
        r.sync()
        ref = orc.render(osc, cam)
        np.testing.assert_array_equal(vis.cpu().numpy().view(np.uint64), ref)
        rf, r8, rl = orc.resolve_textured(osc, cam, ref, textures)
        np.testing.assert_array_equal(lev.cpu().numpy(), rl)
        np.testing.assert_array_equal(u8.cpu().numpy(), r8)
        np.testing.assert_allclose(f32.cpu().numpy(), rf, atol=1e-6, rtol=0)
        seen |= set(np.unique(rl).tolist()) - {255}
    assert len(seen) >= min_levels, seen
    del keep, dev_tex
    r.close()


def test_small_workload_textured(api):
    """The small workload's heightfield textured (uv = grid coordinates, a
    256^2 mip chain), its ground triangles untextured (vertex colours)."""
    sc = S.scene_small(n=128, W=320, H=240)
    tex = [(S.grid_uv(128), S.texture_mip_chain(8, seed=3), 8), None]
    _check(api, sc, tex, sc.cameras, min_levels=4)


def test_heightfield_poses_textured(api):
    """Close-up poses (footprints below a texel: level 0) to whole-mesh views
    (coarse levels) of a 300^2 heightfield with a 4096^2 mip chain."""
    hf = S.heightfield_mesh(300, seed=100)
    sc = Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))], [])
    tex = [(S.grid_uv(300), S.texture_mip_chain(12, seed=5), 12)]
    cams = [S.camera_unique_pose(k, 480, 270) for k in range(8)]
    _check(api, sc, tex, cams, min_levels=6)


def test_grazing_plane_and_instances(api):
    """Two instances of a large textured quad seen at a grazing angle (the
    footprint grows towards the horizon and differs along x and y, the
    texture repeats: uv well outside [0, 1]), one rotated and scaled; the
    texel coordinates clamp at the level's edges."""
    pos = np.array([[-2.0, 0.0, 3.0], [3.0, 0.0, 3.0], [-2.0, 0.0, -6.0], [3.0, 0.0, -6.0]], np.float32)
    idx = np.array([[0, 1, 2], [2, 1, 3]], np.int32)
    uv = np.array([[0.0, 0.0], [2.5, -0.7], [-0.6, 3.1], [1.9, 2.4]], np.float32)
    m = Mesh(pos=torch.tensor(pos), idx=torch.tensor(idx),
             rgba8=torch.tensor(np.full((4, 4), 200, np.uint8)))
    rot = np.eye(4, dtype=np.float32)
    c, s_ = np.cos(0.4), np.sin(0.4)
    rot[:3, :3] = np.array([[c, 0, s_], [0, 1, 0], [-s_, 0, c]], np.float32) * 0.7
    rot[:3, 3] = (0.5, 0.02, -1.0)
    sc = Scene([m], [Instance(0, np.eye(4, dtype=np.float32)), Instance(0, rot)], [])
    tex = [(torch.tensor(uv), S.texture_mip_chain(9, seed=8), 9)]
    cams = [Camera(S.look_at((0.3, 0.35, 2.2), (0.55, 0.0, -0.4)), S.perspective(70.0, 1.5, 0.01, 100.0), 360, 240),
            Camera(S.look_at((-1.0, 2.0, 4.0), (0.5, 0.0, -2.0)), S.perspective(50.0, 1.0, 0.01, 100.0), 256, 256)]
    _check(api, sc, tex, cams, min_levels=5)


def test_texture_argument_checks(api):
    hf = S.heightfield_mesh(8, seed=1)
    r = api.Renderer(0)
    keep = upload(r, Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))]))
    uv = S.grid_uv(8).cuda()
    with pytest.raises(ValueError):
        r.set_mesh_texture(0, uv, torch.zeros(100, dtype=torch.uint8, device="cuda"), 4)
    with pytest.raises(api.CurastError):
        r.set_mesh_texture(7, uv, S.texture_mip_chain(2, seed=1).cuda(), 2)
    r.set_mesh_texture(0, None, None)
    del keep
    r.close()
