"""The paper's ray-cast stage 3 (Section 4.3) through the C ABI: with
stage3_raycast on, triangles whose visible bbox holds more than
stage2_max_pixels pixel centres are covered by view-space pixel rays, and the
visibility buffers equal the oracle's orc_render_paper bit for bit."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import oracle as orc
from synthetic.scenes import Instance, Scene

from gpu_util import assert_vis_equal, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api as A
    return A


def _renderer(api, **cfg):
    r = api.Renderer(0)
    r.set_config(stage3_raycast=1, **cfg)
    return r


def _paper(scene, cam, s1=128, s2=4096):
    return orc.render_paper(orc.OracleScene(scene), cam, s1, s2)


@pytest.mark.parametrize("cfg", [dict(), dict(stage2_max_pixels=32), dict(stage1_max_pixels=16, stage2_max_pixels=64),
                                 dict(stage2_max_pixels=100000), dict(tile_log2=4),
                                 dict(stage2_max_pixels=32, stage3_tile_buffer=1),
                                 dict(tile_log2=5, stage3_tile_buffer=1)])
def test_small_workload_ray_cast_equals_oracle(api, cfg):
    """The heightfield plus two ground triangles crossing the near plane;
    thresholds moved so that few, many or no triangles are ray cast."""
    sc = S.scene_small()
    cam = sc.cameras[0]
    r = _renderer(api, **cfg)
    keep = upload(r, sc)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    f32, u8 = r.resolve(cam.view, cam.proj, vis)
    r.sync()
    c = r.config
    ref = _paper(sc, cam, c.stage1_max_pixels, c.stage2_max_pixels)
    assert_vis_equal(vis, ref, f"ray-cast mode {cfg}")
    osc = orc.OracleScene(sc)
    rf, r8 = orc.resolve(osc, cam, ref)
    np.testing.assert_allclose(f32.cpu().numpy(), rf, atol=1e-6, rtol=0)
    np.testing.assert_array_equal(u8.cpu().numpy(), r8)
    del keep


def test_ray_cast_differs_from_the_fixed_point_rule(api):
    """The mode is live: the ground triangles' depths come from the rays."""
    sc = S.scene_small()
    cam = sc.cameras[0]
    r = _renderer(api)
    keep = upload(r, sc)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H).cpu().numpy().view(np.uint64)
    r.sync()
    fixed = orc.render(orc.OracleScene(sc), cam)
    assert (vis != fixed).sum() > 1000
    del keep


def test_room_around_the_camera(api):
    """The camera inside a closed box (12 triangles facing inwards): every
    face crosses the near plane or the guard band, so every one reaches
    stage 2 and, being huge, the ray cast; with queue capacities of 1 the
    overflow paths ray cast in place."""
    sc = S.scene_room()
    for cfg in (dict(), dict(queue1_capacity=1, queue2_capacity=1), dict(stage3_tile_buffer=1),
                dict(stage3_tile_buffer=1, queue2_capacity=7)):
        r = _renderer(api, **cfg)
        keep = upload(r, sc)
        for cam in sc.cameras:
            vis = r.render(cam.view, cam.proj, cam.W, cam.H)
            r.sync()
            ref = _paper(sc, cam)
            assert (ref != orc.EMPTY).sum() > 0.9 * cam.W * cam.H
            assert_vis_equal(vis, ref, f"room {cam.W}x{cam.H} {cfg}")
        del keep


def test_close_up_poses_ray_cast(api):
    """Close-up poses of a 300^2 heightfield, triangles of hundreds of
    pixels: with stage2_max_pixels = 32 most of them are ray cast."""
    hf = S.heightfield_mesh(300, seed=100)
    sc = Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))], [])
    r = _renderer(api, stage2_max_pixels=32)
    keep = upload(r, sc)
    for k in (0, 3, 5):
        cam = S.camera_unique_pose(k, 480, 270)
        vis = r.render(cam.view, cam.proj, cam.W, cam.H)
        r.sync()
        assert_vis_equal(vis, _paper(sc, cam, 128, 32), f"pose {k}")
    del keep


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_views_ray_cast(api, use_graph):
    from test_gpu_parity import _mixed_scene
    sc = _mixed_scene()
    r = _renderer(api, pairs_per_segment=7, stage2_max_pixels=64)
    keep = upload(r, sc)
    views = [(c.view, c.proj, c.W, c.H, None) for c in sc.cameras]
    for frame in range(2):
        out = r.render_batch(views, use_graph=use_graph)
        r.sync()
        for c, v in zip(sc.cameras, out):
            assert_vis_equal(v, _paper(sc, c, 128, 64), f"batched {c.W}x{c.H} frame {frame}")
    del keep


def test_thin_triangle_routed_by_extent(api):
    """A long thin triangle within stage 1's pixel limit leaves stage 1 for its
    64-pixel extent and, past stage2_max_pixels, takes the ray cast."""
    tri = np.array([[-2.6, -0.05, -3.2], [2.5, -0.035, -3.8], [0.1, 0.01, -3.5]], np.float32)
    m = S.Mesh(pos=torch.tensor(tri), idx=torch.tensor([[0, 1, 2]], dtype=torch.int32), rgba8=None)
    sc = Scene([m], [Instance(0, np.eye(4, dtype=np.float32))], [])
    cam = S.Camera(np.eye(4, dtype=np.float32), S.perspective(60, 200 / 60, 0.05, 100.0), 200, 60)
    r = _renderer(api, stage2_max_pixels=32)
    keep = upload(r, sc, with_colour=False)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    r.sync()
    ref = _paper(sc, cam, 128, 32)
    assert (ref != orc.EMPTY).sum() > 20
    assert_vis_equal(vis, ref, "thin triangle")
    assert (ref != orc.render(orc.OracleScene(sc), cam)).any()
    del keep
