"""GPU path vs the oracle through the C ABI: visibility buffers bit-exact,
resolved colours within 1e-6 (FP32, same operation order)."""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import oracle as orc
from synthetic.scenes import Camera, Instance, Mesh, Scene

from gpu_util import assert_vis_equal, oracle_vis, u64, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api as A
    return A


def _renderer(api, **cfg):
    r = api.Renderer(0)
    if cfg:
        r.set_config(**cfg)
    return r


@pytest.fixture(scope="module")
def small():
    return S.scene_small()


def test_small_workload_bit_exact_and_resolve(api, small):
    """Heightfield of 256^2 cells + 2 near-crossing ground triangles, 512^2."""
    cam = small.cameras[0]
    r = _renderer(api, collect_stats=1)
    keep = upload(r, small)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    f32, u8 = r.resolve(cam.view, cam.proj, vis)
    st = r.sync()
    osc = orc.OracleScene(small)
    ref = orc.render(osc, cam)
    assert_vis_equal(vis, ref, "small")
    rf, r8 = orc.resolve(osc, cam, ref)
    np.testing.assert_allclose(f32.cpu().numpy(), rf, atol=1e-6, rtol=0)
    np.testing.assert_array_equal(u8.cpu().numpy(), r8)
    # every stage took part: the ground triangles cross the near plane
    assert st["stage1_rasterized"] > 0 and st["queued_stage2"] > 0 and st["queued_stage3"] > 0
    assert st["triangles_in"] == small.total_triangles
    del keep


@pytest.mark.parametrize("cfg", [
    dict(stage1_max_pixels=1), dict(stage1_max_pixels=1024, stage2_max_pixels=32),
    dict(stage2_max_pixels=1 << 30), dict(tile_log2=4), dict(tile_log2=7),
    dict(stage1_tri_per_thread=1), dict(stage1_tri_per_thread=3),
    dict(queue1_capacity=1, queue2_capacity=1), dict(queue1_capacity=7, queue2_capacity=3),
    dict(stage1_bitmap_bytes=1 << 12), dict(stage1_bitmap_bytes=1 << 12, stage1_tri_per_thread=1),
    dict(stage1_exact_all=1), dict(stage1_exact_all=1, stage1_bitmap_bytes=1 << 12),
    dict(stage1_vertex_reuse=1), dict(stage1_vertex_reuse=1, stage1_tri_per_thread=3),
    dict(stage3_tile_buffer=1), dict(stage3_tile_buffer=1, tile_log2=4), dict(stage3_tile_buffer=1, tile_log2=7),
])
def test_stage_choices_never_change_visibility(api, small, cfg):
    """Thresholds, tile size, batch shape and queue overflow move triangles
    between stages but the buffer stays bit-identical."""
    cam = small.cameras[0]
    r = _renderer(api, **cfg)
    keep = upload(r, small)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    st = r.sync()
    assert_vis_equal(vis, oracle_vis(small, cam), str(cfg))
    if cfg.get("queue1_capacity", 1 << 30) < 2:
        assert st["queue1_overflow"] > 0
    if cfg.get("stage1_bitmap_bytes", 1 << 30) < 1 << 14:
        assert r.last_frame()["rounds"] > 1          # stage 1 ran in several cull + exact rounds
    del keep


@pytest.mark.parametrize("ss", [1, 2, 4])
def test_supersampled_resolve_equals_oracle(api, small, ss):
    """Super sampling: the view rendered at ss times the resolution per axis
    (bit-exact), box-filtered by curast_resolve_ss (within 1e-6, RGBA8 equal)."""
    cam = small.cameras[0]
    fine = Camera(cam.view, cam.proj, ss * cam.W, ss * cam.H)
    r = _renderer(api)
    keep = upload(r, small)
    vis = r.render(fine.view, fine.proj, fine.W, fine.H)
    f32, u8 = r.resolve_ss(cam.view, cam.proj, vis, ss)
    r.sync()
    osc = orc.OracleScene(small)
    ref = orc.render(osc, fine)
    assert_vis_equal(vis, ref, f"ss={ss}")
    rf, r8 = orc.resolve_ss(osc, fine, ref, ss)
    np.testing.assert_allclose(f32.cpu().numpy(), rf, atol=1e-6, rtol=0)
    np.testing.assert_array_equal(u8.cpu().numpy(), r8)
    if ss == 1:
        g32, g8 = r.resolve(cam.view, cam.proj, vis)
        assert torch.equal(g32, f32) and torch.equal(g8, u8)
    del keep


def _mixed_scene():
    meshes = [S.heightfield_mesh(40, seed=11), S.sphere_mesh(12, seed=12), S.heightfield_mesh(7, seed=13),
              Mesh(pos=torch.zeros((3, 3)), idx=torch.zeros((0, 3), dtype=torch.int32),
                   rgba8=torch.zeros((3, 4), dtype=torch.uint8)), S.ground_mesh(half=30.0, y=-0.3)]
    rng = np.random.default_rng(3)
    inst = []
    for k in range(40):
        m = [0, 1, 2, 3, 1][k % 5]
        M = np.eye(4)
        a = rng.uniform(0, 2 * np.pi)
        M[:3, :3] = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]]) * rng.uniform(0.3, 1.5)
        M[:3, 3] = [rng.uniform(-4, 4), rng.uniform(-0.2, 0.5), rng.uniform(-4, 4)]
        inst.append(Instance(m, M.astype(np.float32)))
    inst.append(Instance(4, np.eye(4, dtype=np.float32)))
    cams = [Camera(S.look_at((0.0, 2.5, -7.0), (0, 0, 0)), S.perspective(60, 320 / 200, 0.05, 100.0), 320, 200),
            Camera(S.look_at((5.0, 1.0, 1.0), (-1, 0, 0)), S.perspective(75, 1.0, 0.02, 100.0), 160, 160),
            Camera(S.look_at((0.5, 0.4, 0.5), (3, 0, 2)), S.perspective(90, 2.0, 0.01, 100.0), 257, 129)]
    return Scene(meshes, inst, cams)


@pytest.fixture(scope="module")
def mixed():
    return _mixed_scene()


@pytest.mark.parametrize("use_graph,bitmap,exact_all", [(False, 1 << 30, 0), (True, 1 << 30, 0), (True, 1 << 12, 0),
                                                        (True, 1 << 30, 1)])
def test_batched_views_equal_oracle(api, mixed, use_graph, bitmap, exact_all):
    """Many meshes, rotated/scaled instances (some culled), an empty mesh and
    three views of different sizes in one batched launch (graph or not; one
    stage-1 round or several; with or without the conservative cull)."""
    r = _renderer(api, pairs_per_segment=7, stage1_bitmap_bytes=bitmap, stage1_exact_all=exact_all)
    keep = upload(r, mixed)
    views = [(c.view, c.proj, c.W, c.H, None) for c in mixed.cameras]
    for frame in range(2):   # the second frame replays the captured graph
        out = r.render_batch(views, use_graph=use_graph)
        r.sync()
        for c, v in zip(mixed.cameras, out):
            assert_vis_equal(v, oracle_vis(mixed, c), f"view {c.W}x{c.H} frame {frame}")
    del keep


@pytest.fixture(scope="module")
def many_small():
    """The many-mesh workload's structure scaled down: 16 meshes of 2e3..5e4
    triangles, 200 randomly rotated instances of scale 0.1..10 over a
    200 x 200 area, two views; most instances cover a few pixels, so many of
    the instanced cull's groups hold no pixel centre and the rest do."""
    return S.scene_batched(n_meshes=16, n_instances=200, tmin=2e3, tmax=5e4,
                           views=((640, 360), (320, 180)), seed=31)


@pytest.mark.parametrize("pps,group_min", [(1, 2), (3, 2), (64, 2), (64, 1), (64, 0)])
def test_many_small_instances_equal_oracle(api, many_small, pps, group_min):
    """Instanced items test each step's triangles per pair as a group first
    (one to 64 pairs an item; from 1 or 2 pairs, or never); the buffers stay
    identical to the oracle's."""
    r = _renderer(api, pairs_per_segment=pps, collect_stats=1, stage1_group_min_pairs=group_min)
    keep = upload(r, many_small, with_colour=False)
    views = [(c.view, c.proj, c.W, c.H, None) for c in many_small.cameras]
    out = r.render_batch(views, use_graph=False)
    st = r.sync()
    for c, v in zip(many_small.cameras, out):
        assert_vis_equal(v, oracle_vis(many_small, c), f"many small instances {c.W}x{c.H} pps {pps}")
    assert st["culled_tiny"] > 0 and st["stage1_rasterized"] > 0
    del keep


def test_per_mesh_launches_equal_oracle(api, mixed):
    """The one-launch-per-mesh-per-view path composes to the same buffer."""
    r = _renderer(api)
    keep = upload(r, mixed)
    for c in mixed.cameras:
        vis = r.new_vis(c.W, c.H)
        r.clear(vis)
        for m in range(len(mixed.meshes)):
            r.render_mesh(m, c.view, c.proj, c.W, c.H, vis)
        r.sync()
        assert_vis_equal(vis, oracle_vis(mixed, c), f"per-mesh {c.W}x{c.H}")
    del keep


def _permuted(mesh, seed):
    """The same mesh with its triangles in a seeded random order (vertex
    indices scattered over the whole mesh within every work item)."""
    perm = np.random.default_rng(seed).permutation(mesh.idx.shape[0])
    return Mesh(pos=mesh.pos, idx=mesh.idx[torch.from_numpy(perm)].contiguous(), rgba8=mesh.rgba8)


@pytest.mark.parametrize("tpt", [4, 3, 1])
def test_vertex_windows_edge_cases(api, tpt):
    """The single-pair cull stages the vertex ranges of each work item in
    shared memory.  Items that straddle grid rows (300 cells a row), a mesh
    whose triangles come in random order (the windows are dropped), a
    position buffer that starts off a 16-byte boundary (no bulk copy), a
    mesh of 3 vertices (below the 4-vertex copy granule) and the 4-vertex
    ground quad: each equal to the oracle, with and without vertex reuse."""
    hf = S.heightfield_mesh(300, seed=100)
    tiny = Mesh(pos=torch.tensor([[0.2, 0.01, 0.2], [0.8, 0.01, 0.3], [0.5, 0.02, 0.9]], dtype=torch.float32),
                idx=torch.tensor([[0, 2, 1]], dtype=torch.int32))
    meshes = [hf, _permuted(S.heightfield_mesh(150, seed=7), 3), tiny, S.ground_mesh()]
    sc = Scene(meshes, [Instance(k, np.eye(4, dtype=np.float32)) for k in range(len(meshes))])
    cams = [S.camera_unique_pose(k, 480, 270) for k in (0, 3, 6)]
    refs = [oracle_vis(sc, c) for c in cams]
    for reuse in (1, 0):
        r = _renderer(api, stage1_tri_per_thread=tpt, stage1_vertex_reuse=reuse)
        keep = []
        for k, m in enumerate(meshes):
            pos = m.pos.cuda().contiguous()
            if k == 0:                               # the same floats, 4 bytes past a 16-byte boundary
                buf = torch.empty(pos.numel() + 1, dtype=torch.float32, device="cuda")
                buf[1:] = pos.reshape(-1)
                pos = buf[1:].view(-1, 3)
                assert pos.data_ptr() % 16 == 4
            idx = m.idx.cuda().contiguous()
            keep.append((pos, idx))
            r.upload_mesh(pos, idx)
        for it in sc.instances:
            r.add_instance(it.mesh, it.model)
        for c, ref in zip(cams, refs):
            vis = r.render(c.view, c.proj, c.W, c.H)
            r.sync()
            assert_vis_equal(vis, ref, f"tpt {tpt} reuse {reuse} {c.W}x{c.H}")
        del keep


@pytest.mark.parametrize("tile_log2", [4, 6, 7])
def test_stage3_tile_buffer_room_and_close_ups(api, tile_log2):
    """Stage-3 workloads -- the camera inside a closed box (every face clipped
    and split into tile parts over the whole screen) and close-up poses with
    stage2_max_pixels = 32 (many mid-sized triangles, tens of parts a tile) --
    with the shared-memory tile buffer and without it, each equal to the
    oracle; with queue 2 of capacity 5 the overflow path joins in."""
    room = S.scene_room()
    hf = S.heightfield_mesh(300, seed=100)
    close = Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))], [])
    cases = [(room, c) for c in room.cameras] + [(close, S.camera_unique_pose(k, 480, 270)) for k in (0, 3, 5)]
    refs = [oracle_vis(sc, c) for sc, c in cases]
    for cfg in (dict(stage3_tile_buffer=1), dict(stage3_tile_buffer=0), dict(stage3_tile_buffer=1, queue2_capacity=5)):
        for (sc, c), ref in zip(cases, refs):
            r = _renderer(api, tile_log2=tile_log2, stage2_max_pixels=32, collect_stats=1, **cfg)
            keep = upload(r, sc)
            vis = r.render(c.view, c.proj, c.W, c.H)
            st = r.sync()
            assert st["queued_stage3"] > 0
            assert_vis_equal(vis, ref, f"{cfg} tile 2^{tile_log2} {c.W}x{c.H}")
            del keep


def test_unique_heightfield_poses_reduced(api):
    """The 100M-triangle workload's structure at 600^2 cells: 8 seeded poses
    from whole-mesh views to close-ups."""
    sc = S.scene_unique(n=600)
    r = _renderer(api)
    keep = upload(r, sc)
    osc = orc.OracleScene(sc)
    for k in range(8):
        cam = S.camera_unique_pose(k, 480, 270)
        vis = r.render(cam.view, cam.proj, cam.W, cam.H)
        r.sync()
        assert_vis_equal(vis, orc.render(osc, cam), f"pose {k}")
    del keep


def test_tiled_terrain_reduced(api):
    """The billion-triangle workload's layout (8 x 8 tiles, frustum culls
    some) at 48^2 cells per tile."""
    sc = S.scene_billion(n=48)
    cam = S.camera_billion(W=384, H=216)
    r = _renderer(api)
    keep = upload(r, sc)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    r.sync()
    assert_vis_equal(vis, oracle_vis(sc, cam), "tiles")
    del keep


def test_edge_cases(api):
    """1x1 and odd sizes, no instances, only an empty mesh."""
    r = _renderer(api)
    hf = S.heightfield_mesh(16, seed=5)
    keep = upload(r, Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))]))
    cam = S.scene_small().cameras[0]
    for W, H in [(1, 1), (3, 517), (1023, 2)]:
        vis = r.render(cam.view, S.perspective(60, W / H, 1e-3, 10), W, H)
        r.sync()
        ref = oracle_vis(Scene([hf], [Instance(0, np.eye(4, dtype=np.float32))]), Camera(cam.view, S.perspective(60, W / H, 1e-3, 10), W, H))
        assert_vis_equal(vis, ref, f"{W}x{H}")
    r.clear_instances()
    vis = r.render(cam.view, cam.proj, 64, 64)
    r.sync()
    assert (u64(vis) == orc.EMPTY).all()
    del keep


def test_out_of_range_index_is_reported(api):
    r = _renderer(api)
    hf = S.heightfield_mesh(8, seed=5)
    idx = hf.idx.clone()
    idx[5, 1] = hf.V + 1000
    pos, idx_d = hf.pos.cuda(), idx.cuda()
    r.upload_mesh(pos, idx_d)
    r.add_instance(0)
    cam = S.scene_small().cameras[0]
    r.render(cam.view, cam.proj, 64, 64)
    with pytest.raises(api.CurastError) as e:
        r.sync()
    assert e.value.status == -4
    # the error is latched once; the context keeps working
    r.sync()


def test_invalid_arguments_rejected(api):
    r = _renderer(api)
    cam = S.scene_small().cameras[0]
    bad = cam.proj.copy()
    bad[0, 2] = 0.5
    with pytest.raises(api.CurastError):
        r.render(cam.view, bad, 8, 8)
    v = cam.view.copy()
    v[3, 0] = 1.0
    with pytest.raises(api.CurastError):
        r.render(v, cam.proj, 8, 8)
    with pytest.raises(api.CurastError):
        r.set_config(tile_log2=9)
    with pytest.raises(api.CurastError):
        r.set_config(stage1_group_min_pairs=65)


def test_autotune_keeps_result(api, mixed):
    r = _renderer(api)
    keep = upload(r, mixed)
    views = [(c.view, c.proj, c.W, c.H, r.new_vis(c.W, c.H)) for c in mixed.cameras]
    cfg = r.autotune(views)
    assert cfg["stage1_max_pixels"] >= 1
    out = r.render_batch([(c.view, c.proj, c.W, c.H, None) for c in mixed.cameras])
    r.sync()
    for c, v in zip(mixed.cameras, out):
        assert_vis_equal(v, oracle_vis(mixed, c), "after autotune")
    del keep
