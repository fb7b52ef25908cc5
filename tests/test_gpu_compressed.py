"""Compressed geometry (Section 4.6) through the C ABI: the device encoding
equals the oracle's, and compressed meshes render bit-exactly what the
oracle renders from the decoded meshes -- alone, mixed with uncompressed
meshes, batched over several views and over several stage-1 rounds."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import oracle as orc

from gpu_util import assert_vis_equal, decoded_scene, oracle_vis, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api as A
    return A


class _DeviceArray:
    """A view of a device buffer by pointer (CUDA array interface); only read."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False), "version": 2}


def _device_words(ptr, n, typestr):
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda").cpu().numpy().copy()


def test_device_encoding_equals_oracle(api):
    sc = S.scene_small()
    r = api.Renderer(0)
    keep = upload(r, sc, compressed={0, 1})
    for k, m in enumerate(sc.meshes):
        info = r.mesh_info(k)
        f, _, _ = orc.compress_mesh(m.pos.numpy(), m.idx.numpy().view(np.uint32))
        assert info["compressed"] == 1
        assert info["index_bits"] == f["bits"] and info["index_min"] == f["imin"]
        np.testing.assert_array_equal(np.array(info["pos_lo"], np.float32), f["lo"])
        np.testing.assert_array_equal(np.array(info["pos_step"], np.float32), f["step"])
        nw = (3 * m.T * f["bits"] + 31) // 32
        words = _device_words(info["packed_indices"], nw, "<u4")
        np.testing.assert_array_equal(words, f["words"][:nw])
        q = _device_words(info["quantized_positions"], 3 * m.V, "<u2")
        np.testing.assert_array_equal(q.reshape(-1, 3), f["q"])
        assert info["geometry_bytes"] == 4 * nw + 6 * m.V
    del keep


def test_compressed_small_scene_equals_decoded_oracle(api):
    """The heightfield and the near-crossing ground triangles compressed:
    every stage (1, 2, 3) and the resolve run on the decoded geometry."""
    sc = S.scene_small()
    cam = sc.cameras[0]
    r = api.Renderer(0)
    r.set_config(collect_stats=1)
    keep = upload(r, sc, compressed={0, 1})
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    f32, u8 = r.resolve(cam.view, cam.proj, vis)
    st = r.sync()
    dsc = decoded_scene(sc, {0, 1})
    osc = orc.OracleScene(dsc)
    ref = orc.render(osc, cam)
    assert_vis_equal(vis, ref, "compressed small scene")
    rf, r8 = orc.resolve(osc, cam, ref)
    np.testing.assert_allclose(f32.cpu().numpy(), rf, atol=1e-6, rtol=0)
    np.testing.assert_array_equal(u8.cpu().numpy(), r8)
    assert st["stage1_rasterized"] > 0 and st["queued_stage2"] > 0
    del keep


@pytest.mark.parametrize("use_graph,bitmap", [(False, 1 << 32), (True, 1 << 32), (True, 1 << 12)])
def test_mixed_compressed_batched(api, use_graph, bitmap):
    """Compressed and uncompressed meshes in one batched frame (their
    stage-1 rounds kept apart), three views, graph replay, several rounds."""
    from test_gpu_parity import _mixed_scene
    sc = _mixed_scene()
    comp = {0, 2}
    r = api.Renderer(0)
    r.set_config(pairs_per_segment=7, stage1_bitmap_bytes=bitmap)
    keep = upload(r, sc, compressed=comp)
    views = [(c.view, c.proj, c.W, c.H, None) for c in sc.cameras]
    dsc = decoded_scene(sc, comp)
    for frame in range(2):
        out = r.render_batch(views, use_graph=use_graph)
        r.sync()
        for c, v in zip(sc.cameras, out):
            assert_vis_equal(v, oracle_vis(dsc, c), f"view {c.W}x{c.H} frame {frame}")
    assert r.last_frame()["rounds"] >= 2
    del keep


def test_compressed_tiles_equal_decoded_oracle(api):
    """Two heightfield tiles of 384^2 cells compressed, the overview camera
    of the billion-triangle layout scaled down."""
    sc = S.scene_billion(tiles=2, n=384)
    cam = S.camera_billion(640, 360, 2)
    r = api.Renderer(0)
    keep = upload(r, sc, compressed={0, 1, 2, 3})
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    r.sync()
    assert_vis_equal(vis, oracle_vis(decoded_scene(sc, {0, 1, 2, 3}), cam), "compressed tiles")
    del keep


def test_compressed_mesh_limits(api):
    sc = S.scene_small()
    r = api.Renderer(0)
    keep = upload(r, sc, compressed={0})
    m = sc.meshes[0]
    with pytest.raises(api.CurastError):
        r.update_mesh(0, pos=m.pos.cuda())
    cam = sc.cameras[0]
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    col = torch.zeros((m.V, 3), device="cuda")
    with pytest.raises(api.CurastError):
        r.interpolate(0, cam.view, cam.proj, vis, col)
    bad = m.idx.clone()
    bad[5, 1] = m.V
    with pytest.raises(api.CurastError):
        r.upload_mesh(m.pos.cuda(), bad.cuda(), compressed=True)
    del keep


def _grid_flags_expected(idx: np.ndarray, V: int) -> np.ndarray:
    """The grid flags by their definition: group G of 128 triangles is set
    when it lies wholly in the mesh and every run of four triangles of it is
    the strip of two grid rows, (s0 s1 s2) (s2 s1 s3) (s2 s3 s4) (s4 s3 s5)
    with s2 = s0 + 1, s4 = s0 + 2, s3 = s1 + 1, s5 = s1 + 2, all below V."""
    T = idx.shape[0]
    ng = (T + 127) // 128
    words = np.zeros((ng + 31) // 32, np.uint32)
    x = idx.astype(np.int64)
    for G in range(T // 128):
        r = x[128 * G:128 * G + 128].reshape(32, 12)
        s0, s1 = r[:, 0], r[:, 1]
        pat = np.stack([s0, s1, s0 + 1, s0 + 1, s1, s1 + 1, s0 + 1, s1 + 1, s0 + 2, s0 + 2, s1 + 1, s1 + 2], 1)
        if np.array_equal(r, pat) and (s0 + 2 < V).all() and (s1 + 2 < V).all():
            words[G // 32] |= np.uint32(1 << (G % 32))
    return words


def _grid_meshes():
    """Grid meshes whose 128-triangle groups are all, some or none grid rows:
    an even row of 96 cells (every group), an odd row of 97 cells (groups
    whose runs straddle two rows are not), the 96-cell grid in shuffled
    triangle order (none), and the 96-cell grid with one triangle of group 5
    stretched to a far vertex (every group but that one)."""
    a = S.heightfield_mesh(96, seed=5)
    b = S.heightfield_mesh(97, seed=6)
    g = torch.Generator().manual_seed(7)
    c = S.Mesh(pos=a.pos.clone(), idx=a.idx[torch.randperm(a.T, generator=g)].contiguous(), rgba8=a.rgba8.clone(),
               aabb=a.aabb)
    d_idx = a.idx.clone()
    d_idx[5 * 128 + 9, 2] = a.V - 1
    d = S.Mesh(pos=a.pos.clone(), idx=d_idx, rgba8=a.rgba8.clone(), aabb=a.aabb)
    return [a, b, c, d]


def test_grid_flags_follow_their_definition(api):
    meshes = _grid_meshes()
    r = api.Renderer(0)
    keep = [(m.pos.cuda(), m.idx.cuda(), m.rgba8.cuda()) for m in meshes]
    for p, i, c in keep:
        r.upload_mesh(p, i, c, compressed=True)
    got = []
    for k, m in enumerate(meshes):
        info = r.mesh_info(k)
        exp = _grid_flags_expected(m.idx.numpy().view(np.uint32), m.V)
        words = _device_words(info["grid_flags"], exp.size, "<u4")
        np.testing.assert_array_equal(words, exp, err_msg=f"mesh {k}")
        got.append(int(np.unpackbits(exp.view(np.uint8)).sum()))
    ng = [(m.T + 127) // 128 for m in meshes]
    assert got[0] == ng[0] and 0 < got[1] < ng[1] and got[2] == 0 and got[3] == ng[3] - 1
    del keep


def test_grid_groups_render_as_decoded_oracle(api):
    """Each mesh of _grid_meshes alone (single-pair frames, so the strip cull
    of compressed meshes runs), seen from above and obliquely: bit-exact
    against the oracle on the decoded mesh."""
    for k, m in enumerate(_grid_meshes()):
        sc = S.Scene(meshes=[m], instances=[S.Instance(0, np.eye(4, dtype=np.float32))])
        for eye, target in (((0.5, 1.4, 0.5), (0.5, 0.0, 0.501)), ((-0.4, 0.6, -0.3), (0.5, 0.05, 0.5))):
            cam = S.Camera(S.look_at(eye, target), S.perspective(60.0, 320 / 240, 1e-3, 100.0), 320, 240)
            r = api.Renderer(0)
            keep = upload(r, sc, compressed={0})
            vis = r.render(cam.view, cam.proj, cam.W, cam.H)
            r.sync()
            assert_vis_equal(vis, oracle_vis(decoded_scene(sc, {0}), cam), f"mesh {k}")
            del keep
