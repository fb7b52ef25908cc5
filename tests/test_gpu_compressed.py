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
