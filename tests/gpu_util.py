"""Helpers shared by the GPU tests: upload a synthetic scene to a Renderer
and compare its output with the oracle."""
import numpy as np
import torch

from oracle import oracle as orc


def upload(renderer, scene, with_colour=True, compressed=()):
    """Uploads every mesh of the scene; the meshes numbered in `compressed`
    go up with the Section 4.6 encoding."""
    dev = renderer.device
    keep = []
    for k, m in enumerate(scene.meshes):
        pos = m.pos.to(dev).contiguous()
        idx = m.idx.to(dev).contiguous()
        col = m.rgba8.to(dev).contiguous() if (with_colour and m.rgba8 is not None) else None
        keep.append((pos, idx, col))
        renderer.upload_mesh(pos, idx, col, compressed=k in compressed)
    for it in scene.instances:
        renderer.add_instance(it.mesh, it.model)
    return keep


def u64(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def assert_vis_equal(got, ref, what=""):
    g = u64(got) if isinstance(got, torch.Tensor) else got
    if not np.array_equal(g, ref):
        bad = np.argwhere(g != ref)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} pixels differ from the oracle; first at (x={x}, y={y}): "
                             f"got {int(g[y, x]):#018x} want {int(ref[y, x]):#018x}")


def oracle_vis(scene, cam):
    return orc.render(orc.OracleScene(scene), cam)


def decoded_scene(scene, compressed):
    """The scene as a compressed upload renders it: meshes numbered in
    `compressed` replaced by the oracle's decoding of their encoding."""
    from synthetic.scenes import Mesh, Scene
    meshes = []
    for k, m in enumerate(scene.meshes):
        if k in compressed and m.T > 0:
            _, dpos, didx = orc.compress_mesh(m.pos.numpy(), m.idx.numpy().view(np.uint32))
            m = Mesh(pos=torch.from_numpy(dpos), idx=torch.from_numpy(didx.view(np.int32).reshape(-1, 3)),
                     rgba8=m.rgba8)
        meshes.append(m)
    return Scene(meshes, scene.instances, scene.cameras)
