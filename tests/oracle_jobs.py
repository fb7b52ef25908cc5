"""Oracle jobs for a spawn process pool (full-size parity tests).

Each job generates its inputs with the seeded generators (bit-identical to
the GPU-side generation) or maps them from .npy files, runs the C oracle on
its share of the scene and returns a visibility buffer; the caller merges
shares with an element-wise minimum, which is exact because the buffer is a
per-pixel minimum over all fragments.
"""
import os

import numpy as np


def _init():
    import torch
    torch.set_num_threads(1)


def pool(n=None):
    import multiprocessing as mp
    n = n or max(1, min(16, (os.cpu_count() or 2)))
    return mp.get_context("spawn").Pool(n, initializer=_init)


def billion_tiles(tiles_k, tiles, n, W, H):
    """Renders the given tiles of the tiled terrain with ids numbered over all
    tiles; returns the min-merged buffer."""
    import synthetic as S
    from oracle import oracle as O
    cam = S.camera_billion(W, H, tiles)
    out = np.full((H, W), O.EMPTY, np.uint64)
    counts = [2 * n * n] * (tiles * tiles)
    for k in tiles_k:
        sc = S.scene_billion(tiles=tiles, n=n, only=[k], colours=False)
        osc = O.OracleScene(sc, tri_counts=counts)
        O.render(osc, cam, first=k, count=1, out=out)
        del sc, osc
    return out


def unique_pose(path_pos, path_idx, k, W, H):
    """One pose of the single large heightfield (inputs memory-mapped)."""
    import torch
    import synthetic as S
    from oracle import oracle as O
    from synthetic.scenes import Instance, Mesh, Scene
    pos = np.load(path_pos, mmap_mode="r")
    idx = np.load(path_idx, mmap_mode="r")
    m = Mesh(pos=torch.from_numpy(np.asarray(pos)), idx=torch.from_numpy(np.asarray(idx)))
    sc = Scene([m], [Instance(0, np.eye(4, dtype=np.float32))])
    cam = S.camera_unique_pose(k, W, H)
    return O.render(O.OracleScene(sc), cam)


def batched_meshes(mesh_ids):
    """The many-mesh workload's instances of the given meshes rendered into
    every view (ids numbered over all instances, as in the full scene); the
    meshes are built here on the CPU.  Returns one buffer per view."""
    import synthetic as S
    from oracle import oracle as O
    specs = S.batched_mesh_specs()
    sc = S.scene_batched(device="cpu", only=set(mesh_ids))
    osc = O.OracleScene(sc, tri_counts=[sp[3] for sp in specs])
    cams = [c for c in sc.cameras]
    out = [np.full((c.H, c.W), O.EMPTY, np.uint64) for c in cams]
    for i, it in enumerate(sc.instances):
        if it.mesh in mesh_ids:
            for c, buf in zip(cams, out):
                O.render(osc, c, first=i, count=1, out=buf)
    return out
