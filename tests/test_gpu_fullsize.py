"""Parity at the full workload sizes, in the launch configuration bench.py
times (default configuration, curast_render / curast_render_batch):

- the billion-triangle terrain (64 tiles of 4096^2 cells, 3840x2160):
  the whole frame against the oracle, tile by tile in a process pool;
- the 100M-triangle heightfield, 8 poses at 1920x1080 and 3840x2160;
- the many-mesh batched workload (256 meshes, 10,000 instances, 4 views):
  batched (graph) against the oracle in full, every pixel of every view;
  batched == one launch per mesh per view; and the same structure at
  reduced size;
- the differentiable workload (1448^2 cells, 1024^2): forward against the
  FP32 oracle, backward against the FP64 adjoint and central differences.

Inputs for the oracle side are generated on the CPU by the same seeded code
that builds them on the GPU; the first test checks that both are identical.
"""
import os
import tempfile

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import oracle as O

import oracle_jobs as J
from gpu_util import assert_vis_equal, u64, upload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def workers():
    p = J.pool()
    yield p
    p.close()
    p.join()


def test_generator_identical_on_cpu_and_gpu():
    a = S.heightfield_mesh(4096, seed=227, device="cpu")
    b = S.heightfield_mesh(4096, seed=227, device="cuda")
    assert torch.equal(a.pos, b.pos.cpu()) and torch.equal(a.idx, b.idx.cpu())
    assert torch.equal(a.rgba8, b.rgba8.cpu())


def test_billion_triangle_frame_bit_exact(api, workers):
    tiles, n, W, H = 8, 4096, 3840, 2160
    sc = S.scene_billion(device="cuda", tiles=tiles, n=n, colours=False)
    cam = S.camera_billion(W, H, tiles)
    r = api.Renderer(0)
    for m in sc.meshes:
        r.upload_mesh(m.pos, m.idx)
    for it in sc.instances:
        r.add_instance(it.mesh, it.model)
    vis = r.render(cam.view, cam.proj, W, H)
    r.sync()
    got = u64(vis)
    info = r.last_frame()
    assert info["pairs"] == 46 and info["triangles"] == 46 * 2 * n * n
    r.close()
    del sc, vis
    torch.cuda.empty_cache()
    # every tile, culled or not: a culled tile must not own a pixel either
    chunks = [list(range(k, tiles * tiles, 16)) for k in range(16)]
    parts = workers.starmap(J.billion_tiles, [(c, tiles, n, W, H) for c in chunks])
    ref = parts[0]
    for p in parts[1:]:
        np.minimum(ref, p, out=ref)
    assert (ref != O.EMPTY).mean() > 0.5
    assert_vis_equal(got, ref, "billion-triangle frame")


def test_unique_100m_all_poses(api, workers):
    n = 7072
    cpu = S.heightfield_mesh(n, seed=100, device="cpu", colours=False)
    tmp = tempfile.mkdtemp(prefix="curast_")
    pp, pi = os.path.join(tmp, "pos.npy"), os.path.join(tmp, "idx.npy")
    np.save(pp, cpu.pos.numpy())
    np.save(pi, cpu.idx.numpy())
    jobs = [(pp, pi, k, W, H) for k in range(8) for (W, H) in ((1920, 1080), (3840, 2160))]
    pending = workers.starmap_async(J.unique_pose, jobs)
    r = api.Renderer(0)
    pos, idx = cpu.pos.cuda(), cpu.idx.cuda()
    del cpu
    r.upload_mesh(pos, idx)
    r.add_instance(0)
    got = []
    for (_, _, k, W, H) in jobs:
        cam = S.camera_unique_pose(k, W, H)
        vis = r.render(cam.view, cam.proj, W, H)
        r.sync()
        got.append(u64(vis))
    refs = pending.get()
    for (_, _, k, W, H), g, ref in zip(jobs, got, refs):
        assert_vis_equal(g, ref, f"pose {k} at {W}x{H}")
    for f in (pp, pi):
        os.unlink(f)
    os.rmdir(tmp)


def _batched_renderer(api, sc):
    r = api.Renderer(0)
    for m in sc.meshes:
        r.upload_mesh(m.pos, m.idx, m.rgba8)
    for it in sc.instances:
        r.add_instance(it.mesh, it.model)
    return r


def test_batched_full_size_equals_per_mesh_launches(api):
    """At full size: the batched launch (replayed from a CUDA graph), the same
    launch without the instanced group test, and one launch per mesh per view
    give identical buffers, and every sampled winning fragment is the
    oracle's fragment of that triangle there."""
    sc = S.scene_batched(device="cuda")
    r = _batched_renderer(api, sc)
    views = [(c.view, c.proj, c.W, c.H, None) for c in sc.cameras]
    out = r.render_batch(views, use_graph=True)
    out = r.render_batch(views, use_graph=True)     # second frame: graph replay
    r.sync()
    cfg = r.config
    r.set_config(stage1_group_min_pairs=0)
    no_group = r.render_batch(views, use_graph=False)
    r.sync()
    for v, w in zip(out, no_group):
        assert torch.equal(v, w), "the group test changed a visibility buffer"
    del no_group
    r.set_config(stage1_group_min_pairs=cfg.stage1_group_min_pairs)
    for c, v in zip(sc.cameras, out):
        plain = r.new_vis(c.W, c.H)
        r.clear(plain)
        for m in range(len(sc.meshes)):
            r.render_mesh(m, c.view, c.proj, c.W, c.H, plain)
        r.sync()
        assert torch.equal(plain, v)
    # sampled winners: re-rasterize the winning triangle alone with the oracle
    bases = np.concatenate([[0], np.cumsum([sc.meshes[i.mesh].T for i in sc.instances])]).astype(np.uint64)
    rng = np.random.default_rng(0)
    for c, v in zip(sc.cameras, out):
        w = u64(v)
        ys, xs = np.nonzero(w != O.EMPTY)
        assert len(ys) > 1000
        for s in rng.choice(len(ys), 64, replace=False):
            y, x = ys[s], xs[s]
            key = w[y, x]
            gid = int(key & O.ID_MASK)
            i = int(np.searchsorted(bases, gid, side="right") - 1)
            t = gid - int(bases[i])
            m = sc.meshes[sc.instances[i].mesh]
            corners = m.pos[m.idx[t].long()].cpu()
            one = S.Scene([S.Mesh(pos=corners, idx=torch.tensor([[0, 1, 2]], dtype=torch.int32))],
                          [S.Instance(0, sc.instances[i].model)])
            ref = O.render(O.OracleScene(one), c)
            assert ref[y, x] != O.EMPTY, "the winning triangle does not cover its pixel"
            assert (ref[y, x] >> np.uint64(36)) == (key >> np.uint64(36)), "depth of the winner differs"
    r.close()


def test_batched_full_size_equals_oracle(api, workers):
    """The many-mesh workload at full size (256 meshes, 10,000 instances, 4
    views, about 9.8e10 triangle-instance-views) rendered by the batched
    launch replayed from its CUDA graph, against the oracle in full: every
    pixel of every view.  The oracle runs in a process pool, each process
    building its share of the meshes on the CPU and rendering all of their
    instances; the shares' buffers merge by an element-wise minimum, which
    is exact because a visibility word is the minimum over all fragments.
    Heightfields are built on the GPU (bit-identical to the CPU build);
    spheres, whose sin/cos may round differently there, are built on the
    CPU and uploaded."""
    specs = S.batched_mesh_specs()
    cams = S.scene_batched(device="cpu", only=set()).cameras
    # shares of about equal work: meshes by triangles x instances, largest first
    inst = np.bincount([it.mesh for it in S.scene_batched(device="cpu", only=set()).instances], minlength=len(specs))
    work = [(sp[3] * int(inst[m]), m) for m, sp in enumerate(specs)]
    nshare = max(1, min(64, (os.cpu_count() or 2) * 2))
    shares = [[] for _ in range(nshare)]
    load = [0] * nshare
    for w, m in sorted(work, reverse=True):
        k = int(np.argmin(load))
        shares[k].append(m)
        load[k] += w
    jobs = [workers.apply_async(J.batched_meshes, (sh,)) for sh in shares if sh]
    sc = S.scene_batched(device="cuda", only={m for m, sp in enumerate(specs) if sp[0] == "heightfield"})
    for m, sp in enumerate(specs):
        if sp[0] == "sphere":
            cpu = S.batched_mesh(sp)
            sc.meshes[m] = S.Mesh(pos=cpu.pos.cuda(), idx=cpu.idx.cuda(), rgba8=cpu.rgba8.cuda(), aabb=cpu.aabb)
    r = _batched_renderer(api, sc)
    out = r.render_batch([(c.view, c.proj, c.W, c.H, None) for c in sc.cameras], use_graph=True)
    out = r.render_batch([(c.view, c.proj, c.W, c.H, o) for c, o in zip(sc.cameras, out)], use_graph=True)
    r.sync()
    got = [u64(v) for v in out]
    r.close()
    del sc, out
    torch.cuda.empty_cache()
    ref = None
    for j in jobs:
        part = j.get(timeout=3000)
        ref = part if ref is None else [np.minimum(a, b) for a, b in zip(ref, part)]
    for c, g, w in zip(cams, got, ref):
        assert (w != O.EMPTY).sum() > 0.5 * c.W * c.H
        assert_vis_equal(g, w, f"batched full size {c.W}x{c.H}")


def test_batched_reduced_equals_oracle(api):
    sc = S.scene_batched(device="cpu", n_meshes=24, n_instances=160, tmin=200, tmax=4e4, area=30.0,
                         views=((480, 270), (480, 270), (240, 136), (240, 136)))
    r = _batched_renderer(api, S.Scene([S.Mesh(m.pos.cuda(), m.idx.cuda(), m.rgba8.cuda()) for m in sc.meshes],
                                       sc.instances, sc.cameras))
    views = [(c.view, c.proj, c.W, c.H, None) for c in sc.cameras]
    out = r.render_batch(views, use_graph=True)
    r.sync()
    osc = O.OracleScene(sc)
    for c, v in zip(sc.cameras, out):
        assert_vis_equal(v, O.render(osc, c), f"batched view {c.W}x{c.H}")


def test_differentiable_full_size(api):
    from oracle import adjoint as A
    sc, col = S.scene_differentiable()
    cam = sc.cameras[0]
    m = sc.meshes[0]
    r = api.Renderer(0)
    pos, idx = m.pos.cuda(), m.idx.cuda()
    r.upload_mesh(pos, idx)
    r.add_instance(0)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    r.sync()
    osc = O.OracleScene(sc)
    ref = O.render(osc, cam)
    assert_vis_equal(vis, ref, "differentiable workload")
    noise = S.target_colour_noise(m.V)
    colc = col.cuda()
    target = r.interpolate(0, cam.view, cam.proj, vis, (col + noise).cuda())
    p = pos.clone().requires_grad_(True)
    c = colc.clone().requires_grad_(True)
    out = api.InterpolateFn.apply(r, 0, p, c, vis, cam.view, cam.proj)
    want, _ = O.interpolate(osc, cam, ref, 0, col.numpy())
    np.testing.assert_allclose(out.detach().cpu().numpy(), want, atol=1e-6, rtol=0)
    loss = ((out - target) ** 2).sum()
    loss.backward()
    fx, fy, _ = O.camera_params(cam.proj)
    mv = O.model_view(cam.view, np.eye(4, dtype=np.float32))
    tri = A.pixel_triangles(u64(vis), 0, m.T)
    g = (2.0 * (out.detach() - target)).cpu().numpy().astype(np.float64).reshape(-1, 3)
    P, I, Cl = m.pos.numpy().astype(np.float64), m.idx.numpy(), col.numpy().astype(np.float64)
    dcol, dpos = A.adjoint64(P, I, Cl, mv, fx, fy, cam.W, cam.H, tri, g)

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    assert rel(c.grad.cpu().numpy(), dcol) <= 1e-4
    assert rel(p.grad.cpu().numpy(), dpos) <= 1e-4
    # central differences of the FP64 forward on 1,000 sampled vertices, step
    # 1e-3 of the grid spacing; only the pixels of the vertex's triangles move
    tgt64 = target.cpu().numpy().astype(np.float64).reshape(-1, 3)
    Tm = I.reshape(-1, 3)
    cov = np.nonzero(tri >= 0)[0]
    order = np.argsort(tri[cov], kind="stable")
    ts, ps = tri[cov][order], cov[order]
    v_tris = {}
    for tt in np.unique(ts):
        for k in range(3):
            v_tris.setdefault(int(Tm[tt, k]), []).append(int(tt))
    lo, hi = np.searchsorted(ts, np.arange(m.T)), np.searchsorted(ts, np.arange(m.T), side="right")
    rng = np.random.default_rng(1)
    h = 1e-3 / 1448
    fd, an = [], []
    for v in rng.choice(np.array(sorted(v_tris)), 1000, replace=False):
        pix = np.concatenate([ps[lo[t]:hi[t]] for t in v_tris[v]])

        def L(q):
            return A.loss_at_pixels64(q, I, Cl, mv, fx, fy, cam.W, cam.H, pix, tri[pix], tgt64[pix])

        for ax in range(3):
            orig = P[v, ax]
            P[v, ax] = orig + h
            lp = L(P)
            P[v, ax] = orig - h
            lm = L(P)
            P[v, ax] = orig
            fd.append((lp - lm) / (2 * h))
            an.append(dpos[v, ax])
    fd, an = np.array(fd), np.array(an)
    assert rel(fd, an) <= 1e-4
