"""curast_render_static -- the render for callers that cannot allocate device
memory (real-time loops that must not allocate, plug-ins whose host owns all
device memory) -- must give the same visibility buffers as the context API,
call after call, even though all its calls share one fixed scratch array.

This file is collected last on purpose: it needs nothing from the other
tests and passes on its own in a fresh process as well as after them.
"""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _instances():
    out = []
    for k, (x, z, a) in enumerate([(0.0, 0.0, 0.0), (1.1, 0.2, 0.5), (-0.4, 1.3, 2.0)]):
        m = np.eye(4)
        m[:3, :3] = [[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]]
        m[:3, 3] = [x, 0.05 * k, z]
        out.append(m.astype(np.float32))
    return out


def test_static_render_matches_context_render_on_consecutive_calls():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api

    hf = S.heightfield_mesh(96, seed=21)
    pos, idx = hf.pos.cuda(), hf.idx.cuda()
    models = _instances()
    r = api.Renderer(0)
    r.upload_mesh(pos, idx)
    for m in models:
        r.add_instance(0, m)
    cams = [S.Camera(S.look_at((0.4, 1.6, -1.8), (0.5, 0.0, 0.6)), S.perspective(60, 320 / 240, 1e-3, 50.0), 320, 240),
            S.Camera(S.look_at((2.5, 0.5, 2.5), (0.3, 0.0, 0.3)), S.perspective(75, 1.0, 1e-2, 50.0), 200, 200)]
    for cam in cams:   # two calls in a row, different sizes: the shared scratch is reused
        want = r.render(cam.view, cam.proj, cam.W, cam.H)
        r.sync()
        got = api.render_static(pos, idx, models, cam.view, cam.proj, cam.W, cam.H)
        torch.cuda.synchronize()
        assert (want != -1).any()
        assert torch.equal(got, want)      # visibility words are integers: bit-exact


def test_static_render_single_instance_and_limit():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api

    sc = S.scene_small(n=48, W=160, H=120)
    hf = sc.meshes[0]
    cam = sc.cameras[0]
    pos, idx = hf.pos.cuda(), hf.idx.cuda()
    r = api.Renderer(0)
    r.upload_mesh(pos, idx)
    r.add_instance(0)
    for _ in range(2):
        want = r.render(cam.view, cam.proj, cam.W, cam.H)
        r.sync()
        got = api.render_static(pos, idx, None, cam.view, cam.proj, cam.W, cam.H)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
    with pytest.raises(api.CurastError) as e:
        api.render_static(pos, idx, [np.eye(4)] * (api.STATIC_MAX_INSTANCES + 1), cam.view, cam.proj, 8, 8)
    assert e.value.status == -10


def test_static_render_stages_2_3_and_queue_overflow():
    """A camera inside nested closed boxes at 3840 x 2160: every face crosses
    the near plane or the guard band, so stage 2 clips it and stage 3 gets
    tens of thousands of tile parts -- more than the static path's queue 2
    holds (16,384), so its overflow path rasterizes the rest in place.  The
    context renderer, run with the static path's capacities and counters on,
    shows that the workload takes those paths; the static render must still
    equal the context render bit for bit, twice in a row."""
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api

    room = S.scene_room()
    mesh = room.meshes[0]
    pos, idx = mesh.pos.cuda(), mesh.idx.cuda()
    models = []
    for k in range(6):
        m = np.eye(4, dtype=np.float32)
        m[:3, :3] *= np.float32(1.0 + 0.15 * k)
        models.append(m)
    cam = S.Camera(room.cameras[0].view, S.perspective(80, 3840 / 2160, 0.05, 100.0), 3840, 2160)
    probe = api.Renderer(0)
    probe.set_config(queue1_capacity=1 << 16, queue2_capacity=1 << 14, collect_stats=1)
    probe.upload_mesh(pos, idx)
    for m in models:
        probe.add_instance(0, m)
    probe.render(cam.view, cam.proj, cam.W, cam.H)
    st = probe.sync()
    assert st["queued_stage2"] > 0 and st["queued_stage3"] > 0 and st["queue2_overflow"] > 0, st
    r = api.Renderer(0)
    r.upload_mesh(pos, idx)
    for m in models:
        r.add_instance(0, m)
    want = r.render(cam.view, cam.proj, cam.W, cam.H)
    r.sync()
    assert (want != -1).all()
    for _ in range(2):
        got = api.render_static(pos, idx, models, cam.view, cam.proj, cam.W, cam.H)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
