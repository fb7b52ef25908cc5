"""curast_render_static -- the render for callers that cannot allocate device
memory (for example code running while a CUDA graph is being captured) --
must give the same visibility buffers as the context API, call after call,
even though all its calls share one fixed scratch array.

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
