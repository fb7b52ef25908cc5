"""Differentiable interpolation on the GPU: forward vs the FP32 oracle
(1e-6 absolute), backward vs the FP64 adjoint (1e-4 relative, normwise per
tensor) and through torch.autograd."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import adjoint as A
from oracle import oracle as orc

from gpu_util import assert_vis_equal, u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2604_21749_gb300 import api as A_
    return A_


def _setup(api, n=96, W=192, H=160):
    sc, col = S.scene_differentiable(n=n, W=W, H=H)
    cam = sc.cameras[0]
    m = sc.meshes[0]
    r = api.Renderer(0)
    pos, idx = m.pos.cuda(), m.idx.cuda()
    r.upload_mesh(pos, idx)
    r.add_instance(0)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    r.sync()
    return sc, col, cam, r, pos, idx, vis


def rel_err(got, ref):
    return np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)


def test_forward_matches_oracle(api):
    sc, col, cam, r, pos, idx, vis = _setup(api)
    osc = orc.OracleScene(sc)
    ref = orc.render(osc, cam)
    assert_vis_equal(vis, ref, "differentiable scene")
    out = r.interpolate(0, cam.view, cam.proj, vis, col.cuda())
    want, _ = orc.interpolate(osc, cam, ref, 0, col.numpy())
    np.testing.assert_allclose(out.cpu().numpy(), want, atol=1e-6, rtol=0)


def test_backward_matches_fp64_adjoint(api):
    sc, col, cam, r, pos, idx, vis = _setup(api)
    m = sc.meshes[0]
    tgt = torch.rand((cam.H, cam.W, 3), generator=torch.Generator().manual_seed(3))
    colc = col.cuda()
    out = r.interpolate(0, cam.view, cam.proj, vis, colc)
    g = 2.0 * (out - tgt.cuda())
    gc, gp = r.interpolate_backward(0, cam.view, cam.proj, vis, colc, g)
    fx, fy, _ = orc.camera_params(cam.proj)
    mv = orc.model_view(cam.view, np.eye(4, dtype=np.float32))
    tri = A.pixel_triangles(u64(vis), 0, m.T)
    dcol, dpos = A.adjoint64(m.pos.numpy(), m.idx.numpy(), col.numpy(), mv, fx, fy, cam.W, cam.H, tri,
                             g.cpu().numpy().astype(np.float64).reshape(-1, 3))
    assert rel_err(gc.cpu().numpy(), dcol) <= 1e-4
    assert rel_err(gp.cpu().numpy(), dpos) <= 1e-4
    big = np.abs(dpos) > 1e-3 * np.abs(dpos).max()
    np.testing.assert_allclose(gp.cpu().numpy()[big], dpos[big], rtol=2e-3)


def test_autograd_function(api):
    sc, col, cam, r, pos, idx, vis = _setup(api, n=48, W=96, H=80)
    p = pos.clone().requires_grad_(True)
    c = col.cuda().requires_grad_(True)
    out = api.InterpolateFn.apply(r, 0, p, c, vis, cam.view, cam.proj)
    tgt = torch.full_like(out, 0.5)
    loss = ((out - tgt) ** 2).sum()
    loss.backward()
    gc, gp = r.interpolate_backward(0, cam.view, cam.proj, vis, col.cuda(), 2.0 * (out.detach() - tgt), pos=pos)
    np.testing.assert_allclose(c.grad.cpu().numpy(), gc.cpu().numpy(), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(p.grad.cpu().numpy(), gp.cpu().numpy(), rtol=1e-4, atol=1e-5)
