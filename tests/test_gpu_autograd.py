"""HandRenderLoss, the torch.autograd.Function around one refinement iteration:
loss.backward() through the hand-written adjoint kernels (re-traced samples, then
the skinning adjoint) against the oracle's whole chain on the same seeded inputs:
oracle.skin -> render_fwd -> loss -> render_bwd (interior + edges + normals) ->
skin_bwd.  Bars: the loss to 1e-4 relative (the per-pixel bar), each of the 61 gradient entries to the
per-entry gradient tolerance (1e-3 relative, floor 1e-3 of the largest entry).

The Function skins on the GPU, so its vertices differ from the oracle's float64
skinning rounded to float32 by float32 rounding (below 2e-6 m, checked
separately); the 61-entry gradient sums over every traced sample and every edge
sample, so the rare sample whose hit that rounding could decide moves it far less
than the bar."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import grad_ok, hand, require_gpu, scene, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    require_gpu()
    from paper_2107_05509_gb300 import binding
    return binding


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _refiner(B, sc):
    from paper_2107_05509_gb300 import pipeline as P
    h = hand()
    views = P.Views(cams=_t(sc.cams), background=_t(sc.bg), observed=_t(sc.observed), mask=_t(sc.mask),
                    H=sc.H, W=sc.W)
    opts = sc.gpu_opts(sc.opts(), B.HR_BWD_REUSE_FWD)
    return P.Refiner(B.Model(h), views, opts)


def _oracle_chain(sc, x):
    h = hand()
    verts = oracle.skin(h, x).astype(np.float32)
    normals = oracle.vertex_normals(verts, h.faces, h.vf_offsets, h.vf_faces)
    o = sc.opts()
    img = oracle.render_fwd(verts, h.faces, normals, h.albedo, sc.cams, sc.H, sc.W, sc.bg, o).astype(np.float32)
    L, A = oracle.loss(img, sc.observed, sc.mask)
    dV, _ = oracle.render_bwd(h, verts, sc.cams, sc.H, sc.W, sc.bg, o, A.astype(np.float32), normals=normals)
    return L, oracle.skin_bwd(h, x, dV)


@pytest.mark.parametrize("name", ["tiny", "ragged"])
def test_loss_backward_matches_oracle_chain(B, name):
    from paper_2107_05509_gb300.pipeline import HandRenderLoss
    sc = scene(name)
    x = sc.x0.astype(np.float32)
    L_ref, g_ref = _oracle_chain(sc, x.astype(np.float64))
    ref = _refiner(B, sc)

    p = _t(x).requires_grad_(True)
    loss = HandRenderLoss.apply(p, ref)
    assert loss.shape == () and loss.requires_grad
    loss.backward()
    assert abs(loss.item() - L_ref) <= 1e-4 * abs(L_ref)
    g = p.grad.cpu().numpy().astype(np.float64)
    ok = grad_ok(g, g_ref)
    assert np.abs(g_ref).max() > 0
    assert ok.all(), (np.argwhere(~ok).ravel(), g[~ok], g_ref[~ok])

    # a constant factor on the loss scales the gradient (the chain rule's grad_out)
    q = _t(x).requires_grad_(True)
    (-2.5 * HandRenderLoss.apply(q, ref)).backward()
    gq = q.grad.cpu().numpy().astype(np.float64)
    ok = grad_ok(gq, -2.5 * g_ref)
    assert ok.all(), (np.argwhere(~ok).ravel(), gq[~ok], -2.5 * g_ref[~ok])
    assert B.hr_get_status(ref.ctx) == B.HR_OK


def test_backward_after_another_forward_raises(B):
    """The Refiner's buffers hold its latest forward; a backward of an older loss
    raises instead of returning the newer forward's gradient, and the newer loss
    still back-propagates."""
    from paper_2107_05509_gb300.pipeline import HandRenderLoss, StaleRenderError
    sc = scene("tiny")
    ref = _refiner(B, sc)
    x = sc.x0.astype(np.float32)
    p1 = _t(x).requires_grad_(True)
    p2 = _t(x + np.float32(0.01)).requires_grad_(True)
    l1 = HandRenderLoss.apply(p1, ref)
    l2 = HandRenderLoss.apply(p2, ref)
    with pytest.raises(StaleRenderError):
        l1.backward()
    l2.backward()
    assert p2.grad is not None and torch.isfinite(p2.grad).all() and p2.grad.abs().max() > 0
    # the same gradient as the Refiner's own step at p2
    loss, d = ref.step(p2.detach())
    assert torch.allclose(p2.grad, d, rtol=1e-5, atol=1e-7 * float(d.abs().max()))
    with pytest.raises(ValueError):
        HandRenderLoss.apply(_t(x[:60]), ref)
