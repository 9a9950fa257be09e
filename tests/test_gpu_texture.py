"""GPU parity of the textured render (bilinear albedo texture at the interpolated
texture coordinates): forward pixels, the vertex gradient (through the barycentrics
and the texture coordinates, plus edges and the normal adjoint) and the texture
gradient, against the oracle, on the hand and on its twice-subdivided version."""
import functools

import numpy as np
import pytest

import oracle
from paper_2107_05509_gb300 import inputs as I
from tests.gpu_common import grad_ok, pixel_ok, require_gpu, torch

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _hand(fine):
    h = I.make_hand(0)
    return I.subdivide_hand(h, 2) if fine else h


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("fine", [False, True])
def test_textured_render_and_gradients_match_oracle(fine):
    require_gpu()
    from paper_2107_05509_gb300 import binding as B
    h = _hand(fine)
    cfg = I.SceneConfig("tex", views=2, width=96, height=80, spp=4, edge_samples=1024, elevation_deg=20.0,
                        azimuths_deg=(10.0, 200.0), seed=21)
    cams = I.pack_cameras(I.make_cameras(cfg, h.v_template.mean(0)))
    for c in cams:
        c[0:2] *= 2.5
    N, H, W = cfg.views, cfg.height, cfg.width
    x = I.perturb_params(I.gt_params(cfg.seed), cfg.seed).astype(np.float32)
    verts = oracle.skin(h, x).astype(np.float32)
    normals = oracle.vertex_normals(verts, h.faces, h.vf_offsets, h.vf_faces)
    bg = I.background(cfg.seed, N, H, W)
    tex = I.texture(cfg.seed, 64)
    o = oracle.make_opts(seed=31, spp=cfg.spp, edge_samples=cfg.edge_samples, ka=I.K_AMBIENT, kd=I.K_DIFFUSE,
                         light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB, edge_eps=I.EDGE_EPS_PX, texture=tex, uv=h.uv)
    ref = oracle.render_fwd(verts, h.faces, normals, h.albedo, cams, H, W, bg, o)
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, N, W, H)
    vt, ct, bt, tt = _t(verts), _t(cams), _t(bg), _t(tex)
    dtex = torch.zeros_like(tt)
    go = B.render_opts(seed=31, spp=cfg.spp, edge_samples=cfg.edge_samples, ka=I.K_AMBIENT, kd=I.K_DIFFUSE,
                       light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB, edge_eps_px=I.EDGE_EPS_PX, texture=tt,
                       d_texture=dtex, flags=B.HR_BWD_REUSE_FWD)
    img = torch.empty((N, H, W, 3), device="cuda")
    B.hr_build_bvh(ctx, model, vt)
    B.hr_render_fwd(ctx, model, vt, ct, H, W, bt, go, img)
    g = img.cpu().numpy()
    ok = pixel_ok(g, ref)
    assert ok.all(), (np.argwhere(~ok)[:5], np.abs(g - ref).max())
    # an adjoint on every 4th row (a real loss adjoint's magnitude)
    rng = np.random.default_rng(3)
    A = np.zeros((N, H, W, 3), np.float32)
    A[:, ::4] = rng.choice([-1.0, 1.0], size=A[:, ::4].shape).astype(np.float32) * 1e-4
    dT_ref = np.zeros(tex.shape, np.float64)
    dv_ref, _ = oracle.render_bwd(h, verts, cams, H, W, bg, o, A, normals=normals, d_texture=dT_ref)
    dv = torch.empty((h.V, 3), device="cuda")
    B.hr_render_bwd(ctx, model, vt, ct, H, W, bt, go, _t(A), dv)
    gd = dv.cpu().numpy()
    ok = grad_ok(gd, dv_ref)
    assert ok.all(), (np.argwhere(~ok)[:5], gd[~ok][:5], dv_ref[~ok][:5])
    gt = dtex.cpu().numpy()
    assert np.abs(dT_ref).max() > 0
    ok = grad_ok(gt, dT_ref)
    assert ok.all(), (np.argwhere(~ok)[:5], gt[~ok][:5], dT_ref[~ok][:5])
    assert B.hr_get_status(ctx) == B.HR_OK
