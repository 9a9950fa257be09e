"""One refinement iteration of the paper's method on the GPU, and the Adam loop.

Section 3: the parameters h + dh are refined by minimising the multiview
backprojection error E_1 (Eq. 3, D_c term of Eq. 4) with Adam (Section 3.3).  Every
step below is one handrt C-ABI call; PyTorch only holds device memory and streams.

    Refiner.step(params)  ->  loss, d_params
        hr_skin -> hr_build_bvh -> hr_render_fwd -> hr_loss -> hr_render_bwd -> hr_skin_bwd
    Refiner.adam(params, ...) -> hr_adam_step after every step

HandRenderLoss is the same iteration behind one torch.autograd.Function: the
forward renders and keeps the adjoint image, the backward re-traces the samples
(hr_render_bwd) instead of storing per-sample hit records.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import binding as B
from . import inputs as I


@dataclasses.dataclass
class Views:
    """Device-resident observations of one multiframe."""
    cams: torch.Tensor        # [N][20] float32 camera records
    background: torch.Tensor  # [N][H][W][3]
    observed: torch.Tensor    # [N][H][W][3]
    mask: torch.Tensor        # [N][H][W] uint8
    H: int
    W: int

    @property
    def N(self):
        return self.cams.shape[0]


class Refiner:
    """Buffers and context for refining one hand instance against one multiframe."""

    def __init__(self, model: B.Model, views: Views, opts: B.hr_render_opts, ctx: B.Context | None = None):
        self.model = model
        self.views = views
        self.opts = opts
        N, H, W = views.N, views.H, views.W
        hand = model.hand
        self.ctx = ctx or B.Context(hand.V, hand.F, hand.E, max(N, 1), W, H)
        dev = views.cams.device
        self.verts = torch.empty((hand.V, 3), device=dev)
        self.image = torch.empty((N, H, W, 3), device=dev)
        self.adjoint = torch.empty((N, H, W, 3), device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.d_verts = torch.empty((hand.V, 3), device=dev)
        self.d_params = torch.empty(61, device=dev)

    def forward(self, params, stream=None):
        ctx, m, v = self.ctx, self.model, self.views
        B.hr_skin(ctx, m, params, self.verts, stream)
        B.hr_build_bvh(ctx, m, self.verts, stream)
        B.hr_render_fwd(ctx, m, self.verts, v.cams, v.H, v.W, v.background, self.opts, self.image, stream)
        B.hr_loss(ctx, self.image, v.observed, v.mask, self.loss, self.adjoint, stream)
        return self.loss

    def backward(self, params, stream=None):
        ctx, m, v = self.ctx, self.model, self.views
        B.hr_render_bwd(ctx, m, self.verts, v.cams, v.H, v.W, v.background, self.opts, self.adjoint, self.d_verts,
                        stream)
        B.hr_skin_bwd(ctx, m, params, self.d_verts, self.d_params, stream)
        return self.d_params

    def step(self, params, stream=None):
        loss = self.forward(params, stream)
        return loss, self.backward(params, stream)

    def adam(self, params, iters, lr=0.01, betas=(0.9, 0.999), eps=1e-8, callback=None, stream=None):
        """Plain refinement: `iters` Adam steps on params (device float[61], updated
        in place).  The sample seed advances with the iteration."""
        m1 = torch.zeros_like(params)
        m2 = torch.zeros_like(params)
        base_iter = self.opts.iter
        for it in range(iters):
            self.opts.iter = base_iter + it
            self.step(params, stream)
            B.hr_adam_step(params, self.d_params, m1, m2, float(lr), betas[0], betas[1], eps, it + 1, stream)
            if callback is not None:
                callback(it, self)
        self.opts.iter = base_iter
        return params


class HandRenderLoss(torch.autograd.Function):
    """loss = E_1(params); backward re-traces the samples (no stored hit records)."""

    @staticmethod
    def forward(ctx, params, refiner: Refiner):
        p = params.detach().contiguous()
        loss = refiner.forward(p).clone()
        ctx.refiner = refiner
        ctx.save_for_backward(p)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        (p,) = ctx.saved_tensors
        g = ctx.refiner.backward(p)
        return g * grad_out, None


# --------------------------------------------------------------------------------------
# Synthetic multiframes
# --------------------------------------------------------------------------------------

def opts_for(cfg: I.SceneConfig, spp=None, seed=None, iter=0, iter_dev=None):
    return B.render_opts(seed=cfg.seed * 7919 + 17 if seed is None else seed, iter=iter, spp=spp or cfg.spp,
                         edge_samples=cfg.edge_samples, ka=I.K_AMBIENT, kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR,
                         light_rgb=I.LIGHT_RGB, edge_eps_px=I.EDGE_EPS_PX, iter_dev=iter_dev)


def make_views(cfg: I.SceneConfig, model: B.Model, x_gt, device="cuda", ctx=None):
    """Observations by this library's own renderer: the GT render at cfg.obs_spp
    samples per pixel plus N(0, sigma) noise; mask = render differs from the plate,
    dilated by cfg.mask_dilate_px (the recipe of the synthetic multiframes)."""
    hand = model.hand
    cams = torch.as_tensor(I.pack_cameras(I.make_cameras(cfg, hand.v_template.mean(0))), device=device)
    bg_np = I.background(cfg.seed, cfg.views, cfg.height, cfg.width)
    bg = torch.as_tensor(bg_np, device=device)
    N, H, W = cfg.views, cfg.height, cfg.width
    ctx = ctx or B.Context(hand.V, hand.F, hand.E, N, W, H)
    verts = torch.empty((hand.V, 3), device=device)
    p = torch.as_tensor(np.asarray(x_gt, np.float32), device=device)
    B.hr_skin(ctx, model, p, verts)
    B.hr_build_bvh(ctx, model, verts)
    clean = torch.empty((N, H, W, 3), device=device)
    o = opts_for(cfg, spp=cfg.obs_spp, seed=cfg.seed * 7919 + 1)
    B.hr_render_fwd(ctx, model, verts, cams, H, W, bg, o, clean)
    clean_np = clean.cpu().numpy()
    obs = I.add_noise(clean_np, cfg.seed, cfg.noise_sigma)
    mask = I.coverage_mask(clean_np, bg_np, cfg.mask_dilate_px)
    return Views(cams=cams, background=bg, observed=torch.as_tensor(obs, device=device),
                 mask=torch.as_tensor(mask, device=device), H=H, W=W), verts
