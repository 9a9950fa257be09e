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
import json
import os

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
        # counts forward() calls: backward() differentiates the state the latest
        # forward left (vertices, BVH, candidate lists, adjoint image)
        self.generation = 0

    def forward(self, params, stream=None, skin=True, build=True):
        ctx, m, v = self.ctx, self.model, self.views
        self.generation += 1
        if skin:
            B.hr_skin(ctx, m, params, self.verts, stream)
        if build:
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

    def capture_step(self, params):
        """step(params) recorded once as a CUDA graph and returned: each replay re-reads
        `params`, the views' tensors and, through opts.iter_dev when it is set, the
        device iteration counter, so a caller refreshes those tensors in place (host
        copies, a counter) and replays; loss, image, adjoint and d_params are written
        as by step().  The first launches run eagerly on a side stream (kernel loading
        is not capturable)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step(params, s)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.step(params, s)
        return g

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


@dataclasses.dataclass
class HostFrame:
    """One step's inputs in pinned host memory: a multiframe (the shapes and dtypes of
    Views' tensors), the 61 parameters and the sample-stream counter (int32[1])."""
    observed: torch.Tensor
    mask: torch.Tensor
    background: torch.Tensor
    cams: torch.Tensor
    params: torch.Tensor
    iter: torch.Tensor


@dataclasses.dataclass
class _Slot:
    ref: Refiner
    params: torch.Tensor
    counter: torch.Tensor
    graph: torch.cuda.CUDAGraph
    free: torch.cuda.Event   # the last step on this slot has been read back


class StreamedRefiner:
    """Refiner.step over a sequence of host-resident frames, each step's inputs copied
    to the device while the step before runs.

    Two device copies of the inputs alternate, each with its own Refiner (one shared
    context) and its own captured step.  For step k a copy stream fills slot k % 2
    from pinned host memory once the step that last used the slot has been read
    back; the caller's stream waits for that copy and replays the slot's graph; a
    read-back stream copies the loss and the parameter gradient to pinned host
    memory.  The copy of step k + 1 thus overlaps the render of step k, and the
    steps themselves run one after another on the caller's stream (they share the
    context's scratch)."""

    def __init__(self, model: B.Model, views: Views, opts: B.hr_render_opts, ctx: B.Context | None = None,
                 params: torch.Tensor | None = None):
        """views: a device multiframe whose shapes and dtypes every frame has; its
        contents, and params (device float[61], zeros if None), seed the capture.
        opts: the render options (each slot takes a copy whose iter_dev points at the
        slot's own counter)."""
        dev = views.cams.device
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.read_stream = torch.cuda.Stream(device=dev)
        self.slots = []
        for _ in range(2):
            counter = torch.zeros(1, dtype=torch.int32, device=dev)
            o = B.hr_render_opts.from_buffer_copy(opts)
            o.iter_dev = counter.data_ptr()
            v = Views(cams=views.cams.clone(), background=views.background.clone(), observed=views.observed.clone(),
                      mask=views.mask.clone(), H=views.H, W=views.W)
            ref = Refiner(model, v, o, ctx=ctx)
            ctx = ref.ctx
            p = params.clone() if params is not None else torch.zeros(61, device=dev)
            graph = ref.capture_step(p)
            slot = _Slot(ref, p, counter, graph, torch.cuda.Event())
            slot.free.record(torch.cuda.current_stream(dev))
            self.slots.append(slot)
        self.ctx = ctx
        self.k = 0

    def order_after(self, stream=None):
        """Start the next copies only after the work already queued on `stream`."""
        s = stream or torch.cuda.current_stream()
        self.copy_stream.wait_stream(s)

    def submit(self, frame: HostFrame, h_loss: torch.Tensor, h_grad: torch.Tensor, stream=None):
        """Queue one step on `frame`; its loss (float[1]) and d_params (float[61]) land
        in the pinned tensors h_loss and h_grad.  Returns (copied, done): events after
        which the frame's host memory may be reused and the outputs are valid."""
        s = stream or torch.cuda.current_stream()
        slot = self.slots[self.k % 2]
        self.k += 1
        v = slot.ref.views
        cs = self.copy_stream
        cs.wait_event(slot.free)
        with torch.cuda.stream(cs):
            for dst, src in ((v.observed, frame.observed), (v.mask, frame.mask), (v.background, frame.background),
                             (v.cams, frame.cams), (slot.params, frame.params), (slot.counter, frame.iter)):
                dst.copy_(src, non_blocking=True)
        copied = torch.cuda.Event()
        copied.record(cs)
        s.wait_event(copied)
        with torch.cuda.stream(s):
            slot.graph.replay()
        rs = self.read_stream
        rs.wait_stream(s)
        with torch.cuda.stream(rs):
            h_loss.copy_(slot.ref.loss, non_blocking=True)
            h_grad.copy_(slot.ref.d_params, non_blocking=True)
        slot.free = torch.cuda.Event()
        slot.free.record(rs)
        return copied, slot.free

    def join(self, stream=None):
        """Make `stream` wait for every queued copy and read-back."""
        s = stream or torch.cuda.current_stream()
        s.wait_stream(self.copy_stream)
        s.wait_stream(self.read_stream)


class StaleRenderError(RuntimeError):
    """backward of a HandRenderLoss after its Refiner rendered again."""


class HandRenderLoss(torch.autograd.Function):
    """loss = E_1(params) (Eq. 3 with the D_c term of Eq. 4) as a scalar tensor;
    backward re-traces the forward's samples (hr_render_bwd, no stored hit records)
    and applies the skinning adjoint, scaled by the incoming gradient.

    The Refiner's buffers (vertices, BVH, candidate lists, adjoint image) hold the
    state of its latest forward and are what the backward differentiates, so each
    loss must be back-propagated before the same Refiner renders again: a backward
    after another forward raises StaleRenderError instead of returning the other
    forward's gradient.  Use one Refiner per loss term that must stay alive (for
    example two terms summed before one backward).  params: device float32[61]."""

    @staticmethod
    def forward(ctx, params, refiner: Refiner):
        if params.dtype != torch.float32 or params.numel() != 61 or not params.is_cuda:
            raise ValueError("params must be a CUDA float32 tensor of 61 entries")
        p = params.detach().contiguous()
        loss = refiner.forward(p).clone()
        ctx.refiner = refiner
        ctx.generation = refiner.generation
        ctx.save_for_backward(p)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        (p,) = ctx.saved_tensors
        r = ctx.refiner
        if r.generation != ctx.generation:
            raise StaleRenderError(
                f"the Refiner rendered {r.generation - ctx.generation} more time(s) after this loss was computed; "
                "back-propagate each HandRenderLoss before the next forward on the same Refiner")
        g = r.backward(p)
        return (g * grad_out).reshape(p.shape), None


# --------------------------------------------------------------------------------------
# Synthetic multiframes
# --------------------------------------------------------------------------------------

def opts_for(cfg: I.SceneConfig, spp=None, seed=None, iter=0, iter_dev=None, flags=B.HR_BWD_REUSE_FWD,
             texture=None, d_texture=None):
    """Render options of a workload; the backward reuses the forward's candidate lists
    (a refinement iteration renders and differentiates the same scene)."""
    return B.render_opts(seed=cfg.seed * 7919 + 17 if seed is None else seed, iter=iter, spp=spp or cfg.spp,
                         edge_samples=cfg.edge_samples, ka=I.K_AMBIENT, kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR,
                         light_rgb=I.LIGHT_RGB, edge_eps_px=I.EDGE_EPS_PX, iter_dev=iter_dev, flags=flags,
                         texture=texture, d_texture=d_texture)


def make_views(cfg: I.SceneConfig, model: B.Model, x_gt, device="cuda", ctx=None, texture=None):
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
    o = opts_for(cfg, spp=cfg.obs_spp, seed=cfg.seed * 7919 + 1, texture=texture)
    B.hr_render_fwd(ctx, model, verts, cams, H, W, bg, o, clean)
    clean_np = clean.cpu().numpy()
    obs = I.add_noise(clean_np, cfg.seed, cfg.noise_sigma)
    mask = I.coverage_mask(clean_np, bg_np, cfg.mask_dilate_px)
    return Views(cams=cams, background=bg, observed=torch.as_tensor(obs, device=device),
                 mask=torch.as_tensor(mask, device=device), H=H, W=W), verts


# --------------------------------------------------------------------------------------
# Batches: many instances refined together, one launch per kernel per iteration
# --------------------------------------------------------------------------------------

# iterations per full BVH rebuild in the captured refinement loops (refits between)
REBUILD_EVERY = 8

# Adam step sizes per parameter group [beta(10), theta(45), phi(3), tau(3)]: shape
# coefficients, radians, radians, metres (Adam's step is about lr whatever the
# gradient's scale, so each group gets a step in its own unit)
LR_GROUPS = (0.1, 0.02, 0.02, 1e-3)


def lr_scale_vector(groups=LR_GROUPS, device="cuda"):
    s = np.empty(I.N_PARAMS, np.float32)
    s[I.P_BETA:I.P_BETA + I.N_SHAPE] = groups[0]
    s[I.P_THETA:I.P_THETA + I.N_POSE] = groups[1]
    s[I.P_THETA + I.N_POSE:I.P_TAU] = groups[2]
    s[I.P_TAU:I.P_TAU + 3] = groups[3]
    return torch.as_tensor(s, device=device)


@dataclasses.dataclass
class BatchViews:
    """Device-resident observations of a batch, concatenated in instance order."""
    cams: torch.Tensor        # [views][20]
    background: torch.Tensor  # [P][3]
    observed: torch.Tensor    # [P][3]
    mask: torch.Tensor        # [P] uint8


def make_batch_views(cfgs, model: B.Model, x_gts, device="cuda", texture=None):
    """Observations of every instance (the recipe of make_views: the GT render at
    cfg.obs_spp with the instance's own Philox instance field, plus noise, and the
    dilated coverage mask), concatenated in instance order; `texture`: the albedo
    texture of the model (its uv) for the observations."""
    hand = model.hand
    cams, bgs, obss, masks = [], [], [], []
    for i, (cfg, x) in enumerate(zip(cfgs, x_gts)):
        N, H, W = cfg.views, cfg.height, cfg.width
        ctx = B.Context(hand.V, hand.F, hand.E, N, W, H)
        c = torch.as_tensor(I.pack_cameras(I.make_cameras(cfg, hand.v_template.mean(0))), device=device)
        bg_np = I.background(cfg.seed, N, H, W)
        bg = torch.as_tensor(bg_np, device=device)
        verts = torch.empty((hand.V, 3), device=device)
        B.hr_skin(ctx, model, torch.as_tensor(np.asarray(x, np.float32), device=device), verts)
        B.hr_build_bvh(ctx, model, verts)
        clean = torch.empty((N, H, W, 3), device=device)
        o = opts_for(cfg, spp=cfg.obs_spp, seed=cfg.seed * 7919 + 1, texture=texture)
        o.instance = i
        B.hr_render_fwd(ctx, model, verts, c, H, W, bg, o, clean)
        clean_np = clean.cpu().numpy()
        ctx.close()
        cams.append(c)
        bgs.append(bg.reshape(-1, 3))
        obss.append(torch.as_tensor(I.add_noise(clean_np, cfg.seed, cfg.noise_sigma).reshape(-1, 3), device=device))
        masks.append(torch.as_tensor(I.coverage_mask(clean_np, bg_np, cfg.mask_dilate_px).reshape(-1),
                                     device=device))
    return BatchViews(cams=torch.cat(cams), background=torch.cat(bgs), observed=torch.cat(obss),
                      mask=torch.cat(masks))


class BatchRefiner:
    """Plain refinement of every instance of a batch at once.  One iteration is
    hr_skin_batch -> hr_update_bvh -> hr_render_fwd_batch -> hr_loss_batch ->
    hr_render_bwd_batch -> hr_skin_bwd_batch -> hr_adam_step_dev, plus (with ground
    truth vertices) hr_vertex_error into the error table: a fixed sequence of launches
    over all instances that capture() records once as a CUDA graph.

    retire: None (every instance refined every iteration), "converged" (an instance
    leaves the batch once its vertex error is <= retire_mm; needs ref_verts: the
    benchmark's per-instance criterion) or "plateau" (an instance leaves once its loss
    has not fallen by rel_tol for `patience` iterations).  A retired instance is
    skipped by every batch kernel and its Adam steps are zeroed, on the device, so the
    captured iteration gets cheaper as instances converge."""

    def __init__(self, model: B.Model, batch: B.Batch, views: BatchViews, seed=17, lr=1.0, lr_groups=LR_GROUPS,
                 ref_verts=None, max_iters=1024, device="cuda", retire=None, retire_mm=1.0, rel_tol=1e-3,
                 patience=10, texture=None):
        self.model, self.batch, self.views = model, batch, views
        n, V, P = batch.n, model.V, batch.total_pixels
        if retire not in (None, "converged", "plateau"):
            raise ValueError(f"retire: {retire}")
        if retire == "converged" and ref_verts is None:
            raise ValueError("retire='converged' needs the ground-truth vertices")
        self.retire, self.retire_m, self.rel_tol, self.patience = retire, retire_mm * 1e-3, rel_tol, patience
        self.counter = torch.zeros(1, dtype=torch.int32, device=device)
        self.opts = B.render_opts(seed=seed, ka=I.K_AMBIENT, kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR,
                                  light_rgb=I.LIGHT_RGB, edge_eps_px=I.EDGE_EPS_PX, iter_dev=self.counter,
                                  flags=B.HR_BWD_REUSE_FWD, texture=texture)
        self.params = torch.zeros((n, I.N_PARAMS), device=device)
        self.verts = torch.empty((n, V, 3), device=device)
        self.image = torch.empty((P, 3), device=device)
        self.adjoint = torch.empty((P, 3), device=device)
        self.loss = torch.zeros(n, device=device)
        self.d_verts = torch.empty((n, V, 3), device=device)
        self.d_params = torch.empty((n, I.N_PARAMS), device=device)
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.lr = float(lr)
        # per-entry steps [n][61] (the groups' steps repeated): retiring an instance
        # zeroes its row
        self.lr_scale0 = lr_scale_vector(lr_groups, device).repeat(n)
        self.lr_scale = self.lr_scale0.clone()
        self.active = torch.ones(n, dtype=torch.int32, device=device)
        self.best = torch.full((n,), float("inf"), device=device)
        self.stall = torch.zeros(n, dtype=torch.int32, device=device)
        B.hr_batch_set_active(batch, self.active)
        batch.active_mask = self.active   # the context reads it for as long as it lives
        self.ref_verts = ref_verts
        self.err = torch.full((max_iters, n), float("nan"), device=device)
        self.graph = None

    def reset(self, params):
        self.params.copy_(params)
        self.m1.zero_()
        self.m2.zero_()
        self.counter.zero_()
        self.err.fill_(float("nan"))
        self.active.fill_(1)
        self.lr_scale.copy_(self.lr_scale0)
        self.best.fill_(float("inf"))
        self.stall.zero_()

    def iteration(self, stream=None):
        bt, m, v = self.batch, self.model, self.views
        # the batch calls read this refiner's mask (the context may be shared with
        # another refiner; a captured iteration keeps the pointer given here)
        B.hr_batch_set_active(bt, self.active)
        bt.active_mask = self.active
        B.hr_skin_batch(bt, m, self.params, self.verts, stream)
        if self.ref_verts is not None:
            B.hr_vertex_error(self.verts, self.ref_verts, self.err, self.counter, stream)
            if self.retire == "converged":
                B.hr_retire_converged(self.err, self.counter, self.retire_m, self.active, self.lr_scale, stream)
        B.hr_update_bvh(bt, m, self.verts, self.counter, REBUILD_EVERY, stream)
        B.hr_render_fwd_batch(bt, m, self.verts, v.cams, v.background, self.opts, self.image, stream)
        B.hr_loss_batch(bt, self.image, v.observed, v.mask, self.loss, self.adjoint, stream)
        if self.retire == "plateau":
            B.hr_retire_plateau(self.loss, self.rel_tol, self.patience, self.best, self.stall, self.active,
                                self.lr_scale, stream)
        B.hr_render_bwd_batch(bt, m, self.verts, v.cams, v.background, self.opts, self.adjoint, self.d_verts, stream)
        B.hr_skin_bwd_batch(bt, m, self.params, self.d_verts, self.d_params, stream)
        B.hr_adam_step_dev(self.params, self.d_params, self.m1, self.m2, self.lr, 0.9, 0.999, 1e-8, self.counter,
                           lr_scale=self.lr_scale, stream=stream)

    def render_pass(self, stream=None):
        """Forward and backward of the current parameters without an update (what the
        autotuner times)."""
        bt, m, v = self.batch, self.model, self.views
        B.hr_batch_set_active(bt, self.active)
        bt.active_mask = self.active
        B.hr_skin_batch(bt, m, self.params, self.verts, stream)
        B.hr_build_bvh_batch(bt, m, self.verts, stream)
        B.hr_render_fwd_batch(bt, m, self.verts, v.cams, v.background, self.opts, self.image, stream)
        B.hr_loss_batch(bt, self.image, v.observed, v.mask, self.loss, self.adjoint, stream)
        B.hr_render_bwd_batch(bt, m, self.verts, v.cams, v.background, self.opts, self.adjoint, self.d_verts, stream)

    def capture(self):
        """Record one iteration as a CUDA graph (warm up first: the first launches of
        a process load the kernels)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        # the warm-up iteration's effects are undone afterwards (retirement state too)
        names = ("params", "m1", "m2", "counter", "active", "lr_scale", "best", "stall")
        state = [getattr(self, k) for k in names if hasattr(self, k)]
        saved = [t.clone() for t in state]
        with torch.cuda.stream(s):
            self.iteration(s)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.iteration(s)
        self.graph = g
        for t, v in zip(state, saved):
            t.copy_(v)
        return g


class PlainRefiner:
    """Plain per-instance refinement through the single-instance calls, one
    iteration captured as a CUDA graph: hr_skin -> (hr_vertex_error) -> hr_update_bvh
    -> hr_render_fwd -> hr_loss -> hr_render_bwd -> hr_skin_bwd -> hr_adam_step_dev
    with per-group step sizes; the device counter advances the sample streams."""

    def __init__(self, model: B.Model, views: Views, cfg: I.SceneConfig, instance=0, seed=17, lr=1.0,
                 lr_groups=LR_GROUPS, ref_verts=None, max_iters=1024, ctx=None, device="cuda", texture=None):
        self.counter = torch.zeros(1, dtype=torch.int32, device=device)
        opts = B.render_opts(seed=seed, instance=instance, spp=cfg.spp, edge_samples=cfg.edge_samples,
                             ka=I.K_AMBIENT, kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB,
                             edge_eps_px=I.EDGE_EPS_PX, iter_dev=self.counter, flags=B.HR_BWD_REUSE_FWD,
                             texture=texture)
        self.r = Refiner(model, views, opts, ctx=ctx)
        self.params = torch.zeros(I.N_PARAMS, device=device)
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.lr = float(lr)
        self.lr_scale = lr_scale_vector(lr_groups, device)
        self.ref_verts = ref_verts
        self.err = torch.full((max_iters, 1), float("nan"), device=device)
        self.graph = None

    def reset(self, params):
        self.params.copy_(params)
        self.m1.zero_()
        self.m2.zero_()
        self.counter.zero_()
        self.err.fill_(float("nan"))

    def iteration(self, stream=None):
        r = self.r
        B.hr_skin(r.ctx, r.model, self.params, r.verts, stream)
        if self.ref_verts is not None:
            B.hr_vertex_error(r.verts, self.ref_verts, self.err, self.counter, stream)
        B.hr_update_bvh(r.ctx, r.model, r.verts, self.counter, REBUILD_EVERY, stream)
        r.forward(self.params, stream, skin=False, build=False)
        r.backward(self.params, stream)
        B.hr_adam_step_dev(self.params, r.d_params, self.m1, self.m2, self.lr, 0.9, 0.999, 1e-8, self.counter,
                           lr_scale=self.lr_scale, stream=stream)

    def render_pass(self, stream=None):
        self.r.step(self.params, stream)

    capture = BatchRefiner.capture


# --------------------------------------------------------------------------------------
# Autotuner of the render kernels' launch shapes
# --------------------------------------------------------------------------------------

TUNING_SPACE = {
    "rays_per_lane": (1, 2, 4),
    "cand_per_chunk": (8, 16, 32),
    "max_chunks": (8, 16),
    "blocks_per_sm": (4, 6, 8),
    "bwd_blocks_per_sm": (2, 3, 4, 6),
    "bwd_rays_per_lane": (1, 2, 4),
    "bwd_cand_per_chunk": (8, 16, 32),
    "edge_lanes": (2, 4, 8),
}


def tuning_cache_path():
    return os.environ.get("HANDRT_TUNING_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "handrt",
                                                              "tuning.json"))


def workload_key(model: B.Model, layout) -> str:
    """Cache key: device, mesh size and the view layout ((views, W, H, spp, edge
    samples) per instance)."""
    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|V{model.V}|F{model.struct.F}|" + ";".join("x".join(str(int(x)) for x in d) for d in layout)


def _time_ms(run, reps):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    run()   # warm-up: first launch of a new kernel variant loads it
    for a, b in ev:
        a.record()
        run()
        b.record()
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ev]))


def autotune(ctx: B.Context, run, key: str, reps=3, space=TUNING_SPACE, cache=True, log=None):
    """Pick the context's launch shapes for a workload: coordinate descent over
    `space` from the cached (else current) setting -- each parameter in turn takes the
    value with the lowest median device time of `run()` (one render forward + backward
    of the workload) with the others fixed, two sweeps -- then set the best and cache
    it under `key`.  Returns (tuning, ms of the start setting, ms of the best)."""
    path = tuning_cache_path()
    table = {}
    if cache and os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if cache and key in table:
        ctx.set_tuning(**table[key]["tuning"])
        return table[key]["tuning"], table[key]["start_ms"], table[key]["best_ms"]
    best = ctx.get_tuning()
    start_ms = best_ms = _time_ms(run, reps)
    for _sweep in range(2):
        changed = False
        for name, values in space.items():
            for v in values:
                if v == best[name]:
                    continue
                trial = dict(best, **{name: v})
                ctx.set_tuning(**trial)
                ms = _time_ms(run, reps)
                if log:
                    log(f"tune {trial}: {ms:.4f} ms")
                if ms < best_ms * 0.99:
                    best, best_ms, changed = trial, ms, True
            ctx.set_tuning(**best)
        if not changed:
            break
    ctx.set_tuning(**best)
    if cache:
        table[key] = {"tuning": best, "start_ms": start_ms, "best_ms": best_ms}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path + ".tmp", "w") as f:
                json.dump(table, f, indent=1)
            os.replace(path + ".tmp", path)
        except OSError:
            pass
    return best, start_ms, best_ms


# --------------------------------------------------------------------------------------
# The paper's full objective with its optimisation schedule
# --------------------------------------------------------------------------------------

class PaperRefiner:
    """Refinement of geometry, colour map and per-camera colour transforms (Section 3:
    E = E_1(dh, c, T) + lambda E_2(dh), the data term f_1 = D_c + edge_weight D_e of
    Eq. 4) with the schedule of Section 3.3: a warm-up in which only T and V_low move,
    then all of (dh, c, T).

    One iteration: hr_skin_joints -> hr_joint_prior (target: the joints of the initial
    estimate) -> hr_update_bvh -> hr_colour_map -> hr_render_fwd (texture V(c)) ->
    hr_loss_ct (D_c with T) -> hr_edge_loss (D_e, adding to the same adjoint and dT) ->
    hr_render_bwd (vertex and texture gradients) -> hr_colour_map_bwd ->
    hr_skin_bwd_joints -> hr_adam_step_dev over the whole parameter vector
    [h (61) | T (N x 9) | V_low | V_high], with per-entry step sizes (zero for the
    parameters a phase keeps fixed).  Both phases are captured as CUDA graphs."""

    def __init__(self, model: B.Model, views: Views, cfg: I.SceneConfig, tex_size=512, low_size=8, gamma=0.005,
                 weight=1e-3, lr_groups=LR_GROUPS, lr_T=0.01, lr_low=0.02, lr_high=0.01, ref_verts=None,
                 max_iters=1024, ctx=None, device="cuda", edge_weight=1.0):
        hand = model.hand
        N = views.N
        self.model, self.views, self.cfg = model, views, cfg
        self.ctx = ctx or B.Context(hand.V, hand.F, hand.E, N, views.W, views.H)
        self.gamma, self.weight = gamma, weight
        self.S, self.Sl = tex_size, low_size
        nJ = hand.j_template.shape[0]
        self.o_h, self.o_T = 0, 61
        self.o_lo = self.o_T + 9 * N
        self.o_hi = self.o_lo + 3 * low_size * low_size
        self.n = self.o_hi + 3 * tex_size * tex_size
        f = lambda *shape: torch.zeros(shape, device=device)
        self.p, self.g, self.m1, self.m2 = f(self.n), f(self.n), f(self.n), f(self.n)
        self.verts, self.d_verts = f(hand.V, 3), f(hand.V, 3)
        self.joints, self.d_joints, self.target = f(nJ, 3), f(nJ, 3), f(nJ, 3)
        self.tex = f(tex_size, tex_size, 3)
        self.image, self.adjoint = f(N, views.H, views.W, 3), f(N, views.H, views.W, 3)
        self.loss, self.prior, self.edge_loss = f(1), f(1), f(1)
        self.edge_weight = float(edge_weight)
        self.edges_obs = f(N, views.H, views.W)
        if self.edge_weight:
            # the observation's blurred edge map, once (this first edge call also
            # allocates the context's edge scratch, outside any graph capture)
            B.hr_edges(self.ctx, views.observed, self.edges_obs)
        self.counter = torch.zeros(1, dtype=torch.int32, device=device)
        self.opts = opts_for(cfg, iter_dev=self.counter, texture=self.tex,
                             d_texture=self.g[self.o_hi:].view(tex_size, tex_size, 3))
        self.ref_verts = ref_verts
        self.err = torch.full((max_iters, 1), float("nan"), device=device)
        base = np.zeros(self.n, np.float32)
        base[:61] = lr_scale_vector(lr_groups, "cpu").numpy()
        base[self.o_T:self.o_lo] = lr_T
        base[self.o_lo:self.o_hi] = lr_low
        base[self.o_hi:] = lr_high
        warm = base.copy()
        warm[:61] = 0.0
        warm[self.o_hi:] = 0.0
        self.scale_warm = torch.as_tensor(warm, device=device)
        self.scale_main = torch.as_tensor(base, device=device)
        self.graphs = {}

    # views of the parameter vector
    def h(self):
        return self.p[:61]

    def T(self):
        return self.p[self.o_T:self.o_lo].view(-1, 9)

    def reset(self, h0, v_low=0.5):
        """Start from estimate h0, identity transforms, a flat low map and no detail;
        the prior's target is h0's joints."""
        self.p.zero_()
        self.p[:61].copy_(torch.as_tensor(np.asarray(h0, np.float32), device=self.p.device))
        self.T().copy_(torch.eye(3, device=self.p.device).reshape(1, 9).expand(self.views.N, 9))
        self.p[self.o_lo:self.o_hi].fill_(v_low)
        self.m1.zero_()
        self.m2.zero_()
        self.counter.zero_()
        self.err.fill_(float("nan"))
        B.hr_skin_joints(self.ctx, self.model, self.h(), self.verts, self.target)

    def iteration(self, scale, stream=None):
        ctx, m, v = self.ctx, self.model, self.views
        S, Sl = self.S, self.Sl
        B.hr_skin_joints(ctx, m, self.h(), self.verts, self.joints, stream)
        if self.ref_verts is not None:
            B.hr_vertex_error(self.verts, self.ref_verts, self.err, self.counter, stream)
        B.hr_joint_prior(self.joints, self.target, self.gamma, self.weight, self.prior, self.d_joints, stream)
        B.hr_update_bvh(ctx, m, self.verts, self.counter, REBUILD_EVERY, stream)
        lo = self.p[self.o_lo:self.o_hi].view(Sl, Sl, 3)
        hi = self.p[self.o_hi:].view(S, S, 3)
        B.hr_colour_map(lo, hi, self.tex, stream)
        B.hr_render_fwd(ctx, m, self.verts, v.cams, v.H, v.W, v.background, self.opts, self.image, stream)
        B.hr_loss_ct(ctx, self.image, v.observed, v.mask, self.T(), self.loss, self.adjoint,
                     self.g[self.o_T:self.o_lo].view(-1, 9), stream)
        if self.edge_weight:
            B.hr_edge_loss(ctx, self.image, self.edges_obs, v.mask, self.edge_loss, self.adjoint, T=self.T(),
                           dT=self.g[self.o_T:self.o_lo].view(-1, 9), weight=self.edge_weight, stream=stream)
        self.g[self.o_hi:].zero_()   # the texture gradient accumulates
        B.hr_render_bwd(ctx, m, self.verts, v.cams, v.H, v.W, v.background, self.opts, self.adjoint, self.d_verts,
                        stream)
        B.hr_colour_map_bwd(self.g[self.o_hi:].view(S, S, 3), self.g[self.o_lo:self.o_hi].view(Sl, Sl, 3), stream)
        B.hr_skin_bwd_joints(ctx, m, self.h(), self.d_verts, self.d_joints, self.g[:61], stream)
        B.hr_adam_step_dev(self.p, self.g, self.m1, self.m2, 1.0, 0.9, 0.999, 1e-8, self.counter, lr_scale=scale,
                           stream=stream)

    def capture(self):
        """Graphs of a warm-up and a main iteration (state restored afterwards)."""
        saved = [t.clone() for t in (self.p, self.m1, self.m2, self.counter)]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        for name, sc in (("warm", self.scale_warm), ("main", self.scale_main)):
            with torch.cuda.stream(s):
                self.iteration(sc, s)
            torch.cuda.current_stream().wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                self.iteration(sc, s)
            self.graphs[name] = g
        for t, v in zip((self.p, self.m1, self.m2, self.counter), saved):
            t.copy_(v)
        return self.graphs

    def run(self, warm=50, main=150):
        """The schedule of Section 3.3 (50 warm-up + 150 iterations by default)."""
        if not self.graphs:
            self.capture()
        for _ in range(warm):
            self.graphs["warm"].replay()
        for _ in range(main):
            self.graphs["main"].replay()


def make_paper_views(cfg: I.SceneConfig, model: B.Model, x_gt, tex_gt, T_gt, device="cuda", ctx=None):
    """Observations for the full objective: the ground truth rendered with the colour
    map tex_gt ([S][S][3]) at cfg.obs_spp, every pixel of camera i's image transformed
    by its T_gt[i] ([N][3][3], near identity: the camera's colour response, which the
    data term models as T_i R), plus noise; mask as in make_views."""
    hand = model.hand
    cams = torch.as_tensor(I.pack_cameras(I.make_cameras(cfg, hand.v_template.mean(0))), device=device)
    bg_np = I.background(cfg.seed, cfg.views, cfg.height, cfg.width)
    bg = torch.as_tensor(bg_np, device=device)
    N, H, W = cfg.views, cfg.height, cfg.width
    ctx = ctx or B.Context(hand.V, hand.F, hand.E, N, W, H)
    verts = torch.empty((hand.V, 3), device=device)
    B.hr_skin(ctx, model, torch.as_tensor(np.asarray(x_gt, np.float32), device=device), verts)
    B.hr_build_bvh(ctx, model, verts)
    clean = torch.empty((N, H, W, 3), device=device)
    tex = torch.as_tensor(np.asarray(tex_gt, np.float32), device=device)
    B.hr_render_fwd(ctx, model, verts, cams, H, W, bg, opts_for(cfg, spp=cfg.obs_spp, seed=cfg.seed * 7919 + 1,
                                                                texture=tex), clean)
    clean_np = clean.cpu().numpy()
    Tt = np.asarray(T_gt, np.float64)
    coloured = np.einsum("nij,nhwj->nhwi", Tt, clean_np).astype(np.float32)
    obs = I.add_noise(coloured, cfg.seed, cfg.noise_sigma)
    mask = I.coverage_mask(clean_np, bg_np, cfg.mask_dilate_px)
    return Views(cams=cams, background=bg, observed=torch.as_tensor(obs, device=device),
                 mask=torch.as_tensor(mask, device=device), H=H, W=W)
