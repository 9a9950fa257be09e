"""Learned proposal for the refinement (an extension: the paper's Section 3 refines by
gradient descent alone).  A network (hr_net_*, bf16 on the tensor cores) maps the
residual images of an estimate to a parameter update; it is trained on pairs that
this library's renderer generates, and used for the first updates of a refinement,
with the photometric loss deciding per instance whether a proposal is kept -- the
plain method stays the fallback and the judge of its error.

Training pairs (the training rig: 8 views of 256 x 256 on a ring at 0.6 m, elevation
30 degrees): ground truth h ~ pose N(0, 0.4 rad) clipped to +-1.2, shape N(0, 1);
estimate h0 = h + u (pose and root rotation N(0, 0.1 rad), shape N(0, 0.5),
translation N(0, 5 mm)) with u ~ U(0.15, 1) per pair.  Each step renders the ground
truth over a fresh noise plate (observation + N(0, 0.01)) and the estimate, forms the
network's inputs, predicts h0 + delta, and takes the mean squared vertex distance
to the ground truth after skinning (hr_vertex_mse); its gradient returns through
hr_skin_bwd_batch to the network (hr_net_backward) -- every step is a library kernel.
"""
from __future__ import annotations

import dataclasses
import json
import os
import time

import numpy as np
import torch

from . import binding as B
from . import inputs as I
from . import pipeline as P

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "proposal_bf16.npz")

RIG = I.SceneConfig("rig-8x256x256", views=8, width=256, height=256, spp=16, edge_samples=4096,
                    elevation_deg=30.0, azimuths_deg=tuple(45.0 * k for k in range(8)), seed=3000)
TRAIN_SPP = 4


def init_params(seed=0):
    """He-normal weights over each layer's real inputs (padding columns zero), zero
    biases; the output layer starts small."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 9001]))
    cin = (8, 32, 64, 128, 128)
    cout = (32, 64, 128, 128, 128)
    spec = [(cout[l], (9 * cin[l] + 63) // 64 * 64, 9 * cin[l], cout[l], np.sqrt(2.0 / (9 * cin[l])))
            for l in range(5)]
    spec += [(256, 2112, 2060, 256, np.sqrt(2.0 / 2060)), (256, 256, 256, 256, np.sqrt(2.0 / 256)),
             (64, 256, 256, 61, 0.1 / 16.0)]
    parts = []
    for n_rows, k_cols, fan, n_real, std in spec:
        W = np.zeros((n_rows, k_cols), np.float32)
        W[:n_real, :fan] = rng.normal(0.0, std, (n_real, fan))
        parts += [W.reshape(-1), np.zeros(n_rows, np.float32)]
    p = np.concatenate(parts)
    assert p.size == int(B.lib().hr_net_param_count())
    return p


def save_weights(params: np.ndarray, meta: dict, path=WEIGHTS):
    """bf16 bit patterns of the parameters (what inference uses) plus metadata."""
    os.makedirs(os.path.dirname(path), exist_ok=True)
    bits = (np.ascontiguousarray(params, np.float32).view(np.uint32) + 0x7FFF +
            ((np.ascontiguousarray(params, np.float32).view(np.uint32) >> 16) & 1)) >> 16
    np.savez_compressed(path, bf16=bits.astype(np.uint16), meta=json.dumps(meta))


def load_weights(path=WEIGHTS):
    z = np.load(path)
    params = (z["bf16"].astype(np.uint32) << 16).view(np.float32)
    return params, json.loads(str(z["meta"]))


def sample_pairs(rng, n):
    """(ground truth, estimate) parameter arrays [n][61] of the training distribution."""
    gt = np.zeros((n, I.N_PARAMS))
    gt[:, I.P_BETA:I.P_BETA + I.N_SHAPE] = rng.normal(0.0, 1.0, (n, I.N_SHAPE))
    gt[:, I.P_THETA:I.P_THETA + I.N_POSE] = np.clip(rng.normal(0.0, 0.4, (n, I.N_POSE)), -1.2, 1.2)
    u = rng.uniform(0.15, 1.0, (n, 1))
    d = np.zeros((n, I.N_PARAMS))
    d[:, I.P_BETA:I.P_BETA + I.N_SHAPE] = rng.normal(0.0, 0.5, (n, I.N_SHAPE))
    d[:, I.P_THETA:I.P_TAU] = rng.normal(0.0, 0.1, (n, I.N_POSE + 3))
    d[:, I.P_TAU:I.P_TAU + 3] = rng.normal(0.0, 0.005, (n, 3))
    return gt.astype(np.float32), (gt + u * d).astype(np.float32)


class Trainer:
    """Training of the proposal network on renderer-generated pairs, B per step."""

    def __init__(self, model: B.Model, batch=128, seed=0, lr=3e-4, device="cuda"):
        self.model, self.B, self.seed, self.lr = model, batch, seed, lr
        hand = model.hand
        rig = RIG
        self.bt = B.Batch(hand.V, hand.F, hand.E, [(rig.views, rig.width, rig.height, TRAIN_SPP, 0, i)
                                                    for i in range(batch)])
        self.net = B.Net(batch, rig.views)
        cams1 = I.pack_cameras(I.make_cameras(rig, hand.v_template.mean(0)))
        self.cams = torch.as_tensor(np.concatenate([cams1] * batch), device=device)
        Pix = self.bt.total_pixels
        self.plate = torch.empty((Pix, 3), device=device)
        self.obs = torch.empty((Pix, 3), device=device)
        self.img = torch.empty((Pix, 3), device=device)
        V = hand.V
        self.v_gt = torch.empty((batch, V, 3), device=device)
        self.v0 = torch.empty((batch, V, 3), device=device)
        self.v_pred = torch.empty((batch, V, 3), device=device)
        self.dv = torch.empty((batch, V, 3), device=device)
        self.x_gt = torch.empty((batch, 61), device=device)
        self.x0 = torch.empty((batch, 61), device=device)
        self.x_pred = torch.empty((batch, 61), device=device)
        self.dx = torch.empty((batch, 61), device=device)
        self.loss = torch.empty(batch, device=device)
        self.loss0 = torch.empty(batch, device=device)
        self.h_in = torch.empty((2, batch, 61)).pin_memory()
        self.opts = B.render_opts(seed=seed * 7919 + 5, ka=I.K_AMBIENT, kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR,
                                  light_rgb=I.LIGHT_RGB, edge_eps_px=I.EDGE_EPS_PX)
        self.step_no = 0

    def set_params(self, params):
        self.net.set_params(torch.as_tensor(np.asarray(params, np.float32), device=self.cams.device))

    def _render(self, x, verts, out):
        bt, m = self.bt, self.model
        B.hr_skin_batch(bt, m, x, verts)
        B.hr_build_bvh_batch(bt, m, verts)
        B.hr_render_fwd_batch(bt, m, verts, self.cams, self.plate, self.opts, out)

    def step(self, train=True):
        """One batch of fresh pairs; returns (mean epsilon_v of the estimates, of the
        proposals) in mm, computed on the device (hr_vertex_mse of the squared
        distance is the loss; the mm figures come from hr_vertex_error)."""
        rng = np.random.default_rng(np.random.SeedSequence([self.seed, 17, self.step_no]))
        gt, x0 = sample_pairs(rng, self.B)
        self.h_in[0].copy_(torch.from_numpy(gt))
        self.h_in[1].copy_(torch.from_numpy(x0))
        self.x_gt.copy_(self.h_in[0], non_blocking=True)
        self.x0.copy_(self.h_in[1], non_blocking=True)
        self.opts.iter = self.step_no
        k = 1 + 4 * self.step_no
        # plate ~ 0.5 + N(0, 0.29) (the spread of U(0, 1)), then the observation
        self.plate.fill_(0.5)
        B.hr_add_noise(self.plate, 0.29, (self.seed << 40) + k)
        self._render(self.x_gt, self.v_gt, self.obs)
        B.hr_add_noise(self.obs, 0.01, (self.seed << 40) + k + 1)
        self._render(self.x0, self.v0, self.img)
        net = self.net
        net.inputs(self.img, self.obs)
        net.forward(self.cams, self.x_pred, base=self.x0)
        B.hr_skin_batch(self.bt, self.model, self.x_pred, self.v_pred)
        B.hr_vertex_mse(self.v_pred, self.v_gt, self.loss, self.dv)
        err = torch.empty((2, self.B), device=self.cams.device)
        B.hr_vertex_error(self.v0, self.v_gt, err[0:1])
        B.hr_vertex_error(self.v_pred, self.v_gt, err[1:2])
        if train:
            B.hr_skin_bwd_batch(self.bt, self.model, self.x_pred, self.dv, self.dx)
            net.backward(self.dx)
            net.adam(self.lr, self.step_no + 1)
        self.step_no += 1
        return err


def train(model: B.Model, pairs=200_000, batch=128, seed=0, lr=3e-4, log=print, init=None):
    """Train on `pairs` fresh pairs; returns (float32 parameters, metadata)."""
    tr = Trainer(model, batch=batch, seed=seed, lr=lr)
    tr.set_params(init_params(seed) if init is None else init)
    steps = (pairs + batch - 1) // batch
    hist = []
    t0 = time.time()
    for s in range(steps):
        if s == int(0.8 * steps):
            tr.lr = lr * 0.1
        e = tr.step()
        if s % 50 == 0 or s == steps - 1:
            e = e.cpu().numpy() * 1e3
            hist.append((s, float(e[0].mean()), float(e[1].mean())))
            log(f"step {s}/{steps}: eps_v estimate {e[0].mean():.2f} mm -> proposal {e[1].mean():.2f} mm "
                f"({time.time() - t0:.1f} s)")
    if tr.net.status() != B.HR_OK or B.hr_get_status(tr.bt) != B.HR_OK:
        raise RuntimeError("device status after training")
    params = torch.empty(tr.net.P, device=tr.cams.device)
    tr.net.get_params(params=params)
    torch.cuda.synchronize()
    meta = dict(pairs=steps * batch, batch=batch, steps=steps, lr=lr, seed=seed, train_spp=TRAIN_SPP,
                seconds=round(time.time() - t0, 1), history=hist)
    return params.cpu().numpy(), meta


def evaluate(model: B.Model, params, batches=4, batch=128, seed=12345):
    """Mean epsilon_v (mm) of estimates and of one proposal on held-out pairs."""
    tr = Trainer(model, batch=batch, seed=seed)
    tr.set_params(params)
    e = np.concatenate([tr.step(train=False).cpu().numpy() for _ in range(batches)], axis=1) * 1e3
    return float(e[0].mean()), float(e[1].mean())


# --------------------------------------------------------------------------------------
# inference: proposal steps in front of the plain batched refinement
# --------------------------------------------------------------------------------------

def rig_views(cfgs, views: P.BatchViews, view_offsets, pixel_offsets):
    """The training rig's views of instances captured by other rigs: every instance
    must have a view at each of the rig's cameras (same elevation, radius and
    azimuths) at an integer multiple f of the rig's resolution.  Those views are
    reduced by f x f box means (hr_box_downsample; masks by block maxima) and their
    intrinsics scaled by 1/f, so the network sees its own camera layout.  Returns the
    rig-layout BatchViews (instances in order, the rig's view order)."""
    cams, bgs, obss, masks = [], [], [], []
    for i, cfg in enumerate(cfgs):
        f = cfg.width // RIG.width
        if (f < 1 or cfg.width != f * RIG.width or cfg.height != f * RIG.height or
                cfg.elevation_deg != RIG.elevation_deg or cfg.radius != RIG.radius):
            raise ValueError(f"instance {i}: its views do not contain the proposal rig's")
        idx = []
        for r in RIG.azimuths_deg:
            k = [j for j, az in enumerate(cfg.azimuths_deg) if abs((az - r + 180.0) % 360.0 - 180.0) < 1e-6]
            if not k:
                raise ValueError(f"instance {i}: no view at azimuth {r}")
            idx.append(k[0])
        H, W = cfg.height, cfg.width
        v0, p0 = int(view_offsets[i]), int(pixel_offsets[i])
        for k in idx:
            c = views.cams[v0 + k].clone()
            c[0:4] /= f
            cams.append(c)
            sl = slice(p0 + k * H * W, p0 + (k + 1) * H * W)
            out = []
            for src in (views.background, views.observed):
                dst = torch.empty((1, H // f, W // f, 3), device=src.device)
                B.hr_box_downsample(src[sl].reshape(1, H, W, 3), f, dst)
                out.append(dst.reshape(-1, 3))
            m = torch.empty((1, H // f, W // f), dtype=torch.uint8, device=views.mask.device)
            B.hr_mask_downsample(views.mask[sl].reshape(1, H, W), f, m)
            bgs.append(out[0])
            obss.append(out[1])
            masks.append(m.reshape(-1))
    return P.BatchViews(cams=torch.stack(cams), background=torch.cat(bgs), observed=torch.cat(obss),
                        mask=torch.cat(masks))


class Proposer:
    """Proposal steps for a BatchRefiner whose instances all use the training rig's
    layout (views x 256 x 256): candidates x_0 (the refiner's parameters) and
    x_{k+1} = x_k + delta(residuals of x_k); each candidate's masked photometric loss
    (hr_loss_batch at the refiner's samples) is recorded, and every instance keeps
    its lowest-loss candidate (hr_select_best) -- an instance whose proposals do not
    lower the loss keeps its initial estimate."""

    def __init__(self, refiner: P.BatchRefiner, params, steps=3):
        n, views = refiner.batch.n, refiner.batch.descs[0][0]
        for d in refiner.batch.descs:
            if (d[0], d[1], d[2]) != (views, 256, 256):
                raise ValueError("the proposal network takes instances of views x 256 x 256")
        self.r, self.steps = refiner, steps
        self.net = B.Net(n, views)
        self.net.set_params(torch.as_tensor(np.asarray(params, np.float32), device=refiner.params.device))
        dev = refiner.params.device
        self.cand = torch.empty((steps + 1, n, 61), device=dev)
        self.losses = torch.empty((steps + 1, n), device=dev)
        self.chosen = torch.empty(n, dtype=torch.int32, device=dev)

    def run(self, stream=None):
        r = self.r
        bt, m, v = r.batch, r.model, r.views
        B.hr_batch_set_active(bt, r.active)
        bt.active_mask = r.active
        self.cand[0].copy_(r.params)
        for k in range(self.steps + 1):
            x = self.cand[k]
            B.hr_skin_batch(bt, m, x, r.verts, stream)
            B.hr_build_bvh_batch(bt, m, r.verts, stream)
            B.hr_render_fwd_batch(bt, m, r.verts, v.cams, v.background, r.opts, r.image, stream)
            B.hr_loss_batch(bt, r.image, v.observed, v.mask, self.losses[k], r.adjoint, stream)
            if k < self.steps:
                self.net.inputs(r.image, v.observed, stream=stream)
                self.net.forward(v.cams, self.cand[k + 1], base=x, stream=stream)
        B.hr_select_best(self.cand, self.losses, r.params, self.chosen, stream)


def main():
    import argparse
    ap = argparse.ArgumentParser(description="train the proposal network on renderer-generated pairs")
    ap.add_argument("--pairs", type=int, default=200_000)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()
    hand = I.make_hand(0)
    model = B.Model(hand)
    params, meta = train(model, pairs=args.pairs, batch=args.batch, seed=args.seed, lr=args.lr)
    e0, e1 = evaluate(model, params)
    meta["heldout_eps_v_mm"] = {"estimate": round(e0, 3), "proposal": round(e1, 3)}
    print(json.dumps(meta["heldout_eps_v_mm"]), flush=True)
    save_weights(params, meta, args.out)
    print("saved", args.out, flush=True)


if __name__ == "__main__":
    main()
