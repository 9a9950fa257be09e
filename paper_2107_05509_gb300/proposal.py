"""Learned proposal for the refinement (an extension: the paper's Section 3 refines by
gradient descent alone).  A network (hr_net_*, bf16 on the tensor cores) maps the
residual images of an estimate to a parameter update; it is trained on pairs that
this library's renderer generates, and used for the first updates of a refinement,
with the photometric loss deciding per instance whether a proposal is kept -- the
plain method stays the fallback and the judge of its error.

Training pairs, in one of two camera layouts: "rig", the training rig (8 views of
256 x 256 on a ring at 0.6 m, elevation 30 degrees, azimuths 45 k); or "ring", the
views of a random ring of 4-16 cameras (elevation 30 degrees, evenly spaced from a
random start azimuth, native resolution 256 x 256, 512 x 384 or 512 x 512) placed in
the network's 8 slots by view_slots and area-resampled to 256 x 256 (a 512 x 384
view's pixels become anisotropic: fy scales by 256/384, fx by 256/512).  Each pair's
ground truth h ~ pose N(0, 0.4 rad) clipped to +-1.2, shape N(0, 1);
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
WEIGHTS_RING = os.path.join(HERE, "weights", "proposal_ring_bf16.npz")
LAYOUTS = ("rig", "ring")
SLOTS = 8                # views per instance the network takes (its view maximum)
NET_SIZE = 256           # their resolution (the network's inputs are 2 x 2 means)

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


def view_slots(k, slots=SLOTS):
    """The views of a k-view ring that fill the network's slots: evenly spread over
    the ring, each view taken twice or more when k < slots (a repeated view changes
    nothing in the maximum over views)."""
    if k < 1:
        raise ValueError("an instance needs a view")
    return [j * k // slots for j in range(slots)]


def ring_cameras(azimuths_deg, elevation_deg, radius, target, native_wh, size=NET_SIZE):
    """Packed cameras [n][20] of views on a ring looking at `target` (as
    inputs.make_cameras builds them at native resolution (W, H) = native_wh[i]),
    with the intrinsics scaled to a size x size image of the same field of view:
    fx, cx by size / W and fy, cy by size / H.  Vectorised: training draws a thousand
    cameras per step."""
    az = np.radians(np.asarray(azimuths_deg, np.float64))
    el = np.radians(elevation_deg)
    d = np.stack([np.sin(az) * np.cos(el), np.full_like(az, np.sin(el)), np.cos(az) * np.cos(el)], axis=1)
    pos = np.asarray(target, np.float64)[None, :] + radius * d
    fwd = np.asarray(target, np.float64)[None, :] - pos
    fwd /= np.linalg.norm(fwd, axis=1, keepdims=True)
    right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right, axis=1, keepdims=True)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)                 # [n][3][3], rows
    t = -np.einsum("nij,nj->ni", R, pos)
    wh = np.asarray(native_wh, np.float64).reshape(-1, 2)
    f = 1.2 * wh[:, 0]                                      # inputs.look_at_camera's focal length
    out = np.zeros((az.size, I.CAM_FLOATS), np.float32)
    out[:, 0] = (f * (size / wh[:, 0])).astype(np.float32)
    out[:, 1] = (f * (size / wh[:, 1])).astype(np.float32)
    out[:, 2] = (wh[:, 0] / 2.0 * (size / wh[:, 0])).astype(np.float32)
    out[:, 3] = (wh[:, 1] / 2.0 * (size / wh[:, 1])).astype(np.float32)
    out[:, 4:13] = R.reshape(-1, 9)
    out[:, 13:16] = t
    out[:, 16:19] = pos
    return out


def sample_ring_layouts(rng, n, target, slots=SLOTS, views=(4, 16)):
    """Cameras [n * slots][20] of n random ring layouts (the heterogeneous batch's
    distribution: view count uniform in `views`, start azimuth uniform, native
    resolution uniform over inputs.BATCH_RESOLUTIONS, elevation 30 degrees, 0.6 m),
    each instance's views placed in the slots by view_slots."""
    az, wh = [], []
    for _ in range(n):
        k = int(rng.integers(views[0], views[1] + 1))
        a0 = float(rng.uniform(0.0, 360.0))
        res = I.BATCH_RESOLUTIONS[int(rng.integers(0, len(I.BATCH_RESOLUTIONS)))]
        az += [a0 + 360.0 * j / k for j in view_slots(k, slots)]
        wh += [res] * slots
    return ring_cameras(az, RIG.elevation_deg, RIG.radius, target, wh)


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

    def __init__(self, model: B.Model, batch=128, seed=0, lr=3e-4, device="cuda", layout="rig"):
        if layout not in LAYOUTS:
            raise ValueError(f"layout: {layout}")
        self.model, self.B, self.seed, self.lr, self.layout = model, batch, seed, lr, layout
        hand = model.hand
        self.target = hand.v_template.mean(0)
        rig = RIG
        self.bt = B.Batch(hand.V, hand.F, hand.E, [(rig.views, rig.width, rig.height, TRAIN_SPP, 0, i)
                                                    for i in range(batch)])
        self.net = B.Net(batch, rig.views)
        cams1 = I.pack_cameras(I.make_cameras(rig, hand.v_template.mean(0)))
        self.cams = torch.as_tensor(np.concatenate([cams1] * batch), device=device)
        self.cams_in = torch.empty(tuple(self.cams.shape)).pin_memory()
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
        torch.cuda.current_stream().synchronize()    # the pinned staging buffers are free
        self.h_in[0].copy_(torch.from_numpy(gt))
        self.h_in[1].copy_(torch.from_numpy(x0))
        self.x_gt.copy_(self.h_in[0], non_blocking=True)
        self.x0.copy_(self.h_in[1], non_blocking=True)
        if self.layout == "ring":
            self.cams_in.copy_(torch.from_numpy(sample_ring_layouts(rng, self.B, self.target)))
            self.cams.copy_(self.cams_in, non_blocking=True)
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


def train(model: B.Model, pairs=200_000, batch=128, seed=0, lr=3e-4, log=print, init=None, layout="rig"):
    """Train on `pairs` fresh pairs; returns (float32 parameters, metadata)."""
    tr = Trainer(model, batch=batch, seed=seed, lr=lr, layout=layout)
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
                layout=layout, seconds=round(time.time() - t0, 1), history=hist)
    return params.cpu().numpy(), meta


def evaluate(model: B.Model, params, batches=4, batch=128, seed=12345, layout="rig"):
    """Mean epsilon_v (mm) of estimates and of one proposal on held-out pairs."""
    tr = Trainer(model, batch=batch, seed=seed, layout=layout)
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


def ring_views(cfgs, views: P.BatchViews, view_offsets, pixel_offsets, slots=SLOTS, size=NET_SIZE):
    """The network's views of instances on any camera layout (the "ring" network's
    inputs): each instance's views view_slots(k) area-resampled to size x size
    (hr_area_resample for plates and observations, hr_mask_resample for masks), with
    fx, cx scaled by size / W and fy, cy by size / H.  Returns the BatchViews of
    len(cfgs) x slots views of size x size (instances in order)."""
    n = len(cfgs)
    dev = views.cams.device
    NV, Pv = n * slots, size * size
    cams = torch.empty((NV, I.CAM_FLOATS), device=dev)
    bg = torch.empty((NV, size, size, 3), device=dev)
    obs = torch.empty((NV, size, size, 3), device=dev)
    mask = torch.empty((NV, size, size), dtype=torch.uint8, device=views.mask.device)
    scale = torch.empty(I.CAM_FLOATS, device=dev)
    for i, cfg in enumerate(cfgs):
        H, W = cfg.height, cfg.width
        v0, p0 = int(view_offsets[i]), int(pixel_offsets[i])
        if int(view_offsets[i + 1]) - v0 != cfg.views or int(pixel_offsets[i + 1]) - p0 != cfg.views * H * W:
            raise ValueError(f"instance {i}: layout does not match its config")
        scale.fill_(1.0)
        scale[0] = size / W
        scale[2] = size / W
        scale[1] = size / H
        scale[3] = size / H
        for j, k in enumerate(view_slots(cfg.views, slots)):
            d = i * slots + j
            torch.mul(views.cams[v0 + k], scale, out=cams[d])
            sl = slice(p0 + k * H * W, p0 + (k + 1) * H * W)
            B.hr_area_resample(views.background[sl].view(1, H, W, 3), bg[d:d + 1])
            B.hr_area_resample(views.observed[sl].view(1, H, W, 3), obs[d:d + 1])
            B.hr_mask_resample(views.mask[sl].view(1, H, W), mask[d:d + 1])
    return P.BatchViews(cams=cams, background=bg.view(NV * Pv, 3), observed=obs.view(NV * Pv, 3),
                        mask=mask.view(NV * Pv))


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
    ap.add_argument("--layout", choices=LAYOUTS, default="rig")
    ap.add_argument("--out", default=None, help="weights file (default: the layout's file in weights/)")
    args = ap.parse_args()
    if args.out is None:
        args.out = WEIGHTS if args.layout == "rig" else WEIGHTS_RING
    hand = I.make_hand(0)
    model = B.Model(hand)
    params, meta = train(model, pairs=args.pairs, batch=args.batch, seed=args.seed, lr=args.lr,
                         layout=args.layout)
    e0, e1 = evaluate(model, params, layout=args.layout)
    meta["heldout_eps_v_mm"] = {"estimate": round(e0, 3), "proposal": round(e1, 3)}
    print(json.dumps(meta["heldout_eps_v_mm"]), flush=True)
    save_weights(params, meta, args.out)
    print("saved", args.out, flush=True)


if __name__ == "__main__":
    main()
