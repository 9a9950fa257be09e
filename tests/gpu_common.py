"""Shared set-up for the GPU parity tests: seeded scenes whose every input and
expected value comes from the seeded generators and the CPU oracle, never from the
CUDA path."""
import functools

import numpy as np
import pytest

import oracle
from paper_2107_05509_gb300 import inputs as I

torch = pytest.importorskip("torch")

# tolerances (spec bar, with the floors that keep near-zero entries meaningful)
PIX_REL, PIX_FLOOR = 1e-4, 1e-2
GRAD_REL, GRAD_FLOOR = 1e-3, 1e-3


def pixel_ok(gpu, ref):
    return np.abs(gpu - ref) <= PIX_REL * np.maximum(np.abs(ref), PIX_FLOOR)


def grad_ok(gpu, ref):
    floor = GRAD_FLOOR * np.abs(ref).max()
    return np.abs(gpu - ref) <= GRAD_REL * np.maximum(np.abs(ref), floor)


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05509_gb300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def hand():
    return I.make_hand(0)


class Scene:
    """A seeded multiframe: cameras, plate, observation (oracle render of the GT
    parameters plus noise), mask, init parameters and the init vertices from the
    oracle's skinning (rounded to float32: the shared input of the render stages)."""

    def __init__(self, cfg: I.SceneConfig, obs_spp=16):
        h = hand()
        self.cfg = cfg
        self.N, self.H, self.W = cfg.views, cfg.height, cfg.width
        self.cams = I.pack_cameras(I.make_cameras(cfg, h.v_template.mean(0)))
        self.bg = I.background(cfg.seed, self.N, self.H, self.W)
        self.x_gt = I.gt_params(cfg.seed)
        self.x0 = I.perturb_params(self.x_gt, cfg.seed)
        self.obs_spp = obs_spp
        self._obs = None
        self.verts = oracle.skin(h, self.x0).astype(np.float32)
        self.normals = oracle.vertex_normals(self.verts, h.faces, h.vf_offsets, h.vf_faces)

    def _observe(self):
        if self._obs is None:
            h = hand()
            v_gt = oracle.skin(h, self.x_gt).astype(np.float32)
            n_gt = oracle.vertex_normals(v_gt, h.faces, h.vf_offsets, h.vf_faces)
            o_obs = self.opts(spp=self.obs_spp, seed=self.cfg.seed * 7919 + 1)
            clean = oracle.render_fwd(v_gt, h.faces, n_gt, h.albedo, self.cams, self.H, self.W, self.bg, o_obs)
            clean32 = clean.astype(np.float32)
            self._obs = (I.add_noise(clean32, self.cfg.seed, self.cfg.noise_sigma),
                         I.coverage_mask(clean32, self.bg, self.cfg.mask_dilate_px))
        return self._obs

    @property
    def observed(self):
        return self._observe()[0]

    @property
    def mask(self):
        return self._observe()[1]

    def opts(self, spp=None, seed=None, iter=0, edge_samples=None):
        cfg = self.cfg
        return oracle.make_opts(seed=cfg.seed * 7919 + 17 if seed is None else seed, iter=iter, spp=spp or cfg.spp,
                                edge_samples=cfg.edge_samples if edge_samples is None else edge_samples,
                                ka=I.K_AMBIENT, kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB,
                                edge_eps=I.EDGE_EPS_PX)

    def gpu_opts(self, o, flags=0):
        from paper_2107_05509_gb300 import binding as B
        return B.render_opts(seed=o.seed_lo | (o.seed_hi << 32), iter=o.iter, instance=o.instance, spp=o.spp,
                             edge_samples=o.edge_samples, ka=o.ka, kd=o.kd, light_dir=tuple(o.light_dir),
                             light_rgb=tuple(o.light_rgb), edge_eps_px=o.edge_eps, flags=flags)


@functools.lru_cache(maxsize=None)
def scene(name):
    if name == "tiny":
        return Scene(I.TINY)
    if name == "ragged":
        cfg = I.SceneConfig("ragged-3x75x100-3spp", views=3, width=100, height=75, spp=3, edge_samples=777,
                            elevation_deg=25.0, azimuths_deg=(10.0, 130.0, 250.0), seed=7)
        return Scene(cfg)
    if name == "paper":
        return Scene(I.PAPER, obs_spp=4)
    raise KeyError(name)
