"""GPU parity of the batched path: several hand instances with different view
counts, ragged resolutions, samples per pixel and edge-sample counts go through the
batch entry points in one launch per kernel, and every instance is compared with the
CPU oracle run on that instance alone (its own Philox instance field, spp and edge
samples).  Same bars as the single-instance parity tests."""
import numpy as np
import pytest

import oracle
from paper_2107_05509_gb300 import inputs as I
from tests.gpu_common import grad_ok, hand, pixel_ok, require_gpu, torch

pytestmark = pytest.mark.gpu

# (views, width, height, spp, edge samples, Philox instance, azimuth offset, seed)
DESCS = [
    (2, 64, 48, 4, 512, 5, 0.0, 11),
    (3, 37, 29, 3, 300, 9, 40.0, 12),    # ragged: neither size a multiple of the 8x4 sub-tile
    (1, 72, 64, 2, 0, 2, 200.0, 13),     # no edge samples
]


class Inst:
    def __init__(self, d):
        N, W, H, spp, ne, inst, az0, seed = d
        h = hand()
        cfg = I.SceneConfig(f"batch-{seed}", views=N, width=W, height=H, spp=spp, edge_samples=ne,
                            elevation_deg=20.0, azimuths_deg=tuple(az0 + 90.0 * k for k in range(N)), seed=seed)
        cams = I.pack_cameras(I.make_cameras(cfg, h.v_template.mean(0)))
        for c in cams:   # zoom in so that the hand fills the small images
            c[0:2] *= 2.5
        self.N, self.W, self.H, self.spp, self.ne, self.inst = N, W, H, spp, ne, inst
        self.cams = cams
        self.bg = I.background(seed, N, H, W)
        self.x = I.perturb_params(I.gt_params(seed), seed).astype(np.float32)
        self.verts = oracle.skin(h, self.x).astype(np.float32)
        self.normals = oracle.vertex_normals(self.verts, h.faces, h.vf_offsets, h.vf_faces)
        self.opts = oracle.make_opts(seed=4242, iter=3, instance=inst, spp=spp, edge_samples=ne, ka=I.K_AMBIENT,
                                     kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB,
                                     edge_eps=I.EDGE_EPS_PX)
        self.ref = oracle.render_fwd(self.verts, h.faces, self.normals, h.albedo, cams, H, W, self.bg, self.opts)
        self.observed = I.add_noise(self.bg, seed, 0.05)
        self.mask = np.ones((N, H, W), np.uint8)
        self.mask[:, : H // 3] = 0   # a partial mask


@pytest.fixture(scope="module")
def setup():
    require_gpu()
    from paper_2107_05509_gb300 import binding as B
    h = hand()
    insts = [Inst(d) for d in DESCS]
    bt = B.Batch(h.V, h.F, h.E, [(i.N, i.W, i.H, i.spp, i.ne, i.inst) for i in insts])
    model = B.Model(h)
    return B, h, insts, bt, model


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _cat(arrs, shape_tail):
    return np.concatenate([np.asarray(a, np.float32).reshape((-1,) + shape_tail) for a in arrs])


def _gopts(B, o, flags=0):
    return B.render_opts(seed=o.seed_lo | (o.seed_hi << 32), iter=o.iter, ka=o.ka, kd=o.kd,
                         light_dir=tuple(o.light_dir), light_rgb=tuple(o.light_rgb), edge_eps_px=o.edge_eps,
                         flags=flags)


def test_layout(setup):
    B, h, insts, bt, model = setup
    assert list(bt.view_offsets) == list(np.cumsum([0] + [i.N for i in insts]))
    assert list(bt.pixel_offsets) == list(np.cumsum([0] + [i.N * i.H * i.W for i in insts]))


def test_batch_skin_and_adjoint(setup):
    B, h, insts, bt, model = setup
    n = len(insts)
    params = _t(np.stack([i.x for i in insts]))
    verts = torch.empty((n, h.V, 3), device="cuda")
    B.hr_skin_batch(bt, model, params, verts)
    g = verts.cpu().numpy()
    for k, i in enumerate(insts):
        assert np.abs(g[k] - oracle.skin(h, i.x)).max() < 2e-6
    rng = np.random.default_rng(1)
    dV = rng.normal(0, 1, (n, h.V, 3)).astype(np.float32)
    dp = torch.empty((n, 61), device="cuda")
    B.hr_skin_bwd_batch(bt, model, params, _t(dV), dp)
    gp = dp.cpu().numpy()
    for k, i in enumerate(insts):
        ok = grad_ok(gp[k], oracle.skin_bwd(h, i.x, dV[k]))
        assert ok.all(), (k, np.argwhere(~ok))
    assert B.hr_get_status(bt) == B.HR_OK


def test_batch_forward_loss_backward(setup):
    B, h, insts, bt, model = setup
    n = len(insts)
    verts = _t(np.stack([i.verts for i in insts]))
    cams = _t(_cat([i.cams for i in insts], (I.CAM_FLOATS,)))
    bg = _t(_cat([i.bg for i in insts], (3,)))
    obs = _t(_cat([i.observed for i in insts], (3,)))
    mask = _t(np.concatenate([i.mask.reshape(-1) for i in insts]))
    P = bt.total_pixels
    img = torch.empty((P, 3), device="cuda")
    go = _gopts(B, insts[0].opts)
    B.hr_build_bvh_batch(bt, model, verts)
    B.hr_render_fwd_batch(bt, model, verts, cams, bg, go, img)
    g_img = img.cpu().numpy()
    po = bt.pixel_offsets
    for k, i in enumerate(insts):
        gi = g_img[po[k]:po[k + 1]].reshape(i.N, i.H, i.W, 3)
        ok = pixel_ok(gi, i.ref)
        assert ok.all(), (k, np.argwhere(~ok)[:5], np.abs(gi - i.ref).max())
    # per-instance loss and adjoint of the oracle's render
    ref_img = _t(_cat([i.ref.astype(np.float32) for i in insts], (3,)))
    loss = torch.zeros(n, device="cuda")
    adj = torch.empty((P, 3), device="cuda")
    B.hr_loss_batch(bt, ref_img, obs, mask, loss, adj)
    L = loss.cpu().numpy()
    A = adj.cpu().numpy()
    A_refs = []
    for k, i in enumerate(insts):
        L_ref, A_ref = oracle.loss(i.ref.astype(np.float32), i.observed, i.mask)
        assert abs(L[k] - L_ref) <= 1e-5 * abs(L_ref), (k, L[k], L_ref)
        a = A[po[k]:po[k + 1]].reshape(i.N, i.H, i.W, 3)
        assert np.array_equal(np.sign(a), np.sign(A_ref))
        assert np.abs(a - A_ref).max() <= 1e-7 * np.abs(A_ref).max()
        A_refs.append(A_ref.astype(np.float32))
    # backward of the oracle's adjoint, every term, per instance
    dv = torch.empty((n, h.V, 3), device="cuda")
    A_all = _t(_cat(A_refs, (3,)))
    refs = [oracle.render_bwd(h, i.verts, i.cams, i.H, i.W, i.bg, i.opts, A_refs[k], normals=i.normals)[0]
            for k, i in enumerate(insts)]
    # a traversal of its own, the forward's candidate lists (HR_BWD_REUSE_FWD), and
    # fixed-point sums (HR_DETERMINISTIC: a repeated call is bit-identical)
    for flags in (0, B.HR_BWD_REUSE_FWD, B.HR_DETERMINISTIC):
        B.hr_render_bwd_batch(bt, model, verts, cams, bg, _gopts(B, insts[0].opts, flags), A_all, dv)
        gd = dv.cpu().numpy()
        for k, i in enumerate(insts):
            ref = refs[k]
            assert np.abs(ref).max() > 0
            ok = grad_ok(gd[k], ref)
            assert ok.all(), (flags, k, np.argwhere(~ok)[:5], gd[k][~ok][:5], ref[~ok][:5])
        if flags == B.HR_DETERMINISTIC:
            again = torch.empty_like(dv)
            B.hr_render_bwd_batch(bt, model, verts, cams, bg, _gopts(B, insts[0].opts, flags), A_all, again)
            assert torch.equal(again, dv)
    assert B.hr_get_status(bt) == B.HR_OK


def test_batch_of_one_equals_single_context(setup):
    """A one-instance batch renders the same image, bit for bit, as a single-instance
    context given that instance's spp, edge samples and instance field."""
    B, h, insts, bt, model = setup
    i = insts[1]
    b1 = B.Batch(h.V, h.F, h.E, [(i.N, i.W, i.H, i.spp, i.ne, i.inst)])
    ctx = B.Context(h.V, h.F, h.E, i.N, i.W, i.H)
    v = _t(i.verts)
    cams, bg = _t(i.cams), _t(i.bg)
    a = torch.empty((i.N, i.H, i.W, 3), device="cuda")
    b = torch.empty_like(a)
    B.hr_build_bvh(ctx, model, v)
    o = i.opts
    single = B.render_opts(seed=o.seed_lo | (o.seed_hi << 32), iter=o.iter, instance=o.instance, spp=o.spp,
                           edge_samples=o.edge_samples, ka=o.ka, kd=o.kd, light_dir=tuple(o.light_dir),
                           light_rgb=tuple(o.light_rgb), edge_eps_px=o.edge_eps)
    B.hr_render_fwd(ctx, model, v, cams, i.H, i.W, bg, single, a)
    B.hr_build_bvh_batch(b1, model, v.reshape(1, h.V, 3))
    B.hr_render_fwd_batch(b1, model, v.reshape(1, h.V, 3), cams, bg, _gopts(B, o), b.reshape(-1, 3))
    assert torch.equal(a, b)
    assert B.hr_get_status(ctx) == B.HR_OK and B.hr_get_status(b1) == B.HR_OK


def test_batch_calls_reject_single_context(setup):
    B, h, insts, bt, model = setup
    i = insts[0]
    ctx = B.Context(h.V, h.F, h.E, i.N, i.W, i.H)
    v = _t(i.verts)
    with pytest.raises(B.HandrtError):
        B.hr_build_bvh_batch(ctx, model, v)
    with pytest.raises(B.HandrtError):
        B.hr_build_bvh(bt, model, v)


def test_vertex_error_matches_oracle(setup):
    B, h, insts, bt, model = setup
    n = len(insts)
    a = np.stack([i.verts for i in insts])
    b = np.stack([oracle.skin(h, I.gt_params(7 + k)).astype(np.float32) for k in range(n)])
    out = torch.full((4, n), -1.0, device="cuda")
    ctr = torch.full((1,), 2, dtype=torch.int32, device="cuda")
    B.hr_vertex_error(_t(a), _t(b), out, ctr)
    got = out.cpu().numpy()
    for k in range(n):
        assert abs(got[2, k] * 1e3 - oracle.vertex_error_mm(a[k], b[k])) <= 1e-5 * oracle.vertex_error_mm(a[k], b[k])
    assert (got[[0, 1, 3]] == -1.0).all()   # only row *iter_dev is written


def test_retired_instance_is_skipped_and_the_rest_unchanged(setup):
    """hr_batch_set_active: a retired instance (mask 0) is skipped by every batch call
    -- its vertices, image, loss and parameter gradient keep the values they had --
    while the active instances get exactly what an all-active call gives them."""
    B, h, insts, bt, model = setup
    n = len(insts)
    params = _t(np.stack([i.x for i in insts]))
    cams = _t(_cat([i.cams for i in insts], (I.CAM_FLOATS,)))
    bg = _t(_cat([i.bg for i in insts], (3,)))
    obs = _t(_cat([i.observed for i in insts], (3,)))
    mask = _t(np.concatenate([i.mask.reshape(-1) for i in insts]))
    P = bt.total_pixels
    po = bt.pixel_offsets
    go = _gopts(B, insts[0].opts, B.HR_DETERMINISTIC)

    def run(sentinel):
        verts = torch.full((n, h.V, 3), sentinel, device="cuda")
        img = torch.full((P, 3), sentinel, device="cuda")
        adj = torch.empty((P, 3), device="cuda")
        loss = torch.full((n,), sentinel, device="cuda")
        dv = torch.empty((n, h.V, 3), device="cuda")
        dp = torch.full((n, 61), sentinel, device="cuda")
        B.hr_skin_batch(bt, model, params, verts)
        B.hr_build_bvh_batch(bt, model, verts)
        B.hr_render_fwd_batch(bt, model, verts, cams, bg, go, img)
        B.hr_loss_batch(bt, img, obs, mask, loss, adj)
        B.hr_render_bwd_batch(bt, model, verts, cams, bg, go, adj, dv)
        B.hr_skin_bwd_batch(bt, model, params, dv, dp)
        return [t.cpu().numpy() for t in (verts, img, loss, dp)]

    B.hr_batch_set_active(bt, None)
    full = run(0.0)
    active = torch.tensor([1, 0, 1], dtype=torch.int32, device="cuda")
    B.hr_batch_set_active(bt, active)
    part = run(-7.0)
    B.hr_batch_set_active(bt, None)
    verts_f, img_f, loss_f, dp_f = full
    verts_p, img_p, loss_p, dp_p = part
    for k in (0, 2):
        assert np.array_equal(verts_p[k], verts_f[k])
        assert np.array_equal(img_p[po[k]:po[k + 1]], img_f[po[k]:po[k + 1]])
        assert loss_p[k] == loss_f[k]
        assert np.array_equal(dp_p[k], dp_f[k])    # fixed-point sums: order-free
    assert (verts_p[1] == -7.0).all() and (img_p[po[1]:po[2]] == -7.0).all()
    assert loss_p[1] == -7.0 and (dp_p[1] == -7.0).all()
    assert B.hr_get_status(bt) == B.HR_OK


def test_retire_converged_and_plateau_kernels(setup):
    B = setup[0]
    n = 5
    err = torch.tensor([[5e-3, 2e-3, 9e-4, 1e-3, 3e-3], [1e-4, 1e-4, 1e-4, 1e-4, 1e-4]], device="cuda")
    ctr = torch.zeros(1, dtype=torch.int32, device="cuda")
    active = torch.ones(n, dtype=torch.int32, device="cuda")
    scale = torch.ones((n, 61), device="cuda")
    B.hr_retire_converged(err, ctr, 1e-3, active, scale)
    # row 0: instances 2 and 3 are at or below 1 mm
    assert active.tolist() == [1, 1, 0, 0, 1]
    sc = scale.cpu().numpy()
    assert (sc[[2, 3]] == 0).all() and (sc[[0, 1, 4]] == 1).all()
    # the plateau rule: retire after `patience` calls without a relative improvement
    loss = torch.tensor([1.0, 1.0, 1.0, 1.0, 1.0], device="cuda")
    best = torch.full((n,), float("inf"), device="cuda")
    stall = torch.zeros(n, dtype=torch.int32, device="cuda")
    active.fill_(1)
    seq = [[1.0, 1.0, 1.0, 1.0, 1.0], [0.9, 1.0, 0.9995, 1.0, 0.5], [0.8, 1.0, 0.9993, 0.95, 0.4],
           [0.7, 1.0, 0.9992, 0.95, 0.3]]
    for row in seq:
        loss.copy_(torch.tensor(row, device="cuda"))
        B.hr_retire_plateau(loss, 1e-3, 3, best, stall, active)
    # instance 1 never improves and instance 2 by less than 0.1 % of its best: three
    # stalls each after the first call; instance 3 improves once (a reset), then stalls
    # twice; instances 0 and 4 keep improving
    assert active.tolist() == [1, 0, 0, 1, 1]
    assert stall.tolist()[3] == 1
    assert B.hr_get_status(setup[3]) == B.HR_OK
