"""C-ABI behaviour on the GPU: the device iteration counter, the device-counted
Adam step, CUDA-graph replay of a whole iteration, and device-detected errors
reported through the status word (never a trap)."""
import ctypes

import numpy as np
import pytest

from tests.gpu_common import hand, require_gpu, scene, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    require_gpu()
    from paper_2107_05509_gb300 import binding
    return binding


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_iter_dev_matches_host_iter(B):
    sc = scene("tiny")
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    vt = _t(sc.verts)
    B.hr_build_bvh(ctx, model, vt)
    img_a = torch.empty((sc.N, sc.H, sc.W, 3), device="cuda")
    img_b = torch.empty_like(img_a)
    o = sc.opts(iter=7)
    B.hr_render_fwd(ctx, model, vt, _t(sc.cams), sc.H, sc.W, _t(sc.bg), sc.gpu_opts(o), img_a)
    counter = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    go = sc.gpu_opts(sc.opts(iter=0))
    go.iter_dev = counter.data_ptr()
    B.hr_render_fwd(ctx, model, vt, _t(sc.cams), sc.H, sc.W, _t(sc.bg), go, img_b)
    assert torch.equal(img_a, img_b)
    # a different iteration draws different samples
    o8 = sc.opts(iter=8)
    B.hr_render_fwd(ctx, model, vt, _t(sc.cams), sc.H, sc.W, _t(sc.bg), sc.gpu_opts(o8), img_b)
    assert not torch.equal(img_a, img_b)
    assert B.hr_get_status(ctx) == B.HR_OK


@pytest.mark.parametrize("n", [61, 786757])   # one block; many blocks and a separate counter advance
def test_adam_step_dev_matches_host_step_and_advances(B, n):
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=n).astype(np.float32)
    gr = rng.normal(size=n).astype(np.float32)
    pa, pb = _t(p0), _t(p0)
    ma, va, mb, vb = (torch.zeros(n, device="cuda") for _ in range(4))
    g = _t(gr)
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    for step in range(1, 4):
        B.hr_adam_step(pa, g, ma, va, 0.01, 0.9, 0.999, 1e-8, step)
        B.hr_adam_step_dev(pb, g, mb, vb, 0.01, 0.9, 0.999, 1e-8, counter)
    torch.cuda.synchronize()
    assert int(counter.item()) == 3
    assert torch.allclose(pa, pb, rtol=0, atol=1e-6)


def test_graph_replay_equals_eager_iteration(B):
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P
    sc = scene("tiny")
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    views = P.Views(cams=_t(sc.cams), background=_t(sc.bg), observed=_t(sc.observed), mask=_t(sc.mask),
                    H=sc.H, W=sc.W)
    counter = torch.full((1,), 2, dtype=torch.int32, device="cuda")
    opts = P.opts_for(sc.cfg, iter_dev=counter)
    ref = P.Refiner(model, views, opts, ctx=ctx)
    x = _t(sc.x0.astype(np.float32))
    loss_e, grad_e = ref.step(x)
    loss_e, grad_e = loss_e.clone(), grad_e.clone()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ref.step(x)
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        ref.step(x)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ref.loss, loss_e)
    assert torch.allclose(ref.d_params, grad_e, rtol=1e-5, atol=1e-7 * float(grad_e.abs().max()))
    assert B.hr_get_status(ctx) == B.HR_OK
    del I


def test_nonfinite_params_reported_in_status(B):
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, 1, 8, 8)
    x = np.zeros(61, np.float32)
    x[12] = np.nan
    v = torch.empty((h.V, 3), device="cuda")
    B.hr_skin(ctx, model, _t(x), v)
    assert B.hr_get_status(ctx) == B.HR_ERR_NONFINITE
    assert B.hr_get_status(ctx) == B.HR_OK          # read clears the word


def test_bad_face_index_reported_not_faulted(B):
    h = hand()
    model = B.Model(h)
    bad = model.t["faces"].clone()
    bad[5, 1] = h.V + 100                          # out of range: rejected by the build
    model.struct.faces = bad.data_ptr()
    ctx = B.Context(h.V, h.F, h.E, 1, 8, 8)
    B.hr_build_bvh(ctx, model, _t(h.v_template))
    assert B.hr_get_status(ctx) == B.HR_ERR_ARG
    model.struct.faces = model.t["faces"].data_ptr()
    B.hr_build_bvh(ctx, model, _t(h.v_template))
    assert B.hr_get_status(ctx) == B.HR_OK


def test_model_check_rejects_out_of_order_parents_and_bad_indices(B):
    """hr_model_check: the skinning kernels walk the kinematic chain from the root,
    so a parent table not in tree order is an argument error on the host, as are
    indices out of range; the model as generated passes."""
    h = hand()
    model = B.Model(h)                  # checked on creation
    assert B.lib().hr_model_check(ctypes.byref(model.struct)) == B.HR_OK
    good = model.t["parents"]
    for bad_parents in ([-1, 2, 0] + list(h.parents[3:]),      # joint 1's parent comes after it
                        [0] + list(h.parents[1:]),              # the root has a parent
                        list(h.parents[:5]) + [5] + list(h.parents[6:])):   # a joint is its own parent
        p = torch.as_tensor(np.asarray(bad_parents, np.int32), device="cuda")
        model.struct.parents = p.data_ptr()
        assert B.lib().hr_model_check(ctypes.byref(model.struct)) == B.HR_ERR_ARG
    model.struct.parents = good.data_ptr()
    bad = model.t["faces"].clone()
    bad[7, 2] = -1
    model.struct.faces = bad.data_ptr()
    assert B.lib().hr_model_check(ctypes.byref(model.struct)) == B.HR_ERR_ARG
    model.struct.faces = model.t["faces"].data_ptr()
    bad = model.t["edge_faces"].clone()
    bad[3, 0] = h.F
    model.struct.edge_faces = bad.data_ptr()
    assert B.lib().hr_model_check(ctypes.byref(model.struct)) == B.HR_ERR_ARG
    model.struct.edge_faces = model.t["edge_faces"].data_ptr()
    assert B.lib().hr_model_check(ctypes.byref(model.struct)) == B.HR_OK


def test_host_argument_errors(B):
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, 2, 16, 16)
    img = torch.empty((3, 16, 16, 3), device="cuda")
    cams = torch.zeros((3, 20), device="cuda")
    bg = torch.zeros_like(img)
    v = _t(h.v_template)
    B.hr_build_bvh(ctx, model, v)
    with pytest.raises(B.HandrtError) as e:           # 3 views > the context's 2
        B.hr_render_fwd(ctx, model, v, cams, 16, 16, bg, B.render_opts(), img)
    assert e.value.code == B.HR_ERR_ARG
    with pytest.raises(B.HandrtError) as e:           # spp 0
        B.hr_render_fwd(ctx, model, v, cams[:2], 16, 16, bg[:2], B.render_opts(spp=0), img[:2])
    assert e.value.code == B.HR_ERR_ARG
    with pytest.raises(B.HandrtError) as e:           # edge offset beyond the candidate lists' reach
        B.hr_render_fwd(ctx, model, v, cams[:2], 16, 16, bg[:2], B.render_opts(edge_eps_px=0.5), img[:2])
    assert e.value.code == B.HR_ERR_ARG
    lim = B.hr_limits(100000, 10, 10, 1, 8, 8)
    hnd = ctypes.c_void_p()
    assert B.lib().hr_context_create(ctypes.byref(lim), ctypes.byref(hnd)) == B.HR_ERR_UNSUPPORTED


def test_refit_gives_the_rebuilt_tree_results(B):
    """hr_update_bvh refits the previous tree (topology of another pose) on device
    iterations that are not multiples of rebuild_every: the render and the closest
    hits equal those of a full rebuild over the same vertices, bit for bit, and the
    render matches the oracle."""
    import oracle
    from tests.gpu_common import pixel_ok
    sc = scene("tiny")
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    v_a = _t(sc.verts)
    vb_np = oracle.skin(h, sc.x_gt).astype(np.float32)     # another pose, same faces
    v_b = _t(vb_np)
    cams, bg = _t(sc.cams), _t(sc.bg)
    o = sc.gpu_opts(sc.opts())
    img_refit = torch.empty((sc.N, sc.H, sc.W, 3), device="cuda")
    img_full = torch.empty_like(img_refit)
    rng = np.random.default_rng(2)
    nray = 4096
    cam = sc.cams[rng.integers(0, sc.N, nray)]
    orig = _t(cam[:, 16:19].copy())
    dirs = _t((vb_np[rng.integers(0, h.V, nray)] - cam[:, 16:19]).astype(np.float32))
    tri_r = torch.empty(nray, dtype=torch.int32, device="cuda")
    tri_f = torch.empty_like(tri_r)
    tuv_r = torch.empty((nray, 3), device="cuda")
    tuv_f = torch.empty_like(tuv_r)
    B.hr_build_bvh(ctx, model, v_a)
    counter = torch.full((1,), 3, dtype=torch.int32, device="cuda")
    B.hr_update_bvh(ctx, model, v_b, counter, 8)            # 3 % 8 != 0: refit
    B.hr_render_fwd(ctx, model, v_b, cams, sc.H, sc.W, bg, o, img_refit)
    B.hr_trace(ctx, orig, dirs, tri_r, tuv_r)
    B.hr_build_bvh(ctx, model, v_b)
    B.hr_render_fwd(ctx, model, v_b, cams, sc.H, sc.W, bg, o, img_full)
    B.hr_trace(ctx, orig, dirs, tri_f, tuv_f)
    assert torch.equal(img_refit, img_full)
    assert torch.equal(tri_r, tri_f) and torch.equal(tuv_r, tuv_f)
    n_b = oracle.vertex_normals(vb_np, h.faces, h.vf_offsets, h.vf_faces)
    ref = oracle.render_fwd(vb_np, h.faces, n_b, h.albedo, sc.cams, sc.H, sc.W, sc.bg, sc.opts())
    assert pixel_ok(img_refit.cpu().numpy(), ref).all()
    assert B.hr_get_status(ctx) == B.HR_OK


def test_lazy_refit_serves_per_ray_traversal(B):
    """On a refit iteration hr_update_bvh rewrites only the triangle records.  A
    forward whose sub-tiles meet more triangles than a candidate list holds (the
    whole hand inside a 16x16 view) traces them ray by ray through the BVH, whose
    boxes -- still those of another pose -- the render refits first.  The image
    equals the one after a full rebuild bit for bit and matches the oracle, and the
    forward's counters show the traversal."""
    import oracle
    from paper_2107_05509_gb300 import inputs as I
    from tests.gpu_common import Scene, pixel_ok
    cfg = I.SceneConfig("far-2x16x16-4spp", views=2, width=16, height=16, spp=4, edge_samples=64,
                        elevation_deg=20.0, azimuths_deg=(0.0, 90.0), seed=5)
    sc = Scene(cfg)
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    vb_np = oracle.skin(h, sc.x_gt).astype(np.float32)     # another pose, same faces
    v_a, v_b = _t(sc.verts), _t(vb_np)
    cams, bg = _t(sc.cams), _t(sc.bg)
    img_lazy = torch.empty((sc.N, sc.H, sc.W, 3), device="cuda")
    img_full = torch.empty_like(img_lazy)
    B.hr_build_bvh(ctx, model, v_a)
    counter = torch.full((1,), 3, dtype=torch.int32, device="cuda")
    B.hr_update_bvh(ctx, model, v_b, counter, 8)            # 3 % 8 != 0: records only
    B.hr_get_stats(ctx)                                     # clears the counters
    B.hr_render_fwd(ctx, model, v_b, cams, sc.H, sc.W, bg, sc.gpu_opts(sc.opts(), flags=B.HR_STATS), img_lazy)
    assert B.hr_get_stats(ctx)[0, 2] > 0                    # BVH nodes visited by per-ray traversal
    B.hr_build_bvh(ctx, model, v_b)
    B.hr_render_fwd(ctx, model, v_b, cams, sc.H, sc.W, bg, sc.gpu_opts(sc.opts()), img_full)
    assert torch.equal(img_lazy, img_full)
    n_b = oracle.vertex_normals(vb_np, h.faces, h.vf_offsets, h.vf_faces)
    ref = oracle.render_fwd(vb_np, h.faces, n_b, h.albedo, sc.cams, sc.H, sc.W, sc.bg, sc.opts())
    assert pixel_ok(img_lazy.cpu().numpy(), ref).all()
    assert B.hr_get_status(ctx) == B.HR_OK


def test_tunings_keep_results(B):
    """Every launch-shape setting renders and differentiates to the oracle's values
    (work-item splits change only the float32 summation grouping); invalid settings
    are refused on the host."""
    import oracle
    from tests.gpu_common import grad_ok, pixel_ok
    sc = scene("ragged")
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    vt, cams, bg = _t(sc.verts), _t(sc.cams), _t(sc.bg)
    o = sc.opts()
    ref = oracle.render_fwd(sc.verts, h.faces, sc.normals, h.albedo, sc.cams, sc.H, sc.W, sc.bg, o)
    _, A = oracle.loss(ref.astype(np.float32), sc.observed, sc.mask)
    A = A.astype(np.float32)
    g_ref, _ = oracle.render_bwd(h, sc.verts, sc.cams, sc.H, sc.W, sc.bg, o, A, normals=sc.normals)
    img = torch.empty((sc.N, sc.H, sc.W, 3), device="cuda")
    dv = torch.empty((h.V, 3), device="cuda")
    B.hr_build_bvh(ctx, model, vt)
    for t in ({"rays_per_lane": 1, "cand_per_chunk": 8, "max_chunks": 16, "blocks_per_sm": 4, "bwd_blocks_per_sm": 2,
               "bwd_rays_per_lane": 2, "bwd_cand_per_chunk": 16, "edge_lanes": 2},
              {"rays_per_lane": 2, "cand_per_chunk": 32, "max_chunks": 8, "blocks_per_sm": 8, "bwd_blocks_per_sm": 6,
               "bwd_rays_per_lane": 4, "bwd_cand_per_chunk": 8, "edge_lanes": 8},
              {"rays_per_lane": 4, "cand_per_chunk": 1, "max_chunks": 1, "blocks_per_sm": 1, "bwd_blocks_per_sm": 1,
               "bwd_rays_per_lane": 1, "bwd_cand_per_chunk": 1, "edge_lanes": 32}):
        ctx.set_tuning(**t)
        assert ctx.get_tuning() == t
        B.hr_render_fwd(ctx, model, vt, cams, sc.H, sc.W, bg, sc.gpu_opts(o), img)
        assert pixel_ok(img.cpu().numpy(), ref).all(), t
        B.hr_render_bwd(ctx, model, vt, cams, sc.H, sc.W, bg, sc.gpu_opts(o, B.HR_BWD_REUSE_FWD), _t(A), dv)
        assert grad_ok(dv.cpu().numpy(), g_ref).all(), t
    for bad in ({"rays_per_lane": 3}, {"max_chunks": 17}, {"blocks_per_sm": 0}, {"bwd_blocks_per_sm": 9},
                {"cand_per_chunk": 0}, {"bwd_rays_per_lane": 3}, {"bwd_cand_per_chunk": 0}, {"edge_lanes": 3},
                {"edge_lanes": 64}):
        with pytest.raises(B.HandrtError):
            ctx.set_tuning(**bad)
    assert B.hr_get_status(ctx) == B.HR_OK


def test_item_region_overflow_matches_oracle(B):
    """Sub-tiles whose work items do not fit the item region are handed whole to the
    overflow kernel; forward pixels and the backward gradient stay the oracle's.  A
    zoomed 2 x 64x48 scene at 16 spp with one candidate per work item asks for more
    items than the region holds (2 x sub-tiles + 1024): counted here from below by the
    distinct triangles covering each sub-tile's pixel centres."""
    import oracle
    from paper_2107_05509_gb300 import inputs as I
    from tests.gpu_common import grad_ok, pixel_ok
    h = hand()
    cfg = I.SceneConfig("overflow", views=2, width=64, height=48, spp=16, edge_samples=256, elevation_deg=20.0,
                        azimuths_deg=(30.0, 210.0), seed=41)
    cams = I.pack_cameras(I.make_cameras(cfg, h.v_template.mean(0)))
    for c in cams:
        c[0:2] *= 3.0
    N, H, W = cfg.views, cfg.height, cfg.width
    x = I.perturb_params(I.gt_params(cfg.seed), cfg.seed).astype(np.float32)
    verts = oracle.skin(h, x).astype(np.float32)
    normals = oracle.vertex_normals(verts, h.faces, h.vf_offsets, h.vf_faces)
    bg = I.background(cfg.seed, N, H, W)
    # lower bound on the items requested: a triangle covering a pixel centre of a
    # sub-tile meets its frustum, so it is among the sub-tile's candidates
    need = 0
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    for v in range(N):
        fx, fy, cx, cy = cams[v][:4]
        R, t = cams[v][4:13].reshape(3, 3).astype(np.float64), cams[v][13:16].astype(np.float64)
        P = verts.astype(np.float64) @ R.T + t
        sx, sy = fx * P[:, 0] / P[:, 2] + cx, fy * P[:, 1] / P[:, 2] + cy
        cover = [set() for _ in range((W // 8) * (H // 4))]
        for f, (i0, i1, i2) in enumerate(h.faces):
            ax, ay, bx, by, qx, qy = sx[i0], sy[i0], sx[i1], sy[i1], sx[i2], sy[i2]
            x0, x1 = int(max(0, np.floor(min(ax, bx, qx)))), int(min(W - 1, np.ceil(max(ax, bx, qx))))
            y0, y1 = int(max(0, np.floor(min(ay, by, qy)))), int(min(H - 1, np.ceil(max(ay, by, qy))))
            if x0 > x1 or y0 > y1 or min(P[i0, 2], P[i1, 2], P[i2, 2]) <= 0:
                continue
            px, py = xs[y0:y1 + 1, x0:x1 + 1], ys[y0:y1 + 1, x0:x1 + 1]
            e0 = (bx - ax) * (py - ay) - (by - ay) * (px - ax)
            e1 = (qx - bx) * (py - by) - (qy - by) * (px - bx)
            e2 = (ax - qx) * (py - qy) - (ay - qy) * (px - qx)
            inside = ((e0 > 0) & (e1 > 0) & (e2 > 0)) | ((e0 < 0) & (e1 < 0) & (e2 < 0))
            for yy, xx in zip(*np.nonzero(inside)):
                cover[((y0 + yy) // 4) * (W // 8) + (x0 + xx) // 8].add(f)
        need += sum(min(len(c), 16) for c in cover)
    subtiles = N * ((W + 7) // 8) * ((H + 3) // 4)
    assert need > 2 * subtiles + 1024, (need, subtiles)
    o = oracle.make_opts(seed=77, spp=cfg.spp, edge_samples=cfg.edge_samples, ka=I.K_AMBIENT, kd=I.K_DIFFUSE,
                         light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB, edge_eps=I.EDGE_EPS_PX)
    ref = oracle.render_fwd(verts, h.faces, normals, h.albedo, cams, H, W, bg, o)
    obs = I.add_noise(bg, cfg.seed, 0.05)
    mask = np.ones((N, H, W), np.uint8)
    _, A = oracle.loss(ref.astype(np.float32), obs, mask)
    A = A.astype(np.float32)
    g_ref, _ = oracle.render_bwd(h, verts, cams, H, W, bg, o, A, normals=normals)
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, N, W, H)
    ctx.set_tuning(rays_per_lane=4, cand_per_chunk=1, max_chunks=16, blocks_per_sm=8, bwd_blocks_per_sm=4,
                   bwd_rays_per_lane=4, bwd_cand_per_chunk=1)
    vt, ct, bt = _t(verts), _t(cams), _t(bg)
    img = torch.empty((N, H, W, 3), device="cuda")
    dv = torch.empty((h.V, 3), device="cuda")
    go = B.render_opts(seed=77, spp=cfg.spp, edge_samples=cfg.edge_samples, ka=I.K_AMBIENT, kd=I.K_DIFFUSE,
                       light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB, edge_eps_px=I.EDGE_EPS_PX)
    B.hr_build_bvh(ctx, model, vt)
    B.hr_render_fwd(ctx, model, vt, ct, H, W, bt, go, img)
    g = img.cpu().numpy()
    ok = pixel_ok(g, ref)
    assert ok.all(), (np.argwhere(~ok)[:5], np.abs(g - ref).max())
    for flags in (0, B.HR_BWD_REUSE_FWD):   # a gather of its own, and the forward's lists
        go.flags = flags
        B.hr_render_bwd(ctx, model, vt, ct, H, W, bt, go, _t(A), dv)
        gd = dv.cpu().numpy()
        ok = grad_ok(gd, g_ref)
        assert ok.all(), (flags, np.argwhere(~ok)[:5], gd[~ok][:5], g_ref[~ok][:5])
    assert B.hr_get_status(ctx) == B.HR_OK


def test_deterministic_backward_repeats_bit_for_bit(B):
    """HR_DETERMINISTIC: the vertex gradient of repeated backward calls with the same
    inputs is identical bit for bit (fixed-point sums), with a traversal of its own and
    with the forward's candidate lists, and it is still the oracle's gradient."""
    import oracle
    from tests.gpu_common import grad_ok
    sc = scene("ragged")
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    vt, cams, bg = _t(sc.verts), _t(sc.cams), _t(sc.bg)
    o = sc.opts()
    ref = oracle.render_fwd(sc.verts, h.faces, sc.normals, h.albedo, sc.cams, sc.H, sc.W, sc.bg, o)
    _, A = oracle.loss(ref.astype(np.float32), sc.observed, sc.mask)
    A = A.astype(np.float32)
    g_ref, _ = oracle.render_bwd(h, sc.verts, sc.cams, sc.H, sc.W, sc.bg, o, A, normals=sc.normals)
    img = torch.empty((sc.N, sc.H, sc.W, 3), device="cuda")
    B.hr_build_bvh(ctx, model, vt)
    B.hr_render_fwd(ctx, model, vt, cams, sc.H, sc.W, bg, sc.gpu_opts(o), img)
    At = _t(A)
    for flags in (B.HR_DETERMINISTIC, B.HR_DETERMINISTIC | B.HR_BWD_REUSE_FWD):
        outs = []
        for _ in range(3):
            dv = torch.empty((h.V, 3), device="cuda")
            B.hr_render_bwd(ctx, model, vt, cams, sc.H, sc.W, bg, sc.gpu_opts(o, flags), At, dv)
            outs.append(dv)
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2]), flags
        g = outs[0].cpu().numpy()
        ok = grad_ok(g, g_ref)
        assert ok.all(), (flags, np.argwhere(~ok)[:5], g[~ok][:5], g_ref[~ok][:5])
    assert B.hr_get_status(ctx) == B.HR_OK


def test_capture_step_replays_the_eager_step(B):
    """Refiner.capture_step: replaying the recorded step gives the eager step's loss
    (bit for bit) and gradient; a new value of the device counter draws new samples."""
    from paper_2107_05509_gb300 import pipeline as P
    sc = scene("tiny")
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    views = P.Views(cams=_t(sc.cams), background=_t(sc.bg), observed=_t(sc.observed), mask=_t(sc.mask),
                    H=sc.H, W=sc.W)
    counter = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    ref = P.Refiner(model, views, P.opts_for(sc.cfg, iter_dev=counter), ctx=ctx)
    x = _t(sc.x0.astype(np.float32))
    loss_e, grad_e = ref.step(x)
    loss_e, grad_e = loss_e.clone(), grad_e.clone()
    g = ref.capture_step(x)
    ref.loss.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ref.loss, loss_e)
    assert torch.allclose(ref.d_params, grad_e, rtol=1e-5, atol=1e-7 * float(grad_e.abs().max()))
    counter.fill_(6)
    g.replay()
    torch.cuda.synchronize()
    assert not torch.equal(ref.loss, loss_e)
    assert B.hr_get_status(ctx) == B.HR_OK


def test_streamed_refiner_matches_eager_steps(B):
    """StreamedRefiner: every submitted frame (its own parameters and counter, copied
    from pinned host memory while the step before runs) gives the loss of an eager
    step on the same inputs, bit for bit, and its gradient."""
    from paper_2107_05509_gb300 import pipeline as P
    sc = scene("tiny")
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, sc.N, sc.W, sc.H)
    views = P.Views(cams=_t(sc.cams), background=_t(sc.bg), observed=_t(sc.observed), mask=_t(sc.mask),
                    H=sc.H, W=sc.W)
    x0 = sc.x0.astype(np.float32)
    xs = [x0, x0 + np.float32(0.01), x0, x0 - np.float32(0.01), x0]
    counters = [5, 6, 7, 8, 9]
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    opts = P.opts_for(sc.cfg, iter_dev=counter)
    ref = P.Refiner(model, views, opts, ctx=ctx)
    want = []
    for x, c in zip(xs, counters):
        counter.fill_(c)
        loss, grad = ref.step(_t(x))
        want.append((loss.clone(), grad.clone()))
    pin = lambda t: t.cpu().pin_memory()
    frames = [P.HostFrame(observed=pin(views.observed), mask=pin(views.mask), background=pin(views.background),
                          cams=pin(views.cams), params=torch.from_numpy(x).pin_memory(),
                          iter=torch.tensor([c], dtype=torch.int32).pin_memory()) for x, c in zip(xs, counters)]
    streamer = P.StreamedRefiner(model, views, opts, ctx=ctx, params=_t(x0))
    h_loss = torch.zeros(len(frames)).pin_memory()
    h_grad = torch.zeros(len(frames), 61).pin_memory()
    s = torch.cuda.current_stream()
    streamer.order_after(s)
    for i, f in enumerate(frames):
        streamer.submit(f, h_loss[i:i + 1], h_grad[i], s)
    streamer.join(s)
    torch.cuda.synchronize()
    for i, (loss, grad) in enumerate(want):
        assert float(h_loss[i]) == float(loss.cpu()[0]), i
        g = grad.cpu()
        assert torch.allclose(h_grad[i], g, rtol=1e-5, atol=1e-7 * float(g.abs().max())), i
    assert float(h_loss[0]) != float(h_loss[1])
    assert B.hr_get_status(ctx) == B.HR_OK
