"""Oracle pins for the Monte Carlo renderer and its derivative (Section 3.1,
"Rendering": pixel values are integrals, estimated with samples per pixel; the
renderer of Li et al. 2018 adds an edge-sampling term for visibility changes).

P3  one constant-colour triangle: the MC pixel estimate matches the exact
    pixel coverage (polygon clipping) within 4 sigma;
P4  its edge-sampling gradient matches the finite difference of the exact
    coverage; a front triangle over a back one gives contributions weighted by
    (front colour - back colour);
P5  away from visibility changes the interior gradient (plus the vertex-normal
    adjoint) matches central finite differences of the render with common
    random numbers.
"""
import numpy as np
import pytest

import oracle
from paper_2107_05509_gb300 import inputs as I
from tests import _exact_area as X


def _cam(W, H, f):
    return np.array([f, f, W / 2, H / 2, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0], np.float32)


def _flat_opts(seed, spp, edge_samples=0):
    # f = albedo * (ka + kd * sigma) with ka = 1, kd = 0: constant colour = albedo
    return oracle.make_opts(seed=seed, spp=spp, edge_samples=edge_samples, ka=1.0, kd=0.0,
                            light_dir=(0, 0, -1))


TRI = np.array([[-0.21, -0.13, 1.0], [0.27, -0.05, 1.1], [-0.02, 0.24, 0.95]], np.float32)


def test_coverage_matches_exact_area():
    H = W = 8
    cam = _cam(W, H, 12.0)
    faces = np.array([[0, 1, 2]], np.int32)
    ones = np.ones((3, 3), np.float32)
    normals = np.tile(np.array([0, 0, -1], np.float32), (3, 1))
    bg = np.zeros((1, H, W, 3), np.float32)
    S = 1 << 16
    img = oracle.render_fwd(TRI, faces, normals, ones, cam[None], H, W, bg, _flat_opts(11, S))[0, :, :, 0]
    exact = X.coverage(X.project(cam, TRI), H, W)
    assert exact.sum() > 3.0 and (exact > 0).sum() > 10 and ((exact > 0) & (exact < 1)).sum() > 8
    sigma = np.sqrt(exact * (1 - exact) / S) + 1.0 / S
    assert np.all(np.abs(img - exact) <= 4 * sigma)
    # a dropped sample, a shifted jitter or a half-pixel offset would all fail:
    assert np.abs(img - exact).max() < 0.01


def _edge_estimates(verts, faces, albedo, cam, H, W, A, n_seeds, n_samples):
    normals = np.tile(np.array([0, 0, -1], np.float32), (len(verts), 1))
    bg = np.zeros((1, H, W, 3), np.float32)
    edges, ef, _, _ = I.mesh_topology(faces, len(verts))
    sl, sc = oracle.silhouette_lists(verts, faces, edges, ef, cam[None])
    ests = []
    for s in range(n_seeds):
        o = _flat_opts(100 + s, 1, n_samples)
        ests.append(oracle.render_bwd_edges(verts, faces, normals, albedo, cam[None], H, W, bg, o, A, edges, sl, sc))
    ests = np.array(ests)
    return ests.mean(0), ests.std(0, ddof=1) / np.sqrt(n_seeds)


def test_edge_gradient_matches_exact_area_derivative():
    H = W = 8
    cam = _cam(W, H, 12.0)
    faces = np.array([[0, 1, 2]], np.int32)
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (1, H, W, 3)).astype(np.float32)
    Aw = A[0].astype(np.float64).sum(-1)     # colour 1 in every channel
    ones = np.ones((3, 3), np.float32)
    mean, se = _edge_estimates(TRI, faces, ones, cam, H, W, A, 16, 1 << 15)

    def objective(V):
        return float((Aw * X.coverage(X.project(cam, V), H, W)).sum())

    V64 = TRI.astype(np.float64)
    fd = np.zeros_like(V64)
    h = 1e-7
    for i in range(3):
        for c in range(3):
            Vp, Vm = V64.copy(), V64.copy()
            Vp[i, c] += h
            Vm[i, c] -= h
            fd[i, c] = (objective(Vp) - objective(Vm)) / (2 * h)
    assert np.abs(fd).max() > 1.0
    assert np.all(np.abs(mean - fd) <= 4 * se + 1e-6), (mean, fd, se)
    # sign and scale: a flipped normal or a missing N_sil factor is far outside
    assert np.abs(mean - fd).max() < 0.05 * np.abs(fd).max()


def test_edge_gradient_occlusion_weighted_by_colour_difference():
    H = W = 8
    cam = _cam(W, H, 12.0)
    front = np.array([[-0.2, -0.15, 1.0], [0.12, -0.1, 1.0], [-0.05, 0.2, 1.0]])
    back = np.array([[-0.3, -0.3, 2.0], [0.5, -0.2, 2.0], [0.0, 0.55, 2.0]])
    verts = np.concatenate([front, back]).astype(np.float32)
    faces = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    cF, cB = np.array([0.9, 0.6, 0.3]), np.array([0.2, 0.5, 0.7])
    albedo = np.concatenate([np.tile(cF, (3, 1)), np.tile(cB, (3, 1))]).astype(np.float32)
    rng = np.random.default_rng(4)
    A = rng.uniform(0.2, 1, (1, H, W, 3)).astype(np.float32)
    mean, se = _edge_estimates(verts, faces, albedo, cam, H, W, A, 16, 1 << 15)

    def objective(Vf):
        img = X.two_layer_image(X.project(cam, Vf), X.project(cam, back), cF, cB, H, W)
        return float((A[0] * img).sum())

    fd = np.zeros((3, 3))
    h = 1e-7
    for i in range(3):
        for c in range(3):
            Vp, Vm = front.copy(), front.copy()
            Vp[i, c] += h
            Vm[i, c] -= h
            fd[i, c] = (objective(Vp) - objective(Vm)) / (2 * h)
    assert np.all(np.abs(mean[:3] - fd) <= 4 * se[:3] + 1e-6), (mean[:3], fd, se[:3])
    # the back triangle lies fully inside the image with the front one inside it,
    # so its own edges see only (back colour - black)
    assert np.abs(mean[3:]).max() > 0


def _octahedron(rng):
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    v += rng.normal(0, 0.08, v.shape)
    f = np.array([[4, 0, 2], [4, 2, 1], [4, 1, 3], [4, 3, 0], [5, 2, 0], [5, 1, 2], [5, 3, 1], [5, 0, 3]], np.int32)
    return v.astype(np.float32), f


@pytest.mark.parametrize("light", [(0.3, 0.5, 0.8), (0.9, -0.2, 0.3)])
def test_interior_gradient_matches_fd_inside_closed_mesh(light):
    # camera inside a closed convex mesh: no silhouette edges, so the whole
    # derivative is the interior term plus the vertex-normal adjoint
    rng = np.random.default_rng(7)
    verts, faces = _octahedron(rng)
    _, _, vfo, vff = I.mesh_topology(faces, len(verts))
    albedo = rng.uniform(0.2, 0.9, (6, 3)).astype(np.float32)
    H = W = 24
    cam = _cam(W, H, 14.0)
    l = np.asarray(light) / np.linalg.norm(light)
    bg = np.zeros((1, H, W, 3), np.float32)
    A = rng.uniform(0.5, 1.5, (1, H, W, 3)).astype(np.float32)
    o = oracle.make_opts(seed=9, spp=16, edge_samples=0, ka=0.4, kd=0.6, light_dir=tuple(l))

    def L(V):
        n = oracle.vertex_normals(V, faces, vfo, vff)
        return float((A.astype(np.float64) * oracle.render_fwd(V, faces, n, albedo, cam[None], H, W, bg, o)).sum())

    n = oracle.vertex_normals(verts, faces, vfo, vff)
    dVi, dN = oracle.render_bwd_interior(verts, faces, n, albedo, cam[None], H, W, bg, o, A)
    grad = dVi + oracle.normal_adjoint(verts, faces, dN)
    h = 2e-4
    fd = np.zeros((6, 3))
    for i in range(6):
        for c in range(3):
            Vp, Vm = verts.copy(), verts.copy()
            Vp[i, c] += h
            Vm[i, c] -= h
            fd[i, c] = (L(Vp) - L(Vm)) / (Vp[i, c] - Vm[i, c])
    scale = np.abs(fd).max()
    assert scale > 1.0
    assert np.all(np.abs(grad - fd) <= 2e-3 * np.maximum(np.abs(fd), 0.05 * scale)), (grad, fd)
    # the normal adjoint is a real part of it
    assert np.abs(oracle.normal_adjoint(verts, faces, dN)).max() > 0.05 * scale


def test_interior_gradient_matches_fd_on_hand_away_from_silhouettes():
    hand = I.make_hand(0)
    cfg = I.TINY
    # a mild pose: strongly contorted poses make the procedural hand interpenetrate,
    # and intersection curves are visibility changes that lie on no mesh edge
    x = np.zeros(61, np.float32)
    x[0:10] = I.gt_params(cfg.seed)[0:10]
    x[55:58] = (0.1, 0.2, 0.0)
    x[10:55] = np.random.default_rng(8).normal(0, 0.05, 45)
    verts = oracle.skin(hand, x).astype(np.float32)
    cams = I.pack_cameras(I.make_cameras(cfg, hand.v_template.mean(0)))
    H, W = cfg.height, cfg.width
    bg = I.background(cfg.seed, cfg.views, H, W)
    o = oracle.make_opts(seed=5, spp=4, edge_samples=0, light_dir=I.LIGHT_DIR)
    # adjoint: positive weights, zero within 2 px of every silhouette edge
    A = np.random.default_rng(1).uniform(0.5, 1.5, (cfg.views, H, W, 3)).astype(np.float32)
    sl, sc = oracle.silhouette_lists(verts, hand.faces, hand.edges, hand.edge_faces, cams)
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    for v in range(cfg.views):
        P = X.project(cams[v], verts)
        for e in sl[v, :sc[v]]:
            a, b = P[hand.edges[e, 0]], P[hand.edges[e, 1]]
            ab = b - a
            t = np.clip(((xx - a[0]) * ab[0] + (yy - a[1]) * ab[1]) / max(ab @ ab, 1e-12), 0, 1)
            d = np.hypot(xx - a[0] - t * ab[0], yy - a[1] - t * ab[1])
            A[v][d < 2.5] = 0.0
    assert (A != 0).any(axis=-1).sum() > 300

    def L(V):
        n = oracle.vertex_normals(V, hand.faces, hand.vf_offsets, hand.vf_faces)
        return float((A.astype(np.float64) * oracle.render_fwd(V, hand.faces, n, hand.albedo, cams, H, W, bg, o)).sum())

    n = oracle.vertex_normals(verts, hand.faces, hand.vf_offsets, hand.vf_faces)
    dVi, dN = oracle.render_bwd_interior(verts, hand.faces, n, hand.albedo, cams, H, W, bg, o, A)
    grad = dVi + oracle.normal_adjoint(verts, hand.faces, dN)
    rng = np.random.default_rng(2)
    k = rng.normal(0, 1, (3, 3)) * 40.0
    smooth = np.sin(verts.astype(np.float64) @ k + rng.uniform(0, 6.28, 3))
    # along the gradient itself (every term positive) and along a smooth random field
    for dirn, rel in ((grad / np.abs(grad).max(), 2e-3), (smooth, 5e-3)):
        h = 4e-6
        Vp = (verts + h * dirn).astype(np.float32)
        Vm = (verts - h * dirn).astype(np.float32)
        fd = (L(Vp) - L(Vm)) / (2 * h)
        step = (Vp.astype(np.float64) - Vm) / (2 * h)     # the float32 step actually taken
        an = float((grad * step).sum())
        assert abs(an - fd) <= rel * float(np.abs(grad * step).sum()), (an, fd)
