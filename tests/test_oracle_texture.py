"""Pins of the oracle's albedo texture (bilinear lookup at the hit's interpolated uv,
texel (i, j) centred at ((i + 0.5) / W, (j + 0.5) / H), clamp-to-edge) and of its
adjoint: the texel-centre convention on a mesh whose vertices share one uv; a
constant texture against the same constant per-vertex albedo; the texture gradient
against central differences (the render is linear in the texels, the hits do not
move); the vertex gradient through the texture coordinates against central
differences inside a closed mesh (no silhouettes)."""
import numpy as np
import pytest

import oracle
from paper_2107_05509_gb300 import inputs as I


def _octahedron(rng):
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    v += rng.normal(0, 0.08, v.shape)
    f = np.array([[4, 0, 2], [4, 2, 1], [4, 1, 3], [4, 3, 0], [5, 2, 0], [5, 1, 2], [5, 3, 1], [5, 0, 3]], np.int32)
    return v.astype(np.float32), f


def _inside_cam(W, H, f):
    c = np.zeros(20, np.float32)
    c[0:4] = (f, f, W / 2, H / 2)
    c[4:13] = np.eye(3).reshape(-1)
    return c


def _scene(seed=7, light=(0.3, 0.5, 0.8)):
    rng = np.random.default_rng(seed)
    verts, faces = _octahedron(rng)
    _, _, vfo, vff = I.mesh_topology(faces, len(verts))
    H = W = 20
    cam = _inside_cam(W, H, 12.0)
    l = np.asarray(light) / np.linalg.norm(light)
    return rng, verts, faces, vfo, vff, H, W, cam, tuple(l)


def _render(verts, faces, vfo, vff, cam, H, W, o, albedo=None):
    n = oracle.vertex_normals(verts, faces, vfo, vff)
    alb = albedo if albedo is not None else np.zeros((len(verts), 3), np.float32)
    return oracle.render_fwd(verts, faces, n, alb, cam[None], H, W, np.zeros((1, H, W, 3), np.float32), o)


@pytest.mark.parametrize("ux,expect", [(0.25, (1.0, 0.0)), (0.5, (0.5, 0.5)), (0.75, (0.0, 1.0)), (0.05, (1.0, 0.0)),
                                       (0.99, (0.0, 1.0))])
def test_texel_centres_and_clamping(ux, expect):
    """A 2x1 texture [c0, c1] seen at uv_x = 0.25 / 0.5 / 0.75 gives c0 / the mean / c1
    (texel centres at 0.25 and 0.75); beyond the centres the lookup clamps."""
    rng, verts, faces, vfo, vff, H, W, cam, l = _scene()
    c0, c1 = np.array([0.2, 0.5, 0.8]), np.array([0.9, 0.1, 0.4])
    tex = np.stack([c0, c1])[None].astype(np.float32)          # [1][2][3]
    uv = np.tile([ux, 0.5], (len(verts), 1)).astype(np.float32)
    o_t = oracle.make_opts(seed=3, spp=4, edge_samples=0, light_dir=l, texture=tex, uv=uv)
    alb = (expect[0] * c0 + expect[1] * c1).astype(np.float32)
    o_v = oracle.make_opts(seed=3, spp=4, edge_samples=0, light_dir=l)
    ref = _render(verts, faces, vfo, vff, cam, H, W, o_v, np.tile(alb, (len(verts), 1)))
    got = _render(verts, faces, vfo, vff, cam, H, W, o_t)
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-7)


def test_constant_texture_equals_constant_albedo():
    rng, verts, faces, vfo, vff, H, W, cam, l = _scene()
    tex = np.full((5, 7, 3), 0.37, np.float32)
    uv = rng.uniform(0.0, 1.0, (len(verts), 2)).astype(np.float32)
    o_t = oracle.make_opts(seed=4, spp=4, edge_samples=0, light_dir=l, texture=tex, uv=uv)
    o_v = oracle.make_opts(seed=4, spp=4, edge_samples=0, light_dir=l)
    ref = _render(verts, faces, vfo, vff, cam, H, W, o_v, np.full((len(verts), 3), 0.37, np.float32))
    assert np.allclose(_render(verts, faces, vfo, vff, cam, H, W, o_t), ref, rtol=1e-12, atol=1e-12)


def test_texture_gradient_matches_central_differences():
    rng, verts, faces, vfo, vff, H, W, cam, l = _scene(seed=8)
    tex = rng.uniform(0.2, 0.9, (16, 16, 3)).astype(np.float32)
    uv = rng.uniform(0.1, 0.9, (len(verts), 2)).astype(np.float32)
    A = rng.uniform(0.5, 1.5, (1, H, W, 3)).astype(np.float32)
    n = oracle.vertex_normals(verts, faces, vfo, vff)
    alb = np.zeros((len(verts), 3), np.float32)
    bg = np.zeros((1, H, W, 3), np.float32)

    def L(T):
        o = oracle.make_opts(seed=5, spp=8, edge_samples=0, light_dir=l, texture=T, uv=uv)
        return float((A.astype(np.float64) * oracle.render_fwd(verts, faces, n, alb, cam[None], H, W, bg, o)).sum())

    o = oracle.make_opts(seed=5, spp=8, edge_samples=0, light_dir=l, texture=tex, uv=uv)
    dT = np.zeros((16, 16, 3))
    oracle.render_bwd_interior(verts, faces, n, alb, cam[None], H, W, bg, o, A, d_texture=dT)
    assert np.abs(dT).max() > 0
    picks = list(zip(*np.nonzero(np.abs(dT) > 1e-3 * np.abs(dT).max())))
    idx = rng.choice(len(picks), size=min(20, len(picks)), replace=False)
    for k in idx:
        j, i, c = picks[k]
        Tp, Tm = tex.copy(), tex.copy()
        Tp[j, i, c] += 0.01
        Tm[j, i, c] -= 0.01
        fd = (L(Tp) - L(Tm)) / (float(Tp[j, i, c]) - float(Tm[j, i, c]))
        assert abs(fd - dT[j, i, c]) <= 1e-6 * max(abs(fd), 1e-3), (j, i, c, fd, dT[j, i, c])


@pytest.mark.parametrize("light", [(0.3, 0.5, 0.8), (0.9, -0.2, 0.3)])
def test_vertex_gradient_through_texture_matches_central_differences(light):
    rng, verts, faces, vfo, vff, H, W, cam, l = _scene(seed=9, light=light)
    y, x = np.mgrid[0:32, 0:32] / 32.0
    tex = np.stack([0.5 + 0.3 * np.sin(6 * x + 2 * y), 0.5 + 0.3 * np.cos(5 * y - x), 0.4 + 0.2 * x],
                   -1).astype(np.float32)
    uv = rng.uniform(0.15, 0.85, (len(verts), 2)).astype(np.float32)
    A = rng.uniform(0.5, 1.5, (1, H, W, 3)).astype(np.float32)
    alb = np.zeros((len(verts), 3), np.float32)
    bg = np.zeros((1, H, W, 3), np.float32)
    o = oracle.make_opts(seed=9, spp=16, edge_samples=0, light_dir=l, texture=tex, uv=uv)

    def L(V):
        n = oracle.vertex_normals(V, faces, vfo, vff)
        return float((A.astype(np.float64) * oracle.render_fwd(V, faces, n, alb, cam[None], H, W, bg, o)).sum())

    n = oracle.vertex_normals(verts, faces, vfo, vff)
    dVi, dN = oracle.render_bwd_interior(verts, faces, n, alb, cam[None], H, W, bg, o, A)
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
    assert np.all(np.abs(grad - fd) <= 5e-3 * np.maximum(np.abs(fd), 0.05 * scale)), (grad, fd)
