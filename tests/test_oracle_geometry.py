"""Oracle pins: ray-triangle intersection, closest-hit choice, vertex normals,
silhouette edges.

The renderer's visibility (Section 3.1, "Rendering") rests on a Moller-Trumbore
hit test; these tests pin the oracle's float32 implementation against exact
answers on axis-aligned cases, against a float64 evaluation on random rays, and
the silhouette classification against a geometric invariant of convex meshes.
"""
import numpy as np

import oracle
from paper_2107_05509_gb300 import inputs as I


def _tri():
    verts = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 1.0], [0.0, 1.0, 1.0]], np.float32)
    return verts, np.array([[0, 1, 2]], np.int32)


def test_axis_aligned_exact():
    v, f = _tri()
    o = np.array([[0.25, 0.25, 0.0], [0.5, 0.5, 0.0], [0.6, 0.6, 0.0], [0.25, 0.25, 2.0], [0.0, 0.0, 0.0]],
                 np.float32)
    d = np.array([[0, 0, 1], [0, 0, 1], [0, 0, 1], [0, 0, 1], [0, 0, 1]], np.float32)
    tri, tuv = oracle.closest_hits(o, d, v, f)
    # interior point: t = 1, (u, v) = (x, y)
    assert tri[0] == 0 and tuple(tuv[0]) == (1.0, 0.25, 0.25)
    # on the hypotenuse u + v = 1 exactly: inside (closed triangle)
    assert tri[1] == 0 and tuple(tuv[1]) == (1.0, 0.5, 0.5)
    # outside
    assert tri[2] == -1
    # behind the origin (t < 0): miss
    assert tri[3] == -1
    # through a vertex: inside
    assert tri[4] == 0 and tuple(tuv[4]) == (1.0, 0.0, 0.0)


def test_parallel_ray_misses():
    v, f = _tri()
    tri, _ = oracle.closest_hits(np.array([[0.2, 0.2, 1.0]], np.float32), np.array([[1, 0, 0]], np.float32), v, f)
    assert tri[0] == -1


def test_double_sided_and_tie_rule():
    v, f = _tri()
    # reversed winding (back face) is still hit
    tri, tuv = oracle.closest_hits(np.array([[0.25, 0.25, 0.0]], np.float32), np.array([[0, 0, 1]], np.float32),
                                   v, f[:, ::-1].copy())
    assert tri[0] == 0
    # two coincident triangles: equal t, the lower id wins; a nearer one wins outright
    v2 = np.concatenate([v, v, v - np.array([0, 0, 0.5], np.float32)])
    f2 = np.array([[3, 4, 5], [0, 1, 2], [6, 7, 8]], np.int32)
    o = np.array([[0.25, 0.25, 0.0]], np.float32)
    tri, tuv = oracle.closest_hits(o, np.array([[0, 0, 1]], np.float32), v2, f2[:2])
    assert tri[0] == 0
    tri, tuv = oracle.closest_hits(o, np.array([[0, 0, 1]], np.float32), v2, f2)
    assert tri[0] == 2 and tuv[0, 0] == 0.5


def _mt64_all(o, d, V64, faces):
    """float64 Moller-Trumbore of one ray against every triangle: (t, u, v) arrays."""
    v0, v1, v2 = V64[faces[:, 0]], V64[faces[:, 1]], V64[faces[:, 2]]
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d[None], e2)
    det = np.einsum("ij,ij->i", e1, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = o[None] - v0
        u = np.einsum("ij,ij->i", s, p) / det
        q = np.cross(s, e1)
        v = (q @ d) / det
        t = np.einsum("ij,ij->i", e2, q) / det
    return t, u, v


def test_closest_hit_matches_float64_on_hand():
    hand = I.make_hand(0)
    verts = hand.v_template
    rng = np.random.default_rng(5)
    n = 2000
    target = verts[rng.integers(0, hand.V, n)].astype(np.float64)
    origins = target + 0.5 * I.random_unit(rng, n)
    dirs = (target - origins) + rng.normal(0, 0.01, (n, 3))
    tri, tuv = oracle.closest_hits(origins.astype(np.float32), dirs.astype(np.float32), verts, hand.faces)
    V64 = verts.astype(np.float64)
    checked = hits = 0
    for i in range(n):
        o = origins[i].astype(np.float32).astype(np.float64)
        d = dirs[i].astype(np.float32).astype(np.float64)
        t, u, v = _mt64_all(o, d, V64, hand.faces)
        m = np.minimum(np.minimum(u, v), 1 - u - v)
        ok = np.isfinite(t)
        if np.any(ok & (np.abs(m) < 1e-4) & (t > 0)):
            continue   # too close to an edge for an unambiguous answer
        inside = ok & (m >= 0) & (t > 0)
        best = int(np.argmin(np.where(inside, t, np.inf))) if inside.any() else -1
        checked += 1
        assert tri[i] == best
        if best >= 0:
            hits += 1
            assert abs(tuv[i, 0] - t[best]) <= 1e-5 * t[best]
    assert checked > 1500 and hits > 300


def test_vertex_normals_match_float64():
    hand = I.make_hand(0)
    v = hand.v_template
    n32 = oracle.vertex_normals(v, hand.faces, hand.vf_offsets, hand.vf_faces)
    V64 = v.astype(np.float64)
    f = hand.faces
    c = np.cross(V64[f[:, 1]] - V64[f[:, 0]], V64[f[:, 2]] - V64[f[:, 0]])
    m = np.zeros_like(V64)
    for k in range(3):
        np.add.at(m, f[:, k], c)
    n64 = m / np.linalg.norm(m, axis=1, keepdims=True)
    assert np.abs(n32 - n64).max() < 2e-6
    # outward: normals point away from the local centroid on the palm's front (+z)
    front = (v[:, 2] > 0.013) & (v[:, 1] > 0.03) & (v[:, 1] < 0.08)
    assert (n32[front, 2] > 0.5).all()


def _uv_sphere(nlat=12, nlon=16, r=0.05):
    verts = [(0, 0, r)]
    for i in range(1, nlat):
        th = np.pi * i / nlat
        for j in range(nlon):
            ph = 2 * np.pi * j / nlon
            verts.append((r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)))
    verts.append((0, 0, -r))
    faces = []
    for j in range(nlon):
        faces.append((0, 1 + j, 1 + (j + 1) % nlon))
    for i in range(nlat - 2):
        a, b = 1 + i * nlon, 1 + (i + 1) * nlon
        for j in range(nlon):
            j1 = (j + 1) % nlon
            faces.append((a + j, b + j, b + j1))
            faces.append((a + j, b + j1, a + j1))
    last = len(verts) - 1
    base = 1 + (nlat - 2) * nlon
    for j in range(nlon):
        faces.append((base + j, last, base + (j + 1) % nlon))
    return np.array(verts, np.float32), np.array(faces, np.int32)


def test_silhouette_convex_loop():
    # On a convex closed mesh every silhouette vertex has exactly two silhouette
    # edges (the silhouette is one closed loop), and every silhouette edge's
    # midpoint sees the camera almost tangentially.
    v, f = _uv_sphere()
    edges, ef, _, _ = I.mesh_topology(f, len(v))
    rng = np.random.default_rng(2)
    for _ in range(5):
        cam = I.pack_cameras([I.look_at_camera(0.6 * I.random_unit(rng, 1)[0] + np.array([0, 0.0, 0.0]),
                                               np.zeros(3), 64, 64)])[0]
        sil = oracle.silhouettes(v, f, edges, ef, cam)
        assert len(sil) >= 8
        deg = np.bincount(edges[sil].ravel(), minlength=len(v))
        assert set(np.unique(deg[deg > 0])) == {2}
        c = cam[16:19].astype(np.float64)
        mid = v[edges[sil]].astype(np.float64).mean(1)
        cosang = np.abs(np.einsum("ij,ij->i", mid / np.linalg.norm(mid, axis=1, keepdims=True),
                                  (mid - c) / np.linalg.norm(mid - c, axis=1, keepdims=True)))
        assert cosang.max() < 0.35


def test_silhouette_includes_boundary_edges():
    hand = I.make_hand(0)
    cams = I.pack_cameras(I.make_cameras(I.TINY, hand.v_template.mean(0)))
    sil = oracle.silhouettes(hand.v_template, hand.faces, hand.edges, hand.edge_faces, cams[0])
    boundary = np.nonzero(hand.edge_faces[:, 1] < 0)[0]
    assert set(boundary).issubset(set(sil))
    assert np.all(np.diff(sil) > 0)
