"""Synthetic inputs: the procedural hand's topology and the camera rig."""
import numpy as np

from paper_2107_05509_gb300 import inputs as I


def test_hand_counts_and_topology():
    h = I.make_hand(0)
    assert (h.V, h.F, h.E) == (778, 1538, 2315)
    boundary = h.edge_faces[:, 1] < 0
    assert boundary.sum() == 16
    assert h.V - h.E + h.F == 1                     # a disc: one boundary loop
    # consistent orientation: every directed edge appears once
    d = set()
    for f in h.faces:
        for k in range(3):
            e = (int(f[k]), int(f[(k + 1) % 3]))
            assert e not in d
            d.add(e)
    assert np.allclose(h.weights.sum(1), 1.0, atol=1e-6)
    assert (h.parents[1:] < np.arange(1, 16)).all()
    assert h.vf_offsets[-1] == 3 * h.F
    for v in range(0, h.V, 37):
        fs = h.vf_faces[h.vf_offsets[v]:h.vf_offsets[v + 1]]
        assert np.all(np.diff(fs) > 0) and all(v in h.faces[f] for f in fs)


def test_seeded_and_reproducible():
    a, b = I.make_hand(3), I.make_hand(3)
    assert np.array_equal(a.shapedirs, b.shapedirs) and np.array_equal(a.albedo, b.albedo)
    assert not np.array_equal(I.make_hand(4).albedo, a.albedo)
    assert np.array_equal(I.gt_params(5), I.gt_params(5))


def test_camera_rig_looks_at_hand():
    h = I.make_hand(0)
    target = h.v_template.mean(0)
    cams = I.pack_cameras(I.make_cameras(I.PAPER, target))
    assert cams.shape == (8, 20)
    for c in cams:
        R = c[4:13].reshape(3, 3).astype(np.float64)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
        P = R @ target + c[13:16]
        assert abs(P[0]) < 1e-6 and abs(P[1]) < 1e-6 and abs(P[2] - 0.6) < 1e-6
        assert np.allclose(-R.T @ c[13:16], c[16:19], atol=1e-6)


def test_loop_subdivision_of_the_hand():
    """Two Loop subdivisions: V + E new vertices per level (778 -> 3093 -> 12337), four
    faces per face, the one wrist loop kept (16 -> 64 boundary edges), Euler
    characteristic unchanged, orientation consistent (every interior edge traversed once
    each way), skin weights still a partition of unity, the surface inside the coarse
    mesh's bounding box (Loop's rules are convex combinations)."""
    h = I.make_hand(0)
    s = I.subdivide_hand(h, 2)
    assert (s.V, s.F) == (12337, 24608)
    assert int((s.edge_faces[:, 1] < 0).sum()) == 64
    assert s.V - s.E + s.F == h.V - h.E + h.F
    directed = {}
    for f in s.faces:
        for k in range(3):
            e = (int(f[k]), int(f[(k + 1) % 3]))
            assert e not in directed
            directed[e] = True
    interior = sum(1 for (a, b) in directed if (b, a) in directed) // 2
    assert interior == int((s.edge_faces[:, 1] >= 0).sum())
    assert np.abs(s.weights.sum(1) - 1.0).max() < 1e-5
    lo, hi = h.v_template.min(0), h.v_template.max(0)
    assert (s.v_template >= lo - 1e-6).all() and (s.v_template <= hi + 1e-6).all()
