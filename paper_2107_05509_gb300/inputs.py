"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module holds input *generation* only: a procedural hand model (template mesh,
shape blendshapes, skin weights, joints, albedo), calibrated pinhole cameras on a
ring around the hand, random background plates, parameter draws and observation
noise.  It contains none of the method's arithmetic (no skinning, no ray tracing,
no loss, no derivatives), so both sides of a parity test can import it without
sharing any computation.

The hand stands in for the MANO model the paper uses (Section 3: 10 shape, 45 pose,
3 root-rotation and 3 root-translation parameters, 61 in total); MANO itself is
licensed data and is not reproduced.  The mesh is a single welded manifold with
one boundary loop at the wrist: a palm tube (16-vertex rings that widen into
32-vertex rings) whose top ring splits into five 8-vertex finger tubes, each
closed by a two-vertex ridge cap.  With 3 + 8 palm rings and 10/12/12/12/12
finger rings it has exactly 778 vertices, 1538 triangles and a 16-edge wrist
loop (F = 2V - 2 - b for a disc).

Units are metres.  Rest pose: wrist at the origin, fingers along +y, palm normal +z.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_JOINTS = 16
N_SHAPE = 10
N_POSE = 45
N_PARAMS = 61          # [beta(10), theta(45), phi(3), tau(3)]
P_BETA, P_THETA, P_PHI, P_TAU = 0, 10, 55, 58

# ----------------------------------------------------------------------------------
# Workload configurations (multiview hand captures; the paper's rig averages about 30
# calibrated views at 16 samples per pixel, Section 3.3).
# ----------------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class SceneConfig:
    name: str
    views: int
    width: int
    height: int
    spp: int
    edge_samples: int            # silhouette-edge samples per view
    elevation_deg: float
    azimuths_deg: tuple
    radius: float = 0.6
    obs_spp: int = 64            # samples per pixel of the noise-free observation
    noise_sigma: float = 0.01
    mask_dilate_px: int = 8
    seed: int = 0


TINY = SceneConfig("tiny-2x128x128-4spp", views=2, width=128, height=128, spp=4,
                   edge_samples=1024, elevation_deg=20.0, azimuths_deg=(0.0, 90.0),
                   seed=0)
PAPER = SceneConfig("paper-8x512x384-16spp", views=8, width=512, height=384, spp=16,
                    edge_samples=4096, elevation_deg=30.0,
                    azimuths_deg=tuple(45.0 * k for k in range(8)), seed=1000)
CONFIGS = {0: TINY, 1: PAPER}

# Batched workload: independently seeded instances with their own view count,
# resolution (W, H) and samples per pixel; 4096 edge samples per view.
BATCH_RESOLUTIONS = ((256, 256), (512, 384), (512, 512))


def batch_configs(n: int = 64, seed_base: int = 2000, views=(4, 16), spp=(8, 32), edge_samples: int = 4096):
    """n instance scene configs: instance i has seed seed_base + i, a view count
    uniform in [views[0], views[1]], a resolution drawn from BATCH_RESOLUTIONS, spp
    uniform in [spp[0], spp[1]], cameras on a ring at 0.6 m (elevation 30 degrees,
    evenly spaced azimuths from a random start)."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(np.random.SeedSequence([seed_base + i, 77]))
        nv = int(rng.integers(views[0], views[1] + 1))
        w, h = BATCH_RESOLUTIONS[int(rng.integers(0, len(BATCH_RESOLUTIONS)))]
        s = int(rng.integers(spp[0], spp[1] + 1))
        az0 = float(rng.uniform(0.0, 360.0))
        out.append(SceneConfig(f"batch{seed_base}-{i}-{nv}x{w}x{h}-{s}spp", views=nv, width=w, height=h, spp=s,
                               edge_samples=edge_samples, elevation_deg=30.0,
                               azimuths_deg=tuple(az0 + 360.0 * k / nv for k in range(nv)), seed=seed_base + i))
    return out


# Scale workload: the hand Loop-subdivided twice (12,337 vertices, 24,608 triangles),
# 16 views of 1024 x 1024, 64 spp, 32768 edge samples per view.
SCALE = SceneConfig("scale-16x1024x1024-64spp", views=16, width=1024, height=1024, spp=64,
                    edge_samples=32768, elevation_deg=30.0, azimuths_deg=tuple(22.5 * k for k in range(16)),
                    seed=4000)


# ----------------------------------------------------------------------------------
# Procedural hand mesh
# ----------------------------------------------------------------------------------

# Fingers: thumb, index, middle, ring, pinky.
_FINGER_RINGS = (10, 12, 12, 12, 12)                 # rings beyond the knuckle ring
_FINGER_LEN = ((0.034, 0.029, 0.024), (0.040, 0.025, 0.020), (0.045, 0.028, 0.022),
               (0.042, 0.027, 0.021), (0.033, 0.021, 0.018))
_FINGER_RADIUS = ((0.0088, 0.0074), (0.0078, 0.0064), (0.0080, 0.0066),
                  (0.0077, 0.0063), (0.0071, 0.0058))
_FINGER_SPLAY_DEG = (48.0, 7.0, 0.0, -6.0, -13.0)   # rotation about +z, positive toward -x
_FINGER_LIFT = (0.55, 0.0, 0.0, 0.0, 0.0)           # +z component added to the direction
_PALM_Y16 = (0.0, 0.010, 0.020)
_PALM_Y32 = tuple(np.linspace(0.030, 0.085, 8))
_PALM_HALF_W = (0.030, 0.0425)                      # wrist, palm
_PALM_HALF_T = (0.018, 0.014)
_SUPERELLIPSE_P = 3.0


def _ring_section(ncol, half_w, half_t):
    """Ring of 2*ncol points on a flattened superellipse, ordered front row left to
    right, then back row right to left (x across, z = thickness)."""
    xs = half_w * (-1.0 + (2.0 * np.arange(ncol) + 1.0) / ncol)
    zs = half_t * np.clip(1.0 - np.abs(xs / half_w) ** _SUPERELLIPSE_P, 0.0, 1.0) ** (1.0 / _SUPERELLIPSE_P)
    front = np.stack([xs, zs], 1)
    back = np.stack([xs[::-1], -zs[::-1]], 1)
    return np.concatenate([front, back], 0)


def _strip(ring_a, ring_b):
    """Triangles joining two rings of equal size (quads split along a fixed diagonal)."""
    n = len(ring_a)
    tris = []
    for i in range(n):
        j = (i + 1) % n
        tris.append((ring_a[i], ring_b[i], ring_b[j]))
        tris.append((ring_a[i], ring_b[j], ring_a[j]))
    return tris


def _stitch_16_32(ring_a, ring_b):
    """Triangles joining a 16-ring to a 32-ring (vertex i of the small ring faces
    vertices 2i and 2i+1 of the large one)."""
    n = len(ring_a)
    m = len(ring_b)
    assert m == 2 * n
    tris = []
    for i in range(n):
        i1 = (i + 1) % n
        b0, b1, b2 = ring_b[2 * i], ring_b[2 * i + 1], ring_b[(2 * i + 2) % m]
        tris.append((ring_a[i], b0, b1))
        tris.append((ring_a[i], b1, ring_a[i1]))
        tris.append((ring_a[i1], b1, b2))
    return tris


def _ridge_cap(ring, a, b):
    """Close an 8-ring with a two-vertex ridge (a covers ring[0..3], b ring[4..7])."""
    r = ring
    return [(a, r[0], r[1]), (a, r[1], r[2]), (a, r[2], r[3]),
            (b, r[4], r[5]), (b, r[5], r[6]), (b, r[6], r[7]),
            (a, r[3], b), (b, r[3], r[4]), (b, r[7], a), (a, r[7], r[0])]


def _orient_outward(verts, faces, boundary_centre):
    """Make the orientation of a connected manifold consistent (breadth-first over edge
    neighbours) and outward (positive volume once the boundary is closed by a fan)."""
    faces = [list(f) for f in faces]
    edge_faces = {}
    for fi, f in enumerate(faces):
        for k in range(3):
            a, b = f[k], f[(k + 1) % 3]
            edge_faces.setdefault((min(a, b), max(a, b)), []).append(fi)
    done = np.zeros(len(faces), bool)
    done[0] = True
    queue = [0]
    while queue:
        fi = queue.pop()
        f = faces[fi]
        for k in range(3):
            a, b = f[k], f[(k + 1) % 3]
            for gj in edge_faces[(min(a, b), max(a, b))]:
                if gj == fi or done[gj]:
                    continue
                g = faces[gj]
                # consistent neighbours traverse the shared edge in opposite directions
                same_dir = any(g[m] == a and g[(m + 1) % 3] == b for m in range(3))
                if same_dir:
                    g[1], g[2] = g[2], g[1]
                done[gj] = True
                queue.append(gj)
    assert done.all(), "mesh is not connected"
    f = np.asarray(faces, np.int64)
    v = verts.astype(np.float64)
    c = boundary_centre
    vol = np.einsum("ij,ij->i", v[f[:, 0]] - c, np.cross(v[f[:, 1]] - c, v[f[:, 2]] - c)).sum()
    if vol < 0:
        f = f[:, [0, 2, 1]]
    return f


@dataclasses.dataclass
class HandModel:
    """Arrays of the procedural hand (all float32 / int32, C-contiguous)."""
    v_template: np.ndarray     # [V][3]
    shapedirs: np.ndarray      # [V][3][K]
    weights: np.ndarray        # [V][J]
    j_template: np.ndarray     # [J][3]
    j_shapedirs: np.ndarray    # [J][3][K]
    parents: np.ndarray        # [J]   (parents[0] = -1, parents[j] < j)
    faces: np.ndarray          # [F][3]
    edges: np.ndarray          # [E][2]   (a < b)
    edge_faces: np.ndarray     # [E][2]   (-1 = boundary)
    vf_offsets: np.ndarray     # [V+1]   vertex -> incident faces, CSR
    vf_faces: np.ndarray       # [3F]    ascending face ids per vertex
    albedo: np.ndarray         # [V][3]
    uv: np.ndarray = None      # [V][2] texture coordinates (planar projection of the rest pose)

    @property
    def V(self):
        return self.v_template.shape[0]

    @property
    def F(self):
        return self.faces.shape[0]

    @property
    def E(self):
        return self.edges.shape[0]


def mesh_topology(faces, n_verts):
    """Edge list (with adjacent faces) and the vertex->face CSR of a triangle mesh."""
    emap = {}
    for fi, f in enumerate(faces):
        for k in range(3):
            a, b = int(f[k]), int(f[(k + 1) % 3])
            emap.setdefault((min(a, b), max(a, b)), []).append(fi)
    keys = sorted(emap)
    edges = np.array(keys, np.int32)
    ef = np.full((len(keys), 2), -1, np.int32)
    for i, k in enumerate(keys):
        fl = sorted(emap[k])
        assert len(fl) <= 2, "non-manifold edge"
        ef[i, :len(fl)] = fl
    counts = np.zeros(n_verts + 1, np.int64)
    for f in faces:
        for v in f:
            counts[v + 1] += 1
    offsets = np.cumsum(counts).astype(np.int32)
    vf = np.zeros(offsets[-1], np.int32)
    fill = offsets[:-1].copy()
    for fi, f in enumerate(faces):           # faces visited in ascending id order
        for v in f:
            vf[fill[v]] = fi
            fill[v] += 1
    return edges, ef, offsets, vf


def _segment_distance(p, a, b):
    ab = b - a
    t = np.clip(((p - a) @ ab) / max(float(ab @ ab), 1e-30), 0.0, 1.0)
    return np.linalg.norm(p - (a + t[:, None] * ab), axis=1)


def make_hand(seed: int = 0) -> HandModel:
    """Build the procedural hand; `seed` drives blendshapes and albedo only."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 778]))
    verts = []
    faces = []

    def add_ring(points3):
        base = len(verts)
        verts.extend(points3)
        return list(range(base, base + len(points3)))

    # palm
    rings16, rings32 = [], []
    for y in _PALM_Y16:
        s = min(1.0, y / 0.03)
        hw = _PALM_HALF_W[0] + (_PALM_HALF_W[1] - _PALM_HALF_W[0]) * s
        ht = _PALM_HALF_T[0] + (_PALM_HALF_T[1] - _PALM_HALF_T[0]) * s
        sec = _ring_section(8, hw, ht)
        rings16.append(add_ring([(x, y, z) for x, z in sec]))
    for y in _PALM_Y32:
        sec = _ring_section(16, _PALM_HALF_W[1], _PALM_HALF_T[1])
        rings32.append(add_ring([(x, y, z) for x, z in sec]))
    for r0, r1 in zip(rings16[:-1], rings16[1:]):
        faces += _strip(r0, r1)
    faces += _stitch_16_32(rings16[-1], rings32[0])
    for r0, r1 in zip(rings32[:-1], rings32[1:]):
        faces += _strip(r0, r1)
    knuckle = rings32[-1]

    # fingers
    joints = [np.zeros(3)]
    parents = [-1]
    bones = []                       # (joint index, segment start, segment end)
    for k in range(5):
        idx = [3 * k, 3 * k + 1, 3 * k + 2, 3 * k + 3,
               31 - (3 * k + 3), 31 - (3 * k + 2), 31 - (3 * k + 1), 31 - 3 * k]
        base_ring = [knuckle[i] for i in idx]
        base_pts = np.array([verts[i] for i in base_ring])
        centre = base_pts.mean(0)
        ang = math.radians(_FINGER_SPLAY_DEG[k])
        d = np.array([-math.sin(ang), math.cos(ang), _FINGER_LIFT[k]])
        d /= np.linalg.norm(d)
        zf = np.array([0.0, 0.0, 1.0]) - d[2] * d
        zf /= np.linalg.norm(zf)
        xf = np.cross(d, zf)
        L = _FINGER_LEN[k]
        total = sum(L)
        r0, r1 = _FINGER_RADIUS[k]
        nr = _FINGER_RINGS[k]
        prev = base_ring
        s_last = total - 0.5 * r1
        for j in range(1, nr + 1):
            s = s_last * j / nr
            rad = r0 + (r1 - r0) * s / total
            psi = np.radians(157.5 - 45.0 * np.arange(8))
            circ = centre + s * d + rad * (np.cos(psi)[:, None] * xf + np.sin(psi)[:, None] * zf)
            alpha = {1: 0.6, 2: 0.9}.get(j, 1.0)
            pts = alpha * circ + (1.0 - alpha) * (base_pts + s * d)
            ring = add_ring([tuple(p) for p in pts])
            faces += _strip(prev, ring)
            prev = ring
        tip_c = centre + total * d
        a = add_ring([tuple(tip_c - 0.2 * r1 * d + 0.35 * r1 * zf)])[0]
        b = add_ring([tuple(tip_c - 0.2 * r1 * d - 0.35 * r1 * zf)])[0]
        faces += _ridge_cap(prev, a, b)
        # joints: MCP, PIP, DIP; bones run to the next joint / the fingertip
        pts = [centre, centre + L[0] * d, centre + (L[0] + L[1]) * d, tip_c]
        for m in range(3):
            jid = len(joints)
            joints.append(pts[m])
            parents.append(0 if m == 0 else jid - 1)
            bones.append((jid, pts[m], pts[m + 1]))

    v = np.asarray(verts, np.float64)
    f = _orient_outward(v, faces, np.zeros(3))
    V, F = len(v), len(f)
    edges, ef, vfo, vff = mesh_topology(f, V)

    # skin weights: softmax of -distance / 5 mm to each joint's bone; the root's
    # "bone" is the palm plate (x in [-w+1cm, w-1cm], y in [0, knuckles-1.2cm], z=0)
    J = N_JOINTS
    dist = np.zeros((V, J))
    hw = _PALM_HALF_W[1] - 0.010
    px = np.clip(v[:, 0], -hw, hw)
    py = np.clip(v[:, 1], 0.0, _PALM_Y32[-1] - 0.012)
    dist[:, 0] = np.sqrt((v[:, 0] - px) ** 2 + (v[:, 1] - py) ** 2 + v[:, 2] ** 2)
    for jid, a, b in bones:
        dist[:, jid] = _segment_distance(v, np.asarray(a), np.asarray(b))
    logits = -dist / 0.005
    logits -= logits.max(1, keepdims=True)
    w = np.exp(logits)
    w /= w.sum(1, keepdims=True)

    # shape blendshapes: N(0, 2 mm) per vertex coordinate, 10 rounds of uniform
    # Laplacian smoothing (step 0.5), then rescaled to 2 mm RMS per shape
    nbrs = [[] for _ in range(V)]
    for a_, b_ in edges:
        nbrs[a_].append(b_)
        nbrs[b_].append(a_)
    S = rng.normal(0.0, 0.002, size=(V, 3, N_SHAPE))
    for _ in range(10):
        mean_n = np.stack([S[nb].mean(0) for nb in nbrs])
        S = S + 0.5 * (mean_n - S)
    S *= 0.002 / np.sqrt((S ** 2).mean(axis=(0, 1), keepdims=True))

    # joint regressor: J(beta) = J_template + SJ beta, SJ = weight-normalised mean of
    # each blendshape's displacement over the joint's vertices
    wsum = w.sum(0)
    SJ = np.einsum("vj,vck->jck", w, S) / wsum[:, None, None]

    # albedo: smooth value noise (sum of random 3-D sinusoids), remapped to [0.2, 0.9]
    alb = np.zeros((V, 3))
    for c in range(3):
        acc = np.zeros(V)
        for _ in range(6):
            omega = rng.normal(0.0, 1.0, 3) * (2 * math.pi / 0.06)
            acc += rng.uniform(0.5, 1.0) * np.sin(v @ omega + rng.uniform(0, 2 * math.pi))
        acc = (acc - acc.min()) / max(acc.max() - acc.min(), 1e-12)
        alb[:, c] = 0.2 + 0.7 * acc

    return HandModel(
        v_template=np.ascontiguousarray(v, np.float32),
        shapedirs=np.ascontiguousarray(S, np.float32),
        weights=np.ascontiguousarray(w, np.float32),
        j_template=np.ascontiguousarray(np.asarray(joints), np.float32),
        j_shapedirs=np.ascontiguousarray(SJ, np.float32),
        parents=np.asarray(parents, np.int32),
        faces=np.ascontiguousarray(f, np.int32),
        edges=edges, edge_faces=ef, vf_offsets=vfo, vf_faces=vff,
        albedo=np.ascontiguousarray(alb, np.float32),
        uv=planar_uv(v),
    )


def planar_uv(v):
    """Texture coordinates of the rest pose: its (x, y) projection scaled to the unit
    square (front and back share texels; there is no seam)."""
    v = np.asarray(v, np.float64)
    lo, hi = v[:, :2].min(0), v[:, :2].max(0)
    return np.ascontiguousarray((v[:, :2] - lo) / (hi - lo), np.float32)


def texture(seed: int, size: int = 256):
    """Albedo texture [size][size][3] from smooth noise (eight random 2-D sinusoids per
    channel, remapped to [0.2, 0.9])."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 256]))
    y, x = np.mgrid[0:size, 0:size] / size
    out = np.zeros((size, size, 3))
    for c in range(3):
        acc = np.zeros((size, size))
        for _ in range(8):
            k = rng.normal(0.0, 12.0, 2)
            acc += rng.uniform(0.5, 1.0) * np.sin(k[0] * x + k[1] * y + rng.uniform(0, 2 * math.pi))
        out[..., c] = 0.2 + 0.7 * (acc - acc.min()) / max(acc.max() - acc.min(), 1e-12)
    return np.ascontiguousarray(out, np.float32)


# ----------------------------------------------------------------------------------
# Cameras: pinhole, OpenCV convention (x right, y down, z forward), world -> camera
# ----------------------------------------------------------------------------------

CAM_FLOATS = 20   # fx fy cx cy R[9] t[3] centre[3] + pad; width/height passed separately


def look_at_camera(position, target, width, height, focal_scale=1.2):
    """Camera at `position` looking at `target`, world +y as the up hint."""
    pos = np.asarray(position, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ pos
    f = focal_scale * width
    return dict(fx=f, fy=f, cx=width / 2.0, cy=height / 2.0, R=R, t=t, centre=pos,
                width=width, height=height)


def make_cameras(cfg: SceneConfig, target):
    cams = []
    el = math.radians(cfg.elevation_deg)
    for az_deg in cfg.azimuths_deg:
        az = math.radians(az_deg)
        direction = np.array([math.sin(az) * math.cos(el), math.sin(el), math.cos(az) * math.cos(el)])
        cams.append(look_at_camera(np.asarray(target) + cfg.radius * direction, target,
                                   cfg.width, cfg.height))
    return cams


def pack_cameras(cams):
    """[N][20] float32 records: fx, fy, cx, cy, R (row-major 9), t (3), centre (3), 0.

    The camera centre is stored explicitly (the position the camera was built
    from, rounded once to float32) so that every consumer starts primary rays
    from the same float32 origin."""
    out = np.zeros((len(cams), CAM_FLOATS), np.float32)
    for i, c in enumerate(cams):
        out[i, 0:4] = (c["fx"], c["fy"], c["cx"], c["cy"])
        out[i, 4:13] = np.asarray(c["R"]).reshape(9)
        out[i, 13:16] = c["t"]
        out[i, 16:19] = c["centre"]
    return out


# ----------------------------------------------------------------------------------
# Parameters, backgrounds, observation noise, masks
# ----------------------------------------------------------------------------------


def gt_params(seed: int):
    """Ground-truth 61-vector: pose N(0, 0.4 rad) clipped to +-1.2, shape N(0, 1),
    root rotation and translation zero."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 61]))
    x = np.zeros(N_PARAMS, np.float64)
    x[P_BETA:P_BETA + N_SHAPE] = rng.normal(0.0, 1.0, N_SHAPE)
    x[P_THETA:P_THETA + N_POSE] = np.clip(rng.normal(0.0, 0.4, N_POSE), -1.2, 1.2)
    return x.astype(np.float32)


def perturb_params(x_gt, seed: int, pose_sigma=0.1, shape_sigma=0.5, trans_sigma=0.005):
    """Initial estimate: GT + pose (theta and root rotation) N(0, 0.1 rad),
    shape N(0, 0.5), root translation N(0, 5 mm)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 62]))
    x = np.asarray(x_gt, np.float64).copy()
    x[P_BETA:P_BETA + N_SHAPE] += rng.normal(0.0, shape_sigma, N_SHAPE)
    x[P_THETA:P_TAU] += rng.normal(0.0, pose_sigma, N_POSE + 3)
    x[P_TAU:P_TAU + 3] += rng.normal(0.0, trans_sigma, 3)
    return x.astype(np.float32)


def background(seed: int, n, h, w):
    """Background plates: i.i.d. U(0, 1) RGB per pixel, [N][H][W][3] float32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 3]))
    return rng.random((n, h, w, 3), dtype=np.float32)


def add_noise(image, seed: int, sigma=0.01):
    rng = np.random.default_rng(np.random.SeedSequence([seed, 4]))
    return (image + rng.normal(0.0, sigma, image.shape)).astype(np.float32)


def dilate(mask, radius):
    """Chebyshev (square) dilation of a [N][H][W] boolean mask by `radius` pixels."""
    m = mask.copy()
    for _ in range(radius):
        p = np.pad(m, ((0, 0), (1, 1), (1, 1)))
        acc = np.zeros_like(m)
        for dy in (0, 1, 2):
            for dx in (0, 1, 2):
                acc |= p[:, dy:dy + m.shape[1], dx:dx + m.shape[2]]
        m = acc
    return m


def coverage_mask(clean_render, plate, radius):
    """Mask M = pixels whose noise-free render differs from the background plate
    in any channel (at least one sample hit the hand), dilated by `radius` px."""
    hit = np.any(clean_render != plate, axis=-1)
    return dilate(hit, radius).astype(np.uint8)


def random_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


LIGHT_DIR = tuple((np.array([0.3, 0.5, 0.8]) / np.linalg.norm([0.3, 0.5, 0.8])).astype(np.float32).tolist())
LIGHT_RGB = (1.0, 1.0, 1.0)
K_AMBIENT = 0.4
K_DIFFUSE = 0.6
EDGE_EPS_PX = 1e-3


# ----------------------------------------------------------------------------------
# Loop subdivision (the scale workload's finer hand)
# ----------------------------------------------------------------------------------

def loop_subdivision_matrix(faces, n_verts):
    """Sparse linear map (rows of (index, weight) per new vertex) of one Loop
    subdivision step, and the new faces.  New vertex i < n_verts is the even (old)
    vertex: interior (1 - n b) v + b sum(neighbours), b = (5/8 - (3/8 + cos(2 pi / n)
    / 4)^2) / n (Loop 1987); boundary 3/4 v + 1/8 (its two boundary neighbours).  New
    vertex n_verts + e is the odd vertex on edge e = (a, b): interior 3/8 (a + b) +
    1/8 (c + d) with c, d opposite the edge; boundary (a + b) / 2.  Each face splits
    into four with the orientation kept."""
    faces = np.asarray(faces, np.int64)
    edges, edge_faces, _, _ = mesh_topology(faces, n_verts)
    eidx = {(int(a), int(b)): i for i, (a, b) in enumerate(edges)}
    nbrs = [set() for _ in range(n_verts)]
    bnd_nbrs = [[] for _ in range(n_verts)]
    for i, (a, b) in enumerate(edges):
        a, b = int(a), int(b)
        nbrs[a].add(b)
        nbrs[b].add(a)
        if edge_faces[i, 1] < 0:
            bnd_nbrs[a].append(b)
            bnd_nbrs[b].append(a)
    rows = []
    for v in range(n_verts):
        if bnd_nbrs[v]:
            b1, b2 = bnd_nbrs[v][:2]
            rows.append([(v, 0.75), (b1, 0.125), (b2, 0.125)])
        else:
            n = len(nbrs[v])
            beta = (5.0 / 8.0 - (3.0 / 8.0 + 0.25 * np.cos(2.0 * np.pi / n)) ** 2) / n
            rows.append([(v, 1.0 - n * beta)] + [(u, beta) for u in sorted(nbrs[v])])
    for i, (a, b) in enumerate(edges):
        a, b = int(a), int(b)
        if edge_faces[i, 1] < 0:
            rows.append([(a, 0.5), (b, 0.5)])
            continue
        opp = []
        for fi in edge_faces[i]:
            f = faces[fi]
            opp.append(int([x for x in f if x != a and x != b][0]))
        rows.append([(a, 0.375), (b, 0.375), (opp[0], 0.125), (opp[1], 0.125)])
    new_faces = []
    for f in faces:
        a, b, c = (int(x) for x in f)
        ab = n_verts + eidx[(min(a, b), max(a, b))]
        bc = n_verts + eidx[(min(b, c), max(b, c))]
        ca = n_verts + eidx[(min(c, a), max(c, a))]
        new_faces += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return rows, np.asarray(new_faces, np.int32)


def _apply_rows(rows, x):
    x = np.asarray(x, np.float64)
    out = np.zeros((len(rows),) + x.shape[1:])
    for i, r in enumerate(rows):
        for j, w in r:
            out[i] += w * x[j]
    return out


def subdivide_hand(hand: HandModel, levels: int = 2) -> HandModel:
    """The hand after `levels` Loop subdivisions: positions, shape blendshapes, skin
    weights and albedo all follow the same (affine, rows summing to one) linear map;
    the skeleton and joint regressor are unchanged."""
    v, sd, w, alb, uv, faces = hand.v_template, hand.shapedirs, hand.weights, hand.albedo, hand.uv, hand.faces
    for _ in range(levels):
        rows, faces = loop_subdivision_matrix(faces, v.shape[0])
        v, sd, w, alb, uv = (_apply_rows(rows, a) for a in (v, sd, w, alb, uv))
    edges, edge_faces, vf_off, vf = mesh_topology(faces, v.shape[0])
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    return HandModel(v_template=f32(v), shapedirs=f32(sd), weights=f32(w), j_template=hand.j_template,
                     j_shapedirs=hand.j_shapedirs, parents=hand.parents, faces=np.ascontiguousarray(faces, np.int32),
                     edges=edges, edge_faces=edge_faces, vf_offsets=vf_off, vf_faces=vf, albedo=f32(alb),
                     uv=f32(uv))
