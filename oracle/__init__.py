"""CPU oracle of the hand-refinement hot path (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the bench's CPU-baseline / reference leg may
import this package.  It shares no code with the CUDA library and never imports it.

What it computes, step by step (Karvounas et al. 2021, Section 3):
  * skin(params)                -> vertices            G_v of Eq. 3 (LBS stand-in for MANO)
  * vertex_normals(verts)       -> shading normals     (float32 decision operands)
  * render_fwd(...)             -> image               R of Eq. 3, Monte Carlo pixel means
  * loss(image, obs, mask)      -> L, dL/dimage        D_c of Eq. 4, masked mean
  * render_bwd(...)             -> dL/dverts           interior + edge-sampling terms
  * skin_bwd(params, dverts)    -> dL/dparams          adjoint of G_v

Skinning, loss, normal adjoint: numpy float64, written out plainly.
Rendering: hr_oracle.c, brute force over all triangles (float32 decisions, float64
values).  Sample streams: Philox4x32-10.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i = ctypes.c_int
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_closest_hits.argtypes = [P, P, i, P, P, i, P, P]
        L.oracle_vertex_normals.argtypes = [P, i, P, P, P, P]
        L.oracle_silhouettes.argtypes = [P, P, P, P, i, P, P]
        L.oracle_silhouettes.restype = i
        L.oracle_render_fwd.argtypes = [P, i, P, i, P, P, P, i, i, i, P, P, P, i, i, i, i, i]
        L.oracle_render_bwd_interior.argtypes = [P, i, P, i, P, P, P, i, i, i, P, P, P, P, P, P, i, i, i, i, i]
        L.oracle_render_bwd_edges.argtypes = [P, i, P, i, P, P, P, i, i, i, P, P, P, P, P, P, i, P, i, i]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def _i32(a):
    return np.ascontiguousarray(a, np.int32)


def n_threads():
    return max(1, len(os.sched_getaffinity(0)))


# ------------------------------------------------------------------------------------
# Philox4x32-10
# ------------------------------------------------------------------------------------

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


# ------------------------------------------------------------------------------------
# Render options (the same fields the CUDA library takes)
# ------------------------------------------------------------------------------------

class Opts(ctypes.Structure):
    _fields_ = [("seed_lo", ctypes.c_uint32), ("seed_hi", ctypes.c_uint32), ("iter", ctypes.c_uint32),
                ("instance", ctypes.c_uint32), ("spp", ctypes.c_int32), ("edge_samples", ctypes.c_int32),
                ("ka", ctypes.c_float), ("kd", ctypes.c_float), ("light_dir", ctypes.c_float * 3),
                ("light_rgb", ctypes.c_float * 3), ("edge_eps", ctypes.c_float),
                ("texture", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("tex_w", ctypes.c_int32),
                ("tex_h", ctypes.c_int32)]


def make_opts(seed=0, iter=0, instance=0, spp=4, edge_samples=1024, ka=0.4, kd=0.6,
              light_dir=(0.0, 0.0, 1.0), light_rgb=(1.0, 1.0, 1.0), edge_eps=1e-3, texture=None, uv=None):
    """Render options; with `texture` ([H][W][3]) and `uv` ([V][2]) the albedo is the
    bilinear texture lookup at the hit's interpolated uv."""
    o = Opts()
    if texture is not None:
        o._tex = np.ascontiguousarray(texture, np.float32)
        o._uv = np.ascontiguousarray(uv, np.float32)
        o.texture = o._tex.ctypes.data
        o.uv = o._uv.ctypes.data
        o.tex_h, o.tex_w = o._tex.shape[0], o._tex.shape[1]
    o.seed_lo = seed & 0xFFFFFFFF
    o.seed_hi = (seed >> 32) & 0xFFFFFFFF
    o.iter = iter
    o.instance = instance
    o.spp = spp
    o.edge_samples = edge_samples
    o.ka, o.kd = ka, kd
    o.light_dir[:] = list(light_dir)
    o.light_rgb[:] = list(light_rgb)
    o.edge_eps = edge_eps
    return o


# ------------------------------------------------------------------------------------
# Geometry helpers (float32 decision operands)
# ------------------------------------------------------------------------------------

def closest_hits(origins, dirs, verts, faces):
    o, d, v, f = _f32(origins), _f32(dirs), _f32(verts), _i32(faces)
    n = o.shape[0]
    tri = np.zeros(n, np.int32)
    tuv = np.zeros((n, 3), np.float32)
    lib().oracle_closest_hits(_p(o), _p(d), n, _p(v), _p(f), f.shape[0], _p(tri), _p(tuv))
    return tri, tuv


def vertex_normals(verts, faces, vf_offsets, vf_faces):
    v = _f32(verts)
    out = np.zeros_like(v)
    lib().oracle_vertex_normals(_p(v), v.shape[0], _p(_i32(faces)), _p(_i32(vf_offsets)),
                                _p(_i32(vf_faces)), _p(out))
    return out


def silhouettes(verts, faces, edges, edge_faces, cam_record):
    v, e = _f32(verts), _i32(edges)
    out = np.zeros(e.shape[0], np.int32)
    cam = _f32(cam_record)
    n = lib().oracle_silhouettes(_p(v), _p(_i32(faces)), _p(e), _p(_i32(edge_faces)), e.shape[0],
                                 _p(cam), _p(out))
    return out[:n].copy()


# ------------------------------------------------------------------------------------
# Rendering (brute force)
# ------------------------------------------------------------------------------------

def render_fwd(verts, faces, normals, albedo, cams, H, W, background, opts, threads=None,
               rows=None, cols=None):
    """Forward render in float64: [N][H][W][3].  `rows` = (r0, r1) over the N*H stacked
    rows and `cols` = (c0, c1) restrict the work (other pixels stay 0)."""
    v, f, n, a = _f32(verts), _i32(faces), _f32(normals), _f32(albedo)
    cams = _f32(cams)
    N = cams.shape[0]
    bg = _f32(background)
    img = np.zeros((N, H, W, 3), np.float64)
    r0, r1 = rows if rows else (0, N * H)
    c0, c1 = cols if cols else (0, W)
    lib().oracle_render_fwd(_p(v), v.shape[0], _p(f), f.shape[0], _p(n), _p(a), _p(cams), N, H, W, _p(bg),
                            ctypes.byref(opts), _p(img), threads or n_threads(), r0, r1, c0, c1)
    return img


def render_bwd_interior(verts, faces, normals, albedo, cams, H, W, background, opts, adjoint,
                        threads=None, rows=None, cols=None, d_texture=None):
    """(dV, dN); with a texture in `opts`, dL/dtexture is added into d_texture
    (float64 [H_t][W_t][3]) when given."""
    v, f, n, a = _f32(verts), _i32(faces), _f32(normals), _f32(albedo)
    cams = _f32(cams)
    N = cams.shape[0]
    bg, A = _f32(background), _f32(adjoint)
    dV = np.zeros((v.shape[0], 3), np.float64)
    dN = np.zeros((v.shape[0], 3), np.float64)
    r0, r1 = rows if rows else (0, N * H)
    c0, c1 = cols if cols else (0, W)
    dT = d_texture if d_texture is not None else None
    if dT is not None:
        assert dT.dtype == np.float64 and dT.flags.c_contiguous
    lib().oracle_render_bwd_interior(_p(v), v.shape[0], _p(f), f.shape[0], _p(n), _p(a), _p(cams), N, H, W,
                                     _p(bg), ctypes.byref(opts), _p(A), _p(dV), _p(dN),
                                     None if dT is None else dT.ctypes.data_as(ctypes.c_void_p),
                                     threads or n_threads(), r0, r1, c0, c1)
    return dV, dN


def silhouette_lists(verts, faces, edges, edge_faces, cams):
    cams = _f32(cams)
    E = np.asarray(edges).shape[0]
    lists = np.zeros((cams.shape[0], E), np.int32)
    counts = np.zeros(cams.shape[0], np.int32)
    for i in range(cams.shape[0]):
        s = silhouettes(verts, faces, edges, edge_faces, cams[i])
        lists[i, :len(s)] = s
        counts[i] = len(s)
    return lists, counts


def render_bwd_edges(verts, faces, normals, albedo, cams, H, W, background, opts, adjoint, edges,
                     sil_lists, sil_counts, k_range=None):
    v, f, n, a = _f32(verts), _i32(faces), _f32(normals), _f32(albedo)
    cams = _f32(cams)
    N = cams.shape[0]
    bg, A = _f32(background), _f32(adjoint)
    sl, sc = _i32(sil_lists), _i32(sil_counts)
    dV = np.zeros((v.shape[0], 3), np.float64)
    k0, k1 = k_range if k_range else (0, opts.edge_samples)
    lib().oracle_render_bwd_edges(_p(v), v.shape[0], _p(f), f.shape[0], _p(n), _p(a), _p(cams), N, H, W,
                                  _p(bg), ctypes.byref(opts), _p(A), _p(_i32(edges)), _p(sl), _p(sc),
                                  sl.shape[1], _p(dV), k0, k1)
    return dV


def normal_adjoint(verts, faces, dN):
    """dL/dverts from dL/d(unit vertex normals), n_v = m_v/|m_v|,
    m_v = sum over incident faces of (v1-v0) x (v2-v0).  float64."""
    v = np.asarray(verts, np.float64)
    f = np.asarray(faces, np.int64)
    e1 = v[f[:, 1]] - v[f[:, 0]]
    e2 = v[f[:, 2]] - v[f[:, 0]]
    c = np.cross(e1, e2)
    m = np.zeros_like(v)
    for k in range(3):
        np.add.at(m, f[:, k], c)
    ln = np.linalg.norm(m, axis=1)
    safe = np.where(ln > 0, ln, 1.0)
    n = m / safe[:, None]
    dm = (dN - n * np.einsum("ij,ij->i", n, dN)[:, None]) / safe[:, None]
    dm[ln == 0] = 0.0
    dc = dm[f[:, 0]] + dm[f[:, 1]] + dm[f[:, 2]]
    de1 = np.cross(e2, dc)        # d(e1 x e2) . dc  w.r.t. e1
    de2 = np.cross(dc, e1)        # ... w.r.t. e2
    dV = np.zeros_like(v)
    np.add.at(dV, f[:, 1], de1)
    np.add.at(dV, f[:, 2], de2)
    np.add.at(dV, f[:, 0], -(de1 + de2))
    return dV


def render_bwd(hand, verts, cams, H, W, background, opts, adjoint, normals=None, threads=None, d_texture=None):
    """Full dL/dverts = interior + edge sampling + normal adjoint (float64); with a
    texture, dL/dtexture (interior only: the texture moves no edge) into d_texture."""
    if normals is None:
        normals = vertex_normals(verts, hand.faces, hand.vf_offsets, hand.vf_faces)
    dVi, dN = render_bwd_interior(verts, hand.faces, normals, hand.albedo, cams, H, W, background, opts,
                                  adjoint, threads=threads, d_texture=d_texture)
    sl, sc = silhouette_lists(verts, hand.faces, hand.edges, hand.edge_faces, cams)
    dVe = render_bwd_edges(verts, hand.faces, normals, hand.albedo, cams, H, W, background, opts, adjoint,
                           hand.edges, sl, sc)
    dVn = normal_adjoint(verts, hand.faces, dN)
    return dVi + dVe + dVn, dict(interior=dVi, edges=dVe, normals=dVn, dN=dN, sil_counts=sc)


# ------------------------------------------------------------------------------------
# Loss: masked mean L1 (D_c of Eq. 4 summed over views as in Eq. 3), float64
# ------------------------------------------------------------------------------------

def loss(image, observed, mask):
    """L = sum_p M_p sum_c |R - O| / (3 sum_p M_p); A = dL/dR = M sign(R - O) / (3 sum M),
    with sign(0) = 0.  An empty mask gives L = 0 and A = 0."""
    R = np.asarray(image, np.float64)
    O = np.asarray(observed, np.float64)
    M = np.asarray(mask).astype(np.float64)[..., None]
    cnt = 3.0 * M.sum()
    if cnt == 0:
        return 0.0, np.zeros_like(R)
    diff = R - O
    L = float((M * np.abs(diff)).sum() / cnt)
    A = M * np.sign(diff) / cnt
    return L, A


# ------------------------------------------------------------------------------------
# Skinning (G_v) and its adjoint, float64
# ------------------------------------------------------------------------------------

def _skew(r):
    return np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])


def _rod_coeffs(th):
    """A = sin t / t, B = (1 - cos t)/t^2, C = A'(t)/t, D = B'(t)/t (series near 0)."""
    if th < 1e-3:
        t2 = th * th
        A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0
        B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0
        C = -1.0 / 3.0 + t2 / 30.0 - t2 * t2 / 840.0
        D = -1.0 / 12.0 + t2 / 180.0 - t2 * t2 / 6720.0
    else:
        s, c = np.sin(th), np.cos(th)
        A = s / th
        B = (1.0 - c) / (th * th)
        C = (th * c - s) / th ** 3
        D = (th * s - 2.0 * (1.0 - c)) / th ** 4
    return A, B, C, D


def rodrigues(r):
    """Rotation matrix of the axis-angle vector r: I + A K + B K^2, K = [r]x."""
    r = np.asarray(r, np.float64)
    A, B, _, _ = _rod_coeffs(float(np.linalg.norm(r)))
    K = _skew(r)
    return np.eye(3) + A * K + B * (K @ K)


def rodrigues_grad(r, dR):
    """sum_ab dR[a,b] * dR[a,b]/dr_k for k = 0..2."""
    r = np.asarray(r, np.float64)
    th = float(np.linalg.norm(r))
    A, B, C, D = _rod_coeffs(th)
    K = _skew(r)
    K2 = K @ K
    out = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        Ek = _skew(e)
        dRk = A * Ek + B * (Ek @ K + K @ Ek) + C * r[k] * K + D * r[k] * K2
        out[k] = float((dR * dRk).sum())
    return out


def skin(hand, params, return_state=False):
    """v = sum_j w_vj (A_j [v_shaped; 1]) + tau with A_j = G_j [I | -J_j],
    G_j = G_parent [R_j | J_j - J_parent], G_0 = [R(phi) | J_0]."""
    x = np.asarray(params, np.float64)
    beta, theta, phi, tau = x[0:10], x[10:55], x[55:58], x[58:61]
    S = hand.shapedirs.astype(np.float64)
    vt = hand.v_template.astype(np.float64) + S @ beta
    Jr = hand.j_template.astype(np.float64) + hand.j_shapedirs.astype(np.float64) @ beta
    par = hand.parents
    nj = Jr.shape[0]
    Rl = [rodrigues(phi)] + [rodrigues(theta[3 * (j - 1):3 * j]) for j in range(1, nj)]
    RG = [None] * nj
    tG = [None] * nj
    for j in range(nj):
        if par[j] < 0:
            RG[j] = Rl[j]
            tG[j] = Jr[j].copy()
        else:
            p = par[j]
            RG[j] = RG[p] @ Rl[j]
            tG[j] = RG[p] @ (Jr[j] - Jr[p]) + tG[p]
    RA = np.stack(RG)                                     # [J,3,3]
    tA = np.stack([tG[j] - RG[j] @ Jr[j] for j in range(nj)])
    W = hand.weights.astype(np.float64)
    posed = np.einsum("jab,vb->vja", RA, vt) + tA[None]    # [V,J,3]
    verts = np.einsum("vj,vja->va", W, posed) + tau
    if return_state:
        return verts, dict(vt=vt, J=Jr, Rl=Rl, RG=RG, tG=tG, RA=RA, tA=tA)
    return verts


def skin_joints(hand, params):
    """G_J (Section 3, the prior term): the posed 3-D joint locations, the origin of
    each joint's global frame plus the root translation, [J][3]."""
    _, st = skin(hand, params, return_state=True)
    return np.stack(st["tG"]) + np.asarray(params, np.float64)[58:61]


def skin_bwd(hand, params, dverts, djoints=None):
    """dL/dparams [61] for upstream dL/dverts [V][3] and, optionally, dL/d(posed
    joints) [J][3] (reverse of `skin` and `skin_joints`)."""
    x = np.asarray(params, np.float64)
    theta, phi = x[10:55], x[55:58]
    dV = np.asarray(dverts, np.float64)
    _, st = skin(hand, params, return_state=True)
    W = hand.weights.astype(np.float64)
    vt, Jr, RA, RG, Rl = st["vt"], st["J"], st["RA"], st["RG"], st["Rl"]
    par = hand.parents
    nj = Jr.shape[0]
    g = np.zeros(61)
    g[58:61] = dV.sum(0)                                        # tau
    dJt = np.zeros((len(par), 3)) if djoints is None else np.asarray(djoints, np.float64)
    g[58:61] += dJt.sum(0)
    dRA = np.einsum("vj,va,vb->jab", W, dV, vt)                # [J,3,3]
    dtA = np.einsum("vj,va->ja", W, dV)                        # [J,3]
    dvt = np.einsum("vj,jab,va->vb", W, RA, dV)                # [V,3]
    S = hand.shapedirs.astype(np.float64)                      # [V,3,K]
    g[0:10] = np.einsum("vck,vc->k", S, dvt)
    # A_j = [RG_j | tG_j - RG_j J_j]
    dRG = [dRA[j] - np.outer(dtA[j], Jr[j]) for j in range(nj)]
    dtG = [dtA[j] + dJt[j] for j in range(nj)]
    dJ = [-RG[j].T @ dtA[j] for j in range(nj)]
    dRl = [None] * nj
    for j in range(nj - 1, -1, -1):
        p = par[j]
        if p < 0:
            dRl[j] = dRG[j]
            dJ[j] = dJ[j] + dtG[j]
        else:
            dRl[j] = RG[p].T @ dRG[j]
            dRG[p] = dRG[p] + dRG[j] @ Rl[j].T + np.outer(dtG[j], Jr[j] - Jr[p])
            dtG[p] = dtG[p] + dtG[j]
            dJ[j] = dJ[j] + RG[p].T @ dtG[j]
            dJ[p] = dJ[p] - RG[p].T @ dtG[j]
    g[55:58] = rodrigues_grad(phi, dRl[0])
    for j in range(1, nj):
        g[10 + 3 * (j - 1):10 + 3 * j] = rodrigues_grad(theta[3 * (j - 1):3 * j], dRl[j])
    SJ = hand.j_shapedirs.astype(np.float64)                   # [J,3,K]
    g[0:10] += np.einsum("jck,jc->k", SJ, np.stack(dJ))
    return g


def vertex_error_mm(verts_a, verts_b):
    """epsilon_v: mean per-vertex Euclidean distance in millimetres (Section 4.1)."""
    return float(np.linalg.norm(np.asarray(verts_a, np.float64) - np.asarray(verts_b, np.float64), axis=1).mean() * 1e3)


def adam_step(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, lr_scale=None):
    """One Adam step (Section 3.3 optimises with Adam; Kingma and Ba's update, in
    float64):
        m <- beta1 m + (1 - beta1) g
        v <- beta2 v + (1 - beta2) g^2
        p <- p - lr_i (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps)
    with step >= 1 counting the steps taken so far, this one included.  Entry i uses
    lr_i = lr * lr_scale[i % len(lr_scale)] when a scale vector is given (parameters
    of different units each get their own step), else lr.  Returns new arrays
    (params, m, v); the inputs are not modified."""
    if step < 1:
        raise ValueError("Adam's step count starts at 1")
    p = np.asarray(params, np.float64)
    g = np.asarray(grad, np.float64)
    m1 = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    m2 = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m1 / (1.0 - beta1 ** step)
    v_hat = m2 / (1.0 - beta2 ** step)
    lr_i = np.full(p.shape, float(lr))
    if lr_scale is not None:
        s = np.asarray(lr_scale, np.float64).reshape(-1)
        lr_i = lr * s[np.arange(p.size) % s.size].reshape(p.shape)
    return p - lr_i * m_hat / (np.sqrt(v_hat) + eps), m1, m2


def _fma32(a, b, c):
    """float32 fused multiply-add (the product of two float32 is exact in float64)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def loss_ct(render, observed, mask, T):
    """Data term with per-camera 3x3 colour transforms (Eq. 2): T_i R evaluated in
    float32 as fma(t2, r2, fma(t1, r1, t0 r0)) (the order the kernels use), d = T R - O;
    L = sum M |d| / (3 sum M), adjoint dL/dR = T^T (M sign(d) / (3 sum M)),
    dT_i = sum_p (M sign(d) / (3 sum M)) R_p^T."""
    R = np.asarray(render, np.float32)
    O = np.asarray(observed, np.float32)
    M = (np.asarray(mask) != 0).astype(np.float64)
    T = np.asarray(T, np.float32).reshape(-1, 3, 3)
    N = R.shape[0]
    cnt = M.sum()
    scale = 1.0 / (3.0 * cnt) if cnt > 0 else 0.0
    TR = np.empty_like(R)
    for c in range(3):
        t = T[:, c, :][:, None, None, :]
        TR[..., c] = _fma32(t[..., 2], R[..., 2], _fma32(t[..., 1], R[..., 1],
                                                          (t[..., 0].astype(np.float32) * R[..., 0]).astype(np.float32)))
    # the exact difference of the float32 transformed value and the observation (its
    # sign is that of the float32 difference the kernels take)
    d = TR.astype(np.float64) - O.astype(np.float64)
    s = np.sign(d) * M[..., None] * scale
    L = float((M[..., None] * np.abs(d)).sum() * scale)
    A = np.einsum("nji,nhwj->nhwi", T.astype(np.float64), s)
    dT = np.einsum("nhwi,nhwj->nij", s, R.astype(np.float64)).reshape(N, 9)
    return L, A, dT


def joint_prior(joints, target, gamma, weight):
    """E_2 (the prior term): weight * sum over joints and coordinates of the smooth L1
    f_2(x, y) = 0.5 (x - y)^2 / gamma for |x - y| < gamma, |x - y| - 0.5 gamma otherwise,
    between the target joints x and the model's joints y; returns (E_2, dE_2/dy)."""
    y = np.asarray(joints, np.float64)
    x = np.asarray(target, np.float64)
    d = y - x
    a = np.abs(d)
    quad = a < gamma
    f = np.where(quad, 0.5 * d * d / gamma, a - 0.5 * gamma)
    g = np.where(quad, d / gamma, np.sign(d))
    return float(weight * f.sum()), weight * g


def colour_map(v_low, v_high):
    """V(c) = V_low scaled up by nearest neighbour to V_high's size + V_high."""
    lo = np.asarray(v_low, np.float64)
    hi = np.asarray(v_high, np.float64)
    fy, fx = hi.shape[0] // lo.shape[0], hi.shape[1] // lo.shape[1]
    return np.repeat(np.repeat(lo, fy, axis=0), fx, axis=1) + hi


def colour_map_bwd(d_v, low_shape):
    """dL/dV_low: sums of dL/dV over each low texel's block."""
    d = np.asarray(d_v, np.float64)
    hl, wl = low_shape[0], low_shape[1]
    return d.reshape(hl, d.shape[0] // hl, wl, d.shape[1] // wl, 3).sum(axis=(1, 3))
