"""Thin Python binding of the handrt C ABI (include/handrt.h).

Argument marshalling only: every function forwards device pointers of torch tensors
(and the current CUDA stream) to the library, checks the returned status code and
raises HandrtError on failure.  All computation happens in the CUDA kernels; there
is no CPU or PyTorch fallback, and loading fails loudly when the library has not
been built (``python -m paper_2107_05509_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhandrt.so")

HR_OK = 0
HR_ERR_ARG = -1
HR_ERR_CUDA = -2
HR_ERR_LIMIT = -3
HR_ERR_NONFINITE = -4
HR_ERR_UNSUPPORTED = -5
HR_ERR_INTERNAL = -6
HR_ERR_TIMEOUT = -7
HR_BWD_NO_INTERIOR = 1
HR_BWD_NO_EDGES = 2
HR_BWD_NO_NORMALS = 4
HR_STATS = 8
HR_TIMING = 16
HR_BWD_REUSE_FWD = 32
HR_DETERMINISTIC = 64
KERNEL_TIMES = ("fwd_gather", "fwd_shade", "fwd_combine", "bwd_gather", "bwd_shade", "bwd_reduce", "silhouettes",
                "edge_samples", "normal_adjoint")

EXPORTS = ("hr_context_create", "hr_context_destroy", "hr_skin", "hr_skin_bwd", "hr_build_bvh", "hr_render_fwd",
           "hr_loss", "hr_render_bwd", "hr_adam_step", "hr_trace", "hr_get_normals", "hr_silhouettes",
           "hr_get_stats", "hr_get_status", "hr_status_string", "hr_skin_bwd_noalloc", "hr_kernel_times",
           "hr_adam_step_dev", "hr_vertex_error", "hr_batch_create", "hr_batch_layout", "hr_skin_batch",
           "hr_skin_bwd_batch", "hr_build_bvh_batch", "hr_render_fwd_batch", "hr_loss_batch", "hr_render_bwd_batch",
           "hr_gemm_bf16", "hr_net_param_count", "hr_net_create", "hr_net_destroy", "hr_net_set_params",
           "hr_net_get_params", "hr_net_inputs", "hr_net_set_inputs_bf16", "hr_net_forward", "hr_net_backward",
           "hr_net_adam", "hr_net_status", "hr_vertex_mse", "hr_add_noise", "hr_select_best", "hr_update_bvh",
           "hr_set_tuning", "hr_get_tuning", "hr_loss_ct",
           "hr_skin_joints", "hr_skin_bwd_joints", "hr_joint_prior", "hr_colour_map", "hr_colour_map_bwd",
           "hr_edges", "hr_edge_loss", "hr_model_check",
           "hr_batch_set_active", "hr_retire_converged", "hr_retire_plateau", "hr_box_downsample",
           "hr_mask_downsample", "hr_area_resample", "hr_mask_resample")


class HandrtError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {code} ({status_string(code)})")
        self.code = code


class hr_model(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int32), ("F", ctypes.c_int32), ("E", ctypes.c_int32), ("J", ctypes.c_int32),
                ("K", ctypes.c_int32)] + [(n, ctypes.c_void_p) for n in (
                    "v_template", "shapedirs", "weights", "j_template", "j_shapedirs", "parents", "faces", "edges",
                    "edge_faces", "vf_offsets", "vf_faces", "albedo", "uv")]


class hr_render_opts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("iter", ctypes.c_uint32), ("instance", ctypes.c_uint32),
                ("spp", ctypes.c_int32), ("edge_samples", ctypes.c_int32), ("ka", ctypes.c_float),
                ("kd", ctypes.c_float), ("light_dir", ctypes.c_float * 3), ("light_rgb", ctypes.c_float * 3),
                ("edge_eps_px", ctypes.c_float), ("flags", ctypes.c_uint32), ("iter_dev", ctypes.c_void_p),
                ("texture", ctypes.c_void_p), ("tex_w", ctypes.c_int32), ("tex_h", ctypes.c_int32),
                ("d_texture", ctypes.c_void_p)]


class hr_instance_desc(ctypes.Structure):
    _fields_ = [("views", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("spp", ctypes.c_int32), ("edge_samples", ctypes.c_int32), ("instance", ctypes.c_uint32)]


class hr_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("rays_per_lane", "cand_per_chunk", "max_chunks", "blocks_per_sm",
                                              "bwd_blocks_per_sm", "bwd_rays_per_lane", "bwd_cand_per_chunk",
                                              "edge_lanes")]


class hr_limits(ctypes.Structure):
    _fields_ = [("max_V", ctypes.c_int32), ("max_F", ctypes.c_int32), ("max_E", ctypes.c_int32),
                ("max_views", ctypes.c_int32), ("max_width", ctypes.c_int32), ("max_height", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"handrt CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -m paper_2107_05509_gb300.build`)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        sig = {
            "hr_context_create": [P, P],
            "hr_context_destroy": [P],
            "hr_skin": [P, P, P, P, P],
            "hr_skin_bwd": [P, P, P, P, P, P],
            "hr_skin_bwd_noalloc": [P, P, P, P, P],
            "hr_model_check": [P],
            "hr_batch_set_active": [P, P],
            "hr_box_downsample": [P, I, I, I, I, P, P],
            "hr_mask_downsample": [P, I, I, I, I, P, P],
            "hr_area_resample": [P, I, I, I, P, I, I, P],
            "hr_mask_resample": [P, I, I, I, P, I, I, P],
            "hr_retire_converged": [P, P, I, I, F, P, P, I, P],
            "hr_retire_plateau": [P, I, F, I, P, P, P, P, I, P],
            "hr_build_bvh": [P, P, P, P],
            "hr_update_bvh": [P, P, P, P, I, P],
            "hr_set_tuning": [P, P],
            "hr_loss_ct": [P, P, P, P, P, I, I, I, P, P, P, P],
            "hr_skin_joints": [P, P, P, P, P, P],
            "hr_skin_bwd_joints": [P, P, P, P, P, P, P],
            "hr_joint_prior": [P, P, I, I, F, F, P, P, P],
            "hr_colour_map": [P, I, I, P, I, I, P, P],
            "hr_colour_map_bwd": [P, I, I, I, I, P, P],
            "hr_edges": [P, P, P, I, I, I, F, F, P, P],
            "hr_edge_loss": [P, P, P, P, P, I, I, I, F, F, F, P, P, P, P],
            "hr_get_tuning": [P, P],
            "hr_render_fwd": [P, P, P, P, I, I, I, P, P, P, P],
            "hr_loss": [P, P, P, P, I, I, I, P, P, P],
            "hr_render_bwd": [P, P, P, P, I, I, I, P, P, P, P, P],
            "hr_adam_step": [P, P, P, P, I, F, F, F, F, I, P],
            "hr_adam_step_dev": [P, P, P, P, I, F, F, F, F, P, I, P, P],
            "hr_vertex_error": [P, P, I, I, P, P, I, P],
            "hr_batch_create": [P, P, I, P],
            "hr_batch_layout": [P, P, P],
            "hr_skin_batch": [P, P, P, P, P],
            "hr_skin_bwd_batch": [P, P, P, P, P, P],
            "hr_build_bvh_batch": [P, P, P, P],
            "hr_render_fwd_batch": [P, P, P, P, P, P, P, P],
            "hr_loss_batch": [P, P, P, P, P, P, P],
            "hr_render_bwd_batch": [P, P, P, P, P, P, P, P, P],
            "hr_gemm_bf16": [P, P, I, P, I, I, I, I, P, I, P, I, I, I, P, P],
            "hr_net_param_count": [],
            "hr_net_create": [I, I, P],
            "hr_net_destroy": [P],
            "hr_net_set_params": [P, P, P],
            "hr_net_get_params": [P, P, P, P],
            "hr_net_inputs": [P, P, P, I, I, P],
            "hr_net_set_inputs_bf16": [P, P, P],
            "hr_net_forward": [P, P, P, P, P],
            "hr_net_backward": [P, P, P],
            "hr_net_adam": [P, F, F, F, F, I, P],
            "hr_net_status": [P, P],
            "hr_vertex_mse": [P, P, I, I, P, P, P],
            "hr_add_noise": [P, ctypes.c_int64, F, ctypes.c_uint64, P],
            "hr_select_best": [P, P, I, I, P, P, P],
            "hr_trace": [P, P, P, I, P, P, P],
            "hr_get_normals": [P, P, P],
            "hr_silhouettes": [P, P, P, P, I, P, P, P],
            "hr_get_stats": [P, P, P],
            "hr_kernel_times": [P, P, I],
            "hr_get_status": [P, P],
            "hr_status_string": [I],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "hr_status_string" else ctypes.c_int
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().hr_status_string(int(code)).decode()


def _check(name, code):
    if code != HR_OK:
        raise HandrtError(name, code)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("handrt takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("handrt takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32(t):
    assert t.dtype == torch.float32, t.dtype
    return _ptr(t)


# --------------------------------------------------------------------------------------
# Objects owning C-side state
# --------------------------------------------------------------------------------------

class Context:
    """An hr_context: device scratch, BVH and status word, sized by the limits."""

    def __init__(self, max_V, max_F, max_E, max_views, max_width, max_height):
        lim = hr_limits(max_V, max_F, max_E, max_views, max_width, max_height)
        h = ctypes.c_void_p()
        _check("hr_context_create", lib().hr_context_create(ctypes.byref(lim), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().hr_context_destroy(self.handle)
            self.handle = None

    def set_tuning(self, **kw):
        """Set launch shapes (hr_tuning fields); unspecified fields keep their value."""
        t = hr_tuning()
        _check("hr_get_tuning", lib().hr_get_tuning(self.handle, ctypes.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check("hr_set_tuning", lib().hr_set_tuning(self.handle, ctypes.byref(t)))

    def get_tuning(self):
        t = hr_tuning()
        _check("hr_get_tuning", lib().hr_get_tuning(self.handle, ctypes.byref(t)))
        return {n: int(getattr(t, n)) for n, _ in hr_tuning._fields_}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(Context):
    """A batch context (hr_batch_create) for instances described by
    (views, width, height, spp, edge_samples, instance) tuples; `view_offsets` and
    `pixel_offsets` (numpy, n + 1 entries) locate each instance in the concatenated
    camera and image arrays."""

    def __init__(self, max_V, max_F, max_E, descs):
        lim = hr_limits(max_V, max_F, max_E, 0, 0, 0)
        n = len(descs)
        arr = (hr_instance_desc * n)(*[hr_instance_desc(*map(int, d)) for d in descs])
        h = ctypes.c_void_p()
        _check("hr_batch_create", lib().hr_batch_create(ctypes.byref(lim), arr, n, ctypes.byref(h)))
        self.handle = h
        self.n = n
        self.descs = [tuple(int(x) for x in d) for d in descs]
        vo = (ctypes.c_int32 * (n + 1))()
        po = (ctypes.c_int64 * (n + 1))()
        _check("hr_batch_layout", lib().hr_batch_layout(h, vo, po))
        self.view_offsets = np.array(vo[:], np.int64)
        self.pixel_offsets = np.array(po[:], np.int64)

    @property
    def total_views(self):
        return int(self.view_offsets[-1])

    @property
    def total_pixels(self):
        return int(self.pixel_offsets[-1])


class Model:
    """Device copy of a hand model (inputs.HandModel) and its hr_model struct."""

    def __init__(self, hand, device="cuda"):
        def f(a):
            return torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)

        def i(a):
            return torch.as_tensor(np.ascontiguousarray(a, np.int32), device=device)

        self.hand = hand
        self.t = dict(v_template=f(hand.v_template), shapedirs=f(hand.shapedirs), weights=f(hand.weights),
                      j_template=f(hand.j_template), j_shapedirs=f(hand.j_shapedirs), parents=i(hand.parents),
                      faces=i(hand.faces), edges=i(hand.edges), edge_faces=i(hand.edge_faces),
                      vf_offsets=i(hand.vf_offsets), vf_faces=i(hand.vf_faces), albedo=f(hand.albedo))
        if getattr(hand, "uv", None) is not None:
            self.t["uv"] = f(hand.uv)
        m = hr_model()
        m.V, m.F, m.E = hand.V, hand.F, hand.E
        m.J, m.K = hand.weights.shape[1], hand.shapedirs.shape[2]
        for k, v in self.t.items():
            setattr(m, k, v.data_ptr())
        self.struct = m
        self.check()

    def check(self):
        """hr_model_check: the parent table in tree order and every index in range
        (synchronous; raises HandrtError)."""
        _check("hr_model_check", lib().hr_model_check(ctypes.byref(self.struct)))

    @property
    def V(self):
        return self.struct.V


def render_opts(seed=0, iter=0, instance=0, spp=4, edge_samples=1024, ka=0.4, kd=0.6, light_dir=(0.0, 0.0, 1.0),
                light_rgb=(1.0, 1.0, 1.0), edge_eps_px=1e-3, flags=0, iter_dev=None, texture=None, d_texture=None):
    """Render options; texture: device float [H_t][W_t][3] albedo texture (needs the
    model's uv); d_texture: device float buffer of the same shape that the backward adds
    dL/dtexture into."""
    o = hr_render_opts()
    o.seed = seed
    o.iter = iter
    o.instance = instance
    o.spp = spp
    o.edge_samples = edge_samples
    o.ka, o.kd = ka, kd
    o.light_dir[:] = list(light_dir)
    o.light_rgb[:] = list(light_rgb)
    o.edge_eps_px = edge_eps_px
    o.flags = flags
    o.iter_dev = None if iter_dev is None else iter_dev.data_ptr()
    if texture is not None:
        assert texture.is_cuda and texture.is_contiguous() and texture.dtype == torch.float32
        o.texture = texture.data_ptr()
        o.tex_h, o.tex_w = int(texture.shape[0]), int(texture.shape[1])
    if d_texture is not None:
        assert d_texture.is_cuda and d_texture.is_contiguous() and d_texture.dtype == torch.float32
        o.d_texture = d_texture.data_ptr()
    return o


# --------------------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# --------------------------------------------------------------------------------------

def hr_skin(ctx, model, params, verts, stream=None):
    _check("hr_skin", lib().hr_skin(ctx.handle, ctypes.byref(model.struct), _f32(params), _f32(verts),
                                    _stream(stream)))


def hr_skin_bwd(ctx, model, params, d_verts, d_params, stream=None):
    _check("hr_skin_bwd", lib().hr_skin_bwd(ctx.handle, ctypes.byref(model.struct), _f32(params), _f32(d_verts),
                                            _f32(d_params), _stream(stream)))


def hr_skin_bwd_noalloc(model, params, d_verts, d_params, stream=None):
    """hr_skin_bwd without a context; its scratch is a static device array in the
    library (for callers that cannot let a library allocate device memory)."""
    _check("hr_skin_bwd_noalloc", lib().hr_skin_bwd_noalloc(ctypes.byref(model.struct), _f32(params), _f32(d_verts),
                                                            _f32(d_params), _stream(stream)))


def hr_build_bvh(ctx, model, verts, stream=None):
    _check("hr_build_bvh", lib().hr_build_bvh(ctx.handle, ctypes.byref(model.struct), _f32(verts),
                                              _stream(stream)))


def hr_update_bvh(ctx, model, verts, iter_dev=None, rebuild_every=1, stream=None):
    """Rebuild when *iter_dev % rebuild_every == 0 (decided on the device), refit
    otherwise; single-instance or batch context."""
    assert iter_dev is None or (iter_dev.dtype == torch.int32 and iter_dev.numel() == 1)
    _check("hr_update_bvh", lib().hr_update_bvh(ctx.handle, ctypes.byref(model.struct), _f32(verts),
                                                None if iter_dev is None else _ptr(iter_dev), int(rebuild_every),
                                                _stream(stream)))


def hr_render_fwd(ctx, model, verts, cams, H, W, background, opts, image, stream=None):
    N = cams.shape[0]
    _check("hr_render_fwd", lib().hr_render_fwd(ctx.handle, ctypes.byref(model.struct), _f32(verts), _f32(cams), N,
                                                H, W, _f32(background), ctypes.byref(opts), _f32(image),
                                                _stream(stream)))


def hr_loss(ctx, image, observed, mask, loss, adjoint, stream=None):
    N, H, W = mask.shape
    assert mask.dtype == torch.uint8
    _check("hr_loss", lib().hr_loss(ctx.handle, _f32(image), _f32(observed), _ptr(mask), N, H, W, _f32(loss),
                                    _f32(adjoint), _stream(stream)))


def hr_skin_joints(ctx, model, params, verts, joints, stream=None):
    _check("hr_skin_joints", lib().hr_skin_joints(ctx.handle, ctypes.byref(model.struct), _f32(params), _f32(verts),
                                                  _f32(joints), _stream(stream)))


def hr_skin_bwd_joints(ctx, model, params, d_verts, d_joints, d_params, stream=None):
    _check("hr_skin_bwd_joints", lib().hr_skin_bwd_joints(ctx.handle, ctypes.byref(model.struct), _f32(params),
                                                          _f32(d_verts), None if d_joints is None else _f32(d_joints),
                                                          _f32(d_params), _stream(stream)))


def hr_joint_prior(joints, target, gamma, weight, loss, d_joints=None, stream=None):
    J = joints.shape[-2]
    n = joints.numel() // (3 * J)
    _check("hr_joint_prior", lib().hr_joint_prior(_f32(joints), _f32(target), J, n, float(gamma), float(weight),
                                                  _f32(loss), None if d_joints is None else _f32(d_joints),
                                                  _stream(stream)))


def hr_colour_map(v_low, v_high, out, stream=None):
    hl, wl = v_low.shape[0], v_low.shape[1]
    H, W = v_high.shape[0], v_high.shape[1]
    _check("hr_colour_map", lib().hr_colour_map(_f32(v_low), wl, hl, _f32(v_high), W, H, _f32(out), _stream(stream)))


def hr_colour_map_bwd(d_v, d_low, stream=None):
    hl, wl = d_low.shape[0], d_low.shape[1]
    H, W = d_v.shape[0], d_v.shape[1]
    _check("hr_colour_map_bwd", lib().hr_colour_map_bwd(_f32(d_v), W, H, wl, hl, _f32(d_low), _stream(stream)))


def hr_loss_ct(ctx, image, observed, mask, T, loss, adjoint, dT=None, stream=None):
    """Masked L1 loss of T_i R against O per camera; adjoint = dL/dR; dT = dL/dT [N][9]."""
    N, H, W = mask.shape
    assert mask.dtype == torch.uint8
    _check("hr_loss_ct", lib().hr_loss_ct(ctx.handle, _f32(image), _f32(observed), _ptr(mask),
                                          None if T is None else _f32(T), N, H, W, _f32(loss), _f32(adjoint),
                                          None if dT is None else _f32(dT), _stream(stream)))


# thresholds of the edge detector on the /8-normalised gradient magnitude (a step of
# contrast c peaks near 0.32 c)
EDGE_LOW, EDGE_HIGH = 0.05, 0.1


def hr_edges(ctx, image, edges, T=None, low=EDGE_LOW, high=EDGE_HIGH, stream=None):
    """Canny(T R) * K per view (the edge term's blurred edge map): image [N][H][W][3],
    edges [N][H][W], T [N][9] or None."""
    N, H, W = edges.shape
    _check("hr_edges", lib().hr_edges(ctx.handle, _f32(image), None if T is None else _f32(T), N, H, W, float(low),
                                      float(high), _f32(edges), _stream(stream)))


def hr_edge_loss(ctx, image, edges_obs, mask, loss, adjoint, T=None, dT=None, weight=1.0, low=EDGE_LOW,
                 high=EDGE_HIGH, stream=None):
    """L_e = weight sum M |E_r - E_o| / sum M into loss; ADDS dL_e/dR into adjoint and
    dL_e/dT into dT."""
    N, H, W = mask.shape
    assert mask.dtype == torch.uint8
    _check("hr_edge_loss", lib().hr_edge_loss(ctx.handle, _f32(image), None if T is None else _f32(T),
                                              _f32(edges_obs), _ptr(mask), N, H, W, float(low), float(high),
                                              float(weight), _f32(loss), _f32(adjoint),
                                              None if dT is None else _f32(dT), _stream(stream)))


def hr_render_bwd(ctx, model, verts, cams, H, W, background, opts, adjoint, d_verts, stream=None):
    N = cams.shape[0]
    _check("hr_render_bwd", lib().hr_render_bwd(ctx.handle, ctypes.byref(model.struct), _f32(verts), _f32(cams), N,
                                                H, W, _f32(background), ctypes.byref(opts), _f32(adjoint),
                                                _f32(d_verts), _stream(stream)))


def hr_adam_step(params, grad, m, v, lr, beta1, beta2, eps, step, stream=None):
    _check("hr_adam_step", lib().hr_adam_step(_f32(params), _f32(grad), _f32(m), _f32(v), params.numel(), lr, beta1,
                                              beta2, eps, step, _stream(stream)))


def hr_adam_step_dev(params, grad, m, v, lr, beta1, beta2, eps, iter_dev, lr_scale=None, stream=None):
    """lr_scale: optional device float tensor; entry i steps by lr * lr_scale[i % len]."""
    assert iter_dev.dtype == torch.int32 and iter_dev.numel() == 1   # holds a uint32 counter
    n_scale = 0 if lr_scale is None else lr_scale.numel()
    _check("hr_adam_step_dev", lib().hr_adam_step_dev(_f32(params), _f32(grad), _f32(m), _f32(v), params.numel(), lr,
                                                      beta1, beta2, eps, None if lr_scale is None else _f32(lr_scale),
                                                      n_scale, _ptr(iter_dev), _stream(stream)))


def hr_vertex_error(verts, ref, out, iter_dev=None, stream=None):
    """epsilon_v per instance (metres): verts, ref [n][V][3] (or [V][3]); out [rows][n],
    row = *iter_dev (0 without a counter)."""
    V = verts.shape[-2]
    n = verts.numel() // (3 * V)
    rows = out.numel() // n
    _check("hr_vertex_error", lib().hr_vertex_error(_f32(verts), _f32(ref), V, n, _f32(out),
                                                    None if iter_dev is None else _ptr(iter_dev), rows,
                                                    _stream(stream)))


def hr_gemm_bf16(ctx, A, Bm, C, bias=None, relu=False, splits=1, split_buf=None, stream=None):
    """C = act(A Bm^T + bias) on the tensor cores: A [M][K], Bm [N][K] bf16 (row
    pitch = stride(0)), C [M][N] bf16 or float32."""
    assert A.dtype == torch.bfloat16 and Bm.dtype == torch.bfloat16 and A.stride(1) == 1 and Bm.stride(1) == 1
    assert C.dtype in (torch.bfloat16, torch.float32) and C.stride(1) == 1
    M, K = A.shape
    N = Bm.shape[0]
    assert Bm.shape[1] == K and C.shape[0] == M and C.shape[1] >= N
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    _check("hr_gemm_bf16", lib().hr_gemm_bf16(ctx.handle, ptr(A), A.stride(0), ptr(Bm), Bm.stride(0), M, N, K,
                                              None if bias is None else _f32(bias), int(bool(relu)), ptr(C),
                                              C.stride(0), int(C.dtype == torch.bfloat16), int(splits),
                                              None if split_buf is None else _f32(split_buf), _stream(stream)))


class Net:
    """The proposal network (hr_net_*) for B instances of `views` views."""

    def __init__(self, B, views):
        h = ctypes.c_void_p()
        _check("hr_net_create", lib().hr_net_create(int(B), int(views), ctypes.byref(h)))
        self.handle = h
        self.B, self.views = int(B), int(views)
        self.P = int(lib().hr_net_param_count())

    def close(self):
        if self.handle:
            lib().hr_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, stream=None):
        assert params.numel() == self.P
        _check("hr_net_set_params", lib().hr_net_set_params(self.handle, _f32(params), _stream(stream)))

    def get_params(self, params=None, grads=None, stream=None):
        _check("hr_net_get_params", lib().hr_net_get_params(self.handle, None if params is None else _f32(params),
                                                            None if grads is None else _f32(grads), _stream(stream)))

    def inputs(self, render, observed, W=256, H=256, stream=None):
        _check("hr_net_inputs", lib().hr_net_inputs(self.handle, _f32(render), _f32(observed), W, H,
                                                    _stream(stream)))

    def set_inputs_bf16(self, x0, stream=None):
        assert x0.dtype == torch.bfloat16
        _check("hr_net_set_inputs_bf16", lib().hr_net_set_inputs_bf16(self.handle, _ptr(x0), _stream(stream)))

    def forward(self, cams, out, base=None, stream=None):
        _check("hr_net_forward", lib().hr_net_forward(self.handle, _f32(cams), None if base is None else _f32(base),
                                                      _f32(out), _stream(stream)))

    def backward(self, d_out, stream=None):
        _check("hr_net_backward", lib().hr_net_backward(self.handle, _f32(d_out), _stream(stream)))

    def adam(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check("hr_net_adam", lib().hr_net_adam(self.handle, lr, beta1, beta2, eps, int(step), _stream(stream)))

    def status(self, stream=None):
        return int(lib().hr_net_status(self.handle, _stream(stream)))


def hr_batch_set_active(ctx, active):
    """active: device int32 tensor [n] (kept alive by the caller) or None."""
    assert active is None or (active.dtype == torch.int32 and active.is_cuda)
    _check("hr_batch_set_active", lib().hr_batch_set_active(ctx.handle, None if active is None else _ptr(active)))


def hr_retire_converged(err, iter_dev, threshold, active, lr_scale=None, stream=None):
    """err: device float [rows][n] (hr_vertex_error's table); lr_scale: device float
    [n][per] per-entry Adam steps, zeroed for retired instances."""
    rows, n = err.shape
    per = 0 if lr_scale is None else lr_scale.numel() // n
    _check("hr_retire_converged", lib().hr_retire_converged(
        _f32(err), None if iter_dev is None else _ptr(iter_dev), rows, n, float(threshold), _ptr(active),
        None if lr_scale is None else _f32(lr_scale), per, _stream(stream)))


def hr_retire_plateau(loss, rel_tol, patience, best, stall, active, lr_scale=None, stream=None):
    n = loss.numel()
    per = 0 if lr_scale is None else lr_scale.numel() // n
    _check("hr_retire_plateau", lib().hr_retire_plateau(
        _f32(loss), n, float(rel_tol), int(patience), _f32(best), _ptr(stall), _ptr(active),
        None if lr_scale is None else _f32(lr_scale), per, _stream(stream)))


def hr_box_downsample(src, f, dst, stream=None):
    """src: device float [N][H][W][3]; dst: [N][H/f][W/f][3] box means."""
    N, H, W, _ = src.shape
    _check("hr_box_downsample", lib().hr_box_downsample(_f32(src), N, H, W, int(f), _f32(dst), _stream(stream)))


def hr_mask_downsample(src, f, dst, stream=None):
    """src: device uint8 [N][H][W]; dst: [N][H/f][W/f] block maxima."""
    assert src.dtype == torch.uint8 and dst.dtype == torch.uint8
    N, H, W = src.shape
    _check("hr_mask_downsample", lib().hr_mask_downsample(_ptr(src), N, H, W, int(f), _ptr(dst), _stream(stream)))


def hr_area_resample(src, dst, stream=None):
    """src: device float [N][H][W][3]; dst: [N][Ho][Wo][3] area means over each output
    pixel's footprint."""
    N, H, W, _ = src.shape
    No, Ho, Wo, _ = dst.shape
    assert No == N and src.is_contiguous() and dst.is_contiguous()
    _check("hr_area_resample", lib().hr_area_resample(_f32(src), N, H, W, _f32(dst), Ho, Wo, _stream(stream)))


def hr_mask_resample(src, dst, stream=None):
    """src: device uint8 [N][H][W]; dst: [N][Ho][Wo] maxima over each footprint."""
    assert src.dtype == torch.uint8 and dst.dtype == torch.uint8
    N, H, W = src.shape
    No, Ho, Wo = dst.shape
    assert No == N and src.is_contiguous() and dst.is_contiguous()
    _check("hr_mask_resample", lib().hr_mask_resample(_ptr(src), N, H, W, _ptr(dst), Ho, Wo, _stream(stream)))


def hr_vertex_mse(verts, ref, loss, d_verts=None, stream=None):
    V = verts.shape[-2]
    n = verts.numel() // (3 * V)
    _check("hr_vertex_mse", lib().hr_vertex_mse(_f32(verts), _f32(ref), V, n, _f32(loss),
                                                None if d_verts is None else _f32(d_verts), _stream(stream)))


def hr_add_noise(image, sigma, seed, stream=None):
    _check("hr_add_noise", lib().hr_add_noise(_f32(image), image.numel(), float(sigma), int(seed), _stream(stream)))


def hr_select_best(candidates, losses, params, chosen=None, stream=None):
    K, n = losses.shape
    assert chosen is None or chosen.dtype == torch.int32
    _check("hr_select_best", lib().hr_select_best(_f32(candidates), _f32(losses), K, n, _f32(params),
                                                  None if chosen is None else _ptr(chosen), _stream(stream)))


# batches (hr_batch_create): concatenated per-instance arrays, see include/handrt.h

def hr_skin_batch(ctx, model, params, verts, stream=None):
    _check("hr_skin_batch", lib().hr_skin_batch(ctx.handle, ctypes.byref(model.struct), _f32(params), _f32(verts),
                                                _stream(stream)))


def hr_skin_bwd_batch(ctx, model, params, d_verts, d_params, stream=None):
    _check("hr_skin_bwd_batch", lib().hr_skin_bwd_batch(ctx.handle, ctypes.byref(model.struct), _f32(params),
                                                        _f32(d_verts), _f32(d_params), _stream(stream)))


def hr_build_bvh_batch(ctx, model, verts, stream=None):
    _check("hr_build_bvh_batch", lib().hr_build_bvh_batch(ctx.handle, ctypes.byref(model.struct), _f32(verts),
                                                          _stream(stream)))


def hr_render_fwd_batch(ctx, model, verts, cams, background, opts, image, stream=None):
    _check("hr_render_fwd_batch", lib().hr_render_fwd_batch(ctx.handle, ctypes.byref(model.struct), _f32(verts),
                                                            _f32(cams), _f32(background), ctypes.byref(opts),
                                                            _f32(image), _stream(stream)))


def hr_loss_batch(ctx, image, observed, mask, loss, adjoint, stream=None):
    assert mask.dtype == torch.uint8
    _check("hr_loss_batch", lib().hr_loss_batch(ctx.handle, _f32(image), _f32(observed), _ptr(mask), _f32(loss),
                                                _f32(adjoint), _stream(stream)))


def hr_render_bwd_batch(ctx, model, verts, cams, background, opts, adjoint, d_verts, stream=None):
    _check("hr_render_bwd_batch", lib().hr_render_bwd_batch(ctx.handle, ctypes.byref(model.struct), _f32(verts),
                                                            _f32(cams), _f32(background), ctypes.byref(opts),
                                                            _f32(adjoint), _f32(d_verts), _stream(stream)))


def hr_trace(ctx, origins, dirs, tri, tuv, stream=None):
    assert tri.dtype == torch.int32
    _check("hr_trace", lib().hr_trace(ctx.handle, _f32(origins), _f32(dirs), origins.shape[0], _ptr(tri), _f32(tuv),
                                      _stream(stream)))


def hr_get_normals(ctx, normals, stream=None):
    _check("hr_get_normals", lib().hr_get_normals(ctx.handle, _f32(normals), _stream(stream)))


def hr_silhouettes(ctx, model, verts, cams, lists, counts, stream=None):
    _check("hr_silhouettes", lib().hr_silhouettes(ctx.handle, ctypes.byref(model.struct), _f32(verts), _f32(cams),
                                                  cams.shape[0], _ptr(lists), _ptr(counts), _stream(stream)))


def hr_get_stats(ctx, stream=None):
    """Work counters [3][6] (forward, interior backward, edge rays) x (estimator
    samples resolved, rays made individually, BVH nodes visited, Moller-Trumbore
    tests, hits, candidate screen-box tests) accumulated by calls made with
    HR_STATS; cleared on read."""
    out = (ctypes.c_uint64 * 18)()
    _check("hr_get_stats", lib().hr_get_stats(ctx.handle, out, _stream(stream)))
    return np.array(out[:], np.uint64).reshape(3, 6)


def hr_kernel_times(ctx):
    """Internal kernel times (ms) of the last HR_TIMING render calls, by KERNEL_TIMES."""
    out = (ctypes.c_float * len(KERNEL_TIMES))()
    _check("hr_kernel_times", lib().hr_kernel_times(ctx.handle, out, len(KERNEL_TIMES)))
    return dict(zip(KERNEL_TIMES, out[:]))


def hr_get_status(ctx, stream=None):
    return int(lib().hr_get_status(ctx.handle, _stream(stream)))
