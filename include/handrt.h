/*
 * handrt -- GB300 (sm_103a) library for multiview hand-geometry refinement by
 * differentiable Monte Carlo ray tracing (Karvounas et al., "Multiview Image-based
 * Hand Geometry Refinement using Differentiable Monte Carlo Ray Tracing", BMVC 2021).
 *
 * One refinement iteration (Section 3, Eq. 1-3) is
 *
 *     verts  = G_v(h + dh)                       hr_skin          (Section 3.1, "Geometry")
 *     accel  = BVH + vertex normals of verts     hr_build_bvh
 *     R_i    = R(verts, colour, C_i)             hr_render_fwd    (Section 3.1, "Rendering")
 *     E_1    = sum_i D_c(O_i, R_i), dE_1/dR_i    hr_loss          (Eq. 3 and Eq. 4, D_c term)
 *     dE/dverts                                  hr_render_bwd    (interior + edge sampling)
 *     dE/d(h + dh)                               hr_skin_bwd
 *     h + dh <- Adam step                        hr_adam_step     (Section 3.3)
 *
 * Conventions shared by every call:
 *   - Array pointers are caller-owned DEVICE memory unless stated otherwise; the
 *     library never frees them and keeps no reference after the call returns
 *     (the context keeps its own copies of what later calls need).
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) and never synchronises, except hr_get_status.
 *   - Return value: HR_OK (0) or a negative HR_ERR_* code for errors detected on
 *     the host (bad arguments, a failed launch).  Errors found by a kernel (a
 *     traversal stack overflow, non-finite parameters) are OR-ed into the
 *     context's device status word; hr_get_status reads and clears it.  No call
 *     traps on the device.
 *   - Calls that share one context must be ordered on one stream; use one context
 *     per concurrent stream.
 *   - Layouts are C-contiguous, float32 unless stated.  Images are [N][H][W][3]
 *     (views, rows, columns, RGB); pixel (x, y) covers [x, x+1) x [y, y+1).
 *   - Parameters h are float[61] = [beta(10) shape, theta(45) pose as 15 axis-angle
 *     triples, phi(3) root axis-angle, tau(3) root translation in metres]
 *     (Section 3: the 61 parameters {beta, theta, tau, phi} of the hand model).
 */
#ifndef HANDRT_H
#define HANDRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HR_OK 0
#define HR_ERR_ARG (-1)         /* invalid argument (null pointer, size out of range) */
#define HR_ERR_CUDA (-2)        /* a CUDA runtime call or launch failed */
#define HR_ERR_LIMIT (-3)       /* a device-side limit was hit (traversal stack) */
#define HR_ERR_NONFINITE (-4)   /* non-finite parameters reached the skinning kernel */
#define HR_ERR_UNSUPPORTED (-5) /* sizes beyond what the context was created for */
#define HR_ERR_INTERNAL (-6)    /* a kernel read an internal index out of range and skipped it */
#define HR_ERR_TIMEOUT (-7)     /* a bounded device-side wait ran out; that kernel's work was abandoned */

typedef void* hr_stream; /* a cudaStream_t */

/* Pinhole camera, OpenCV convention (x right, y down, z forward), world -> camera:
 * X_cam = R X_world + t.  `centre` is the camera position in world coordinates
 * (-R^T t, given explicitly so that all primary rays start from the same float32
 * point).  80 bytes.  (Section 3: calibrated views with intrinsics and extrinsics.) */
typedef struct hr_camera {
    float fx, fy, cx, cy;
    float R[9];      /* row-major */
    float t[3];
    float centre[3];
    float pad;
} hr_camera;

/* Hand model (device arrays, caller-owned).  A linear-blend-skinned mesh standing in
 * for the MANO model of Section 3: K shape blendshapes, J joints, parents[j] < j. */
typedef struct hr_model {
    int32_t V, F, E, J, K;
    const float* v_template;   /* [V][3] rest vertices                             */
    const float* shapedirs;    /* [V][3][K] shape blendshapes                       */
    const float* weights;      /* [V][J] skin weights                               */
    const float* j_template;   /* [J][3] rest joints                                */
    const float* j_shapedirs;  /* [J][3][K] joint regressor per shape component     */
    const int32_t* parents;    /* [J] parent joint, -1 for the root (joint 0)       */
    const int32_t* faces;      /* [F][3] triangles, outward counter-clockwise       */
    const int32_t* edges;      /* [E][2] unique edges (a < b)                       */
    const int32_t* edge_faces; /* [E][2] adjacent faces, second = -1 on a boundary  */
    const int32_t* vf_offsets; /* [V+1] vertex -> incident faces, CSR offsets       */
    const int32_t* vf_faces;   /* [3F]  incident faces, ascending per vertex        */
    const float* albedo;       /* [V][3] per-vertex RGB albedo                      */
    const float* uv;           /* [V][2] texture coordinates in [0, 1]^2, or NULL;
                                  used when the render options give a texture        */
} hr_model;

/* Check a model's index tables once, after filling the struct (synchronous: copies
 * the tables from the device; not for the refinement loop).  Returns HR_ERR_ARG for
 * a parent table that is not in tree order (parents[0] = -1 and 0 <= parents[j] < j
 * for j > 0: the skinning kernels compose and differentiate the kinematic chain of
 * Section 3 level by level from the root), face, edge or incident-face indices out
 * of range, or vertex->face offsets that are not a CSR table; HR_ERR_UNSUPPORTED for
 * more than 16 joints or 10 shape components; HR_ERR_CUDA if a copy fails.  The
 * other calls only check sizes and pointers on the host; their kernels report index
 * errors they meet through the status word. */
int hr_model_check(const hr_model* model);

/* Allocation-free variant of hr_skin_bwd (the paper has no counterpart: it is an
 * interface for callers that cannot let a library allocate device memory, such as
 * host applications that hand out all device memory from their own pool, processes
 * under a fixed device-memory quota, and latency-bound loops that cannot afford
 * cudaMalloc's implicit device synchronisation).  Same arguments and result as
 * hr_skin_bwd, without a context: the reduction scratch is a static device array
 * of about 52 KB inside this library, which every GPU that loads the library keeps
 * until the process exits.  No device memory is allocated or freed by the call.
 *   - The array's device address is looked up, on the current device, by every
 *     call whose stream is not being captured (so a device reset does not leave a
 *     stale address); other calls use the device's last looked-up address.  Make
 *     the first call on a device, and the first call after a device reset, before
 *     any stream capture.
 *   - model->V <= 16384, model->J <= 16, model->K <= 10, else HR_ERR_UNSUPPORTED.
 *   - All calls share the one array: calls that may overlap on the GPU (different
 *     streams, or different host threads on one device) race and must be ordered
 *     by the caller.  The call clears what must start at zero itself.
 *   - Device-detected errors (non-finite parameters, parent indices out of range)
 *     are not reported by this variant; its outputs are then undefined. */
int hr_skin_bwd_noalloc(const hr_model* model, const float* params, const float* d_verts, float* d_params,
                        hr_stream stream);

/* Render options.  Samples are drawn from Philox4x32-10 keyed by `seed` with counters
 * built from (pixel, view | instance << 16, sample, iter << 4 | stream), so a render
 * is a deterministic function of (seed, iter, instance).  Shading is Lambertian with
 * one directional light: f = albedo * light_rgb * (ka + kd * max(0, n . light_dir)),
 * n the interpolated, normalised vertex normal; light_dir points toward the light. */
typedef struct hr_render_opts {
    uint64_t seed;
    uint32_t iter;
    uint32_t instance;
    int32_t spp;            /* primary samples per pixel, 1 .. 65536                */
    int32_t edge_samples;   /* silhouette-edge samples per view (>= 0)              */
    float ka, kd;
    float light_dir[3];
    float light_rgb[3];
    float edge_eps_px;      /* offset of the two edge-sample rays, in pixels, in
                               (0, 0.25]: the offset rays use the candidate list of the
                               sub-tile holding the sample, which is complete for
                               screen points within half a pixel of the sub-tile   */
    uint32_t flags;         /* HR_BWD_* bits; 0 = every term                        */
    const uint32_t* iter_dev; /* optional device counter read instead of `iter` (so a
                                 captured iteration replays with fresh samples); NULL = use iter */
    /* Albedo texture (optional; needs model->uv).  When given, the albedo of a hit is
     * the bilinear lookup of `texture` (device float[tex_h][tex_w][3], texel (i, j)
     * centred at ((i + 0.5) / tex_w, (j + 0.5) / tex_h), clamp-to-edge) at the
     * interpolated uv, instead of the interpolated per-vertex albedo.  The texel
     * coordinates x = uv_x tex_w - 0.5, y = uv_y tex_h - 0.5 and their floors are
     * float32 decisions.  hr_render_bwd adds dL/dtexture into d_texture (device
     * float[tex_h][tex_w][3], accumulated: the caller clears it) when it is not NULL. */
    const float* texture;
    int32_t tex_w, tex_h;
    float* d_texture;
} hr_render_opts;

#define HR_BWD_NO_INTERIOR 1u  /* hr_render_bwd: skip the interior term            */
#define HR_BWD_NO_EDGES 2u     /* hr_render_bwd: skip the edge-sampling term       */
#define HR_BWD_NO_NORMALS 4u   /* hr_render_bwd: skip the vertex-normal adjoint    */
#define HR_STATS 8u            /* count rays, BVH nodes, triangle tests and hits   */
#define HR_TIMING 16u          /* record CUDA events around the internal kernels   */
#define HR_BWD_REUSE_FWD 32u   /* hr_render_bwd: take the candidate lists of the last
                                  hr_render_fwd on this context instead of gathering
                                  its own from the BVH -- honoured only when that forward used
                                  the same vertex and camera pointers, sizes and spp and
                                  no hr_build_bvh came after it; the caller guarantees
                                  that the contents of both arrays are unchanged      */
#define HR_DETERMINISTIC 64u   /* hr_render_bwd: d_verts bit-identical on every call
                                  with the same inputs -- each vertex-gradient
                                  contribution is rounded to a multiple of 2^-40 and
                                  summed as a 64-bit integer (exact, so the order of
                                  the atomics does not matter); the interior shader
                                  traces one sample per lane (whichever kernel traces
                                  a sample does the same arithmetic) and the edge term
                                  runs on the caller's stream.  d_texture sums stay
                                  in float atomics (order-dependent rounding)         */

/* Sizes a context is created for; all scratch is allocated once, up front. */
typedef struct hr_limits {
    int32_t max_V;      /* vertices (<= 65536; up to 8192 the backward sums in shared
                           memory, beyond that with global atomics)             */
    int32_t max_F;      /* triangles (<= 65536; the BVH build runs in one block per
                           instance up to ~2400, in a multi-block build beyond)  */
    int32_t max_E;      /* edges                                                 */
    int32_t max_views;  /* views per call                                        */
    int32_t max_width;  /* image width W per call                                */
    int32_t max_height; /* image height H per call                               */
} hr_limits;

typedef struct hr_context hr_context;

/* Launch shapes of the render kernels (hr_set_tuning; see pipeline.autotune for the
 * project's autotuner, which times candidates on a workload and caches the best):
 *   rays_per_lane      samples each lane of the forward shader traces together
 *                      against a candidate (1, 2, 4)
 *   cand_per_chunk     candidates per work item when splitting a sub-tile (>= 1)
 *   max_chunks         work items per sub-tile at most (1 .. 16)
 *   blocks_per_sm      persistent blocks per SM of the forward shader, the list sort
 *                      and the backward's own list gather (1 .. 8)
 *   bwd_blocks_per_sm  persistent blocks per SM of the backward shader (1 .. 8)
 *   bwd_rays_per_lane  rays_per_lane of the backward shader (1, 2, 4)
 *   bwd_cand_per_chunk cand_per_chunk of the backward's work items (>= 1)
 *   edge_lanes         lanes per silhouette-edge sample in the edge-sampling kernel
 *                      (2, 4, 8, 16, 32: a warp takes 32 / edge_lanes samples)
 * Every setting gives the same results (the backward up to float32 summation order);
 * only the speed changes.  Defaults: 2, 8, 16, 8, 4, 4, 16, 4. */
typedef struct hr_tuning {
    int32_t rays_per_lane;
    int32_t cand_per_chunk;
    int32_t max_chunks;
    int32_t blocks_per_sm;
    int32_t bwd_blocks_per_sm;
    int32_t bwd_rays_per_lane;
    int32_t bwd_cand_per_chunk;
    int32_t edge_lanes;
} hr_tuning;

/* Create a context on the current CUDA device: device scratch for the given
 * limits (the BVH, vertex normals, the render kernels' per-sub-tile candidate pool
 * and work items, reduction partials) and the device status word.
 * Returns HR_ERR_ARG for non-positive or too large limits, HR_ERR_CUDA when an
 * allocation fails (nothing is leaked).  The context is owned by the caller. */
int hr_context_create(const hr_limits* limits, hr_context** out);

/* Free a context and all its device memory (synchronises the device first). */
int hr_context_destroy(hr_context* ctx);

/* Set / read the context's launch shapes (HR_ERR_ARG for values out of range). */
int hr_set_tuning(hr_context* ctx, const hr_tuning* tuning);
int hr_get_tuning(hr_context* ctx, hr_tuning* tuning);

/* Skinning G_v (Section 3.1, "Geometry": x in R^61 decoded into 3-D vertices).
 *   v = sum_j w_vj (A_j [v_template + S beta; 1]) + tau,  A_j = G_j [I | -J_j],
 *   G_0 = [R(phi) | J_0],  G_j = G_parent(j) [R(theta_j) | J_j - J_parent(j)],
 *   J = j_template + SJ beta, R(.) = Rodrigues.
 * params: device float[61]; verts: device float[V][3] (written).
 * Non-finite params set HR_ERR_NONFINITE in the status word (outputs then undefined). */
int hr_skin(hr_context* ctx, const hr_model* model, const float* params, float* verts, hr_stream stream);

/* Adjoint of hr_skin: d_params (device float[61], overwritten) = (dverts/dparams)^T d_verts
 * for d_verts device float[V][3]. */
int hr_skin_bwd(hr_context* ctx, const hr_model* model, const float* params, const float* d_verts,
                float* d_params, hr_stream stream);

/* Rebuild the context's scene from the current vertices: a Morton-code linear BVH
 * over the model's faces (rebuilt, not refitted, every call) and the area-weighted
 * unit vertex normals used for shading.  verts: device float[V][3]. */
int hr_build_bvh(hr_context* ctx, const hr_model* model, const float* verts, hr_stream stream);

/* Rebuild or refit: with iter_dev (device uint32) and rebuild_every > 1, the tree is
 * rebuilt when *iter_dev is a multiple of rebuild_every (or when this context has no
 * tree of the model's faces yet) and otherwise refitted -- the topology and leaf
 * order of the last build kept, triangle records recomputed from verts -- the choice
 * taken on the device, so a captured iteration replays it.  On meshes the one-block
 * build holds (the paper-sized hand), a refit iteration rewrites only the records;
 * the boxes are refitted from them by the first later call that traverses the tree:
 * a forward render with a sub-tile left to per-ray traversal, a backward without
 * HR_BWD_REUSE_FWD, or hr_trace (the forward's candidate lists come from the
 * records' screen boxes, not from the tree).  Any tree whose boxes contain their
 * children gives the same hits and candidate sets, so refitting changes speed only.
 * iter_dev NULL or rebuild_every = 1: hr_build_bvh.  Works on single-instance and
 * batch contexts (verts [n][V][3] for a batch); the vertex normals are recomputed
 * every call. */
int hr_update_bvh(hr_context* ctx, const hr_model* model, const float* verts, const uint32_t* iter_dev,
                  int rebuild_every, hr_stream stream);

/* Forward render R (Section 3.1, "Rendering"): every pixel value is the Monte Carlo
 * estimate (1/spp) sum_s f(x_s) of its box-filtered integral, x_s uniform in the
 * pixel, f the radiance of the closest hit of the primary ray through x_s (double-
 * sided Moller-Trumbore; ties in distance go to the lower triangle id), or the
 * background pixel on a miss.  Requires hr_build_bvh for the same verts.
 * cams: device hr_camera[N]; background and image: device float[N][H][W][3]. */
int hr_render_fwd(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N,
                  int H, int W, const float* background, const hr_render_opts* opts, float* image,
                  hr_stream stream);

/* Masked photometric loss (Eq. 3 with the D_c term of Eq. 4, summed over views):
 *   L = sum_p M_p sum_c |R_pc - O_pc| / (3 sum_p M_p),
 *   adjoint_pc = dL/dR_pc = M_p sign(R_pc - O_pc) / (3 sum_p M_p), sign(0) = 0.
 * An all-zero mask gives L = 0 and a zero adjoint.  image, observed, adjoint: device
 * float[N][H][W][3]; mask: device uint8[N][H][W] (non-zero = 1); loss: device float[1].
 * The reduction order is fixed, so repeated calls return identical values. */
int hr_loss(hr_context* ctx, const float* image, const float* observed, const uint8_t* mask, int N, int H,
            int W, float* loss, float* adjoint, hr_stream stream);

/* The data term with the per-camera colour transform (Eq. 2: camera i's rendering
 * enters the comparison as T_i R, T_i a 3x3 matrix applied to every pixel's RGB):
 *   L = sum_p M_p sum_c |(T_i R_p)_c - O_pc| / (3 sum_p M_p),
 *   adjoint_p = dL/dR_p = T_i^T (M_p sign(T_i R_p - O_p) / (3 sum M)),
 *   dT[i] = dL/dT_i = sum over camera i's pixels of (M sign(...) / (3 sum M)) R_p^T.
 * T: device float[N][9] row-major (NULL = identity, the plain hr_loss); dT: device
 * float[N][9] (overwritten) or NULL.  Sums in a fixed order; N <= 113.  Single-
 * instance contexts. */
int hr_loss_ct(hr_context* ctx, const float* image, const float* observed, const uint8_t* mask, const float* T,
               int N, int H, int W, float* loss, float* adjoint, float* dT, hr_stream stream);

/* The edge term D_e of the data term (Eq. 4): |Canny(o) * K - Canny(r) * K| with K the
 * 11 x 11 Gaussian of sigma 5 (zero padding), r = T_i R the colour-transformed render
 * of camera i (Eq. 2).  Canny's detector, per view: luma g = a . R with a = T_i^T w,
 * w = (0.299, 0.587, 0.114); 5-tap Gaussian of sigma 1 along x then y; Sobel / 8
 * ((1/4, 1/2, 1/4) smoothing, (-1/2, 0, 1/2) differences); m = sqrt(gx^2 + gy^2 +
 * 1e-12); non-maximum suppression along the gradient direction quantised to 0, 45, 90
 * or 135 degrees (a pixel survives when m >= m at both neighbours, coordinates clamped);
 * candidates m > low, strong m > high; hysteresis keeps the candidates 8-connected
 * through candidates to a strong pixel.  The detector's passes replicate the image
 * border.  Canny(x) is m on the kept pixels and 0 elsewhere: the selection is
 * piecewise constant, so the derivative flows through m with the selection fixed.
 * Everything up to the blurred map is float32 with one rounding per multiply and per
 * add, taps summed from the most negative offset up (the selection and the loss's
 * signs are reproducible decisions).
 *
 * hr_edges writes Canny(T R) * K (device float[N][H][W]; T device float[N][9]
 * row-major or NULL for none): the observation's map, computed once.
 * hr_edge_loss evaluates, for edges_obs = hr_edges of the observation,
 *   L_e = weight sum_p M_p |E_r - E_o| / sum_p M_p  (into loss, device float[1];
 *         0 without masked pixels),
 * ADDS dL_e/dR into adjoint (device float[N][H][W][3]) and, when dT is not NULL,
 * dL_e/dT into dT (device float[N][9]).  Call it after hr_loss_ct, which overwrites
 * both, to form the whole data term.  The per-pixel scratch (23 bytes per pixel of
 * the context's maximum image stack) is allocated by the first edge call on a
 * context, so make that call outside stream capture.  Single-instance contexts;
 * N H W <= INT_MAX; 0 <= low <= high, finite.  A union-find that ran past its bound
 * reports HR_ERR_LIMIT through hr_get_status. */
int hr_edges(hr_context* ctx, const float* image, const float* T, int N, int H, int W, float low, float high,
             float* edges, hr_stream stream);
int hr_edge_loss(hr_context* ctx, const float* image, const float* T, const float* edges_obs, const uint8_t* mask,
                 int N, int H, int W, float low, float high, float weight, float* loss, float* adjoint, float* dT,
                 hr_stream stream);

/* Backward of hr_render_fwd for adjoint image A = dL/dR (Section 1 and Section 3.1:
 * the ray tracer of Li et al. 2018 handles visibility discontinuities in the
 * backward pass).  d_verts (device float[V][3], overwritten) is the sum of
 *   interior : the forward's samples re-traced (same Philox counters); at each hit
 *              g^T df/dverts at the fixed ray (barycentrics, albedo, normals);
 *   edges    : edge_samples per view on the view's silhouette edges, uniform over the
 *              edge list and along the edge, each tracing f+ and f- at +-edge_eps_px
 *              along the edge's screen normal: A[p] . (f+ - f-) dalpha/d(endpoints)
 *              times N_sil / edge_samples, mapped to vertices by the projection;
 *   normals  : the vertex-normal adjoint of the interior term's normal gradient.
 * Requires hr_build_bvh for the same verts; background as in the forward. */
int hr_render_bwd(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N,
                  int H, int W, const float* background, const hr_render_opts* opts, const float* adjoint,
                  float* d_verts, hr_stream stream);

/* One Adam step (Section 3.3: the parameters are optimised with Adam) on n floats:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps),  step >= 1. */
int hr_adam_step(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1,
                 float beta2, float eps, int step, hr_stream stream);

/* Adam step with the step number kept on the device: step = *iter_dev + 1, and the
 * call then advances *iter_dev by one (device uint32).  With the same counter given
 * to the render calls as hr_render_opts.iter_dev, a whole refinement iteration can
 * be replayed (for example from a CUDA graph) with fresh sample streams and correct
 * bias correction every time.  lr_scale (device float[scale_len], or NULL) gives
 * entry i the step size lr * lr_scale[i % scale_len]: parameters of different units
 * (radians, shape coefficients, metres) get their own step, and scale_len = 61
 * repeats one scale over the instances of a batch. */
int hr_adam_step_dev(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1,
                     float beta2, float eps, const float* lr_scale, int scale_len, uint32_t* iter_dev,
                     hr_stream stream);

/* G_J, the model's 3-D joint locations (Section 3, the prior term E_2): hr_skin plus
 * the posed joints (each joint frame's origin plus the root translation), joints:
 * device float[J][3] ([n][J][3] on a batch context).  hr_skin_bwd_joints is
 * hr_skin_bwd with an optional upstream gradient of those joints (d_joints, same
 * layout, or NULL) added to the kinematic chain's adjoint.  Single-instance or batch
 * contexts. */
int hr_skin_joints(hr_context* ctx, const hr_model* model, const float* params, float* verts, float* joints,
                   hr_stream stream);
int hr_skin_bwd_joints(hr_context* ctx, const hr_model* model, const float* params, const float* d_verts,
                       const float* d_joints, float* d_params, hr_stream stream);

/* The prior term E_2 per instance (Section 3): weight * sum over joints and coordinates
 * of f_2(x, y) = 0.5 (x - y)^2 / gamma for |x - y| < gamma, |x - y| - 0.5 gamma
 * otherwise, x the target joints, y the model's (device float[n][J][3] each); loss:
 * device float[n]; d_joints (device float[n][J][3] or NULL) = dE_2/dy.  The paper
 * uses gamma = 5 mm and weight 1e-3.  J <= 1024. */
int hr_joint_prior(const float* joints, const float* target, int J, int n, float gamma, float weight, float* loss,
                   float* d_joints, hr_stream stream);

/* The two-level colour map (Section 3, "Color mapping"): out = V_low scaled up by
 * nearest neighbour to W x H + V_high, all device float [rows][cols][3]
 * (V_low [hl][wl][3], V_high and out [H][W][3]; W, H multiples of wl, hl).
 * hr_colour_map_bwd: dL/dV_low (device float[hl][wl][3], overwritten) from dL/dV
 * (the gradient of V_high is dL/dV itself); block sums in a fixed order. */
int hr_colour_map(const float* v_low, int wl, int hl, const float* v_high, int W, int H, float* out,
                  hr_stream stream);
int hr_colour_map_bwd(const float* d_v, int W, int H, int wl, int hl, float* d_low, hr_stream stream);

/* Mean vertex error epsilon_v (Section 4.1: mean Euclidean distance between the
 * vertices of the estimate and of the ground truth), per instance, in metres:
 * out[row * n + i] = mean_v |verts[i][v] - ref[i][v]| for verts, ref device
 * float[n][V][3].  row = *iter_dev when iter_dev (device uint32) is given, else 0;
 * rows >= `rows` are not written (out: device float[rows][n]), so one call in a
 * captured iteration records the error trajectory.  Summed in a fixed order. */
int hr_vertex_error(const float* verts, const float* ref, int V, int n, float* out, const uint32_t* iter_dev,
                    int rows, hr_stream stream);

/* ---------------------------------------------------------------------------------
 * Batches: many hand instances refined together.  Each instance has its own
 * parameters, cameras, resolution (shared by its views), samples per pixel and edge
 * samples per view; all share one hand model (topology, blendshapes, weights,
 * albedo).  A batch context fixes that layout once; every batch call then runs all
 * instances in ONE launch per kernel (skinning, one BVH build block per instance, the
 * render kernels over all views' sub-tiles, per-instance loss reductions), so a whole
 * iteration of all instances is a short fixed sequence of launches that a CUDA graph
 * can capture.  Device arrays of a batch are the per-instance arrays concatenated in
 * instance order:
 *   params, d_params   float[n][61]
 *   verts, d_verts     float[n][V][3]
 *   cams               hr_camera[sum_i views_i], instance-major
 *   images, background,
 *   observed, adjoint  float[P][3], P = sum_i views_i H_i W_i; instance i's views are
 *                      [N_i][H_i][W_i][3] starting at pixel pixel_offsets[i]
 *   mask               uint8[P]
 *   loss               float[n]
 * Samples of instance i use hr_instance_desc.instance as the Philox instance field,
 * so instance i renders exactly what a single-instance context renders with
 * hr_render_opts.instance = that value, its spp and edge_samples (up to float32
 * summation order in the backward).  Single-instance calls on a batch context, and
 * batch calls on a single-instance context, return HR_ERR_ARG.
 * --------------------------------------------------------------------------------- */
typedef struct hr_instance_desc {
    int32_t views;          /* N_i >= 1                                              */
    int32_t width, height;  /* W_i, H_i of all its views                             */
    int32_t spp;            /* primary samples per pixel, 1 .. 65536                 */
    int32_t edge_samples;   /* silhouette-edge samples per view (>= 0)               */
    uint32_t instance;      /* Philox instance field, < 65536                        */
} hr_instance_desc;

/* Create a batch context on the current CUDA device for the n instances of `desc`
 * (host array).  limits->max_V, max_F, max_E bound the model as for
 * hr_context_create (the view and image fields are not used).  All scratch is
 * allocated here, once.  HR_ERR_ARG for invalid descriptors, HR_ERR_UNSUPPORTED for
 * layouts beyond 2^27 sub-tiles of 8x4 pixels, HR_ERR_CUDA when an allocation fails.
 * Destroy with hr_context_destroy. */
int hr_batch_create(const hr_limits* limits, const hr_instance_desc* desc, int n, hr_context** out);

/* Host copies of the layout: view_offsets[i] = first camera of instance i,
 * pixel_offsets[i] = first pixel of instance i (host arrays of n + 1; the last
 * entries are the totals). */
int hr_batch_layout(hr_context* ctx, int32_t* view_offsets, int64_t* pixel_offsets);

/* The single-instance calls above, over every instance of a batch.  opts supplies the
 * seed, iteration (or iter_dev), shading, edge offset and flags; spp, edge_samples and
 * the instance field come from the descriptors.  hr_loss_batch writes one loss per
 * instance (each the mean over that instance's own masked pixel-channels). */
int hr_skin_batch(hr_context* ctx, const hr_model* model, const float* params, float* verts, hr_stream stream);
int hr_skin_bwd_batch(hr_context* ctx, const hr_model* model, const float* params, const float* d_verts,
                      float* d_params, hr_stream stream);
int hr_build_bvh_batch(hr_context* ctx, const hr_model* model, const float* verts, hr_stream stream);
int hr_render_fwd_batch(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams,
                        const float* background, const hr_render_opts* opts, float* image, hr_stream stream);
int hr_loss_batch(hr_context* ctx, const float* image, const float* observed, const uint8_t* mask, float* loss,
                  float* adjoint, hr_stream stream);
int hr_render_bwd_batch(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams,
                        const float* background, const hr_render_opts* opts, const float* adjoint, float* d_verts,
                        hr_stream stream);

/* Retiring converged instances of a batch (Section 3.3 refines each multiframe until
 * its estimate stops improving; in a batch an instance that has converged would
 * otherwise keep costing a full share of every launch).  hr_batch_set_active gives
 * the batch context a device int32[n] mask (NULL: every instance active), read by
 * every batch call at each launch (so a captured iteration sees later changes):
 * instances with 0 are skipped by hr_skin_batch, hr_skin_bwd_batch, hr_update_bvh /
 * hr_build_bvh_batch (single-block builds), hr_render_fwd_batch, hr_loss_batch and
 * hr_render_bwd_batch, and their outputs keep their previous values.  The two calls
 * below clear mask entries on the device; with lr_scale (the per-entry step sizes of
 * hr_adam_step_dev, device float[n][per_instance]) they also zero the retired
 * instance's steps, so that Adam leaves its parameters where they are.
 *   hr_retire_converged: instance i retires when err[*iter_dev][i] <= threshold (err
 *     as written by hr_vertex_error, rows rows; a criterion with ground truth, the
 *     benchmark's 1 mm).
 *   hr_retire_plateau: instance i retires once loss[i] (hr_loss_batch) has not fallen
 *     below (1 - rel_tol) best[i] for `patience` calls in a row; best (device
 *     float[n], start at +inf) and stall (device int32[n], start at 0) are its state. */
int hr_batch_set_active(hr_context* ctx, const int32_t* active);
int hr_retire_converged(const float* err, const uint32_t* iter_dev, int rows, int n, float threshold,
                        int32_t* active, float* lr_scale, int per_instance, hr_stream stream);
int hr_retire_plateau(const float* loss, int n, float rel_tol, int patience, float* best, int32_t* stall,
                      int32_t* active, float* lr_scale, int per_instance, hr_stream stream);

/* Lower-resolution copies of a multiframe, for the learned proposal, whose network
 * takes views of its training rig's resolution: hr_box_downsample writes the f x f
 * box means of device float[N][H][W][3] images into float[N][H/f][W/f][3] (a pixel
 * of the result covers the f x f pixels it averages, so the cameras' intrinsics scale
 * by 1/f); hr_mask_downsample the maximum of f x f blocks of uint8[N][H][W] masks.
 * H and W multiples of f, else HR_ERR_ARG. */
int hr_box_downsample(const float* src, int N, int H, int W, int f, float* dst, hr_stream stream);
int hr_mask_downsample(const uint8_t* src, int N, int H, int W, int f, uint8_t* dst, hr_stream stream);

/* Area resampling to the proposal network's grid from views of any size (the
 * heterogeneous batch's 512 x 384 views become 256 x 256 with anisotropic pixels):
 * hr_area_resample writes into device float[N][Ho][Wo][3] the overlap-weighted mean
 * of device float[N][H][W][3] over each output pixel's footprint
 * [x W/Wo, (x+1) W/Wo) x [y H/Ho, (y+1) H/Ho) (pixel (x, y) of an image covers
 * [x, x+1) x [y, y+1), so a camera's fx, cx scale by Wo/W and fy, cy by Ho/H);
 * integer factors give the box means of hr_box_downsample.  hr_mask_resample writes
 * the maximum of uint8[N][H][W] masks over the input pixels each output pixel
 * overlaps.  Sizes 1 .. 65536 and src != dst, else HR_ERR_ARG (the two buffers must
 * not overlap at all; only equality is checked); asynchronous. */
int hr_area_resample(const float* src, int N, int H, int W, float* dst, int Ho, int Wo, hr_stream stream);
int hr_mask_resample(const uint8_t* src, int N, int H, int W, uint8_t* dst, int Ho, int Wo, hr_stream stream);

/* BF16 matrix product on the tensor cores (tcgen05, float32 accumulation), the
 * building block of the learned proposal network:
 *   C[M][N] = act(A[M][K] B[N][K]^T + bias[N]),  act = ReLU when relu != 0.
 * A, B: device bf16, row-major with K contiguous and row pitches lda, ldb (elements;
 * multiples of 8, base addresses 16-byte aligned); K a multiple of 64.  bias: device
 * float[N] or NULL.  C: device bf16 (out_bf16 != 0) or float32, row pitch ldc.
 * splits > 1 divides K among that many CTAs per output tile (for long K) and needs
 * split_buf, device float[splits][M][N]; the partials are summed in split order.
 * A bounded wait that runs out sets HR_ERR_TIMEOUT in the context's status word. */
int hr_gemm_bf16(hr_context* ctx, const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                 const float* bias, int relu, void* C, int ldc, int out_bf16, int splits, float* split_buf,
                 hr_stream stream);

/* ---------------------------------------------------------------------------------
 * Learned proposal (an extension: the paper refines by gradient descent alone).  A
 * small network maps per-view residual images of an estimate to a parameter update;
 * refinement takes its proposals first and keeps each instance's best candidate by
 * the photometric loss, so the plain method stays the fallback and the judge.
 *
 * Network, per view of each of B instances with `views` views (B * views a multiple
 * of 4), all weights and activations bf16 with float32 accumulation on the tensor
 * cores (hr_gemm_bf16):
 *   input   128x128x8: 2x2 means of a 256x256 render R and observation O, as
 *           (R - O, O, 0, 0)
 *   conv    five 3x3 convolutions, stride 2, padding 1, ReLU: 8->32, 32->64, 64->128,
 *           128->128, 128->128 (output 4x4x128)
 *   view    ReLU(Wv [features(2048), camera R (9), camera centre / 0.6 m (3), 0] + bv),
 *           256 per view; the maximum over the instance's views
 *   head    ReLU(W1 . + b1) (256), W2 . + b2 (61) times the per-group scales
 *           (0.5 shape, 0.1 rad pose, 0.1 rad root rotation, 0.005 m translation)
 * Parameters: one float32 vector of hr_net_param_count() entries: per layer W [N][K]
 * row-major then b [N], for the five convolutions (K = 9 Cin rounded up to 64, tap-
 * major then channel: k = (3 ky + kx) Cin + c, the padding columns zero), the view
 * layer (K = 2112), W1 (K = 256), W2 (N = 64: rows 61-63 zero).
 * --------------------------------------------------------------------------------- */
typedef struct hr_net hr_net;

int hr_net_param_count(void);
/* Allocate a network for B instances of `views` views (all scratch up front). */
int hr_net_create(int B, int views, hr_net** out);
int hr_net_destroy(hr_net* net);
/* Load parameters (device float[hr_net_param_count()]) and reset the Adam moments. */
int hr_net_set_params(hr_net* net, const float* params, hr_stream stream);
/* Copy the parameters and/or the last gradient (device float[count], either NULL). */
int hr_net_get_params(hr_net* net, float* params, float* grads, hr_stream stream);
/* Inputs from renders and observations: device float[B * views][H][W][3] with
 * W = H = 256 (instances' views consecutive). */
int hr_net_inputs(hr_net* net, const float* render, const float* observed, int W, int H, hr_stream stream);
/* Inputs given directly: device bf16[B * views][128][128][8]. */
int hr_net_set_inputs_bf16(hr_net* net, const void* x0, hr_stream stream);
/* Forward: out[b] = base[b] + delta[b] (device float[B][61]; base NULL = 0).
 * cams: device hr_camera[B * views]. */
int hr_net_forward(hr_net* net, const float* cams, const float* base, float* out, hr_stream stream);
/* Backward of the last forward for d_out = dL/d delta (device float[B][61]): the
 * parameter gradient, kept in the network (hr_net_get_params). */
int hr_net_backward(hr_net* net, const float* d_out, hr_stream stream);
/* Adam step (step >= 1) on the parameters with the last gradient. */
int hr_net_adam(hr_net* net, float lr, float beta1, float beta2, float eps, int step, hr_stream stream);
/* Synchronise and return/clear the network's status (HR_OK or HR_ERR_TIMEOUT). */
int hr_net_status(hr_net* net, hr_stream stream);

/* Training loss of the proposal: loss[i] = (1/V) sum_v |verts[i][v] - ref[i][v]|^2 and,
 * when d_verts is given, d_verts = d((1/n) sum_i loss[i]) / d verts (device arrays
 * float[n][V][3], loss float[n]). */
int hr_vertex_mse(const float* verts, const float* ref, int V, int n, float* loss, float* d_verts,
                  hr_stream stream);
/* image[i] += sigma * N(0, 1) for i < n (Philox4x32-10 keyed by seed, Box-Muller). */
int hr_add_noise(float* image, int64_t n, float sigma, uint64_t seed, hr_stream stream);
/* Per instance i < n, the candidate with the lowest loss (the earliest on ties):
 * params[i] = candidates[k*][i] for candidates device float[K][n][61], losses float[K][n];
 * chosen (device int32[n] or NULL) receives k*. */
int hr_select_best(const float* candidates, const float* losses, int K, int n, float* params, int32_t* chosen,
                   hr_stream stream);

/* Diagnostics over the context's current scene (used by the tests; on a batch
 * context they see instance 0):
 *   hr_trace:        closest hit of n rays (origins, dirs: device float[n][3]) against
 *                    the last built BVH: tri (device int32[n], -1 = miss), tuv
 *                    (device float[n][3] = t, u, v);
 *   hr_get_normals:  copy the unit vertex normals to device float[V][3];
 *   hr_silhouettes:  per-view silhouette edge ids (ascending) into lists (device
 *                    int32[N][E]) and counts (device int32[N]). */
int hr_trace(hr_context* ctx, const float* origins, const float* dirs, int n, int32_t* tri, float* tuv,
             hr_stream stream);
int hr_get_normals(hr_context* ctx, float* normals, hr_stream stream);
int hr_silhouettes(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N,
                   int32_t* lists, int32_t* counts, hr_stream stream);

/* Work counters of the calls made with HR_STATS since the last read: synchronise
 * `stream`, copy 18 counters to host `out` and clear them.  out[0..5] = forward,
 * out[6..11] = the interior backward, out[12..17] = the edge-sample rays, each
 * (estimator samples resolved, rays made individually, BVH nodes visited,
 * Moller-Trumbore tests, hits, candidate screen-box tests).  A sample is resolved
 * without its own ray when no triangle's screen box meets its sub-tile (the forward)
 * or its sub-tile's frustum misses the scene (the backward's own lists). */
int hr_get_stats(hr_context* ctx, uint64_t* out, hr_stream stream);

/* Device times (ms) of the internal kernels of the most recent hr_render_fwd and
 * hr_render_bwd made with HR_TIMING, from CUDA events recorded on their stream:
 * ms[0..2] forward candidate lists / shading / combine, ms[3..5] backward work items /
 * shading / partial reduction, ms[6] silhouettes, ms[7] edge samples, ms[8] normal
 * adjoint; -1 for a kernel that did not run.  n >= 9.  Waits for those events. */
int hr_kernel_times(hr_context* ctx, float* ms, int n);

/* Synchronise `stream`, then return and clear the device status word: HR_OK, or the
 * HR_ERR_* code of a device-detected error since the last call (HR_ERR_ARG for face
 * or parent indices out of range, then HR_ERR_INTERNAL, HR_ERR_NONFINITE,
 * HR_ERR_LIMIT, HR_ERR_TIMEOUT). */
int hr_get_status(hr_context* ctx, hr_stream stream);

/* Static text for a status code. */
const char* hr_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* HANDRT_H */
