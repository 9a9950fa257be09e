// C ABI of handrt: context management, argument checks and the entry points
// declared in include/handrt.h.  Every entry point returns an HR_* code and never
// throws; device-side errors go to the context's status word.
#include <cstdlib>
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "hr_internal.h"

using hr::Cam;
using hr::Context;

namespace {

struct Alloc {
  void** slots[48];
  int n = 0;
};

template <class T>
bool dev_alloc(T** p, size_t count, Alloc& list) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  list.slots[list.n++] = reinterpret_cast<void**>(p);
  return true;
}

void free_ctx(Context* c) {
  hr::free_edge_buffers(c);
  for (int i = 0; i < 2 * hr::kTimeSlots; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  void* ptrs[] = {c->nodes,   c->tris,    c->normals,   c->normal_len, c->partials,      c->dN,
                  c->sil,     c->sil_count, c->loss_partials, c->counters,   c->skin_partials,
                  c->status,  c->stats,   c->pool_bb,   c->pool_z,     c->pool_rec,      c->st_info,
                  c->items,   c->item_part, c->extra,   c->work_ctr,   c->vt,            c->it,
                  c->bvh_parent, c->bvh_valid, c->bvh_keys, c->bvh_flags, c->bvh_bounds, c->bvh_bad,
                  c->bvh_mode, c->extra64, c->ct_partials, c->dedge, c->ovf_list, c->acc_fx, c->act_off,
                  c->trace_list, c->st_done, c->cand_st, c->bin_cnt, c->bvh_stale, c->bvh_need};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete[] c->hvt;
  delete[] c->hit;
  delete c;
}

bool model_ok(const hr_model* m, const Context* c) {
  if (!m) return false;
  if (m->V <= 0 || m->F <= 0 || m->E <= 0 || m->J <= 0 || m->K < 0) return false;
  if (m->V > c->lim.max_V || m->F > c->lim.max_F || m->E > c->lim.max_E) return false;
  if (m->J > hr::kMaxJ || m->K > hr::kMaxK) return false;
  return m->v_template && m->shapedirs && m->weights && m->j_template && m->j_shapedirs && m->parents && m->faces &&
         m->edges && m->edge_faces && m->vf_offsets && m->vf_faces && m->albedo;
}

// a texture needs its size and the model's texture coordinates
bool tex_ok(const hr_render_opts* o, const hr_model* m) {
  return !o->texture || (m && m->uv && o->tex_w >= 1 && o->tex_h >= 1 && o->tex_w <= 16384 && o->tex_h <= 16384);
}

bool opts_ok(const hr_render_opts* o) {
  return o && o->spp >= 1 && o->spp <= 65536 && o->edge_samples >= 0 && o->edge_eps_px > 0.0f &&
         o->edge_eps_px <= 0.25f;
}

bool image_ok(const Context* c, int N, int H, int W) {
  return N >= 1 && H >= 1 && W >= 1 && N <= c->lim.max_views && W <= c->lim.max_width && H <= c->lim.max_height;
}

bool limits_ok(const hr_limits* lim, bool batch) {
  if (lim->max_V <= 0 || lim->max_F <= 0 || lim->max_E <= 0) return false;
  if (batch) return true;
  return lim->max_views > 0 && lim->max_width > 0 && lim->max_height > 0;
}

// Allocate a context for `n` instances whose views hold `views` views, `subtiles`
// sub-tiles and `items` work-item slots in all (single instance: the limits' maxima).
int create_ctx(const hr_limits* lim, int n, size_t views, size_t subtiles, size_t items, int loss_blocks,
               Context** out) {
  Context* c = new (std::nothrow) Context();
  if (!c) return HR_ERR_CUDA;
  std::memset(c, 0, sizeof(Context));
  c->lim = *lim;
  c->n_inst = n;
  c->tune = hr_tuning{2, 8, 16, 8, 4, 4, 16, 4};
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return HR_ERR_CUDA;
  }
  if (hr::render_grid(c->device, &c->render_blocks, &c->render_threads, &c->num_sms) != HR_OK) {
    delete c;
    return HR_ERR_CUDA;
  }
  Alloc a;
  const size_t V = lim->max_V, F = lim->max_F, ni = (size_t)n;
  c->pool_cap = (int)std::min<size_t>((size_t)1 << 28, 16 * subtiles + 4096);
  c->item_cap = (int)items;
  c->loss_blocks = loss_blocks;
  // partials of the single-instance backward, one per SM (V <= kPartialMaxV)
  const size_t partial_blocks = (n == 1 && V <= (size_t)hr::kPartialMaxV) ? (size_t)c->num_sms : 1;
  const size_t nviews = views;
  bool ok = dev_alloc(&c->nodes, ni * F, a) && dev_alloc(&c->tris, ni * 3 * F, a) &&
            dev_alloc(&c->normals, ni * 3 * V, a) && dev_alloc(&c->normal_len, ni * V, a) &&
            dev_alloc(&c->partials, partial_blocks * 6 * V, a) && dev_alloc(&c->dN, ni * 3 * V, a) &&
            dev_alloc(&c->dedge, ni * 3 * V, a) && dev_alloc(&c->acc_fx, ni * 6 * V, a) &&
            dev_alloc(&c->sil, nviews * lim->max_E, a) &&
            dev_alloc(&c->sil_count, nviews, a) &&
            dev_alloc(&c->loss_partials, ni * hr::kLossStride(c->loss_blocks), a) &&
            dev_alloc(&c->counters, ni * 4, a) && dev_alloc(&c->skin_partials, ni * hr::kSkinBlocks * hr::kSkinAcc, a) &&
            dev_alloc(&c->status, 1, a) && dev_alloc(&c->stats, 3 * hr::kStatsPer, a) &&
            dev_alloc(&c->pool_bb, c->pool_cap, a) && dev_alloc(&c->pool_z, c->pool_cap, a) &&
            dev_alloc(&c->pool_rec, c->pool_cap, a) && dev_alloc(&c->st_info, subtiles, a) &&
            dev_alloc(&c->items, c->item_cap, a) && dev_alloc(&c->item_part, (size_t)c->item_cap * 32, a) &&
            dev_alloc(&c->extra, ni * 6 * V, a) && dev_alloc(&c->work_ctr, hr::ctr_words(ni), a) &&
            dev_alloc(&c->ovf_list, subtiles, a) && dev_alloc(&c->trace_list, c->item_cap, a) &&
            dev_alloc(&c->st_done, subtiles, a) && dev_alloc(&c->cand_st, subtiles, a) &&
            dev_alloc(&c->bin_cnt, subtiles, a) &&
            dev_alloc(&c->bvh_parent, ni * 2 * F, a) && dev_alloc(&c->bvh_valid, ni, a) &&
            dev_alloc(&c->bvh_bounds, ni * 6, a) && dev_alloc(&c->bvh_bad, ni, a) && dev_alloc(&c->bvh_mode, ni, a) &&
            dev_alloc(&c->bvh_stale, ni, a) && dev_alloc(&c->bvh_need, ni, a);
  // keys of the multi-block build, for meshes beyond one block's shared memory
  c->bvh_pmax = 1;
  while ((size_t)c->bvh_pmax < F) c->bvh_pmax <<= 1;
  if (ok && F > 2048)
    ok = dev_alloc(&c->bvh_keys, ni * (size_t)c->bvh_pmax, a) && dev_alloc(&c->bvh_flags, ni * F, a);
  if (ok && V > 8192) ok = dev_alloc(&c->extra64, ni * 6 * V, a);
  if (ok && n == 1) ok = dev_alloc(&c->ct_partials, views * 64 * 10, a);
  if (ok) ok = cudaMemset(c->counters, 0, ni * 4 * sizeof(unsigned)) == cudaSuccess &&
               cudaMemset(c->status, 0, sizeof(int)) == cudaSuccess &&
               cudaMemset(c->stats, 0, 3 * hr::kStatsPer * sizeof(unsigned long long)) == cudaSuccess &&
               cudaMemset(c->nodes, 0, ni * F * sizeof(hr::Node)) == cudaSuccess &&
               cudaMemset(c->bvh_valid, 0, ni * sizeof(int)) == cudaSuccess &&
               cudaMemset(c->st_done, 0, subtiles * sizeof(unsigned)) == cudaSuccess &&
               cudaMemset(c->bin_cnt, 0, subtiles * sizeof(unsigned)) == cudaSuccess &&
               cudaMemset(c->bvh_stale, 0, ni * sizeof(int)) == cudaSuccess &&
               cudaMemset(c->bvh_need, 0, ni * sizeof(int)) == cudaSuccess;
  for (int i = 0; ok && i < 2 * hr::kTimeSlots; ++i) ok = cudaEventCreate(&c->ev[i]) == cudaSuccess;
  if (ok)
    ok = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
  // kernel attributes are set here, once, so that the per-iteration calls are only
  // launches and asynchronous memsets
  if (ok)
    ok = hr::configure_bvh_kernels() == HR_OK &&
         hr::configure_gemm_kernels() == HR_OK;
  if (!ok) {
    cudaGetLastError();
    free_ctx(c);
    return HR_ERR_CUDA;
  }
  *out = c;
  return HR_OK;
}

}  // namespace

extern "C" {

int hr_context_create(const hr_limits* lim, hr_context** out) {
  if (!lim || !out) return HR_ERR_ARG;
  *out = nullptr;
  if (!limits_ok(lim, false)) return HR_ERR_ARG;
  if (lim->max_V > 65536 || lim->max_F > 65536 || lim->max_views > 65535 || lim->max_width > 16384 ||
      lim->max_height > 16384 || (long long)lim->max_views * lim->max_width * lim->max_height > (1ll << 31) / 3)
    return HR_ERR_UNSUPPORTED;
  const size_t subtiles = (size_t)hr::subtiles_for(lim->max_views, lim->max_width, lim->max_height);
  Context* c = nullptr;
  int rc = create_ctx(lim, 1, (size_t)lim->max_views, subtiles,
                      std::min<size_t>((size_t)1 << 26, 2 * subtiles + 1024), hr::kLossBlocks, &c);
  if (rc != HR_OK) return rc;
  *out = reinterpret_cast<hr_context*>(c);
  return HR_OK;
}

int hr_batch_create(const hr_limits* lim, const hr_instance_desc* desc, int n, hr_context** out) {
  if (!lim || !desc || !out || n < 1) return HR_ERR_ARG;
  *out = nullptr;
  if (!limits_ok(lim, true)) return HR_ERR_ARG;
  if (lim->max_V > 65536 || lim->max_F > 65536 || n > 65536) return HR_ERR_UNSUPPORTED;
  long long views = 0, subtiles = 0, pixels = 0, items = 0;
  for (int i = 0; i < n; ++i) {
    const hr_instance_desc& d = desc[i];
    if (d.views < 1 || d.width < 1 || d.height < 1 || d.spp < 1 || d.spp > 65536 || d.edge_samples < 0)
      return HR_ERR_ARG;
    if (d.views > 65535 || d.width > 16384 || d.height > 16384 || d.instance > 65535u) return HR_ERR_UNSUPPORTED;
    const long long st = (long long)d.views * hr::subtiles_for(1, d.width, d.height);
    views += d.views;
    subtiles += st;
    pixels += (long long)d.views * d.width * d.height;
    items += 2 * st + 64;
  }
  if (subtiles > (1ll << 27) || items > (1ll << 28) || views > (1ll << 24)) return HR_ERR_UNSUPPORTED;
  hr::ViewRec* hv = new (std::nothrow) hr::ViewRec[views];
  hr::InstRec* hi = new (std::nothrow) hr::InstRec[n];
  if (!hv || !hi) {
    delete[] hv;
    delete[] hi;
    return HR_ERR_CUDA;
  }
  int g = 0, st0 = 0, ib = 0, max_ne = 0;
  long long pix0 = 0;
  bool vec = true;
  for (int i = 0; i < n; ++i) {
    const hr_instance_desc& d = desc[i];
    hr::InstRec& r = hi[i];
    r.view0 = g;
    r.nviews = d.views;
    r.pix0 = pix0;
    r.ctr1_hi = d.instance << 16;
    r.spp = d.spp;
    r.ne = d.edge_samples;
    r.st0 = st0;
    const int per_view = hr::subtiles_for(1, d.width, d.height);
    r.nst = d.views * per_view;
    r.ibase = ib;
    r.icap = 2 * r.nst + 64;
    ib += r.icap;
    vec = vec && (pix0 % 4) == 0;
    for (int v = 0; v < d.views; ++v, ++g) {
      hr::ViewRec& w = hv[g];
      w.inst = i;
      w.ctr1 = (uint32_t)v | (d.instance << 16);
      w.H = d.height;
      w.W = d.width;
      w.spp = d.spp;
      w.ne = d.edge_samples;
      w.st0 = st0;
      w.nsx = hr::subtile_columns(d.width);
      w.pix0 = pix0;
      st0 += per_view;
      pix0 += (long long)d.width * d.height;
    }
    r.npix = pix0 - r.pix0;
    max_ne = std::max(max_ne, d.edge_samples);
  }
  Context* c = nullptr;
  int rc = create_ctx(lim, n, (size_t)views, (size_t)subtiles, (size_t)items, hr::kLossBlocksBatch, &c);
  if (rc != HR_OK) {
    delete[] hv;
    delete[] hi;
    return rc;
  }
  c->hvt = hv;
  c->hit = hi;
  c->nviews = (int)views;
  c->total_st = (int)subtiles;
  c->total_pix = pixels;
  c->max_ne = max_ne;
  c->loss_vec = vec;
  if (cudaMalloc(reinterpret_cast<void**>(&c->vt), sizeof(hr::ViewRec) * views) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&c->it), sizeof(hr::InstRec) * n) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&c->act_off), sizeof(int) * 2 * ((size_t)n + 1)) != cudaSuccess ||
      cudaMemcpy(c->vt, hv, sizeof(hr::ViewRec) * views, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->it, hi, sizeof(hr::InstRec) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    free_ctx(c);
    return HR_ERR_CUDA;
  }
  *out = reinterpret_cast<hr_context*>(c);
  return HR_OK;
}

int hr_batch_set_active(hr_context* ctx, const int32_t* active) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt) return HR_ERR_ARG;
  c->active = active;
  return HR_OK;
}

int hr_retire_converged(const float* err, const uint32_t* iter_dev, int rows, int n, float threshold,
                        int32_t* active, float* lr_scale, int per_instance, hr_stream stream) {
  if (!err || !active || rows < 1 || n < 1 || !std::isfinite(threshold) || (lr_scale && per_instance < 1))
    return HR_ERR_ARG;
  return hr::launch_retire_converged(err, iter_dev, rows, n, threshold, active, lr_scale, per_instance,
                                     (cudaStream_t)stream);
}

int hr_retire_plateau(const float* loss, int n, float rel_tol, int patience, float* best, int32_t* stall,
                      int32_t* active, float* lr_scale, int per_instance, hr_stream stream) {
  if (!loss || !best || !stall || !active || n < 1 || !(rel_tol >= 0.0f && rel_tol < 1.0f) || patience < 1 ||
      (lr_scale && per_instance < 1))
    return HR_ERR_ARG;
  return hr::launch_retire_plateau(loss, n, rel_tol, patience, best, stall, active, lr_scale, per_instance,
                                   (cudaStream_t)stream);
}

int hr_box_downsample(const float* src, int N, int H, int W, int f, float* dst, hr_stream stream) {
  if (!src || !dst || N < 1 || f < 1 || H < f || W < f || H % f || W % f || (long long)N * H * W > (1ll << 40))
    return HR_ERR_ARG;
  return hr::launch_box_downsample(src, N, H, W, f, dst, (cudaStream_t)stream);
}

int hr_mask_downsample(const uint8_t* src, int N, int H, int W, int f, uint8_t* dst, hr_stream stream) {
  if (!src || !dst || N < 1 || f < 1 || H < f || W < f || H % f || W % f || (long long)N * H * W > (1ll << 40))
    return HR_ERR_ARG;
  return hr::launch_mask_downsample(src, N, H, W, f, dst, (cudaStream_t)stream);
}

static bool resample_args_ok(const void* src, int N, int H, int W, int Ho, int Wo, const void* dst) {
  return src && dst && src != dst && N >= 1 && H >= 1 && W >= 1 && Ho >= 1 && Wo >= 1 && H <= (1 << 16) && W <= (1 << 16) &&
         Ho <= (1 << 16) && Wo <= (1 << 16) && (long long)N * H * W <= (1ll << 40) &&
         (long long)N * Ho * Wo <= (1ll << 40);
}

int hr_area_resample(const float* src, int N, int H, int W, float* dst, int Ho, int Wo, hr_stream stream) {
  if (!resample_args_ok(src, N, H, W, Ho, Wo, dst)) return HR_ERR_ARG;
  return hr::launch_area_resample(src, N, H, W, Ho, Wo, dst, (cudaStream_t)stream);
}

int hr_mask_resample(const uint8_t* src, int N, int H, int W, uint8_t* dst, int Ho, int Wo, hr_stream stream) {
  if (!resample_args_ok(src, N, H, W, Ho, Wo, dst)) return HR_ERR_ARG;
  return hr::launch_mask_resample(src, N, H, W, Ho, Wo, dst, (cudaStream_t)stream);
}

int hr_batch_layout(hr_context* ctx, int32_t* view_offsets, int64_t* pixel_offsets) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt || !view_offsets || !pixel_offsets) return HR_ERR_ARG;
  for (int i = 0; i < c->n_inst; ++i) {
    view_offsets[i] = c->hit[i].view0;
    pixel_offsets[i] = c->hit[i].pix0;
  }
  view_offsets[c->n_inst] = c->nviews;
  pixel_offsets[c->n_inst] = c->total_pix;
  return HR_OK;
}

int hr_set_tuning(hr_context* ctx, const hr_tuning* t) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !t) return HR_ERR_ARG;
  const auto rays_ok = [](int r) { return r == 1 || r == 2 || r == 4; };
  if (!rays_ok(t->rays_per_lane) || !rays_ok(t->bwd_rays_per_lane) || t->cand_per_chunk < 1 ||
      t->bwd_cand_per_chunk < 1 ||
      t->max_chunks < 1 || t->max_chunks > 16 || t->blocks_per_sm < 1 || t->blocks_per_sm > 8 ||
      t->bwd_blocks_per_sm < 1 || t->bwd_blocks_per_sm > 8 ||
      !(t->edge_lanes == 2 || t->edge_lanes == 4 || t->edge_lanes == 8 || t->edge_lanes == 16 ||
        t->edge_lanes == 32))
    return HR_ERR_ARG;
  c->tune = *t;
  return HR_OK;
}

int hr_get_tuning(hr_context* ctx, hr_tuning* t) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !t) return HR_ERR_ARG;
  *t = c->tune;
  return HR_OK;
}

int hr_context_destroy(hr_context* ctx) {
  if (!ctx) return HR_ERR_ARG;
  Context* c = reinterpret_cast<Context*>(ctx);
  cudaDeviceSynchronize();
  free_ctx(c);
  return HR_OK;
}

// host copy of n int32 from device memory (synchronous)
static bool copy_ints(std::vector<int32_t>& dst, const int32_t* src, size_t n) {
  dst.resize(n);
  if (n == 0) return true;
  if (cudaMemcpy(dst.data(), src, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

int hr_model_check(const hr_model* m) {
  if (!m || m->V <= 0 || m->F <= 0 || m->E <= 0 || m->J <= 0 || m->K < 0) return HR_ERR_ARG;
  if (m->J > hr::kMaxJ || m->K > hr::kMaxK) return HR_ERR_UNSUPPORTED;
  if (!m->v_template || !m->shapedirs || !m->weights || !m->j_template || !m->j_shapedirs || !m->parents ||
      !m->faces || !m->edges || !m->edge_faces || !m->vf_offsets || !m->vf_faces || !m->albedo)
    return HR_ERR_ARG;
  const int V = m->V, F = m->F, E = m->E, J = m->J;
  std::vector<int32_t> a;
  // the kinematic tree: the root first, every parent before its children
  if (!copy_ints(a, m->parents, J)) return HR_ERR_CUDA;
  if (a[0] != -1) return HR_ERR_ARG;
  for (int j = 1; j < J; ++j)
    if (a[j] < 0 || a[j] >= j) return HR_ERR_ARG;
  if (!copy_ints(a, m->faces, 3 * (size_t)F)) return HR_ERR_CUDA;
  for (int32_t x : a)
    if (x < 0 || x >= V) return HR_ERR_ARG;
  if (!copy_ints(a, m->edges, 2 * (size_t)E)) return HR_ERR_CUDA;
  for (int32_t x : a)
    if (x < 0 || x >= V) return HR_ERR_ARG;
  if (!copy_ints(a, m->edge_faces, 2 * (size_t)E)) return HR_ERR_CUDA;
  for (int e = 0; e < E; ++e)
    if (a[2 * e] < 0 || a[2 * e] >= F || a[2 * e + 1] < -1 || a[2 * e + 1] >= F) return HR_ERR_ARG;
  if (!copy_ints(a, m->vf_offsets, (size_t)V + 1)) return HR_ERR_CUDA;
  if (a[0] != 0 || a[V] > 3 * F) return HR_ERR_ARG;
  for (int v = 0; v < V; ++v)
    if (a[v + 1] < a[v]) return HR_ERR_ARG;
  const int n_inc = a[V];
  if (!copy_ints(a, m->vf_faces, (size_t)n_inc)) return HR_ERR_CUDA;
  for (int32_t x : a)
    if (x < 0 || x >= F) return HR_ERR_ARG;
  return HR_OK;
}

int hr_skin(hr_context* ctx, const hr_model* model, const float* params, float* verts, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || c->vt || !model_ok(model, c) || !params || !verts) return HR_ERR_ARG;
  return hr::launch_skin(c, model, params, verts, nullptr, (cudaStream_t)stream);
}

int hr_skin_bwd(hr_context* ctx, const hr_model* model, const float* params, const float* d_verts, float* d_params,
                hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || c->vt || !model_ok(model, c) || !params || !d_verts || !d_params) return HR_ERR_ARG;
  return hr::launch_skin_bwd(c, model, params, d_verts, nullptr, d_params, (cudaStream_t)stream);
}

int hr_build_bvh(hr_context* ctx, const hr_model* model, const float* verts, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || c->vt || !model_ok(model, c) || !verts) return HR_ERR_ARG;
  return hr::launch_build_bvh(c, model, verts, (cudaStream_t)stream);
}

int hr_update_bvh(hr_context* ctx, const hr_model* model, const float* verts, const uint32_t* iter_dev,
                  int rebuild_every, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !verts || rebuild_every < 1) return HR_ERR_ARG;
  return hr::launch_update_bvh(c, model, verts, iter_dev, rebuild_every, (cudaStream_t)stream);
}

int hr_render_fwd(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N, int H,
                  int W, const float* background, const hr_render_opts* opts, float* image, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || c->vt || !model_ok(model, c) || !verts || !cams || !background || !image || !opts_ok(opts) ||
      !image_ok(c, N, H, W) || !tex_ok(opts, model))
    return HR_ERR_ARG;
  if (c->F != model->F || c->V != model->V) return HR_ERR_ARG;  // hr_build_bvh first
  return hr::launch_render_fwd(c, model, verts, reinterpret_cast<const Cam*>(cams), N, H, W, background, opts, image,
                               (cudaStream_t)stream);
}

int hr_loss(hr_context* ctx, const float* image, const float* observed, const uint8_t* mask, int N, int H, int W,
            float* loss, float* adjoint, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || c->vt || !image || !observed || !mask || !loss || !adjoint || !image_ok(c, N, H, W)) return HR_ERR_ARG;
  return hr::launch_loss(c, image, observed, mask, (long long)N * H * W, loss, adjoint, (cudaStream_t)stream);
}

int hr_loss_ct(hr_context* ctx, const float* image, const float* observed, const uint8_t* mask, const float* T,
               int N, int H, int W, float* loss, float* adjoint, float* dT, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || c->vt || !c->ct_partials || !image || !observed || !mask || !loss || !adjoint || !image_ok(c, N, H, W) ||
      9 * N > 1024)
    return HR_ERR_ARG;
  return hr::launch_loss_ct(c, image, observed, mask, T, N, (long long)H * W, loss, adjoint, dT,
                            (cudaStream_t)stream);
}

static bool edge_args_ok(const Context* c, int N, int H, int W, float low, float high) {
  return c && !c->vt && image_ok(c, N, H, W) && (long long)N * H * W <= INT_MAX && std::isfinite(low) &&
         std::isfinite(high) && low >= 0.0f && high >= low;
}

int hr_edges(hr_context* ctx, const float* image, const float* T, int N, int H, int W, float low, float high,
             float* edges, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!edge_args_ok(c, N, H, W, low, high) || !image || !edges) return HR_ERR_ARG;
  const int rc = hr::edge_buffers(c);
  if (rc != HR_OK) return rc;
  return hr::launch_edges(c, image, T, N, H, W, low, high, edges, (cudaStream_t)stream);
}

int hr_edge_loss(hr_context* ctx, const float* image, const float* T, const float* edges_obs, const uint8_t* mask,
                 int N, int H, int W, float low, float high, float weight, float* loss, float* adjoint, float* dT,
                 hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!edge_args_ok(c, N, H, W, low, high) || !image || !edges_obs || !mask || !loss || !adjoint ||
      !std::isfinite(weight))
    return HR_ERR_ARG;
  const int rc = hr::edge_buffers(c);
  if (rc != HR_OK) return rc;
  return hr::launch_edge_loss(c, image, T, edges_obs, mask, N, H, W, low, high, weight, loss, adjoint, dT,
                              (cudaStream_t)stream);
}

int hr_render_bwd(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N, int H,
                  int W, const float* background, const hr_render_opts* opts, const float* adjoint, float* d_verts,
                  hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || c->vt || !model_ok(model, c) || !verts || !cams || !background || !adjoint || !d_verts ||
      !opts_ok(opts) || !image_ok(c, N, H, W) || !tex_ok(opts, model))
    return HR_ERR_ARG;
  if (c->F != model->F || c->V != model->V) return HR_ERR_ARG;
  return hr::launch_render_bwd(c, model, verts, reinterpret_cast<const Cam*>(cams), N, H, W, background, opts,
                               adjoint, d_verts, (cudaStream_t)stream);
}

// ---- batches: the same steps over every instance of a batch context, one launch each
int hr_skin_batch(hr_context* ctx, const hr_model* model, const float* params, float* verts, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt || !model_ok(model, c) || !params || !verts) return HR_ERR_ARG;
  return hr::launch_skin(c, model, params, verts, nullptr, (cudaStream_t)stream);
}

int hr_skin_bwd_batch(hr_context* ctx, const hr_model* model, const float* params, const float* d_verts,
                      float* d_params, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt || !model_ok(model, c) || !params || !d_verts || !d_params) return HR_ERR_ARG;
  return hr::launch_skin_bwd(c, model, params, d_verts, nullptr, d_params, (cudaStream_t)stream);
}

int hr_build_bvh_batch(hr_context* ctx, const hr_model* model, const float* verts, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt || !model_ok(model, c) || !verts) return HR_ERR_ARG;
  return hr::launch_build_bvh(c, model, verts, (cudaStream_t)stream);
}

int hr_render_fwd_batch(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams,
                        const float* background, const hr_render_opts* opts, float* image, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt || !model_ok(model, c) || !verts || !cams || !background || !image || !opts ||
      !(opts->edge_eps_px > 0.0f) || !tex_ok(opts, model))
    return HR_ERR_ARG;
  if (c->F != model->F || c->V != model->V) return HR_ERR_ARG;  // hr_build_bvh_batch first
  return hr::launch_render_fwd(c, model, verts, reinterpret_cast<const Cam*>(cams), 0, 0, 0, background, opts,
                               image, (cudaStream_t)stream);
}

int hr_loss_batch(hr_context* ctx, const float* image, const float* observed, const uint8_t* mask, float* loss,
                  float* adjoint, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt || !image || !observed || !mask || !loss || !adjoint) return HR_ERR_ARG;
  return hr::launch_loss(c, image, observed, mask, c->total_pix, loss, adjoint, (cudaStream_t)stream);
}

int hr_render_bwd_batch(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams,
                        const float* background, const hr_render_opts* opts, const float* adjoint, float* d_verts,
                        hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !c->vt || !model_ok(model, c) || !verts || !cams || !background || !adjoint || !d_verts || !opts ||
      !(opts->edge_eps_px > 0.0f) || !tex_ok(opts, model))
    return HR_ERR_ARG;
  if (c->F != model->F || c->V != model->V) return HR_ERR_ARG;
  return hr::launch_render_bwd(c, model, verts, reinterpret_cast<const Cam*>(cams), 0, 0, 0, background, opts,
                               adjoint, d_verts, (cudaStream_t)stream);
}

int hr_skin_joints(hr_context* ctx, const hr_model* model, const float* params, float* verts, float* joints,
                   hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !params || !verts || !joints) return HR_ERR_ARG;
  return hr::launch_skin(c, model, params, verts, joints, (cudaStream_t)stream);
}

int hr_skin_bwd_joints(hr_context* ctx, const hr_model* model, const float* params, const float* d_verts,
                       const float* d_joints, float* d_params, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !params || !d_verts || !d_params) return HR_ERR_ARG;
  return hr::launch_skin_bwd(c, model, params, d_verts, d_joints, d_params, (cudaStream_t)stream);
}

int hr_joint_prior(const float* joints, const float* target, int J, int n, float gamma, float weight, float* loss,
                   float* d_joints, hr_stream stream) {
  if (!joints || !target || !loss || J < 1 || J > 1024 || n < 1 || !(gamma > 0.0f)) return HR_ERR_ARG;
  return hr::launch_joint_prior(joints, target, J, n, gamma, weight, loss, d_joints, (cudaStream_t)stream);
}

int hr_colour_map(const float* v_low, int wl, int hl, const float* v_high, int W, int H, float* out,
                  hr_stream stream) {
  if (!v_low || !v_high || !out || wl < 1 || hl < 1 || W < wl || H < hl || W % wl || H % hl) return HR_ERR_ARG;
  return hr::launch_colour_map(v_low, wl, hl, v_high, W, H, out, (cudaStream_t)stream);
}

int hr_colour_map_bwd(const float* d_v, int W, int H, int wl, int hl, float* d_low, hr_stream stream) {
  if (!d_v || !d_low || wl < 1 || hl < 1 || W < wl || H < hl || W % wl || H % hl) return HR_ERR_ARG;
  return hr::launch_colour_map_bwd(d_v, W, H, wl, hl, d_low, (cudaStream_t)stream);
}

int hr_vertex_error(const float* verts, const float* ref, int V, int n, float* out, const uint32_t* iter_dev,
                    int rows, hr_stream stream) {
  if (!verts || !ref || !out || V < 1 || n < 1 || rows < 1) return HR_ERR_ARG;
  return hr::launch_vertex_error(verts, ref, V, n, out, iter_dev, rows, (cudaStream_t)stream);
}

int hr_gemm_bf16(hr_context* ctx, const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                 const float* bias, int relu, void* C, int ldc, int out_bf16, int splits, float* split_buf,
                 hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !A || !B || !C || ldc < N) return HR_ERR_ARG;
  return hr::launch_gemm(A, lda, B, ldb, M, N, K, bias, relu, C, ldc, out_bf16, splits, split_buf, c->status,
                         (cudaStream_t)stream);
}

int hr_vertex_mse(const float* verts, const float* ref, int V, int n, float* loss, float* d_verts,
                  hr_stream stream) {
  if (!verts || !ref || !loss || V < 1 || n < 1) return HR_ERR_ARG;
  return hr::launch_vertex_mse(verts, ref, V, n, loss, d_verts, (cudaStream_t)stream);
}

int hr_add_noise(float* image, int64_t n, float sigma, uint64_t seed, hr_stream stream) {
  if (!image || n < 0) return HR_ERR_ARG;
  if (n == 0) return HR_OK;
  return hr::launch_add_noise(image, n, sigma, seed, (cudaStream_t)stream);
}

int hr_select_best(const float* candidates, const float* losses, int K, int n, float* params, int32_t* chosen,
                   hr_stream stream) {
  if (!candidates || !losses || !params || K < 1 || n < 1) return HR_ERR_ARG;
  return hr::launch_select_best(candidates, losses, K, n, params, chosen, (cudaStream_t)stream);
}

int hr_adam_step(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                 float eps, int step, hr_stream stream) {
  if (!params || !grad || !m || !v || n <= 0 || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return HR_ERR_ARG;
  return hr::launch_adam(params, grad, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
}

int hr_adam_step_dev(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                     float eps, const float* lr_scale, int scale_len, uint32_t* iter_dev, hr_stream stream) {
  if (!params || !grad || !m || !v || !iter_dev || n <= 0 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) || (lr_scale && scale_len < 1))
    return HR_ERR_ARG;
  return hr::launch_adam_dev(params, grad, m, v, n, lr, beta1, beta2, eps, lr_scale, scale_len, iter_dev,
                             (cudaStream_t)stream);
}

int hr_trace(hr_context* ctx, const float* origins, const float* dirs, int n, int32_t* tri, float* tuv,
             hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !origins || !dirs || !tri || !tuv || n < 0 || c->F <= 0) return HR_ERR_ARG;
  if (n == 0) return HR_OK;
  return hr::launch_trace(c, origins, dirs, n, tri, tuv, (cudaStream_t)stream);
}

int hr_get_normals(hr_context* ctx, float* normals, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !normals || c->V <= 0) return HR_ERR_ARG;
  if (cudaMemcpyAsync(normals, c->normals, sizeof(float) * 3 * c->V, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream) != cudaSuccess)
    return HR_ERR_CUDA;
  return HR_OK;
}

int hr_silhouettes(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N,
                   int32_t* lists, int32_t* counts, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !verts || !cams || !lists || !counts || N < 1 || N > c->lim.max_views)
    return HR_ERR_ARG;
  return hr::launch_silhouettes(c, model, verts, reinterpret_cast<const Cam*>(cams), N, lists, model->E, counts,
                                (cudaStream_t)stream);
}

int hr_get_stats(hr_context* ctx, uint64_t* out, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !out) return HR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpy(out, c->stats, 3 * hr::kStatsPer * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      cudaMemset(c->stats, 0, 3 * hr::kStatsPer * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  return HR_OK;
}

static_assert(2 * hr::kTimeSlots <= (int)(sizeof(hr::Context::ev) / sizeof(cudaEvent_t)), "event slots");

int hr_kernel_times(hr_context* ctx, float* ms, int n) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !ms || n < hr::kTimeSlots) return HR_ERR_ARG;
  const int need[hr::kTimeSlots] = {1, 1, 1, 4, 4, 4, 8, 8, 16};
  for (int i = 0; i < hr::kTimeSlots; ++i) {
    ms[i] = -1.0f;
    if (!(c->ev_ready & need[i])) continue;
    if (cudaEventSynchronize(c->ev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms[i], c->ev[2 * i], c->ev[2 * i + 1]) != cudaSuccess) {
      cudaGetLastError();
      return HR_ERR_CUDA;
    }
  }
  return HR_OK;
}

int hr_get_status(hr_context* ctx, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c) return HR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  int host = 0;
  if (cudaMemcpy(&host, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  if (host & hr::kStatusBadModel) return HR_ERR_ARG;
  if (host & hr::kStatusIndex) return HR_ERR_INTERNAL;
  if (host & hr::kStatusNonfinite) return HR_ERR_NONFINITE;
  if (host & hr::kStatusLimit) return HR_ERR_LIMIT;
  if (host & hr::kStatusTimeout) return HR_ERR_TIMEOUT;
  return HR_OK;
}

const char* hr_status_string(int code) {
  switch (code) {
    case HR_OK: return "ok";
    case HR_ERR_ARG: return "invalid argument";
    case HR_ERR_CUDA: return "CUDA runtime error";
    case HR_ERR_LIMIT: return "device limit reached (BVH traversal stack)";
    case HR_ERR_NONFINITE: return "non-finite parameters";
    case HR_ERR_UNSUPPORTED: return "size beyond the context's limits";
    case HR_ERR_INTERNAL: return "internal index out of range (access skipped)";
    case HR_ERR_TIMEOUT: return "a bounded device wait ran out (work abandoned)";
    default: return "unknown status";
  }
}

}  // extern "C"
