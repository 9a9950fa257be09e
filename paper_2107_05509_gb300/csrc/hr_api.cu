// C ABI of handrt: context management, argument checks and the entry points
// declared in include/handrt.h.  Every entry point returns an HR_* code and never
// throws; device-side errors go to the context's status word.
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>

#include "hr_internal.h"

using hr::Cam;
using hr::Context;

namespace {

struct Alloc {
  void** slots[40];
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
  for (int i = 0; i < 2 * hr::kTimeSlots; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  void* ptrs[] = {c->nodes, c->tris,          c->normals,      c->normal_len, c->partials,
                  c->dN,    c->dm,            c->sil,          c->sil_count,  c->loss_partials,
                  c->counters, c->skin_partials, c->status, c->keys, c->parent, c->stats, c->tile_counters,
                  c->pool_bb, c->pool_z, c->pool_rec, c->st_info, c->items, c->item_part, c->extra, c->work_ctr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
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

bool opts_ok(const hr_render_opts* o) {
  return o && o->spp >= 1 && o->spp <= 65536 && o->edge_samples >= 0 && o->edge_eps_px > 0.0f;
}

bool image_ok(const Context* c, int N, int H, int W) {
  return N >= 1 && H >= 1 && W >= 1 && N <= c->lim.max_views && W <= c->lim.max_width && H <= c->lim.max_height;
}

}  // namespace

extern "C" {

int hr_context_create(const hr_limits* lim, hr_context** out) {
  if (!lim || !out) return HR_ERR_ARG;
  *out = nullptr;
  if (lim->max_V <= 0 || lim->max_F <= 0 || lim->max_E <= 0 || lim->max_views <= 0 || lim->max_width <= 0 ||
      lim->max_height <= 0)
    return HR_ERR_ARG;
  if (lim->max_V > 8192 || lim->max_F > 8192 || lim->max_views > 65535 || lim->max_width > 16384 ||
      lim->max_height > 16384 || (long long)lim->max_views * lim->max_width * lim->max_height > (1ll << 31) / 3)
    return HR_ERR_UNSUPPORTED;
  Context* c = new (std::nothrow) Context();
  if (!c) return HR_ERR_CUDA;
  std::memset(c, 0, sizeof(Context));
  c->lim = *lim;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return HR_ERR_CUDA;
  }
  if (hr::render_grid(c->device, &c->render_blocks, &c->render_threads, &c->num_sms) != HR_OK) {
    delete c;
    return HR_ERR_CUDA;
  }
  Alloc a;
  const size_t V = lim->max_V, F = lim->max_F;
  const size_t subtiles = (size_t)hr::subtiles_for(lim->max_views, lim->max_width, lim->max_height);
  c->pool_cap = (int)std::min<size_t>((size_t)1 << 28, 16 * subtiles + 4096);
  c->item_cap = (int)std::min<size_t>((size_t)1 << 26, 2 * subtiles + 1024);
  bool ok = dev_alloc(&c->nodes, F, a) && dev_alloc(&c->tris, 3 * F, a) && dev_alloc(&c->normals, 3 * V, a) &&
            dev_alloc(&c->normal_len, V, a) && dev_alloc(&c->partials, (size_t)c->render_blocks * 6 * V, a) &&
            dev_alloc(&c->dN, 3 * V, a) && dev_alloc(&c->dm, 3 * V, a) &&
            dev_alloc(&c->sil, (size_t)lim->max_views * lim->max_E, a) &&
            dev_alloc(&c->sil_count, (size_t)lim->max_views, a) &&
            dev_alloc(&c->loss_partials, (size_t)4 * hr::kLossBlocks + 8, a) && dev_alloc(&c->counters, 8, a) &&
            dev_alloc(&c->skin_partials, (size_t)hr::kSkinBlocks * hr::kSkinAcc, a) && dev_alloc(&c->status, 1, a) && dev_alloc(&c->stats, 3 * hr::kStatsPer, a) &&
            dev_alloc(&c->tile_counters, 4, a) && dev_alloc(&c->pool_bb, c->pool_cap, a) &&
            dev_alloc(&c->pool_z, c->pool_cap, a) && dev_alloc(&c->pool_rec, c->pool_cap, a) &&
            dev_alloc(&c->st_info, subtiles, a) && dev_alloc(&c->items, c->item_cap, a) &&
            dev_alloc(&c->item_part, (size_t)c->item_cap * 32, a) && dev_alloc(&c->extra, 6 * V, a) &&
            dev_alloc(&c->work_ctr, 4, a);
  if (ok) ok = cudaMemset(c->counters, 0, 8 * sizeof(unsigned)) == cudaSuccess &&
               cudaMemset(c->status, 0, sizeof(int)) == cudaSuccess &&
               cudaMemset(c->stats, 0, 3 * hr::kStatsPer * sizeof(unsigned long long)) == cudaSuccess &&
               cudaMemset(c->nodes, 0, F * sizeof(hr::Node)) == cudaSuccess;
  for (int i = 0; ok && i < 2 * hr::kTimeSlots; ++i) ok = cudaEventCreate(&c->ev[i]) == cudaSuccess;
  // kernel attributes are set here, once, so that the per-iteration calls are only
  // launches and asynchronous memsets
  if (ok) ok = hr::configure_bvh_kernels() == HR_OK && hr::configure_render_kernels(lim->max_V) == HR_OK;
  if (!ok) {
    cudaGetLastError();
    free_ctx(c);
    return HR_ERR_CUDA;
  }
  *out = reinterpret_cast<hr_context*>(c);
  return HR_OK;
}

int hr_context_destroy(hr_context* ctx) {
  if (!ctx) return HR_ERR_ARG;
  Context* c = reinterpret_cast<Context*>(ctx);
  cudaDeviceSynchronize();
  free_ctx(c);
  return HR_OK;
}

int hr_skin(hr_context* ctx, const hr_model* model, const float* params, float* verts, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !params || !verts) return HR_ERR_ARG;
  return hr::launch_skin(c, model, params, verts, (cudaStream_t)stream);
}

int hr_skin_bwd(hr_context* ctx, const hr_model* model, const float* params, const float* d_verts, float* d_params,
                hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !params || !d_verts || !d_params) return HR_ERR_ARG;
  return hr::launch_skin_bwd(c, model, params, d_verts, d_params, (cudaStream_t)stream);
}

int hr_build_bvh(hr_context* ctx, const hr_model* model, const float* verts, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !verts) return HR_ERR_ARG;
  return hr::launch_build_bvh(c, model, verts, (cudaStream_t)stream);
}

int hr_render_fwd(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N, int H,
                  int W, const float* background, const hr_render_opts* opts, float* image, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !verts || !cams || !background || !image || !opts_ok(opts) ||
      !image_ok(c, N, H, W))
    return HR_ERR_ARG;
  if (c->F != model->F || c->V != model->V) return HR_ERR_ARG;  // hr_build_bvh first
  return hr::launch_render_fwd(c, model, verts, reinterpret_cast<const Cam*>(cams), N, H, W, background, opts, image,
                               (cudaStream_t)stream);
}

int hr_loss(hr_context* ctx, const float* image, const float* observed, const uint8_t* mask, int N, int H, int W,
            float* loss, float* adjoint, hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !image || !observed || !mask || !loss || !adjoint || !image_ok(c, N, H, W)) return HR_ERR_ARG;
  return hr::launch_loss(c, image, observed, mask, (long long)N * H * W, loss, adjoint, (cudaStream_t)stream);
}

int hr_render_bwd(hr_context* ctx, const hr_model* model, const float* verts, const hr_camera* cams, int N, int H,
                  int W, const float* background, const hr_render_opts* opts, const float* adjoint, float* d_verts,
                  hr_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !model_ok(model, c) || !verts || !cams || !background || !adjoint || !d_verts || !opts_ok(opts) ||
      !image_ok(c, N, H, W))
    return HR_ERR_ARG;
  if (c->F != model->F || c->V != model->V) return HR_ERR_ARG;
  return hr::launch_render_bwd(c, model, verts, reinterpret_cast<const Cam*>(cams), N, H, W, background, opts,
                               adjoint, d_verts, (cudaStream_t)stream);
}

int hr_adam_step(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                 float eps, int step, hr_stream stream) {
  if (!params || !grad || !m || !v || n <= 0 || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return HR_ERR_ARG;
  return hr::launch_adam(params, grad, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
}

int hr_adam_step_dev(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                     float eps, uint32_t* iter_dev, hr_stream stream) {
  if (!params || !grad || !m || !v || !iter_dev || n <= 0 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return HR_ERR_ARG;
  return hr::launch_adam_dev(params, grad, m, v, n, lr, beta1, beta2, eps, iter_dev, (cudaStream_t)stream);
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
    default: return "unknown status";
  }
}

}  // extern "C"
