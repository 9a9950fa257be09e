// Host-side launchers shared between the handrt translation units.
#pragma once

#include <cuda_runtime.h>

#include "hr_device.cuh"

namespace hr {

int launch_skin(Context* ctx, const hr_model* m, const float* params, float* verts, float* joints, cudaStream_t s);
int launch_skin_bwd(Context* ctx, const hr_model* m, const float* params, const float* d_verts,
                    const float* d_joints, float* d_params, cudaStream_t s);
int launch_joint_prior(const float* joints, const float* target, int J, int n, float gamma, float weight,
                       float* loss, float* d_joints, cudaStream_t s);
int launch_colour_map(const float* v_low, int wl, int hl, const float* v_high, int W, int H, float* out,
                      cudaStream_t s);
int launch_colour_map_bwd(const float* d_v, int W, int H, int wl, int hl, float* d_low, cudaStream_t s);
int launch_build_bvh(Context* ctx, const hr_model* m, const float* verts, cudaStream_t s);
int launch_update_bvh(Context* ctx, const hr_model* m, const float* verts, const uint32_t* iter_dev,
                      int rebuild_every, cudaStream_t s);
int launch_bvh_lazy_refit(Context* ctx, int force, cudaStream_t s);
int launch_render_fwd(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int H, int W,
                      const float* bg, const hr_render_opts* o, float* image, cudaStream_t s);
int launch_render_bwd(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int H, int W,
                      const float* bg, const hr_render_opts* o, const float* adjoint, float* d_verts,
                      cudaStream_t s);
int launch_silhouettes(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int* lists,
                       int list_stride, int* counts, cudaStream_t s);
int launch_trace(Context* ctx, const float* o, const float* d, int n, int* tri, float* tuv, cudaStream_t s);
int launch_loss(Context* ctx, const float* image, const float* obs, const uint8_t* mask, long long P,
                float* loss, float* adjoint, cudaStream_t s);
int launch_loss_ct(Context* ctx, const float* image, const float* obs, const uint8_t* mask, const float* T, int N,
                   long long HW, float* loss, float* adjoint, float* dT, cudaStream_t s);
// the edge term D_e (hr_edge.cu); edge_buffers allocates the context's scratch once
int edge_buffers(Context* c);
void free_edge_buffers(Context* c);
int launch_edges(Context* c, const float* image, const float* T, int N, int H, int W, float low, float high,
                 float* edges, cudaStream_t s);
int launch_edge_loss(Context* c, const float* image, const float* T, const float* edges_obs, const uint8_t* mask,
                     int N, int H, int W, float low, float high, float weight, float* loss, float* adjoint,
                     float* dT, cudaStream_t s);
int launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                int step, cudaStream_t s);
int launch_adam_dev(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                    const float* lr_scale, int scale_len, uint32_t* iter_dev, cudaStream_t s);
int launch_retire_converged(const float* err, const uint32_t* iter_dev, int rows, int n, float thr, int* active,
                            float* lr_scale, int per, cudaStream_t s);
int launch_retire_plateau(const float* loss, int n, float rel_tol, int patience, float* best, int* stall, int* active,
                          float* lr_scale, int per, cudaStream_t s);
int launch_box_downsample(const float* src, int N, int H, int W, int f, float* dst, cudaStream_t s);
int launch_mask_downsample(const uint8_t* src, int N, int H, int W, int f, uint8_t* dst, cudaStream_t s);
int launch_area_resample(const float* src, int N, int H, int W, int Ho, int Wo, float* dst, cudaStream_t s);
int launch_mask_resample(const uint8_t* src, int N, int H, int W, int Ho, int Wo, uint8_t* dst, cudaStream_t s);
int launch_vertex_mse(const float* a, const float* b, int V, int n, float* loss, float* grad, cudaStream_t s);
int launch_add_noise(float* img, long long n, float sigma, uint64_t seed, cudaStream_t s);
int launch_select_best(const float* cand, const float* losses, int K, int n, float* out, int* chosen,
                       cudaStream_t s);
int launch_vertex_error(const float* verts, const float* ref, int V, int n, float* out, const uint32_t* iter_dev,
                        int rows, cudaStream_t s);

// bf16 tensor-core GEMM C = act(A B^T + bias) (hr_gemm.cu); splits > 1 needs
// split_buf of splits * M * N floats
int launch_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const float* bias, int relu,
                void* C, int ldc, int out_bf16, int splits, float* split_buf, int* status, cudaStream_t s);
int configure_gemm_kernels();

// per-device properties of the render kernels (persistent grid)
int render_grid(int device, int* blocks, int* threads, int* num_sms);
int subtiles_for(int views, int W, int H);
int subtile_columns(int W);
// one-time kernel attributes (shared-memory opt-in) on the current device
int configure_bvh_kernels();

}  // namespace hr
