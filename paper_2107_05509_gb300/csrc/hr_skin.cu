// Skinning G_v (Section 3.1, "Geometry": the 61 hand parameters decoded into
// vertices) as linear blend skinning, and its adjoint.
//
//   k_skin      every block first builds the J joint transforms in shared memory
//               (one thread walks the kinematic chain: Rodrigues per joint, parents
//               before children), then each thread blends one vertex.
//   k_skin_bwd  per vertex the gradients w.r.t. the blended transforms A_j, the
//               shape coefficients (through the blendshapes) and the translation;
//               warp sums accumulate per warp in shared memory (no atomics), blocks
//               write one partial each, and the last block to finish sums the
//               partials in block order and runs the chain backward in one thread.
//               Fully deterministic.
#include <mutex>

#include "hr_internal.h"

namespace hr {

namespace {

constexpr int kSkinThreads = 256;

struct Chain {
  float Rl[kMaxJ][9];   // local rotations
  float RG[kMaxJ][9];   // global rotations
  float tG[kMaxJ][3];   // global translations
  float RA[kMaxJ][9];   // blended rotation = RG
  float tA[kMaxJ][3];   // blended translation = tG - RG J
  float J[kMaxJ][3];    // shaped joints
  float beta[kMaxK];
  float tau[3];
};

__device__ void rod_coeffs(float t, float& A, float& B, float& C, float& D) {
  if (t < 0.5f) {
    float t2 = t * t, t4 = t2 * t2, t6 = t4 * t2;
    A = 1.0f - t2 / 6.0f + t4 / 120.0f - t6 / 5040.0f;
    B = 0.5f - t2 / 24.0f + t4 / 720.0f - t6 / 40320.0f;
    C = -1.0f / 3.0f + t2 / 30.0f - t4 / 840.0f + t6 / 45360.0f;
    D = -1.0f / 12.0f + t2 / 180.0f - t4 / 6720.0f + t6 / 453600.0f;
  } else {
    float s = sinf(t), c = cosf(t), sh = sinf(0.5f * t);
    float omc = 2.0f * sh * sh;  // 1 - cos t without cancellation
    A = s / t;
    B = omc / (t * t);
    C = (t * c - s) / (t * t * t);
    D = (t * s - 2.0f * omc) / (t * t * t * t);
  }
}

__device__ void skew(const float r[3], float K[9]) {
  K[0] = 0.0f; K[1] = -r[2]; K[2] = r[1];
  K[3] = r[2]; K[4] = 0.0f; K[5] = -r[0];
  K[6] = -r[1]; K[7] = r[0]; K[8] = 0.0f;
}

__device__ void matmul3(const float A[9], const float B[9], float C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

__device__ void rodrigues(const float r[3], float R[9]) {
  float t = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  float A, B, C, D;
  rod_coeffs(t, A, B, C, D);
  float K[9], K2[9];
  skew(r, K);
  matmul3(K, K, K2);
  for (int i = 0; i < 9; ++i) R[i] = A * K[i] + B * K2[i] + ((i % 4 == 0) ? 1.0f : 0.0f);
}

// sum_ab G[a,b] dR[a,b]/dr_k
__device__ void rodrigues_grad(const float r[3], const float G[9], float out[3]) {
  float t = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  float A, B, C, D;
  rod_coeffs(t, A, B, C, D);
  float K[9], K2[9];
  skew(r, K);
  matmul3(K, K, K2);
  float gK = 0.0f, gK2 = 0.0f;
  for (int i = 0; i < 9; ++i) {
    gK += G[i] * K[i];
    gK2 += G[i] * K2[i];
  }
  for (int k = 0; k < 3; ++k) {
    float e[3] = {0.0f, 0.0f, 0.0f};
    e[k] = 1.0f;
    float E[9], EK[9], KE[9];
    skew(e, E);
    matmul3(E, K, EK);
    matmul3(K, E, KE);
    float gE = 0.0f, gS = 0.0f;
    for (int i = 0; i < 9; ++i) {
      gE += G[i] * E[i];
      gS += G[i] * (EK[i] + KE[i]);
    }
    out[k] = A * gE + B * gS + C * r[k] * gK + D * r[k] * gK2;
  }
}

struct ModelArgs {
  const float *v_template, *shapedirs, *weights, *j_template, *j_shapedirs;
  const int* parents;
  int V, J, K;
};

// the forward kinematic chain into shared memory, called by every thread of the
// block: per-joint work (shaped joint, local rotation) in parallel, then one thread
// composes parents before children
__device__ void build_chain(const ModelArgs& m, const float* __restrict__ params, Chain& ch, int* status) {
  const int tid = threadIdx.x;
  if (tid < 61 && !isfinite(params[tid])) set_status(status, kStatusNonfinite);
  if (tid < m.K) ch.beta[tid] = params[tid];
  if (tid < 3) ch.tau[tid] = params[58 + tid];
  __syncthreads();
  if (tid < 3 * m.J) {
    const int j = tid / 3, c = tid % 3;
    float acc = m.j_template[3 * j + c];
    for (int k = 0; k < m.K; ++k) acc += m.j_shapedirs[(3 * j + c) * m.K + k] * ch.beta[k];
    ch.J[j][c] = acc;
  }
  if (tid >= 64 && tid < 64 + m.J) {
    const int j = tid - 64;
    const float* r = (j == 0) ? params + 55 : params + 10 + 3 * (j - 1);
    float rr[3] = {r[0], r[1], r[2]};
    rodrigues(rr, ch.Rl[j]);
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < m.J; ++j) {
      int p = m.parents[j];
      if (p >= j || p < -1 || (j == 0) != (p < 0)) {   // parents must precede children; only joint 0 is a root
        set_status(status, kStatusBadModel);
        p = j == 0 ? -1 : 0;
      }
      if (p < 0) {
        for (int i = 0; i < 9; ++i) ch.RG[j][i] = ch.Rl[j][i];
        for (int c = 0; c < 3; ++c) ch.tG[j][c] = ch.J[j][c];
      } else {
        matmul3(ch.RG[p], ch.Rl[j], ch.RG[j]);
        for (int a = 0; a < 3; ++a) {
          float acc = ch.tG[p][a];
          for (int b = 0; b < 3; ++b) acc += ch.RG[p][3 * a + b] * (ch.J[j][b] - ch.J[p][b]);
          ch.tG[j][a] = acc;
        }
      }
      for (int i = 0; i < 9; ++i) ch.RA[j][i] = ch.RG[j][i];
      for (int a = 0; a < 3; ++a)
        ch.tA[j][a] = ch.tG[j][a] - (ch.RG[j][3 * a] * ch.J[j][0] + ch.RG[j][3 * a + 1] * ch.J[j][1] +
                                     ch.RG[j][3 * a + 2] * ch.J[j][2]);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float3 shaped_vertex(const ModelArgs& m, const Chain& ch, int v) {
  float p[3];
  for (int c = 0; c < 3; ++c) {
    float acc = m.v_template[3 * v + c];
    const float* S = m.shapedirs + (size_t)(3 * v + c) * m.K;
    for (int k = 0; k < m.K; ++k) acc += S[k] * ch.beta[k];
    p[c] = acc;
  }
  return make_float3(p[0], p[1], p[2]);
}

// blockIdx.y selects the instance: params [61] and verts [V][3] of instance y; block 0
// also writes the posed joints G_J (each joint frame's origin plus the root
// translation, [J][3]) when `joints_all` is given
__global__ void __launch_bounds__(kSkinThreads) k_skin(ModelArgs m, const float* __restrict__ params_all,
                                                       float* __restrict__ verts_all, float* __restrict__ joints_all,
                                                       int* status) {
  __shared__ Chain ch;
  const float* params = params_all + (size_t)blockIdx.y * 61;
  float* verts = verts_all + (size_t)blockIdx.y * 3 * m.V;
  build_chain(m, params, ch, status);
  if (joints_all && blockIdx.x == 0 && threadIdx.x < 3 * m.J) {
    const int j = threadIdx.x / 3, c = threadIdx.x % 3;
    joints_all[((size_t)blockIdx.y * m.J + j) * 3 + c] = ch.tG[j][c] + ch.tau[c];
  }
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < m.V; v += gridDim.x * blockDim.x) {
    float3 p = shaped_vertex(m, ch, v);
    float out[3] = {ch.tau[0], ch.tau[1], ch.tau[2]};
    const float* w = m.weights + (size_t)v * m.J;
    for (int j = 0; j < m.J; ++j) {
      float wj = w[j];
      if (wj == 0.0f) continue;
      for (int a = 0; a < 3; ++a)
        out[a] += wj * (ch.RA[j][3 * a] * p.x + ch.RA[j][3 * a + 1] * p.y + ch.RA[j][3 * a + 2] * p.z + ch.tA[j][a]);
    }
    verts[3 * v] = out[0];
    verts[3 * v + 1] = out[1];
    verts[3 * v + 2] = out[2];
  }
}

__device__ __forceinline__ float warp_sum(float x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// accumulator layout: [j*12 + 0..8] dRA_j (row-major), [j*12 + 9..11] dtA_j,
// [16*12 + k] dbeta_k (blendshape part), [16*12 + 10 + c] dtau_c.
// blockIdx.y selects the instance: params / dparams [61], dverts [V][3], partials
// [kSkinBlocks][kSkinAcc] and the last-block counter at counter_all + y * cstride;
// djoints_all (optional, [J][3] per instance) is dL/d(posed joints).
__global__ void __launch_bounds__(kSkinThreads) k_skin_bwd(ModelArgs m, const float* __restrict__ params_all,
                                                           const float* __restrict__ dverts_all,
                                                           const float* __restrict__ djoints_all,
                                                           float* __restrict__ partials_all, unsigned* counter_all,
                                                           int cstride, float* __restrict__ dparams_all,
                                                           int* status) {
  __shared__ Chain ch;
  const float* params = params_all + (size_t)blockIdx.y * 61;
  const float* dverts = dverts_all + (size_t)blockIdx.y * 3 * m.V;
  float* partials = partials_all + (size_t)blockIdx.y * kSkinBlocks * kSkinAcc;
  unsigned* counter = counter_all + (size_t)blockIdx.y * cstride;
  float* dparams = dparams_all + (size_t)blockIdx.y * 61;
  __shared__ float wacc[kSkinThreads / 32][kSkinAcc];
  __shared__ float bacc[kSkinAcc];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = lane; i < kSkinAcc; i += 32) wacc[warp][i] = 0.0f;
  build_chain(m, params, ch, status);
  const int nv_iter = (m.V + gridDim.x * blockDim.x - 1) / (gridDim.x * blockDim.x);
  for (int it = 0; it < nv_iter; ++it) {
    int v = (it * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    bool ok = v < m.V;
    float3 g = ok ? ld3(dverts + 3 * v) : make_float3(0.0f, 0.0f, 0.0f);
    float3 p = ok ? shaped_vertex(m, ch, v) : make_float3(0.0f, 0.0f, 0.0f);
    const float* w = m.weights + (size_t)(ok ? v : 0) * m.J;
    float dvt[3] = {0.0f, 0.0f, 0.0f};
    for (int j = 0; j < kMaxJ; ++j) {
      float wj = (ok && j < m.J) ? w[j] : 0.0f;
      float gw[3] = {wj * g.x, wj * g.y, wj * g.z};
      float pv[3] = {p.x, p.y, p.z};
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
          float s = warp_sum(gw[a] * pv[b]);
          if (lane == 0) wacc[warp][12 * j + 3 * a + b] += s;
        }
        float s = warp_sum(gw[a]);
        if (lane == 0) wacc[warp][12 * j + 9 + a] += s;
      }
      if (j < m.J)
        for (int b = 0; b < 3; ++b) dvt[b] += ch.RA[j][b] * gw[0] + ch.RA[j][3 + b] * gw[1] + ch.RA[j][6 + b] * gw[2];
    }
    for (int k = 0; k < kMaxK; ++k) {
      float s = 0.0f;
      if (ok && k < m.K)
        for (int c = 0; c < 3; ++c) s += m.shapedirs[(size_t)(3 * v + c) * m.K + k] * dvt[c];
      s = warp_sum(s);
      if (lane == 0) wacc[warp][16 * 12 + k] += s;
    }
    float gt[3] = {g.x, g.y, g.z};
    for (int c = 0; c < 3; ++c) {
      float s = warp_sum(gt[c]);
      if (lane == 0) wacc[warp][16 * 12 + 10 + c] += s;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSkinAcc; i += blockDim.x) {
    float s = 0.0f;
    for (int q = 0; q < kSkinThreads / 32; ++q) s += wacc[q][i];
    partials[(size_t)blockIdx.x * kSkinAcc + i] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = threadIdx.x; i < kSkinAcc; i += blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(&partials[(size_t)b * kSkinAcc + i]);
    bacc[i] = s;
  }
  __syncthreads();
  // chain backward: one thread walks children before parents; the per-joint
  // Rodrigues gradients and the shape gradient then run in parallel
  __shared__ float sdRl[kMaxJ][9];
  __shared__ float sdJ[kMaxJ][3];
  if (threadIdx.x == 0) {
    *counter = 0u;
    float dRG[kMaxJ][9], dtG[kMaxJ][3];
    const float* djoints = djoints_all ? djoints_all + (size_t)blockIdx.y * 3 * m.J : nullptr;
    for (int j = 0; j < m.J; ++j) {
      const float* dRA = &bacc[12 * j];
      const float* dtA = &bacc[12 * j + 9];
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) dRG[j][3 * a + b] = dRA[3 * a + b] - dtA[a] * ch.J[j][b];
        dtG[j][a] = dtA[a] + (djoints ? djoints[3 * j + a] : 0.0f);
        sdJ[j][a] = -(ch.RG[j][a] * dtA[0] + ch.RG[j][3 + a] * dtA[1] + ch.RG[j][6 + a] * dtA[2]);
      }
    }
    for (int j = m.J - 1; j >= 0; --j) {
      int p = m.parents[j];
      if (p >= j || p < -1 || (j == 0) != (p < 0)) p = j == 0 ? -1 : 0;   // reported by build_chain
      if (p < 0) {
        for (int i = 0; i < 9; ++i) sdRl[j][i] = dRG[j][i];
        for (int a = 0; a < 3; ++a) sdJ[j][a] += dtG[j][a];
        continue;
      }
      const float* Rp = ch.RG[p];
      // dRl_j = Rp^T dRG_j
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          sdRl[j][3 * a + b] = Rp[a] * dRG[j][b] + Rp[3 + a] * dRG[j][3 + b] + Rp[6 + a] * dRG[j][6 + b];
      // dRG_p += dRG_j Rl_j^T + dtG_j (J_j - J_p)^T
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          dRG[p][3 * a + b] += dRG[j][3 * a] * ch.Rl[j][3 * b] + dRG[j][3 * a + 1] * ch.Rl[j][3 * b + 1] +
                               dRG[j][3 * a + 2] * ch.Rl[j][3 * b + 2] + dtG[j][a] * (ch.J[j][b] - ch.J[p][b]);
      for (int a = 0; a < 3; ++a) {
        float rt = Rp[a] * dtG[j][0] + Rp[3 + a] * dtG[j][1] + Rp[6 + a] * dtG[j][2];
        dtG[p][a] += dtG[j][a];
        sdJ[j][a] += rt;
        sdJ[p][a] -= rt;
      }
    }
  }
  __syncthreads();
  const int tid = threadIdx.x;
  if (tid < m.J) {
    const int j = tid;
    const float* r = (j == 0) ? params + 55 : params + 10 + 3 * (j - 1);
    float rr[3] = {r[0], r[1], r[2]}, out[3];
    rodrigues_grad(rr, sdRl[j], out);
    float* dst = (j == 0) ? dparams + 55 : dparams + 10 + 3 * (j - 1);
    for (int c = 0; c < 3; ++c) dst[c] = out[c];
  } else if (tid >= 32 && tid < 32 + m.K) {
    const int k = tid - 32;
    float s = bacc[16 * 12 + k];
    for (int j = 0; j < m.J; ++j)
      for (int c = 0; c < 3; ++c) s += m.j_shapedirs[(3 * j + c) * m.K + k] * sdJ[j][c];
    dparams[k] = s;
  } else if (tid >= 64 && tid < 67) {
    const int c = tid - 64;
    float dt = bacc[16 * 12 + 10 + c];
    if (djoints_all)
      for (int j = 0; j < m.J; ++j) dt += djoints_all[((size_t)blockIdx.y * m.J + j) * 3 + c];
    dparams[58 + c] = dt;
  }
}

ModelArgs model_args(const hr_model* m) {
  ModelArgs a;
  a.v_template = m->v_template;
  a.shapedirs = m->shapedirs;
  a.weights = m->weights;
  a.j_template = m->j_template;
  a.j_shapedirs = m->j_shapedirs;
  a.parents = m->parents;
  a.V = m->V;
  a.J = m->J;
  a.K = m->K;
  return a;
}

}  // namespace

int launch_skin(Context* ctx, const hr_model* m, const float* params, float* verts, float* joints, cudaStream_t s) {
  int blocks = (m->V + kSkinThreads - 1) / kSkinThreads;
  k_skin<<<dim3(blocks, ctx->n_inst), kSkinThreads, 0, s>>>(model_args(m), params, verts, joints, ctx->status);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_skin_bwd(Context* ctx, const hr_model* m, const float* params, const float* d_verts,
                    const float* d_joints, float* d_params, cudaStream_t s) {
  int blocks = (m->V + kSkinThreads - 1) / kSkinThreads;
  if (blocks > kSkinBlocks) blocks = kSkinBlocks;
  k_skin_bwd<<<dim3(blocks, ctx->n_inst), kSkinThreads, 0, s>>>(model_args(m), params, d_verts, d_joints,
                                                                ctx->skin_partials, ctx->counters + 2, 4, d_params,
                                                                ctx->status);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

}  // namespace hr

// ---------------------------------------------------------------------------------
// Allocation-free skinning adjoint.
//
// Some callers cannot let a library allocate device memory: host applications that
// hand every byte of device memory out of their own pool and forbid side
// allocations, processes running under a fixed device-memory quota, and
// latency-bound loops that cannot afford the implicit device synchronisation of
// cudaMalloc.  hr_skin_bwd_noalloc computes exactly what hr_skin_bwd computes, with
// the same kernel, but its reduction scratch (one partial per block, the
// last-block counter and a status word) lives in the file-scope array below, which
// every GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------------
namespace hr {
namespace {

constexpr int kNoAllocMaxV = kSkinBlocks * kSkinThreads;   // 16384 vertices
constexpr size_t kNoAllocPartialBytes = sizeof(float) * kSkinBlocks * kSkinAcc;
constexpr size_t kNoAllocBytes = kNoAllocPartialBytes + 256;   // + counter and status word

static __device__ __align__(256) unsigned char g_skin_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// device address of the scratch array on the current device (looked up once per
// device; the host-side symbol is only a stand-in and must never reach a kernel)
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return HR_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_skin_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HR_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return HR_OK;
}

}  // namespace
}  // namespace hr

extern "C" int hr_skin_bwd_noalloc(const hr_model* m, const float* params, const float* d_verts, float* d_params,
                                   hr_stream stream) {
  using namespace hr;
  if (!m || !params || !d_verts || !d_params) return HR_ERR_ARG;
  if (m->V <= 0 || m->J <= 0 || m->K < 0 || !m->v_template || !m->shapedirs || !m->weights || !m->j_template ||
      !m->j_shapedirs || !m->parents)
    return HR_ERR_ARG;
  if (m->V > kNoAllocMaxV || m->J > kMaxJ || m->K > kMaxK) return HR_ERR_UNSUPPORTED;
  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != HR_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  float* partials = reinterpret_cast<float*>(b);
  unsigned* counter = reinterpret_cast<unsigned*>(b + kNoAllocPartialBytes);
  int* status = reinterpret_cast<int*>(b + kNoAllocPartialBytes + 128);
  cudaStream_t s = (cudaStream_t)stream;
  // the last-block counter must start at zero; the rest is overwritten by the call
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  int blocks = (m->V + kSkinThreads - 1) / kSkinThreads;
  k_skin_bwd<<<blocks, kSkinThreads, 0, s>>>(model_args(m), params, d_verts, nullptr, partials, counter, 0, d_params,
                                             status);
  HR_CHECK_LAUNCH();
  return HR_OK;
}
