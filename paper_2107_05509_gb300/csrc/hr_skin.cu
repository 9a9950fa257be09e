// Skinning G_v (Section 3.1, "Geometry": the 61 hand parameters decoded into
// vertices) as linear blend skinning, and its adjoint.
//
//   k_skin      every block first builds the J joint transforms in shared memory
//               (Rodrigues per joint in parallel, then the kinematic tree composed
//               level by level, parents before children), then each thread blends
//               one vertex.
//   k_skin_bwd  per vertex the gradients w.r.t. the blended transforms A_j, the
//               shape coefficients (through the blendshapes) and the translation:
//               the block stages its vertices' terms in shared memory and one
//               thread per output sums them in vertex order (no atomics), blocks
//               write one partial each, and the last block to finish sums the
//               partials in block order and runs the chain backward level by level
//               (children before parents).  Fully deterministic.
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
  int par[kMaxJ];       // checked parent of each joint (-1 for the root)
  int depth[kMaxJ];     // level of each joint in the kinematic tree (root 0)
  int levels;           // 1 + the deepest level
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

// joint j's parent as the chain uses it: parents must precede children and only joint
// 0 is a root; a parent that breaks this is taken as joint 0 (as -1 for joint 0) and
// reported (report = true) in the status word
__device__ __forceinline__ int chain_parent(const ModelArgs& m, int j, int* status, bool report) {
  int p = m.parents[j];
  if (p >= j || p < -1 || (j == 0) != (p < 0)) {
    if (report) set_status(status, kStatusBadModel);
    p = j == 0 ? -1 : 0;
  }
  return p;
}

// the forward kinematic chain into shared memory, called by every thread of the
// block: per-joint work (shaped joint, local rotation) in parallel, then the
// composition level by level of the kinematic tree (thread j composes joint j once
// its parent, one level up, is done; one barrier per level, the same arithmetic per
// joint as a parents-first walk)
__device__ void build_chain(const ModelArgs& m, const float* __restrict__ params, Chain& ch, int* status) {
  const int tid = threadIdx.x;
  if (tid < 61 && !isfinite(params[tid])) set_status(status, kStatusNonfinite);
  if (tid < m.K) ch.beta[tid] = params[tid];
  if (tid < 3) ch.tau[tid] = params[58 + tid];
  if (tid < m.J) {   // depth of joint j (a chain of checked parents ends within j steps)
    const int p = chain_parent(m, tid, status, true);
    int d = 0;
    for (int q = p; q >= 0; q = chain_parent(m, q, status, false)) ++d;
    ch.par[tid] = p;
    ch.depth[tid] = d;
  }
  __syncthreads();
  if (tid < 3 * m.J) {
    const int j = tid / 3, c = tid % 3;
    const float* row = m.j_shapedirs + (3 * j + c) * m.K;
    float Sj[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) Sj[k] = k < m.K ? __ldg(row + k) : 0.0f;
    float acc = __ldg(m.j_template + 3 * j + c);
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
      if (k < m.K) acc += Sj[k] * ch.beta[k];
    ch.J[j][c] = acc;
  }
  if (tid >= 64 && tid < 64 + m.J) {
    const int j = tid - 64;
    const float* r = (j == 0) ? params + 55 : params + 10 + 3 * (j - 1);
    float rr[3] = {r[0], r[1], r[2]};
    rodrigues(rr, ch.Rl[j]);
  }
  if (tid == 0) {
    int d = 0;
    for (int j = 0; j < m.J; ++j) d = max(d, ch.depth[j]);
    ch.levels = d + 1;
  }
  __syncthreads();
  const int levels = ch.levels;
  for (int L = 0; L < levels; ++L) {
    if (tid < m.J && ch.depth[tid] == L) {
      const int j = tid, p = ch.par[j];
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
    __syncthreads();
  }
}

// vertex v's rows of the blendshape basis, S[c][k] = shapedirs[3v + c][k] (zero for
// k >= K) and its skinning weights wv[j] (zero for j >= J): loaded up front so that
// the loads are in flight together (loops over the run-time K and J issue them one
// round trip at a time)
__device__ __forceinline__ void load_vertex_rows(const ModelArgs& m, int v, float (&S)[3][kMaxK], float (&wv)[kMaxJ]) {
  const float* row = m.shapedirs + (size_t)3 * v * m.K;
  const float* w = m.weights + (size_t)v * m.J;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) S[c][k] = k < m.K ? __ldg(row + c * m.K + k) : 0.0f;
#pragma unroll
  for (int j = 0; j < kMaxJ; ++j) wv[j] = j < m.J ? __ldg(w + j) : 0.0f;
}

// the shaped vertex: template + sum_k S[c][k] beta_k, summed in k order
__device__ __forceinline__ float3 shaped_vertex(const ModelArgs& m, const Chain& ch, int v, const float (&S)[3][kMaxK]) {
  float p[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float acc = __ldg(m.v_template + 3 * v + c);
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
      if (k < m.K) acc += S[c][k] * ch.beta[k];
    p[c] = acc;
  }
  return make_float3(p[0], p[1], p[2]);
}

// blockIdx.y selects the instance: params [61] and verts [V][3] of instance y; block 0
// also writes the posed joints G_J (each joint frame's origin plus the root
// translation, [J][3]) when `joints_all` is given
__global__ void __launch_bounds__(kSkinThreads) k_skin(ModelArgs m, const float* __restrict__ params_all,
                                                       float* __restrict__ verts_all, float* __restrict__ joints_all,
                                                       int* status, const int* __restrict__ active) {
  pdl_wait();
  __shared__ Chain ch;
  if (active && !active[blockIdx.y]) return;   // a retired instance of a batch
  const float* params = params_all + (size_t)blockIdx.y * 61;
  float* verts = verts_all + (size_t)blockIdx.y * 3 * m.V;
  build_chain(m, params, ch, status);
  if (joints_all && blockIdx.x == 0 && threadIdx.x < 3 * m.J) {
    const int j = threadIdx.x / 3, c = threadIdx.x % 3;
    joints_all[((size_t)blockIdx.y * m.J + j) * 3 + c] = ch.tG[j][c] + ch.tau[c];
  }
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < m.V; v += gridDim.x * blockDim.x) {
    float S[3][kMaxK], wv[kMaxJ];
    load_vertex_rows(m, v, S, wv);
    float3 p = shaped_vertex(m, ch, v, S);
    float out[3] = {ch.tau[0], ch.tau[1], ch.tau[2]};
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) {
      const float wj = wv[j];
      if (j >= m.J || wj == 0.0f) continue;
      for (int a = 0; a < 3; ++a)
        out[a] += wj * (ch.RA[j][3 * a] * p.x + ch.RA[j][3 * a + 1] * p.y + ch.RA[j][3 * a + 2] * p.z + ch.tA[j][a]);
    }
    verts[3 * v] = out[0];
    verts[3 * v + 1] = out[1];
    verts[3 * v + 2] = out[2];
  }
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
                                                           int* status, const int* __restrict__ active) {
  pdl_wait();
  __shared__ Chain ch;
  if (active && !active[blockIdx.y]) return;   // a retired instance of a batch
  const float* params = params_all + (size_t)blockIdx.y * 61;
  const float* dverts = dverts_all + (size_t)blockIdx.y * 3 * m.V;
  float* partials = partials_all + (size_t)blockIdx.y * kSkinBlocks * kSkinAcc;
  unsigned* counter = counter_all + (size_t)blockIdx.y * cstride;
  float* dparams = dparams_all + (size_t)blockIdx.y * 61;
  // per-vertex terms of the block's current vertices (rows padded against bank
  // conflicts): g_a p_b and g_a, the skinning weights, and dL/d(shaped vertex)
  __shared__ float sgp[kSkinThreads][13];
  __shared__ float sw[kSkinThreads][kMaxJ + 1];
  __shared__ float sy[kSkinThreads][kMaxK + 1];
  __shared__ float bacc[kSkinAcc];
  __shared__ bool last;
  build_chain(m, params, ch, status);
  // thread i < kSkinAcc owns output i: it sums the block's vertices in vertex order
  // (dRA_j[a][b] = sum_v w_vj g_va p_vb, dtA_j[a] = sum_v w_vj g_va, dbeta_k through
  // the blendshapes, dtau = sum_v g_v)
  float tot = 0.0f;
  const int nv_iter = (m.V + gridDim.x * blockDim.x - 1) / (gridDim.x * blockDim.x);
  for (int it = 0; it < nv_iter; ++it) {
    const int v0 = (it * gridDim.x + blockIdx.x) * blockDim.x;
    const int v = v0 + threadIdx.x;
    const bool ok = v < m.V;
    float S[3][kMaxK], wv[kMaxJ];
    load_vertex_rows(m, ok ? v : 0, S, wv);
    const float3 g = ok ? ld3(dverts + 3 * v) : make_float3(0.0f, 0.0f, 0.0f);
    const float3 p = ok ? shaped_vertex(m, ch, v, S) : make_float3(0.0f, 0.0f, 0.0f);
    // dL/d(shaped vertex) through the blend, then its blendshape terms
    float dvt[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) {
      const float wj = ok ? wv[j] : 0.0f;
      sw[threadIdx.x][j] = wj;
      if (j >= m.J) continue;
      const float gw[3] = {wj * g.x, wj * g.y, wj * g.z};
      for (int b = 0; b < 3; ++b) dvt[b] += ch.RA[j][b] * gw[0] + ch.RA[j][3 + b] * gw[1] + ch.RA[j][6 + b] * gw[2];
    }
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
      float y = 0.0f;
      if (ok)
        for (int c = 0; c < 3; ++c) y += S[c][k] * dvt[c];
      sy[threadIdx.x][k] = y;
    }
    const float gv[3] = {g.x, g.y, g.z}, pv[3] = {p.x, p.y, p.z};
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) sgp[threadIdx.x][3 * a + b] = gv[a] * pv[b];
      sgp[threadIdx.x][9 + a] = gv[a];
    }
    __syncthreads();
    const int nv = max(0, min((int)blockDim.x, m.V - v0));
    const int i = threadIdx.x;
    if (i < 16 * 12) {
      const int j = i / 12, c = i % 12;
      if (j < m.J)
#pragma unroll 4
        for (int u = 0; u < nv; ++u) tot += sw[u][j] * sgp[u][c];
    } else if (i < 16 * 12 + kMaxK) {
      const int k = i - 16 * 12;
      if (k < m.K)
#pragma unroll 4
        for (int u = 0; u < nv; ++u) tot += sy[u][k];
    } else if (i < kSkinAcc) {
      const int c = i - 16 * 12 - 10;
#pragma unroll 4
      for (int u = 0; u < nv; ++u) tot += sgp[u][9 + c];
    }
    __syncthreads();
  }
  if (threadIdx.x < kSkinAcc) partials[(size_t)blockIdx.x * kSkinAcc + threadIdx.x] = tot;
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
  // chain backward, level by level from the deepest: the thread of joint p takes its
  // children in descending order (each child's own children were done one level
  // deeper), so every sum gets its terms in the order of a children-before-parents
  // walk; the per-joint Rodrigues gradients and the shape gradient then run in
  // parallel
  __shared__ float sdRl[kMaxJ][9];
  __shared__ float sdJ[kMaxJ][3];
  __shared__ float sdRG[kMaxJ][9];
  __shared__ float sdtG[kMaxJ][3];
  const float* djoints = djoints_all ? djoints_all + (size_t)blockIdx.y * 3 * m.J : nullptr;
  if (threadIdx.x == 0) *counter = 0u;
  if (threadIdx.x < m.J) {
    const int j = threadIdx.x;
    const float* dRA = &bacc[12 * j];
    const float* dtA = &bacc[12 * j + 9];
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) sdRG[j][3 * a + b] = dRA[3 * a + b] - dtA[a] * ch.J[j][b];
      sdtG[j][a] = dtA[a] + (djoints ? djoints[3 * j + a] : 0.0f);
      sdJ[j][a] = -(ch.RG[j][a] * dtA[0] + ch.RG[j][3 + a] * dtA[1] + ch.RG[j][6 + a] * dtA[2]);
    }
  }
  __syncthreads();
  for (int L = ch.levels - 2; L >= 0; --L) {
    if (threadIdx.x < m.J && ch.depth[threadIdx.x] == L) {
      // joint p's sums stay in registers over its children (through shared memory
      // every access would wait on the one before)
      const int p = threadIdx.x;
      float Rp[9], gRp[9], gtp[3], gJp[3], Jp[3];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        Rp[i] = ch.RG[p][i];
        gRp[i] = sdRG[p][i];
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gtp[a] = sdtG[p][a];
        gJp[a] = sdJ[p][a];
        Jp[a] = ch.J[p][a];
      }
      for (int j = m.J - 1; j > p; --j) {
        if (ch.par[j] != p) continue;
        float gRj[9], Rlj[9], gtj[3], Jj[3], gJj[3];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          gRj[i] = sdRG[j][i];
          Rlj[i] = ch.Rl[j][i];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          gtj[a] = sdtG[j][a];
          Jj[a] = ch.J[j][a];
          gJj[a] = sdJ[j][a];
        }
        // dRl_j = Rp^T dRG_j
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) sdRl[j][3 * a + b] = Rp[a] * gRj[b] + Rp[3 + a] * gRj[3 + b] + Rp[6 + a] * gRj[6 + b];
        // dRG_p += dRG_j Rl_j^T + dtG_j (J_j - J_p)^T
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            gRp[3 * a + b] += gRj[3 * a] * Rlj[3 * b] + gRj[3 * a + 1] * Rlj[3 * b + 1] + gRj[3 * a + 2] * Rlj[3 * b + 2] +
                              gtj[a] * (Jj[b] - Jp[b]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float rt = Rp[a] * gtj[0] + Rp[3 + a] * gtj[1] + Rp[6 + a] * gtj[2];
          gtp[a] += gtj[a];
          gJj[a] += rt;
          gJp[a] -= rt;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) sdJ[j][a] = gJj[a];
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) sdRG[p][i] = gRp[i];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        sdtG[p][a] = gtp[a];
        sdJ[p][a] = gJp[a];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < m.J && ch.par[threadIdx.x] < 0) {   // the root
    const int j = threadIdx.x;
    for (int i = 0; i < 9; ++i) sdRl[j][i] = sdRG[j][i];
    for (int a = 0; a < 3; ++a) sdJ[j][a] += sdtG[j][a];
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
    float Sj[3 * kMaxJ];
#pragma unroll
    for (int q = 0; q < 3 * kMaxJ; ++q) Sj[q] = q < 3 * m.J ? __ldg(m.j_shapedirs + q * m.K + k) : 0.0f;
    float s = bacc[16 * 12 + k];
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j)
      if (j < m.J)
        for (int c = 0; c < 3; ++c) s += Sj[3 * j + c] * sdJ[j][c];
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
  launch_pdl(k_skin, dim3(blocks, ctx->n_inst), dim3(kSkinThreads), 0, s, model_args(m), params, verts, joints,
             ctx->status, (const int*)ctx->active);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_skin_bwd(Context* ctx, const hr_model* m, const float* params, const float* d_verts,
                    const float* d_joints, float* d_params, cudaStream_t s) {
  int blocks = (m->V + kSkinThreads - 1) / kSkinThreads;
  if (blocks > kSkinBlocks) blocks = kSkinBlocks;
  launch_pdl(k_skin_bwd, dim3(blocks, ctx->n_inst), dim3(kSkinThreads), 0, s, model_args(m), params, d_verts,
             d_joints, ctx->skin_partials, ctx->counters + 2, 4, d_params, ctx->status, (const int*)ctx->active);
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

// device address of the scratch array on the current device (the host-side symbol
// is only a stand-in and must never reach a kernel).  Looked up again on every call
// whose stream is not being captured, so a device reset (which reloads the module,
// possibly elsewhere) cannot leave a stale address; a call on a capturing stream
// takes the address of the device's last uncaptured call, or looks it up when there
// was none.
int noalloc_scratch(cudaStream_t s, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return HR_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev] || cap == cudaStreamCaptureStatusNone) {
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
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  int rc = noalloc_scratch(s, &base);
  if (rc != HR_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  float* partials = reinterpret_cast<float*>(b);
  unsigned* counter = reinterpret_cast<unsigned*>(b + kNoAllocPartialBytes);
  int* status = reinterpret_cast<int*>(b + kNoAllocPartialBytes + 128);
  // the last-block counter must start at zero; the rest is overwritten by the call
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  int blocks = (m->V + kSkinThreads - 1) / kSkinThreads;
  k_skin_bwd<<<blocks, kSkinThreads, 0, s>>>(model_args(m), params, d_verts, nullptr, partials, counter, 0, d_params,
                                             status, nullptr);
  HR_CHECK_LAUNCH();
  return HR_OK;
}
