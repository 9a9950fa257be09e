// Masked photometric loss (Eq. 3 with the D_c term of Eq. 4, summed over views)
// and its adjoint, plus the Adam update (Section 3.3).
//
//   k_mask_count    integer count of masked pixels; the last block to finish sums the
//                   per-block counts in block order and stores 1 / (3 sum M).
//   k_loss_adjoint  adjoint = M sign(R - O) / (3 sum M) and per-block partial sums of
//                   M |R - O|; the last block sums the partials in block order (in
//                   double) into the loss.  Both reductions are deterministic.
// The image is streamed as float4 (4 pixels = 3 float4 per thread) when its
// pointers are 16-byte aligned.  A batch reduces every instance separately (its own
// mean over its own masked pixels): grid row blockIdx.y is instance y, whose pixels
// are one contiguous range, with its own partials and last-block counters.
#include <algorithm>

#include "hr_internal.h"

namespace hr {

namespace {

constexpr int kLossThreads = 256;

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x, unsigned long long* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  unsigned long long s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

__device__ __forceinline__ float block_sum_f(float x, float* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  float s = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// pixel range of grid row blockIdx.y: the instance's from the batch table, else [0, P)
__device__ __forceinline__ void inst_range(const InstRec* it, long long P, long long& p0, long long& n) {
  if (it) {
    p0 = it[blockIdx.y].pix0;
    n = it[blockIdx.y].npix;
  } else {
    p0 = 0;
    n = P;
  }
}

// per-instance scratch (lstride floats): counts[blocks] (u64), partials[blocks],
// scale; counters [4] per instance: 0 mask count, 1 loss
__global__ void __launch_bounds__(kLossThreads) k_mask_count(const uint8_t* __restrict__ mask_all,
                                                             const InstRec* __restrict__ it, long long P,
                                                             float* __restrict__ scratch_all, int lstride,
                                                             unsigned* counters_all, const int* __restrict__ active) {
  pdl_wait();
  __shared__ unsigned long long red[32];
  __shared__ bool last;
  if (active && !active[blockIdx.y]) return;   // a retired instance of a batch
  long long p0, n;
  inst_range(it, P, p0, n);
  const uint8_t* mask = mask_all + p0;
  float* scratch = scratch_all + (size_t)blockIdx.y * lstride;
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(scratch);
  float* scale = scratch + 3 * gridDim.x;
  unsigned* counter = counters_all + 4 * blockIdx.y;
  unsigned long long c = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long head = 0;
  if ((reinterpret_cast<uintptr_t>(mask) & 15) == 0) {
    // 16 mask bytes per load; a byte is non-zero iff the high bit of
    // ((b & 0x7f) + 0x7f) | b is set
    const uint4* m16 = reinterpret_cast<const uint4*>(mask);
    const long long q = n / 16;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < q; i += stride) {
      const uint4 w = m16[i];
      const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) c += __popc((((ws[k] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | ws[k]) & 0x80808080u);
    }
    head = 16 * q;
  }
  for (long long i = head + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) c += mask[i] != 0;
  unsigned long long s = block_sum_u64(c, red);
  if (threadIdx.x == 0) {
    counts[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: each thread sums a strided set of block counts, then a fixed
  // pairing tree (integer sums, exact in any order anyway)
  unsigned long long part = 0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) part += __ldcg(&counts[b]);
  __syncthreads();
  unsigned long long tot = block_sum_u64(part, red);
  if (threadIdx.x != 0) return;
  scale[0] = tot > 0 ? (float)(1.0 / (3.0 * (double)tot)) : 0.0f;
  *counter = 0u;
}

__device__ __forceinline__ float sgn(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

__global__ void __launch_bounds__(kLossThreads) k_loss_adjoint(const float* __restrict__ image_all,
                                                               const float* __restrict__ obs_all,
                                                               const uint8_t* __restrict__ mask_all,
                                                               const InstRec* __restrict__ it, long long P,
                                                               float* __restrict__ scratch_all, int lstride,
                                                               unsigned* counters_all,
                                                               float* __restrict__ adjoint_all,
                                                               float* __restrict__ loss_all, bool vec,
                                                               const int* __restrict__ active) {
  pdl_wait();
  __shared__ float red[32];
  __shared__ bool last;
  if (active && !active[blockIdx.y]) return;   // a retired instance of a batch
  long long p0;
  inst_range(it, P, p0, P);
  const float* image = image_all + 3 * p0;
  const float* obs = obs_all + 3 * p0;
  const uint8_t* mask = mask_all + p0;
  float* adjoint = adjoint_all + 3 * p0;
  float* scratch = scratch_all + (size_t)blockIdx.y * lstride;
  float* partials = scratch + 2 * gridDim.x;
  const float sc = scratch[3 * gridDim.x];
  unsigned* counter = counters_all + 4 * blockIdx.y + 1;
  float* loss = loss_all + blockIdx.y;
  float acc = 0.0f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (vec) {
    // 4 pixels = 12 floats = 3 float4 per step
    const long long Q = P / 4;
    const float4* R4 = reinterpret_cast<const float4*>(image);
    const float4* O4 = reinterpret_cast<const float4*>(obs);
    float4* A4 = reinterpret_cast<float4*>(adjoint);
    const uchar4* M4 = reinterpret_cast<const uchar4*>(mask);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += stride) {
      uchar4 m4 = M4[q];
      float mk[4] = {m4.x ? 1.0f : 0.0f, m4.y ? 1.0f : 0.0f, m4.z ? 1.0f : 0.0f, m4.w ? 1.0f : 0.0f};
      float r[12], o[12], a[12];
      for (int k = 0; k < 3; ++k) {
        float4 rv = R4[3 * q + k], ov = O4[3 * q + k];
        r[4 * k] = rv.x; r[4 * k + 1] = rv.y; r[4 * k + 2] = rv.z; r[4 * k + 3] = rv.w;
        o[4 * k] = ov.x; o[4 * k + 1] = ov.y; o[4 * k + 2] = ov.z; o[4 * k + 3] = ov.w;
      }
      for (int e = 0; e < 12; ++e) {
        float m = mk[e / 3];
        float d = r[e] - o[e];
        a[e] = m * sgn(d) * sc;
        acc += m * fabsf(d);
      }
      for (int k = 0; k < 3; ++k) A4[3 * q + k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
    }
    for (long long p = 4 * Q + (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
      float m = mask[p] ? 1.0f : 0.0f;
      for (int c = 0; c < 3; ++c) {
        float d = image[3 * p + c] - obs[3 * p + c];
        adjoint[3 * p + c] = m * sgn(d) * sc;
        acc += m * fabsf(d);
      }
    }
  } else {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
      float m = mask[p] ? 1.0f : 0.0f;
      for (int c = 0; c < 3; ++c) {
        float d = image[3 * p + c] - obs[3 * p + c];
        adjoint[3 * p + c] = m * sgn(d) * sc;
        acc += m * fabsf(d);
      }
    }
  }
  float s = block_sum_f(acc, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: thread i sums partials i, i + blockDim, ... in order (double),
  // then a fixed pairing tree over the threads -- the same order on every call
  __shared__ double dred[kLossThreads];
  double part = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) part += (double)__ldcg(&partials[b]);
  dred[threadIdx.x] = part;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) dred[threadIdx.x] += dred[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  loss[0] = (float)(dred[0] * (double)sc);
  *counter = 0u;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.0f - b1) * gi;
  float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// one block: bias corrections from the device step counter, then the counter
// advances; entry i steps by lr * lr_scale[i % scale_len] when a scale is given
// Grid-stride over the entries.  A one-block launch also advances the counter; a
// multi-block launch leaves that to k_counter_advance, launched after it on the same
// stream (no block may advance it while another still reads it).
__global__ void k_adam_dev(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                           const float* __restrict__ lr_scale, int scale_len, uint32_t* __restrict__ iter_dev) {
  pdl_wait();
  const float step = (float)(*iter_dev + 1u);
  const float c1 = 1.0f - powf(b1, step), c2 = 1.0f - powf(b2, step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float li = lr_scale ? lr * lr_scale[i % scale_len] : lr;
    p[i] -= li * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
  if (gridDim.x == 1) {
    __syncthreads();
    if (threadIdx.x == 0) *iter_dev += 1u;
  }
}

__global__ void k_counter_advance(uint32_t* iter_dev) { *iter_dev += 1u; }

// retire an instance of a batch: it is skipped from now on, and the Adam step sizes
// of its `per` parameters are zeroed so that its estimate stays where it is
__device__ __forceinline__ void retire(int i, int* active, float* lr_scale, int per) {
  active[i] = 0;
  if (lr_scale)
    for (int j = 0; j < per; ++j) lr_scale[(size_t)i * per + j] = 0.0f;
}

// instances whose error in the current row (err[*iter_dev][i]) is at most `thr`
__global__ void k_retire_converged(const float* __restrict__ err, const uint32_t* iter_dev, int rows, int n,
                                   float thr, int* __restrict__ active, float* __restrict__ lr_scale, int per) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !active[i]) return;
  const unsigned row = iter_dev ? *iter_dev : 0u;
  if (row >= (unsigned)rows) return;
  const float e = err[(size_t)row * n + i];
  if (e <= thr) retire(i, active, lr_scale, per);
}

// instances whose loss has not fallen below (1 - rel_tol) x its best for `patience`
// calls in a row
__global__ void k_retire_plateau(const float* __restrict__ loss, int n, float rel_tol, int patience,
                                 float* __restrict__ best, int* __restrict__ stall, int* __restrict__ active,
                                 float* __restrict__ lr_scale, int per) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !active[i]) return;
  const float l = loss[i];
  if (l < best[i] * (1.0f - rel_tol)) {
    best[i] = l;
    stall[i] = 0;
  } else if (++stall[i] >= patience) {
    retire(i, active, lr_scale, per);
  }
}

// epsilon_v of instance blockIdx.x: mean over vertices of |verts - ref| (metres),
// summed in a fixed order, into out[row][instance] with row = *iter_dev (row 0 when
// no counter is given); rows past the table are not written
constexpr int kErrThreads = 256;
__global__ void __launch_bounds__(kErrThreads) k_vertex_error(const float* __restrict__ verts,
                                                             const float* __restrict__ ref, int V,
                                                             float* __restrict__ out, const uint32_t* iter_dev,
                                                             int rows) {
  __shared__ double red[kErrThreads];
  const size_t o = (size_t)blockIdx.x * 3 * V;
  double acc = 0.0;
  for (int v = threadIdx.x; v < V; v += kErrThreads) {
    const double dx = (double)verts[o + 3 * v] - ref[o + 3 * v];
    const double dy = (double)verts[o + 3 * v + 1] - ref[o + 3 * v + 1];
    const double dz = (double)verts[o + 3 * v + 2] - ref[o + 3 * v + 2];
    acc += sqrt(dx * dx + dy * dy + dz * dz);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kErrThreads >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const unsigned row = iter_dev ? *iter_dev : 0u;
  if (row < (unsigned)rows) out[(size_t)row * gridDim.x + blockIdx.x] = (float)(red[0] / V);
}

// training loss of the proposal network: per instance (block) the mean squared
// vertex distance L_i = (1/V) sum_v |a - b|^2 (fixed-order sum), and the gradient of
// (1/n) sum_i L_i with respect to a
__global__ void __launch_bounds__(kErrThreads) k_vertex_mse(const float* __restrict__ a, const float* __restrict__ b,
                                                           int V, float* __restrict__ loss,
                                                           float* __restrict__ grad) {
  __shared__ double red[kErrThreads];
  const size_t o = (size_t)blockIdx.x * 3 * V;
  const float sc = 2.0f / ((float)V * (float)gridDim.x);
  double acc = 0.0;
  for (int i = threadIdx.x; i < 3 * V; i += kErrThreads) {
    const float d = a[o + i] - b[o + i];
    acc += (double)d * d;
    if (grad) grad[o + i] = sc * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kErrThreads >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[blockIdx.x] = (float)(red[0] / V);
}

// image[i] += sigma * N(0, 1): Philox4x32-10 keyed by seed, counter (i / 4, 0, 0, 0),
// two Box-Muller pairs per counter
__global__ void k_add_noise(float* __restrict__ img, long long n, float sigma, uint2 key) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * t >= n) return;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0u, 0u), key);
  const float u[4] = {((r.x >> 8) + 1) * 5.9604644775390625e-08f, (r.y >> 8) * 5.9604644775390625e-08f,
                      ((r.z >> 8) + 1) * 5.9604644775390625e-08f, (r.w >> 8) * 5.9604644775390625e-08f};
  float z[4];
  for (int k = 0; k < 2; ++k) {
    const float rad = sqrtf(-2.0f * logf(u[2 * k]));
    float sn, cs;
    sincospif(2.0f * u[2 * k + 1], &sn, &cs);
    z[2 * k] = rad * cs;
    z[2 * k + 1] = rad * sn;
  }
  for (int k = 0; k < 4 && 4 * t + k < n; ++k) img[4 * t + k] += sigma * z[k];
}

// per instance, the candidate with the lowest loss (the earliest on ties) of K
// candidates: out[i] = cand[k*][i], losses [K][n], cand [K][n][61]
__global__ void k_select_best(const float* __restrict__ cand, const float* __restrict__ losses, int K, int n,
                              float* __restrict__ out, int* __restrict__ chosen) {
  const int i = blockIdx.x;
  if (i >= n) return;
  int best = 0;
  float bl = losses[i];
  for (int k = 1; k < K; ++k) {
    const float l = losses[(size_t)k * n + i];
    if (l < bl) {
      bl = l;
      best = k;
    }
  }
  for (int j = threadIdx.x; j < 61; j += blockDim.x) out[(size_t)i * 61 + j] = cand[((size_t)best * n + i) * 61 + j];
  if (chosen && threadIdx.x == 0) chosen[i] = best;
}

// Colour-transformed loss (Eq. 2: the rendering of camera i enters the comparison as
// T_i R): per view, blocks over the view's pixels compute d = T R - O, the adjoint
// with respect to R, A = T^T (M sign(d) scale), and partial sums of M |d| and of
// dL/dT = (M sign(d) scale) R^T; a final block adds the partials in a fixed order.
constexpr int kCtBlocks = 64;
constexpr int kCtVals = 10;   // |d| sum, dT (9)
__global__ void __launch_bounds__(kLossThreads) k_loss_ct(const float* __restrict__ image,
                                                          const float* __restrict__ obs,
                                                          const uint8_t* __restrict__ mask,
                                                          const float* __restrict__ T, long long HW,
                                                          const float* __restrict__ scale_p,
                                                          float* __restrict__ adjoint,
                                                          float* __restrict__ part) {
  __shared__ float red[kCtVals][kLossThreads / 32];
  const int view = blockIdx.y;
  const float sc = scale_p[0];
  float t[9] = {1.0f, 0.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f, 0.0f, 1.0f};
  if (T)
    for (int k = 0; k < 9; ++k) t[k] = T[view * 9 + k];
  float acc[kCtVals] = {};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < HW; q += (long long)gridDim.x * blockDim.x) {
    const long long p = view * HW + q;
    const float m = mask[p] ? 1.0f : 0.0f;
    const float r[3] = {image[3 * p], image[3 * p + 1], image[3 * p + 2]};
    float sg[3];
    for (int c = 0; c < 3; ++c) {
      // the sign of d decides the adjoint: float32 with a fixed operation order
      const float tr = __fmaf_rn(t[3 * c + 2], r[2], __fmaf_rn(t[3 * c + 1], r[1], __fmul_rn(t[3 * c], r[0])));
      const float d = __fsub_rn(tr, obs[3 * p + c]);
      acc[0] += m * fabsf(d);
      sg[c] = m * sgn(d) * sc;
    }
    for (int c = 0; c < 3; ++c) {
      adjoint[3 * p + c] = t[c] * sg[0] + t[3 + c] * sg[1] + t[6 + c] * sg[2];
      for (int k = 0; k < 3; ++k) acc[1 + 3 * c + k] += sg[c] * r[k];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < kCtVals; ++k) {
    float x = acc[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < kCtVals) {
    float x = 0.0f;
    for (int w = 0; w < kLossThreads / 32; ++w) x += red[threadIdx.x][w];
    part[((size_t)view * gridDim.x + blockIdx.x) * kCtVals + threadIdx.x] = x;
  }
}

// loss = scale sum_views sum_blocks |d| (double, fixed order); dT[view] = its partials
__global__ void k_loss_ct_final(const float* __restrict__ part, int N, int nb, const float* __restrict__ scale_p,
                                float* __restrict__ loss, float* __restrict__ dT) {
  if (threadIdx.x < 9 * N && dT) {
    const int view = threadIdx.x / 9, k = threadIdx.x % 9;
    float x = 0.0f;
    for (int b = 0; b < nb; ++b) x += part[((size_t)view * nb + b) * kCtVals + 1 + k];
    dT[view * 9 + k] = x;
  }
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int v = 0; v < N; ++v)
      for (int b = 0; b < nb; ++b) tot += part[((size_t)v * nb + b) * kCtVals];
    loss[0] = (float)(tot * (double)scale_p[0]);
  }
}

// E_2 (the prior term), per instance (block): weight * sum over joints and
// coordinates of the smooth L1 f_2 between the target joints x and the model's joints
// y (0.5 d^2 / gamma for |d| < gamma, |d| - gamma / 2 beyond, d = y - x), and dE_2/dy
__global__ void k_joint_prior(const float* __restrict__ joints, const float* __restrict__ target, int J,
                              float gamma, float weight, float* __restrict__ loss, float* __restrict__ d_joints) {
  __shared__ double red[1024];
  const size_t o = (size_t)blockIdx.x * 3 * J;
  double f = 0.0;
  for (int i = threadIdx.x; i < 3 * J; i += blockDim.x) {
    const float d = joints[o + i] - target[o + i];
    const float a = fabsf(d);
    const bool quad = a < gamma;
    f += quad ? 0.5 * (double)d * d / gamma : (double)a - 0.5 * gamma;
    if (d_joints) d_joints[o + i] = weight * (quad ? d / gamma : (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f)));
  }
  red[threadIdx.x] = f;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[blockIdx.x] = (float)(weight * red[0]);
}

// V(c) = V_low scaled up by nearest neighbour + V_high (the two-level colour map)
__global__ void k_colour_map(const float* __restrict__ v_low, int wl, int hl, const float* __restrict__ v_high, int W,
                             int H, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)W * H * 3) return;
  const int c = (int)(i % 3);
  const long long p = i / 3;
  const int x = (int)(p % W), y = (int)(p / W);
  const int xl = x / (W / wl), yl = y / (H / hl);
  out[i] = v_low[((size_t)yl * wl + xl) * 3 + c] + v_high[i];
}

// dL/dV_low: the sum of dL/dV over each low texel's block (one block of threads per
// low texel and channel; strided sums added in a fixed tree order)
__global__ void __launch_bounds__(256) k_colour_low_grad(const float* __restrict__ d_v, int W, int H, int wl, int hl,
                                                         float* __restrict__ d_low) {
  __shared__ float red[256];
  const int c = blockIdx.y, xl = blockIdx.x % wl, yl = blockIdx.x / wl;
  const int bw = W / wl, bh = H / hl;
  float acc = 0.0f;
  for (int k = threadIdx.x; k < bw * bh; k += blockDim.x) {
    const int x = xl * bw + k % bw, y = yl * bh + k / bw;
    acc += d_v[((size_t)y * W + x) * 3 + c];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) d_low[((size_t)yl * wl + xl) * 3 + c] = red[0];
}

}  // namespace

int launch_adam_dev(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                    const float* lr_scale, int scale_len, uint32_t* iter_dev, cudaStream_t s) {
  // one block up to 16 entries per thread (the pose vector of one or a few
  // instances), else enough blocks to stream the five arrays at memory speed
  constexpr int kThreads = 256;
  const int blocks = n <= 16 * kThreads ? 1 : (int)std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 8);
  launch_pdl(k_adam_dev, dim3(blocks), dim3(kThreads), 0, s, p, g, m, v, n, lr, b1, b2, eps, lr_scale, scale_len,
             iter_dev);
  HR_CHECK_LAUNCH();
  if (blocks > 1) {
    k_counter_advance<<<1, 1, 0, s>>>(iter_dev);
    HR_CHECK_LAUNCH();
  }
  return HR_OK;
}

int launch_retire_converged(const float* err, const uint32_t* iter_dev, int rows, int n, float thr, int* active,
                            float* lr_scale, int per, cudaStream_t s) {
  k_retire_converged<<<(n + 127) / 128, 128, 0, s>>>(err, iter_dev, rows, n, thr, active, lr_scale, per);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_retire_plateau(const float* loss, int n, float rel_tol, int patience, float* best, int* stall, int* active,
                          float* lr_scale, int per, cudaStream_t s) {
  k_retire_plateau<<<(n + 127) / 128, 128, 0, s>>>(loss, n, rel_tol, patience, best, stall, active, lr_scale, per);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

// f x f box mean of [N][H][W][3] images (H, W multiples of f): one thread per output
// value; and the maximum of f x f blocks of [N][H][W] uint8 masks
__global__ void k_box_downsample(const float* __restrict__ src, long long n_out, int Ho, int Wo, int f,
                                 float* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  const int c = (int)(i % 3);
  const long long px = i / 3;
  const int x = (int)(px % Wo);
  const long long r = px / Wo;
  const int y = (int)(r % Ho);
  const long long v = r / Ho;
  const long long W = (long long)Wo * f, H = (long long)Ho * f;
  float acc = 0.0f;
  for (int dy = 0; dy < f; ++dy)
    for (int dx = 0; dx < f; ++dx) acc += src[((v * H + (long long)y * f + dy) * W + (long long)x * f + dx) * 3 + c];
  dst[i] = acc / (float)(f * f);
}

__global__ void k_mask_downsample(const uint8_t* __restrict__ src, long long n_out, int Ho, int Wo, int f,
                                  uint8_t* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  const int x = (int)(i % Wo);
  const long long r = i / Wo;
  const int y = (int)(r % Ho);
  const long long v = r / Ho;
  const long long W = (long long)Wo * f, H = (long long)Ho * f;
  uint8_t m = 0;
  for (int dy = 0; dy < f; ++dy)
    for (int dx = 0; dx < f; ++dx) m = max(m, src[(v * H + (long long)y * f + dy) * W + (long long)x * f + dx]);
  dst[i] = m;
}

// Area resampling of [N][H][W][3] images to [N][Ho][Wo][3] (any sizes): output pixel
// (x, y) covers input [x W / Wo, (x + 1) W / Wo) x [y H / Ho, (y + 1) H / Ho) and is
// the overlap-weighted mean of the input pixels there.  Measured in units of 1/Wo
// (1/Ho) of an input pixel the overlaps are integers, so the weights are exact; the
// sum runs over input rows, then columns, in increasing order.  The mask version takes
// the maximum over the input pixels with a positive overlap.
__device__ __forceinline__ long long area_overlap(long long o, long long n_in, long long n_out, long long k) {
  // [o n_in, (o + 1) n_in) against input pixel k's [k n_out, (k + 1) n_out)
  return min((o + 1) * n_in, (k + 1) * n_out) - max(o * n_in, k * n_out);
}

__global__ void k_area_resample(const float* __restrict__ src, long long n_out, int H, int W, int Ho, int Wo,
                                float* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  const int c = (int)(i % 3);
  const long long px = i / 3;
  const int x = (int)(px % Wo);
  const long long r = px / Wo;
  const int y = (int)(r % Ho);
  const long long v = r / Ho;
  const long long y_lo = (long long)y * H / Ho, x_lo = (long long)x * W / Wo;
  float acc = 0.0f;
  for (long long iy = y_lo; iy < H && iy * Ho < (long long)(y + 1) * H; ++iy) {
    const long long oy = area_overlap(y, H, Ho, iy);
    if (oy <= 0) continue;
    const float* row = src + ((v * H + iy) * W) * 3 + c;
    for (long long ix = x_lo; ix < W && ix * Wo < (long long)(x + 1) * W; ++ix) {
      const long long ox = area_overlap(x, W, Wo, ix);
      if (ox > 0) acc = fmaf((float)(oy * ox), row[ix * 3], acc);
    }
  }
  dst[i] = acc / ((float)H * (float)W);
}

__global__ void k_mask_resample(const uint8_t* __restrict__ src, long long n_out, int H, int W, int Ho, int Wo,
                                uint8_t* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  const int x = (int)(i % Wo);
  const long long r = i / Wo;
  const int y = (int)(r % Ho);
  const long long v = r / Ho;
  const long long y_lo = (long long)y * H / Ho, x_lo = (long long)x * W / Wo;
  uint8_t m = 0;
  for (long long iy = y_lo; iy < H && iy * Ho < (long long)(y + 1) * H; ++iy) {
    if (area_overlap(y, H, Ho, iy) <= 0) continue;
    for (long long ix = x_lo; ix < W && ix * Wo < (long long)(x + 1) * W; ++ix)
      if (area_overlap(x, W, Wo, ix) > 0) m = max(m, src[(v * H + iy) * W + ix]);
  }
  dst[i] = m;
}

int launch_area_resample(const float* src, int N, int H, int W, int Ho, int Wo, float* dst, cudaStream_t s) {
  const long long n = (long long)N * Ho * Wo * 3;
  k_area_resample<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, H, W, Ho, Wo, dst);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_mask_resample(const uint8_t* src, int N, int H, int W, int Ho, int Wo, uint8_t* dst, cudaStream_t s) {
  const long long n = (long long)N * Ho * Wo;
  k_mask_resample<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, H, W, Ho, Wo, dst);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_box_downsample(const float* src, int N, int H, int W, int f, float* dst, cudaStream_t s) {
  const long long n = (long long)N * (H / f) * (W / f) * 3;
  k_box_downsample<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, H / f, W / f, f, dst);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_mask_downsample(const uint8_t* src, int N, int H, int W, int f, uint8_t* dst, cudaStream_t s) {
  const long long n = (long long)N * (H / f) * (W / f);
  k_mask_downsample<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, H / f, W / f, f, dst);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_vertex_mse(const float* a, const float* b, int V, int n, float* loss, float* grad, cudaStream_t s) {
  k_vertex_mse<<<n, kErrThreads, 0, s>>>(a, b, V, loss, grad);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_add_noise(float* img, long long n, float sigma, uint64_t seed, cudaStream_t s) {
  const long long t = (n + 3) / 4;
  k_add_noise<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(img, n, sigma,
                                                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_select_best(const float* cand, const float* losses, int K, int n, float* out, int* chosen,
                       cudaStream_t s) {
  k_select_best<<<n, 64, 0, s>>>(cand, losses, K, n, out, chosen);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_joint_prior(const float* joints, const float* target, int J, int n, float gamma, float weight,
                       float* loss, float* d_joints, cudaStream_t s) {
  int threads = 32;
  while (threads < 3 * J && threads < 1024) threads <<= 1;
  k_joint_prior<<<n, threads, 0, s>>>(joints, target, J, gamma, weight, loss, d_joints);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_colour_map(const float* v_low, int wl, int hl, const float* v_high, int W, int H, float* out,
                      cudaStream_t s) {
  const long long n = (long long)W * H * 3;
  k_colour_map<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v_low, wl, hl, v_high, W, H, out);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_colour_map_bwd(const float* d_v, int W, int H, int wl, int hl, float* d_low, cudaStream_t s) {
  k_colour_low_grad<<<dim3(wl * hl, 3), 256, 0, s>>>(d_v, W, H, wl, hl, d_low);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_vertex_error(const float* verts, const float* ref, int V, int n, float* out, const uint32_t* iter_dev,
                        int rows, cudaStream_t s) {
  k_vertex_error<<<n, kErrThreads, 0, s>>>(verts, ref, V, out, iter_dev, rows);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_loss(Context* ctx, const float* image, const float* obs, const uint8_t* mask, long long P, float* loss,
                float* adjoint, cudaStream_t s) {
  int blocks;
  bool vec = ((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(obs) |
               reinterpret_cast<uintptr_t>(adjoint)) & 15) == 0 &&
             (reinterpret_cast<uintptr_t>(mask) & 3) == 0;
  if (ctx->vt) {   // a batch: every instance's range, its own reduction
    blocks = ctx->loss_blocks;
    vec = vec && ctx->loss_vec;
    P = 0;
  } else {
    long long want = (P + kLossThreads - 1) / kLossThreads;
    blocks = (int)(want < kLossBlocks ? (want > 0 ? want : 1) : kLossBlocks);
  }
  const int lstride = kLossStride(ctx->loss_blocks);
  const dim3 grid(blocks, ctx->vt ? ctx->n_inst : 1);
  const InstRec* it = ctx->vt ? ctx->it : nullptr;
  launch_pdl(k_mask_count, grid, dim3(kLossThreads), 0, s, mask, it, P, ctx->loss_partials, lstride, ctx->counters,
             (const int*)(ctx->vt ? ctx->active : nullptr));
  HR_CHECK_LAUNCH();
  launch_pdl(k_loss_adjoint, grid, dim3(kLossThreads), 0, s, image, obs, mask, it, P, ctx->loss_partials, lstride,
             ctx->counters, adjoint, loss, vec, (const int*)(ctx->vt ? ctx->active : nullptr));
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_loss_ct(Context* ctx, const float* image, const float* obs, const uint8_t* mask, const float* T, int N,
                   long long HW, float* loss, float* adjoint, float* dT, cudaStream_t s) {
  const long long P = (long long)N * HW;
  const long long want = (P + kLossThreads - 1) / kLossThreads;
  const int blocks = (int)(want < kLossBlocks ? (want > 0 ? want : 1) : kLossBlocks);
  float* scale = ctx->loss_partials + 3 * blocks;   // where k_mask_count leaves 1 / (3 sum M)
  k_mask_count<<<dim3(blocks, 1), kLossThreads, 0, s>>>(mask, nullptr, P, ctx->loss_partials, 0, ctx->counters,
                                                        nullptr);
  HR_CHECK_LAUNCH();
  k_loss_ct<<<dim3(kCtBlocks, N), kLossThreads, 0, s>>>(image, obs, mask, T, HW, scale, adjoint, ctx->ct_partials);
  HR_CHECK_LAUNCH();
  k_loss_ct_final<<<1, 32 * ((9 * N + 31) / 32 > 0 ? (9 * N + 31) / 32 : 1), 0, s>>>(ctx->ct_partials, N, kCtBlocks,
                                                                                     scale, loss, dT);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps, int step,
                cudaStream_t s) {
  float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(n + 127) / 128, 128, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

}  // namespace hr
