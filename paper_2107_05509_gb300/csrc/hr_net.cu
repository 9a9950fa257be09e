// The learned proposal network: from per-view residual images to a parameter update.
// (The paper refines by gradient descent alone; this network is an extension that
// proposes the first updates, with the plain method as the fallback and judge.)
//
// Architecture, per view v of instance b (B instances x nv views, NV = B nv):
//   X0  [128][128][8]  2x2-averaged render minus observation (3), observation (3), 0, 0
//   Y1..Y5             3x3 convolutions, stride 2, padding 1, ReLU:
//                      8->32 (64x64), 32->64 (32x32), 64->128 (16x16), 128->128 (8x8),
//                      128->128 (4x4)
//   Z   [2112]         Y5 flattened (2048) + camera rotation (9) + centre / 0.6 m (3) + 0
//   F   [256]          ReLU(Wv Z + bv), per view, shared weights
//   P   [256]          max over the instance's views (the first maximum on ties)
//   H   [256]          ReLU(W1 P + b1)
//   O   [61]           W2 H + b2;  delta = s * O with s the per-group scale
// Weights and activations are bf16, products accumulate in float32 on the tensor
// cores (hr_gemm.cu): a convolution is im2col + GEMM (cols [pixels][9 Cin padded to
// 64] x W [Cout][same]^T = the NHWC output), its weight gradient dPre^T cols (split
// over pixels), its input gradient dPre W followed by col2im (a gather, so every sum
// has a fixed order).  Master weights, gradients and the Adam moments are float32.
#include <cuda_bf16.h>

#include <cstring>
#include <new>

#include "hr_internal.h"

namespace hr {

namespace {

constexpr int kIn = 128, kC0 = 8;
constexpr int kConv = 5;
constexpr int kCin[kConv] = {8, 32, 64, 128, 128};
constexpr int kCout[kConv] = {32, 64, 128, 128, 128};
constexpr int kKp[kConv] = {128, 320, 576, 1152, 1152};   // 9 Cin rounded up to 64
constexpr int kHin[kConv] = {128, 64, 32, 16, 8};        // input side; output side = kHin / 2
constexpr int kFeat = 2048, kZ = 2112, kHid = 256, kOut = 61, kOutPad = 64;
constexpr int kSplitMax = 128;

// per-group output scales: shape, pose (rad), root rotation (rad), translation (m)
__constant__ float c_out_scale[4] = {0.5f, 0.1f, 0.1f, 0.005f};
__device__ __forceinline__ float out_scale(int j) {
  return j < 10 ? c_out_scale[0] : (j < 55 ? c_out_scale[1] : (j < 58 ? c_out_scale[2] : c_out_scale[3]));
}

__host__ __device__ constexpr int round64(int x) { return (x + 63) & ~63; }

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------------
// glue kernels
// ---------------------------------------------------------------------------------

// X0 of every view: 2x2 means of the 256x256 render R and observation O
__global__ void k_net_inputs(const float* __restrict__ R, const float* __restrict__ O, int NV, int W, int H,
                             bf16* __restrict__ X0) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)NV * kIn * kIn) return;
  const int v = (int)(i / (kIn * kIn)), p = (int)(i % (kIn * kIn)), y = p / kIn, x = p % kIn;
  float r[3] = {0.0f, 0.0f, 0.0f}, o[3] = {0.0f, 0.0f, 0.0f};
  for (int dy = 0; dy < 2; ++dy)
    for (int dx = 0; dx < 2; ++dx) {
      const size_t q = 3 * (((size_t)v * H + 2 * y + dy) * W + 2 * x + dx);
      for (int c = 0; c < 3; ++c) {
        r[c] += R[q + c];
        o[c] += O[q + c];
      }
    }
  bf16* out = X0 + i * kC0;
  for (int c = 0; c < 3; ++c) {
    out[c] = __float2bfloat16_rn(0.25f * (r[c] - o[c]));
    out[3 + c] = __float2bfloat16_rn(0.25f * o[c]);
  }
  out[6] = out[7] = __float2bfloat16_rn(0.0f);
}

// cols[(v, oy, ox)][(ky 3 + kx) Cin + c] = X[v][2 oy - 1 + ky][2 ox - 1 + kx][c] (0 outside),
// padded with zeros to Kp columns; transposed (colsT[k][row], pitch ldt) when T
template <bool T>
__global__ void k_im2col(const bf16* __restrict__ X, int NV, int Hin, int Cin, int Kp, bf16* __restrict__ out,
                         long long ldt) {
  const int Ho = Hin / 2;
  const long long rows = (long long)NV * Ho * Ho;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * Kp) return;
  long long row;
  int k;
  if (T) {   // consecutive threads along rows: coalesced stores of colsT
    k = (int)(i / rows);
    row = i % rows;
  } else {
    row = i / Kp;
    k = (int)(i % Kp);
  }
  bf16 val = __float2bfloat16_rn(0.0f);
  if (k < 9 * Cin) {
    const int tap = k / Cin, c = k % Cin, ky = tap / 3, kx = tap % 3;
    const int v = (int)(row / (Ho * Ho)), p = (int)(row % (Ho * Ho)), oy = p / Ho, ox = p % Ho;
    const int y = 2 * oy - 1 + ky, x = 2 * ox - 1 + kx;
    if (y >= 0 && y < Hin && x >= 0 && x < Hin) val = X[(((size_t)v * Hin + y) * Hin + x) * Cin + c];
  }
  if (T)
    out[(size_t)k * ldt + row] = val;
  else
    out[(size_t)row * Kp + k] = val;
}

// dX[v][y][x][c] = sum over the taps that read (y, x): dcols[(v, oy, ox)][(ky 3 + kx) Cin + c]
__global__ void k_col2im(const bf16* __restrict__ dcols, int NV, int Hin, int Cin, int Kp, bf16* __restrict__ dX) {
  const int Ho = Hin / 2;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)NV * Hin * Hin * Cin) return;
  const int c = (int)(i % Cin);
  const long long pix = i / Cin;
  const int v = (int)(pix / (Hin * Hin)), p = (int)(pix % (Hin * Hin)), y = p / Hin, x = p % Hin;
  float acc = 0.0f;
  for (int ky = 0; ky < 3; ++ky) {
    const int ty = y + 1 - ky;   // = 2 oy
    if (ty < 0 || (ty & 1) || ty / 2 >= Ho) continue;
    for (int kx = 0; kx < 3; ++kx) {
      const int tx = x + 1 - kx;
      if (tx < 0 || (tx & 1) || tx / 2 >= Ho) continue;
      const size_t row = ((size_t)v * Ho + ty / 2) * Ho + tx / 2;
      acc += __bfloat162float(dcols[row * Kp + (ky * 3 + kx) * Cin + c]);
    }
  }
  dX[i] = __float2bfloat16_rn(acc);
}

// out[c][r] = in[r][c] for r < rows, c < cols; columns [rows, ldo) of out are zero
__global__ void k_transpose(const bf16* __restrict__ in, long long rows, int cols, int ldi, bf16* __restrict__ out,
                            long long ldo) {
  __shared__ bf16 tile[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long long r = r0 + j;
    const int c = c0 + threadIdx.x;
    tile[j][threadIdx.x] = (r < rows && c < cols) ? in[r * ldi + c] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j;
    const long long r = r0 + threadIdx.x;
    if (c < cols && r < ldo) out[(size_t)c * ldo + r] = tile[threadIdx.x][j];
  }
}

// dPre = dY * (Y > 0), elementwise
__global__ void k_relu_grad(const bf16* __restrict__ dY, const bf16* __restrict__ Y, long long n,
                            bf16* __restrict__ dPre) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dPre[i] = __bfloat162float(Y[i]) > 0.0f ? dY[i] : __float2bfloat16_rn(0.0f);
}

// column sums of a [rows][cols] bf16 matrix (cols <= 256) into out[cols] (float32):
// block b takes a fixed slice of rows; warp w of the block sums rows w, w + 8, ... of
// the slice for 32 columns at a time; the warps' sums are added in warp order, and
// the last block to finish adds the block sums in block order
constexpr int kColBlocks = 128;
__global__ void __launch_bounds__(256) k_colsum(const bf16* __restrict__ in, long long rows, int cols,
                                                float* __restrict__ part, unsigned* counter, float* __restrict__ out) {
  __shared__ float red[8][32];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long per = (rows + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
  for (int c0 = 0; c0 < cols; c0 += 32) {
    const int c = c0 + lane;
    float acc = 0.0f;
    if (c < cols) {
#pragma unroll 4
      for (long long r = r0 + warp; r < r1; r += 8) acc += __bfloat162float(in[r * cols + c]);
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < cols) {
      float t = 0.0f;
      for (int w = 0; w < 8; ++w) t += red[w][lane];
      part[(size_t)blockIdx.x * cols + c] = t;
    }
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    float acc = 0.0f;
    for (int b = 0; b < (int)gridDim.x; ++b) acc += __ldcg(&part[(size_t)b * cols + c]);
    out[c] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// Z[v] = Y5[v] (2048) | camera R (9) | centre / 0.6 (3) | zeros
__global__ void k_features(const bf16* __restrict__ Y5, const float* __restrict__ cams, int NV, bf16* __restrict__ Z) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)NV * kZ) return;
  const int v = (int)(i / kZ), k = (int)(i % kZ);
  float val = 0.0f;
  if (k < kFeat) {
    Z[i] = Y5[(size_t)v * kFeat + k];
    return;
  }
  if (k < kFeat + 9)
    val = cams[v * 20 + 4 + (k - kFeat)];
  else if (k < kFeat + 12)
    val = cams[v * 20 + 16 + (k - kFeat - 9)] * (1.0f / 0.6f);
  Z[i] = __float2bfloat16_rn(val);
}

// P[b][c] = max_v F[b nv + v][c] (first maximum), idx = that v
__global__ void k_viewpool(const bf16* __restrict__ F, int B, int nv, bf16* __restrict__ P, int* __restrict__ idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * kHid) return;
  const int b = i / kHid, c = i % kHid;
  float best = -INFINITY;
  int bi = 0;
  for (int v = 0; v < nv; ++v) {
    const float x = __bfloat162float(F[((size_t)b * nv + v) * kHid + c]);
    if (x > best) {
      best = x;
      bi = v;
    }
  }
  P[i] = __float2bfloat16_rn(best);
  idx[i] = bi;
}

__global__ void k_viewpool_bwd(const bf16* __restrict__ dP, const int* __restrict__ idx, int B, int nv,
                               bf16* __restrict__ dF) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * nv * kHid) return;
  const int bv = i / kHid, c = i % kHid, b = bv / nv, v = bv % nv;
  dF[i] = idx[b * kHid + c] == v ? dP[b * kHid + c] : __float2bfloat16_rn(0.0f);
}

// out[b][j] = base[b][j] + s_j O[b][j] (base optional)
__global__ void k_net_out(const float* __restrict__ O, int B, const float* __restrict__ base, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * kOut) return;
  const int b = i / kOut, j = i % kOut;
  out[i] = (base ? base[i] : 0.0f) + out_scale(j) * O[(size_t)b * kOutPad + j];
}

// dO[b][j] = s_j d_out[b][j] (bf16, padded to 64 columns with zeros), and db2
__global__ void k_net_dout(const float* __restrict__ dout, int B, bf16* __restrict__ dO) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * kOutPad) return;
  const int b = i / kOutPad, j = i % kOutPad;
  dO[i] = __float2bfloat16_rn(j < kOut ? out_scale(j) * dout[b * kOut + j] : 0.0f);
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, long long n, bf16* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------------
// the network object
// ---------------------------------------------------------------------------------
struct Layer {   // a dense layer y = W x + b over K inputs (W [N][K], K a multiple of 64)
  int N, K;
  size_t w, b;   // offsets into the parameter vector
};

struct Net {
  int B, nv, NV;
  int Bp, NVp;   // batch and view counts rounded up to 64 (reduction dims of weight gradients)
  Layer conv[kConv], fv, f1, f2;
  size_t P;      // parameter count
  float *w32, *g32, *m, *v;
  bf16* w16;     // bf16 copy of the weights (same offsets)
  bf16* wT[kConv + 3];   // transposed weights [K][N] for the input gradients
  bf16* act[kConv + 1];  // X0, Y1..Y5 (NHWC)
  bf16 *Z, *F, *Pool, *H;
  int* pidx;
  float* O;
  bf16 *cols, *colsT, *dcols, *dA, *dB, *dPre, *dPreT;
  bf16 *dZ, *dF, *dP, *dH, *dO;
  float* split;
  float* colpart;
  unsigned* counter;
  int* status;
  size_t cols_elems;
};

Layer make_layer(int N, int K, size_t& off) {
  Layer l;
  l.N = N;
  l.K = K;
  l.w = off;
  off += (size_t)N * K;
  l.b = off;
  off += (size_t)N;
  return l;
}

void free_net(Net* n) {
  void* ptrs[] = {n->w32, n->g32,  n->m,    n->v,     n->w16,  n->Z,     n->F,      n->Pool, n->H,
                  n->pidx, n->O,   n->cols, n->colsT, n->dcols, n->dA,   n->dB,     n->dPre, n->dPreT,
                  n->dZ,  n->dF,   n->dP,   n->dH,    n->dO,   n->split, n->colpart, n->counter, n->status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < kConv + 3; ++i)
    if (n->wT[i]) cudaFree(n->wT[i]);
  for (int i = 0; i <= kConv; ++i)
    if (n->act[i]) cudaFree(n->act[i]);
  delete n;
}

template <class T>
bool nalloc(T** p, size_t count) {
  if (cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

int gemm(Net* n, const bf16* A, int lda, const bf16* Bm, int ldb, int M, int N, int K, const float* bias, int relu,
         void* C, int ldc, bool out_bf16, cudaStream_t s, int splits = 1) {
  return launch_gemm(A, lda, Bm, ldb, M, N, K, bias, relu, C, ldc, out_bf16 ? 1 : 0, splits, n->split, n->status, s);
}

// split count for a weight-gradient GEMM with a long reduction: about two CTAs per
// SM over the output tiles, each split at least 8 K-steps
int wgrad_splits(int M, int N, long long K) {
  const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
  int s = (2 * 152 + tiles - 1) / tiles;
  const long long ksteps = K / 64;
  while (s > 1 && ksteps / s < 8) --s;
  return s < 1 ? 1 : (s > kSplitMax ? kSplitMax : s);
}

// refresh the bf16 weights and their transposes from the float32 master copy
int refresh_weights(Net* n, cudaStream_t s) {
  k_f32_to_bf16<<<nblk((long long)n->P), 256, 0, s>>>(n->w32, (long long)n->P, n->w16);
  HR_CHECK_LAUNCH();
  const Layer* ls[kConv + 3] = {&n->conv[0], &n->conv[1], &n->conv[2], &n->conv[3], &n->conv[4],
                                &n->fv,      &n->f1,      &n->f2};
  for (int i = 1; i < kConv + 3; ++i) {   // layer 1 needs no input gradient
    const Layer& l = *ls[i];
    dim3 grid((unsigned)((l.N + 31) / 32), (unsigned)((l.K + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(n->w16 + l.w, l.N, l.K, l.K, n->wT[i], l.N);
    HR_CHECK_LAUNCH();
  }
  return HR_OK;
}

int net_forward(Net* n, const float* cams, cudaStream_t s) {
  int rc;
  for (int l = 0; l < kConv; ++l) {
    const int Hin = kHin[l], Ho = Hin / 2;
    const long long rows = (long long)n->NV * Ho * Ho;
    k_im2col<false><<<nblk(rows * kKp[l]), 256, 0, s>>>(n->act[l], n->NV, Hin, kCin[l], kKp[l], n->cols, 0);
    HR_CHECK_LAUNCH();
    const Layer& L = n->conv[l];
    if ((rc = gemm(n, n->cols, kKp[l], n->w16 + L.w, L.K, (int)rows, L.N, L.K, n->w32 + L.b, 1, n->act[l + 1], L.N,
                   true, s)) != HR_OK)
      return rc;
  }
  k_features<<<nblk((long long)n->NV * kZ), 256, 0, s>>>(n->act[kConv], cams, n->NV, n->Z);
  HR_CHECK_LAUNCH();
  if ((rc = gemm(n, n->Z, kZ, n->w16 + n->fv.w, kZ, n->NV, kHid, kZ, n->w32 + n->fv.b, 1, n->F, kHid, true, s)) !=
      HR_OK)
    return rc;
  k_viewpool<<<nblk(n->B * kHid), 256, 0, s>>>(n->F, n->B, n->nv, n->Pool, n->pidx);
  HR_CHECK_LAUNCH();
  if ((rc = gemm(n, n->Pool, kHid, n->w16 + n->f1.w, kHid, n->B, kHid, kHid, n->w32 + n->f1.b, 1, n->H, kHid, true,
                 s)) != HR_OK)
    return rc;
  return gemm(n, n->H, kHid, n->w16 + n->f2.w, kHid, n->B, kOutPad, kHid, n->w32 + n->f2.b, 0, n->O, kOutPad, false,
              s);
}

// gradients of a dense layer y = act(W x + b) given dPre = dL/d(W x + b) [rows][N]:
// db = column sums, dW [N][K] = dPre^T x (x [rows][K]); dx = dPre W when dx != null
int dense_bwd(Net* n, const Layer& L, int li, const bf16* dPre, const bf16* x, long long rows, long long rows_p,
              bf16* dx, cudaStream_t s) {
  int rc;
  k_colsum<<<kColBlocks, 256, 0, s>>>(dPre, rows, L.N, n->colpart, n->counter, n->g32 + L.b);
  HR_CHECK_LAUNCH();
  // dPre^T [N][rows_p] and x^T [K][rows_p], zero-padded along the reduction
  k_transpose<<<dim3((unsigned)((rows_p + 31) / 32), (unsigned)((L.N + 31) / 32)), dim3(32, 8), 0, s>>>(
      dPre, rows, L.N, L.N, n->dPreT, rows_p);
  HR_CHECK_LAUNCH();
  k_transpose<<<dim3((unsigned)((rows_p + 31) / 32), (unsigned)((L.K + 31) / 32)), dim3(32, 8), 0, s>>>(
      x, rows, L.K, L.K, n->colsT, rows_p);
  HR_CHECK_LAUNCH();
  const int sp = wgrad_splits(L.N, L.K, rows_p);
  if ((rc = gemm(n, n->dPreT, (int)rows_p, n->colsT, (int)rows_p, L.N, L.K, (int)rows_p, nullptr, 0, n->g32 + L.w,
                 L.K, false, s, sp)) != HR_OK)
    return rc;
  if (dx)
    return gemm(n, dPre, L.N, n->wT[li], L.N, (int)rows, L.K, L.N, nullptr, 0, dx, L.K, true, s);
  return HR_OK;
}

int net_backward(Net* n, const float* d_out, cudaStream_t s) {
  int rc;
  const long long Bp = n->Bp, NVp = n->NVp;
  // output layer (linear)
  k_net_dout<<<nblk(n->B * kOutPad), 256, 0, s>>>(d_out, n->B, n->dO);
  HR_CHECK_LAUNCH();
  if ((rc = dense_bwd(n, n->f2, 7, n->dO, n->H, n->B, Bp, n->dH, s)) != HR_OK) return rc;
  // hidden layer
  k_relu_grad<<<nblk((long long)n->B * kHid), 256, 0, s>>>(n->dH, n->H, (long long)n->B * kHid, n->dPre);
  HR_CHECK_LAUNCH();
  if ((rc = dense_bwd(n, n->f1, 6, n->dPre, n->Pool, n->B, Bp, n->dP, s)) != HR_OK) return rc;
  // view pooling, per-view layer
  k_viewpool_bwd<<<nblk((long long)n->NV * kHid), 256, 0, s>>>(n->dP, n->pidx, n->B, n->nv, n->dF);
  HR_CHECK_LAUNCH();
  k_relu_grad<<<nblk((long long)n->NV * kHid), 256, 0, s>>>(n->dF, n->F, (long long)n->NV * kHid, n->dPre);
  HR_CHECK_LAUNCH();
  if ((rc = dense_bwd(n, n->fv, 5, n->dPre, n->Z, n->NV, NVp, n->dZ, s)) != HR_OK) return rc;
  // dY5 = the first 2048 columns of dZ
  bf16* dY = n->dA;
  bf16* dnext = n->dB;
  if (cudaMemcpy2DAsync(dY, kFeat * sizeof(bf16), n->dZ, kZ * sizeof(bf16), kFeat * sizeof(bf16), n->NV,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HR_ERR_CUDA;
  for (int l = kConv - 1; l >= 0; --l) {
    const int Hin = kHin[l], Ho = Hin / 2;
    const long long rows = (long long)n->NV * Ho * Ho;
    const Layer& L = n->conv[l];
    k_relu_grad<<<nblk(rows * L.N), 256, 0, s>>>(dY, n->act[l + 1], rows * L.N, n->dPre);
    HR_CHECK_LAUNCH();
    k_colsum<<<kColBlocks, 256, 0, s>>>(n->dPre, rows, L.N, n->colpart, n->counter, n->g32 + L.b);
    HR_CHECK_LAUNCH();
    k_transpose<<<dim3((unsigned)((rows + 31) / 32), (unsigned)((L.N + 31) / 32)), dim3(32, 8), 0, s>>>(
        n->dPre, rows, L.N, L.N, n->dPreT, rows);
    HR_CHECK_LAUNCH();
    k_im2col<true><<<nblk(rows * kKp[l]), 256, 0, s>>>(n->act[l], n->NV, Hin, kCin[l], kKp[l], n->colsT, rows);
    HR_CHECK_LAUNCH();
    const int sp = wgrad_splits(L.N, L.K, rows);
    if ((rc = gemm(n, n->dPreT, (int)rows, n->colsT, (int)rows, L.N, L.K, (int)rows, nullptr, 0, n->g32 + L.w, L.K,
                   false, s, sp)) != HR_OK)
      return rc;
    if (l == 0) break;
    if ((rc = gemm(n, n->dPre, L.N, n->wT[l], L.N, (int)rows, L.K, L.N, nullptr, 0, n->dcols, L.K, true, s)) !=
        HR_OK)
      return rc;
    k_col2im<<<nblk((long long)n->NV * Hin * Hin * kCin[l]), 256, 0, s>>>(n->dcols, n->NV, Hin, kCin[l], kKp[l],
                                                                          dnext);
    HR_CHECK_LAUNCH();
    bf16* t = dY;
    dY = dnext;
    dnext = t;
  }
  return HR_OK;
}

}  // namespace

}  // namespace hr

using hr::Net;

extern "C" {

int hr_net_param_count(void) {
  size_t off = 0;
  for (int l = 0; l < hr::kConv; ++l) hr::make_layer(hr::kCout[l], hr::kKp[l], off);
  hr::make_layer(hr::kHid, hr::kZ, off);
  hr::make_layer(hr::kHid, hr::kHid, off);
  hr::make_layer(hr::kOutPad, hr::kHid, off);
  return (int)off;
}

int hr_net_create(int B, int views, hr_net** out) {
  using namespace hr;
  // the weight gradient of the last convolution reduces over 16 NV rows: a multiple
  // of the GEMM's 64-wide K step when NV is a multiple of 4
  if (!out || B < 1 || views < 1 || B > 4096 || views > 64 || (B * views) % 4 != 0) return HR_ERR_ARG;
  *out = nullptr;
  Net* n = new (std::nothrow) Net();
  if (!n) return HR_ERR_CUDA;
  std::memset(n, 0, sizeof(Net));
  n->B = B;
  n->nv = views;
  n->NV = B * views;
  n->Bp = round64(B);
  n->NVp = round64(n->NV);
  size_t off = 0;
  for (int l = 0; l < kConv; ++l) n->conv[l] = make_layer(kCout[l], kKp[l], off);
  n->fv = make_layer(kHid, kZ, off);
  n->f1 = make_layer(kHid, kHid, off);
  n->f2 = make_layer(kOutPad, kHid, off);
  n->P = off;
  const size_t NV = n->NV;
  size_t cols = 0, act_max = 0;
  for (int l = 0; l < kConv; ++l) {
    const size_t rows = NV * (kHin[l] / 2) * (kHin[l] / 2);
    cols = std::max(cols, rows * kKp[l]);
    act_max = std::max(act_max, rows * kCout[l]);
  }
  cols = std::max(cols, (size_t)n->NVp * kZ);
  n->cols_elems = cols;
  const size_t big = std::max<size_t>(act_max, NV * kZ);
  bool ok = nalloc(&n->w32, n->P) && nalloc(&n->g32, n->P) && nalloc(&n->m, n->P) && nalloc(&n->v, n->P) &&
            nalloc(&n->w16, n->P) && nalloc(&n->Z, NV * kZ) && nalloc(&n->F, NV * kHid) &&
            nalloc(&n->Pool, (size_t)B * kHid) && nalloc(&n->H, (size_t)B * kHid) && nalloc(&n->pidx, (size_t)B * kHid) &&
            nalloc(&n->O, (size_t)B * kOutPad) && nalloc(&n->cols, cols) && nalloc(&n->colsT, cols) &&
            nalloc(&n->dcols, cols) && nalloc(&n->dA, big) && nalloc(&n->dB, big) &&
            nalloc(&n->dPre, std::max<size_t>(act_max, NV * kHid)) &&
            nalloc(&n->dPreT, std::max<size_t>(act_max, (size_t)kHid * n->NVp)) && nalloc(&n->dZ, NV * kZ) &&
            nalloc(&n->dF, NV * kHid) && nalloc(&n->dP, (size_t)B * kHid) && nalloc(&n->dH, (size_t)B * kHid) &&
            nalloc(&n->dO, (size_t)B * kOutPad) &&
            nalloc(&n->split, (size_t)kSplitMax * kHid * kZ) && nalloc(&n->colpart, (size_t)kColBlocks * kZ) &&
            nalloc(&n->counter, 1) && nalloc(&n->status, 1);
  const Layer* ls[kConv + 3] = {&n->conv[0], &n->conv[1], &n->conv[2], &n->conv[3], &n->conv[4],
                                &n->fv,      &n->f1,      &n->f2};
  for (int i = 1; ok && i < kConv + 3; ++i) ok = nalloc(&n->wT[i], (size_t)ls[i]->N * ls[i]->K);
  ok = ok && nalloc(&n->act[0], NV * kIn * kIn * kC0);
  for (int l = 0; ok && l < kConv; ++l) {
    const size_t rows = NV * (kHin[l] / 2) * (kHin[l] / 2);
    ok = nalloc(&n->act[l + 1], rows * kCout[l]);
  }
  if (ok)
    ok = cudaMemset(n->counter, 0, sizeof(unsigned)) == cudaSuccess &&
         cudaMemset(n->status, 0, sizeof(int)) == cudaSuccess &&
         cudaMemset(n->w32, 0, n->P * sizeof(float)) == cudaSuccess &&
         cudaMemset(n->m, 0, n->P * sizeof(float)) == cudaSuccess &&
         cudaMemset(n->v, 0, n->P * sizeof(float)) == cudaSuccess && configure_gemm_kernels() == HR_OK;
  if (!ok) {
    cudaGetLastError();
    free_net(n);
    return HR_ERR_CUDA;
  }
  *out = reinterpret_cast<hr_net*>(n);
  return HR_OK;
}

int hr_net_destroy(hr_net* net) {
  if (!net) return HR_ERR_ARG;
  cudaDeviceSynchronize();
  hr::free_net(reinterpret_cast<Net*>(net));
  return HR_OK;
}

int hr_net_set_params(hr_net* net, const float* params, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n || !params) return HR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(n->w32, params, n->P * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(n->m, 0, n->P * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(n->v, 0, n->P * sizeof(float), s) != cudaSuccess)
    return HR_ERR_CUDA;
  return hr::refresh_weights(n, s);
}

int hr_net_get_params(hr_net* net, float* params, float* grads, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n || (!params && !grads)) return HR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (params && cudaMemcpyAsync(params, n->w32, n->P * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HR_ERR_CUDA;
  if (grads && cudaMemcpyAsync(grads, n->g32, n->P * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HR_ERR_CUDA;
  return HR_OK;
}

int hr_net_inputs(hr_net* net, const float* render, const float* observed, int W, int H, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n || !render || !observed || W != 2 * hr::kIn || H != 2 * hr::kIn) return HR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  hr::k_net_inputs<<<hr::nblk((long long)n->NV * hr::kIn * hr::kIn), 256, 0, s>>>(render, observed, n->NV, W, H,
                                                                                  n->act[0]);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int hr_net_set_inputs_bf16(hr_net* net, const void* x0, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n || !x0) return HR_ERR_ARG;
  if (cudaMemcpyAsync(n->act[0], x0, (size_t)n->NV * hr::kIn * hr::kIn * hr::kC0 * 2, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream) != cudaSuccess)
    return HR_ERR_CUDA;
  return HR_OK;
}

int hr_net_forward(hr_net* net, const float* cams, const float* base, float* out, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n || !cams || !out) return HR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = hr::net_forward(n, cams, s);
  if (rc != HR_OK) return rc;
  hr::k_net_out<<<hr::nblk(n->B * hr::kOut), 256, 0, s>>>(n->O, n->B, base, out);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int hr_net_backward(hr_net* net, const float* d_out, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n || !d_out) return HR_ERR_ARG;
  return hr::net_backward(n, d_out, (cudaStream_t)stream);
}

int hr_net_adam(hr_net* net, float lr, float beta1, float beta2, float eps, int step, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n || step < 1 || !(lr >= 0.0f)) return HR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = hr::launch_adam(n->w32, n->g32, n->m, n->v, (int)n->P, lr, beta1, beta2, eps, step, s);
  if (rc != HR_OK) return rc;
  return hr::refresh_weights(n, s);
}

int hr_net_status(hr_net* net, hr_stream stream) {
  Net* n = reinterpret_cast<Net*>(net);
  if (!n) return HR_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  int host = 0;
  if (cudaMemcpy(&host, n->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(n->status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  return (host & hr::kStatusTimeout) ? HR_ERR_TIMEOUT : HR_OK;
}

}  // extern "C"
