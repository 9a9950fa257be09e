// The edge term D_e of Eq. 4: Canny's detector applied to camera i's colour-
// transformed rendering T_i R, its edge strength blurred by K (an 11 x 11 Gaussian of
// sigma 5), and the masked L1 difference to the observation's blurred edge map, with
// the adjoint into R and into T.
//
// Detector (Canny 1986, textbook steps): luma g = a . R with a = T^T w (w the Rec. 601
// weights), 5-tap Gaussian (sigma 1) along x then y, Sobel / 8 as (1/4, 1/2, 1/4)
// smoothing and (-1/2, 0, 1/2) differences, m = sqrt(gx^2 + gy^2 + 1e-12), non-maximum
// suppression along the gradient direction quantised to 0/45/90/135 degrees (pixel
// survives when m >= both neighbours, neighbour coordinates clamped), candidates
// m > low, strong m > high, hysteresis = candidates 8-connected to a strong pixel.
// The edge strength E is m on kept pixels; E_hat = K_y K_x E with zero padding.  The
// detector's passes replicate the image border (every read clamps its coordinates).
//
// Layout: images [N][H][W][3] float32, masks and edge maps [N][H][W], pixel p =
// (view H + y) W + x.  The forward up to E_hat is float32 with one rounding per
// multiply and per add, taps summed from the most negative offset up: the selection
// and the sign of E_hat_r - E_hat_o are decisions.  Kernels:
//   k_canny      32 x 8 output tiles: luma, smoothing, Sobel, magnitude and
//                suppression in shared memory (4-pixel halo); writes (gx, gy), the
//                candidate/strong bits, and union-find parents after joining the
//                tile's candidates in shared memory
//   k_cc_border  candidates on tile borders join their W, NW, N, NE candidate
//                neighbours in other tiles (lock-free union by atomicMin on roots;
//                parents only decrease)
//   k_cc_flag    every candidate points at its root; strong pixels mark the root
//                (kept = candidate whose root is marked: one hop afterwards)
//   k_edge_blur  tiles with a 5-pixel halo: E from (gx, gy) on kept pixels, K along x
//                then y; writes E_hat, or the loss's sign map and block partials
//   k_edge_final block partials in a fixed order: loss and weight / sum M
//   k_edge_bwd1  K^T of the sign map on tiles, then through the magnitude: (gbar_x,
//                gbar_y) = mbar (gx, gy) / m on kept pixels
//   k_edge_bwd2  tiles with a 3-pixel halo: the transposed Sobel and Gaussian passes
//                (a replicated border folds the gradient of clamped reads back onto
//                the border pixel), adjoint += a gbar, per-tile sums of gbar R
//   k_edge_dT    dT[i][r][c] += w_r sum over the view's tiles (fixed order)
#include <algorithm>
#include <climits>
#include <cmath>

#include "hr_internal.h"

namespace hr {
namespace {

constexpr int kTX = 32, kTY = 8, kEThreads = kTX * kTY;
constexpr int kUnionIters = 1 << 20;
constexpr int kFinalThreads = 256;

struct EdgeW {
  float g5[5];     // Canny's smoothing, offsets -2..2
  float k11[11];   // K, offsets -5..5
  float gray[3];   // luma weights
  float t1, t2;    // tan(22.5 deg), tan(67.5 deg)
  float low, high;
};

// normalised Gaussian taps: exp(-k^2 / (2 sigma^2)) in double, divided by their sum
// (added from the most negative offset up), rounded to float
void gauss_taps(int r, double sigma, float* out) {
  double e[16], tot = 0.0;
  for (int k = -r; k <= r; ++k) e[k + r] = std::exp(-(double)(k * k) / (2.0 * sigma * sigma));
  for (int i = 0; i <= 2 * r; ++i) tot += e[i];
  for (int i = 0; i <= 2 * r; ++i) out[i] = (float)(e[i] / tot);
}

EdgeW make_weights(float low, float high) {
  EdgeW w;
  gauss_taps(2, 1.0, w.g5);
  gauss_taps(5, 5.0, w.k11);
  w.gray[0] = 0.299f;
  w.gray[1] = 0.587f;
  w.gray[2] = 0.114f;
  w.t1 = (float)(std::sqrt(2.0) - 1.0);
  w.t2 = (float)(std::sqrt(2.0) + 1.0);
  w.low = low;
  w.high = high;
  return w;
}

__device__ __constant__ float kSmooth[3] = {0.25f, 0.5f, 0.25f};
__device__ __constant__ float kDeriv[3] = {-0.5f, 0.0f, 0.5f};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// a = T^T w for view `view` (a = w without T): a_c = (w0 T0c + w1 T1c) + w2 T2c
__device__ __forceinline__ float3 luma_weights(const float* T, int view, const EdgeW& w) {
  if (!T) return make_float3(w.gray[0], w.gray[1], w.gray[2]);
  const float* t = T + 9 * view;
  float a[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    a[c] = __fadd_rn(__fadd_rn(__fmul_rn(w.gray[0], t[c]), __fmul_rn(w.gray[1], t[3 + c])),
                     __fmul_rn(w.gray[2], t[6 + c]));
  return make_float3(a[0], a[1], a[2]);
}

__device__ __forceinline__ float magnitude(float gx, float gy) {
  return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), 1e-12f));
}

// ---- union-find over candidate pixels (parent[x] <= x always)
__device__ __forceinline__ int cc_find(const int* parent, int x) {
  int p = __ldcg(parent + x);
  while (p != x) {
    x = p;
    p = __ldcg(parent + x);
  }
  return x;
}

__device__ void cc_unite(int* parent, int a, int b, int* status) {
  for (int it = 0; it < kUnionIters; ++it) {
    a = cc_find(parent, a);
    b = cc_find(parent, b);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    // link root b under a; if b gained a parent meanwhile, join that one instead
    const int old = atomicMin(parent + b, a);
    if (old == b) return;
    b = old;
  }
  atomicOr(status, kStatusLimit);
}

// a kept pixel: a candidate whose root holds a strong pixel (parents flattened)
__device__ __forceinline__ bool kept(const uint8_t* cls, const int* parent, const uint8_t* flag, int p) {
  return (cls[p] & 1) && flag[parent[p]];
}

// the same on a tile's labels in shared memory
__device__ __forceinline__ int find_local(const int* lab, int x) {
  const volatile int* v = lab;
  int p = v[x];
  while (p != x) {
    x = p;
    p = v[x];
  }
  return x;
}

__device__ void unite_local(int* lab, int a, int b, int* status) {
  for (int it = 0; it < kUnionIters; ++it) {
    a = find_local(lab, a);
    b = find_local(lab, b);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(lab + b, a);
    if (old == b) return;
    b = old;
  }
  atomicOr(status, kStatusLimit);
}

// ---- the detector on one 32 x 8 tile.  Shared-memory stages and the global
// coordinates they cover (tile origin x0, y0); each stage is evaluated at in-image
// coordinates only and reads its input at clamped coordinates:
//   luma        x0-4 .. x0+35, y0-4 .. y0+11
//   h  (G5, x)  x0-2 .. x0+33, y0-4 .. y0+11
//   s  (G5, y)  x0-2 .. x0+33, y0-2 .. y0+9
//   v  (S, y)   x0-2 .. x0+33, y0-1 .. y0+8      gx = D_x v
//   u  (S, x)   x0-1 .. x0+32, y0-2 .. y0+9      gy = D_y u
//   gx, gy, m   x0-1 .. x0+32, y0-1 .. y0+8
struct CannySmem {
  float sl[kTY + 8][kTX + 8];
  float sh[kTY + 8][kTX + 4];
  float ss[kTY + 4][kTX + 4];
  float sv[kTY + 2][kTX + 4];
  float su[kTY + 4][kTX + 2];
  float sgx[kTY + 2][kTX + 2], sgy[kTY + 2][kTX + 2], sm[kTY + 2][kTX + 2];
  int lab[kEThreads];
};

// INNER: the tile's 4-pixel halo lies inside the image, so no coordinate needs a
// clamp or a bounds check (the same arithmetic as the general path, fewer
// instructions)
template <bool INNER>
__device__ __forceinline__ void canny_tile(CannySmem& S, const float* __restrict__ img, float3 a, int view, int x0,
                                           int y0, int H, int W, const EdgeW& w, float2* __restrict__ gxy,
                                           uint8_t* __restrict__ cls, uint8_t* __restrict__ flag,
                                           int* __restrict__ parent, int* status) {
  constexpr int LX = kTX + 8, LY = kTY + 8;
  constexpr int HX = kTX + 4, HY = kTY + 8;
  constexpr int SX = kTX + 4, SY = kTY + 4;
  constexpr int VX = kTX + 4, VY = kTY + 2;
  constexpr int UX = kTX + 2, UY = kTY + 4;
  constexpr int MX = kTX + 2, MY = kTY + 2;
  const int tid = threadIdx.x;
  auto cx = [&](int x) { return INNER ? x : clampi(x, 0, W - 1); };
  auto cy = [&](int y) { return INNER ? y : clampi(y, 0, H - 1); };
  auto outside = [&](int x, int y) { return !INNER && (x < 0 || x >= W || y < 0 || y >= H); };
  for (int i = tid; i < LX * LY; i += kEThreads) {
    const int ry = i / LX, rx = i % LX, x = x0 - 4 + rx, y = y0 - 4 + ry;
    if (outside(x, y)) continue;
    const float* px = img + ((size_t)y * W + x) * 3;
    S.sl[ry][rx] = __fadd_rn(__fadd_rn(__fmul_rn(a.x, px[0]), __fmul_rn(a.y, px[1])), __fmul_rn(a.z, px[2]));
  }
  __syncthreads();
  for (int i = tid; i < HX * HY; i += kEThreads) {
    const int ry = i / HX, rx = i % HX, x = x0 - 2 + rx, y = y0 - 4 + ry;
    if (outside(x, y)) continue;
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const float term = __fmul_rn(w.g5[t], S.sl[ry][cx(x + t - 2) - (x0 - 4)]);
      acc = t ? __fadd_rn(acc, term) : term;
    }
    S.sh[ry][rx] = acc;
  }
  __syncthreads();
  for (int i = tid; i < SX * SY; i += kEThreads) {
    const int ry = i / SX, rx = i % SX, x = x0 - 2 + rx, y = y0 - 2 + ry;
    if (outside(x, y)) continue;
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const float term = __fmul_rn(w.g5[t], S.sh[cy(y + t - 2) - (y0 - 4)][rx]);
      acc = t ? __fadd_rn(acc, term) : term;
    }
    S.ss[ry][rx] = acc;
  }
  __syncthreads();
  for (int i = tid; i < VX * VY + UX * UY; i += kEThreads) {
    if (i < VX * VY) {
      const int ry = i / VX, rx = i % VX, x = x0 - 2 + rx, y = y0 - 1 + ry;
      if (outside(x, y)) continue;
      float acc = 0.0f;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const float term = __fmul_rn(kSmooth[t], S.ss[cy(y + t - 1) - (y0 - 2)][rx]);
        acc = t ? __fadd_rn(acc, term) : term;
      }
      S.sv[ry][rx] = acc;
    } else {
      const int j = i - VX * VY, ry = j / UX, rx = j % UX, x = x0 - 1 + rx, y = y0 - 2 + ry;
      if (outside(x, y)) continue;
      float acc = 0.0f;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const float term = __fmul_rn(kSmooth[t], S.ss[ry][cx(x + t - 1) - (x0 - 2)]);
        acc = t ? __fadd_rn(acc, term) : term;
      }
      S.su[ry][rx] = acc;
    }
  }
  __syncthreads();
  for (int i = tid; i < MX * MY; i += kEThreads) {
    const int ry = i / MX, rx = i % MX, x = x0 - 1 + rx, y = y0 - 1 + ry;
    if (outside(x, y)) continue;
    float gx = 0.0f, gy = 0.0f;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const float tx = __fmul_rn(kDeriv[t], S.sv[ry][cx(x + t - 1) - (x0 - 2)]);
      const float ty = __fmul_rn(kDeriv[t], S.su[cy(y + t - 1) - (y0 - 2)][rx]);
      gx = t ? __fadd_rn(gx, tx) : tx;
      gy = t ? __fadd_rn(gy, ty) : ty;
    }
    S.sgx[ry][rx] = gx;
    S.sgy[ry][rx] = gy;
    S.sm[ry][rx] = magnitude(gx, gy);
  }
  __syncthreads();
  const int tx = tid % kTX, ty = tid / kTX, x = x0 + tx, y = y0 + ty;
  const bool in = INNER || (x < W && y < H);
  bool cand = false;
  if (in) {
    const float gx = S.sgx[ty + 1][tx + 1], gy = S.sgy[ty + 1][tx + 1], m = S.sm[ty + 1][tx + 1];
    const float ax = fabsf(gx), ay = fabsf(gy);
    const bool along_x = ay <= __fmul_rn(w.t1, ax);
    const bool along_y = !along_x && ay >= __fmul_rn(w.t2, ax);
    const int dx = along_y ? 0 : 1;
    const int dy = along_x ? 0 : (along_y ? 1 : (((gx > 0.0f) == (gy > 0.0f)) ? 1 : -1));
    const float m1 = S.sm[cy(y + dy) - (y0 - 1)][cx(x + dx) - (x0 - 1)];
    const float m2 = S.sm[cy(y - dy) - (y0 - 1)][cx(x - dx) - (x0 - 1)];
    cand = m >= m1 && m >= m2 && m > w.low;
    const bool strong = cand && m > w.high;
    const int p = (view * H + y) * W + x;
    gxy[p] = make_float2(gx, gy);
    cls[p] = (uint8_t)((cand ? 1 : 0) | (strong ? 2 : 0));
    flag[p] = 0;
  }
  // the tile's candidates joined in shared memory (local index l = ty 32 + tx; a
  // component's root is its smallest index, so a pixel's global parent, the root's
  // global index, never exceeds its own)
  int* lab = S.lab;
  lab[tid] = cand ? tid : -1;
  __syncthreads();
  if (cand) {
    if (tx > 0 && lab[tid - 1] >= 0) unite_local(lab, tid, tid - 1, status);
    if (ty > 0) {
      if (tx > 0 && lab[tid - kTX - 1] >= 0) unite_local(lab, tid, tid - kTX - 1, status);
      if (lab[tid - kTX] >= 0) unite_local(lab, tid, tid - kTX, status);
      if (tx + 1 < kTX && lab[tid - kTX + 1] >= 0) unite_local(lab, tid, tid - kTX + 1, status);
    }
  }
  __syncthreads();
  if (in) {
    int root = -1;
    if (cand) {
      const int r = find_local(lab, tid);
      root = (view * H + y0 + r / kTX) * W + x0 + r % kTX;
    }
    parent[(view * H + y) * W + x] = root;
  }
}

__global__ void __launch_bounds__(kEThreads) k_canny(const float* __restrict__ image, const float* __restrict__ T,
                                                     int H, int W, EdgeW w, float2* __restrict__ gxy,
                                                     uint8_t* __restrict__ cls, uint8_t* __restrict__ flag,
                                                     int* __restrict__ parent, int* status) {
  __shared__ CannySmem S;
  const int view = blockIdx.z, x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const float3 a = luma_weights(T, view, w);
  const float* img = image + (size_t)view * H * W * 3;
  if (x0 >= 4 && x0 + kTX + 4 <= W && y0 >= 4 && y0 + kTY + 4 <= H)
    canny_tile<true>(S, img, a, view, x0, y0, H, W, w, gxy, cls, flag, parent, status);
  else
    canny_tile<false>(S, img, a, view, x0, y0, H, W, w, gxy, cls, flag, parent, status);
}

// candidates on a tile's border join their candidate neighbours in other tiles (the
// W, NW, N, NE neighbours that lie outside the tile), on the global forest
__global__ void __launch_bounds__(kEThreads) k_cc_border(const uint8_t* __restrict__ cls, int* parent, int H, int W,
                                                         int* status) {
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  if (ty != 0 && tx != 0 && tx != kTX - 1) return;
  const int view = blockIdx.z, x = blockIdx.x * kTX + tx, y = blockIdx.y * kTY + ty;
  if (x >= W || y >= H) return;
  const int p = (view * H + y) * W + x;
  if (!(cls[p] & 1)) return;
  // neighbour (x + ox, y + oy) for the four earlier neighbours, when outside the tile
  const int ox[4] = {-1, -1, 0, 1}, oy[4] = {0, -1, -1, -1};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int nx = x + ox[k], ny = y + oy[k], ntx = tx + ox[k], nty = ty + oy[k];
    if (nx < 0 || nx >= W || ny < 0) continue;
    if (ntx >= 0 && ntx < kTX && nty >= 0) continue;   // inside the tile: joined already
    const int q = (view * H + ny) * W + nx;
    if (cls[q] & 1) cc_unite(parent, p, q, status);
  }
}

// every candidate points at its root (flattening; a concurrent find reads either an
// ancestor or the root), and strong pixels mark their root
__global__ void k_cc_flag(const uint8_t* __restrict__ cls, int* parent, uint8_t* flag, int P) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const uint8_t c = cls[p];
    if (!(c & 1)) continue;
    const int r = cc_find(parent, p);
    parent[p] = r;
    if (c & 2) flag[r] = 1;
  }
}

// fixed-order block sum (warp shuffles, then the warps in order); thread 0 holds the
// totals afterwards
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float (*red)[kEThreads / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float x = 0.0f;
      for (int i = 0; i < kEThreads / 32; ++i) x += red[k][i];
      v[k] = x;
    }
  }
}

// E_hat = K_y K_x E on a tile (E from (gx, gy) on kept pixels, zero outside the image).
// Without `obs`: writes E_hat to `out`.  With `obs` (the observation's E_hat) and
// `mask`: sign map gs = M sign(E_hat - obs) and per-tile (sum M |d|, sum M).
__global__ void __launch_bounds__(kEThreads) k_edge_blur(const uint8_t* __restrict__ cls,
                                                         const int* __restrict__ parent,
                                                         const uint8_t* __restrict__ flag,
                                                         const float2* __restrict__ gxy, int H, int W, EdgeW w,
                                                         float* __restrict__ out, const float* __restrict__ obs,
                                                         const uint8_t* __restrict__ mask,
                                                         int8_t* __restrict__ gs, float2* __restrict__ part) {
  constexpr int EX = kTX + 10, EY = kTY + 10;
  __shared__ float se[EY][EX], sb[EY][kTX];
  __shared__ float red[2][kEThreads / 32];
  const int view = blockIdx.z, x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, tid = threadIdx.x;
  for (int i = tid; i < EX * EY; i += kEThreads) {
    const int ry = i / EX, rx = i % EX, x = x0 - 5 + rx, y = y0 - 5 + ry;
    float e = 0.0f;
    if (x >= 0 && x < W && y >= 0 && y < H) {
      const int p = (view * H + y) * W + x;
      if (kept(cls, parent, flag, p)) {
        const float2 g = gxy[p];
        e = magnitude(g.x, g.y);
      }
    }
    se[ry][rx] = e;
  }
  __syncthreads();
  for (int i = tid; i < kTX * EY; i += kEThreads) {
    const int ry = i / kTX, rx = i % kTX;
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < 11; ++t) {
      const float term = __fmul_rn(w.k11[t], se[ry][rx + t]);
      acc = t ? __fadd_rn(acc, term) : term;
    }
    sb[ry][rx] = acc;
  }
  __syncthreads();
  const int tx = tid % kTX, ty = tid / kTX, x = x0 + tx, y = y0 + ty;
  const bool in = x < W && y < H;
  float acc = 0.0f;
#pragma unroll
  for (int t = 0; t < 11; ++t) {
    const float term = __fmul_rn(w.k11[t], sb[ty + t][tx]);
    acc = t ? __fadd_rn(acc, term) : term;
  }
  const int p = (view * H + y) * W + x;
  if (!obs) {
    if (in) out[p] = acc;
    return;
  }
  float v[2] = {0.0f, 0.0f};
  if (in) {
    const float d = __fsub_rn(acc, obs[p]);
    const bool m = mask[p] != 0;
    gs[p] = (int8_t)(m ? (d > 0.0f) - (d < 0.0f) : 0);
    if (m) {
      v[0] = fabsf(d);
      v[1] = 1.0f;
    }
  }
  block_sum<2>(v, red);
  if (tid == 0) part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = make_float2(v[0], v[1]);
}

// loss = weight sum |d| / sum M and scale = weight / sum M (0 without masked pixels);
// each thread sums a fixed stride of the tiles in double, then a fixed-order tree
__global__ void __launch_bounds__(kFinalThreads) k_edge_final(const float2* __restrict__ part, int n, float weight,
                                                              float* __restrict__ loss, float* __restrict__ scale) {
  __shared__ double sa[kFinalThreads], sc[kFinalThreads];
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += kFinalThreads) {
    const float2 v = part[i];
    a += v.x;
    c += v.y;
  }
  sa[threadIdx.x] = a;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int s = kFinalThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sc[threadIdx.x] += sc[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sc_ = sc[0] > 0.0 ? (double)weight / sc[0] : 0.0;
    loss[0] = (float)(sa[0] * sc_);
    scale[0] = (float)sc_;
  }
}

// mbar = kept ? scale (K_x^T K_y^T gs) : 0 (K is symmetric and zero-padded, so each
// transpose is the same tap sum), then (gbar_x, gbar_y) = mbar (gx, gy) / m
__global__ void __launch_bounds__(kEThreads) k_edge_bwd1(const int8_t* __restrict__ gs,
                                                         const uint8_t* __restrict__ cls,
                                                         const int* __restrict__ parent,
                                                         const uint8_t* __restrict__ flag,
                                                         const float2* __restrict__ gxy, int H, int W, EdgeW w,
                                                         const float* __restrict__ scale,
                                                         float2* __restrict__ gbar) {
  constexpr int EX = kTX + 10, EY = kTY + 10;
  __shared__ float sg[EY][EX], sb[kTY][EX];
  const int view = blockIdx.z, x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, tid = threadIdx.x;
  for (int i = tid; i < EX * EY; i += kEThreads) {
    const int ry = i / EX, rx = i % EX, x = x0 - 5 + rx, y = y0 - 5 + ry;
    sg[ry][rx] = (x >= 0 && x < W && y >= 0 && y < H) ? (float)gs[(view * H + y) * W + x] : 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < kTY * EX; i += kEThreads) {
    const int ry = i / EX, rx = i % EX;
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < 11; ++t) acc += w.k11[t] * sg[ry + t][rx];
    sb[ry][rx] = acc;
  }
  __syncthreads();
  const int tx = tid % kTX, ty = tid / kTX, x = x0 + tx, y = y0 + ty;
  if (x >= W || y >= H) return;
  const int p = (view * H + y) * W + x;
  float2 out = make_float2(0.0f, 0.0f);
  if (kept(cls, parent, flag, p)) {
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < 11; ++t) acc += w.k11[t] * sb[ty][tx + t];
    const float2 g = gxy[p];
    const float mb = acc * scale[0] / magnitude(g.x, g.y);
    out = make_float2(mb * g.x, mb * g.y);
  }
  gbar[p] = out;
}

// The adjoint of a replicated-border tap pass y[i] = sum_t w_t x[clamp(i + t - R)]
// at output j (0 <= j < n): x_bar[j] = sum over the reads that landed on j.  The
// input element of coordinate i along the pass is y[(i - origin) * stride].  INNER:
// j - R .. j + R lie inside (1 .. n - 2), so neither bounds nor folds apply.
template <int R, bool INNER>
__device__ __forceinline__ float tap_T(const float* w, int j, int n, const float* y, int origin, int stride) {
  float acc = 0.0f;
#pragma unroll
  for (int t = 0; t <= 2 * R; ++t) {
    const int i = j + R - t;
    if (INNER || (i >= 0 && i < n)) acc += w[t] * y[(i - origin) * stride];
  }
  if (INNER) return acc;
  if (j == 0) {   // reads below the border were clamped onto coordinate 0
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (i < n)
#pragma unroll
        for (int t = 0; t < R - i; ++t) acc += w[t] * y[(i - origin) * stride];
  }
  if (j == n - 1) {   // and reads beyond it onto n - 1 (i = n - 1 - q)
#pragma unroll
    for (int q = 0; q < R; ++q)
      if (n - 1 - q >= 0)
#pragma unroll
        for (int t = R + q + 1; t <= 2 * R; ++t) acc += w[t] * y[(n - 1 - q - origin) * stride];
  }
  return acc;
}

// Transposed Sobel and smoothing passes on a tile, then adjoint += a gbar and the
// tile's sums of gbar R (for dT).  Stages (in-image coordinates only):
//   (gbar_x, gbar_y)  x0-3 .. x0+34, y0-3 .. y0+10
//   vb = D_x^T gbar_x x0-2 .. x0+33, y0-3 .. y0+10
//   ub = D_y^T gbar_y x0-3 .. x0+34, y0-2 .. y0+9
//   sb = S_y^T vb + S_x^T ub          x0-2 .. x0+33, y0-2 .. y0+9
//   hb = G5_y^T sb                    x0-2 .. x0+33, y0 .. y0+7
//   gb = G5_x^T hb                    the tile
struct Bwd2Smem {
  float sbx[kTY + 6][kTX + 6], sby[kTY + 6][kTX + 6];
  float sv[kTY + 6][kTX + 4];
  float su[kTY + 4][kTX + 6];
  float ssb[kTY + 4][kTX + 4];
  float shb[kTY][kTX + 4];
  float red[3][kEThreads / 32];
};

template <bool INNER>
__device__ __forceinline__ void bwd2_tile(Bwd2Smem& S, const float2* __restrict__ gbar,
                                          const float* __restrict__ image, float3 a, int view, int x0, int y0, int H,
                                          int W, const EdgeW& w, float* __restrict__ adjoint,
                                          float4* __restrict__ part) {
  constexpr int BX = kTX + 6, BY = kTY + 6;
  constexpr int VX = kTX + 4, VY = kTY + 6;
  constexpr int UX = kTX + 6, UY = kTY + 4;
  constexpr int SX = kTX + 4, SY = kTY + 4;
  constexpr int HX = kTX + 4;
  const int tid = threadIdx.x;
  auto outside = [&](int x, int y) { return !INNER && (x < 0 || x >= W || y < 0 || y >= H); };
  for (int i = tid; i < BX * BY; i += kEThreads) {
    const int ry = i / BX, rx = i % BX, x = x0 - 3 + rx, y = y0 - 3 + ry;
    float2 g = make_float2(0.0f, 0.0f);
    if (!outside(x, y)) g = gbar[(view * H + y) * W + x];
    S.sbx[ry][rx] = g.x;
    S.sby[ry][rx] = g.y;
  }
  __syncthreads();
  for (int i = tid; i < VX * VY + UX * UY; i += kEThreads) {
    if (i < VX * VY) {
      const int ry = i / VX, rx = i % VX, x = x0 - 2 + rx, y = y0 - 3 + ry;
      if (outside(x, y)) continue;
      S.sv[ry][rx] = tap_T<1, INNER>(kDeriv, x, W, &S.sbx[ry][0], x0 - 3, 1);
    } else {
      const int j = i - VX * VY, ry = j / UX, rx = j % UX, x = x0 - 3 + rx, y = y0 - 2 + ry;
      if (outside(x, y)) continue;
      S.su[ry][rx] = tap_T<1, INNER>(kDeriv, y, H, &S.sby[0][rx], y0 - 3, BX);
    }
  }
  __syncthreads();
  for (int i = tid; i < SX * SY; i += kEThreads) {
    const int ry = i / SX, rx = i % SX, x = x0 - 2 + rx, y = y0 - 2 + ry;
    if (outside(x, y)) continue;
    S.ssb[ry][rx] = tap_T<1, INNER>(kSmooth, y, H, &S.sv[0][rx], y0 - 3, VX) +
                    tap_T<1, INNER>(kSmooth, x, W, &S.su[ry][0], x0 - 3, 1);
  }
  __syncthreads();
  for (int i = tid; i < HX * kTY; i += kEThreads) {
    const int ry = i / HX, rx = i % HX, x = x0 - 2 + rx, y = y0 + ry;
    if (outside(x, y)) continue;
    S.shb[ry][rx] = tap_T<2, INNER>(w.g5, y, H, &S.ssb[0][rx], y0 - 2, SX);
  }
  __syncthreads();
  const int tx = tid % kTX, ty = tid / kTX, x = x0 + tx, y = y0 + ty;
  float v[3] = {0.0f, 0.0f, 0.0f};
  if (INNER || (x < W && y < H)) {
    const float g = tap_T<2, INNER>(w.g5, x, W, &S.shb[ty][0], x0 - 2, 1);
    const size_t p = (size_t)(view * H + y) * W + x;
    const float* r = image + 3 * p;
    float* ad = adjoint + 3 * p;
    ad[0] += a.x * g;
    ad[1] += a.y * g;
    ad[2] += a.z * g;
    v[0] = g * r[0];
    v[1] = g * r[1];
    v[2] = g * r[2];
  }
  block_sum<3>(v, S.red);
  if (tid == 0)
    part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = make_float4(v[0], v[1], v[2], 0.0f);
}

__global__ void __launch_bounds__(kEThreads) k_edge_bwd2(const float2* __restrict__ gbar,
                                                         const float* __restrict__ image,
                                                         const float* __restrict__ T, int H, int W, EdgeW w,
                                                         float* __restrict__ adjoint, float4* __restrict__ part) {
  __shared__ Bwd2Smem S;
  const int view = blockIdx.z, x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const float3 a = luma_weights(T, view, w);
  if (x0 >= 3 && x0 + kTX + 3 <= W && y0 >= 3 && y0 + kTY + 3 <= H)
    bwd2_tile<true>(S, gbar, image, a, view, x0, y0, H, W, w, adjoint, part);
  else
    bwd2_tile<false>(S, gbar, image, a, view, x0, y0, H, W, w, adjoint, part);
}

// dT[view][r][c] += w_r sum over the view's tiles of sum gbar R_c: one block per view,
// each thread a fixed stride of tiles in double, then a fixed-order tree
__global__ void __launch_bounds__(kFinalThreads) k_edge_dT(const float4* __restrict__ part, int tiles, EdgeW w,
                                                           float* __restrict__ dT) {
  __shared__ double red[3][kFinalThreads];
  const int view = blockIdx.x;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int t = threadIdx.x; t < tiles; t += kFinalThreads) {
    const float4 v = part[(size_t)view * tiles + t];
    a += v.x;
    b += v.y;
    c += v.z;
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int s = kFinalThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 9) {
    const int r = threadIdx.x / 3, col = threadIdx.x % 3;
    dT[view * 9 + threadIdx.x] += (float)(w.gray[r] * red[col][0]);
  }
}

int grid_blocks(long long P, int threads) {
  return (int)std::min<long long>((P + threads - 1) / threads, 152LL * 16);
}

// the detector and the hysteresis for N views: k_canny (with the tiles' own unions),
// k_cc_border, k_cc_flag
int run_detector(Context* c, const float* image, const float* T, int N, int H, int W, const EdgeW& w,
                 cudaStream_t s) {
  const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, N);
  const int P = N * H * W;
  k_canny<<<grid, kEThreads, 0, s>>>(image, T, H, W, w, c->edge_gxy, c->edge_cls, c->edge_flag, c->edge_parent,
                                     c->status);
  HR_CHECK_LAUNCH();
  k_cc_border<<<grid, kEThreads, 0, s>>>(c->edge_cls, c->edge_parent, H, W, c->status);
  HR_CHECK_LAUNCH();
  k_cc_flag<<<grid_blocks(P, 256), 256, 0, s>>>(c->edge_cls, c->edge_parent, c->edge_flag, P);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

}  // namespace

int edge_buffers(Context* c) {
  if (c->edge_gxy) return HR_OK;
  const size_t P = (size_t)c->lim.max_views * c->lim.max_width * c->lim.max_height;
  const size_t tiles = (size_t)c->lim.max_views * ((c->lim.max_width + kTX - 1) / kTX) *
                       ((c->lim.max_height + kTY - 1) / kTY);
  bool ok = cudaMalloc(&c->edge_gxy, P * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&c->edge_gbar, P * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&c->edge_parent, P * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->edge_cls, P) == cudaSuccess && cudaMalloc(&c->edge_flag, P) == cudaSuccess &&
            cudaMalloc(&c->edge_gs, P) == cudaSuccess &&
            cudaMalloc(&c->edge_part, tiles * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&c->edge_scale, sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_edge_buffers(c);
    return HR_ERR_CUDA;
  }
  return HR_OK;
}

void free_edge_buffers(Context* c) {
  void* ptrs[] = {c->edge_gxy, c->edge_gbar, c->edge_parent, c->edge_cls, c->edge_flag,
                  c->edge_gs,  c->edge_part, c->edge_scale};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->edge_gxy = c->edge_gbar = nullptr;
  c->edge_parent = nullptr;
  c->edge_cls = c->edge_flag = nullptr;
  c->edge_gs = nullptr;
  c->edge_part = nullptr;
  c->edge_scale = nullptr;
}

int launch_edges(Context* c, const float* image, const float* T, int N, int H, int W, float low, float high,
                 float* edges, cudaStream_t s) {
  const EdgeW w = make_weights(low, high);
  int rc = run_detector(c, image, T, N, H, W, w, s);
  if (rc != HR_OK) return rc;
  const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, N);
  k_edge_blur<<<grid, kEThreads, 0, s>>>(c->edge_cls, c->edge_parent, c->edge_flag, c->edge_gxy, H, W, w, edges,
                                         nullptr, nullptr, nullptr, nullptr);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_edge_loss(Context* c, const float* image, const float* T, const float* edges_obs, const uint8_t* mask,
                     int N, int H, int W, float low, float high, float weight, float* loss, float* adjoint,
                     float* dT, cudaStream_t s) {
  const EdgeW w = make_weights(low, high);
  int rc = run_detector(c, image, T, N, H, W, w, s);
  if (rc != HR_OK) return rc;
  const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, N);
  const int tiles = (int)(grid.x * grid.y), n = tiles * N;
  float2* part2 = reinterpret_cast<float2*>(c->edge_part);
  k_edge_blur<<<grid, kEThreads, 0, s>>>(c->edge_cls, c->edge_parent, c->edge_flag, c->edge_gxy, H, W, w, nullptr,
                                         edges_obs, mask, c->edge_gs, part2);
  HR_CHECK_LAUNCH();
  k_edge_final<<<1, kFinalThreads, 0, s>>>(part2, n, weight, loss, c->edge_scale);
  HR_CHECK_LAUNCH();
  k_edge_bwd1<<<grid, kEThreads, 0, s>>>(c->edge_gs, c->edge_cls, c->edge_parent, c->edge_flag, c->edge_gxy, H, W,
                                         w, c->edge_scale, c->edge_gbar);
  HR_CHECK_LAUNCH();
  k_edge_bwd2<<<grid, kEThreads, 0, s>>>(c->edge_gbar, image, T, H, W, w, adjoint, c->edge_part);
  HR_CHECK_LAUNCH();
  if (dT) {
    k_edge_dT<<<N, kFinalThreads, 0, s>>>(c->edge_part, tiles, w, dT);
    HR_CHECK_LAUNCH();
  }
  return HR_OK;
}

}  // namespace hr
