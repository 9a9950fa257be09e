// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the learned proposal
// network: C[M][N] = act(A[M][K] B[N][K]^T + bias), A and B bf16 with K contiguous,
// accumulation in float32 in tensor memory, C stored as bf16 or float32.
//
// One CTA computes a 128 x BN tile of C:
//   warp 0      TMA producer: 128 x 64 tiles of A and BN x 64 tiles of B into a ring of
//               shared-memory stages (128-byte swizzle), one mbarrier per stage that
//               completes when both copies have landed
//   warp 1      allocates BN tensor-memory columns; one thread issues the
//               tcgen05.mma (M = 128, N = BN, K = 16) of every stage and commits each
//               stage back to the producer, and the last one to the epilogue
//   warps 2-5   epilogue: tcgen05.ld of the accumulator rows of their lane quarter,
//               bias, ReLU, conversion, stores
// Split-K (gridDim.z > 1): CTA z takes K range z of gridDim.z and writes float32
// partials to C + z * ldc_split (no bias, no activation); a separate reduction sums
// them in split order.
//
// Every mbarrier wait is bounded (about one second of device time); a wait that
// runs out sets a status bit, the CTA stops issuing work, waits (bounded) for its own
// copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "hr_internal.h"

namespace hr {

namespace {

constexpr int kBM = 128, kBK = 64, kStages = 3, kGemmThreads = 192;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase of `parity` to complete; false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > 1000000000ull) return false;   // 1 s
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major operand tile whose rows are 128
// bytes (64 bf16), 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// instruction descriptor of kind::f16: bf16 x bf16 -> f32, both K-major, M x N
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct GemmArgs {
  int M, N, K;
  int kt_per_split;    // 64-wide K steps per split
  const float* bias;   // [N] or null
  int relu;
  void* C;
  int ldc;             // elements
  long long split_stride;   // elements between split outputs (split-K partials)
  int out_bf16;
  int* status;
};

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_bf16(const __grid_constant__ CUtensorMap tmA,
                                                               const __grid_constant__ CUtensorMap tmB,
                                                               GemmArgs g) {
  constexpr int kTmemCols = BN < 32 ? 32 : BN;
  constexpr uint32_t kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  // 1024-byte aligned stage buffers (the 128-byte swizzle pattern repeats every 1024 B)
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = base;
  unsigned char* sB = base + kStages * kABytes;
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int kt0 = blockIdx.z * g.kt_per_split;
  const int kt_total = (g.K / kBK);
  const int nkt = max(0, min(g.kt_per_split, kt_total - kt0));

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer
    int issued = 0;
    for (int kt = 0; kt < nkt; ++kt) {
      const int s = kt % kStages;
      if (kt >= kStages && !mbar_wait(smem_u32(&empty_bar[s]), ((kt / kStages) + 1) & 1)) {
        set_status(g.status, kStatusTimeout);
        atomicExch(&abort_flag, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(&abort_flag)) break;
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, kABytes + kBBytes);
      tma_load_2d(smem_u32(sA + s * kABytes), &tmA, (kt0 + kt) * kBK, m0, fb);
      tma_load_2d(smem_u32(sB + s * kBBytes), &tmB, (kt0 + kt) * kBK, n0, fb);
      ++issued;
    }
    // copies still in flight must land before the CTA may exit
    for (int kt = max(0, issued - kStages); kt < issued; ++kt)
      mbar_wait(smem_u32(&full_bar[kt % kStages]), (kt / kStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = mma_idesc(kBM, BN);
    bool ok = true;
    for (int kt = 0; kt < nkt; ++kt) {
      const int s = kt % kStages;
      if (!mbar_wait(smem_u32(&full_bar[s]), (kt / kStages) & 1)) {
        set_status(g.status, kStatusTimeout);
        atomicExch(&abort_flag, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k)
        mma_bf16(tmem, sw128_desc(a0 + k * 32), sw128_desc(b0 + k * 32), idesc, (kt > 0 || k > 0) ? 1u : 0u);
      mma_commit(smem_u32(&empty_bar[s]));   // the stage is free once these MMAs have read it
    }
    if (ok && nkt > 0) mma_commit(smem_u32(&done_bar));
    if (!ok || nkt == 0) {
      // nothing (more) will be computed: release the epilogue
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&done_bar)) : "memory");
    }
  } else if (warp >= 2) {
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 = tile rows
    const bool ok = mbar_wait(smem_u32(&done_bar), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      set_status(g.status, kStatusTimeout);
    } else if (!*reinterpret_cast<volatile int*>(&abort_flag)) {
      const int q = warp & 3;
      const int row = m0 + q * 32 + lane;
      const bool split = gridDim.z > 1;
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        if (nkt > 0) {
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.0f;
        }
        if (row >= g.M) continue;
        const int col = n0 + c;
        if (!split) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (g.bias && col + i < g.N) v[i] += g.bias[col + i];
            if (g.relu) v[i] = fmaxf(v[i], 0.0f);
          }
        }
        if (g.out_bf16) {
          __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(g.C) + (size_t)row * g.ldc + col;
          if (col + 16 <= g.N && ((reinterpret_cast<uintptr_t>(out) & 15) == 0)) {
            uint32_t w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
              w[i] = *reinterpret_cast<uint32_t*>(&h);
            }
            reinterpret_cast<uint4*>(out)[0] = make_uint4(w[0], w[1], w[2], w[3]);
            reinterpret_cast<uint4*>(out)[1] = make_uint4(w[4], w[5], w[6], w[7]);
          } else {
            for (int i = 0; i < 16 && col + i < g.N; ++i) out[i] = __float2bfloat16_rn(v[i]);
          }
        } else {
          float* out = reinterpret_cast<float*>(g.C) + (split ? blockIdx.z * g.split_stride : 0) +
                       (size_t)row * g.ldc + col;
          if (col + 16 <= g.N && ((reinterpret_cast<uintptr_t>(out) & 15) == 0)) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              reinterpret_cast<float4*>(out)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          } else {
            for (int i = 0; i < 16 && col + i < g.N; ++i) out[i] = v[i];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// fixed-order sum of split-K partials: out[i] = act(sum_z part[z][i] + bias[col])
__global__ void k_split_reduce(const float* __restrict__ part, int splits, long long stride, int M, int N, int ldc,
                               const float* __restrict__ bias, int relu, void* out, int ldo, int out_bf16) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)M * N) return;
  const int r = (int)(i / N), c = (int)(i % N);
  float acc = 0.0f;
  for (int z = 0; z < splits; ++z) acc += part[z * stride + (size_t)r * ldc + c];
  if (bias) acc += bias[c];
  if (relu) acc = fmaxf(acc, 0.0f);
  if (out_bf16)
    reinterpret_cast<__nv_bfloat16*>(out)[(size_t)r * ldo + c] = __float2bfloat16_rn(acc);
  else
    reinterpret_cast<float*>(out)[(size_t)r * ldo + c] = acc;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_encode_mutex;
EncodeTiledFn g_encode = nullptr;

EncodeTiledFn encode_fn() {
  std::lock_guard<std::mutex> lock(g_encode_mutex);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return g_encode;
}

// 2-D bf16 tensor map over rows x K (K contiguous, row pitch ld elements), box 64 x box_rows
bool make_map(CUtensorMap* map, const void* ptr, int rows, int K, int ld, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
size_t gemm_smem() {
  return 1024 + (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2);
}

template <int BN>
int launch_gemm_bn(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int splits, cudaStream_t s) {
  const size_t smem = gemm_smem<BN>();
  dim3 grid((g.M + kBM - 1) / kBM, (g.N + BN - 1) / BN, splits);
  k_gemm_bf16<BN><<<grid, kGemmThreads, smem, s>>>(ta, tb, g);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

}  // namespace

int configure_gemm_kernels() {
  if (cudaFuncSetAttribute(k_gemm_bf16<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<32>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_gemm_bf16<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<64>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_gemm_bf16<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<128>()) !=
          cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  return HR_OK;
}

int launch_gemm(const void* A, int lda, const void* Bm, int ldb, int M, int N, int K, const float* bias, int relu,
                void* C, int ldc, int out_bf16, int splits, float* split_buf, int* status, cudaStream_t s) {
  if (M < 1 || N < 1 || K < kBK || K % kBK != 0 || lda < K || ldb < K || lda % 8 || ldb % 8 || splits < 1)
    return HR_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bm)) & 15) return HR_ERR_ARG;
  const int BN = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K, lda, kBM) || !make_map(&tb, Bm, N, K, ldb, BN)) return HR_ERR_CUDA;
  const int kt_total = K / kBK;
  if (splits > kt_total) splits = kt_total;
  GemmArgs g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.kt_per_split = (kt_total + splits - 1) / splits;
  splits = (kt_total + g.kt_per_split - 1) / g.kt_per_split;
  g.status = status;
  if (splits > 1) {
    if (!split_buf) return HR_ERR_ARG;
    g.bias = nullptr;
    g.relu = 0;
    g.C = split_buf;
    g.ldc = N;
    g.split_stride = (long long)M * N;
    g.out_bf16 = 0;
  } else {
    g.bias = bias;
    g.relu = relu;
    g.C = C;
    g.ldc = ldc;
    g.split_stride = 0;
    g.out_bf16 = out_bf16;
  }
  int rc = BN == 32 ? launch_gemm_bn<32>(ta, tb, g, splits, s)
                    : (BN == 64 ? launch_gemm_bn<64>(ta, tb, g, splits, s) : launch_gemm_bn<128>(ta, tb, g, splits, s));
  if (rc != HR_OK || splits == 1) return rc;
  const long long n = (long long)M * N;
  k_split_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(split_buf, splits, (long long)M * N, M, N, N, bias, relu,
                                                             C, ldc, out_bf16);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

}  // namespace hr
