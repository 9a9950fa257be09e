// Device-side building blocks shared by the handrt kernels: the context layout,
// Philox4x32-10 sample streams, and the float32 "decision arithmetic" -- every
// operation whose result decides a branch or an integer (which triangle a sample
// hits, lit or unlit, silhouette or not, which pixel an edge sample lands in) is
// written with explicitly rounded intrinsics (__fmul_rn, __fadd_rn, __fsub_rn,
// __fdiv_rn, __fsqrt_rn, __fmaf_rn), so the compiler cannot contract or reorder it
// and the result is the same float32 value on every run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/handrt.h"

namespace hr {

constexpr int kStack = 64;          // BVH traversal stack entries per ray
constexpr int kStatusLimit = 1;     // device status bits
constexpr int kStatusNonfinite = 2;
constexpr int kStatusBadModel = 4;  // a face or parent index out of range
constexpr int kStatusIndex = 8;     // an internal index read from device memory out of range
constexpr int kStatusTimeout = 16;  // a bounded device-side wait ran out
// HR_TIMING event slots: forward gather/shade/combine, backward gather/shade/reduce/
// silhouettes/edges/normal adjoint
constexpr int kTimeFwdGather = 0, kTimeFwdShade = 1, kTimeFwdCombine = 2, kTimeBwdGather = 3, kTimeBwdShade = 4,
              kTimeBwdReduce = 5, kTimeBwdSil = 6, kTimeBwdEdges = 7, kTimeBwdNormals = 8, kTimeSlots = 9;

// ---------------------------------------------------------------------------------
// BVH layout (binary LBVH, F-1 internal nodes, leaves = triangle records)
//   node n: float4 a = (lminx, lminy, lminz, lmaxx)
//           float4 b = (lmaxy, lmaxz, rminx, rminy)
//           float4 c = (rminz, rmaxx, rmaxy, rmaxz)
//           int4   d = (left, right, -, -); child >= 0: internal node, < 0: leaf ~idx
//   triangle record k (in Morton order): float4 (v0.xyz, e1.x), (e1.yz, e2.xy),
//                                        (e2.z, tri_id bits, 0, 0)
// ---------------------------------------------------------------------------------
struct Node {
  float4 a, b, c;
  int4 d;
};

// Batch layout (hr_batch_create): instances of one hand model, each with its own
// parameters, cameras, resolution, samples per pixel and edge samples.  Views are
// numbered instance-major; sub-tiles and pixels are numbered view-major within that,
// so every per-instance buffer is one contiguous range.
struct ViewRec {
  int inst;         // instance of this view
  uint32_t ctr1;    // Philox counter word: view index within the instance | instance << 16
  int H, W;
  int spp;
  int ne;           // edge samples of this view
  int st0;          // first sub-tile of the view (global numbering)
  int nsx;          // sub-tiles per row
  long long pix0;   // first pixel of the view (global numbering)
};
struct InstRec {
  int view0, nviews;   // global views [view0, view0 + nviews)
  long long pix0, npix;
  uint32_t ctr1_hi;    // Philox instance field << 16
  int spp, ne;
  int ibase, icap;     // the instance's region of the work-item table
  int st0, nst;        // the instance's sub-tiles
};

struct Context {
  hr_limits lim;
  // batch layout: n_inst == 1 and vt == nullptr for a single-instance context
  int n_inst;
  int nviews;
  int total_st;
  long long total_pix;
  int max_ne;            // largest edge-sample count of a view
  bool loss_vec;         // every instance's first pixel is a multiple of 4
  ViewRec* vt;           // device [nviews]
  const int* active;     // device [n_inst] of a batch: instances with 0 are skipped, or
                         // NULL (every instance); hr_batch_set_active
  int* act_off;          // device [2][n_inst + 1] of a batch: prefix sums over the active
                         // instances of their sub-tiles (row 0) and views (row 1)
  InstRec* it;           // device [n_inst]
  ViewRec* hvt;          // host copies
  InstRec* hit;
  int device;
  int num_sms;
  int render_blocks;     // largest persistent grid of the render kernels
  int render_threads;
  hr_tuning tune;        // launch shapes (hr_set_tuning)
  // scene, one per instance (per-instance arrays are [n_inst][...], contiguous)
  int V, F;              // sizes of the last hr_build_bvh
  unsigned bvh_gen;      // builds so far
  int* bvh_parent;       // [n_inst][2 max_F] parents of the internal nodes and leaves
  int* bvh_valid;        // [n_inst] 1 once a tree of bvh_faces exists (refits need it)
  const int* bvh_faces;  // the face array of the last build
  // one-block trees: hr_update_bvh's refit iterations rewrite only the triangle
  // records and mark the boxes stale; a render call refits them when one of its
  // sub-tiles needs per-ray traversal (the shared-memory layout of the last update)
  int* bvh_stale;        // [n_inst] boxes older than the records
  int* bvh_need;         // [n_inst] this forward has a sub-tile without a candidate list
  bool bvh_lazy;         // the last update was a one-block build or record update
  int bvh_P;             // its key count (power of two >= F)
  size_t bvh_smem;       // its dynamic shared memory
  bool bvh_snodes;       // its nodes held in shared memory
  // multi-block build (meshes beyond one block's shared memory)
  int bvh_pmax;                  // keys per instance (power of two >= max_F)
  unsigned long long* bvh_keys;  // [n_inst][bvh_pmax]
  int* bvh_flags;                // [n_inst][max_F] refit arrival counters
  unsigned* bvh_bounds;          // [n_inst][6] centroid bounds (order-preserving)
  int* bvh_bad;                  // [n_inst] a face index out of range
  int* bvh_mode;                 // [n_inst] this call: 1 refit, 0 full build
  // the last forward render (its candidate pool serves a backward with
  // HR_BWD_REUSE_FWD): vertices, cameras, sizes and the build it used
  const void* fwd_verts;
  const void* fwd_cams;
  int fwd_N, fwd_H, fwd_W, fwd_spp;
  unsigned fwd_gen;
  bool fwd_valid;
  Node* nodes;           // [n_inst][max_F]
  float4* tris;          // [n_inst][max_F][3]
  float* normals;        // [n_inst][max_V][3] unit vertex normals
  float* normal_len;     // [n_inst][max_V]    |m_v|
  // sub-tile candidate pool and work items of the render kernels
  float4* pool_bb;       // [pool_cap]
  float* pool_z;         // [pool_cap]
  int* pool_rec;         // [pool_cap]
  int pool_cap;
  int2* st_info;         // [sub-tiles]
  int4* items;           // [item_cap], one region per instance
  float4* item_part;     // [item_cap][32]
  int item_cap;
  float* extra;          // [n_inst][max_V][6]
  double* extra64;       // [n_inst][max_V][6] backward sums when max_V > 8192
  unsigned* work_ctr;    // [3 + 2 n_inst]
  int* ovf_list;         // [sub-tiles] sub-tiles whose items overflowed their region
  int* trace_list;       // [item_cap] items of sub-tiles without a candidate list (per-ray traversal)
  unsigned* st_done;     // [sub-tiles] forward items finished per sub-tile (zero between launches)
  int4* cand_st;         // [sub-tiles] forward lists to sort: (sub-tile, pool offset, K, 0)
  unsigned* bin_cnt;     // [sub-tiles] records binned per sub-tile (zeroed by every forward)
  // backward scratch
  float* partials;       // [render_blocks][max_V][6] (single-instance contexts)
  float* dN;             // [n_inst][max_V][3]
  float* dedge;          // [n_inst][max_V][3] the edge-sampling term's vertex sums
  unsigned long long* acc_fx;   // [n_inst][max_V][6] fixed-point backward sums (HR_DETERMINISTIC)
  cudaStream_t side;     // the edge-sampling term runs here, beside the interior term
  cudaEvent_t ev_fork, ev_join;
  int* sil;              // [views][max_E]
  int* sil_count;        // [views]
  // loss scratch: per instance kLossStride(loss_blocks) floats
  float* loss_partials;
  int loss_blocks;       // blocks per instance of the loss kernels
  float* ct_partials;    // [max_views][64][10] colour-transformed loss partials
  unsigned int* counters;// [n_inst][4] last-block counters (mask count, loss, skin adjoint)
  // skin scratch
  float* skin_partials;  // [n_inst][kSkinBlocks][kSkinAcc]
  // edge-term scratch (single-instance contexts; allocated by the first edge call),
  // per pixel of max_views x max_height x max_width
  float2* edge_gxy;      // Sobel gradient of the last detector run
  float2* edge_gbar;     // adjoint of the gradient
  int* edge_parent;      // union-find parents of the candidates (-1 elsewhere)
  uint8_t* edge_cls;     // bit 0 candidate, bit 1 strong
  uint8_t* edge_flag;    // a component root holding a strong pixel
  int8_t* edge_gs;       // M sign(E_hat_r - E_hat_o)
  float4* edge_part;     // per-tile partial sums
  float* edge_scale;     // weight / sum M of the last edge loss
  // kernel timing (HR_TIMING): events around the render kernels of the last call
  cudaEvent_t ev[32];          // >= 2 * kTimeSlots
  int ev_ready;
  // status and work counters
  int* status;
  unsigned long long* stats;  // [3][kStatsPer]
};

// work counters of the render kernels for n instances: 3 + 3n words, the trace-list
// count, the count of lists to sort, then (from an even word) one 64-bit item-allocation
// word per instance
__host__ __device__ constexpr int ctr_trace(int n) { return 3 + 3 * n; }
__host__ __device__ constexpr int ctr_sort(int n) { return 4 + 3 * n; }
__host__ __device__ constexpr int ctr_alloc_base(int n) { return (5 + 3 * n + 1) & ~1; }
__host__ __device__ constexpr int ctr_words(int n) { return ctr_alloc_base(n) + 2 * n; }
// meshes up to this many vertices take float backward sums (per block of the shader
// in a single-instance context); larger ones float64 sums
constexpr int kPartialMaxV = 8192;
constexpr int kLossBlocks = 304;         // loss blocks of a single-instance context (2 per SM of a GB300)
constexpr int kLossBlocksBatch = 128;    // per instance in a batch
// per-instance loss scratch: block counts (u64), block sums, 1 / (3 sum M), padding
__host__ __device__ constexpr int kLossStride(int blocks) { return 4 * blocks + 8; }
constexpr int kStatsPer = 6;   // samples, rays, BVH nodes, triangle tests, hits, candidate box tests
constexpr int kSkinBlocks = 64;
constexpr int kSkinAcc = 16 * 12 + 10 + 3;   // dA_j (J=16 x 3x4), dbeta, dtau
constexpr int kMaxJ = 16;
constexpr int kMaxK = 10;

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// uniform in [0, 1): the top 24 bits, exact in float32
__device__ __forceinline__ float u24(uint32_t r) {
  return __fmul_rn(__uint2float_rn(r >> 8), 5.9604644775390625e-08f);
}

// ---------------------------------------------------------------------------------
// float32 decision arithmetic
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float3 dsub(float3 a, float3 b) {
  return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ float3 dcross(float3 a, float3 b) {
  return make_float3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
                     __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float ddot(float3 a, float3 b) {
  return __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, __fmul_rn(a.z, b.z)));
}

struct Cam {
  float fx, fy, cx, cy, R[9], t[3], c[3], pad;
};
static_assert(sizeof(Cam) == sizeof(hr_camera), "camera layout");

// world-space direction of the primary ray through screen point (sx, sy)
__device__ __forceinline__ float3 primary_dir(const Cam& cam, float sx, float sy) {
  float dcx = __fdiv_rn(__fsub_rn(sx, cam.cx), cam.fx);
  float dcy = __fdiv_rn(__fsub_rn(sy, cam.cy), cam.fy);
  return make_float3(__fmaf_rn(cam.R[0], dcx, __fmaf_rn(cam.R[3], dcy, cam.R[6])),
                     __fmaf_rn(cam.R[1], dcx, __fmaf_rn(cam.R[4], dcy, cam.R[7])),
                     __fmaf_rn(cam.R[2], dcx, __fmaf_rn(cam.R[5], dcy, cam.R[8])));
}

// Moller-Trumbore, double-sided; true on a hit with t > 0
__device__ __forceinline__ bool mt_hit(float3 o, float3 d, float3 v0, float3 e1, float3 e2, float& t,
                                       float& u, float& v) {
  float3 p = dcross(d, e2);
  float det = ddot(e1, p);
  if (det == 0.0f) return false;
  float inv = __fdiv_rn(1.0f, det);
  float3 s = dsub(o, v0);
  u = __fmul_rn(ddot(s, p), inv);
  float3 q = dcross(s, e1);
  v = __fmul_rn(ddot(d, q), inv);
  t = __fmul_rn(ddot(e2, q), inv);
  return u >= 0.0f && u <= 1.0f && v >= 0.0f && __fadd_rn(u, v) <= 1.0f && t > 0.0f;
}

// lit/unlit decision: sign of n_interp . l with n_interp = w n0 + u n1 + v n2
__device__ __forceinline__ float3 interp_normal(float u, float v, float3 n0, float3 n1, float3 n2) {
  float w = __fsub_rn(__fsub_rn(1.0f, u), v);
  return make_float3(__fmaf_rn(v, n2.x, __fmaf_rn(u, n1.x, __fmul_rn(w, n0.x))),
                     __fmaf_rn(v, n2.y, __fmaf_rn(u, n1.y, __fmul_rn(w, n0.y))),
                     __fmaf_rn(v, n2.z, __fmaf_rn(u, n1.z, __fmul_rn(w, n0.z))));
}

// pinhole projection of a vertex to screen; false when Z <= 1e-3
__device__ __forceinline__ bool project(const Cam& cam, float3 p, float& ax, float& ay) {
  float X = __fmaf_rn(cam.R[0], p.x, __fmaf_rn(cam.R[1], p.y, __fmaf_rn(cam.R[2], p.z, cam.t[0])));
  float Y = __fmaf_rn(cam.R[3], p.x, __fmaf_rn(cam.R[4], p.y, __fmaf_rn(cam.R[5], p.z, cam.t[1])));
  float Z = __fmaf_rn(cam.R[6], p.x, __fmaf_rn(cam.R[7], p.y, __fmaf_rn(cam.R[8], p.z, cam.t[2])));
  if (!(Z > 1e-3f)) return false;
  ax = __fmaf_rn(cam.fx, __fdiv_rn(X, Z), cam.cx);
  ay = __fmaf_rn(cam.fy, __fdiv_rn(Y, Z), cam.cy);
  return true;
}

__device__ __forceinline__ float3 ld3(const float* p) { return make_float3(p[0], p[1], p[2]); }

__device__ __forceinline__ void set_status(int* status, int bit) { atomicOr(status, bit); }

// Programmatic dependent launch: kernels on the iteration's critical path are
// launched with launch_pdl, so their launch is processed while the kernel before them
// in the stream finishes.  Each such kernel calls pdl_wait() before its first access
// to device memory: it returns once the previous grid has completed and its writes
// are visible (without the launch attribute, at once).  No kernel signals its
// dependents early: blocks of the next kernel waiting beside a running one took SM
// slots from it (the backward lost 22 us per iteration), so each dependent grid
// starts when its predecessor's blocks have exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace hr

// launch helpers implemented per translation unit; every host entry returns an HR code
#define HR_CHECK_LAUNCH()                                   \
  do {                                                      \
    if (cudaPeekAtLastError() != cudaSuccess) {             \
      cudaGetLastError();                                   \
      return HR_ERR_CUDA;                                   \
    }                                                       \
  } while (0)
