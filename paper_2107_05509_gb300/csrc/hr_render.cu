// Monte Carlo ray tracing of the hand (Section 3.1, "Rendering") and its derivative
// with edge sampling for the visibility discontinuities (the renderer of Li et al.
// 2018 that the paper builds on; Section 1 and Section 3.1).
//
//   k_render_fwd       persistent blocks over 16x8 pixel tiles; per sample: Philox
//                      jitter -> primary ray -> LBVH traversal -> Moller-Trumbore ->
//                      Lambertian shading; per pixel the sample mean.
//   k_render_bwd       the same samples re-traced (no hit records are stored); at each
//                      hit the derivative of the shaded value w.r.t. the triangle's
//                      vertices (through the barycentrics at the fixed ray) and its
//                      vertex normals, accumulated in shared memory per block and
//                      written as one partial per block.
//   k_reduce_partials  fixed-order sum of the per-block partials (deterministic).
//   k_silhouettes      per view, the edges whose two faces face opposite ways as seen
//                      from the camera (plus boundary edges), compacted in id order.
//   k_edge_samples     the boundary term: samples on silhouette edges, f+ and f- by
//                      two traced rays, mapped to vertices by the projection Jacobian.
//   k_normal_dm / k_normal_gather   adjoint of the area-weighted vertex normals.
#include "hr_internal.h"

namespace hr {

namespace {

constexpr int kTileW = 16, kTileH = 8, kRenderThreads = kTileW * kTileH;

struct Hit {
  int tri;
  float t, u, v;
};

__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz, float3 o,
                                     float3 inv, float tmax_in, float& tentry) {
  float t0x = (lx - o.x) * inv.x, t1x = (hx - o.x) * inv.x;
  float t0y = (ly - o.y) * inv.y, t1y = (hy - o.y) * inv.y;
  float t0z = (lz - o.z) * inv.z, t1z = (hz - o.z) * inv.z;
  float tmin = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
  float tmax = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax_in));
  tentry = tmin;
  return tmin <= tmax;
}

__device__ __forceinline__ float safe_inv(float d) {
  return 1.0f / (fabsf(d) > 1e-20f ? d : copysignf(1e-20f, d));
}

__device__ __forceinline__ void isect(const float4* __restrict__ tris, int k, float3 o, float3 d, Hit& h) {
  float4 a = __ldg(&tris[3 * k]), b = __ldg(&tris[3 * k + 1]), c = __ldg(&tris[3 * k + 2]);
  float3 v0 = make_float3(a.x, a.y, a.z), e1 = make_float3(a.w, b.x, b.y), e2 = make_float3(b.z, b.w, c.x);
  int id = __float_as_int(c.y);
  float t, u, v;
  if (mt_hit(o, d, v0, e1, e2, t, u, v)) {
    if (t < h.t || (t == h.t && id < h.tri)) {
      h.tri = id;
      h.t = t;
      h.u = u;
      h.v = v;
    }
  }
}

// per-thread work counters of the statistics build (HR_STATS)
struct Counts {
  unsigned rays = 0, nodes = 0, tris = 0, hits = 0;
};

// closest hit against the LBVH (root = internal node 0); ties in t -> lower id
// At most `max_visits` internal nodes are visited (each node of a well-formed tree is
// visited at most once, so F-1 is never exceeded); past it the status records a
// limit error and the ray returns what it has.
template <bool STATS>
__device__ Hit trace(const Node* __restrict__ nodes, const float4* __restrict__ tris, float3 o, float3 d,
                     int* status, Counts& cnt, int max_visits) {
  Hit h{-1, INFINITY, 0.0f, 0.0f};
  float3 inv = make_float3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
  int stack[kStack];
  int sp = 0;
  int node = 0;
  for (int visits = 0;; ++visits) {
    if (visits >= max_visits) {
      set_status(status, kStatusLimit);
      break;
    }
    const float4* np = reinterpret_cast<const float4*>(nodes + node);
    if (STATS) ++cnt.nodes;
    float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
    int4 dd = __ldg(reinterpret_cast<const int4*>(np + 3));
    float tl, tr;
    bool hl = slab(a.x, a.y, a.z, a.w, b.x, b.y, o, inv, h.t, tl);
    bool hrr = slab(b.z, b.w, c.x, c.y, c.z, c.w, o, inv, h.t, tr);
    if (hl && dd.x < 0) {
      if (STATS) ++cnt.tris;
      isect(tris, ~dd.x, o, d, h);
      hl = false;
    }
    if (hrr && dd.y < 0) {
      if (STATS) ++cnt.tris;
      isect(tris, ~dd.y, o, d, h);
      hrr = false;
    }
    if (hl && hrr) {
      int nearc = dd.x, farc = dd.y;
      if (tr < tl) {
        nearc = dd.y;
        farc = dd.x;
      }
      if (sp < kStack) {
        stack[sp++] = farc;
      } else {
        set_status(status, kStatusLimit);
      }
      node = nearc;
    } else if (hl) {
      node = dd.x;
    } else if (hrr) {
      node = dd.y;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  if (STATS) {
    ++cnt.rays;
    cnt.hits += h.tri >= 0;
  }
  return h;
}

template <bool STATS>
__device__ __forceinline__ void flush_counts(const Counts& c, unsigned long long* out) {
  if (!STATS) return;
  unsigned v[4] = {c.rays, c.nodes, c.tris, c.hits};
  for (int k = 0; k < 4; ++k) {
    unsigned long long x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(out + k, x);
  }
}

struct Shading {
  float3 l, lrgb;
  float ka, kd;
};

struct RenderArgs {
  const Node* nodes;
  const float4* tris;
  const float* verts;
  const int* faces;
  const float* normals;
  const float* albedo;
  const Cam* cams;
  const float* bg;
  int N, H, W, spp, V;
  uint2 key;
  uint32_t ctr1_hi;  // instance << 16
  uint32_t iter4;    // iter << 4
  Shading sh;
  int* status;
  int max_visits;   // F (internal nodes are F - 1)
};

__device__ __forceinline__ float3 shade(const RenderArgs& a, const Hit& h) {
  int i0 = __ldg(&a.faces[3 * h.tri]), i1 = __ldg(&a.faces[3 * h.tri + 1]), i2 = __ldg(&a.faces[3 * h.tri + 2]);
  float3 n0 = ld3(a.normals + 3 * i0), n1 = ld3(a.normals + 3 * i1), n2 = ld3(a.normals + 3 * i2);
  float3 nm = interp_normal(h.u, h.v, n0, n1, n2);
  float ndl = ddot(nm, a.sh.l);
  float sigma = 0.0f;
  if (ndl > 0.0f) sigma = ndl * rsqrtf(nm.x * nm.x + nm.y * nm.y + nm.z * nm.z);
  float w = 1.0f - h.u - h.v;
  float k = a.sh.ka + a.sh.kd * sigma;
  float3 a0 = ld3(a.albedo + 3 * i0), a1 = ld3(a.albedo + 3 * i1), a2 = ld3(a.albedo + 3 * i2);
  return make_float3((w * a0.x + h.u * a1.x + h.v * a2.x) * a.sh.lrgb.x * k,
                     (w * a0.y + h.u * a1.y + h.v * a2.y) * a.sh.lrgb.y * k,
                     (w * a0.z + h.u * a1.z + h.v * a2.z) * a.sh.lrgb.z * k);
}

__device__ __forceinline__ Cam load_cam(const Cam* cams, int view) {
  Cam c;
  const float* src = reinterpret_cast<const float*>(cams + view);
  float* dst = reinterpret_cast<float*>(&c);
#pragma unroll
  for (int i = 0; i < 20; ++i) dst[i] = __ldg(src + i);
  return c;
}

__device__ __forceinline__ void jitter(const RenderArgs& a, int view, int px, int py, int s, float& u1, float& u2) {
  uint4 r = philox4x32_10(make_uint4((uint32_t)(py * a.W + px), (uint32_t)view | a.ctr1_hi, (uint32_t)s, a.iter4),
                          a.key);
  u1 = u24(r.x);
  u2 = u24(r.y);
}

// radiance through screen point (sx, sy); a miss returns background pixel (bx, by)
template <bool STATS>
__device__ __forceinline__ float3 radiance(const RenderArgs& a, const Cam& cam, int view, float sx, float sy, int bx,
                                           int by, Counts& cnt) {
  float3 o = make_float3(cam.c[0], cam.c[1], cam.c[2]);
  float3 d = primary_dir(cam, sx, sy);
  Hit h = trace<STATS>(a.nodes, a.tris, o, d, a.status, cnt, a.max_visits);
  if (h.tri >= 0) return shade(a, h);
  return ld3(a.bg + 3 * (((size_t)view * a.H + by) * a.W + bx));
}

template <bool STATS>
__global__ void __launch_bounds__(kRenderThreads) k_render_fwd(RenderArgs a, float* __restrict__ image,
                                                               unsigned long long* stats) {
  Counts cnt;
  const int tx = (a.W + kTileW - 1) / kTileW, ty = (a.H + kTileH - 1) / kTileH;
  const int per_view = tx * ty, total = a.N * per_view;
  const float inv_spp = 1.0f / (float)a.spp;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int view = tile / per_view, rem = tile - view * per_view;
    int py = (rem / tx) * kTileH + (threadIdx.x / kTileW);
    int px = (rem % tx) * kTileW + (threadIdx.x % kTileW);
    if (px >= a.W || py >= a.H) continue;
    Cam cam = load_cam(a.cams, view);
    float3 o = make_float3(cam.c[0], cam.c[1], cam.c[2]);
    size_t pix = ((size_t)view * a.H + py) * a.W + px;
    float3 acc = make_float3(0.0f, 0.0f, 0.0f);
    int misses = 0;
    for (int s = 0; s < a.spp; ++s) {
      float u1, u2;
      jitter(a, view, px, py, s, u1, u2);
      float3 d = primary_dir(cam, __fadd_rn((float)px, u1), __fadd_rn((float)py, u2));
      Hit h = trace<STATS>(a.nodes, a.tris, o, d, a.status, cnt, a.max_visits);
      if (h.tri >= 0) {
        float3 f = shade(a, h);
        acc.x += f.x;
        acc.y += f.y;
        acc.z += f.z;
      } else {
        ++misses;
      }
    }
    // misses contribute background * (misses / spp): a pixel whose samples all miss
    // is exactly its background value
    float fm = __fdiv_rn((float)misses, (float)a.spp);
    float3 bgc = misses ? ld3(a.bg + 3 * pix) : make_float3(0.0f, 0.0f, 0.0f);
    image[3 * pix] = acc.x * inv_spp + bgc.x * fm;
    image[3 * pix + 1] = acc.y * inv_spp + bgc.y * fm;
    image[3 * pix + 2] = acc.z * inv_spp + bgc.z * fm;
  }
  flush_counts<STATS>(cnt, stats);
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

__device__ __forceinline__ void add3(float* dst, int i, float x, float y, float z) {
  atomicAdd(&dst[3 * i], x);
  atomicAdd(&dst[3 * i + 1], y);
  atomicAdd(&dst[3 * i + 2], z);
}

// dL/dverts (through u, v at the fixed ray) and dL/dnormals of one shaded hit with
// upstream g = dL/df, accumulated into shared sdV = [V][3], sdN = [V][3]
__device__ __forceinline__ void hit_grad(const RenderArgs& a, const Hit& h, float3 o, float3 d, float3 g,
                                         float* sdV, float* sdN) {
  int i0 = __ldg(&a.faces[3 * h.tri]), i1 = __ldg(&a.faces[3 * h.tri + 1]), i2 = __ldg(&a.faces[3 * h.tri + 2]);
  float3 n0 = ld3(a.normals + 3 * i0), n1 = ld3(a.normals + 3 * i1), n2 = ld3(a.normals + 3 * i2);
  float3 a0 = ld3(a.albedo + 3 * i0), a1 = ld3(a.albedo + 3 * i1), a2 = ld3(a.albedo + 3 * i2);
  const float u = h.u, v = h.v, w = 1.0f - u - v;
  float3 nm = interp_normal(u, v, n0, n1, n2);
  bool lit = ddot(nm, a.sh.l) > 0.0f;
  float inv_len = rsqrtf(dot3(nm, nm));
  float3 nh = make_float3(nm.x * inv_len, nm.y * inv_len, nm.z * inv_len);
  float sigma = lit ? dot3(nh, a.sh.l) : 0.0f;
  float k = a.sh.ka + a.sh.kd * sigma;
  float3 dalb = make_float3(g.x * a.sh.lrgb.x * k, g.y * a.sh.lrgb.y * k, g.z * a.sh.lrgb.z * k);
  float3 alb = make_float3(w * a0.x + u * a1.x + v * a2.x, w * a0.y + u * a1.y + v * a2.y,
                           w * a0.z + u * a1.z + v * a2.z);
  float gu = dalb.x * (a1.x - a0.x) + dalb.y * (a1.y - a0.y) + dalb.z * (a1.z - a0.z);
  float gv = dalb.x * (a2.x - a0.x) + dalb.y * (a2.y - a0.y) + dalb.z * (a2.z - a0.z);
  if (lit) {
    float dsig = a.sh.kd * (g.x * alb.x * a.sh.lrgb.x + g.y * alb.y * a.sh.lrgb.y + g.z * alb.z * a.sh.lrgb.z);
    float3 dnh = make_float3(dsig * a.sh.l.x, dsig * a.sh.l.y, dsig * a.sh.l.z);
    float pr = dot3(nh, dnh);
    float3 dnm = make_float3((dnh.x - nh.x * pr) * inv_len, (dnh.y - nh.y * pr) * inv_len,
                             (dnh.z - nh.z * pr) * inv_len);
    gu += dnm.x * (n1.x - n0.x) + dnm.y * (n1.y - n0.y) + dnm.z * (n1.z - n0.z);
    gv += dnm.x * (n2.x - n0.x) + dnm.y * (n2.y - n0.y) + dnm.z * (n2.z - n0.z);
    add3(sdN, i0, w * dnm.x, w * dnm.y, w * dnm.z);
    add3(sdN, i1, u * dnm.x, u * dnm.y, u * dnm.z);
    add3(sdN, i2, v * dnm.x, v * dnm.y, v * dnm.z);
  }
  // barycentrics at the fixed ray: u = [s,d,e2]/D, v = [d,s,e1]/D, D = [e1,d,e2]
  float3 p0 = ld3(a.verts + 3 * i0), p1 = ld3(a.verts + 3 * i1), p2 = ld3(a.verts + 3 * i2);
  float3 s = make_float3(o.x - p0.x, o.y - p0.y, o.z - p0.z);
  float3 e1 = make_float3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z);
  float3 e2 = make_float3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z);
  float3 dxe2 = cross3(d, e2), e1xd = cross3(e1, d), dxs = cross3(d, s);
  float invD = 1.0f / dot3(e1, dxe2);
  float uv = gu * u + gv * v;
  float3 gs = make_float3((gu * dxe2.x + gv * e1xd.x) * invD, (gu * dxe2.y + gv * e1xd.y) * invD,
                          (gu * dxe2.z + gv * e1xd.z) * invD);
  float3 ge1 = make_float3((gv * dxs.x - uv * dxe2.x) * invD, (gv * dxs.y - uv * dxe2.y) * invD,
                           (gv * dxs.z - uv * dxe2.z) * invD);
  float3 ge2 = make_float3((-gu * dxs.x - uv * e1xd.x) * invD, (-gu * dxs.y - uv * e1xd.y) * invD,
                           (-gu * dxs.z - uv * e1xd.z) * invD);
  add3(sdV, i1, ge1.x, ge1.y, ge1.z);
  add3(sdV, i2, ge2.x, ge2.y, ge2.z);
  add3(sdV, i0, -(gs.x + ge1.x + ge2.x), -(gs.y + ge1.y + ge2.y), -(gs.z + ge1.z + ge2.z));
}

// interior term; shared memory: sdV [V][3] then sdN [V][3]; one partial per block
template <bool STATS>
__global__ void __launch_bounds__(kRenderThreads) k_render_bwd(RenderArgs a, const float* __restrict__ adjoint,
                                                               float* __restrict__ partials,
                                                               unsigned long long* stats) {
  extern __shared__ float sacc[];
  Counts cnt;
  float* sdV = sacc;
  float* sdN = sacc + 3 * a.V;
  for (int i = threadIdx.x; i < 6 * a.V; i += blockDim.x) sacc[i] = 0.0f;
  __syncthreads();
  const int tx = (a.W + kTileW - 1) / kTileW, ty = (a.H + kTileH - 1) / kTileH;
  const int per_view = tx * ty, total = a.N * per_view;
  const float inv_spp = 1.0f / (float)a.spp;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int view = tile / per_view, rem = tile - view * per_view;
    int py = (rem / tx) * kTileH + (threadIdx.x / kTileW);
    int px = (rem % tx) * kTileW + (threadIdx.x % kTileW);
    if (px >= a.W || py >= a.H) continue;
    size_t pix = ((size_t)view * a.H + py) * a.W + px;
    float3 A = ld3(adjoint + 3 * pix);
    if (A.x == 0.0f && A.y == 0.0f && A.z == 0.0f) continue;
    float3 g = make_float3(A.x * inv_spp, A.y * inv_spp, A.z * inv_spp);
    Cam cam = load_cam(a.cams, view);
    float3 o = make_float3(cam.c[0], cam.c[1], cam.c[2]);
    for (int s = 0; s < a.spp; ++s) {
      float u1, u2;
      jitter(a, view, px, py, s, u1, u2);
      float3 d = primary_dir(cam, __fadd_rn((float)px, u1), __fadd_rn((float)py, u2));
      Hit h = trace<STATS>(a.nodes, a.tris, o, d, a.status, cnt, a.max_visits);
      if (h.tri >= 0) hit_grad(a, h, o, d, g, sdV, sdN);
    }
  }
  flush_counts<STATS>(cnt, stats);
  __syncthreads();
  float* out = partials + (size_t)blockIdx.x * 6 * a.V;
  for (int i = threadIdx.x; i < 6 * a.V; i += blockDim.x) out[i] = sacc[i];
}

// d_verts[i] = sum_b partials[b][i] (i < 3V), dN[i-3V] = ... (fixed block order)
__global__ void k_reduce_partials(const float* __restrict__ partials, int nblocks, int V, float* __restrict__ d_verts,
                                  float* __restrict__ dN) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * V) return;
  float acc = 0.0f;
  for (int b = 0; b < nblocks; ++b) acc += partials[(size_t)b * 6 * V + i];
  if (i < 3 * V) d_verts[i] = acc;
  else dN[i - 3 * V] = acc;
}

// per view: silhouette flags in edge order, compacted by a block-wide scan
__global__ void k_silhouettes(const float* __restrict__ verts, const int* __restrict__ faces,
                              const int* __restrict__ edges, const int* __restrict__ edge_faces, int E,
                              const Cam* __restrict__ cams, int* __restrict__ lists, int stride,
                              int* __restrict__ counts) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  const int view = blockIdx.x;
  Cam cam = load_cam(cams, view);
  float3 c = make_float3(cam.c[0], cam.c[1], cam.c[2]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int e0 = 0; e0 < E; e0 += blockDim.x) {
    int e = e0 + threadIdx.x;
    bool sil = false;
    if (e < E) {
      int f2 = edge_faces[2 * e + 1];
      if (f2 < 0) {
        sil = true;
      } else {
        float3 w = dsub(ld3(verts + 3 * edges[2 * e]), c);
        int f1 = edge_faces[2 * e];
        bool s[2];
        int fs[2] = {f1, f2};
        for (int k = 0; k < 2; ++k) {
          int f = fs[k];
          float3 p0 = ld3(verts + 3 * faces[3 * f]), p1 = ld3(verts + 3 * faces[3 * f + 1]),
                 p2 = ld3(verts + 3 * faces[3 * f + 2]);
          s[k] = ddot(dcross(dsub(p1, p0), dsub(p2, p0)), w) < 0.0f;
        }
        sil = s[0] != s[1];
      }
    }
    unsigned bal = __ballot_sync(0xffffffffu, sil);
    int within = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, chunk = 0;
    for (int k = 0; k < nw; ++k) {
      int t = warp_tot[k];
      if (k < warp) before += t;
      chunk += t;
    }
    if (sil) lists[(size_t)view * stride + base + before + within] = e;
    __syncthreads();
    if (threadIdx.x == 0) base += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[view] = base;
}

// boundary term (edge sampling); one thread per (view, sample)
template <bool STATS>
__global__ void k_edge_samples(RenderArgs a, const float* __restrict__ adjoint, const int* __restrict__ edges,
                               const int* __restrict__ lists, int stride, const int* __restrict__ counts, int Ne,
                               float eps, float* __restrict__ d_verts, unsigned long long* stats) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)a.N * Ne) return;
  int view = (int)(i / Ne), k = (int)(i - (long long)view * Ne);
  int nsil = counts[view];
  if (nsil == 0) return;
  uint4 r = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)view | a.ctr1_hi, 0u, a.iter4 | 1u), a.key);
  int si = (int)__umulhi(r.x, (uint32_t)nsil);
  float t = u24(r.y);
  int e = lists[(size_t)view * stride + si];
  int ia = edges[2 * e], ib = edges[2 * e + 1];
  Cam cam = load_cam(a.cams, view);
  float3 va = ld3(a.verts + 3 * ia), vb = ld3(a.verts + 3 * ib);
  float ax, ay, bx, by;
  if (!project(cam, va, ax, ay) || !project(cam, vb, bx, by)) return;
  float x = __fmaf_rn(t, __fsub_rn(bx, ax), ax), y = __fmaf_rn(t, __fsub_rn(by, ay), ay);
  float nx = __fsub_rn(ay, by), ny = __fsub_rn(bx, ax);
  float len = __fsqrt_rn(__fmaf_rn(nx, nx, __fmul_rn(ny, ny)));
  if (!(len > 0.0f)) return;
  float nhx = __fdiv_rn(nx, len), nhy = __fdiv_rn(ny, len);
  float fxp = floorf(x), fyp = floorf(y);
  if (fxp < 0.0f || fyp < 0.0f || fxp >= (float)a.W || fyp >= (float)a.H) return;
  int px = (int)fxp, py = (int)fyp;
  float3 A = ld3(adjoint + 3 * (((size_t)view * a.H + py) * a.W + px));
  if (A.x == 0.0f && A.y == 0.0f && A.z == 0.0f) return;
  float xp = __fmaf_rn(eps, nhx, x), yp = __fmaf_rn(eps, nhy, y);
  float xm = __fmaf_rn(-eps, nhx, x), ym = __fmaf_rn(-eps, nhy, y);
  int bxp = (int)fminf(fmaxf(floorf(xp), 0.0f), (float)(a.W - 1));
  int byp = (int)fminf(fmaxf(floorf(yp), 0.0f), (float)(a.H - 1));
  int bxm = (int)fminf(fmaxf(floorf(xm), 0.0f), (float)(a.W - 1));
  int bym = (int)fminf(fmaxf(floorf(ym), 0.0f), (float)(a.H - 1));
  Counts cnt;
  float3 fp = radiance<STATS>(a, cam, view, xp, yp, bxp, byp, cnt);
  float3 fm = radiance<STATS>(a, cam, view, xm, ym, bxm, bym, cnt);
  if (STATS) {
    atomicAdd(stats + 0, (unsigned long long)cnt.rays);
    atomicAdd(stats + 1, (unsigned long long)cnt.nodes);
    atomicAdd(stats + 2, (unsigned long long)cnt.tris);
    atomicAdd(stats + 3, (unsigned long long)cnt.hits);
  }
  float wgt = (A.x * (fp.x - fm.x) + A.y * (fp.y - fm.y) + A.z * (fp.z - fm.z)) * ((float)nsil / (float)Ne);
  if (wgt == 0.0f) return;
  float dax = wgt * (by - y), day = wgt * (x - bx), dbx = wgt * (y - ay), dby = wgt * (ax - x);
  // projection Jacobians d(screen)/d(vertex)
  float3 pv[2] = {va, vb};
  float g2[2][2] = {{dax, day}, {dbx, dby}};
  int ids[2] = {ia, ib};
  for (int q = 0; q < 2; ++q) {
    float3 p = pv[q];
    float X = cam.R[0] * p.x + cam.R[1] * p.y + cam.R[2] * p.z + cam.t[0];
    float Y = cam.R[3] * p.x + cam.R[4] * p.y + cam.R[5] * p.z + cam.t[1];
    float Z = cam.R[6] * p.x + cam.R[7] * p.y + cam.R[8] * p.z + cam.t[2];
    float iz = 1.0f / Z;
    float gx = g2[q][0] * cam.fx * iz, gy = g2[q][1] * cam.fy * iz;
    float gz = -(gx * X + gy * Y) * iz;
    // J^T g = R^T (gx, gy, gz)
    atomicAdd(&d_verts[3 * ids[q]], cam.R[0] * gx + cam.R[3] * gy + cam.R[6] * gz);
    atomicAdd(&d_verts[3 * ids[q] + 1], cam.R[1] * gx + cam.R[4] * gy + cam.R[7] * gz);
    atomicAdd(&d_verts[3 * ids[q] + 2], cam.R[2] * gx + cam.R[5] * gy + cam.R[8] * gz);
  }
}

// dm_v = (I - n n^T) dN_v / |m_v|
__global__ void k_normal_dm(const float* __restrict__ normals, const float* __restrict__ normal_len,
                            const float* __restrict__ dN, int V, float* __restrict__ dm) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float len = normal_len[v];
  float3 n = ld3(normals + 3 * v), g = ld3(dN + 3 * v);
  float3 r = make_float3(0.0f, 0.0f, 0.0f);
  if (len > 0.0f) {
    float pr = dot3(n, g);
    float il = 1.0f / len;
    r = make_float3((g.x - n.x * pr) * il, (g.y - n.y * pr) * il, (g.z - n.z * pr) * il);
  }
  dm[3 * v] = r.x;
  dm[3 * v + 1] = r.y;
  dm[3 * v + 2] = r.z;
}

// d_verts[v] += sum over incident faces of d(e1 x e2)/dv . dc_f, dc_f = sum of dm over f
__global__ void k_normal_gather(const float* __restrict__ verts, const int* __restrict__ faces,
                                const int* __restrict__ vf_off, const int* __restrict__ vf_faces,
                                const float* __restrict__ dm, int V, float* __restrict__ d_verts) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float3 acc = make_float3(0.0f, 0.0f, 0.0f);
  for (int k = vf_off[v]; k < vf_off[v + 1]; ++k) {
    int f = vf_faces[k];
    int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    float3 dc = ld3(dm + 3 * i0);
    float3 t1 = ld3(dm + 3 * i1), t2 = ld3(dm + 3 * i2);
    dc = make_float3(dc.x + t1.x + t2.x, dc.y + t1.y + t2.y, dc.z + t1.z + t2.z);
    float3 p0 = ld3(verts + 3 * i0), p1 = ld3(verts + 3 * i1), p2 = ld3(verts + 3 * i2);
    float3 e1 = make_float3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z);
    float3 e2 = make_float3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z);
    float3 de1 = cross3(e2, dc), de2 = cross3(dc, e1);
    if (v == i1) {
      acc.x += de1.x; acc.y += de1.y; acc.z += de1.z;
    } else if (v == i2) {
      acc.x += de2.x; acc.y += de2.y; acc.z += de2.z;
    } else {
      acc.x -= de1.x + de2.x; acc.y -= de1.y + de2.y; acc.z -= de1.z + de2.z;
    }
  }
  d_verts[3 * v] += acc.x;
  d_verts[3 * v + 1] += acc.y;
  d_verts[3 * v + 2] += acc.z;
}

__global__ void k_trace(const Node* __restrict__ nodes, const float4* __restrict__ tris, const float* __restrict__ o,
                        const float* __restrict__ d, int n, int* __restrict__ tri, float* __restrict__ tuv, int* status,
                        int max_visits) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Counts cnt;
  Hit h = trace<false>(nodes, tris, ld3(o + 3 * i), ld3(d + 3 * i), status, cnt, max_visits);
  tri[i] = h.tri;
  tuv[3 * i] = h.t;
  tuv[3 * i + 1] = h.u;
  tuv[3 * i + 2] = h.v;
}

RenderArgs make_args(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int H, int W,
                     const float* bg, const hr_render_opts* o) {
  RenderArgs a;
  a.nodes = ctx->nodes;
  a.tris = ctx->tris;
  a.verts = verts;
  a.faces = m->faces;
  a.normals = ctx->normals;
  a.albedo = m->albedo;
  a.cams = cams;
  a.bg = bg;
  a.N = N;
  a.H = H;
  a.W = W;
  a.spp = o->spp;
  a.V = m->V;
  a.key = make_uint2((uint32_t)(o->seed & 0xffffffffull), (uint32_t)(o->seed >> 32));
  a.ctr1_hi = o->instance << 16;
  a.iter4 = o->iter << 4;
  a.sh.l = make_float3(o->light_dir[0], o->light_dir[1], o->light_dir[2]);
  a.sh.lrgb = make_float3(o->light_rgb[0], o->light_rgb[1], o->light_rgb[2]);
  a.sh.ka = o->ka;
  a.sh.kd = o->kd;
  a.status = ctx->status;
  a.max_visits = ctx->F + 1;
  return a;
}

}  // namespace

int render_grid(int device, int* blocks, int* threads, int* num_sms) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HR_ERR_CUDA;
  *num_sms = sms;
  *threads = kRenderThreads;
  *blocks = sms * 8;
  return HR_OK;
}

size_t render_bwd_smem(int V) { return (size_t)6 * V * sizeof(float); }

int launch_render_fwd(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int H, int W,
                      const float* bg, const hr_render_opts* o, float* image, cudaStream_t s) {
  RenderArgs a = make_args(ctx, m, verts, cams, N, H, W, bg, o);
  long long tiles = (long long)N * ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
  int blocks = (int)(tiles < ctx->render_blocks ? tiles : ctx->render_blocks);
  if (o->flags & HR_STATS)
    k_render_fwd<true><<<blocks, kRenderThreads, 0, s>>>(a, image, ctx->stats);
  else
    k_render_fwd<false><<<blocks, kRenderThreads, 0, s>>>(a, image, nullptr);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_silhouettes(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int* lists,
                       int list_stride, int* counts, cudaStream_t s) {
  k_silhouettes<<<N, 512, 0, s>>>(verts, m->faces, m->edges, m->edge_faces, m->E, cams, lists, list_stride, counts);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_render_bwd(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int H, int W,
                      const float* bg, const hr_render_opts* o, const float* adjoint, float* d_verts,
                      cudaStream_t s) {
  RenderArgs a = make_args(ctx, m, verts, cams, N, H, W, bg, o);
  const int V = m->V;
  const bool interior = !(o->flags & HR_BWD_NO_INTERIOR);
  const bool edges = !(o->flags & HR_BWD_NO_EDGES) && o->edge_samples > 0;
  const bool normals = !(o->flags & HR_BWD_NO_NORMALS) && interior;
  if (interior) {
    size_t smem = render_bwd_smem(V);
    const bool st = o->flags & HR_STATS;
    auto kern = st ? k_render_bwd<true> : k_render_bwd<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return HR_ERR_CUDA;
    int blocks = ctx->render_blocks;
    kern<<<blocks, kRenderThreads, smem, s>>>(a, adjoint, ctx->partials, st ? ctx->stats + 4 : nullptr);
    HR_CHECK_LAUNCH();
    k_reduce_partials<<<(6 * V + 255) / 256, 256, 0, s>>>(ctx->partials, blocks, V, d_verts, ctx->dN);
    HR_CHECK_LAUNCH();
  } else {
    if (cudaMemsetAsync(d_verts, 0, sizeof(float) * 3 * V, s) != cudaSuccess) return HR_ERR_CUDA;
  }
  if (edges) {
    int rc = launch_silhouettes(ctx, m, verts, cams, N, ctx->sil, ctx->lim.max_E, ctx->sil_count, s);
    if (rc != HR_OK) return rc;
    long long n = (long long)N * o->edge_samples;
    auto kern = (o->flags & HR_STATS) ? k_edge_samples<true> : k_edge_samples<false>;
    kern<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a, adjoint, m->edges, ctx->sil, ctx->lim.max_E, ctx->sil_count,
                                                     o->edge_samples, o->edge_eps_px, d_verts, ctx->stats + 8);
    HR_CHECK_LAUNCH();
  }
  if (normals) {
    k_normal_dm<<<(V + 255) / 256, 256, 0, s>>>(ctx->normals, ctx->normal_len, ctx->dN, V, ctx->dm);
    HR_CHECK_LAUNCH();
    k_normal_gather<<<(V + 255) / 256, 256, 0, s>>>(verts, m->faces, m->vf_offsets, m->vf_faces, ctx->dm, V, d_verts);
    HR_CHECK_LAUNCH();
  }
  return HR_OK;
}

int launch_trace(Context* ctx, const float* o, const float* d, int n, int* tri, float* tuv, cudaStream_t s) {
  k_trace<<<(n + 127) / 128, 128, 0, s>>>(ctx->nodes, ctx->tris, o, d, n, tri, tuv, ctx->status, ctx->F + 1);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

}  // namespace hr
