// Monte Carlo ray tracing of the hand (Section 3.1, "Rendering") and its derivative
// with edge sampling for the visibility discontinuities (the renderer of Li et al.
// 2018 that the paper builds on; Section 1 and Section 3.1).
//
// Primary rays of a pinhole camera are coherent, so the forward and the interior
// backward work on 8x4-pixel sub-tiles, one warp per sub-tile at a time.
//
// Candidate lists (forward).  A sample can hit a triangle only if the sample lies in
// the triangle's screen box (padded by half a pixel), and every shader tests that box
// before intersecting, so a sub-tile needs the triangle records whose boxes meet it:
//   k_bin (count)  each (view, record) pair counts itself into the sub-tiles its box
//                  meets;
//   k_bin_alloc    each sub-tile gets a pool range for its K records and 1-16 work
//                  items of consecutive samples (more for longer lists, so no single
//                  warp holds up the launch);
//   k_background   sub-tiles that no record meets get the background (second stream);
//   k_bin (fill)   the pairs write their records, boxes and depths into the ranges;
//   k_bin_sort     each list is sorted by nearest camera depth.
// k_gather (a frustum walk of the LBVH per sub-tile) makes the backward's own lists
// when the forward's cannot be reused.
//
// Shading:
//   k_shade_fwd    warps take work items; each lane (pixel) makes its samples
//                  (Philox jitter) and walks the candidates that can hold a sample of
//                  its pixel (a bit transpose of the warp's box-against-pixel tests),
//                  in depth order, with the same float32 Moller-Trumbore test and
//                  closest-hit rule as a per-ray traversal, stopping at the first
//                  candidate nearer than none of its hits; shades, and writes per-item
//                  sums.  The warp finishing a sub-tile's last item sums the items in
//                  item order (deterministic) and writes the pixels.
//   k_shade_bwd    the same samples re-traced (no hit records are kept between
//                  the passes); every hit is differentiated at the fixed ray and the
//                  gradient accumulated per run of hits on one triangle in registers,
//                  summed over the warp, and added into one partial per SM.
//   k_reduce_partials  fixed-order sum of the partials.
//
// Per-ray LBVH traversal (trace) serves the hr_trace entry point and the sub-tiles
// with more candidates than a list holds (k_overflow, and edge rays landing there).
//   k_silhouettes  per view, edges whose faces face opposite ways from the camera
//                  (plus boundary edges), compacted in edge order.
//   k_edge_samples the boundary term: samples on silhouette edges, f+ and f- by
//                  two rays over the candidate list of the sample's sub-tile, mapped
//                  to vertices by the projection Jacobian.
//   k_normal_gather  adjoint of the area-weighted vertex normals.
//
// Batches (hr_batch_create): every kernel runs over all instances of the batch in
// one launch.  Sub-tiles are numbered over all views of all instances (a view table
// maps a sub-tile to its view, instance, resolution and samples per pixel); each
// instance has its own BVH, vertices, normals and region of the work-item table.
// Warps take items instance after instance; a batch's backward adds each run's sums
// straight into its instance's gradient.  A single-instance call is a batch of one
// with a uniform view layout (no table).
#include <type_traits>

#include "hr_internal.h"

namespace hr {

namespace {

constexpr int kRenderThreads = 128;   // 4 warps per block
constexpr int kWarps = kRenderThreads / 32;
constexpr int kBwdMinBlocks = 4;      // launch bound of the backward shader (128 registers)
constexpr int kBlocksPerSm = 8;       // largest persistent grid; backward partials are sized for it
constexpr int kSubW = 8, kSubH = 4;   // sub-tile; lane = pixel
constexpr int kLeafCap = 512;         // candidates per sub-tile
constexpr int kFrontCap = 256;        // breadth-first frontier per level (dense meshes need the width)

// Self-check of an index read from device memory (BVH children, candidate records,
// pool offsets, work items): out of range sets a status bit and the caller skips
// the access.
__device__ __forceinline__ bool in_range(int* status, long long i, long long lo, long long hi) {
  if (i >= lo && i < hi) return true;
  set_status(status, kStatusIndex);
  return false;
}

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

// reciprocal for the slab tests only (never for a hit decision): the approximate
// reciprocal is off by a couple of ulp, far inside the padding of the leaf boxes
__device__ __forceinline__ float safe_inv(float d) {
  return __fdividef(1.0f, fabsf(d) > 1e-20f ? d : copysignf(1e-20f, d));
}

// work counters of the statistics build (HR_STATS): estimator samples resolved,
// rays made individually, BVH nodes visited, Moller-Trumbore tests, hits, candidate
// screen-box tests
struct Counts {
  unsigned samples = 0, rays = 0, nodes = 0, tris = 0, hits = 0, cands = 0;
};

template <bool STATS>
__device__ __forceinline__ void isect(const float4* __restrict__ tris, int k, float3 o, float3 d, Hit& h,
                                      Counts& cnt) {
  if (STATS) ++cnt.tris;
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

// Closest hit against the LBVH (root = internal node 0); ties in t go to the lower
// triangle id.  At most `max_visits` internal nodes are visited (a well-formed tree
// never needs more than F - 1); past it the status records a limit error.
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
      isect<STATS>(tris, ~dd.x, o, d, h, cnt);
      hl = false;
    }
    if (hrr && dd.y < 0) {
      isect<STATS>(tris, ~dd.y, o, d, h, cnt);
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
  return h;
}

template <bool STATS>
__device__ __forceinline__ void flush_counts(const Counts& c, unsigned long long* out) {
  if (!STATS) return;
  unsigned v[kStatsPer] = {c.samples, c.rays, c.nodes, c.tris, c.hits, c.cands};
  for (int k = 0; k < kStatsPer; ++k) {
    unsigned long long x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(out + k, x);
  }
}

struct Shading {
  float3 l, lrgb;
  float ka, kd;
};

// candidate pool and work items shared by the gather / shade / combine kernels
struct Work {
  float4* bb;      // [pool] screen box (x0, y0, x1, y1) of the candidate
  float* z;        // [pool] nearest camera depth (sorted within a sub-tile)
  int* rec;        // [pool] triangle record
  int pool_cap;
  int2* st;        // [sub-tiles] (pool offset, K): K = 0 no ray can hit, K < 0 per-ray
                   // traversal (-1: too many candidates; -(n + 1): n found no pool room)
  int4* items;     // [items] (sub-tile, chunk, chunks, first item of the sub-tile)
  int item_cap;
  float4* part;    // [items][32] forward per-item sums (r, g, b, misses)
  double* extra64; // [n_inst][6V] backward sums of meshes beyond shared memory (float64
                   // atomics: long runs of cancelling contributions)
  float* extra;    // [n_inst][6V] backward sums: shading blocks of a batch, and work
                   // done outside the shading blocks
  unsigned* ctr;   // [ctr_words(n_inst)] sub-tile counter, pool fill, per instance
                   // front items and taken items, the overflow count, per instance back
                   // items, then per instance a 64-bit allocation word
  int* ovf;        // [sub-tiles] sub-tiles whose items did not fit their instance's
                   // region (k_overflow does them whole)
  int* trace;      // [items] region slots (+ instance base) of the items of sub-tiles
                   // without a candidate list (k_overflow traces them ray by ray)
  unsigned* st_done;   // [sub-tiles] forward items finished (the last one combines)
  int4* cand_st;       // [sub-tiles] forward lists k_bin_sort orders: (sub-tile, pool offset, K, 0)
                       // (count: ctr_sort)
  unsigned* bin;       // [sub-tiles] records binned per sub-tile, then the fill's slot counter
  int* bvh_need;       // [n_inst] set when a sub-tile is listed for per-ray traversal
  unsigned long long* fx;   // [n_inst][6V] fixed-point backward sums (HR_DETERMINISTIC)
  bool det;                 // HR_DETERMINISTIC: every vertex-gradient sum goes to fx
};

struct RenderArgs {
  const Node* nodes;       // instance 0; instance i at + i node_stride
  const float4* tris;      // instance i at + 3 i node_stride
  const float* verts;      // instance i at + 3 i V
  const int* faces;
  const float* normals;    // instance i at + 3 i V
  const float* albedo;
  const Cam* cams;         // [views]
  const float* bg;
  int N, H, W, spp, V;     // uniform layout (single instance)
  const ViewRec* vt;       // batch view table, nullptr = uniform layout
  const InstRec* it;       // batch instance table
  const int* active;       // batch: instances with 0 are skipped (retired), or null
  const int* act_off;      // with `active`: [2][n_inst + 1] active sub-tile / view prefix sums
  int n_inst, nviews, total_st;
  int node_stride;
  int cand_per_chunk, max_chunks;   // work-item split (tuning)
  const float* uv;        // [V][2] texture coordinates (shared by all instances)
  const float* tex;       // [tex_h][tex_w][3] albedo texture, or null: per-vertex albedo
  int tex_w, tex_h;
  float* d_tex;           // dL/dtexture (accumulated), or null
  uint2 key;
  uint32_t ctr1_hi;  // instance << 16
  uint32_t iter4;    // iter << 4 (kernels refresh it from iter_dev when given)
  const uint32_t* iter_dev;
  Shading sh;
  int* status;
  int max_visits;    // F + 1
  Work wk;
};

// bilinear texture lookup at the interpolated uv of a hit: texel coordinates
// x = uv_x W - 0.5, y = uv_y H - 0.5 and their floors are float32 decisions; the
// four texels (clamped to the edge) and their weights
struct TexSample {
  int i0, i1, j0, j1;
  float fx, fy;
};
__device__ __forceinline__ TexSample tex_coords(const RenderArgs& a, int3 f, float u, float v) {
  const float w = __fsub_rn(__fsub_rn(1.0f, u), v);
  const float2 t0 = __ldg(reinterpret_cast<const float2*>(a.uv) + f.x);
  const float2 t1 = __ldg(reinterpret_cast<const float2*>(a.uv) + f.y);
  const float2 t2 = __ldg(reinterpret_cast<const float2*>(a.uv) + f.z);
  const float ux = __fmaf_rn(v, t2.x, __fmaf_rn(u, t1.x, __fmul_rn(w, t0.x)));
  const float uy = __fmaf_rn(v, t2.y, __fmaf_rn(u, t1.y, __fmul_rn(w, t0.y)));
  const float x = __fmaf_rn(ux, (float)a.tex_w, -0.5f), y = __fmaf_rn(uy, (float)a.tex_h, -0.5f);
  const float xf = floorf(x), yf = floorf(y);
  TexSample ts;
  ts.fx = __fsub_rn(x, xf);
  ts.fy = __fsub_rn(y, yf);
  const int xi = (int)fminf(fmaxf(xf, -1.0f), (float)a.tex_w), yi = (int)fminf(fmaxf(yf, -1.0f), (float)a.tex_h);
  ts.i0 = min(max(xi, 0), a.tex_w - 1);
  ts.i1 = min(max(xi + 1, 0), a.tex_w - 1);
  ts.j0 = min(max(yi, 0), a.tex_h - 1);
  ts.j1 = min(max(yi + 1, 0), a.tex_h - 1);
  return ts;
}

__device__ __forceinline__ float3 tex_texel(const RenderArgs& a, int i, int j) {
  return ld3(a.tex + 3 * ((size_t)j * a.tex_w + i));
}

__device__ __forceinline__ float3 tex_albedo(const RenderArgs& a, const TexSample& ts) {
  const float3 t00 = tex_texel(a, ts.i0, ts.j0), t10 = tex_texel(a, ts.i1, ts.j0);
  const float3 t01 = tex_texel(a, ts.i0, ts.j1), t11 = tex_texel(a, ts.i1, ts.j1);
  const float gx = 1.0f - ts.fx, gy = 1.0f - ts.fy;
  return make_float3(gy * (gx * t00.x + ts.fx * t10.x) + ts.fy * (gx * t01.x + ts.fx * t11.x),
                     gy * (gx * t00.y + ts.fx * t10.y) + ts.fy * (gx * t01.y + ts.fx * t11.y),
                     gy * (gx * t00.z + ts.fx * t10.z) + ts.fy * (gx * t01.z + ts.fx * t11.z));
}

__device__ __forceinline__ float3 shade(const RenderArgs& a, const Hit& h) {
  int i0 = __ldg(&a.faces[3 * h.tri]), i1 = __ldg(&a.faces[3 * h.tri + 1]), i2 = __ldg(&a.faces[3 * h.tri + 2]);
  float3 n0 = ld3(a.normals + 3 * i0), n1 = ld3(a.normals + 3 * i1), n2 = ld3(a.normals + 3 * i2);
  float3 nm = interp_normal(h.u, h.v, n0, n1, n2);
  float ndl = ddot(nm, a.sh.l);
  float sigma = 0.0f;
  if (ndl > 0.0f) sigma = ndl * rsqrtf(nm.x * nm.x + nm.y * nm.y + nm.z * nm.z);
  float w = 1.0f - h.u - h.v;
  float k = a.sh.ka + a.sh.kd * sigma;
  float3 alb;
  if (a.tex) {
    alb = tex_albedo(a, tex_coords(a, make_int3(i0, i1, i2), h.u, h.v));
  } else {
    float3 a0 = ld3(a.albedo + 3 * i0), a1 = ld3(a.albedo + 3 * i1), a2 = ld3(a.albedo + 3 * i2);
    alb = make_float3(w * a0.x + h.u * a1.x + h.v * a2.x, w * a0.y + h.u * a1.y + h.v * a2.y,
                      w * a0.z + h.u * a1.z + h.v * a2.z);
  }
  return make_float3(alb.x * a.sh.lrgb.x * k, alb.y * a.sh.lrgb.y * k, alb.z * a.sh.lrgb.z * k);
}

__device__ __forceinline__ Cam load_cam(const Cam* cams, int view) {
  Cam c;
  const float* src = reinterpret_cast<const float*>(cams + view);
  float* dst = reinterpret_cast<float*>(&c);
#pragma unroll
  for (int i = 0; i < 20; ++i) dst[i] = __ldg(src + i);
  return c;
}

// a work item's camera, copied into the warp's shared-memory slot (lane i < 20 copies
// word i) so that the shaders read it from there instead of holding 20 registers
__device__ __forceinline__ const Cam& warp_cam(Cam* slot, const Cam* cams, int view) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (lane < 20) reinterpret_cast<float*>(slot)[lane] = __ldg(reinterpret_cast<const float*>(cams + view) + lane);
  __syncwarp();
  return *slot;
}

// sample-stream iteration: the device counter when the caller gave one
__device__ __forceinline__ RenderArgs with_iter(RenderArgs a) {
  if (a.iter_dev) a.iter4 = (*a.iter_dev) << 4;
  return a;
}

// the same arguments with the scene pointers of instance `inst`
__device__ __forceinline__ RenderArgs for_inst(RenderArgs a, int inst) {
  a.nodes += (size_t)inst * a.node_stride;
  a.tris += (size_t)inst * 3 * a.node_stride;
  a.verts += (size_t)inst * 3 * a.V;
  a.normals += (size_t)inst * 3 * a.V;
  return a;
}

// a batch instance still being refined (hr_batch_set_active)
__device__ __forceinline__ bool inst_active(const RenderArgs& a, int inst) {
  return !a.active || __ldg(&a.active[inst]) != 0;
}

// work-item region of an instance
__device__ __forceinline__ int inst_ibase(const RenderArgs& a, int inst) { return a.vt ? a.it[inst].ibase : 0; }
__device__ __forceinline__ int inst_icap(const RenderArgs& a, int inst) {
  return a.vt ? a.it[inst].icap : a.wk.item_cap;
}

// sample s of pixel (px, py) of a view of width W whose counter word is ctr1
__device__ __forceinline__ void jitter(const RenderArgs& a, uint32_t ctr1, int W, int px, int py, int s, float& u1,
                                       float& u2) {
  uint4 r = philox4x32_10(make_uint4((uint32_t)(py * W + px), ctr1, (uint32_t)s, a.iter4), a.key);
  u1 = u24(r.x);
  u2 = u24(r.y);
}


__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

template <class T>
__device__ __forceinline__ void add3(T* dst, int i, float x, float y, float z) {
  atomicAdd(&dst[3 * i], x);
  atomicAdd(&dst[3 * i + 1], y);
  atomicAdd(&dst[3 * i + 2], z);
}

// Fixed-point sums (HR_DETERMINISTIC): a contribution x is added as the 64-bit integer
// round(x 2^40) (two's complement in an unsigned word); integer addition is exact and
// associative, so the sums do not depend on the order of the atomics.
constexpr double kFixScale = 1099511627776.0;   // 2^40
__device__ __forceinline__ void add_fixed(unsigned long long* p, float x) {
  atomicAdd(p, (unsigned long long)__double2ll_rn((double)x * kFixScale));
}
template <>
__device__ __forceinline__ void add3<unsigned long long>(unsigned long long* dst, int i, float x, float y, float z) {
  add_fixed(&dst[3 * i], x);
  add_fixed(&dst[3 * i + 1], y);
  add_fixed(&dst[3 * i + 2], z);
}
__device__ __forceinline__ float from_fixed(unsigned long long v) {
  return (float)((double)(long long)v * (1.0 / kFixScale));
}

// ---------------------------------------------------------------------------------
// sub-tiles, frustum gathering
// ---------------------------------------------------------------------------------
struct SubTile {
  int view;          // global view (camera index)
  int inst;          // instance
  int x0, y0;
  int H, W, spp;
  uint32_t ctr1;     // Philox counter word of the view
  long long pix0;    // first pixel of the view
};

__device__ __forceinline__ int subtile_count(const RenderArgs& a) { return a.total_st; }

// global view holding sub-tile st: binary search of the view table (views are in
// sub-tile order)
__device__ __forceinline__ int view_of_subtile(const RenderArgs& a, int st) {
  int lo = 0, hi = a.nviews - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&a.vt[mid].st0) <= st) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the view of global view index g (uniform layout: computed)
__device__ __forceinline__ void view_info(const RenderArgs& a, int g, SubTile& t, int& st0, int& nsx) {
  t.view = g;
  if (a.vt) {
    const ViewRec* v = a.vt + g;
    t.inst = __ldg(&v->inst);
    t.ctr1 = __ldg(&v->ctr1);
    t.H = __ldg(&v->H);
    t.W = __ldg(&v->W);
    t.spp = __ldg(&v->spp);
    t.pix0 = __ldg(&v->pix0);
    st0 = __ldg(&v->st0);
    nsx = __ldg(&v->nsx);
  } else {
    t.inst = 0;
    t.ctr1 = (uint32_t)g | a.ctr1_hi;
    t.H = a.H;
    t.W = a.W;
    t.spp = a.spp;
    t.pix0 = (long long)g * a.H * a.W;
    nsx = (a.W + kSubW - 1) / kSubW;
    st0 = g * nsx * ((a.H + kSubH - 1) / kSubH);
  }
}

__device__ __forceinline__ SubTile subtile(const RenderArgs& a, int st) {
  SubTile t;
  int g;
  if (a.vt) {
    g = view_of_subtile(a, st);
  } else {
    const int nsx = (a.W + kSubW - 1) / kSubW, nsy = (a.H + kSubH - 1) / kSubH;
    g = st / (nsx * nsy);
  }
  int st0, nsx;
  view_info(a, g, t, st0, nsx);
  const int rem = st - st0;
  t.x0 = (rem % nsx) * kSubW;
  t.y0 = (rem / nsx) * kSubH;
  return t;
}

// The sub-tiles a kernel visits: all of them, or in a batch with retired instances
// those of the active instances, numbered 0 .. visit_count - 1 in instance order
// (prefix sums act_off, made by k_active_layout before the render kernels), so that a
// mostly retired batch costs no pass over the retired instances' sub-tiles.
__device__ __forceinline__ int visit_count(const RenderArgs& a) {
  return a.act_off ? __ldg(&a.act_off[a.n_inst]) : a.total_st;
}
// the instance k with off[k] <= i < off[k + 1] (off: n_inst + 1 prefix sums)
__device__ __forceinline__ int active_inst(const int* off, int n, int i) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&off[mid]) <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int visit_subtile(const RenderArgs& a, int i) {
  if (!a.act_off) return i;
  const int k = active_inst(a.act_off, a.n_inst, i);
  return __ldg(&a.it[k].st0) + (i - __ldg(&a.act_off[k]));
}
// views likewise (the edge-sampling kernel)
__device__ __forceinline__ int visit_views(const RenderArgs& a) {
  return a.act_off ? __ldg(&a.act_off[a.n_inst + 1 + a.n_inst]) : a.nviews;
}
__device__ __forceinline__ int visit_view(const RenderArgs& a, int j) {
  if (!a.act_off) return j;
  const int* off = a.act_off + a.n_inst + 1;
  const int k = active_inst(off, a.n_inst, j);
  return __ldg(&a.it[k].view0) + (j - __ldg(&off[k]));
}

// act_off = prefix sums over the instances of (active ? sub-tiles : 0) and
// (active ? views : 0); one block, each thread a contiguous run of instances
constexpr int kLayoutThreads = 1024;
__global__ void __launch_bounds__(kLayoutThreads) k_active_layout(const InstRec* __restrict__ it,
                                                                  const int* __restrict__ active, int n,
                                                                  int* __restrict__ act_off) {
  __shared__ int sst[kLayoutThreads], svw[kLayoutThreads];
  const int per = (n + kLayoutThreads - 1) / kLayoutThreads;
  const int i0 = min(n, threadIdx.x * per), i1 = min(n, i0 + per);
  int st = 0, vw = 0;
  for (int i = i0; i < i1; ++i)
    if (active[i]) {
      st += it[i].nst;
      vw += it[i].nviews;
    }
  sst[threadIdx.x] = st;
  svw[threadIdx.x] = vw;
  __syncthreads();
  for (int d = 1; d < kLayoutThreads; d <<= 1) {   // inclusive scan
    const int a = threadIdx.x >= d ? sst[threadIdx.x - d] : 0, b = threadIdx.x >= d ? svw[threadIdx.x - d] : 0;
    __syncthreads();
    sst[threadIdx.x] += a;
    svw[threadIdx.x] += b;
    __syncthreads();
  }
  st = sst[threadIdx.x] - st;
  vw = svw[threadIdx.x] - vw;
  for (int i = i0; i < i1; ++i) {
    act_off[i] = st;
    act_off[n + 1 + i] = vw;
    if (active[i]) {
      st += it[i].nst;
      vw += it[i].nviews;
    }
  }
  if (threadIdx.x == kLayoutThreads - 1) {
    act_off[n] = sst[threadIdx.x];
    act_off[n + 1 + n] = svw[threadIdx.x];
  }
}

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

__device__ __forceinline__ int warp_append(bool want, int value, int* arr, int count, int cap, bool& ovf) {
  unsigned b = __ballot_sync(0xffffffffu, want);
  int idx = count + __popc(b & lanemask_lt());
  if (want && idx < cap) arr[idx] = value;
  int n = count + __popc(b);
  if (n > cap) ovf = true;
  return n;
}

__device__ __forceinline__ bool box_in_frustum(const float4* pl, float lx, float ly, float lz, float hx, float hy,
                                               float hz) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float4 p = pl[i];
    float x = p.x >= 0.0f ? hx : lx, y = p.y >= 0.0f ? hy : ly, z = p.z >= 0.0f ? hz : lz;
    if (p.x * x + p.y * y + p.z * z < p.w) return false;
  }
  return true;
}

struct GatherSmem {        // per warp
  int leaf[kLeafCap];
  float key[kLeafCap];
  int idx[kLeafCap];
  int front[2][kFrontCap];
  float4 pl[5];
};

// screen box (padded by half a pixel; unbounded if a vertex is not in front of the
// camera) and nearest camera depth of triangle record k
__device__ __forceinline__ void project_record(const RenderArgs& a, const Cam& cam, int k, float4& bb, float& zmin) {
  float4 t0 = __ldg(&a.tris[3 * k]), t1 = __ldg(&a.tris[3 * k + 1]), t2 = __ldg(&a.tris[3 * k + 2]);
  float3 v[3] = {make_float3(t0.x, t0.y, t0.z), make_float3(t0.x + t0.w, t0.y + t1.x, t0.z + t1.y),
                 make_float3(t0.x + t1.z, t0.y + t1.w, t0.z + t2.x)};
  float bx0 = INFINITY, by0 = INFINITY, bx1 = -INFINITY, by1 = -INFINITY;
  zmin = INFINITY;
  bool front = true;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    float X = cam.R[0] * v[m].x + cam.R[1] * v[m].y + cam.R[2] * v[m].z + cam.t[0];
    float Y = cam.R[3] * v[m].x + cam.R[4] * v[m].y + cam.R[5] * v[m].z + cam.t[1];
    float Z = cam.R[6] * v[m].x + cam.R[7] * v[m].y + cam.R[8] * v[m].z + cam.t[2];
    zmin = fminf(zmin, Z);
    front = front && Z > 1e-4f;
    float iz = 1.0f / Z;
    float sx = cam.fx * X * iz + cam.cx, sy = cam.fy * Y * iz + cam.cy;
    bx0 = fminf(bx0, sx);
    bx1 = fmaxf(bx1, sx);
    by0 = fminf(by0, sy);
    by1 = fmaxf(by1, sy);
  }
  if (front) {
    bb = make_float4(bx0 - 0.5f, by0 - 0.5f, bx1 + 0.5f, by1 + 0.5f);
  } else {
    bb = make_float4(-INFINITY, -INFINITY, INFINITY, INFINITY);
    zmin = -INFINITY;
  }
}

// Frustum traversal for the sub-tile with pixels [x0, x0+8) x [y0, y0+4): the four
// planes through the camera centre and the rectangle padded by half a pixel, and
// the camera's forward plane.  Leaves into gs.leaf; returns their count, or -1 when
// the sub-tile needs more than kLeafCap candidates or kFrontCap frontier nodes.
// plane q (0-4) of the sub-tile's frustum: the four planes through the camera centre
// and the rectangle padded by half a pixel, and the camera's forward plane (n, n . c)
__device__ __forceinline__ float4 frustum_plane(const Cam& cam, int x0, int y0, int q) {
  float ax = __fdividef((float)x0 - 0.5f - cam.cx, cam.fx);
  float bx = __fdividef((float)(x0 + kSubW) + 0.5f - cam.cx, cam.fx);
  float ay = __fdividef((float)y0 - 0.5f - cam.cy, cam.fy);
  float by = __fdividef((float)(y0 + kSubH) + 0.5f - cam.cy, cam.fy);
  float3 nc = q == 0   ? make_float3(1.0f, 0.0f, -ax)
              : q == 1 ? make_float3(-1.0f, 0.0f, bx)
              : q == 2 ? make_float3(0.0f, 1.0f, -ay)
              : q == 3 ? make_float3(0.0f, -1.0f, by)
                       : make_float3(0.0f, 0.0f, 1.0f);
  float3 nw = make_float3(cam.R[0] * nc.x + cam.R[3] * nc.y + cam.R[6] * nc.z,
                          cam.R[1] * nc.x + cam.R[4] * nc.y + cam.R[7] * nc.z,
                          cam.R[2] * nc.x + cam.R[5] * nc.y + cam.R[8] * nc.z);
  return make_float4(nw.x, nw.y, nw.z, nw.x * cam.c[0] + nw.y * cam.c[1] + nw.z * cam.c[2]);
}

template <bool STATS>
__device__ int frustum_leaves(const RenderArgs& a, const Cam& cam, int x0, int y0, GatherSmem& gs, Counts& cnt) {
  const int lane = threadIdx.x & 31;
  if (lane < 5) gs.pl[lane] = frustum_plane(cam, x0, y0, lane);
  if (lane == 0) gs.front[0][0] = 0;
  __syncwarp();
  int n = 1, cur = 0, K = 0, levels = 0;
  bool ovf = false;
  while (n > 0 && !ovf) {
    int nn = 0;
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      bool kl = false, kr = false;
      int cl = 0, cr = 0;
      if (i < n) {
        int node = gs.front[cur][i];
        if (!in_range(a.status, node, 0, a.max_visits)) node = 0;
        const float4* np = reinterpret_cast<const float4*>(a.nodes + node);
        float4 p = __ldg(np), q = __ldg(np + 1), r = __ldg(np + 2);
        int4 dd = __ldg(reinterpret_cast<const int4*>(np + 3));
        if (STATS) ++cnt.nodes;
        kl = box_in_frustum(gs.pl, p.x, p.y, p.z, p.w, q.x, q.y);
        kr = box_in_frustum(gs.pl, q.z, q.w, r.x, r.y, r.z, r.w);
        cl = dd.x;
        cr = dd.y;
        if (cl == cr) kr = false;   // a one-triangle tree stores its leaf twice
      }
      nn = warp_append(kl && cl >= 0, cl, gs.front[cur ^ 1], nn, kFrontCap, ovf);
      nn = warp_append(kr && cr >= 0, cr, gs.front[cur ^ 1], nn, kFrontCap, ovf);
      K = warp_append(kl && cl < 0, ~cl, gs.leaf, K, kLeafCap, ovf);
      K = warp_append(kr && cr < 0, ~cr, gs.leaf, K, kLeafCap, ovf);
    }
    __syncwarp();
    cur ^= 1;
    n = nn;
    if (++levels > a.max_visits) {   // deeper than any well-formed tree: report and stop
      if (lane == 0) set_status(a.status, kStatusLimit);
      ovf = true;
    }
  }
  return ovf ? -1 : K;
}

// work items of a sub-tile with K candidates (K < 0: per-ray traversal): one per
// `cand_per_chunk` candidates, at most max_chunks and spp
// (K = -1: more candidates than the gather's list holds; K < -1: -(K + 1) candidates
// that found no room in the pool.)  The split depends on the geometry only, never on
// which sub-tiles the pool served first, so sums over a sub-tile's items are
// reproducible.
__device__ __forceinline__ int chunks_for(const RenderArgs& a, int K, int spp) {
  int c = K == -1 ? a.max_chunks : (K < 0 ? -K - 1 : K) / a.cand_per_chunk;
  return max(1, min(min(c, a.max_chunks), spp));
}

// Work-item order.  A warp's item costs about (samples per lane) x (kSampleCost + K)
// candidate tests: a sample's own work (jitter, direction, shading or
// differentiation) weighs about kSampleCost tests (measured on the paper-shaped
// workload).  Items are taken from one counter, so the launch ends when the last
// item taken finishes; heavy items taken last leave most warps idle for the length
// of one heavy item.  Items whose cost exceeds twice the split's target
// (cand_per_chunk x spp) are therefore allocated from the front of the instance's
// item region and the others from its back, and the shaders take the front first.
// Per instance the counters are: front items (ctr[2 + 2i]), taken items
// (ctr[3 + 2i]), back items (ctr[3 + 2n + i]), and a 64-bit allocation word
// (front | back << 32) that decides, in one atomic, whether a group still fits.
constexpr int kSampleCost = 16;
__device__ __forceinline__ bool heavy_item(const RenderArgs& a, int K, int C, int spp) {
  const int k = K == -1 ? kLeafCap : (K < 0 ? -K - 1 : K);
  const int ns = (spp + C - 1) / C;
  return (long long)ns * (k + kSampleCost) > 2LL * a.cand_per_chunk * spp;
}
__device__ __forceinline__ unsigned* back_count(const RenderArgs& a, int inst) {
  return a.wk.ctr + 3 + 2 * a.n_inst + inst;
}
__device__ __forceinline__ unsigned long long* alloc_word(const RenderArgs& a, int inst) {
  return reinterpret_cast<unsigned long long*>(a.wk.ctr + ctr_alloc_base(a.n_inst)) + inst;
}
// reserve C consecutive slots of instance inst's region (lane 0 calls); -1 when the
// region has no room for them
__device__ __forceinline__ int alloc_items(const RenderArgs& a, int inst, int C, bool heavy, int icap) {
  const unsigned long long v =
      atomicAdd(alloc_word(a, inst), heavy ? (unsigned long long)C : ((unsigned long long)C << 32));
  const long long front = (long long)(v & 0xffffffffull), back = (long long)(v >> 32);
  if (front + back + C > icap) return -1;
  if (heavy) {
    atomicAdd(&a.wk.ctr[2 + 2 * inst], (unsigned)C);
    return (int)front;
  }
  atomicAdd(back_count(a, inst), (unsigned)C);
  return (int)(icap - back - C);
}

// the C items at table index `gi` belong to a sub-tile without a candidate list: list
// them for k_overflow (all lanes call)
__device__ __forceinline__ void note_trace_items(const RenderArgs& a, int gi, int C) {
  int base = 0;
  if ((threadIdx.x & 31) == 0) base = (int)atomicAdd(&a.wk.ctr[ctr_trace(a.n_inst)], (unsigned)C);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int c = threadIdx.x & 31; c < C; c += 32)
    if (base + c < a.wk.item_cap) a.wk.trace[base + c] = gi + c;
}


// bit p of the result: candidate box `b` (screen pixels, closed) meets pixel p of the
// 8x4 sub-tile at (x0, y0), i.e. b.x <= px + 1, b.z >= px, b.y <= py + 1, b.w >= py
// with pixel p at (x0 + p % 8, y0 + p / 8).  The float subtractions round
// monotonically and integers are exact, so the column and row bounds never exclude a
// pixel that meets the box; a NaN bound keeps the whole range.
__device__ __forceinline__ unsigned box_pixel_mask(float4 b, int x0, int y0) {
  const int cx0 = (int)fminf(fmaxf(ceilf(__fsub_rn(b.x, (float)(x0 + 1))), 0.0f), 8.0f);
  const int cx1 = (int)fmaxf(fminf(floorf(__fsub_rn(b.z, (float)x0)), 7.0f), -1.0f);
  const int ry0 = (int)fminf(fmaxf(ceilf(__fsub_rn(b.y, (float)(y0 + 1))), 0.0f), 4.0f);
  const int ry1 = (int)fmaxf(fminf(floorf(__fsub_rn(b.w, (float)y0)), 3.0f), -1.0f);
  if (cx0 > cx1 || ry0 > ry1) return 0u;
  const unsigned cols = (0xffu >> (7 - cx1)) & (0xffu << cx0);
  const unsigned rows = (0xffffffffu >> (8 * (3 - ry1))) & (0xffffffffu << (8 * ry0));
  return rows & (cols * 0x01010101u);
}

// 32 x 32 bit matrix held one row per lane (bit p of lane l's word) -> its transpose
// (bit l of lane p's word), by five butterfly stages that swap off-diagonal blocks
__device__ __forceinline__ unsigned warp_transpose32(unsigned x) {
  const int lane = threadIdx.x & 31;
  const unsigned m[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const unsigned t = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~m[s]) | ((t & ~m[s]) >> j)) : ((x & m[s]) | ((t & m[s]) << j));
  }
  return x;
}

// closest hits of a lane's S rays (same origin, all in pixel (x0 + lane % 8,
// y0 + lane / 8)) among the K pool candidates at `off`, which are sorted by nearest
// depth.  The warp loads the candidates 32 at a time, one per lane (depth, screen box
// and triangle record in three coalesced loads); each lane tests its candidate's box
// against the sub-tile's 32 pixel squares, and a bit transpose gives every lane the
// candidates that can hold a sample of its own pixel.  Each lane then walks only
// those, in depth order, taking their records by shuffles from the lanes that loaded
// them, so the lanes of one iteration each test a different candidate instead of
// idling while the warp steps through candidates that miss their pixel.  A lane stops
// at the first candidate nearer than none of its rays' hits (the list is depth-sorted,
// so no later one is nearer).  Every ray tests the same candidates in the same order
// as a scan of the whole list would, so each gets exactly the hit the one-ray search
// gives it.  `live[j]` rays take part.
template <bool STATS, int S>
__device__ __forceinline__ void closest_candidates(const RenderArgs& a, int off, int K, int x0, int y0,
                                                   const bool (&live)[S], const float (&sx)[S], const float (&sy)[S],
                                                   float3 o, const float3 (&d)[S], Hit (&h)[S], Counts& cnt) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool done = true;
#pragma unroll
  for (int j = 0; j < S; ++j) {
    h[j] = Hit{-1, INFINITY, 0.0f, 0.0f};
    done = done && !live[j];
  }
  for (int c0 = 0; c0 < K; c0 += 32) {
    if (!__any_sync(full, !done)) break;
    // this block of candidates, one per lane; a pool index out of range ends the scan
    const int cl = c0 + lane;
    const bool have = cl < K;
    const bool ok = have && in_range(a.status, off + cl, 0, a.wk.pool_cap);
    float zl = 0.0f;
    float4 bl = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int kl = 0;
    if (ok) {
      zl = __ldg(&a.wk.z[off + cl]);
      bl = __ldg(&a.wk.bb[off + cl]);
      kl = __ldg(&a.wk.rec[off + cl]);
    }
    const unsigned bad = __ballot_sync(full, have && !ok);
    int n = min(32, K - c0);
    if (bad) n = min(n, __ffs(bad) - 1);
    unsigned pm = 0u;
    if (lane < n) {
      pm = box_pixel_mask(bl, x0, y0);
      if (STATS) ++cnt.cands;
    }
    unsigned m = warp_transpose32(pm);   // bit i: candidate c0 + i meets this lane's pixel
    if (done) m = 0u;
    for (;;) {
      const bool act = m != 0u;
      if (!__any_sync(full, act)) break;
      const int i = act ? __ffs(m) - 1 : 0;
      m &= m - 1u;
      const float zm = __shfl_sync(full, zl, i);
      const float bx0 = __shfl_sync(full, bl.x, i), by0 = __shfl_sync(full, bl.y, i);
      const float bx1 = __shfl_sync(full, bl.z, i), by1 = __shfl_sync(full, bl.w, i);
      const int k = __shfl_sync(full, kl, i);
      if (!act) continue;
      const float zlim = zm - (1e-4f * fabsf(zm) + 1e-6f);
      bool want[S];
      bool any = false;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        want[j] = live[j] && !(h[j].t < zlim);
        any = any || want[j];
      }
      if (!any) {   // no later candidate is nearer either
        done = true;
        m = 0u;
        continue;
      }
      bool inside = false;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (STATS && want[j]) ++cnt.cands;
        want[j] = want[j] && sx[j] >= bx0 && sx[j] <= bx1 && sy[j] >= by0 && sy[j] <= by1;
        inside = inside || want[j];
      }
      if (!inside) continue;
      if (!in_range(a.status, k, 0, a.max_visits - 1)) continue;
      const float4 ta = __ldg(&a.tris[3 * k]), tb = __ldg(&a.tris[3 * k + 1]), tc = __ldg(&a.tris[3 * k + 2]);
      const float3 v0 = make_float3(ta.x, ta.y, ta.z), e1 = make_float3(ta.w, tb.x, tb.y),
                   e2 = make_float3(tb.z, tb.w, tc.x);
      const int id = __float_as_int(tc.y);
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (!want[j]) continue;
        if (STATS) ++cnt.tris;
        float t, u, v;
        if (mt_hit(o, d[j], v0, e1, e2, t, u, v) && (t < h[j].t || (t == h[j].t && id < h[j].tri))) {
          h[j].tri = id;
          h[j].t = t;
          h[j].u = u;
          h[j].v = v;
        }
      }
    }
    if (bad) break;
  }
}

// Radiance sums of samples [s0, s1) of this lane's pixel (all lanes call it), traced
// S at a time (the tuning's rays per lane); the radiance is added in sample order.
template <bool STATS, int S, bool TRACE = true>
__device__ __forceinline__ void shade_samples(const RenderArgs& a, const SubTile& t, const Cam& cam, int off, int K,
                                              int s0, int s1, float3& acc, int& misses, Counts& cnt) {
  const int lane = threadIdx.x & 31;
  const int px = t.x0 + (lane % kSubW), py = t.y0 + (lane / kSubW);
  const bool valid = px < t.W && py < t.H;
  const float3 o = make_float3(cam.c[0], cam.c[1], cam.c[2]);
  for (int sb = s0; sb < s1; sb += S) {
    bool live[S];
    float sx[S], sy[S];
    float3 d[S];
    Hit h[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      live[j] = valid && sb + j < s1;
      sx[j] = sy[j] = 0.0f;
      if (live[j]) {
        float u1, u2;
        jitter(a, t.ctr1, t.W, px, py, sb + j, u1, u2);
        sx[j] = __fadd_rn((float)px, u1);
        sy[j] = __fadd_rn((float)py, u2);
        if (STATS) {
          ++cnt.samples;
          ++cnt.rays;
        }
      }
      d[j] = primary_dir(cam, sx[j], sy[j]);
    }
    if (K > 0) {
      closest_candidates<STATS, S>(a, off, K, t.x0, t.y0, live, sx, sy, o, d, h, cnt);
    } else {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        h[j] = Hit{-1, INFINITY, 0.0f, 0.0f};
        // K < 0: no usable candidate list, per-ray traversal (only the overflow kernel
        // meets such sub-tiles; the shaders are built without it)
        if (TRACE && live[j]) h[j] = trace<STATS>(a.nodes, a.tris, o, d[j], a.status, cnt, a.max_visits);
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (!(valid && sb + j < s1)) continue;
      if (h[j].tri >= 0) {
        if (STATS) ++cnt.hits;
        float3 f = shade(a, h[j]);
        acc.x += f.x;
        acc.y += f.y;
        acc.z += f.z;
      } else {
        ++misses;
      }
    }
  }
}

__device__ __forceinline__ void write_pixel(const RenderArgs& a, const SubTile& t, float3 acc, int misses,
                                            float* __restrict__ image) {
  const int lane = threadIdx.x & 31;
  const int px = t.x0 + (lane % kSubW), py = t.y0 + (lane / kSubW);
  if (px >= t.W || py >= t.H) return;
  // misses contribute background * (misses / spp): a pixel whose samples all miss is
  // exactly its background value
  const size_t pix = t.pix0 + (size_t)py * t.W + px;
  const float fm = __fdiv_rn((float)misses, (float)t.spp);
  const float inv_spp = 1.0f / (float)t.spp;
  float3 bgc = misses ? ld3(a.bg + 3 * pix) : make_float3(0.0f, 0.0f, 0.0f);
  image[3 * pix] = acc.x * inv_spp + bgc.x * fm;
  image[3 * pix + 1] = acc.y * inv_spp + bgc.y * fm;
  image[3 * pix + 2] = acc.z * inv_spp + bgc.z * fm;
}

// dL/dverts (through u, v at the fixed ray) and dL/dnormals of one shaded hit with
// upstream g = dL/df: dv[0..8] = dL/d(v0, v1, v2), dn[0..8] = dL/d(n0, n1, n2)
struct HitGrad {
  float dv[9], dn[9];
};

__device__ __forceinline__ void hit_grad(const RenderArgs& a, const Hit& h, const int3 f, float3 d,
                                         float3 g, HitGrad& out) {
  float3 n0 = ld3(a.normals + 3 * f.x), n1 = ld3(a.normals + 3 * f.y), n2 = ld3(a.normals + 3 * f.z);
  float3 a0 = ld3(a.albedo + 3 * f.x), a1 = ld3(a.albedo + 3 * f.y), a2 = ld3(a.albedo + 3 * f.z);
  const float u = h.u, v = h.v, w = 1.0f - u - v;
  float3 nm = interp_normal(u, v, n0, n1, n2);
  bool lit = ddot(nm, a.sh.l) > 0.0f;
  float inv_len = rsqrtf(dot3(nm, nm));
  float3 nh = make_float3(nm.x * inv_len, nm.y * inv_len, nm.z * inv_len);
  float sigma = lit ? dot3(nh, a.sh.l) : 0.0f;
  float k = a.sh.ka + a.sh.kd * sigma;
  float3 dalb = make_float3(g.x * a.sh.lrgb.x * k, g.y * a.sh.lrgb.y * k, g.z * a.sh.lrgb.z * k);
  float gu, gv;
  float3 alb;
  if (a.tex) {
    // albedo = bilinear(texture, uv(u, v)): texel gradients, and the uv chain to (u, v)
    const TexSample ts = tex_coords(a, f, u, v);
    alb = tex_albedo(a, ts);
    const float3 t00 = tex_texel(a, ts.i0, ts.j0), t10 = tex_texel(a, ts.i1, ts.j0);
    const float3 t01 = tex_texel(a, ts.i0, ts.j1), t11 = tex_texel(a, ts.i1, ts.j1);
    const float gx = 1.0f - ts.fx, gy = 1.0f - ts.fy;
    const float dax = (gy * (t10.x - t00.x) + ts.fy * (t11.x - t01.x)) * dalb.x +
                      (gy * (t10.y - t00.y) + ts.fy * (t11.y - t01.y)) * dalb.y +
                      (gy * (t10.z - t00.z) + ts.fy * (t11.z - t01.z)) * dalb.z;
    const float day = (gx * (t01.x - t00.x) + ts.fx * (t11.x - t10.x)) * dalb.x +
                      (gx * (t01.y - t00.y) + ts.fx * (t11.y - t10.y)) * dalb.y +
                      (gx * (t01.z - t00.z) + ts.fx * (t11.z - t10.z)) * dalb.z;
    const float dux = dax * (float)a.tex_w, duy = day * (float)a.tex_h;   // dL/d(uv of the hit)
    const float2 q0 = __ldg(reinterpret_cast<const float2*>(a.uv) + f.x);
    const float2 q1 = __ldg(reinterpret_cast<const float2*>(a.uv) + f.y);
    const float2 q2 = __ldg(reinterpret_cast<const float2*>(a.uv) + f.z);
    gu = dux * (q1.x - q0.x) + duy * (q1.y - q0.y);
    gv = dux * (q2.x - q0.x) + duy * (q2.y - q0.y);
    if (a.d_tex) {
      const float wts[4] = {gx * gy, ts.fx * gy, gx * ts.fy, ts.fx * ts.fy};
      const int ii[4] = {ts.i0, ts.i1, ts.i0, ts.i1}, jj[4] = {ts.j0, ts.j0, ts.j1, ts.j1};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        add3(a.d_tex, jj[q] * a.tex_w + ii[q], wts[q] * dalb.x, wts[q] * dalb.y, wts[q] * dalb.z);
    }
  } else {
    gu = dalb.x * (a1.x - a0.x) + dalb.y * (a1.y - a0.y) + dalb.z * (a1.z - a0.z);
    gv = dalb.x * (a2.x - a0.x) + dalb.y * (a2.y - a0.y) + dalb.z * (a2.z - a0.z);
    alb = make_float3(w * a0.x + u * a1.x + v * a2.x, w * a0.y + u * a1.y + v * a2.y, w * a0.z + u * a1.z + v * a2.z);
  }
  float3 dnm = make_float3(0.0f, 0.0f, 0.0f);
  if (lit) {
    float dsig = a.sh.kd * (g.x * alb.x * a.sh.lrgb.x + g.y * alb.y * a.sh.lrgb.y + g.z * alb.z * a.sh.lrgb.z);
    float3 dnh = make_float3(dsig * a.sh.l.x, dsig * a.sh.l.y, dsig * a.sh.l.z);
    float pr = dot3(nh, dnh);
    dnm = make_float3((dnh.x - nh.x * pr) * inv_len, (dnh.y - nh.y * pr) * inv_len, (dnh.z - nh.z * pr) * inv_len);
    gu += dnm.x * (n1.x - n0.x) + dnm.y * (n1.y - n0.y) + dnm.z * (n1.z - n0.z);
    gv += dnm.x * (n2.x - n0.x) + dnm.y * (n2.y - n0.y) + dnm.z * (n2.z - n0.z);
  }
  out.dn[0] = w * dnm.x; out.dn[1] = w * dnm.y; out.dn[2] = w * dnm.z;
  out.dn[3] = u * dnm.x; out.dn[4] = u * dnm.y; out.dn[5] = u * dnm.z;
  out.dn[6] = v * dnm.x; out.dn[7] = v * dnm.y; out.dn[8] = v * dnm.z;
  // barycentrics at the fixed ray: moving vertex k by dp moves the hit's (u, v, t)
  // by -M^-1 (w_k dp) with M = [e1, e2, -d] and weights (w, u, v), so
  // dL/dp_k = -w_k (gu (d x e2) + gv (e1 x d)) / D, D = e1 . (d x e2) -- written with
  // the triangle's edges and the ray direction only (the camera-to-triangle offset,
  // ~1000x an edge, cancels out of the algebra and would cost float32 digits)
  float3 p0 = ld3(a.verts + 3 * f.x), p1 = ld3(a.verts + 3 * f.y), p2 = ld3(a.verts + 3 * f.z);
  float3 e1 = make_float3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z);
  float3 e2 = make_float3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z);
  float3 dxe2 = cross3(d, e2), e1xd = cross3(e1, d);
  float invD = 1.0f / dot3(e1, dxe2);
  float q[3] = {(gu * dxe2.x + gv * e1xd.x) * invD, (gu * dxe2.y + gv * e1xd.y) * invD,
                (gu * dxe2.z + gv * e1xd.z) * invD};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out.dv[c] = -w * q[c];
    out.dv[3 + c] = -u * q[c];
    out.dv[6 + c] = -v * q[c];
  }
}

template <class T>
__device__ __forceinline__ void flush_tri(int3 f, const HitGrad& acc, T* dV, T* dN) {
  add3(dV, f.x, acc.dv[0], acc.dv[1], acc.dv[2]);
  add3(dV, f.y, acc.dv[3], acc.dv[4], acc.dv[5]);
  add3(dV, f.z, acc.dv[6], acc.dv[7], acc.dv[8]);
  add3(dN, f.x, acc.dn[0], acc.dn[1], acc.dn[2]);
  add3(dN, f.y, acc.dn[3], acc.dn[4], acc.dn[5]);
  add3(dN, f.z, acc.dn[6], acc.dn[7], acc.dn[8]);
}

// End-of-item flush by the whole warp: lanes whose run is on a triangle no other
// lane holds add their sums directly; lanes sharing a triangle (the usual case in a
// coherent 8x4 sub-tile) are summed by a warp butterfly first and one lane adds the
// group's sums, so the shared-memory atomics do not collide on the same addresses.
template <class T>
__device__ __forceinline__ void flush_tri_warp(int cur, int3 cf, const HitGrad& acc, T* dV, T* dN) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned grp = __match_any_sync(full, cur);
  const bool shared = __popc(grp) > 1;
  if (cur >= 0 && !shared) flush_tri(cf, acc, dV, dN);
  unsigned pending = __ballot_sync(full, cur >= 0 && shared && lane == __ffs(grp) - 1);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    pending &= pending - 1;
    const int key = __shfl_sync(full, cur, leader);
    const bool in = cur == key;
    HitGrad sum;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      float x = in ? acc.dv[c] : 0.0f, y = in ? acc.dn[c] : 0.0f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(full, x, o);
        y += __shfl_xor_sync(full, y, o);
      }
      sum.dv[c] = x;
      sum.dn[c] = y;
    }
    if (lane == leader) flush_tri(cf, sum, dV, dN);
  }
}

// Gradient of samples [s0, s1) of this lane's pixel (upstream g, `live` lanes only;
// all lanes call it), traced S at a time and differentiated in sample order; added to
// dV [V][3] / dN [V][3] per run of hits on one triangle.
template <bool STATS, int S, class T, bool TRACE = true>
__device__ __forceinline__ void grad_samples(const RenderArgs& a, const SubTile& t, const Cam& cam, int off, int K,
                                             int s0, int s1, bool live, float3 g, T* dV, T* dN, Counts& cnt) {
  const int lane = threadIdx.x & 31;
  const int px = t.x0 + (lane % kSubW), py = t.y0 + (lane / kSubW);
  const float3 o = make_float3(cam.c[0], cam.c[1], cam.c[2]);
  int cur = -1;
  int3 cf = make_int3(0, 0, 0);
  HitGrad acc;
#pragma unroll
  for (int c = 0; c < 9; ++c) acc.dv[c] = acc.dn[c] = 0.0f;
  for (int sb = s0; sb < s1; sb += S) {
    bool lv[S];
    float sx[S], sy[S];
    float3 d[S];
    Hit h[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      lv[j] = live && sb + j < s1;
      sx[j] = sy[j] = 0.0f;
      if (lv[j]) {
        float u1, u2;
        jitter(a, t.ctr1, t.W, px, py, sb + j, u1, u2);
        sx[j] = __fadd_rn((float)px, u1);
        sy[j] = __fadd_rn((float)py, u2);
        if (STATS) {
          ++cnt.samples;
          ++cnt.rays;
        }
      }
      d[j] = primary_dir(cam, sx[j], sy[j]);
    }
    if (K > 0) {
      closest_candidates<STATS, S>(a, off, K, t.x0, t.y0, lv, sx, sy, o, d, h, cnt);
    } else {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        h[j] = Hit{-1, INFINITY, 0.0f, 0.0f};
        if (TRACE && lv[j]) h[j] = trace<STATS>(a.nodes, a.tris, o, d[j], a.status, cnt, a.max_visits);
      }
    }
    // one copy of the differentiation for the S rays (the trace above is unrolled for
    // its independent loads; unrolling this too multiplies the kernel's largest body
    // S times and the warps then wait on instruction fetch): ray j is picked by
    // selects, which keeps h and d in registers
#pragma unroll 1
    for (int j = 0; j < S; ++j) {
      bool lj = lv[0];
      Hit hj = h[0];
      float3 dj = d[0];
#pragma unroll
      for (int q = 1; q < S; ++q)
        if (j == q) {
          lj = lv[q];
          hj = h[q];
          dj = d[q];
        }
      if (!lj || hj.tri < 0) continue;
      if (STATS) ++cnt.hits;
      if (hj.tri != cur) {
        if (cur >= 0) {
          flush_tri(cf, acc, dV, dN);
#pragma unroll
          for (int c = 0; c < 9; ++c) acc.dv[c] = acc.dn[c] = 0.0f;
        }
        cur = hj.tri;
        cf = make_int3(__ldg(&a.faces[3 * cur]), __ldg(&a.faces[3 * cur + 1]), __ldg(&a.faces[3 * cur + 2]));
      }
      HitGrad hg;
      hit_grad(a, hj, cf, dj, g, hg);
      // rounded adds: no contraction with the products inside hit_grad, so a run's sum
      // is the same in every kernel that traces it
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        acc.dv[c] = __fadd_rn(acc.dv[c], hg.dv[c]);
        acc.dn[c] = __fadd_rn(acc.dn[c], hg.dn[c]);
      }
    }
  }
  flush_tri_warp(cur, cf, acc, dV, dN);
}

// this lane's upstream gradient dL/df / spp; `live` = non-zero adjoint
__device__ __forceinline__ float3 lane_adjoint(const RenderArgs& a, const SubTile& t, const float* __restrict__ adjoint,
                                               bool& live) {
  const int lane = threadIdx.x & 31;
  const int px = t.x0 + (lane % kSubW), py = t.y0 + (lane / kSubW);
  live = false;
  if (px >= t.W || py >= t.H) return make_float3(0.0f, 0.0f, 0.0f);
  float3 g = ld3(adjoint + 3 * (t.pix0 + (size_t)py * t.W + px));
  live = g.x != 0.0f || g.y != 0.0f || g.z != 0.0f;
  const float inv_spp = 1.0f / (float)t.spp;
  return make_float3(g.x * inv_spp, g.y * inv_spp, g.z * inv_spp);
}

// kernels that take a group of consecutive sub-tiles per warp (k_bin_alloc, k_background,
// k_items_bwd): one per lane of the first kGroupSubtiles lanes
constexpr int kGroupThreads = 256;
constexpr int kGroupSubtiles = 8;

// ---------------------------------------------------------------------------------
// forward candidate lists by screen-space binning
// ---------------------------------------------------------------------------------
// The shaders test every sample against a candidate's screen box (project_record:
// padded by half a pixel, unbounded when a vertex is not in front of the camera)
// before intersecting it, so a sub-tile's list needs exactly the triangle records
// whose box meets the sub-tile's sample square [x0, x0 + 8] x [y0, y0 + 4].  The
// forward builds the lists by binning each (view, record) pair into the sub-tiles its
// box meets -- k_bin counts them, k_bin_alloc gives every sub-tile its pool range and
// work items, k_bin in fill mode writes the records, k_bin_sort orders each list by
// nearest depth -- instead of a frustum walk of the BVH per sub-tile.

// sub-tile columns [c0, c1] and rows [r0, r1] of a view (nsx x nsy sub-tiles) whose
// sample squares meet box b: column c meets it iff b.x <= 8c + 8 and b.z >= 8c (rows
// likewise with 4).  The float subtraction rounds monotonically and the scalings by
// 1/8 and 1/4 and the integers are exact, so no column or row that meets the box is
// left out; a NaN bound keeps the whole range.
struct BinRange {
  int c0, c1, r0, r1;
};
__device__ __forceinline__ BinRange bin_range(float4 b, int nsx, int nsy) {
  BinRange r;
  r.c0 = (int)fminf(fmaxf(ceilf(__fmul_rn(__fsub_rn(b.x, (float)kSubW), 1.0f / kSubW)), 0.0f), (float)nsx);
  r.c1 = (int)fmaxf(fminf(floorf(__fmul_rn(b.z, 1.0f / kSubW)), (float)(nsx - 1)), -1.0f);
  r.r0 = (int)fminf(fmaxf(ceilf(__fmul_rn(__fsub_rn(b.y, (float)kSubH), 1.0f / kSubH)), 0.0f), (float)nsy);
  r.r1 = (int)fmaxf(fminf(floorf(__fmul_rn(b.w, 1.0f / kSubH)), (float)(nsy - 1)), -1.0f);
  return r;
}

// the camera depth of record k's three vertices all below -1e-3: no primary ray
// (camera depth t > 0 at parameter t) can meet it
__device__ __forceinline__ bool record_behind(const RenderArgs& a, const Cam& cam, int k) {
  const float4 t0 = __ldg(&a.tris[3 * k]), t1 = __ldg(&a.tris[3 * k + 1]), t2 = __ldg(&a.tris[3 * k + 2]);
  const float3 v[3] = {make_float3(t0.x, t0.y, t0.z), make_float3(t0.x + t0.w, t0.y + t1.x, t0.z + t1.y),
                       make_float3(t0.x + t1.z, t0.y + t1.w, t0.z + t2.x)};
  bool behind = true;
#pragma unroll
  for (int m = 0; m < 3; ++m)
    behind = behind && cam.R[6] * v[m].x + cam.R[7] * v[m].y + cam.R[8] * v[m].z + cam.t[2] < -1e-3f;
  return behind;
}

constexpr int kBinThreads = 256;
constexpr int kBinPairs = 8;   // (view, record) pairs per warp

// one sub-tile of a pair's range: count it, or (FILL) write the record into the
// sub-tile's pool range at the next free slot
template <bool FILL>
__device__ __forceinline__ void bin_visit(const RenderArgs& a, unsigned* __restrict__ bin, int s, int k, float zm,
                                          float4 bb) {
  if (!FILL) {
    atomicAdd(&bin[s], 1u);
    return;
  }
  const int2 pk = a.wk.st[s];
  if (pk.y <= 0) return;   // no list: background, per-ray traversal, or no pool room
  const int slot = (int)atomicAdd(&bin[s], 1u);
  if (slot >= pk.y || !in_range(a.status, (long long)pk.x + slot, 0, a.wk.pool_cap)) return;
  a.wk.rec[pk.x + slot] = k;
  a.wk.z[pk.x + slot] = zm;
  a.wk.bb[pk.x + slot] = bb;
}

// Each warp takes kBinPairs consecutive pairs i = (active view i / F, record i % F),
// one per lane of its first lanes, and projects them; the (pair, sub-tile) visits of
// all its pairs are then spread over the 32 lanes (visit q belongs to the pair whose
// range of prefix sums holds q), so the visits of one warp are in flight together
// whatever the sizes of the pairs' ranges.
template <bool FILL>
__global__ void __launch_bounds__(kBinThreads) k_bin(RenderArgs a0, unsigned* __restrict__ bin) {
  pdl_wait();
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int F = a0.max_visits - 1;
  const long long total = (long long)visit_views(a0) * F;
  const long long nw = (long long)gridDim.x * (kBinThreads / 32);
  for (long long w0 = ((long long)blockIdx.x * (kBinThreads / 32) + (threadIdx.x >> 5)) * kBinPairs; w0 < total;
       w0 += nw * kBinPairs) {
    const long long i = w0 + lane;
    int st0 = 0, nsx = 1, k = 0, area = 0;
    float zm = 0.0f;
    float4 bb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    BinRange r{0, -1, 0, -1};
    if (lane < kBinPairs && i < total) {
      const int g = visit_view(a0, (int)(i / F));
      k = (int)(i % F);
      SubTile t;
      view_info(a0, g, t, st0, nsx);
      if (in_range(a0.status, t.inst, 0, a0.n_inst) && inst_active(a0, t.inst)) {
        const RenderArgs a = for_inst(a0, t.inst);
        const Cam cam = load_cam(a.cams, g);
        if (!record_behind(a, cam, k)) {
          project_record(a, cam, k, bb, zm);
          r = bin_range(bb, nsx, (t.H + kSubH - 1) / kSubH);
          if (r.c0 <= r.c1 && r.r0 <= r.r1) area = (r.c1 - r.c0 + 1) * (r.r1 - r.r0 + 1);
        }
      }
    }
    // inclusive prefix sums of the ranges' sizes over the pairs
    int incl = area;
#pragma unroll
    for (int o = 1; o < kBinPairs; o <<= 1) {
      const int y = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += y;
    }
    const int T = __shfl_sync(full, incl, kBinPairs - 1);
    for (int q0 = 0; q0 < T; q0 += 32) {
      const int q = q0 + lane;
      // owner: the first pair whose inclusive sum exceeds q
      int lo = 0;
#pragma unroll
      for (int step = kBinPairs / 2; step > 0; step >>= 1) {
        const int v = __shfl_sync(full, incl, lo + step - 1);
        if (v <= q) lo += step;
      }
      const int own = min(lo, kBinPairs - 1);
      const int s0 = __shfl_sync(full, st0, own), n = __shfl_sync(full, nsx, own);
      const int c0 = __shfl_sync(full, r.c0, own), c1 = __shfl_sync(full, r.c1, own);
      const int r0 = __shfl_sync(full, r.r0, own);
      const int kk = __shfl_sync(full, k, own), end = __shfl_sync(full, incl, own);
      const int na = __shfl_sync(full, area, own);
      const float z = __shfl_sync(full, zm, own);
      float4 b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (FILL) {
        b.x = __shfl_sync(full, bb.x, own);
        b.y = __shfl_sync(full, bb.y, own);
        b.z = __shfl_sync(full, bb.z, own);
        b.w = __shfl_sync(full, bb.w, own);
      }
      if (q >= T) continue;
      const int w = c1 - c0 + 1, local = q - (end - na);
      bin_visit<FILL>(a0, bin, s0 + (r0 + local / w) * n + c0 + local % w, kk, z, b);
    }
  }
}

// Work items of the sub-tiles held by lanes 0 .. kGroupSubtiles - 1 (all lanes call): each
// `need` lane's sub-tile st (instance inst, candidate count K) gets C consecutive
// items.  One reservation per instance among the lanes -- heavy items from the front
// of the instance's region, the others from its back -- so the instance's counters
// see one atomic per warp, not one per sub-tile.  Sub-tiles without a candidate list
// (K < 0) are listed for k_overflow's per-ray traversal; when the region has no room
// for a group, its sub-tiles go to k_overflow whole.
__device__ __forceinline__ void place_items(const RenderArgs& a0, bool need, int st, int inst, int K, int C,
                                            bool heavy) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int key = need ? inst : -1;
  int hx = 0, lx = 0, ht = 0, lt = 0, leader = -1;
#pragma unroll
  for (int j = 0; j < kGroupSubtiles; ++j) {
    const int kj = __shfl_sync(full, key, j), cj = __shfl_sync(full, C, j);
    const bool hj = __shfl_sync(full, (int)heavy, j) != 0;
    if (need && kj == key) {
      if (leader < 0) leader = j;
      if (hj) {
        ht += cj;
        if (j < lane) hx += cj;
      } else {
        lt += cj;
        if (j < lane) lx += cj;
      }
    }
  }
  unsigned long long v = 0ull;
  if (need && lane == leader) {
    v = atomicAdd(alloc_word(a0, inst), (unsigned long long)ht | ((unsigned long long)lt << 32));
    const long long front = (long long)(v & 0xffffffffull), back = (long long)(v >> 32);
    if (front + back + ht + lt <= inst_icap(a0, inst)) {
      if (ht) atomicAdd(&a0.wk.ctr[2 + 2 * inst], (unsigned)ht);
      if (lt) atomicAdd(back_count(a0, inst), (unsigned)lt);
    }
  }
  const int src = leader < 0 ? 0 : leader;
  const unsigned vlo = __shfl_sync(full, (unsigned)(v & 0xffffffffull), src);
  const unsigned vhi = __shfl_sync(full, (unsigned)(v >> 32), src);
  if (!need) return;
  const int icap = inst_icap(a0, inst), ibase = inst_ibase(a0, inst);
  const long long front = vlo, back = vhi;
  const bool fits = front + back + ht + lt <= icap;
  const int first = fits ? (heavy ? (int)front + hx : icap - (int)back - lt + lx) : -1;
  if (first >= 0) {
    for (int c = 0; c < C; ++c) a0.wk.items[ibase + first + c] = make_int4(st, c, C, ibase + first);
    if (K < 0) {
      const int tb = (int)atomicAdd(&a0.wk.ctr[ctr_trace(a0.n_inst)], (unsigned)C);
      for (int c = 0; c < C; ++c)
        if (tb + c < a0.wk.item_cap) a0.wk.trace[tb + c] = ibase + first + c;
    }
  } else {
    a0.wk.ovf[atomicAdd(&a0.wk.ctr[2 + 2 * a0.n_inst], 1u)] = st;
  }
}

// Each warp takes kGroupSubtiles consecutive sub-tiles, one per lane of its first lanes.
// A sub-tile with no record in its bin sees only the background (k_background writes
// it).  The others get a pool range for their K records (one atomic per warp), the
// work items of their chunks, and an entry in the list k_bin_sort orders; the count
// becomes the fill's slot counter.  A sub-tile with more records than a list holds,
// or whose records find no pool room, is traced ray by ray (K = -1, -(K + 1)).
__global__ void __launch_bounds__(kGroupThreads) k_bin_alloc(RenderArgs a0, unsigned* __restrict__ bin) {
  pdl_wait();
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int total = visit_count(a0);
  const int nw = gridDim.x * (kGroupThreads / 32);
  for (int g0 = (blockIdx.x * (kGroupThreads / 32) + (threadIdx.x >> 5)) * kGroupSubtiles; g0 < total;
       g0 += nw * kGroupSubtiles) {
    int st = -1, K = 0;
    bool listed = false;
    SubTile t{};
    if (lane < kGroupSubtiles && g0 + lane < total) {
      const int s = visit_subtile(a0, g0 + lane);
      if (in_range(a0.status, s, 0, a0.total_st)) {
        t = subtile(a0, s);
        if (in_range(a0.status, t.inst, 0, a0.n_inst)) {
          st = s;
          if (!inst_active(a0, t.inst)) {   // a retired instance: nothing to render
            a0.wk.st[s] = make_int2(0, 0);
          } else {
            K = (int)bin[s];
            bin[s] = 0u;
            if (K == 0) a0.wk.st[s] = make_int2(0, 0);
            else listed = true;
          }
        }
      }
    }
    // pool ranges of the warp's lists: exclusive prefix sums of K over the lanes
    const int want = listed && K <= kLeafCap ? K : 0;
    int incl = want;
#pragma unroll
    for (int o = 1; o < kGroupSubtiles; o <<= 1) {
      const int y = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += y;
    }
    unsigned base = 0u;
    const int tot = __shfl_sync(full, incl, kGroupSubtiles - 1);
    if (lane == 0 && tot > 0) base = atomicAdd(&a0.wk.ctr[1], (unsigned)tot);
    base = __shfl_sync(full, base, 0);
    bool sorted = false, heavy = false;
    int Kc = 0, C = 0;
    long long off = 0;
    if (listed) {
      off = (long long)base + incl - want;
      Kc = K;
      if (K > kLeafCap) Kc = -1;
      else if (off + K > a0.wk.pool_cap) Kc = -(K + 1);
      sorted = Kc > 0;
      if (Kc < 0) a0.wk.bvh_need[t.inst] = 1;   // traced ray by ray: the BVH boxes must be current
      a0.wk.st[st] = make_int2(sorted ? (int)off : 0, Kc);
      C = chunks_for(a0, Kc, t.spp);
      heavy = heavy_item(a0, Kc, C, t.spp);
    }
    place_items(a0, listed, st, t.inst, Kc, C, heavy);
    const unsigned sm = __ballot_sync(full, sorted);
    int lb = 0;
    if (lane == 0 && sm) lb = (int)atomicAdd(&a0.wk.ctr[ctr_sort(a0.n_inst)], (unsigned)__popc(sm));
    lb = __shfl_sync(full, lb, 0);
    if (sorted) a0.wk.cand_st[lb + __popc(sm & lanemask_lt())] = make_int4(st, (int)off, Kc, 0);
  }
}

// Pixels of the sub-tiles whose bins hold no record: the background (the value
// write_pixel gives a sub-tile whose samples all miss).  Each warp takes kGroupSubtiles
// consecutive sub-tiles, one per lane of its first lanes, then writes the background
// ones, lane = pixel, every background load issued before the first store.  Runs on
// the context's second stream beside the fill and the sort, which touch no pixel.
template <bool STATS>
__global__ void __launch_bounds__(kGroupThreads) k_background(RenderArgs a0, float* __restrict__ image,
                                                             unsigned long long* stats) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  Counts cnt;
  const int total = visit_count(a0);
  const int nw = gridDim.x * (kGroupThreads / 32);
  for (int g0 = (blockIdx.x * (kGroupThreads / 32) + (threadIdx.x >> 5)) * kGroupSubtiles; g0 < total;
       g0 += nw * kGroupSubtiles) {
    bool background = false;
    SubTile t{};
    if (lane < kGroupSubtiles && g0 + lane < total) {
      const int s = visit_subtile(a0, g0 + lane);
      if (in_range(a0.status, s, 0, a0.total_st)) {
        t = subtile(a0, s);
        background = in_range(a0.status, t.inst, 0, a0.n_inst) && inst_active(a0, t.inst) && a0.wk.st[s].y == 0;
      }
    }
    const unsigned cm = __ballot_sync(full, background);
    if (!cm) continue;
    float3 bgv[kGroupSubtiles];
    size_t pix[kGroupSubtiles];
    bool valid[kGroupSubtiles];
#pragma unroll
    for (int j = 0; j < kGroupSubtiles; ++j) {
      const int x0 = __shfl_sync(full, t.x0, j), y0 = __shfl_sync(full, t.y0, j);
      const int W = __shfl_sync(full, t.W, j), H = __shfl_sync(full, t.H, j);
      const long long p0 = __shfl_sync(full, t.pix0, j);
      const int px = x0 + (lane % kSubW), py = y0 + (lane / kSubW);
      valid[j] = ((cm >> j) & 1u) && px < W && py < H;
      pix[j] = (size_t)p0 + (size_t)py * W + px;
      bgv[j] = valid[j] ? ld3(a0.bg + 3 * pix[j]) : make_float3(0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int j = 0; j < kGroupSubtiles; ++j) {
      const int spp = __shfl_sync(full, t.spp, j);
      if (!valid[j]) continue;
      if (STATS) cnt.samples += spp;   // resolved by the binning: no record meets the sub-tile
      const float fm = __fdiv_rn((float)spp, (float)spp);
      const float inv_spp = 1.0f / (float)spp;
      image[3 * pix[j]] = 0.0f * inv_spp + bgv[j].x * fm;
      image[3 * pix[j] + 1] = 0.0f * inv_spp + bgv[j].y * fm;
      image[3 * pix[j] + 2] = 0.0f * inv_spp + bgv[j].z * fm;
    }
  }
  flush_counts<STATS>(cnt, stats);
}

// one warp per listed sub-tile: its K records (in fill order) sorted by nearest depth
// (bitonic, padded with +inf: across the lanes' registers for K <= 32, else in shared
// memory, the boxes then projected again from the records), written back in order
struct SortSmem {   // per warp
  int leaf[kLeafCap];
  float key[kLeafCap];
  int idx[kLeafCap];
};
__global__ void __launch_bounds__(kRenderThreads) k_bin_sort(RenderArgs a0) {
  pdl_wait();
  __shared__ SortSmem ssm[kWarps];
  SortSmem& ss = ssm[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int n = (int)min(*reinterpret_cast<volatile unsigned*>(&a0.wk.ctr[ctr_sort(a0.n_inst)]),
                         (unsigned)a0.total_st);
  for (int vi = blockIdx.x * kWarps + (threadIdx.x >> 5); vi < n; vi += gridDim.x * kWarps) {
    const int4 cd = a0.wk.cand_st[vi];
    const int st = cd.x, off = cd.y, K = cd.z;
    if (!in_range(a0.status, st, 0, a0.total_st)) continue;
    if (lane == 0) a0.wk.bin[st] = 0u;   // the fill's slot counter, clear for the next forward
    if (K <= 0 || K > kLeafCap || off < 0 || !in_range(a0.status, (long long)off + K - 1, 0, a0.wk.pool_cap)) continue;
    if (K <= 32) {
      // one record per lane (depth, box and index as the fill wrote them), a bitonic
      // sort of (depth, lane) across the warp; lane c then takes the c-th record's box
      // and index from its lane
      int k = 0;
      float4 bb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float key = INFINITY;
      if (lane < K) {
        k = a0.wk.rec[off + lane];
        key = a0.wk.z[off + lane];
        bb = a0.wk.bb[off + lane];
      }
      int src = lane;
#pragma unroll
      for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
          const float ok = __shfl_xor_sync(0xffffffffu, key, stride);
          const int os = __shfl_xor_sync(0xffffffffu, src, stride);
          const bool take_min = ((lane & stride) == 0) == ((lane & size) == 0);
          const bool take = take_min ? (ok < key || (ok == key && os < src)) : (ok > key || (ok == key && os > src));
          if (take) {
            key = ok;
            src = os;
          }
        }
      }
      const int kc = __shfl_sync(0xffffffffu, k, src);
      const float4 bc = make_float4(__shfl_sync(0xffffffffu, bb.x, src), __shfl_sync(0xffffffffu, bb.y, src),
                                    __shfl_sync(0xffffffffu, bb.z, src), __shfl_sync(0xffffffffu, bb.w, src));
      if (lane < K) {
        a0.wk.bb[off + lane] = bc;
        a0.wk.z[off + lane] = key;
        a0.wk.rec[off + lane] = kc;
      }
      continue;
    }
    const SubTile t = subtile(a0, st);
    if (!in_range(a0.status, t.inst, 0, a0.n_inst)) continue;
    const RenderArgs a = for_inst(a0, t.inst);
    const Cam cam = load_cam(a.cams, t.view);
    int P = 1;
    while (P < K) P <<= 1;
    for (int j = lane; j < P; j += 32) {
      int k = 0;
      float z = INFINITY;
      if (j < K) {
        k = a.wk.rec[off + j];
        z = a.wk.z[off + j];
        if (!in_range(a.status, k, 0, a.max_visits - 1)) k = 0;
      }
      ss.leaf[j] = k;
      ss.key[j] = z;
      ss.idx[j] = j;
    }
    __syncwarp();
    for (int q = 2; q <= P; q <<= 1) {
      for (int j = q >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const float zi = ss.key[i], zj = ss.key[ixj];
            const bool up = (i & q) == 0;
            if ((zi > zj) == up) {
              ss.key[i] = zj;
              ss.key[ixj] = zi;
              const int w = ss.idx[i];
              ss.idx[i] = ss.idx[ixj];
              ss.idx[ixj] = w;
            }
          }
        }
        __syncwarp();
      }
    }
    for (int c = lane; c < K; c += 32) {
      int j = ss.idx[c];
      if (!in_range(a.status, j, 0, K)) j = 0;
      const int k = ss.leaf[j];
      float4 bb;
      float zm;
      project_record(a, cam, k, bb, zm);
      a.wk.bb[off + c] = bb;
      a.wk.z[off + c] = zm;
      a.wk.rec[off + c] = k;
    }
    __syncwarp();
  }
}

// The backward's own candidate lists (without HR_BWD_REUSE_FWD): one warp per
// sub-tile with a non-zero adjoint walks the BVH with the sub-tile's frustum,
// collects the records it meets into the pool sorted by nearest depth, and allocates
// the sub-tile's work items in its instance's region of the item table; sub-tiles
// whose frustum meets nothing have no interior gradient.  When the pool or the item
// region is full the sub-tile is traced ray by ray or done whole by k_overflow.
template <bool STATS>
__global__ void __launch_bounds__(kRenderThreads) k_gather(RenderArgs a_in, const float* __restrict__ adjoint,
                                                          unsigned long long* stats) {
  const RenderArgs a0 = with_iter(a_in);
  __shared__ GatherSmem gsm[kWarps];
  GatherSmem& gs = gsm[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  Counts cnt;
  const int total = visit_count(a0);
  for (;;) {
    int vi = 0;
    if (lane == 0) vi = (int)atomicAdd(&a0.wk.ctr[0], 1u);
    vi = __shfl_sync(0xffffffffu, vi, 0);
    if (vi >= total) break;
    const int st = visit_subtile(a0, vi);
    if (!in_range(a0.status, st, 0, a0.total_st)) continue;
    const SubTile t = subtile(a0, st);
    if (!in_range(a0.status, t.inst, 0, a0.n_inst)) continue;
    if (!inst_active(a0, t.inst)) {   // a retired instance: nothing to render
      if (lane == 0) a0.wk.st[st] = make_int2(0, 0);
      continue;
    }
    const RenderArgs a = for_inst(a0, t.inst);
    bool live;
    lane_adjoint(a, t, adjoint, live);
    if (!__any_sync(0xffffffffu, live)) {
      if (lane == 0) a.wk.st[st] = make_int2(0, 0);
      continue;
    }
    const Cam cam = load_cam(a.cams, t.view);
    int K = frustum_leaves<STATS>(a, cam, t.x0, t.y0, gs, cnt);
    if (K == 0) {
      if (lane == 0) a.wk.st[st] = make_int2(0, 0);
      const int px = t.x0 + (lane % kSubW), py = t.y0 + (lane / kSubW);
      if (STATS && px < t.W && py < t.H && live) cnt.samples += t.spp;   // resolved by the frustum test
      continue;
    }
    int off = 0;
    if (K > 0) {
      // sort the candidates by nearest depth (bitonic, padded with +inf)
      for (int j = lane; j < K; j += 32) {
        float4 bb;
        float zm;
        int k = gs.leaf[j];
        if (!in_range(a.status, k, 0, a.max_visits - 1)) k = 0;
        gs.leaf[j] = k;
        project_record(a, cam, k, bb, zm);
        gs.key[j] = zm;
        gs.idx[j] = j;
      }
      int P = 1;
      while (P < K) P <<= 1;
      for (int j = K + lane; j < P; j += 32) {
        gs.key[j] = INFINITY;
        gs.idx[j] = 0;
      }
      __syncwarp();
      for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = lane; i < P; i += 32) {
            int ixj = i ^ j;
            if (ixj > i) {
              float zi = gs.key[i], zj = gs.key[ixj];
              bool up = (i & k) == 0;
              if ((zi > zj) == up) {
                gs.key[i] = zj;
                gs.key[ixj] = zi;
                int q = gs.idx[i];
                gs.idx[i] = gs.idx[ixj];
                gs.idx[ixj] = q;
              }
            }
          }
          __syncwarp();
        }
      }
      if (lane == 0) off = (int)atomicAdd(&a.wk.ctr[1], (unsigned)K);
      off = __shfl_sync(0xffffffffu, off, 0);
      if (off + K <= a.wk.pool_cap) {
        for (int c = lane; c < K; c += 32) {
          int j = gs.idx[c];
          if (!in_range(a.status, j, 0, K)) j = 0;
          const int k = gs.leaf[j];
          float4 bb;
          float zm;
          project_record(a, cam, k, bb, zm);
          a.wk.bb[off + c] = bb;
          a.wk.z[off + c] = zm;
          a.wk.rec[off + c] = k;
        }
      } else {
        // pool full: per-ray traversal for this sub-tile, with K's count kept as
        // -(K + 1) so that its work items are split as they would be with the list
        K = -(K + 1);
      }
    }
    const int C = chunks_for(a, K, t.spp);
    const int ibase = inst_ibase(a, t.inst), icap = inst_icap(a, t.inst);
    int first = 0;
    if (lane == 0) first = alloc_items(a, t.inst, C, heavy_item(a, K, C, t.spp), icap);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (lane == 0) a.wk.st[st] = make_int2(off, K);
    if (first >= 0) {
      for (int c = lane; c < C; c += 32) a.wk.items[ibase + first + c] = make_int4(st, c, C, ibase + first);
      if (K < 0) note_trace_items(a, ibase + first, C);
    } else if (lane == 0) {
      // item region full: the whole sub-tile goes to k_overflow
      a.wk.ovf[atomicAdd(&a.wk.ctr[2 + 2 * a.n_inst], 1u)] = st;
    }
    __syncwarp();
  }
  flush_counts<STATS>(cnt, stats);
}

// The backward's work items from the forward's candidate lists (HR_BWD_REUSE_FWD).
// Each warp takes kGroupSubtiles consecutive sub-tiles, one per lane of its first lanes;
// only sub-tiles with a candidate list (or per-ray traversal) read the adjoint, the
// whole warp loading all of them first (lane = pixel), and those with a non-zero
// adjoint get their work items (place_items).
template <bool STATS>
__global__ void __launch_bounds__(kGroupThreads, 4) k_items_bwd(RenderArgs a0, const float* __restrict__ adjoint,
                                                               unsigned long long* stats) {
  pdl_wait();
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  Counts cnt;
  const int total = visit_count(a0);
  const int nw = gridDim.x * (kGroupThreads / 32);
  for (int g0 = (blockIdx.x * (kGroupThreads / 32) + (threadIdx.x >> 5)) * kGroupSubtiles; g0 < total;
       g0 += nw * kGroupSubtiles) {
    int st = -1;
    int2 pk = make_int2(0, 0);
    bool ok = false;
    SubTile t{};
    if (lane < kGroupSubtiles && g0 + lane < total) {
      const int s = visit_subtile(a0, g0 + lane);
      if (in_range(a0.status, s, 0, a0.total_st)) {
        t = subtile(a0, s);
        if (in_range(a0.status, t.inst, 0, a0.n_inst) && inst_active(a0, t.inst)) {
          st = s;
          ok = true;
          pk = a0.wk.st[s];
          if (pk.y > 0 && !in_range(a0.status, (long long)pk.x + pk.y - 1, 0, a0.wk.pool_cap)) pk.y = -1;
        }
      }
    }
    // sub-tile j's pixels: lane = pixel; every adjoint load issued before the tests
    const unsigned look = __ballot_sync(full, ok && (STATS || pk.y != 0));
    if (!look) continue;
    float3 g[kGroupSubtiles];
    bool valid[kGroupSubtiles];
#pragma unroll
    for (int j = 0; j < kGroupSubtiles; ++j) {
      const int x0 = __shfl_sync(full, t.x0, j), y0 = __shfl_sync(full, t.y0, j);
      const int W = __shfl_sync(full, t.W, j), H = __shfl_sync(full, t.H, j);
      const long long p0 = __shfl_sync(full, t.pix0, j);
      const int px = x0 + (lane % kSubW), py = y0 + (lane / kSubW);
      valid[j] = ((look >> j) & 1u) && px < W && py < H;
      g[j] = valid[j] ? ld3(adjoint + 3 * ((size_t)p0 + (size_t)py * W + px)) : make_float3(0.0f, 0.0f, 0.0f);
    }
    unsigned live = 0u;
#pragma unroll
    for (int j = 0; j < kGroupSubtiles; ++j) {
      const bool lj = valid[j] && (g[j].x != 0.0f || g[j].y != 0.0f || g[j].z != 0.0f);
      if (__ballot_sync(full, lj)) live |= 1u << j;
      const int kj = __shfl_sync(full, pk.y, j), sppj = __shfl_sync(full, t.spp, j);
      if (STATS && lj && kj == 0) cnt.samples += sppj;   // no ray of the sub-tile can hit
    }
    const bool need = ok && ((live >> lane) & 1u) && pk.y != 0;
    const int C = need ? chunks_for(a0, pk.y, t.spp) : 0;
    const bool heavy = need && heavy_item(a0, pk.y, C, t.spp);
    place_items(a0, need, st, t.inst, pk.y, C, heavy);
  }
  flush_counts<STATS>(cnt, stats);
}

// items of an instance's region that the gather filled (front and back)
__device__ __forceinline__ int front_count(const RenderArgs& a, int inst) {
  return (int)min(*reinterpret_cast<volatile unsigned*>(&a.wk.ctr[2 + 2 * inst]), (unsigned)inst_icap(a, inst));
}
__device__ __forceinline__ int item_count(const RenderArgs& a, int inst) {
  const unsigned b = *reinterpret_cast<volatile unsigned*>(back_count(a, inst));
  return (int)min((unsigned)front_count(a, inst) + b, (unsigned)inst_icap(a, inst));
}
// region slot of the instance's i-th item (0 <= i < item_count): the front items,
// heavy, first; then the back items from the region's end
__device__ __forceinline__ int item_slot(const RenderArgs& a, int inst, int i, int nfront) {
  return i < nfront ? i : inst_icap(a, inst) - 1 - (i - nfront);
}

__device__ __forceinline__ void item_samples(int c, int C, int spp, int& s0, int& s1) {
  s0 = (int)((long long)c * spp / C);
  s1 = (int)((long long)(c + 1) * spp / C);
}

// fetch the next work item of instance `inst` (lane 0 takes it, the warp shares it);
// -1 when the instance's region is exhausted
__device__ __forceinline__ int next_item(const RenderArgs& a, int inst, int n) {
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = (int)atomicAdd(&a.wk.ctr[3 + 2 * inst], 1u);
  it = __shfl_sync(0xffffffffu, it, 0);
  return it < n ? it : -1;
}

// the sub-tile and candidate list of item `gi` (global index); false for a blanked or
// corrupt item
__device__ __forceinline__ bool load_item(const RenderArgs& a, int gi, int4& item, SubTile& t, int2& pk) {
  item = a.wk.items[gi];
  if (item.x < 0) return false;   // a blanked slot
  if (!in_range(a.status, item.x, 0, subtile_count(a))) return false;
  t = subtile(a, item.x);
  if (!in_range(a.status, t.inst, 0, a.n_inst)) return false;
  pk = a.wk.st[item.x];
  if (pk.y > 0 && !in_range(a.status, (long long)pk.x + pk.y - 1, 0, a.wk.pool_cap)) pk.y = -1;
  return true;
}

// A forward work item is done (all lanes call): a sub-tile with one item writes its
// pixels at once; otherwise the item's radiance sums go to its slot of the partials,
// and the warp that finishes the sub-tile's last item (a per-sub-tile counter) adds
// the C partials in item order and writes the pixels -- the same sums, in the same
// order, whichever warps traced the items.
__device__ __forceinline__ void finish_item(const RenderArgs& a, const SubTile& t, const int4& item, int slot,
                                            float3 acc, int misses, float* __restrict__ image) {
  const int lane = threadIdx.x & 31;
  if (item.z == 1) {
    write_pixel(a, t, acc, misses, image);
    return;
  }
  a.wk.part[(size_t)slot * 32 + lane] = make_float4(acc.x, acc.y, acc.z, (float)misses);
  // every lane's sums are visible device-wide before lane 0 counts the item (the fence
  // orders each lane's own store; the warp barrier puts all of them before the count)
  __threadfence();
  __syncwarp();
  unsigned prev = 0;
  if (lane == 0) prev = atomicAdd(&a.wk.st_done[item.x], 1u);
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev != (unsigned)item.z - 1u) return;
  __threadfence();
  if (!in_range(a.status, (long long)item.w + item.z - 1, 0, a.wk.item_cap)) return;
  float3 tot = make_float3(0.0f, 0.0f, 0.0f);
  float tmiss = 0.0f;
  for (int c = 0; c < item.z; ++c) {
    const float4 p = __ldcg(&a.wk.part[(size_t)(item.w + c) * 32 + lane]);   // written on other SMs
    tot.x += p.x;
    tot.y += p.y;
    tot.z += p.z;
    tmiss += p.w;
  }
  write_pixel(a, t, tot, (int)tmiss, image);
  if (lane == 0) a.wk.st_done[item.x] = 0u;   // ready for the next launch
}

// warps take work items, instance after instance; S samples per lane at a time
template <bool STATS, int S>
__global__ void __launch_bounds__(kRenderThreads, 6) k_shade_fwd(RenderArgs a_in, float* __restrict__ image,
                                                                  unsigned long long* stats) {
  pdl_wait();
  __shared__ Cam scam[kWarps];
  const RenderArgs a0 = with_iter(a_in);
  Counts cnt;
  for (int inst = 0; inst < a0.n_inst; ++inst) {
    const int n = item_count(a0, inst), nf = front_count(a0, inst), ibase = inst_ibase(a0, inst);
    const RenderArgs a = for_inst(a0, inst);
    for (;;) {
      const int it = next_item(a, inst, n);
      if (it < 0) break;
      const int slot = ibase + item_slot(a, inst, it, nf);
      int4 item;
      SubTile t;
      int2 pk;
      if (!load_item(a, slot, item, t, pk) || t.inst != inst) continue;
      if (pk.y < 0) continue;   // no candidate list: k_overflow traces this item
      const Cam& cam = warp_cam(&scam[threadIdx.x >> 5], a.cams, t.view);
      int s0, s1;
      item_samples(item.y, item.z, t.spp, s0, s1);
      float3 acc = make_float3(0.0f, 0.0f, 0.0f);
      int misses = 0;
      shade_samples<STATS, S, false>(a, t, cam, pk.x, pk.y, s0, s1, acc, misses, cnt);
      finish_item(a, t, item, slot, acc, misses, image);
    }
  }
  flush_counts<STATS>(cnt, stats);
}

// one warp per sub-tile with items: its item sums in item order, then the pixel
// The rare paths, kept out of the gather and the shaders so that their registers are
// sized for their own work: (1) sub-tiles whose work items did not fit their
// instance's region -- one warp does a whole sub-tile, all its samples, in the chunks
// the items would have had (the forward writes its pixels, the backward adds to the
// instance's extra sums); (2) work items of sub-tiles without a usable candidate list
// (more candidates than the gather's list holds, or the pool full), traced ray by ray.
template <bool BWD, bool STATS>
__global__ void __launch_bounds__(kRenderThreads, BWD ? kBwdMinBlocks : 8) k_overflow(RenderArgs a_in,
                                                                                     const float* __restrict__ adjoint,
                                                            float* __restrict__ image, unsigned long long* stats) {
  pdl_wait();
  const RenderArgs a0 = with_iter(a_in);
  const int total = subtile_count(a0);
  const int n = (int)min(*reinterpret_cast<volatile unsigned*>(&a0.wk.ctr[2 + 2 * a0.n_inst]), (unsigned)total);
  Counts cnt;
  for (int i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < n; i += gridDim.x * kWarps) {
    const int st = a0.wk.ovf[i];
    if (!in_range(a0.status, st, 0, total)) continue;
    const SubTile t = subtile(a0, st);
    if (!in_range(a0.status, t.inst, 0, a0.n_inst)) continue;
    const RenderArgs a = for_inst(a0, t.inst);
    int2 pk = a.wk.st[st];
    if (pk.y > 0 && !in_range(a.status, (long long)pk.x + pk.y - 1, 0, a.wk.pool_cap)) pk.y = -1;
    const Cam cam = load_cam(a.cams, t.view);
    if (BWD) {
      // in the items' chunks too: each chunk's runs are added exactly as its work item
      // would add them, so fixed-point sums do not depend on which sub-tiles overflowed
      bool live;
      const float3 g = lane_adjoint(a, t, adjoint, live);
      const int C = chunks_for(a, pk.y, t.spp);
      for (int c = 0; c < C; ++c) {
        int s0, s1;
        item_samples(c, C, t.spp, s0, s1);
        if (a.wk.det) {
          unsigned long long* ex = a.wk.fx + (size_t)t.inst * 6 * a.V;
          grad_samples<STATS, 1>(a, t, cam, pk.x, pk.y, s0, s1, live, g, ex, ex + 3 * a.V, cnt);
        } else {
          float* ex = a.wk.extra + (size_t)t.inst * 6 * a.V;
          grad_samples<STATS, 1>(a, t, cam, pk.x, pk.y, s0, s1, live, g, ex, ex + 3 * a.V, cnt);
        }
      }
    } else {
      // the same chunks and the same order of sums as the work items and finish_item
      // would use, so a pixel's value does not depend on which path rendered it
      const int C = chunks_for(a, pk.y, t.spp);
      float3 tot = make_float3(0.0f, 0.0f, 0.0f);
      float tmiss = 0.0f;
      for (int c = 0; c < C; ++c) {
        int s0, s1;
        item_samples(c, C, t.spp, s0, s1);
        float3 acc = make_float3(0.0f, 0.0f, 0.0f);
        int misses = 0;
        shade_samples<STATS, 1>(a, t, cam, pk.x, pk.y, s0, s1, acc, misses, cnt);
        tot.x += acc.x;
        tot.y += acc.y;
        tot.z += acc.z;
        tmiss += (float)misses;
      }
      write_pixel(a, t, tot, (int)tmiss, image);
    }
  }
  // work items of sub-tiles without a candidate list (the shaders skip them, the gather
  // lists them): traced ray by ray, the forward finishing each item as the shader
  // would, the backward adding to the instance's extra sums
  const int nt = (int)min(*reinterpret_cast<volatile unsigned*>(&a0.wk.ctr[ctr_trace(a0.n_inst)]),
                          (unsigned)a0.wk.item_cap);
  for (int i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < nt; i += gridDim.x * kWarps) {
    const int slot = a0.wk.trace[i];
    if (!in_range(a0.status, slot, 0, a0.wk.item_cap)) continue;
    int4 item;
    SubTile t;
    int2 pk;
    if (!load_item(a0, slot, item, t, pk) || pk.y >= 0) continue;
    const RenderArgs a = for_inst(a0, t.inst);
    const Cam cam = load_cam(a.cams, t.view);
    int s0, s1;
    item_samples(item.y, item.z, t.spp, s0, s1);
    if (BWD) {
      bool live;
      const float3 g = lane_adjoint(a, t, adjoint, live);
      if (a.wk.det) {
        unsigned long long* ex = a.wk.fx + (size_t)t.inst * 6 * a.V;
        grad_samples<STATS, 1>(a, t, cam, pk.x, pk.y, s0, s1, live, g, ex, ex + 3 * a.V, cnt);
      } else {
        float* ex = a.wk.extra + (size_t)t.inst * 6 * a.V;
        grad_samples<STATS, 1>(a, t, cam, pk.x, pk.y, s0, s1, live, g, ex, ex + 3 * a.V, cnt);
      }
    } else {
      float3 acc = make_float3(0.0f, 0.0f, 0.0f);
      int misses = 0;
      shade_samples<STATS, 1>(a, t, cam, pk.x, pk.y, s0, s1, acc, misses, cnt);
      finish_item(a, t, item, slot, acc, misses, image);
    }
  }
  flush_counts<STATS>(cnt, stats);
}

// interior term: warps take work items.  ACC selects where the gradient collects;
// every mode adds with atomic adds whose result is not read, which retire in L2
// without holding up the warp (float adds to shared memory cost a read and a
// compare-and-swap loop each, and made the sums a quarter of this kernel's time):
//   kAccPartials  block b into partial b % nparts of `nparts` partials [6V]
//                 (L2-resident, zeroed before the launch), summed in partial order by
//                 k_reduce_partials (single instance)
//   kAccDirect    every run of hits on one triangle straight into its instance's
//                 extra [6V] (batches)
//   kAccGlobal    meshes beyond kPartialMaxV vertices: into the instance's float64
//                 extra64 [6V] (long runs of cancelling contributions)
//   kAccFixed     HR_DETERMINISTIC: into the instance's fixed-point sums fx [6V]
//                 (order-free integer atomics)
constexpr int kAccPartials = 0, kAccDirect = 1, kAccGlobal = 2, kAccFixed = 3;
template <bool STATS, int ACC, int S>
__global__ void __launch_bounds__(kRenderThreads, kBwdMinBlocks) k_shade_bwd(RenderArgs a_in,
                                                                             const float* __restrict__ adjoint,
                                                                             float* __restrict__ partials, int nparts,
                                                                             unsigned long long* stats) {
  pdl_wait();
  __shared__ Cam scam[kWarps];
  const RenderArgs a0 = with_iter(a_in);
  float* part = partials + (size_t)(blockIdx.x % nparts) * 6 * a0.V;
  Counts cnt;
  for (int inst = 0; inst < a0.n_inst; ++inst) {
    const int n = item_count(a0, inst), nf = front_count(a0, inst), ibase = inst_ibase(a0, inst);
    const RenderArgs a = for_inst(a0, inst);
    typedef typename std::conditional<
        ACC == kAccGlobal, double, typename std::conditional<ACC == kAccFixed, unsigned long long, float>::type>::type
        AccT;
    AccT* sdV;
    if constexpr (ACC == kAccGlobal)
      sdV = a0.wk.extra64 + (size_t)inst * 6 * a0.V;
    else if constexpr (ACC == kAccFixed)
      sdV = a0.wk.fx + (size_t)inst * 6 * a0.V;
    else if constexpr (ACC == kAccDirect)
      sdV = a0.wk.extra + (size_t)inst * 6 * a0.V;
    else
      sdV = part;
    AccT* sdN = sdV + 3 * a0.V;
    for (;;) {
      const int it = next_item(a, inst, n);
      if (it < 0) break;
      int4 item;
      SubTile t;
      int2 pk;
      if (!load_item(a, ibase + item_slot(a, inst, it, nf), item, t, pk) || t.inst != inst) continue;
      if (pk.y < 0) continue;   // no candidate list: k_overflow traces this item
      bool live;
      const float3 g = lane_adjoint(a, t, adjoint, live);
      const Cam& cam = warp_cam(&scam[threadIdx.x >> 5], a.cams, t.view);
      int s0, s1;
      item_samples(item.y, item.z, t.spp, s0, s1);
      grad_samples<STATS, S, AccT, false>(a, t, cam, pk.x, pk.y, s0, s1, live, g, sdV, sdN, cnt);
    }
  }
  flush_counts<STATS>(cnt, stats);
}

// d_verts[i] = extra[i] + sum_b partials[b][i] (i < 3V), dN[i-3V] likewise.  A block
// covers 32 entries with 16 groups of threads: group g sums partials g, g + 16, ...
// in order, then the 16 group sums are added in group order (a fixed order for every
// call).  blockIdx.y selects the instance (a batch has no partials).
constexpr int kRedEntries = 32, kRedGroups = 16;
__global__ void __launch_bounds__(kRedEntries * kRedGroups) k_reduce_partials(
    const float* __restrict__ partials, const float* __restrict__ extra_all, const double* __restrict__ extra64_all,
    const unsigned long long* __restrict__ fx_all, int nblocks, int V, float* __restrict__ d_verts_all,
    float* __restrict__ dN_all) {
  pdl_wait();
  __shared__ float red[kRedGroups][kRedEntries];
  const int j = threadIdx.x % kRedEntries, g = threadIdx.x / kRedEntries;
  const int i = blockIdx.x * kRedEntries + j;
  float acc = 0.0f;
  if (i < 6 * V) {
#pragma unroll 4
    for (int b = g; b < nblocks; b += kRedGroups) acc += partials[(size_t)b * 6 * V + i];
  }
  red[g][j] = acc;
  __syncthreads();
  if (g != 0 || i >= 6 * V) return;
  const float* extra = extra_all + (size_t)blockIdx.y * 6 * V;
  float* d_verts = d_verts_all + (size_t)blockIdx.y * 3 * V;
  float* dN = dN_all + (size_t)blockIdx.y * 3 * V;
  float tot = extra[i];
  if (extra64_all) tot = (float)(extra64_all[(size_t)blockIdx.y * 6 * V + i] + (double)tot);
  if (fx_all) tot += from_fixed(fx_all[(size_t)blockIdx.y * 6 * V + i]);
  for (int q = 0; q < kRedGroups; ++q) tot += red[q][j];
  if (i < 3 * V) d_verts[i] = tot;
  else dN[i - 3 * V] = tot;
}

// per view: silhouette flags in edge order, compacted by a block-wide scan.  In a
// batch the view's instance (view table) selects the vertices ([V][3] per instance).
__global__ void k_silhouettes(const float* __restrict__ verts_all, const int* __restrict__ faces,
                              const int* __restrict__ edges, const int* __restrict__ edge_faces, int E,
                              const Cam* __restrict__ cams, const ViewRec* __restrict__ vt, int V,
                              int* __restrict__ lists, int stride, int* __restrict__ counts,
                              const int* __restrict__ active) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  const int view = blockIdx.x;
  if (vt && active && !active[__ldg(&vt[view].inst)]) return;   // a retired instance
  const float* verts = verts_all + (vt ? (size_t)__ldg(&vt[view].inst) * 3 * V : 0);
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

// nearer of two hits: smaller t, then the lower triangle id (a miss loses)
__device__ __forceinline__ bool nearer(const Hit& m, const Hit& h) {
  return m.tri >= 0 && (h.tri < 0 || m.t < h.t || (m.t == h.t && m.tri < h.tri));
}

// the nearest hit of a group of L lanes (all 32 lanes call; the result is the same in
// every lane of a group)
template <int L>
__device__ __forceinline__ Hit group_min(Hit m) {
#pragma unroll
  for (int sh = L / 2; sh > 0; sh >>= 1) {
    Hit o;
    o.t = __shfl_xor_sync(0xffffffffu, m.t, sh, L);
    o.tri = __shfl_xor_sync(0xffffffffu, m.tri, sh, L);
    o.u = __shfl_xor_sync(0xffffffffu, m.u, sh, L);
    o.v = __shfl_xor_sync(0xffffffffu, m.v, sh, L);
    if (nearer(o, m)) m = o;
  }
  return m;
}

// boundary term (edge sampling).  A warp takes 32 / L samples, L lanes each: sample i
// of the launch is i % Ne_max of global view i / Ne_max (views with fewer samples skip
// the rest).  The lanes of a group compute the sample's set-up redundantly (same
// values, broadcast loads), then search the depth-sorted candidates of the sub-tile
// under the sample L at a time, lane q of the group testing candidate base + q against
// both offset rays (f+ and f-) and the group keeping the nearest hit of each (t, then
// the lower triangle id).  A ray stops at the first group of candidates whose nearest
// depth lies beyond its hit: the hits are those of testing the candidates one by one
// in depth order.  The group's lanes add the six results (two endpoints x three
// coordinates).
__device__ __forceinline__ void add1(float* p, float x) { atomicAdd(p, x); }
__device__ __forceinline__ void add1(unsigned long long* p, float x) { add_fixed(p, x); }

// T: float sums (dedge [n_inst][3V]) or fixed-point sums (fx [n_inst][6V], dV part);
// L: lanes per sample (the tuning's edge_lanes)
template <bool STATS, class T, int L>
__global__ void __launch_bounds__(kRenderThreads) k_edge_samples(RenderArgs a_in, const float* __restrict__ adjoint,
                                                                 const int* __restrict__ edges,
                                                                 const int* __restrict__ lists, int stride,
                                                                 const int* __restrict__ counts, int Ne_max, float eps,
                                                                 T* __restrict__ d_verts_all, long long inst_stride,
                                                                 unsigned long long* stats) {
  static_assert(L == 2 || L == 4 || L == 8 || L == 16 || L == 32, "lanes per edge sample");
  const unsigned full = 0xffffffffu;
  const RenderArgs a0 = with_iter(a_in);
  const int lane = threadIdx.x & 31, q = lane % L;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long i = warp * (32 / L) + lane / L;
  const int nv = visit_views(a0);
  if (warp * (32 / L) >= (long long)nv * Ne_max) return;   // whole warps leave together
  Counts cnt;
  // ---- set-up (group-uniform); `active` groups go on to the search -------------
  bool active = i < (long long)nv * Ne_max;
  const int jv = active ? (int)(i / Ne_max) : 0, k = active ? (int)(i - (long long)jv * Ne_max) : 0;
  const int view = active ? visit_view(a0, jv) : 0;
  active = active && in_range(a0.status, view, 0, a0.nviews);
  SubTile vw;
  int st0 = 0, nsx = 1;
  RenderArgs a = a0;
  T* d_verts = d_verts_all;
  int nsil = 0, ia = 0, ib = 0, K = 0, off = 0, W = 1;
  float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f, x = 0.f, y = 0.f, xp = 0.f, yp = 0.f, xm = 0.f, ym = 0.f;
  int bxp = 0, byp = 0, bxm = 0, bym = 0;
  float3 A = make_float3(0.f, 0.f, 0.f), va = A, vb = A, dp = A, dm = A, o = A;
  Cam cam;
  if (active) {
    view_info(a0, view, vw, st0, nsx);
    const int Ne = a0.vt ? __ldg(&a0.vt[view].ne) : Ne_max;
    active = k < Ne && in_range(a0.status, vw.inst, 0, a0.n_inst) && inst_active(a0, vw.inst);
    if (active) {
      a = for_inst(a0, vw.inst);
      d_verts = d_verts_all + (size_t)vw.inst * inst_stride;
      nsil = counts[view];
      active = nsil > 0;
    }
    if (active) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)k, vw.ctr1, 0u, a.iter4 | 1u), a.key);
      const int si = (int)__umulhi(r.x, (uint32_t)nsil);
      const float t = u24(r.y);
      const int e = lists[(size_t)view * stride + si];
      ia = edges[2 * e];
      ib = edges[2 * e + 1];
      cam = load_cam(a.cams, view);
      va = ld3(a.verts + 3 * ia);
      vb = ld3(a.verts + 3 * ib);
      active = project(cam, va, ax, ay) && project(cam, vb, bx, by);
      if (active) {
        x = __fmaf_rn(t, __fsub_rn(bx, ax), ax);
        y = __fmaf_rn(t, __fsub_rn(by, ay), ay);
        const float nx = __fsub_rn(ay, by), ny = __fsub_rn(bx, ax);
        const float len = __fsqrt_rn(__fmaf_rn(nx, nx, __fmul_rn(ny, ny)));
        active = len > 0.0f;
        if (active) {
          const float nhx = __fdiv_rn(nx, len), nhy = __fdiv_rn(ny, len);
          const float fxp = floorf(x), fyp = floorf(y);
          W = vw.W;
          const int H = vw.H;
          active = !(fxp < 0.0f || fyp < 0.0f || fxp >= (float)W || fyp >= (float)H);
          if (active) {
            const int px = (int)fxp, py = (int)fyp;
            A = ld3(adjoint + 3 * (vw.pix0 + (size_t)py * W + px));
            active = A.x != 0.0f || A.y != 0.0f || A.z != 0.0f;
            if (active) {
              xp = __fmaf_rn(eps, nhx, x);
              yp = __fmaf_rn(eps, nhy, y);
              xm = __fmaf_rn(-eps, nhx, x);
              ym = __fmaf_rn(-eps, nhy, y);
              bxp = (int)fminf(fmaxf(floorf(xp), 0.0f), (float)(W - 1));
              byp = (int)fminf(fmaxf(floorf(yp), 0.0f), (float)(H - 1));
              bxm = (int)fminf(fmaxf(floorf(xm), 0.0f), (float)(W - 1));
              bym = (int)fminf(fmaxf(floorf(ym), 0.0f), (float)(H - 1));
              // the candidates of the sub-tile holding the centre pixel serve both
              // offset rays: its frustum is padded by half a pixel and the offsets are
              // far smaller
              const int st = st0 + (py / kSubH) * nsx + (px / kSubW);
              int2 pk = a.wk.st[st];
              if (pk.y > 0 && !in_range(a.status, (long long)pk.x + pk.y - 1, 0, a.wk.pool_cap)) pk.y = -1;
              off = pk.x;
              K = pk.y;
              o = make_float3(cam.c[0], cam.c[1], cam.c[2]);
              dp = primary_dir(cam, xp, yp);
              dm = primary_dir(cam, xm, ym);
              if (STATS && q == 0) {
                cnt.samples += 2;
                cnt.rays += 2;
              }
            }
          }
        }
      }
    }
  }
  Hit hp{-1, INFINITY, 0.0f, 0.0f}, hm{-1, INFINITY, 0.0f, 0.0f};
  // ---- no candidate list: lanes 0 and 1 of the group traverse the BVH -----------
  if (__any_sync(full, active && K < 0)) {
    Hit h{-1, INFINITY, 0.0f, 0.0f};
    if (active && K < 0 && q < 2) h = trace<STATS>(a.nodes, a.tris, o, q == 0 ? dp : dm, a.status, cnt, a.max_visits);
    const int g0 = lane - q;
    Hit r0, r1;
    r0.tri = __shfl_sync(full, h.tri, g0);
    r0.t = __shfl_sync(full, h.t, g0);
    r0.u = __shfl_sync(full, h.u, g0);
    r0.v = __shfl_sync(full, h.v, g0);
    r1.tri = __shfl_sync(full, h.tri, g0 + 1);
    r1.t = __shfl_sync(full, h.t, g0 + 1);
    r1.u = __shfl_sync(full, h.u, g0 + 1);
    r1.v = __shfl_sync(full, h.v, g0 + 1);
    if (active && K < 0) {
      hp = r0;
      hm = r1;
    }
  }
  // ---- candidate search, both rays together, L candidates per step ---------------
  bool donep = !(active && K > 0), donem = donep;
  for (int base = 0;; base += L) {
    const bool go = !(donep && donem) && base < K;
    if (!__any_sync(full, go)) break;
    Hit mp{-1, INFINITY, 0.0f, 0.0f}, mm{-1, INFINITY, 0.0f, 0.0f};
    if (go) {
      // group-uniform: no candidate from here on can be nearer than a ray's hit
      const float z0 = __ldg(&a.wk.z[off + base]);
      const float zl0 = z0 - (1e-4f * fabsf(z0) + 1e-6f);
      donep = donep || hp.t < zl0;
      donem = donem || hm.t < zl0;
      const int c = base + q;
      if (!(donep && donem) && c < K && in_range(a.status, off + c, 0, a.wk.pool_cap)) {
        const float zm = __ldg(&a.wk.z[off + c]);
        const float zl = zm - (1e-4f * fabsf(zm) + 1e-6f);
        bool tp = !donep && !(hp.t < zl), tm = !donem && !(hm.t < zl);
        if (tp || tm) {
          const float4 bb = __ldg(&a.wk.bb[off + c]);
          if (STATS) cnt.cands += (unsigned)tp + (unsigned)tm;
          tp = tp && xp >= bb.x && xp <= bb.z && yp >= bb.y && yp <= bb.w;
          tm = tm && xm >= bb.x && xm <= bb.z && ym >= bb.y && ym <= bb.w;
          if (tp || tm) {
            const int kr = __ldg(&a.wk.rec[off + c]);
            if (in_range(a.status, kr, 0, a.max_visits - 1)) {
              if (tp) isect<STATS>(a.tris, kr, o, dp, mp, cnt);
              if (tm) isect<STATS>(a.tris, kr, o, dm, mm, cnt);
            }
          }
        }
      }
    }
    mp = group_min<L>(mp);
    mm = group_min<L>(mm);
    if (go) {
      if (nearer(mp, hp)) hp = mp;
      if (nearer(mm, hm)) hm = mm;
    }
  }
  if (STATS) {
    if (q == 0) cnt.hits += (unsigned)(active && hp.tri >= 0) + (unsigned)(active && hm.tri >= 0);
    unsigned v[kStatsPer] = {cnt.samples, cnt.rays, cnt.nodes, cnt.tris, cnt.hits, cnt.cands};
    for (int s2 = 0; s2 < kStatsPer; ++s2) {
      unsigned long long xq = v[s2];
      for (int o2 = 16; o2 > 0; o2 >>= 1) xq += __shfl_down_sync(full, xq, o2);
      if (lane == 0 && xq) atomicAdd(stats + s2, xq);
    }
  }
  if (!active || q >= 6) return;
  const float3 fp = hp.tri >= 0 ? shade(a, hp) : ld3(a.bg + 3 * (vw.pix0 + (size_t)byp * W + bxp));
  const float3 fm = hm.tri >= 0 ? shade(a, hm) : ld3(a.bg + 3 * (vw.pix0 + (size_t)bym * W + bxm));
  const int Ne = a0.vt ? __ldg(&a0.vt[view].ne) : Ne_max;
  const float wgt = (A.x * (fp.x - fm.x) + A.y * (fp.y - fm.y) + A.z * (fp.z - fm.z)) * ((float)nsil / (float)Ne);
  if (wgt == 0.0f) return;
  const float dax = wgt * (by - y), day = wgt * (x - bx), dbx = wgt * (y - ay), dby = wgt * (ax - x);
  // the six results (endpoint ep = j / 3, coordinate j % 3), lanes q, q + L, ... of the
  // group: the projection Jacobian's transpose, J^T g = R^T (gx, gy, gz)
  for (int j = q; j < 6; j += L) {
    const int ep = j / 3, comp = j % 3;
    const float3 p = ep == 0 ? va : vb;
    const float g2x = ep == 0 ? dax : dbx, g2y = ep == 0 ? day : dby;
    const float X = cam.R[0] * p.x + cam.R[1] * p.y + cam.R[2] * p.z + cam.t[0];
    const float Y = cam.R[3] * p.x + cam.R[4] * p.y + cam.R[5] * p.z + cam.t[1];
    const float Z = cam.R[6] * p.x + cam.R[7] * p.y + cam.R[8] * p.z + cam.t[2];
    const float iz = 1.0f / Z;
    const float gx = g2x * cam.fx * iz, gy = g2y * cam.fy * iz;
    const float gz = -(gx * X + gy * Y) * iz;
    add1(&d_verts[3 * (ep == 0 ? ia : ib) + comp], cam.R[comp] * gx + cam.R[3 + comp] * gy + cam.R[6 + comp] * gz);
  }
}

// dm_u = (I - n n^T) dN_u / |m_u|: the adjoint of the unnormalised normal m_u of
// vertex u from that of its unit normal
__device__ __forceinline__ float3 normal_dm(const float* __restrict__ normals, const float* __restrict__ normal_len,
                                           const float* __restrict__ dN, int u) {
  const float len = normal_len[u];
  const float3 n = ld3(normals + 3 * u), g = ld3(dN + 3 * u);
  if (!(len > 0.0f)) return make_float3(0.0f, 0.0f, 0.0f);
  const float pr = dot3(n, g);
  const float il = 1.0f / len;
  return make_float3((g.x - n.x * pr) * il, (g.y - n.y * pr) * il, (g.z - n.z * pr) * il);
}

// d_verts[v] += sum over incident faces of d(e1 x e2)/dv . dc_f, dc_f = sum of dm
// over f's vertices (dm computed here from dN for each of them: no pass of its own);
// plus the edge term's sums when dedge is given.  blockIdx.y selects the instance.
__global__ void k_normal_gather(const float* __restrict__ verts_all, const int* __restrict__ faces,
                                const int* __restrict__ vf_off, const int* __restrict__ vf_faces,
                                const float* __restrict__ normals_all, const float* __restrict__ normal_len_all,
                                const float* __restrict__ dN_all, int V, const float* __restrict__ dedge_all,
                                float* __restrict__ d_verts_all, const int* __restrict__ active) {
  pdl_wait();
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V || (active && !active[blockIdx.y])) return;
  const size_t o = (size_t)blockIdx.y * 3 * V;
  const float *verts = verts_all + o, *normals = normals_all + o, *dN = dN_all + o;
  const float* normal_len = normal_len_all + (size_t)blockIdx.y * V;
  float* d_verts = d_verts_all + o;
  float3 acc = make_float3(0.0f, 0.0f, 0.0f);
  if (dedge_all) acc = ld3(dedge_all + o + 3 * v);
  for (int k = vf_off[v]; k < vf_off[v + 1]; ++k) {
    int f = vf_faces[k];
    int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    float3 dc = normal_dm(normals, normal_len, dN, i0);
    float3 t1 = normal_dm(normals, normal_len, dN, i1), t2 = normal_dm(normals, normal_len, dN, i2);
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

// d_verts += dedge (the edge term's sums, when the normals' adjoint is off)
__global__ void k_add_edges(const float* __restrict__ dedge, long long n, float* __restrict__ d_verts) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d_verts[i] += dedge[i];
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


// HR_TIMING: event pair (2 slot, 2 slot + 1) around internal kernel `slot`
struct Timer {
  Context* ctx;
  cudaStream_t s;
  bool on;
  void begin(int slot) {
    if (on) cudaEventRecord(ctx->ev[2 * slot], s);
  }
  void end(int slot) {
    if (on) cudaEventRecord(ctx->ev[2 * slot + 1], s);
  }
};

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
  a.iter_dev = o->iter_dev;
  a.sh.l = make_float3(o->light_dir[0], o->light_dir[1], o->light_dir[2]);
  a.sh.lrgb = make_float3(o->light_rgb[0], o->light_rgb[1], o->light_rgb[2]);
  a.sh.ka = o->ka;
  a.sh.kd = o->kd;
  a.status = ctx->status;
  a.max_visits = ctx->F + 1;
  a.wk.bb = ctx->pool_bb;
  a.wk.z = ctx->pool_z;
  a.wk.rec = ctx->pool_rec;
  a.wk.pool_cap = ctx->pool_cap;
  a.wk.st = ctx->st_info;
  a.wk.items = ctx->items;
  a.wk.item_cap = ctx->item_cap;
  a.wk.part = ctx->item_part;
  a.wk.extra = ctx->extra;
  a.wk.extra64 = ctx->extra64;
  a.wk.ctr = ctx->work_ctr;
  a.wk.ovf = ctx->ovf_list;
  a.wk.trace = ctx->trace_list;
  a.wk.st_done = ctx->st_done;
  a.wk.cand_st = ctx->cand_st;
  a.wk.bin = ctx->bin_cnt;
  a.wk.bvh_need = ctx->bvh_need;
  a.wk.fx = ctx->acc_fx;
  a.wk.det = (o->flags & HR_DETERMINISTIC) != 0;
  a.node_stride = ctx->lim.max_F;
  a.cand_per_chunk = ctx->tune.cand_per_chunk;
  a.max_chunks = ctx->tune.max_chunks;
  a.uv = m->uv;
  a.tex = (o->texture && m->uv) ? o->texture : nullptr;
  a.tex_w = o->tex_w;
  a.tex_h = o->tex_h;
  a.d_tex = a.tex ? o->d_texture : nullptr;
  a.active = ctx->vt ? ctx->active : nullptr;
  a.act_off = a.active ? ctx->act_off : nullptr;
  if (ctx->vt) {
    a.vt = ctx->vt;
    a.it = ctx->it;
    a.n_inst = ctx->n_inst;
    a.nviews = ctx->nviews;
    a.total_st = ctx->total_st;
  } else {
    a.vt = nullptr;
    a.it = nullptr;
    a.n_inst = 1;
    a.nviews = N;
    a.total_st = subtiles_for(N, W, H);
  }
  return a;
}

}  // namespace

int render_grid(int device, int* blocks, int* threads, int* num_sms) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HR_ERR_CUDA;
  *num_sms = sms;
  *threads = kRenderThreads;
  *blocks = sms * kBlocksPerSm;
  return HR_OK;
}

int subtiles_for(int views, int W, int H) { return views * ((W + kSubW - 1) / kSubW) * ((H + kSubH - 1) / kSubH); }
int subtile_columns(int W) { return (W + kSubW - 1) / kSubW; }

int launch_render_fwd(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int H, int W,
                      const float* bg, const hr_render_opts* o, float* image, cudaStream_t s) {
  RenderArgs a = make_args(ctx, m, verts, cams, N, H, W, bg, o);
  const bool st = o->flags & HR_STATS;
  Timer tm{ctx, s, (o->flags & HR_TIMING) != 0};
  if (cudaMemsetAsync(ctx->work_ctr, 0, ctr_words(a.n_inst) * sizeof(unsigned), s) != cudaSuccess)
    return HR_ERR_CUDA;
  if (a.act_off) {   // a batch with a mask: the active instances' sub-tiles and views
    k_active_layout<<<1, kLayoutThreads, 0, s>>>(ctx->it, ctx->active, ctx->n_inst, ctx->act_off);
    HR_CHECK_LAUNCH();
  }
  const int blocks = ctx->num_sms * ctx->tune.blocks_per_sm;
  tm.begin(kTimeFwdGather);
  // candidate lists: bin the (view, record) pairs into sub-tiles (count), give each
  // sub-tile its pool range and work items, bin again into the ranges (fill), order
  // each list by nearest depth.  The bins are zero between forwards (cleared once at
  // creation, then by k_bin_alloc and k_bin_sort).  The background sub-tiles' pixels
  // are written on the context's second stream beside the fill and the sort (with
  // kernel timing on, on the caller's stream), joined before the call returns.
  const bool fork = !tm.on;
  cudaStream_t bs = fork ? ctx->side : s;
  {
    const long long pairs = (long long)a.nviews * (a.max_visits - 1);
    const long long bin_warps = (pairs + kBinPairs - 1) / kBinPairs;
    const int bin_blocks = (int)std::min<long long>((bin_warps + kBinThreads / 32 - 1) / (kBinThreads / 32), 8LL * ctx->num_sms);
    launch_pdl(k_bin<false>, dim3(std::max(bin_blocks, 1)), dim3(kBinThreads), 0, s, a, ctx->bin_cnt);
    HR_CHECK_LAUNCH();
    const int group_blocks = ctx->num_sms * 8;
    launch_pdl(k_bin_alloc, dim3(group_blocks), dim3(kGroupThreads), 0, s, a, ctx->bin_cnt);
    HR_CHECK_LAUNCH();
    if (fork && (cudaEventRecord(ctx->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(bs, ctx->ev_fork, 0) != cudaSuccess))
      return HR_ERR_CUDA;
    const int bg_blocks = ctx->num_sms * 4;   // one wave at k_background's 64 registers
    if (st)
      k_background<true><<<bg_blocks, kGroupThreads, 0, bs>>>(a, image, ctx->stats);
    else
      k_background<false><<<bg_blocks, kGroupThreads, 0, bs>>>(a, image, nullptr);
    HR_CHECK_LAUNCH();
    // the boxes of a tree whose update rewrote only the records, refitted if a sub-tile
    // was listed for per-ray traversal (k_overflow is the first to traverse)
    const int rc = launch_bvh_lazy_refit(ctx, 0, bs);
    if (rc != HR_OK) return rc;
    if (fork && cudaEventRecord(ctx->ev_join, bs) != cudaSuccess) return HR_ERR_CUDA;
    launch_pdl(k_bin<true>, dim3(std::max(bin_blocks, 1)), dim3(kBinThreads), 0, s, a, ctx->bin_cnt);
    HR_CHECK_LAUNCH();
    launch_pdl(k_bin_sort, dim3(blocks), dim3(kRenderThreads), 0, s, a);
    HR_CHECK_LAUNCH();
  }
  tm.end(kTimeFwdGather);
  tm.begin(kTimeFwdShade);
  {
    const int S = ctx->tune.rays_per_lane;
    auto kern = st ? (S == 1 ? k_shade_fwd<true, 1> : (S == 2 ? k_shade_fwd<true, 2> : k_shade_fwd<true, 4>))
                   : (S == 1 ? k_shade_fwd<false, 1> : (S == 2 ? k_shade_fwd<false, 2> : k_shade_fwd<false, 4>));
    launch_pdl(kern, dim3(blocks), dim3(kRenderThreads), 0, s, a, image, st ? ctx->stats : nullptr);
  }
  HR_CHECK_LAUNCH();
  if (fork && cudaStreamWaitEvent(s, ctx->ev_join, 0) != cudaSuccess) return HR_ERR_CUDA;
  if (st)
    launch_pdl(k_overflow<false, true>, dim3(blocks), dim3(kRenderThreads), 0, s, a, nullptr, image, ctx->stats);
  else
    launch_pdl(k_overflow<false, false>, dim3(blocks), dim3(kRenderThreads), 0, s, a, nullptr, image,
               (unsigned long long*)nullptr);
  HR_CHECK_LAUNCH();
  tm.end(kTimeFwdShade);
  // the item sums are combined inside the shaders (finish_item): the slot stays, empty
  tm.begin(kTimeFwdCombine);
  tm.end(kTimeFwdCombine);
  if (tm.on) ctx->ev_ready |= 1;
  ctx->fwd_verts = verts;
  ctx->fwd_cams = cams;
  ctx->fwd_N = N;
  ctx->fwd_H = H;
  ctx->fwd_W = W;
  ctx->fwd_spp = o->spp;
  ctx->fwd_gen = ctx->bvh_gen;
  ctx->fwd_valid = true;
  return HR_OK;
}

int launch_silhouettes(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int* lists,
                       int list_stride, int* counts, cudaStream_t s) {
  k_silhouettes<<<N, 512, 0, s>>>(verts, m->faces, m->edges, m->edge_faces, m->E, cams, ctx->vt, m->V, lists,
                                  list_stride, counts, ctx->vt ? ctx->active : nullptr);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_render_bwd(Context* ctx, const hr_model* m, const float* verts, const Cam* cams, int N, int H, int W,
                      const float* bg, const hr_render_opts* o, const float* adjoint, float* d_verts,
                      cudaStream_t s) {
  RenderArgs a = make_args(ctx, m, verts, cams, N, H, W, bg, o);
  a.cand_per_chunk = ctx->tune.bwd_cand_per_chunk;   // the backward's own work-item split
  if (a.act_off) {   // a batch with a mask: the active instances' sub-tiles and views
    k_active_layout<<<1, kLayoutThreads, 0, s>>>(ctx->it, ctx->active, ctx->n_inst, ctx->act_off);
    HR_CHECK_LAUNCH();
  }
  const int V = m->V, ni = a.n_inst, nv = a.nviews;
  const bool batch = ctx->vt != nullptr;
  const int Ne = batch ? ctx->max_ne : o->edge_samples;
  const bool interior = !(o->flags & HR_BWD_NO_INTERIOR);
  const bool edges = !(o->flags & HR_BWD_NO_EDGES) && Ne > 0;
  const bool normals = !(o->flags & HR_BWD_NO_NORMALS) && interior;
  const bool st = o->flags & HR_STATS;
  Timer tm{ctx, s, (o->flags & HR_TIMING) != 0};
  if (interior || edges) {
    // candidates of the sub-tiles with a non-zero adjoint: the interior shader's work
    // items, and the edge rays' candidate lists
    if (cudaMemsetAsync(ctx->work_ctr, 0, ctr_words(ni) * sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(ctx->extra, 0, sizeof(float) * 6 * V * ni, s) != cudaSuccess)
      return HR_ERR_CUDA;
    // the forward's candidate lists still describe this scene when it used the same
    // vertices, cameras and sizes after the last build
    const bool reuse = (o->flags & HR_BWD_REUSE_FWD) && ctx->fwd_valid && ctx->fwd_verts == verts &&
                       ctx->fwd_cams == cams && ctx->fwd_N == N && ctx->fwd_H == H && ctx->fwd_W == W &&
                       (batch || ctx->fwd_spp == o->spp) && ctx->fwd_gen == ctx->bvh_gen;
    tm.begin(kTimeBwdGather);
    if (reuse) {
      if (st)
        launch_pdl(k_items_bwd<true>, dim3(ctx->num_sms * 4), dim3(kGroupThreads), 0, s, a, adjoint, ctx->stats + kStatsPer);
      else
        launch_pdl(k_items_bwd<false>, dim3(ctx->num_sms * 4), dim3(kGroupThreads), 0, s, a, adjoint,
                   (unsigned long long*)nullptr);
    } else {
      // its own lists from a frustum walk of the BVH: the boxes must be current
      const int rc = launch_bvh_lazy_refit(ctx, 1, s);
      if (rc != HR_OK) return rc;
      if (st)
        k_gather<true><<<ctx->num_sms * ctx->tune.blocks_per_sm, kRenderThreads, 0, s>>>(a, adjoint,
                                                                            ctx->stats + kStatsPer);
      else
        k_gather<false><<<ctx->num_sms * ctx->tune.blocks_per_sm, kRenderThreads, 0, s>>>(a, adjoint, nullptr);
    }
    HR_CHECK_LAUNCH();
    tm.end(kTimeBwdGather);
  }
  // The edge-sampling term (silhouettes, edge samples into ctx->dedge) needs only the
  // candidate lists made above; it runs on the context's side stream beside the
  // interior shader and joins before the normals' adjoint adds it to d_verts.  With
  // kernel timing on, everything stays on the caller's stream.  HR_DETERMINISTIC:
  // everything stays on the caller's stream, both terms add their vertex sums to the
  // fixed-point array, and one reduction after both turns it into d_verts and dN.
  const bool det = (o->flags & HR_DETERMINISTIC) != 0;
  const bool fork = edges && !tm.on && !det;
  cudaStream_t es = fork ? ctx->side : s;
  if (det && cudaMemsetAsync(ctx->acc_fx, 0, sizeof(unsigned long long) * 6 * V * ni, s) != cudaSuccess)
    return HR_ERR_CUDA;
  if (edges) {
    if (fork && (cudaEventRecord(ctx->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(es, ctx->ev_fork, 0) != cudaSuccess))
      return HR_ERR_CUDA;
    if (!det && cudaMemsetAsync(ctx->dedge, 0, sizeof(float) * 3 * V * ni, es) != cudaSuccess) return HR_ERR_CUDA;
  }
  const auto reduce = [&](int acc, int nparts) {
    launch_pdl(k_reduce_partials, dim3((6 * V + kRedEntries - 1) / kRedEntries, ni), dim3(kRedEntries * kRedGroups), 0,
               s, (const float*)ctx->partials, (const float*)ctx->extra,
               (const double*)(acc == kAccGlobal ? ctx->extra64 : nullptr),
               (const unsigned long long*)(det ? ctx->acc_fx : nullptr), acc == kAccPartials ? nparts : 0, V, d_verts,
               ctx->dN);
  };
  if (interior) {
    // float sums up to kPartialMaxV vertices (per block, or per instance in a batch),
    // float64 beyond; fixed-point sums when deterministic
    const bool global_acc = V > kPartialMaxV;
    if (!det && global_acc &&
        (!ctx->extra64 || cudaMemsetAsync(ctx->extra64, 0, sizeof(double) * 6 * V * ni, s) != cudaSuccess))
      return ctx->extra64 ? HR_ERR_CUDA : HR_ERR_UNSUPPORTED;
    const int acc = det ? kAccFixed : (global_acc ? kAccGlobal : (batch ? kAccDirect : kAccPartials));
    // deterministic: one ray per lane, the arithmetic of the overflow kernel, which may
    // trace any sub-tile whose candidates found no room in the pool
    const int S = det ? 1 : ctx->tune.bwd_rays_per_lane;
#define HR_BWD_KERNEL(A_) \
  (st ? (S == 1 ? k_shade_bwd<true, A_, 1> : (S == 2 ? k_shade_bwd<true, A_, 2> : k_shade_bwd<true, A_, 4>)) \
      : (S == 1 ? k_shade_bwd<false, A_, 1> : (S == 2 ? k_shade_bwd<false, A_, 2> : k_shade_bwd<false, A_, 4>)))
    auto kern = acc == kAccFixed    ? HR_BWD_KERNEL(kAccFixed)
                : acc == kAccGlobal ? HR_BWD_KERNEL(kAccGlobal)
                                    : (acc == kAccDirect ? HR_BWD_KERNEL(kAccDirect) : HR_BWD_KERNEL(kAccPartials));
#undef HR_BWD_KERNEL
    // one partial per SM (the blocks of a launch share them round-robin), zeroed first
    const int blocks = ctx->num_sms * ctx->tune.bwd_blocks_per_sm;
    const int nparts = ctx->num_sms;
    if (acc == kAccPartials &&
        cudaMemsetAsync(ctx->partials, 0, sizeof(float) * 6 * V * (size_t)nparts, s) != cudaSuccess)
      return HR_ERR_CUDA;
    tm.begin(kTimeBwdShade);
    launch_pdl(kern, dim3(blocks), dim3(kRenderThreads), 0, s, a, adjoint, ctx->partials, nparts,
               st ? ctx->stats + kStatsPer : nullptr);
    HR_CHECK_LAUNCH();
    if (st)
      launch_pdl(k_overflow<true, true>, dim3(blocks), dim3(kRenderThreads), 0, s, a, adjoint, (float*)nullptr,
                 ctx->stats + kStatsPer);
    else
      launch_pdl(k_overflow<true, false>, dim3(blocks), dim3(kRenderThreads), 0, s, a, adjoint, (float*)nullptr,
                 (unsigned long long*)nullptr);
    HR_CHECK_LAUNCH();
    tm.end(kTimeBwdShade);
    if (!det) {
      tm.begin(kTimeBwdReduce);
      reduce(acc, nparts);
      HR_CHECK_LAUNCH();
      tm.end(kTimeBwdReduce);
    }
  } else if (!det) {
    if (cudaMemsetAsync(d_verts, 0, sizeof(float) * 3 * V * ni, s) != cudaSuccess) return HR_ERR_CUDA;
  }
  if (edges) {
    tm.begin(kTimeBwdSil);
    int rc = launch_silhouettes(ctx, m, verts, cams, nv, ctx->sil, ctx->lim.max_E, ctx->sil_count, es);
    if (rc != HR_OK) return rc;
    tm.end(kTimeBwdSil);
    // edge_lanes lanes per edge sample
    const int L = ctx->tune.edge_lanes;
    const long long n = ((long long)nv * Ne + 32 / L - 1) / (32 / L) * 32;
    const unsigned grid = (unsigned)((n + kRenderThreads - 1) / kRenderThreads);
    tm.begin(kTimeBwdEdges);
#define HR_EDGE_KERNEL(T_)                                                                            \
  (st ? (L == 2 ? k_edge_samples<true, T_, 2> : L == 4 ? k_edge_samples<true, T_, 4>                  \
         : L == 8 ? k_edge_samples<true, T_, 8> : L == 16 ? k_edge_samples<true, T_, 16>              \
                                                        : k_edge_samples<true, T_, 32>)               \
      : (L == 2 ? k_edge_samples<false, T_, 2> : L == 4 ? k_edge_samples<false, T_, 4>                \
         : L == 8 ? k_edge_samples<false, T_, 8> : L == 16 ? k_edge_samples<false, T_, 16>            \
                                                         : k_edge_samples<false, T_, 32>))
    if (det) {
      auto kern = HR_EDGE_KERNEL(unsigned long long);
      kern<<<grid, kRenderThreads, 0, es>>>(a, adjoint, m->edges, ctx->sil, ctx->lim.max_E, ctx->sil_count, Ne,
                                            o->edge_eps_px, ctx->acc_fx, 6LL * V, ctx->stats + 2 * kStatsPer);
    } else {
      auto kern = HR_EDGE_KERNEL(float);
      kern<<<grid, kRenderThreads, 0, es>>>(a, adjoint, m->edges, ctx->sil, ctx->lim.max_E, ctx->sil_count, Ne,
                                            o->edge_eps_px, ctx->dedge, 3LL * V, ctx->stats + 2 * kStatsPer);
    }
#undef HR_EDGE_KERNEL
    HR_CHECK_LAUNCH();
    tm.end(kTimeBwdEdges);
    if (fork && (cudaEventRecord(ctx->ev_join, es) != cudaSuccess || cudaStreamWaitEvent(s, ctx->ev_join, 0) != cudaSuccess))
      return HR_ERR_CUDA;
  }
  if (det) {
    tm.begin(kTimeBwdReduce);
    reduce(kAccFixed, 0);
    HR_CHECK_LAUNCH();
    tm.end(kTimeBwdReduce);
  }
  if (normals) {
    tm.begin(kTimeBwdNormals);
    const dim3 g((V + 255) / 256, ni);
    const int* act = batch ? ctx->active : nullptr;
    launch_pdl(k_normal_gather, g, dim3(256), 0, s, verts, m->faces, m->vf_offsets, m->vf_faces,
               (const float*)ctx->normals, (const float*)ctx->normal_len, (const float*)ctx->dN, V,
               (const float*)(edges && !det ? ctx->dedge : nullptr), d_verts, act);
    HR_CHECK_LAUNCH();
    tm.end(kTimeBwdNormals);
  } else if (edges && !det) {
    const long long n3 = 3LL * V * ni;
    k_add_edges<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(ctx->dedge, n3, d_verts);
    HR_CHECK_LAUNCH();
  }
  if (tm.on) ctx->ev_ready |= 2 | (interior ? 4 : 0) | (edges ? 8 : 0) | (normals ? 16 : 0);
  return HR_OK;
}

int launch_trace(Context* ctx, const float* o, const float* d, int n, int* tri, float* tuv, cudaStream_t s) {
  const int rc = launch_bvh_lazy_refit(ctx, 1, s);   // traversal reads the boxes
  if (rc != HR_OK) return rc;
  k_trace<<<(n + 127) / 128, 128, 0, s>>>(ctx->nodes, ctx->tris, o, d, n, tri, tuv, ctx->status, ctx->F + 1);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

}  // namespace hr
