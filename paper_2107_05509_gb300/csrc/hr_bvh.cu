// Per-iteration scene build: a Morton-code linear BVH over the current triangles
// (Karras, "Maximizing parallelism in the construction of BVHs, octrees, and k-d
// trees", HPG 2012) and the area-weighted unit vertex normals used for shading.
//
// Each instance's build runs in ONE thread block (a batch builds all instances in
// one launch, one block each): at a hand's size (1.5k triangles) a build is
// latency-bound, and one block keeps every phase in shared memory with only
// __syncthreads between phases -- centroid bounds, 30-bit Morton codes, a bitonic
// sort of (code << 32 | triangle id) keys (unique, so the hierarchy has no
// duplicate-key special case), the hierarchy, then a bottom-up refit in which the
// second child to arrive at a node (atomic counter in shared memory) writes the
// union box into the parent.  When the nodes fit next to the keys (F up to ~2400) the
// hierarchy and the refit run on a shared-memory copy of the nodes that is written
// out once at the end, so the refit's dependent loads cost shared-memory latency.
// Leaf boxes are padded so that the float32 slab test can never reject a ray that
// the float32 Moller-Trumbore test would accept.
//
// Refit (hr_update_bvh): between full rebuilds the tree keeps its topology and leaf
// order, and only the triangle records and boxes are recomputed bottom-up.  Any tree
// whose boxes contain their children gives the same hits and the same candidate sets
// (a leaf reaches a frustum exactly when its own padded box does), so refitting
// changes speed, not results; the decision (*iter_dev % rebuild_every) is taken on
// the device, so a captured iteration replays it.
#include <cstdio>

#include "hr_internal.h"

namespace hr {

namespace {

constexpr int kBuildThreads = 1024;
// k_build_bvh modes: kBvhFull builds or refits (per the rebuild schedule) with fresh
// boxes; kBvhRecords builds per the schedule but on refit iterations rewrites only
// the triangle records and marks the boxes stale; kBvhLazyRefit refits stale boxes
// from the current records' leaf order when a render call needs traversal
constexpr int kBvhFull = 0, kBvhRecords = 1, kBvhLazyRefit = 2;
constexpr int kBuildSmemCap = 200 * 1024;   // opt-in of k_build_bvh

__device__ __forceinline__ unsigned expand_bits10(unsigned v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__device__ __forceinline__ int delta(const unsigned long long* keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(keys[i] ^ keys[j]);
}

// Internal node i (0 <= i < F - 1) of the hierarchy over F sorted Morton keys
// (Karras 2012, "Maximizing parallelism in the construction of BVHs, octrees, and k-d
// trees"): the direction of its key range from the common-prefix lengths of its
// neighbours, the range's far end by an exponential then a binary search, the split
// position by a binary search for the longest common prefix; children are internal
// nodes or leaves (encoded ~k, k = sorted position), and both record i as their
// parent (leaf k at parent[F + k]).  Keys, nodes and parents may live in shared or
// global memory.
__device__ __forceinline__ void karras_node(const unsigned long long* keys, int F, int i, Node* nodes, int* parent) {
  const int d = (delta(keys, F, i, i + 1) - delta(keys, F, i, i - 1)) > 0 ? 1 : -1;
  const int dmin = delta(keys, F, i, i - d);
  int lmax = 2;
  while (delta(keys, F, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, F, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta(keys, F, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, F, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  const int gamma = i + s * d + min(d, 0);
  const int left = (min(i, j) == gamma) ? ~gamma : gamma;
  const int right = (max(i, j) == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  nodes[i].d = make_int4(left, right, 0, 0);
  if (left >= 0) parent[left] = i; else parent[F + ~left] = i;
  if (right >= 0) parent[right] = i; else parent[F + ~right] = i;
  if (i == 0) parent[0] = -1;
}

__device__ __forceinline__ float warp_min(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct Box {
  float lo[3], hi[3];
};

__device__ __forceinline__ void store_slot(Node* nodes, int p, int slot, const Box& b) {
  volatile float* f = reinterpret_cast<volatile float*>(&nodes[p]);
  int o = slot ? 6 : 0;
  f[o + 0] = b.lo[0];
  f[o + 1] = b.lo[1];
  f[o + 2] = b.lo[2];
  f[o + 3] = b.hi[0];
  f[o + 4] = b.hi[1];
  f[o + 5] = b.hi[2];
}

__device__ __forceinline__ Box load_union(const Node* nodes, int p) {
  const volatile float* f = reinterpret_cast<const volatile float*>(&nodes[p]);
  Box b;
  for (int c = 0; c < 3; ++c) {
    b.lo[c] = fminf(f[c], f[6 + c]);
    b.hi[c] = fmaxf(f[3 + c], f[9 + c]);
  }
  return b;
}

// unit area-weighted normal of vertex v (incident faces in ascending order, float32
// decision arithmetic) and its length, into normals[v] and normal_len[v]
__device__ __forceinline__ void vertex_normal(int v, const float* __restrict__ verts, const int* __restrict__ faces,
                                              const int* __restrict__ vf_off, const int* __restrict__ vf_faces,
                                              int V, int F, float* __restrict__ normals,
                                              float* __restrict__ normal_len, int* status) {
  float3 m = make_float3(0.0f, 0.0f, 0.0f);
  int k0 = vf_off[v], k1 = vf_off[v + 1];
  if (k0 < 0 || k1 < k0 || k1 > 3 * F) {
    set_status(status, kStatusBadModel);
    k1 = k0;
  }
  for (int k = k0; k < k1; ++k) {
    int f = vf_faces[k];
    if (f < 0 || f >= F) {
      set_status(status, kStatusBadModel);
      continue;
    }
    const int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    if (i0 < 0 || i0 >= V || i1 < 0 || i1 >= V || i2 < 0 || i2 >= V) {
      set_status(status, kStatusBadModel);
      continue;
    }
    float3 a = ld3(verts + 3 * i0), b = ld3(verts + 3 * i1), c = ld3(verts + 3 * i2);
    float3 cf = dcross(dsub(b, a), dsub(c, a));
    m = make_float3(__fadd_rn(m.x, cf.x), __fadd_rn(m.y, cf.y), __fadd_rn(m.z, cf.z));
  }
  float len = __fsqrt_rn(ddot(m, m));
  float3 n = len > 0.0f ? make_float3(__fdiv_rn(m.x, len), __fdiv_rn(m.y, len), __fdiv_rn(m.z, len))
                        : make_float3(0.0f, 0.0f, 0.0f);
  normals[3 * v] = n.x;
  normals[3 * v + 1] = n.y;
  normals[3 * v + 2] = n.z;
  normal_len[v] = len;
}

// shared memory: keys [P] u64, parent [2F] int, visit flags [F] int, then (when
// `snodes`) the max(F - 1, 1) nodes.  One block per instance: blockIdx.x selects the instance's
// vertices ([V][3] at blockIdx.x * 3V), nodes ([node_stride] per instance) and
// triangle records ([3 node_stride] float4 per instance).
__global__ void __launch_bounds__(kBuildThreads) k_build_bvh(const float* __restrict__ verts_all,
                                                             const int* __restrict__ faces, int F, int V, int P,
                                                             int node_stride, bool snodes,
                                                             Node* __restrict__ nodes_all,
                                                             float4* __restrict__ tris_all,
                                                             int* __restrict__ parent_all, int* __restrict__ valid,
                                                             const uint32_t* iter_dev, int rebuild_every,
                                                             int* status, const int* __restrict__ active,
                                                             const int* __restrict__ vf_off,
                                                             const int* __restrict__ vf_faces,
                                                             float* __restrict__ normals_all,
                                                             float* __restrict__ normal_len_all, int mode,
                                                             int* __restrict__ stale_all, int* __restrict__ need_all,
                                                             int force) {
  extern __shared__ unsigned long long smem_keys[];
  if (active && !active[blockIdx.x]) return;   // a retired instance of a batch
  unsigned long long* keys = smem_keys;
  int* parent = reinterpret_cast<int*>(keys + P);
  int* flags = parent + 2 * F;
  const float* verts = verts_all ? verts_all + (size_t)blockIdx.x * 3 * V : nullptr;   // null: a lazy refit
  Node* gnodes = nodes_all + (size_t)blockIdx.x * node_stride;
  float4* tris = tris_all + (size_t)blockIdx.x * 3 * node_stride;
  // the node array the hierarchy and refit work on (16-byte aligned after flags)
  Node* nodes = gnodes;
  if (snodes)
    nodes = reinterpret_cast<Node*>(reinterpret_cast<char*>(smem_keys) +
                                    (((size_t)P * 8 + (size_t)3 * F * 4 + 15) & ~(size_t)15));
  __shared__ float red[6][32];
  __shared__ float bounds[6];

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  int* gparent = parent_all + (size_t)blockIdx.x * 2 * node_stride;
  // refit when a tree of these faces exists and this is not a rebuild iteration
  bool refit = rebuild_every > 1 && iter_dev && valid[blockIdx.x] == 1 && (*iter_dev % rebuild_every) != 0;
  if (mode == kBvhLazyRefit) {
    // a render call: refit the stale boxes of an existing tree when a traversal will
    // read them (a sub-tile of this forward without a candidate list, or `force`)
    __shared__ int go;
    if (tid == 0) {
      go = valid[blockIdx.x] == 1 && stale_all[blockIdx.x] && (force || need_all[blockIdx.x]);
      need_all[blockIdx.x] = 0;
    }
    __syncthreads();
    if (!go) return;
    refit = true;
  }
  // hr_update_bvh's refit iterations: the triangle records only, the boxes left stale
  const bool records_only = mode == kBvhRecords && refit;
  if (refit && !records_only) {
    const int nn = F > 1 ? F - 1 : 1;
    if (snodes)   // the refit rewrites every box: only the child indices are read
      for (int i = tid; i < nn; i += blockDim.x) nodes[i].d = gnodes[i].d;
    for (int i = tid; i < 2 * F; i += blockDim.x) parent[i] = gparent[i];
    for (int i = tid; i < F; i += blockDim.x) flags[i] = 0;
    __syncthreads();
  }
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  if (!refit) {   // block-uniform: phases 0-4 of a full build
    // 0. face indices must address [0, V); otherwise record the error and build nothing
    for (int i = tid; i < 3 * F; i += blockDim.x)
      if (faces[i] < 0 || faces[i] >= V) bad = 1;
    __syncthreads();
    if (bad) {
      if (tid == 0) {
        set_status(status, kStatusBadModel);
        gnodes[0].d = make_int4(~0, ~0, 0, 0);   // a one-leaf tree over a degenerate record
        gnodes[0].a = make_float4(1.0f, 1.0f, 1.0f, -1.0f);
        gnodes[0].b = make_float4(-1.0f, -1.0f, 1.0f, 1.0f);
        gnodes[0].c = make_float4(1.0f, -1.0f, -1.0f, -1.0f);
        tris[0] = tris[1] = tris[2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
      return;
    }

    // 1. centroid bounds
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int f = tid; f < F; f += blockDim.x) {
      int3 fc = make_int3(faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]);
      for (int c = 0; c < 3; ++c) {
        float x = (verts[3 * fc.x + c] + verts[3 * fc.y + c] + verts[3 * fc.z + c]) * (1.0f / 3.0f);
        lo[c] = fminf(lo[c], x);
        hi[c] = fmaxf(hi[c], x);
      }
    }
    for (int c = 0; c < 3; ++c) {
      float a = warp_min(lo[c]), b = warp_max(hi[c]);
      if (lane == 0) {
        red[c][warp] = a;
        red[3 + c][warp] = b;
      }
    }
    __syncthreads();
    if (warp == 0) {
      int nw = blockDim.x >> 5;
      for (int c = 0; c < 3; ++c) {
        float a = lane < nw ? red[c][lane] : INFINITY;
        float b = lane < nw ? red[3 + c][lane] : -INFINITY;
        a = warp_min(a);
        b = warp_max(b);
        if (lane == 0) {
          bounds[c] = a;
          bounds[3 + c] = b;
        }
      }
    }
    __syncthreads();

    // 2. Morton keys (code << 32 | triangle id), padded to P with all-ones
    for (int i = tid; i < P; i += blockDim.x) {
      unsigned long long key = ~0ull;
      if (i < F) {
        int3 fc = make_int3(faces[3 * i], faces[3 * i + 1], faces[3 * i + 2]);
        unsigned q[3];
        for (int c = 0; c < 3; ++c) {
          float x = (verts[3 * fc.x + c] + verts[3 * fc.y + c] + verts[3 * fc.z + c]) * (1.0f / 3.0f);
          float ext = bounds[3 + c] - bounds[c];
          float n = ext > 0.0f ? (x - bounds[c]) / ext : 0.5f;
          q[c] = (unsigned)fminf(fmaxf(n * 1024.0f, 0.0f), 1023.0f);
        }
        unsigned code = (expand_bits10(q[0]) << 2) | (expand_bits10(q[1]) << 1) | expand_bits10(q[2]);
        key = ((unsigned long long)code << 32) | (unsigned)i;
      }
      keys[i] = key;
    }
    for (int i = tid; i < F; i += blockDim.x) flags[i] = 0;
    __syncthreads();

    // 3. bitonic sort (ascending)
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < P; i += blockDim.x) {
          int ixj = i ^ j;
          if (ixj > i) {
            unsigned long long a = keys[i], b = keys[ixj];
            bool up = (i & k) == 0;
            if ((a > b) == up) {
              keys[i] = b;
              keys[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }

    // 4. hierarchy (internal nodes 0..F-2; leaves encoded ~k, k = sorted position)
    if (F == 1) {
      if (tid == 0) {
        nodes[0].d = make_int4(~0, ~0, 0, 0);
        parent[0] = -1;
        parent[F + 0] = 0;
      }
    }
    for (int i = tid; i < F - 1; i += blockDim.x) karras_node(keys, F, i, nodes, parent);
    __syncthreads();

  }
  // 5. triangle records and leaf boxes, then the bottom-up refit (a refit reads the
  // leaf order from the previous records).  A thread's leaves (two at F <= 2048) load
  // their triangles together before either walks up the tree.
  constexpr int kLeafPer = 2;
  for (int k0 = tid; k0 < F; k0 += kLeafPer * blockDim.x) {
    int tri[kLeafPer];
    float3 v0[kLeafPer], v1[kLeafPer], v2[kLeafPer];
#pragma unroll
    for (int j = 0; j < kLeafPer; ++j) {
      const int k = k0 + j * blockDim.x;
      tri[j] = -1;
      if (k >= F) continue;
      tri[j] = refit ? __float_as_int(tris[3 * k + 2].y) : (int)(keys[k] & 0xffffffffull);
    }
#pragma unroll
    for (int j = 0; j < kLeafPer; ++j) {
      const int k = k0 + j * blockDim.x;
      if (k >= F) continue;
      if (tri[j] < 0 || tri[j] >= F) {   // a corrupt record: skip it (reported)
        set_status(status, kStatusIndex);
        tri[j] = -1;
        continue;
      }
      if (mode == kBvhLazyRefit) {   // the triangle as the records give it to the intersector
        const float4 ta = tris[3 * k], tb = tris[3 * k + 1], tc = tris[3 * k + 2];
        v0[j] = make_float3(ta.x, ta.y, ta.z);
        v1[j] = make_float3(ta.x + ta.w, ta.y + tb.x, ta.z + tb.y);
        v2[j] = make_float3(ta.x + tb.z, ta.y + tb.w, ta.z + tc.x);
      } else {
        v0[j] = ld3(verts + 3 * faces[3 * tri[j]]);
        v1[j] = ld3(verts + 3 * faces[3 * tri[j] + 1]);
        v2[j] = ld3(verts + 3 * faces[3 * tri[j] + 2]);
      }
    }
#pragma unroll 1
    for (int j = 0; j < kLeafPer; ++j) {
      const int k = k0 + j * blockDim.x;
      if (k >= F || tri[j] < 0) continue;
      if (mode != kBvhLazyRefit) {   // a lazy refit leaves the records (read by the render) alone
        float3 e1 = dsub(v1[j], v0[j]), e2 = dsub(v2[j], v0[j]);
        tris[3 * k + 0] = make_float4(v0[j].x, v0[j].y, v0[j].z, e1.x);
        tris[3 * k + 1] = make_float4(e1.y, e1.z, e2.x, e2.y);
        tris[3 * k + 2] = make_float4(e2.z, __int_as_float(tri[j]), 0.0f, 0.0f);
      }
      if (records_only) continue;
      Box b;
      float amax = 0.0f;
      float p0[3] = {v0[j].x, v0[j].y, v0[j].z}, p1[3] = {v1[j].x, v1[j].y, v1[j].z},
            p2[3] = {v2[j].x, v2[j].y, v2[j].z};
      for (int c = 0; c < 3; ++c) {
        b.lo[c] = fminf(p0[c], fminf(p1[c], p2[c]));
        b.hi[c] = fmaxf(p0[c], fmaxf(p1[c], p2[c]));
        amax = fmaxf(amax, fmaxf(fabsf(b.lo[c]), fabsf(b.hi[c])));
      }
      float pad = 1e-6f + 1e-5f * amax;
      for (int c = 0; c < 3; ++c) {
        b.lo[c] -= pad;
        b.hi[c] += pad;
      }
      int p = parent[F + k];
      int slot = (nodes[p].d.x == ~k) ? 0 : 1;
      if (F == 1) {
        store_slot(nodes, 0, 0, b);
        store_slot(nodes, 0, 1, b);
        continue;
      }
      store_slot(nodes, p, slot, b);
      __threadfence_block();
      for (int up = 0; up < F; ++up) {   // a well-formed tree is at most F - 1 levels deep
        if (atomicAdd(&flags[p], 1) == 0) break;   // the sibling is not done yet
        __threadfence_block();
        Box u = load_union(nodes, p);
        int gp = parent[p];
        if (gp < 0) break;                          // p is the root
        int gslot = (nodes[gp].d.x == p) ? 0 : 1;
        store_slot(nodes, gp, gslot, u);
        __threadfence_block();
        p = gp;
      }
    }
  }
  // 6. the shading normals of the same vertices (threads that finished their walks
  // first start on them)
  if (normals_all) {
    float* normals = normals_all + (size_t)blockIdx.x * 3 * V;
    float* normal_len = normal_len_all + (size_t)blockIdx.x * V;
    for (int v = tid; v < V; v += blockDim.x)
      vertex_normal(v, verts, faces, vf_off, vf_faces, V, F, normals, normal_len, status);
  }
  __syncthreads();
  if (records_only) {
    if (tid == 0) stale_all[blockIdx.x] = 1;
    return;
  }
  if (snodes) {   // a refit changed only the boxes (the first three float4 of a node)
    const int nn = F > 1 ? F - 1 : 1;
    const float4* src = reinterpret_cast<const float4*>(nodes);
    float4* dst = reinterpret_cast<float4*>(gnodes);
    if (refit) {
      for (int i = tid; i < 3 * nn; i += blockDim.x) dst[4 * (i / 3) + i % 3] = src[4 * (i / 3) + i % 3];
    } else {
      for (int i = tid; i < 4 * nn; i += blockDim.x) dst[i] = src[i];
    }
  }
  if (!refit) {   // keep the topology for later refits
    for (int i = tid; i < 2 * F; i += blockDim.x) gparent[i] = parent[i];
    if (tid == 0) valid[blockIdx.x] = 1;
  }
  if (tid == 0 && stale_all) stale_all[blockIdx.x] = 0;
}

// Faces and the vertex->face table come from the caller: an index out of range is
// reported in the status word and its face skipped.
// Batched: blockIdx.y selects the instance ([V][3] vertices and normals, [V] lengths).
__global__ void k_vertex_normals(const float* __restrict__ verts_all, const int* __restrict__ faces,
                                 const int* __restrict__ vf_off, const int* __restrict__ vf_faces, int V, int F,
                                 float* __restrict__ normals_all, float* __restrict__ normal_len_all, int* status,
                                 const int* __restrict__ active) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V || (active && !active[blockIdx.y])) return;
  vertex_normal(v, verts_all + (size_t)blockIdx.y * 3 * V, faces, vf_off, vf_faces, V, F,
                normals_all + (size_t)blockIdx.y * 3 * V, normal_len_all + (size_t)blockIdx.y * V, status);
}


// ---------------------------------------------------------------------------------
// Multi-block build for meshes whose keys do not fit one block's shared memory
// (F above ~2400 with the nodes, ~25k without): the same Morton codes, hierarchy and
// refit over global memory, one instance per grid row, the keys sorted by a bitonic
// network whose stages below 2048 run in shared memory.
// ---------------------------------------------------------------------------------
constexpr int kSortChunk = 2048;    // keys sorted per block in shared memory
constexpr int kGridThreads = 256;

// float <-> order-preserving unsigned (for atomicMin / atomicMax of floats)
__device__ __forceinline__ unsigned f2o(float f) {
  unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// per instance: refit (mode 1) or full build (mode 0), decided once per call before
// the other kernels read it; a full build marks the tree valid for later refits
// (a build over bad faces clears that again) and resets the bounds and the bad flag
__global__ void k_lb_decide(int* __restrict__ mode, int* __restrict__ valid, unsigned* __restrict__ bounds_all,
                            int* __restrict__ bad_all, const uint32_t* iter_dev, int rebuild_every) {
  const int inst = blockIdx.x;
  const bool refit = rebuild_every > 1 && iter_dev && valid[inst] == 1 && (*iter_dev % rebuild_every) != 0;
  mode[inst] = refit ? 1 : 0;
  if (refit) return;
  valid[inst] = 1;
  bad_all[inst] = 0;
  for (int c = 0; c < 3; ++c) {
    bounds_all[inst * 6 + c] = 0xFFFFFFFFu;
    bounds_all[inst * 6 + 3 + c] = 0u;
  }
}

// centroid bounds (ordered unsigned, [n][6]: min xyz, max xyz) and face validation
__global__ void k_lb_bounds(const float* __restrict__ verts_all, const int* __restrict__ faces, int F, int V,
                            unsigned* __restrict__ bounds_all, int* __restrict__ bad_all, const int* mode,
                            int* status) {
  if (mode[blockIdx.y]) return;
  const float* verts = verts_all + (size_t)blockIdx.y * 3 * V;
  unsigned* bounds = bounds_all + blockIdx.y * 6;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
    const int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    if (i0 < 0 || i0 >= V || i1 < 0 || i1 >= V || i2 < 0 || i2 >= V) {
      set_status(status, kStatusBadModel);
      bad_all[blockIdx.y] = 1;
      continue;
    }
    for (int c = 0; c < 3; ++c) {
      const float x = (verts[3 * i0 + c] + verts[3 * i1 + c] + verts[3 * i2 + c]) * (1.0f / 3.0f);
      lo[c] = fminf(lo[c], x);
      hi[c] = fmaxf(hi[c], x);
    }
  }
  for (int c = 0; c < 3; ++c) {
    const float a = warp_min(lo[c]), b = warp_max(hi[c]);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&bounds[c], f2o(a));
      atomicMax(&bounds[3 + c], f2o(b));
    }
  }
}

// keys[i] = morton << 32 | i for i < F, all ones up to P
__global__ void k_lb_morton(const float* __restrict__ verts_all, const int* __restrict__ faces, int F, int V, int P,
                            const unsigned* __restrict__ bounds_all, const int* __restrict__ bad_all,
                            unsigned long long* __restrict__ keys_all, const int* mode) {
  if (mode[blockIdx.y]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  unsigned long long* keys = keys_all + (size_t)blockIdx.y * P;
  unsigned long long key = ~0ull;
  if (i < F && !bad_all[blockIdx.y]) {
    const float* verts = verts_all + (size_t)blockIdx.y * 3 * V;
    const unsigned* bo = bounds_all + blockIdx.y * 6;
    const int i0 = faces[3 * i], i1 = faces[3 * i + 1], i2 = faces[3 * i + 2];
    unsigned q[3];
    for (int c = 0; c < 3; ++c) {
      const float x = (verts[3 * i0 + c] + verts[3 * i1 + c] + verts[3 * i2 + c]) * (1.0f / 3.0f);
      const float l = o2f(bo[c]), ext = o2f(bo[3 + c]) - l;
      const float nrm = ext > 0.0f ? (x - l) / ext : 0.5f;
      q[c] = (unsigned)fminf(fmaxf(nrm * 1024.0f, 0.0f), 1023.0f);
    }
    const unsigned code = (expand_bits10(q[0]) << 2) | (expand_bits10(q[1]) << 1) | expand_bits10(q[2]);
    key = ((unsigned long long)code << 32) | (unsigned)i;
  }
  keys[i] = key;
}

// bitonic stages (k, j) with j < kSortChunk of one 2048-key chunk, in shared memory;
// first = true runs every stage k = 2 .. kSortChunk, otherwise the j-stages of one k
__global__ void __launch_bounds__(1024) k_lb_sort_local(unsigned long long* __restrict__ keys_all, int P, int k_outer,
                                                        bool first, const int* mode) {
  if (mode[blockIdx.y]) return;
  __shared__ unsigned long long sk[kSortChunk];
  unsigned long long* keys = keys_all + (size_t)blockIdx.y * P;
  const int base = blockIdx.x * kSortChunk;
  for (int t = threadIdx.x; t < kSortChunk; t += blockDim.x) sk[t] = keys[base + t];
  __syncthreads();
  const int k_lo = first ? 2 : k_outer, k_hi = first ? kSortChunk : k_outer;
  for (int k = k_lo; k <= k_hi; k <<= 1) {
    for (int j = min(k, kSortChunk) >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < kSortChunk; t += blockDim.x) {
        const int l = t ^ j;
        if (l > t) {
          const bool up = ((base + t) & k) == 0;
          const unsigned long long x = sk[t], y = sk[l];
          if ((x > y) == up) {
            sk[t] = y;
            sk[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < kSortChunk; t += blockDim.x) keys[base + t] = sk[t];
}

// one bitonic stage (k, j) with j >= kSortChunk over global memory
__global__ void k_lb_sort_global(unsigned long long* __restrict__ keys_all, int P, int k, int j, const int* mode) {
  if (mode[blockIdx.y]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int l = t ^ j;
  if (l <= t) return;
  unsigned long long* keys = keys_all + (size_t)blockIdx.y * P;
  const bool up = (t & k) == 0;
  const unsigned long long x = keys[t], y = keys[l];
  if ((x > y) == up) {
    keys[t] = y;
    keys[l] = x;
  }
}

// Karras hierarchy over the sorted keys (internal nodes 0..F-2, leaves ~k)
__global__ void k_lb_hierarchy(const unsigned long long* __restrict__ keys_all, int F, int P, int node_stride,
                               Node* __restrict__ nodes_all, int* __restrict__ parent_all, const int* mode) {
  if (mode[blockIdx.y]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long* keys = keys_all + (size_t)blockIdx.y * P;
  Node* nodes = nodes_all + (size_t)blockIdx.y * node_stride;
  int* parent = parent_all + (size_t)blockIdx.y * 2 * node_stride;
  if (F == 1) {
    if (i == 0) {
      nodes[0].d = make_int4(~0, ~0, 0, 0);
      parent[0] = -1;
      parent[F] = 0;
    }
    return;
  }
  if (i >= F - 1) return;
  karras_node(keys, F, i, nodes, parent);
}

// triangle records and leaf boxes, then the bottom-up refit with global flags (zeroed
// before the launch); a refit takes the leaf order from the previous records
__global__ void k_lb_leaves(const float* __restrict__ verts_all, const int* __restrict__ faces, int F, int V,
                            int P, int node_stride, const unsigned long long* __restrict__ keys_all,
                            Node* __restrict__ nodes_all, float4* __restrict__ tris_all,
                            const int* __restrict__ parent_all, int* __restrict__ flags_all, int* __restrict__ valid,
                            const int* __restrict__ bad_all, const int* mode, int* status) {
  const bool refit = mode[blockIdx.y] == 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  Node* nodes = nodes_all + (size_t)blockIdx.y * node_stride;
  float4* tris = tris_all + (size_t)blockIdx.y * 3 * node_stride;
  if (!refit && bad_all[blockIdx.y]) {   // bad faces: the degenerate one-leaf tree
    if (k == 0) {
      nodes[0].d = make_int4(~0, ~0, 0, 0);
      nodes[0].a = make_float4(1.0f, 1.0f, 1.0f, -1.0f);
      nodes[0].b = make_float4(-1.0f, -1.0f, 1.0f, 1.0f);
      nodes[0].c = make_float4(1.0f, -1.0f, -1.0f, -1.0f);
      tris[0] = tris[1] = tris[2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      valid[blockIdx.y] = 0;
    }
    return;
  }
  if (k >= F) return;
  const float* verts = verts_all + (size_t)blockIdx.y * 3 * V;
  const int* parent = parent_all + (size_t)blockIdx.y * 2 * node_stride;
  int* flags = flags_all + (size_t)blockIdx.y * node_stride;
  const unsigned long long* keys = keys_all + (size_t)blockIdx.y * P;
  const int tri = refit ? __float_as_int(tris[3 * k + 2].y) : (int)(keys[k] & 0xffffffffull);
  if (tri < 0 || tri >= F) {
    set_status(status, kStatusIndex);
    return;
  }
  float3 v0 = ld3(verts + 3 * faces[3 * tri]);
  float3 v1 = ld3(verts + 3 * faces[3 * tri + 1]);
  float3 v2 = ld3(verts + 3 * faces[3 * tri + 2]);
  float3 e1 = dsub(v1, v0), e2 = dsub(v2, v0);
  tris[3 * k + 0] = make_float4(v0.x, v0.y, v0.z, e1.x);
  tris[3 * k + 1] = make_float4(e1.y, e1.z, e2.x, e2.y);
  tris[3 * k + 2] = make_float4(e2.z, __int_as_float(tri), 0.0f, 0.0f);
  Box b;
  float amax = 0.0f;
  float p0[3] = {v0.x, v0.y, v0.z}, p1[3] = {v1.x, v1.y, v1.z}, p2[3] = {v2.x, v2.y, v2.z};
  for (int c = 0; c < 3; ++c) {
    b.lo[c] = fminf(p0[c], fminf(p1[c], p2[c]));
    b.hi[c] = fmaxf(p0[c], fmaxf(p1[c], p2[c]));
    amax = fmaxf(amax, fmaxf(fabsf(b.lo[c]), fabsf(b.hi[c])));
  }
  const float pad = 1e-6f + 1e-5f * amax;
  for (int c = 0; c < 3; ++c) {
    b.lo[c] -= pad;
    b.hi[c] += pad;
  }
  if (F == 1) {
    store_slot(nodes, 0, 0, b);
    store_slot(nodes, 0, 1, b);
    return;
  }
  int p = parent[F + k];
  if (p < 0 || p >= F - 1) {
    set_status(status, kStatusIndex);
    return;
  }
  store_slot(nodes, p, (nodes[p].d.x == ~k) ? 0 : 1, b);
  __threadfence();
  for (int up = 0; up < F; ++up) {   // a well-formed tree is at most F - 1 levels deep
    if (atomicAdd(&flags[p], 1) == 0) break;
    __threadfence();
    Box u = load_union(nodes, p);
    const int gp = parent[p];
    if (gp < 0) break;
    if (gp >= F - 1) {
      set_status(status, kStatusIndex);
      break;
    }
    store_slot(nodes, gp, (nodes[gp].d.x == p) ? 0 : 1, u);
    __threadfence();
    p = gp;
  }
}

}  // namespace

int configure_bvh_kernels() {
  if (cudaFuncSetAttribute(k_build_bvh, cudaFuncAttributeMaxDynamicSharedMemorySize, kBuildSmemCap) !=
      cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  return HR_OK;
}

// the multi-block build (keys beyond one block's shared memory)
int launch_build_bvh_grid(Context* ctx, const hr_model* m, const float* verts, const uint32_t* iter_dev,
                          int rebuild_every, int P, cudaStream_t s) {
  const int F = m->F, V = m->V, ni = ctx->n_inst, ns = ctx->lim.max_F;
  if (P > ctx->bvh_pmax) return HR_ERR_UNSUPPORTED;
  if (ctx->bvh_faces != m->faces || ctx->F != F) {
    if (cudaMemsetAsync(ctx->bvh_valid, 0, sizeof(int) * ni, s) != cudaSuccess) return HR_ERR_CUDA;
    ctx->bvh_faces = m->faces;
  }
  ctx->bvh_lazy = false;   // the multi-block build refits its boxes every call
  k_lb_decide<<<ni, 1, 0, s>>>(ctx->bvh_mode, ctx->bvh_valid, ctx->bvh_bounds, ctx->bvh_bad, iter_dev,
                               rebuild_every);
  HR_CHECK_LAUNCH();
  const unsigned fb = (unsigned)((F + kGridThreads - 1) / kGridThreads);
  k_lb_bounds<<<dim3(fb < 64 ? fb : 64, ni), kGridThreads, 0, s>>>(verts, m->faces, F, V, ctx->bvh_bounds,
                                                                   ctx->bvh_bad, ctx->bvh_mode, ctx->status);
  HR_CHECK_LAUNCH();
  const dim3 gp((unsigned)((P + kGridThreads - 1) / kGridThreads), ni);
  k_lb_morton<<<gp, kGridThreads, 0, s>>>(verts, m->faces, F, V, P, ctx->bvh_bounds, ctx->bvh_bad, ctx->bvh_keys,
                                          ctx->bvh_mode);
  HR_CHECK_LAUNCH();
  const dim3 gc((unsigned)(P / kSortChunk), ni);
  k_lb_sort_local<<<gc, 1024, 0, s>>>(ctx->bvh_keys, P, 0, true, ctx->bvh_mode);
  HR_CHECK_LAUNCH();
  for (int k = 2 * kSortChunk; k <= P; k <<= 1) {
    for (int j = k >> 1; j >= kSortChunk; j >>= 1) {
      k_lb_sort_global<<<gp, kGridThreads, 0, s>>>(ctx->bvh_keys, P, k, j, ctx->bvh_mode);
      HR_CHECK_LAUNCH();
    }
    k_lb_sort_local<<<gc, 1024, 0, s>>>(ctx->bvh_keys, P, k, false, ctx->bvh_mode);
    HR_CHECK_LAUNCH();
  }
  k_lb_hierarchy<<<dim3(fb, ni), kGridThreads, 0, s>>>(ctx->bvh_keys, F, P, ns, ctx->nodes, ctx->bvh_parent,
                                                       ctx->bvh_mode);
  HR_CHECK_LAUNCH();
  if (cudaMemsetAsync(ctx->bvh_flags, 0, sizeof(int) * (size_t)ni * ns, s) != cudaSuccess) return HR_ERR_CUDA;
  k_lb_leaves<<<dim3(fb, ni), kGridThreads, 0, s>>>(verts, m->faces, F, V, P, ns, ctx->bvh_keys, ctx->nodes,
                                                    ctx->tris, ctx->bvh_parent, ctx->bvh_flags, ctx->bvh_valid,
                                                    ctx->bvh_bad, ctx->bvh_mode, ctx->status);
  HR_CHECK_LAUNCH();
  k_vertex_normals<<<dim3((V + 255) / 256, ni), 256, 0, s>>>(verts, m->faces, m->vf_offsets, m->vf_faces, V, F,
                                                             ctx->normals, ctx->normal_len, ctx->status, ctx->active);
  HR_CHECK_LAUNCH();
  ctx->V = V;
  ctx->F = F;
  ++ctx->bvh_gen;
  ctx->fwd_valid = false;
  return HR_OK;
}

// Refit the boxes of a one-block tree whose last update rewrote only the records,
// from the records themselves (the triangles the intersector tests), when this
// forward listed a sub-tile for per-ray traversal (k_bin_alloc sets bvh_need) or
// `force`; otherwise the kernel returns at once.
int launch_bvh_lazy_refit(Context* ctx, int force, cudaStream_t s) {
  if (!ctx->bvh_lazy) return HR_OK;
  k_build_bvh<<<ctx->n_inst, kBuildThreads, ctx->bvh_smem, s>>>(
      nullptr, ctx->bvh_faces, ctx->F, ctx->V, ctx->bvh_P, ctx->lim.max_F, ctx->bvh_snodes, ctx->nodes, ctx->tris,
      ctx->bvh_parent, ctx->bvh_valid, nullptr, 1, ctx->status, ctx->active, nullptr, nullptr, nullptr, nullptr,
      kBvhLazyRefit, ctx->bvh_stale, ctx->bvh_need, force);
  HR_CHECK_LAUNCH();
  return HR_OK;
}

int launch_build_bvh(Context* ctx, const hr_model* m, const float* verts, cudaStream_t s) {
  return launch_update_bvh(ctx, m, verts, nullptr, 1, s);
}

int launch_update_bvh(Context* ctx, const hr_model* m, const float* verts, const uint32_t* iter_dev,
                      int rebuild_every, cudaStream_t s) {
  int F = m->F, V = m->V;
  int P = 1;
  while (P < F) P <<= 1;
  size_t smem = (size_t)P * 8 + (size_t)3 * F * 4;
  if (smem > (size_t)kBuildSmemCap) return launch_build_bvh_grid(ctx, m, verts, iter_dev, rebuild_every, P, s);
  const size_t with_nodes = ((smem + 15) & ~(size_t)15) + (size_t)(F > 1 ? F - 1 : 1) * sizeof(Node);
  const bool snodes = with_nodes <= (size_t)kBuildSmemCap;
  if (snodes) smem = with_nodes;
  // a refit needs a tree built over these faces by this context
  if (ctx->bvh_faces != m->faces || ctx->F != F) {
    if (cudaMemsetAsync(ctx->bvh_valid, 0, sizeof(int) * ctx->n_inst, s) != cudaSuccess) return HR_ERR_CUDA;
    ctx->bvh_faces = m->faces;
  }
  // the vertex normals need only the vertices: they are computed on the context's side
  // stream beside the build (one block per instance), joined before the call returns
  // (in a captured graph, two parallel branches)
  if (cudaEventRecord(ctx->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0) != cudaSuccess)
    return HR_ERR_CUDA;
  k_vertex_normals<<<dim3((V + 255) / 256, ctx->n_inst), 256, 0, ctx->side>>>(
      verts, m->faces, m->vf_offsets, m->vf_faces, V, F, ctx->normals, ctx->normal_len, ctx->status, ctx->active);
  HR_CHECK_LAUNCH();
  // with a rebuild schedule, refit iterations rewrite only the records; the render
  // calls refit the boxes when they need them (launch_bvh_lazy_refit)
  const int mode = (rebuild_every > 1 && iter_dev) ? kBvhRecords : kBvhFull;
  k_build_bvh<<<ctx->n_inst, kBuildThreads, smem, s>>>(verts, m->faces, F, V, P, ctx->lim.max_F, snodes,
                                                       ctx->nodes, ctx->tris, ctx->bvh_parent, ctx->bvh_valid,
                                                       iter_dev, rebuild_every, ctx->status, ctx->active,
                                                       nullptr, nullptr, nullptr, nullptr, mode, ctx->bvh_stale,
                                                       ctx->bvh_need, 0);
  HR_CHECK_LAUNCH();
  ctx->bvh_lazy = true;
  ctx->bvh_P = P;
  ctx->bvh_smem = smem;
  ctx->bvh_snodes = snodes;
  if (cudaEventRecord(ctx->ev_join, ctx->side) != cudaSuccess || cudaStreamWaitEvent(s, ctx->ev_join, 0) != cudaSuccess)
    return HR_ERR_CUDA;
  ctx->V = V;
  ctx->F = F;
  ++ctx->bvh_gen;
  ctx->fwd_valid = false;
  return HR_OK;
}

}  // namespace hr
