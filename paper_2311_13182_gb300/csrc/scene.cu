// Mesh packing and LBVH construction.
//
// The triangle mesh is the scene representation whose vertex positions are the
// optimised parameters (Section 3.1).  The paper gives no acceleration
// structure; this builds a linear BVH: Morton codes of triangle centroids
// (30 bits), a stable radix sort (ties keep the triangle order), the binary
// radix tree of Karras (2012, "Maximizing parallelism in the construction of
// BVHs, octrees, and k-d trees") and a bottom-up AABB refit driven by atomic
// arrival counters (the second child to arrive builds the parent; nothing waits).
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <cmath>

#include <cuda/atomic>

#include "scene.cuh"

namespace sbr {
namespace {

__device__ inline int32_t ord(float f) {
  int32_t i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ inline float unord(int32_t i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_init_bounds(int32_t* b, int32_t* err, uint32_t* hist) {
  if (threadIdx.x < 3) b[threadIdx.x] = 0x7fffffff;           // min x, y, z
  else if (threadIdx.x < 6) b[threadIdx.x] = (int32_t)0x80000000;  // max x, y, z
  else if (threadIdx.x == 6) b[6] = 0;                        // max |coord| (ordered, >= 0)
  else if (threadIdx.x == 7) b[7] = 0;
  if (threadIdx.x == 0) *err = 0;
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) hist[i] = 0u;
}

__device__ inline int face_vert(const int32_t* faces, int f, int c, int nv, int32_t* err) {
  int i = faces[3 * f + c];
  if (i < 0 || i >= nv) {
    atomicOr(err, 1);
    return 0;
  }
  return i;
}

__device__ inline float3 vload(const float* v, int i) { return f3(v[3 * i], v[3 * i + 1], v[3 * i + 2]); }

__global__ void k_bounds(const float* __restrict__ verts, int nv, const int32_t* __restrict__ faces,
                         int nt, int32_t* bounds, int32_t* err) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  float3 lo = f3(INFINITY, INFINITY, INFINITY), hi = f3(-INFINITY, -INFINITY, -INFINITY);
  float mabs = 0.f;
  if (f < nt) {
    float3 a = vload(verts, face_vert(faces, f, 0, nv, err));
    float3 b = vload(verts, face_vert(faces, f, 1, nv, err));
    float3 c = vload(verts, face_vert(faces, f, 2, nv, err));
    float3 m = (a + b + c) * (1.f / 3.f);
    lo = m;
    hi = m;
    mabs = fmaxf(fmaxf(l1(a), l1(b)), l1(c));
  }
  // warp reduce then one atomic per warp
  for (int o = 16; o; o >>= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(~0u, lo.x, o));
    lo.y = fminf(lo.y, __shfl_xor_sync(~0u, lo.y, o));
    lo.z = fminf(lo.z, __shfl_xor_sync(~0u, lo.z, o));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(~0u, hi.x, o));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(~0u, hi.y, o));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(~0u, hi.z, o));
    mabs = fmaxf(mabs, __shfl_xor_sync(~0u, mabs, o));
  }
  if ((threadIdx.x & 31) == 0 && lo.x <= hi.x) {
    atomicMin(&bounds[0], ord(lo.x));
    atomicMin(&bounds[1], ord(lo.y));
    atomicMin(&bounds[2], ord(lo.z));
    atomicMax(&bounds[3], ord(hi.x));
    atomicMax(&bounds[4], ord(hi.y));
    atomicMax(&bounds[5], ord(hi.z));
    atomicMax(&bounds[6], ord(mabs));
  }
}

__device__ inline uint32_t spread10(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

// 30-bit Morton code of the centroid in the centroid box (bounds, ordered ints).
// Triangles spanning more than 1/32 of that box (a ground plane under an object)
// get key bit 30, so the radix tree puts them in their own subtree at the root
// instead of inflating the boxes of their Morton neighbours.
__device__ inline uint32_t morton_key(float3 a, float3 b, float3 c, const int32_t* bounds) {
  const float3 m = (a + b + c) * (1.f / 3.f);
  const float3 lo = f3(unord(__ldcg(&bounds[0])), unord(__ldcg(&bounds[1])), unord(__ldcg(&bounds[2])));
  const float3 hi = f3(unord(__ldcg(&bounds[3])), unord(__ldcg(&bounds[4])), unord(__ldcg(&bounds[5])));
  const float3 ext = hi - lo;
  const float qx = ext.x > 0.f ? (m.x - lo.x) / ext.x : 0.f;
  const float qy = ext.y > 0.f ? (m.y - lo.y) / ext.y : 0.f;
  const float qz = ext.z > 0.f ? (m.z - lo.z) / ext.z : 0.f;
  const uint32_t ix = (uint32_t)fminf(fmaxf(qx * 1024.f, 0.f), 1023.f);
  const uint32_t iy = (uint32_t)fminf(fmaxf(qy * 1024.f, 0.f), 1023.f);
  const uint32_t iz = (uint32_t)fminf(fmaxf(qz * 1024.f, 0.f), 1023.f);
  const float side = fmaxf(fmaxf(fmaxf(fabsf(a.x - b.x), fabsf(b.x - c.x)), fabsf(c.x - a.x)),
                           fmaxf(fmaxf(fmaxf(fabsf(a.y - b.y), fabsf(b.y - c.y)), fabsf(c.y - a.y)),
                                 fmaxf(fmaxf(fabsf(a.z - b.z), fabsf(b.z - c.z)), fabsf(c.z - a.z))));
  const float extent = fmaxf(fmaxf(ext.x, ext.y), ext.z);
  const uint32_t big = (extent > 0.f && side * 32.f > extent) ? (1u << 30) : 0u;
  return big | (spread10(ix) << 2) | (spread10(iy) << 1) | spread10(iz);
}

// Morton keys, and the counts of their four 8-bit digit places for the sort.
__global__ void __launch_bounds__(256) k_morton(const float* __restrict__ verts, int nv,
                                                const int32_t* __restrict__ faces, int nt,
                                                const int32_t* __restrict__ bounds, uint32_t* keys,
                                                int32_t* vals, uint32_t* hist, int32_t* err) {
  __shared__ uint32_t h[4 * 256];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = f < nt;
  uint32_t key = 0u;
  if (ok) {
    const float3 a = vload(verts, face_vert(faces, f, 0, nv, err));
    const float3 b = vload(verts, face_vert(faces, f, 1, nv, err));
    const float3 c = vload(verts, face_vert(faces, f, 2, nv, err));
    key = morton_key(a, b, c, bounds);
    keys[f] = key;
    vals[f] = f;
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < 4; ++p) {  // warp-aggregated counts
    const uint32_t d = (key >> (8 * p)) & 255u;
    const uint32_t peers = warp_peers8(d, ok);
    if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[256 * p + d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void k_pack(const float* __restrict__ verts, int nv, const int32_t* __restrict__ faces,
                       int nt, const int32_t* __restrict__ order, float4* __restrict__ tris,
                       int32_t* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  int f = order[i];
  float3 a = vload(verts, face_vert(faces, f, 0, nv, err));
  float3 b = vload(verts, face_vert(faces, f, 1, nv, err));
  float3 c = vload(verts, face_vert(faces, f, 2, nv, err));
  tris[3 * i + 0] = make_float4(a.x, a.y, a.z, __int_as_float(f));
  tris[3 * i + 1] = make_float4(b.x, b.y, b.z, 0.f);
  tris[3 * i + 2] = make_float4(c.x, c.y, c.z, 0.f);
}

// Length of the common prefix of sorted keys i and j (index bits break ties);
// key(j) reads sorted key j.
template <class KeyAt>
__device__ inline int prefix(const KeyAt& key, uint32_t ki, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t b = key(j);
  if (ki != b) return __clz(ki ^ b);
  return 32 + __clz((uint32_t)(i ^ j));
}

// Children and leaf range [lo, hi] of internal node i of the radix tree.
template <class KeyAt>
__device__ inline void karras_node(const KeyAt& key, int n, int i, int* left, int* right, int* lo, int* hi) {
  const uint32_t ki = key(i);
  // direction of the range covered by node i
  int d = (prefix(key, ki, n, i, i + 1) - prefix(key, ki, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = prefix(key, ki, n, i, i - d);
  int lmax = 2;
  while (prefix(key, ki, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (prefix(key, ki, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = prefix(key, ki, n, i, j);
  // split: last index sharing more than dnode bits with i
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (prefix(key, ki, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int g = i + s * d + (d < 0 ? -1 : 0);
  *lo = min(i, j);
  *hi = max(i, j);
  *left = (*lo == g) ? ~g : g;
  *right = (*hi == g + 1) ? ~(g + 1) : g + 1;
}

__global__ void k_karras(const uint32_t* __restrict__ keys, int n, Node* nodes, int32_t* parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int left, right, lo, hi;
  karras_node([&](int j) { return __ldg(&keys[j]); }, n, i, &left, &right, &lo, &hi);
  nodes[i].child = make_int4(left, right, 0, 0);
  parent[left >= 0 ? left : (n - 1 + ~left)] = i;
  parent[right >= 0 ? right : (n - 1 + ~right)] = i;
  if (i == 0) parent[0] = -1;
}

struct Box {
  float3 lo, hi;
};

__device__ inline Box tri_box(const float4* __restrict__ tris, int slot, float pad) {
  float4 a = tris[3 * slot], b = tris[3 * slot + 1], c = tris[3 * slot + 2];
  Box r;
  r.lo = f3(fminf(fminf(a.x, b.x), c.x) - pad, fminf(fminf(a.y, b.y), c.y) - pad,
            fminf(fminf(a.z, b.z), c.z) - pad);
  r.hi = f3(fmaxf(fmaxf(a.x, b.x), c.x) + pad, fmaxf(fmaxf(a.y, b.y), c.y) + pad,
            fmaxf(fmaxf(a.z, b.z), c.z) + pad);
  return r;
}

__device__ inline Box node_box(const Node* nodes, int i) {
  float4 a = __ldcg(&nodes[i].lxy), b = __ldcg(&nodes[i].rxy), c = __ldcg(&nodes[i].lrz);
  Box r;
  r.lo = f3(fminf(a.x, b.x), fminf(a.z, b.z), fminf(c.x, c.z));
  r.hi = f3(fmaxf(a.y, b.y), fmaxf(a.w, b.w), fmaxf(c.y, c.w));
  return r;
}

__global__ void k_refit(const float4* __restrict__ tris, int n, Node* nodes,
                        const int32_t* __restrict__ parent, uint32_t* visits,
                        const int32_t* __restrict__ bounds) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  // conservative pad: covers the FP32 ray's deviation from its FP64 source and
  // slab-test rounding for rays within the scene's coordinate range
  const float pad = ldexpf(1.f + unord(bounds[6]), -18);
  int node = parent[n - 1 + l];
  for (int depth = 0; node >= 0 && depth < 128; ++depth) {  // tree depth <= 62 (30 + 32 key bits)
    // acquire-release counter: the first arrival's child boxes (written before its
    // own increment) are visible to the second, which builds this node
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> arrivals(visits[node]);
    if (arrivals.fetch_add(1u, cuda::memory_order_acq_rel) == 0u) return;  // sibling subtree not done yet
    int4 ch = __ldcg(&nodes[node].child);
    Box bl = ch.x < 0 ? tri_box(tris, ~ch.x, pad) : node_box(nodes, ch.x);
    Box br = ch.y < 0 ? tri_box(tris, ~ch.y, pad) : node_box(nodes, ch.y);
    __stcg(&nodes[node].lxy, make_float4(bl.lo.x, bl.hi.x, bl.lo.y, bl.hi.y));
    __stcg(&nodes[node].rxy, make_float4(br.lo.x, br.hi.x, br.lo.y, br.hi.y));
    __stcg(&nodes[node].lrz, make_float4(bl.lo.z, bl.hi.z, br.lo.z, br.hi.z));
    node = parent[node];
  }
}

// ---- fused build for meshes of up to kTiledMax triangles ---------------------
//
// Every internal node's index lies inside its leaf range [lo, hi] (a property of
// the Karras tree), so with leaves and node indices cut into tiles of kBuildTile
// a node whose range stays inside one tile ("local") has its whole subtree in
// that tile.  The tree phase of k_build_scene runs one CTA per tile: it packs
// the tile's triangles in sorted order, computes the tile's tree nodes and
// refits the local ones with shared-memory arrival counters.  The last CTA to
// finish then refits the rest ("crossing" nodes, whose range spans a tile
// boundary).  Crossing nodes all contain the two leaves on either side of some
// boundary, so they are the ancestors of at most tiles-1 lowest common
// ancestors: at most 64 per boundary, as the tree depth is bounded by the 63
// prefix bits of key and index.

constexpr int kBuildTile = 1024;
constexpr int kTiledMax = 65536;
// Sorted keys staged in shared memory for the tree searches: all of them up to
// kKeyWindow, else a window around the tile (a local node's searches stay
// within twice its range of it; the rest read global memory).  Sized so the
// window, the tile's leaf boxes and k_build_scene's static arrays fit the
// 227 KB of a CTA.
constexpr int kKeyWindow = 38912;

// exclusive scan of one value per thread over a CTA of whole warps
__device__ inline uint32_t block_exclusive_u32(uint32_t v, uint32_t* total, uint32_t* warp_tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t q = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, q, o);
      if (lane >= o) q += y;
    }
    if (lane < nw) warp_tot[lane] = q;
  }
  __syncthreads();
  const uint32_t r = (w ? warp_tot[w - 1] : 0u) + x - v;
  *total = warp_tot[nw - 1];
  __syncthreads();
  return r;
}

struct SBox {
  float lx, ly, lz, hx, hy, hz;
};
__device__ inline SBox sbox(const Box& b) { return SBox{b.lo.x, b.lo.y, b.lo.z, b.hi.x, b.hi.y, b.hi.z}; }
__device__ inline Box unsbox(const SBox& b) {
  Box r;
  r.lo = f3(b.lx, b.ly, b.lz);
  r.hi = f3(b.hx, b.hy, b.hz);
  return r;
}
__device__ inline Box box_union(const Box& a, const Box& b) {
  Box r;
  r.lo = f3(fminf(a.lo.x, b.lo.x), fminf(a.lo.y, b.lo.y), fminf(a.lo.z, b.lo.z));
  r.hi = f3(fmaxf(a.hi.x, b.hi.x), fmaxf(a.hi.y, b.hi.y), fmaxf(a.hi.z, b.hi.z));
  return r;
}
__device__ inline void write_node(Node* nodes, int i, const Box& l, const Box& r) {
  nodes[i].lxy = make_float4(l.lo.x, l.hi.x, l.lo.y, l.hi.y);
  nodes[i].rxy = make_float4(r.lo.x, r.hi.x, r.lo.y, r.hi.y);
  nodes[i].lrz = make_float4(l.lo.z, l.hi.z, r.lo.z, r.hi.z);
}
// conservative pad: covers the FP32 ray's deviation from its exact source and
// slab-test rounding for rays within the scene's coordinate range (bounds[6]:
// the largest |x| + |y| + |z| of a vertex, written by other CTAs: read through L2)
__device__ inline float refit_pad(const int32_t* bounds) { return ldexpf(1.f + unord(__ldcg(&bounds[6])), -18); }

__device__ inline Box tri_box_cg(const float4* tris, int slot, float pad) {  // written in this kernel
  const float4 a = __ldcg(&tris[3 * slot]), b = __ldcg(&tris[3 * slot + 1]), c = __ldcg(&tris[3 * slot + 2]);
  Box r;
  r.lo = f3(fminf(fminf(a.x, b.x), c.x) - pad, fminf(fminf(a.y, b.y), c.y) - pad,
            fminf(fminf(a.z, b.z), c.z) - pad);
  r.hi = f3(fmaxf(fmaxf(a.x, b.x), c.x) + pad, fmaxf(fmaxf(a.y, b.y), c.y) + pad,
            fmaxf(fmaxf(a.z, b.z), c.z) + pad);
  return r;
}

// Shared memory of the crossing-node refit for a mesh of n triangles.
inline int top_slots(int n) {
  const int tiles = (n + kBuildTile - 1) / kBuildTile;
  int m = 64 * (tiles - 1);
  return m < n - 1 ? m : n - 1;
}
inline size_t top_smem(int n) {
  const int words = (n - 1 + 31) / 32;
  const int slots = top_slots(n) > 0 ? top_slots(n) : 1;
  return (size_t)words * 8 + (size_t)slots * (sizeof(SBox) + 4 + 4 + 4 + 4);
}
// the tree phase's key window, then the tile's leaf boxes (16-byte aligned)
inline __host__ __device__ size_t window_bytes(int n) {
  return ((size_t)(n < kKeyWindow ? n : kKeyWindow) * sizeof(uint32_t) + 15) / 16 * 16;
}
inline size_t tree_smem(int n) {
  const size_t keys = window_bytes(n) + (size_t)kBuildTile * sizeof(SBox);
  const size_t top = top_smem(n);
  return keys > top ? keys : top;
}

// Refit of the crossing nodes by one CTA of 1024 threads (the build's last).
__device__ void refit_crossing(int n, const float4* tris, float pad, Node* nodes, const int32_t* parent,
                               const uint32_t* crossing, int slots, int32_t* err, unsigned char* smem) {
  const int words = (n - 1 + 31) / 32;
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_wpre = s_mask + words;  // crossing nodes before each mask word
  SBox* s_box = reinterpret_cast<SBox*>(s_wpre + words);
  int32_t* s_id = reinterpret_cast<int32_t*>(s_box + slots);
  int32_t* s_pslot = s_id + slots;
  int32_t* s_kids = s_pslot + slots;  // left slot (low 16 bits) and right slot, 0xffff = not crossing
  uint32_t* s_arr = reinterpret_cast<uint32_t*>(s_kids + slots);
  __shared__ uint32_t wt[32];
  __shared__ uint32_t s_total;
  const int t = threadIdx.x;
  // slot of each crossing node = its rank in index order
  uint32_t cnt = 0;
  for (int j = 0; j < 2; ++j) {  // words 2t, 2t+1 (words <= 2048)
    const int wd = 2 * t + j;
    const uint32_t v = wd < words ? __ldcg(&crossing[wd]) : 0u;
    if (wd < words) s_mask[wd] = v;
    cnt += __popc(v);
  }
  uint32_t tot;
  uint32_t pre = block_exclusive_u32(cnt, &tot, wt);
  for (int j = 0; j < 2; ++j) {
    const int wd = 2 * t + j;
    if (wd < words) {
      s_wpre[wd] = pre;
      pre += __popc(s_mask[wd]);
    }
  }
  if (t == 0) s_total = tot;
  __syncthreads();
  const int m = (int)s_total;
  if (m > slots) {  // cannot happen for a radix tree (bound in the comment above)
    if (t == 0) atomicOr(err, 2);
    return;
  }
  if (m == 0) return;
  auto slot_of = [&](int id) -> int {  // -1 if node id is local
    const uint32_t wv = s_mask[id >> 5], bit = 1u << (id & 31);
    return (wv & bit) ? (int)(s_wpre[id >> 5] + __popc(wv & (bit - 1u))) : -1;
  };
  // slot -> node id, then one thread per crossing node (they cluster near tile
  // boundaries, so a thread per mask word would serialise them)
  for (int wd = t; wd < words; wd += 1024) {
    uint32_t v = s_mask[wd];
    int s = (int)s_wpre[wd];
    while (v) {
      s_id[s++] = 32 * wd + __ffs(v) - 1;
      v &= v - 1u;
    }
  }
  __syncthreads();
  // setup: parent slots, crossing children, the other children's boxes
  for (int s = t; s < m; s += 1024) {
    const int id = s_id[s];
    const int pid = __ldcg(&parent[id]);
    const int4 ch = __ldcg(&nodes[id].child);
    s_pslot[s] = pid >= 0 ? slot_of(pid) : -1;
    s_arr[s] = 0u;
    const int ls = ch.x >= 0 ? slot_of(ch.x) : -1, rs = ch.y >= 0 ? slot_of(ch.y) : -1;
    s_kids[s] = (int32_t)(((uint32_t)rs << 16) | ((uint32_t)ls & 0xffffu));
    if (ls < 0 && rs < 0) {  // both children built already: build this node now
      const Box bl = ch.x < 0 ? tri_box_cg(tris, ~ch.x, pad) : node_box(nodes, ch.x);
      const Box br = ch.y < 0 ? tri_box_cg(tris, ~ch.y, pad) : node_box(nodes, ch.y);
      write_node(nodes, id, bl, br);
      s_box[s] = sbox(box_union(bl, br));
    } else if (ls < 0) {
      s_box[s] = sbox(ch.x < 0 ? tri_box_cg(tris, ~ch.x, pad) : node_box(nodes, ch.x));
    } else if (rs < 0) {
      s_box[s] = sbox(ch.y < 0 ? tri_box_cg(tris, ~ch.y, pad) : node_box(nodes, ch.y));
    }
  }
  __syncthreads();
  // climb from the nodes built in setup; the last child to arrive builds the parent
  for (int s0 = t; s0 < m; s0 += 1024) {
    if (s_kids[s0] != -1) continue;  // has a crossing child: built by a climb
    int s = s0;
    for (int depth = 0; depth < 128; ++depth) {
      const int ps = s_pslot[s];
      if (ps < 0) break;  // root
      const int kids = s_kids[ps];
      const int ls = (int16_t)(kids & 0xffff), rs = kids >> 16;
      const uint32_t need = (ls >= 0) + (rs >= 0);
      __threadfence_block();
      if (atomicAdd(&s_arr[ps], 1u) + 1u < need) break;  // other crossing child not done yet
      __threadfence_block();
      const Box bl = unsbox(s_box[ls >= 0 ? ls : ps]);
      const Box br = unsbox(s_box[rs >= 0 ? rs : ps]);
      write_node(nodes, s_id[ps], bl, br);
      s_box[ps] = sbox(box_union(bl, br));
      s = ps;
    }
  }
}

// ---- the whole build as one cooperative kernel -------------------------------
//
// One CTA of 1024 threads per tile of 1024 triangles, all resident at once
// (cooperative launch), with grid-wide barriers between the phases: centroid
// bounds; Morton keys and their digit counts; four stable passes of an 8-bit
// LSD radix sort (each CTA ranks its tile by digit and scatters with the digit
// counts of the tiles before it, which the previous pass's scatter counted by
// destination tile: one barrier per pass); then the tiled tree build above.
// Data written by other CTAs is read through L2 (ld.cg), never through the
// non-coherent L1 path.

constexpr int kBarrierSpins = 1 << 22;  // ~0.3 s of polling before a barrier gives up
constexpr int kSortStride = 257;        // padded per-warp row of 256 digit counters

struct BuildBufs {
  uint32_t* keys[2];
  int32_t* vals[2];
  float4* tris;
  Node* nodes;
  int32_t* parent;
  uint32_t* crossing;
  int32_t* bounds;    // [8] ordered ints: centroid min xyz, max xyz, max |coord|
  uint32_t* hist;     // [4*256] digit counts of all keys
  uint32_t* tile_hist;  // [3][tiles*256] digit counts per tile: pass p's in buffer p % 3
  uint32_t* bar;      // [2] grid barrier: arrivals, generation
  uint32_t* done;     // [1] CTAs finished with the tree
  int32_t* err;
};

// Grid-wide barrier for a cooperative launch.  Waits are bounded: on timeout the
// error word gets bit 2 and false is returned (the caller then exits).
__device__ bool grid_sync(uint32_t* bar, uint32_t nblocks, int32_t* err) {
  __shared__ int s_ok;
  __syncthreads();  // the CTA's writes happen before thread 0's release (cumulative)
  if (threadIdx.x == 0) {
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> cnt(bar[0]), gen(bar[1]);
    const uint32_t g = gen.load(cuda::memory_order_acquire);
    int ok = 1;
    if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == nblocks - 1u) {
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.store(g + 1u, cuda::memory_order_release);
    } else {
      for (int it = 0; gen.load(cuda::memory_order_acquire) == g; ++it) {
        if (it >= kBarrierSpins) {
          atomicOr(err, 4);
          ok = 0;
          break;
        }
        if (it > 256) __nanosleep(64);  // poll tightly at first, then back off
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Barrier between the build's phases: a thread-block cluster's hardware barrier
// (release / acquire at cluster scope) when the whole grid is one cluster, else
// the grid-wide barrier above.  A cluster's CTAs are resident together and take
// no early exit before the last barrier, so the cluster barrier always completes.
__device__ inline bool build_sync(uint32_t* bar, uint32_t nblocks, int32_t* err, bool cluster) {
  if (cluster) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  }
  return grid_sync(bar, nblocks, err);
}

// exclusive scan of 256 counts held in shared memory, by one warp (8 per lane)
__device__ inline void warp_scan256(const uint32_t* in, uint32_t* out) {
  const int lane = threadIdx.x & 31;
  uint32_t c[8], sum = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    c[j] = in[8 * lane + j];
    sum += c[j];
  }
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  uint32_t r = x - sum;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    out[8 * lane + j] = r;
    r += c[j];
  }
}

// Dynamic shared memory: the sort's counters and staging, later reused for the
// key window and the crossing-node refit.
constexpr size_t kSortSmem = (size_t)(32 * kSortStride + 4 * 256 + 3 * 256 + 2 * kBuildTile) * 4;
inline size_t build_smem(int n) {
  const size_t t = tree_smem(n);
  return t > kSortSmem ? t : kSortSmem;
}

// kRefit: the boxes of the tree of the last build for new vertex positions of the
// same mesh (phases 1, 4 and 5: the bounds for the pads, then the packing and the
// refit with the kept triangle order, children and crossing marks).
template <bool kRefit>
__global__ void __launch_bounds__(kBuildTile) k_build_scene(const float* __restrict__ verts, int nv,
                                                            const int32_t* __restrict__ faces, int n,
                                                            BuildBufs B, int slots, bool cluster) {
  __shared__ int32_t s_par_leaf[kBuildTile];  // in-tile parent of leaf c0+t, else -1
  __shared__ int32_t s_par_node[kBuildTile];  // in-tile local parent of node c0+t, else -1
  __shared__ int2 s_child[kBuildTile];
  __shared__ uint32_t s_arr[kBuildTile];
  __shared__ SBox s_box[kBuildTile];  // box of local node c0+t once built
  __shared__ int32_t s_red[32][8];
  __shared__ bool s_last;
  extern __shared__ __align__(16) unsigned char build_sm[];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, c0 = blockIdx.x * kBuildTile, i = c0 + t;
  const uint32_t nb = gridDim.x;
  const bool live = i < n;

  // 1. centroid box and largest coordinate (ordered-int atomics, one set per CTA)
  float3 a = f3(0.f, 0.f, 0.f), b = a, c = a;
  if (live) {
    a = vload(verts, face_vert(faces, i, 0, nv, B.err));
    b = vload(verts, face_vert(faces, i, 1, nv, B.err));
    c = vload(verts, face_vert(faces, i, 2, nv, B.err));
  }
  {
    const float3 m = (a + b + c) * (1.f / 3.f);
    int32_t v[7] = {ord(m.x), ord(m.y), ord(m.z), ord(m.x), ord(m.y), ord(m.z),
                    ord(fmaxf(fmaxf(l1(a), l1(b)), l1(c)))};
    if (!live) {
      v[0] = v[1] = v[2] = 0x7fffffff;
      v[3] = v[4] = v[5] = (int32_t)0x80000000;
      v[6] = 0;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = min(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
#pragma unroll
      for (int k = 3; k < 7; ++k) v[k] = max(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    }
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 7; ++k) s_red[w][k] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[k] = s_red[lane][k];
#pragma unroll
      for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = min(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
#pragma unroll
        for (int k = 3; k < 7; ++k) v[k] = max(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
      }
      int32_t mine = v[0];
#pragma unroll
      for (int k = 1; k < 7; ++k)
        if (lane == k) mine = v[k];
      if (lane < 3) atomicMin(&B.bounds[lane], mine);
      else if (lane < 7) atomicMax(&B.bounds[lane], mine);
    }
  }
  if (!build_sync(B.bar, nb, B.err, cluster)) return;

  if (!kRefit) {
  // 2. Morton keys and the digit counts of all four places
  uint32_t* cnt = reinterpret_cast<uint32_t*>(build_sm);  // [32][kSortStride]
  uint32_t* goff = cnt + 32 * kSortStride;                 // [4][256] start of each digit, whole array
  uint32_t* tot = goff + 4 * 256;                          // [256] tile's digit counts
  uint32_t* lstart = tot + 256;                            // [256] digit start within the tile
  uint32_t* gbase = lstart + 256;                          // [256] output position of the tile's digit d, minus lstart
  uint32_t* stage_k = gbase + 256;                         // [1024] tile grouped by digit
  int32_t* stage_v = reinterpret_cast<int32_t*>(stage_k + kBuildTile);
  uint32_t key = live ? morton_key(a, b, c, B.bounds) : 0u;
  int32_t val = i;
  goff[t] = 0u;  // 1024 threads: the CTA's own counts first
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint32_t d = (key >> (8 * p)) & 255u;
    const uint32_t peers = warp_peers8(d, live);
    if (live && lane == __ffs(peers) - 1) atomicAdd(&goff[256 * p + d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (goff[t]) atomicAdd(&B.hist[t], goff[t]);
  // per-tile digit counts of pass p live in tile_hist[p % 3]: pass 0's are this tile's own
  // keys; the other two buffers start at zero and collect the scatters' counts
  const size_t hrow = (size_t)blockIdx.x * 256, hbuf = (size_t)nb * 256;
  if (t < 256) {
    B.tile_hist[hrow + t] = goff[t];
    B.tile_hist[hbuf + hrow + t] = 0u;
    B.tile_hist[2 * hbuf + hrow + t] = 0u;
  }
  if (!build_sync(B.bar, nb, B.err, cluster)) return;
  if (w < 4) {  // warp p: start of each digit of place p in the sorted array
    uint32_t c8[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c8[j] = __ldcg(&B.hist[256 * w + 8 * lane + j]);
      sum += c8[j];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    uint32_t r = x - sum;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      goff[256 * w + 8 * lane + j] = r;
      r += c8[j];
    }
  }

  // 3. four stable passes; pass p moves keys[p & 1] to keys[(p + 1) & 1], one grid barrier
  // each: the tile counts it needs were added by the previous pass's scatter, which also
  // adds those of the next pass, by destination tile, into tile_hist[(p + 1) % 3]
  const uint32_t lt = (1u << lane) - 1u;
  const int rn = min(n - c0, kBuildTile);
  uint32_t* row = cnt + w * kSortStride;
#pragma unroll 1
  for (int p = 0; p < 4; ++p) {
    const int shift = 8 * p;
    if (p > 0) {
      key = live ? __ldcg(&((p & 1) ? B.keys[1] : B.keys[0])[i]) : 0u;
      val = live ? __ldcg(&((p & 1) ? B.vals[1] : B.vals[0])[i]) : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) row[lane + 32 * j] = 0u;
    __syncwarp();
    const uint32_t d = (key >> shift) & 255u;
    const uint32_t peers = warp_peers8(d, live);
    const uint32_t rank = __popc(peers & lt);
    if (live && lane == __ffs(peers) - 1) row[d] = __popc(peers);
    __syncthreads();
    // per digit: exclusive scan over the warps (warp w: digits w, w+32, ...)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int dd = w + 32 * j;
      const uint32_t cv = cnt[lane * kSortStride + dd];
      uint32_t x = cv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      cnt[lane * kSortStride + dd] = x - cv;
      if (lane == 31) tot[dd] = x;
    }
    __syncthreads();
    if (w == 0) warp_scan256(tot, lstart);
    __syncthreads();
    if (live) {
      const uint32_t q = lstart[d] + row[d] + rank;
      stage_k[q] = key;
      stage_v[q] = val;
    }
    const uint32_t* th = B.tile_hist + (size_t)(p % 3) * hbuf;
    if (t < 256) {  // digit t's output start for this tile: whole-array start + earlier tiles
      uint32_t pre = 0;
      for (uint32_t c2 = 0; c2 < blockIdx.x; ++c2) pre += __ldcg(&th[(size_t)c2 * 256 + t]);
      gbase[t] = goff[256 * p + t] + pre - lstart[t];
      // this tile's row of the buffer pass p + 1 fills, read last by pass p - 2
      if (p == 1) B.tile_hist[hrow + t] = 0u;
    }
    __syncthreads();
    uint32_t* th_next = B.tile_hist + (size_t)((p + 1) % 3) * hbuf;
    if (t < rn) {
      const uint32_t k2 = stage_k[t];
      const uint32_t pos = gbase[(k2 >> shift) & 255u] + (uint32_t)t;
      if (pos < (uint32_t)n) {  // always true when the counts match the keys
        ((p & 1) ? B.keys[0] : B.keys[1])[pos] = k2;
        ((p & 1) ? B.vals[0] : B.vals[1])[pos] = stage_v[t];
        if (p < 3) atomicAdd(&th_next[(size_t)(pos / kBuildTile) * 256 + ((k2 >> (shift + 8)) & 255u)], 1u);
      }
    }
    if (!build_sync(B.bar, nb, B.err, cluster)) return;
  }

  }  // !kRefit

  // 4. tree: this tile's triangles in sorted order, its nodes, the local refit
  const uint32_t* keys = B.keys[0];
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(build_sm);
  const int wlen = min(n, kKeyWindow);
  const int wlo = min(max(c0 + kBuildTile / 2 - kKeyWindow / 2, 0), n - wlen);
  if (!kRefit) {
    // window copy with every load in flight before the stores (a plain loop
    // would wait out one L2 round trip per element it moves)
    constexpr int kU = 8;
    for (int base = 0; base < wlen; base += kU * kBuildTile) {
      uint32_t tmp[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int j = base + u * kBuildTile + t;
        tmp[u] = j < wlen ? __ldcg(&keys[wlo + j]) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int j = base + u * kBuildTile + t;
        if (j < wlen) s_keys[j] = tmp[u];
      }
    }
  }
  s_par_leaf[t] = -1;
  s_par_node[t] = -1;
  s_arr[t] = 0u;
  const float pad = refit_pad(B.bounds);
  Box bx{};
  if (live) {
    const int f = __ldcg(&B.vals[0][i]);
    const float3 p0 = vload(verts, face_vert(faces, f, 0, nv, B.err));
    const float3 p1 = vload(verts, face_vert(faces, f, 1, nv, B.err));
    const float3 p2 = vload(verts, face_vert(faces, f, 2, nv, B.err));
    B.tris[3 * i + 0] = make_float4(p0.x, p0.y, p0.z, __int_as_float(f));
    B.tris[3 * i + 1] = make_float4(p1.x, p1.y, p1.z, 0.f);
    B.tris[3 * i + 2] = make_float4(p2.x, p2.y, p2.z, 0.f);
    bx.lo = f3(fminf(fminf(p0.x, p1.x), p2.x) - pad, fminf(fminf(p0.y, p1.y), p2.y) - pad,
               fminf(fminf(p0.z, p1.z), p2.z) - pad);
    bx.hi = f3(fmaxf(fmaxf(p0.x, p1.x), p2.x) + pad, fmaxf(fmaxf(p0.y, p1.y), p2.y) + pad,
               fmaxf(fmaxf(p0.z, p1.z), p2.z) + pad);
  }
  SBox* s_leaf = reinterpret_cast<SBox*>(build_sm + window_bytes(n));  // box of leaf c0+t
  s_leaf[t] = sbox(bx);
  __syncthreads();
  bool cross = false;
  if (kRefit && i < n - 1) {  // the kept topology: children and crossing marks of the last build
    const int4 ch = __ldcg(&B.nodes[i].child);
    const int left = ch.x, right = ch.y;
    s_child[t] = make_int2(left, right);
    cross = (__ldcg(&B.crossing[i >> 5]) >> (i & 31)) & 1u;
    if (!cross) {
      if (left < 0) s_par_leaf[~left - c0] = i;
      else s_par_node[left - c0] = i;
      if (right < 0) s_par_leaf[~right - c0] = i;
      else s_par_node[right - c0] = i;
    }
  }
  if (!kRefit && i < n - 1) {
    int left, right, lo, hi;
    if (wlen == n) {  // every key in shared memory: plain shared loads in the searches
      karras_node([&](int j) { return s_keys[j]; }, n, i, &left, &right, &lo, &hi);
    } else {  // a window: a lookup that may read either space becomes a generic load, ~3x slower
      karras_node(
          [&](int j) {
            const unsigned r = (unsigned)(j - wlo);
            return r < (unsigned)wlen ? s_keys[r] : __ldcg(&keys[j]);
          },
          n, i, &left, &right, &lo, &hi);
    }
    B.nodes[i].child = make_int4(left, right, 0, 0);
    B.parent[left >= 0 ? left : (n - 1 + ~left)] = i;
    B.parent[right >= 0 ? right : (n - 1 + ~right)] = i;
    s_child[t] = make_int2(left, right);
    cross = (lo / kBuildTile) != (hi / kBuildTile);
    if (!cross) {  // local: both children are in this tile
      if (left < 0) s_par_leaf[~left - c0] = i;
      else s_par_node[left - c0] = i;
      if (right < 0) s_par_leaf[~right - c0] = i;
      else s_par_node[right - c0] = i;
    }
  }
  if (!kRefit) {
    if (i == 0) B.parent[0] = -1;
    const uint32_t mword = __ballot_sync(0xffffffffu, cross);
    if (lane == 0 && i < n - 1) B.crossing[i >> 5] = mword;
  }
  __syncthreads();
  int me = ~i;  // child code of the subtree this thread holds
  int pn = live ? s_par_leaf[t] : -1;
  while (pn >= 0) {
    const int lp = pn - c0;
    if (me >= 0) s_box[me - c0] = sbox(bx);  // leaf boxes are re-read by the sibling
    __threadfence_block();
    if (atomicAdd(&s_arr[lp], 1u) == 0u) break;  // sibling subtree not done yet
    __threadfence_block();
    const int2 ch = s_child[lp];
    const bool is_left = ch.x == me;
    const int sib = is_left ? ch.y : ch.x;
    const Box sb = unsbox(sib < 0 ? s_leaf[~sib - c0] : s_box[sib - c0]);  // both in this tile
    if (is_left) write_node(B.nodes, pn, bx, sb);
    else write_node(B.nodes, pn, sb, bx);
    bx = box_union(bx, sb);
    me = pn;
    pn = s_par_node[lp];
  }

  // 5. the last CTA refits the crossing nodes and resets the counters
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(B.done, 1u) == nb - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  refit_crossing(n, B.tris, pad, B.nodes, B.parent, B.crossing, slots, B.err, build_sm);
  __syncthreads();
  if (t < 3) B.bounds[t] = 0x7fffffff;
  else if (t < 6) B.bounds[t] = (int32_t)0x80000000;
  else if (t < 8) B.bounds[t] = 0;
  B.hist[t] = 0u;
  if (t == 0) *B.done = 0u;
}

// ---- 4-wide collapse ---------------------------------------------------------

__device__ inline float half_area(const Box& b) {
  const float dx = b.hi.x - b.lo.x, dy = b.hi.y - b.lo.y, dz = b.hi.z - b.lo.z;
  return dx * dy + dy * dz + dz * dx;
}
__device__ inline void node_children(const Node* nodes, int i, Box& l, Box& r, int& cl, int& cr) {
  const float4 a = __ldg(&nodes[i].lxy), b = __ldg(&nodes[i].rxy), z = __ldg(&nodes[i].lrz);
  const int4 ch = __ldg(&nodes[i].child);
  l.lo = f3(a.x, a.z, z.x);
  l.hi = f3(a.y, a.w, z.y);
  r.lo = f3(b.x, b.z, z.z);
  r.hi = f3(b.y, b.w, z.w);
  cl = ch.x;
  cr = ch.y;
}

// Entry i of the 4-wide tree: binary node i's grandchildren, then greedy
// expansion of the largest internal slot while fewer than four slots are used.
__global__ void k_collapse4(const Node* __restrict__ nodes, int n, Node4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  Box bx[4];
  int id[4];
  int cnt = 0;
  {
    Box l, r;
    int cl, cr;
    node_children(nodes, i, l, r, cl, cr);
    bx[0] = l;
    id[0] = cl;
    bx[1] = r;
    id[1] = cr;
    cnt = 2;
  }
  for (int it = 0; it < 3 && cnt < 4; ++it) {
    int best = -1;
    float area = -1.f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < cnt && id[k] >= 0 && half_area(bx[k]) > area) {
        area = half_area(bx[k]);
        best = k;
      }
    if (best < 0) break;
    Box l, r;
    int cl, cr;
    node_children(nodes, id[best], l, r, cl, cr);
    bx[best] = l;
    id[best] = cl;
    bx[cnt] = r;  // cnt < 4
    id[cnt] = cr;
    ++cnt;
  }
  Node4 o;
  float* f = reinterpret_cast<float*>(&o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool used = k < cnt;
    f[0 * 4 + k] = used ? bx[k].lo.x : 0.f;
    f[1 * 4 + k] = used ? bx[k].hi.x : 0.f;
    f[2 * 4 + k] = used ? bx[k].lo.y : 0.f;
    f[3 * 4 + k] = used ? bx[k].hi.y : 0.f;
    f[4 * 4 + k] = used ? bx[k].lo.z : 0.f;
    f[5 * 4 + k] = used ? bx[k].hi.z : 0.f;
  }
  o.child = make_int4(cnt > 0 ? id[0] : kEmpty, cnt > 1 ? id[1] : kEmpty, cnt > 2 ? id[2] : kEmpty,
                      cnt > 3 ? id[3] : kEmpty);
  o.pad = make_int4(cnt, 0, 0, 0);
  out[i] = o;
}

// Breadth-first copy of the top kTopLevels levels of the 4-wide tree (one CTA,
// level by level): staged entries link to each other as kStaged + position.
__global__ void __launch_bounds__(128) k_top_table(const Node4* __restrict__ nodes4, int nt, Node4* __restrict__ top,
                                                   int32_t* __restrict__ top_n) {
  __shared__ int idx[kTopMax];  // full-tree index of each staged entry
  __shared__ int lvl_begin, lvl_end;
  const int t = threadIdx.x;
  if (t == 0) {
    lvl_begin = 0;
    lvl_end = nt > 1 ? 1 : 0;
    idx[0] = 0;
  }
  __syncthreads();
  for (int level = 1; level < kTopLevels; ++level) {
    const int b = lvl_begin, e = lvl_end;
    __syncthreads();
    if (t == 0) {  // append the internal children of this level in (entry, slot) order
      int n = e;
      for (int q = b; q < e; ++q) {
        const int4 ch = nodes4[idx[q]].child;
        const int c[4] = {ch.x, ch.y, ch.z, ch.w};
        for (int k = 0; k < 4; ++k)
          if (c[k] >= 0 && n < kTopMax) idx[n++] = c[k];
      }
      lvl_begin = e;
      lvl_end = n;
    }
    __syncthreads();
  }
  const int n = lvl_end;
  for (int q = t; q < n; q += blockDim.x) {
    Node4 o = nodes4[idx[q]];
    int c[4] = {o.child.x, o.child.y, o.child.z, o.child.w};
    for (int k = 0; k < 4; ++k)
      if (c[k] >= 0)
        for (int r = 1; r < n; ++r)
          if (idx[r] == c[k]) {
            c[k] = kStaged + r;
            break;
          }
    o.child = make_int4(c[0], c[1], c[2], c[3]);
    o.pad.y = idx[q];
    top[q] = o;
  }
  if (t == 0) *top_n = n;
}

inline int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

size_t layout(sbr_scene* s, void* mem, int32_t nt) {
  Carver c(mem);
  int64_t n = nt > 0 ? nt : 1;
  int64_t ni = n > 1 ? n - 1 : 1;
  s->tris = c.take<float4>(3 * n);
  s->nodes = c.take<Node>(ni);
  s->nodes4 = c.take<Node4>(ni);
  s->top = c.take<Node4>(kTopMax);
  s->top_n = c.take<int32_t>(1);
  s->parent = c.take<int32_t>(2 * n);
  s->visits = c.take<uint32_t>(ni);
  s->keys[0] = c.take<uint32_t>(n);
  s->keys[1] = c.take<uint32_t>(n);
  s->vals[0] = c.take<int32_t>(n);
  s->vals[1] = c.take<int32_t>(n);
  s->faces = c.take<int32_t>(3 * n);
  s->bounds = c.take<int32_t>(8);
  s->err = c.take<int32_t>(1);
  s->hist = c.take<uint32_t>(4 * 256);
  s->done = c.take<uint32_t>(1);
  s->bar = c.take<uint32_t>(2);
  s->tile_hist = c.take<uint32_t>((size_t)3 * 256 * ((n + kBuildTile - 1) / kBuildTile));
  s->sort_scratch = c.take<char>(sort_scratch_bytes(n));
  return c.bytes();
}

// The whole build, or with refit the boxes of the last build's tree for new vertex
// positions (triangle order, children and crossing marks kept).
sbr_status rebuild(sbr_scene* s, const float* verts, cudaStream_t st, bool refit = false) {
  const int nt = s->nt, nv = s->nv;
  if (s->coop) {  // one cooperative launch; it leaves its counters reset for the next build
    BuildBufs B{{s->keys[0], s->keys[1]}, {s->vals[0], s->vals[1]}, s->tris, s->nodes, s->parent, s->visits,
                s->bounds, s->hist, s->tile_hist, s->bar, s->done, s->err};
    int slots = top_slots(nt), n = nt, nvv = nv;
    const int32_t* faces = s->faces;
    if (s->cluster) {  // the whole grid one cluster: hardware barriers between the phases
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(blocks(nt, kBuildTile));
      cfg.blockDim = dim3(kBuildTile);
      cfg.dynamicSmemBytes = build_smem(nt);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = blocks(nt, kBuildTile);
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      ::sbr::note_launch();
      if (refit) SBR_CUDA(cudaLaunchKernelEx(&cfg, k_build_scene<true>, verts, nv, faces, nt, B, slots, true));
      else SBR_CUDA(cudaLaunchKernelEx(&cfg, k_build_scene<false>, verts, nv, faces, nt, B, slots, true));
      ::sbr::note_launch();
      k_collapse4<<<blocks(nt - 1, 128), 128, 0, st>>>(s->nodes, nt, s->nodes4);
      if (kTopLevels > 0) {
        ::sbr::note_launch();
        k_top_table<<<1, 128, 0, st>>>(s->nodes4, nt, s->top, s->top_n);
      }
      SBR_CUDA(cudaGetLastError());
      return SBR_OK;
    }
    bool no_cluster = false;
    void* args[] = {(void*)&verts, (void*)&nvv, (void*)&faces, (void*)&n, (void*)&B, (void*)&slots,
                    (void*)&no_cluster};
    ::sbr::note_launch();
    SBR_CUDA(cudaLaunchCooperativeKernel(refit ? (const void*)k_build_scene<true> : (const void*)k_build_scene<false>,
                                         dim3(blocks(nt, kBuildTile)), dim3(kBuildTile), args, build_smem(nt), st));
    ::sbr::note_launch();
    k_collapse4<<<blocks(nt - 1, 128), 128, 0, st>>>(s->nodes, nt, s->nodes4);
    if (kTopLevels > 0) {
      ::sbr::note_launch();
      k_top_table<<<1, 128, 0, st>>>(s->nodes4, nt, s->top, s->top_n);
    }
    SBR_CUDA(cudaGetLastError());
    return SBR_OK;
  }
  ::sbr::note_launch();
  k_init_bounds<<<1, 256, 0, st>>>(s->bounds, s->err, s->hist);
  if (nt == 0) {
    SBR_CUDA(cudaGetLastError());
    return SBR_OK;
  }
  ::sbr::note_launch();
  k_bounds<<<blocks(nt, 256), 256, 0, st>>>(verts, nv, s->faces, nt, s->bounds, s->err);
  if (!refit) {
    ::sbr::note_launch();
    k_morton<<<blocks(nt, 256), 256, 0, st>>>(verts, nv, s->faces, nt, s->bounds, s->keys[0],
                                              s->vals[0], s->hist, s->err);
    SBR_CUDA(radix_sort_pairs(s->keys, s->vals, nt, nullptr, 31, s->sort_scratch, st, s->hist));
  }
  ::sbr::note_launch();
  k_pack<<<blocks(nt, 256), 256, 0, st>>>(verts, nv, s->faces, nt, s->vals[0], s->tris, s->err);
  if (nt > 1) {
    if (!refit) {
      ::sbr::note_launch();
      k_karras<<<blocks(nt - 1, 256), 256, 0, st>>>(s->keys[0], nt, s->nodes, s->parent);
    }
    SBR_CUDA(cudaMemsetAsync(s->visits, 0, sizeof(uint32_t) * (nt - 1), st));
    ::sbr::note_launch();
    k_refit<<<blocks(nt, 256), 256, 0, st>>>(s->tris, nt, s->nodes, s->parent, s->visits,
                                             s->bounds);
    ::sbr::note_launch();
    k_collapse4<<<blocks(nt - 1, 128), 128, 0, st>>>(s->nodes, nt, s->nodes4);
  }
  if (kTopLevels > 0) {
    ::sbr::note_launch();
    k_top_table<<<1, 128, 0, st>>>(s->nodes4, nt, s->top, s->top_n);
  }
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}

}  // namespace
}  // namespace sbr

using namespace sbr;

extern "C" size_t sbr_scene_bytes(int32_t nt) {
  sbr_scene s{};
  return layout(&s, nullptr, nt < 0 ? 0 : nt);
}

extern "C" sbr_status sbr_scene_create(const float* d_verts, int32_t nv, const int32_t* d_faces,
                                       int32_t nt, void* d_mem, size_t mem_bytes,
                                       sbr_stream stream, sbr_scene** out) {
  SBR_ARG(out != nullptr, "sbr_scene_create: out is NULL");
  *out = nullptr;
  SBR_ARG(nt >= 0 && nv >= 0, "sbr_scene_create: negative size (nv=%d nt=%d)", nv, nt);
  SBR_ARG(nt <= (1 << 26), "sbr_scene_create: nt=%d above the 2^26 limit", nt);
  SBR_ARG(nt == 0 || (d_verts && d_faces && nv > 0), "sbr_scene_create: NULL mesh pointer");
  SBR_ARG(d_mem && aligned256(d_mem), "sbr_scene_create: d_mem NULL or not 256-byte aligned");
  const size_t need = sbr_scene_bytes(nt);
  if (mem_bytes < need) {
    set_error("sbr_scene_create: region of %zu bytes, %zu needed", mem_bytes, need);
    return SBR_ERR_OOM;
  }
  sbr_scene* s = static_cast<sbr_scene*>(calloc(1, sizeof(sbr_scene)));
  if (!s) {
    set_error("sbr_scene_create: host allocation failed");
    return SBR_ERR_OOM;
  }
  s->nv = nv;
  s->nt = nt;
  s->bytes = layout(s, d_mem, nt);
  {
    // The cooperative build needs every tile's CTA resident at once (1024
    // threads and up to ~224 KB of shared memory each); otherwise the
    // multi-kernel build runs.
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (nt >= 2 && nt <= kTiledMax) {
      int dev = 0, sms = 0, coop = 0, per_sm = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_build_scene<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)build_smem(kTiledMax));  // the largest any scene asks
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_build_scene<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)build_smem(kTiledMax));
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_scene<false>, kBuildTile, build_smem(nt));
      s->coop = e == cudaSuccess && coop && (int64_t)per_sm * sms >= blocks(nt, kBuildTile);
      if (e != cudaSuccess) (void)cudaGetLastError();  // not fatal: the multi-kernel build runs
      // up to 16 tiles the grid can run as one cluster, when the GPU can hold it
      const int tiles = blocks(nt, kBuildTile);
      s->cluster = 0;
      if (s->coop && tiles <= 16) {
        cudaError_t ce = cudaFuncSetAttribute(k_build_scene<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (ce == cudaSuccess)
          ce = cudaFuncSetAttribute(k_build_scene<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(tiles);
        cfg.blockDim = dim3(kBuildTile);
        cfg.dynamicSmemBytes = build_smem(nt);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = tiles;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveClusters(&clusters, k_build_scene<false>, &cfg);
        if (ce == cudaSuccess && clusters >= 1) s->cluster = 1;
        else (void)cudaGetLastError();  // the cooperative launch stays
      }
      e = cudaSuccess;
    }
    // counters of the cooperative build start cleared; bounds start empty
    e = cudaMemsetAsync(s->err, 0, sizeof(int32_t), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->bar, 0, 2 * sizeof(uint32_t), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->done, 0, sizeof(uint32_t), cs);
    if (e == cudaSuccess) {
      ::sbr::note_launch();
      k_init_bounds<<<1, 256, 0, cs>>>(s->bounds, s->err, s->hist);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      set_error("sbr_scene_create: %s", cudaGetErrorString(e));
      free(s);
      return SBR_ERR_CUDA;
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (nt > 0) {
    cudaError_t e = cudaMemcpyAsync(s->faces, d_faces, sizeof(int32_t) * 3 * (size_t)nt,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      set_error("sbr_scene_create: face copy failed: %s", cudaGetErrorString(e));
      free(s);
      return SBR_ERR_CUDA;
    }
  }
  sbr_status r = rebuild(s, d_verts, st);
  if (r != SBR_OK) {
    free(s);
    return r;
  }
  *out = s;
  return SBR_OK;
}

extern "C" sbr_status sbr_scene_update(sbr_scene* scene, const float* d_verts, sbr_stream stream) {
  SBR_ARG(scene != nullptr, "sbr_scene_update: scene is NULL");
  SBR_ARG(scene->nt == 0 || d_verts, "sbr_scene_update: d_verts is NULL");
  return rebuild(scene, d_verts, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" sbr_status sbr_scene_refit(sbr_scene* scene, const float* d_verts, sbr_stream stream) {
  SBR_ARG(scene != nullptr, "sbr_scene_refit: scene is NULL");
  SBR_ARG(scene->nt == 0 || d_verts, "sbr_scene_refit: d_verts is NULL");
  return rebuild(scene, d_verts, reinterpret_cast<cudaStream_t>(stream), true);
}

extern "C" sbr_status sbr_scene_check(const sbr_scene* scene, sbr_stream stream) {
  SBR_ARG(scene != nullptr, "sbr_scene_check: scene is NULL");
  int32_t err = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SBR_CUDA(cudaMemcpyAsync(&err, scene->err, sizeof(err), cudaMemcpyDeviceToHost, st));
  SBR_CUDA(cudaStreamSynchronize(st));
  SBR_ARG((err & 1) == 0, "sbr_scene: face index outside [0, nv) (error word %d)", err);
  if (err) {
    set_error("sbr_scene: tree build failed (error word %d)", err);
    return SBR_ERR_CUDA;
  }
  return SBR_OK;
}

extern "C" void sbr_scene_destroy(sbr_scene* scene) { free(scene); }

extern "C" sbr_status sbr_scene_set_motion(sbr_scene* scene, const sbr_motion* m) {
  SBR_ARG(scene, "sbr_scene_set_motion: scene is NULL");
  if (!m || m->n_objects == 0) {
    scene->n_obj = 0;
    scene->tri_obj = nullptr;
    return SBR_OK;
  }
  SBR_ARG(m->n_objects > 0 && m->n_objects <= SBR_MAX_OBJECTS, "sbr_scene_set_motion: n_objects=%d outside [0, %d]",
          m->n_objects, SBR_MAX_OBJECTS);
  for (int i = 0; i < m->n_objects; ++i)
    for (int j = 0; j < 3; ++j)
      SBR_ARG(std::isfinite(m->velocity[i][j]), "sbr_scene_set_motion: object %d: non-finite velocity", i);
  scene->n_obj = m->n_objects;
  scene->tri_obj = m->tri_object;
  for (int i = 0; i < SBR_MAX_OBJECTS; ++i)
    for (int j = 0; j < 3; ++j) scene->vel[i][j] = i < m->n_objects ? m->velocity[i][j] : 0.f;
  return SBR_OK;
}

extern "C" sbr_status sbr_scene_set_materials(sbr_scene* scene, const sbr_materials* m) {
  SBR_ARG(scene, "sbr_scene_set_materials: scene is NULL");
  if (!m || m->n_materials == 0) {
    scene->n_mat = 0;
    scene->tri_mat = nullptr;
    return SBR_OK;
  }
  SBR_ARG(m->n_materials > 0 && m->n_materials <= SBR_MAX_MATERIALS,
          "sbr_scene_set_materials: n_materials=%d outside [0, %d]", m->n_materials, SBR_MAX_MATERIALS);
  for (int i = 0; i < m->n_materials; ++i) {
    const float er = m->eps_re[i], ei = m->eps_im[i];
    SBR_ARG(std::isfinite(er) && std::isfinite(ei) && ei >= 0.f,
            "sbr_scene_set_materials: material %d: eps_im must be finite and >= 0", i);
    SBR_ARG(er <= 0.f || std::hypot((double)er - 1.0, (double)ei) >= 1e-6,
            "sbr_scene_set_materials: material %d: eps = 1 does not reflect", i);
  }
  scene->n_mat = m->n_materials;
  scene->tri_mat = m->tri_material;
  for (int i = 0; i < SBR_MAX_MATERIALS; ++i) {
    scene->eps_re[i] = i < m->n_materials ? m->eps_re[i] : -1.f;
    scene->eps_im[i] = i < m->n_materials ? m->eps_im[i] : 0.f;
  }
  return SBR_OK;
}
