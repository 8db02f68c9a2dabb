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

#include <cuda/atomic>

#include "scene.cuh"

namespace sbr {
namespace {

__device__ inline int32_t ord(float f) {
  int32_t i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ inline float unord(int32_t i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_init_bounds(int32_t* b, int32_t* err) {
  if (threadIdx.x < 3) b[threadIdx.x] = 0x7fffffff;           // min x, y, z
  else if (threadIdx.x < 6) b[threadIdx.x] = (int32_t)0x80000000;  // max x, y, z
  else if (threadIdx.x == 6) b[6] = 0;                        // max |coord| (ordered, >= 0)
  else if (threadIdx.x == 7) b[7] = 0;
  if (threadIdx.x == 0) *err = 0;
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

__global__ void k_morton(const float* __restrict__ verts, int nv, const int32_t* __restrict__ faces,
                         int nt, const int32_t* __restrict__ bounds, uint32_t* keys, int32_t* vals,
                         int32_t* err) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nt) return;
  float3 a = vload(verts, face_vert(faces, f, 0, nv, err));
  float3 b = vload(verts, face_vert(faces, f, 1, nv, err));
  float3 c = vload(verts, face_vert(faces, f, 2, nv, err));
  float3 m = (a + b + c) * (1.f / 3.f);
  float3 lo = f3(unord(bounds[0]), unord(bounds[1]), unord(bounds[2]));
  float3 hi = f3(unord(bounds[3]), unord(bounds[4]), unord(bounds[5]));
  float3 ext = hi - lo;
  float qx = ext.x > 0.f ? (m.x - lo.x) / ext.x : 0.f;
  float qy = ext.y > 0.f ? (m.y - lo.y) / ext.y : 0.f;
  float qz = ext.z > 0.f ? (m.z - lo.z) / ext.z : 0.f;
  uint32_t ix = (uint32_t)fminf(fmaxf(qx * 1024.f, 0.f), 1023.f);
  uint32_t iy = (uint32_t)fminf(fmaxf(qy * 1024.f, 0.f), 1023.f);
  uint32_t iz = (uint32_t)fminf(fmaxf(qz * 1024.f, 0.f), 1023.f);
  // Triangles spanning more than 1/32 of the centroid box (a ground plane under
  // an object) get key bit 30, so the radix tree puts them in their own subtree
  // at the root instead of inflating the boxes of their Morton neighbours.
  const float side = fmaxf(fmaxf(fmaxf(fabsf(a.x - b.x), fabsf(b.x - c.x)), fabsf(c.x - a.x)),
                           fmaxf(fmaxf(fmaxf(fabsf(a.y - b.y), fabsf(b.y - c.y)), fabsf(c.y - a.y)),
                                 fmaxf(fmaxf(fabsf(a.z - b.z), fabsf(b.z - c.z)), fabsf(c.z - a.z))));
  const float extent = fmaxf(fmaxf(ext.x, ext.y), ext.z);
  const uint32_t big = (extent > 0.f && side * 32.f > extent) ? (1u << 30) : 0u;
  keys[f] = big | (spread10(ix) << 2) | (spread10(iy) << 1) | spread10(iz);
  vals[f] = f;
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

// Length of the common prefix of sorted keys i and j (index bits break ties).
__device__ inline int prefix(const uint32_t* __restrict__ k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint32_t a = k[i], b = k[j];
  if (a != b) return __clz(a ^ b);
  return 32 + __clz((uint32_t)(i ^ j));
}

__global__ void k_karras(const uint32_t* __restrict__ keys, int n, Node* nodes, int32_t* parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  // direction of the range covered by node i
  int d = (prefix(keys, n, i, i + 1) - prefix(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = prefix(keys, n, i, i - d);
  int lmax = 2;
  while (prefix(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (prefix(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = prefix(keys, n, i, j);
  // split: last index sharing more than dnode bits with i
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (prefix(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int g = i + s * d + (d < 0 ? -1 : 0);
  int lo = min(i, j), hi = max(i, j);
  int left = (lo == g) ? ~g : g;
  int right = (hi == g + 1) ? ~(g + 1) : g + 1;
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

inline int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

size_t layout(sbr_scene* s, void* mem, int32_t nt) {
  Carver c(mem);
  int64_t n = nt > 0 ? nt : 1;
  int64_t ni = n > 1 ? n - 1 : 1;
  s->tris = c.take<float4>(3 * n);
  s->nodes = c.take<Node>(ni);
  s->parent = c.take<int32_t>(2 * n);
  s->visits = c.take<uint32_t>(ni);
  s->keys[0] = c.take<uint32_t>(n);
  s->keys[1] = c.take<uint32_t>(n);
  s->vals[0] = c.take<int32_t>(n);
  s->vals[1] = c.take<int32_t>(n);
  s->faces = c.take<int32_t>(3 * n);
  s->bounds = c.take<int32_t>(8);
  s->err = c.take<int32_t>(1);
  s->sort_scratch = c.take<char>(sort_scratch_bytes(n));
  return c.bytes();
}

sbr_status rebuild(sbr_scene* s, const float* verts, cudaStream_t st) {
  const int nt = s->nt, nv = s->nv;
  ::sbr::note_launch();
  k_init_bounds<<<1, 32, 0, st>>>(s->bounds, s->err);
  if (nt == 0) {
    SBR_CUDA(cudaGetLastError());
    return SBR_OK;
  }
  ::sbr::note_launch();
  k_bounds<<<blocks(nt, 256), 256, 0, st>>>(verts, nv, s->faces, nt, s->bounds, s->err);
  ::sbr::note_launch();
  k_morton<<<blocks(nt, 256), 256, 0, st>>>(verts, nv, s->faces, nt, s->bounds, s->keys[0],
                                            s->vals[0], s->err);
  SBR_CUDA(radix_sort_pairs(s->keys, s->vals, nt, nullptr, 31, s->sort_scratch, st));
  ::sbr::note_launch();
  k_pack<<<blocks(nt, 256), 256, 0, st>>>(verts, nv, s->faces, nt, s->vals[0], s->tris, s->err);
  if (nt > 1) {
    ::sbr::note_launch();
    k_karras<<<blocks(nt - 1, 256), 256, 0, st>>>(s->keys[0], nt, s->nodes, s->parent);
    SBR_CUDA(cudaMemsetAsync(s->visits, 0, sizeof(uint32_t) * (nt - 1), st));
    ::sbr::note_launch();
    k_refit<<<blocks(nt, 256), 256, 0, st>>>(s->tris, nt, s->nodes, s->parent, s->visits,
                                             s->bounds);
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

extern "C" sbr_status sbr_scene_check(const sbr_scene* scene, sbr_stream stream) {
  SBR_ARG(scene != nullptr, "sbr_scene_check: scene is NULL");
  int32_t err = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SBR_CUDA(cudaMemcpyAsync(&err, scene->err, sizeof(err), cudaMemcpyDeviceToHost, st));
  SBR_CUDA(cudaStreamSynchronize(st));
  SBR_ARG(err == 0, "sbr_scene: face index outside [0, nv) (error word %d)", err);
  return SBR_OK;
}

extern "C" void sbr_scene_destroy(sbr_scene* scene) { free(scene); }
