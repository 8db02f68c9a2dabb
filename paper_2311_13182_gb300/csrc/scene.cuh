// Scene layout shared by the LBVH builder, the traversal and the trace adjoint.
#pragma once

#include "common.cuh"

namespace sbr {

// BVH2 node with both child boxes stored in the parent (64 B, four float4
// loads).  child >= 0: internal node index; child < 0: leaf ~child = position
// of the triangle in sorted (Morton) order.
struct __align__(16) Node {
  float4 lxy;   // left  lo.x hi.x lo.y hi.y
  float4 rxy;   // right lo.x hi.x lo.y hi.y
  float4 lrz;   // left lo.z hi.z, right lo.z hi.z
  int4 child;   // left, right, unused, unused
};

// 4-wide node for the traversal, collapsed from the binary tree: the entry of
// binary node i holds i's grandchildren (a leaf child stands for itself), then
// the largest internal slot is expanded while a slot is free.  child >= 0:
// internal binary node (its own 4-wide entry); kEmpty: unused slot; otherwise a
// leaf ~slot.  Boxes per axis as float4 over the four slots (112 of 128 bytes).
constexpr int kEmpty = (int)0x80000000;
struct __align__(128) Node4 {
  float4 lox, hix, loy, hiy, loz, hiz;
  int4 child;
  int4 pad;
};

// Shared-memory staging of the top levels of the 4-wide tree: the scene build
// copies the entries of the first kTopLevels levels, breadth first, into a
// table whose links to other staged entries read kStaged + position; every
// trace CTA loads the table into shared memory once.  pad.y of a staged entry
// holds its index in the full tree.  kTopLevels = 0 turns the staging off.
#ifndef SBR_TRACE_TOP_LEVELS
#define SBR_TRACE_TOP_LEVELS 0
#endif
constexpr int kTopLevels = SBR_TRACE_TOP_LEVELS;
constexpr int kTopMax = kTopLevels == 0 ? 1 : ((1 << (2 * kTopLevels)) - 1) / 3;  // 1 + 4 + 16 + ...
constexpr int kStaged = 1 << 30;  // above any node index (nt <= 2^26)

}  // namespace sbr

struct sbr_scene {
  int32_t nv, nt;
  float4* tris;        // [nt*3] sorted: (v0, original id bits), (v1, 0), (v2, 0)
  sbr::Node* nodes;    // [max(nt-1, 1)] binary tree
  sbr::Node4* nodes4;  // [max(nt-1, 1)] 4-wide entries, indexed like the binary nodes
  sbr::Node4* top;     // [kTopMax] breadth-first copy of the top levels (staging), count in top_n
  int32_t* top_n;      // [1]
  int32_t* parent;     // [2nt-1]: internal 0..nt-2, leaves nt-1..2nt-2
  uint32_t* visits;    // [max(nt-1,1)] refit arrival counters, or the crossing-node mask
  uint32_t* keys[2];   // [nt] Morton codes (sort ping-pong)
  int32_t* vals[2];    // [nt] triangle ids (sort ping-pong)
  int32_t* faces;      // [nt*3] copy of the topology
  int32_t* bounds;     // [8] centroid box as ordered ints + pad
  int32_t* err;        // [1] device error word (bit 0: face index out of range)
  uint32_t* hist;      // [4*256] Morton key digit counts (8-bit places) for the sort
  uint32_t* done;      // [1] CTAs of the cooperative build that have finished the tree
  uint32_t* bar;       // [2] grid barrier of the cooperative build: arrivals, generation
  uint32_t* tile_hist; // [3][tiles*256] per-tile digit counts of the cooperative sort (pass p: p % 3)
  int coop;            // build with one cooperative launch (all tiles resident at once)
  int cluster;         // ... launched as one thread-block cluster (at most 16 tiles): hardware barriers
  void* sort_scratch;
  size_t bytes;
  // materials (sbr_scene_set_materials): 0 = perfect conductors everywhere
  int n_mat;
  const int32_t* tri_mat;  // caller's device [nt] or NULL (all material 0)
  float eps_re[SBR_MAX_MATERIALS], eps_im[SBR_MAX_MATERIALS];
  // object motion (sbr_scene_set_motion): 0 = static
  int n_obj;
  const int32_t* tri_obj;  // caller's device [nt] or NULL (all object 0)
  float vel[SBR_MAX_OBJECTS][3];
};

namespace sbr {
// Materials as a kernel argument (by value).
struct MatArg {
  int n;
  const int32_t* tri_mat;
  float2 eps[SBR_MAX_MATERIALS];  // (eps_re, eps_im), eps = eps_re - j eps_im; eps_re <= 0: conductor
};

inline MatArg mat_arg(const sbr_scene* s) {
  MatArg m{};
  m.n = s->n_mat;
  m.tri_mat = s->tri_mat;
  for (int i = 0; i < SBR_MAX_MATERIALS; ++i) m.eps[i] = make_float2(s->eps_re[i], s->eps_im[i]);
  return m;
}

__device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline float2 cdiv(float2 a, float2 b) {
  const float d = 1.f / (b.x * b.x + b.y * b.y);
  return make_float2((a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d);
}
// principal square root (Re >= 0)
__device__ inline float2 csqrt(float2 z) {
  const float r = hypotf(z.x, z.y);
  const float re = sqrtf(fmaxf(0.5f * (r + z.x), 0.f));
  const float im = sqrtf(fmaxf(0.5f * (r - z.x), 0.f));
  return make_float2(re, z.y < 0.f ? -im : im);
}

// Object motion as a kernel argument (by value).
struct MotionArg {
  int n;
  const int32_t* tri_obj;
  float3 vel[SBR_MAX_OBJECTS];
};

inline MotionArg motion_arg(const sbr_scene* s) {
  MotionArg m{};
  m.n = s->n_obj;
  m.tri_obj = s->tri_obj;
  for (int i = 0; i < SBR_MAX_OBJECTS; ++i) m.vel[i] = make_float3(s->vel[i][0], s->vel[i][1], s->vel[i][2]);
  return m;
}

__device__ inline float3 velocity_of(const MotionArg& m, int id) {
  int k = m.tri_obj ? m.tri_obj[id] : 0;
  k = k < 0 ? 0 : (k >= m.n ? m.n - 1 : k);
  return m.vel[k];
}

// Material of triangle `id` (original index), clamped into the table.
__device__ inline int material_of(const MatArg& m, int id) {
  if (!m.tri_mat) return 0;
  const int k = m.tri_mat[id];
  return k < 0 ? 0 : (k >= m.n ? m.n - 1 : k);
}

// Fresnel r_s for incidence cosine c on material e; w = sqrt(eps - 1 + c^2) is returned
// for the adjoint (d log r_s / dc = -2 / w, d log r_s / d eps = c / (w (eps - 1))).
__device__ inline float2 fresnel_rs(float c, float2 e, float2* w_out) {
  const float2 eps = make_float2(e.x, -e.y);
  const float2 w = csqrt(make_float2(eps.x - 1.f + c * c, eps.y));
  if (w_out) *w_out = w;
  return cdiv(make_float2(c - w.x, -w.y), make_float2(c + w.x, w.y));
}
}  // namespace sbr
