// Ray tracing with specular bounces (Section 3.2.1, Eq. 2-3) and path preparation.
//
// One thread per ray.  The ray is carried in float-float (ff.cuh): its FP32 hi
// parts drive a stack traversal of the 4-wide BVH collapsed from the LBVH (a
// node's four child boxes and links as seven float4 loads, triangles as three
// float4 loads) with the Moller-Trumbore (1997) test.  Every
// FP32 decision carries a forward error bound: a triangle is accepted or
// rejected in FP32 only when the bound says exact arithmetic on the exact ray
// would decide the same; otherwise the test is repeated in float-float
// (signs of float-float numerators, ~1e-14 relative).  Nearest-hit ordering is
// decided the same way (interval overlap -> float-float t, exact ties -> lower
// triangle index).  The chosen hit of each bounce is then
// refined in float-float (plane intersection of the exact triangle) and the ray
// is reflected in float-float, so the triangle sequence is that of an FP64
// brute-force search for every ray not within rounding distance of an edge,
// without the FP64 pipe (a small fraction of the FP32 rate on GB300) on the
// per-ray path.
//
// Path preparation (float-float, O(paths x antennas)): per hit k and virtual
// antenna (t, r): L_in = |h_1 - Tx_t| + sum_{j=2..k} |h_j - h_{j-1}|,
// L_out = |Rx_r - h_k|, L = L_in + L_out, tau = L / c; phi0 = frac(f_c tau),
// delta = frac(B tau / N_s) split into delta_hi (a multiple of 2^-12, so
// n * delta_hi is exact in FP32 for n < 4096) and delta_lo; and
// A = omega (-1)^(k-1) |d_k . n_k| / (4 pi L_in L_out).
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "ff.cuh"
#include "scene.cuh"

namespace sbr {
namespace {

struct GridArg {
  ff o[3], ax[3], ua[3], va[3];
  ff start;    // -tan_half + tan_half / G: the first cell centre
  ff step;     // 2 tan_half / G: the cell pitch
  ff lo;       // -tan_half: the first cell's edge (jittered sampling)
  float cell;  // 2 tan_half / G
  int G;
  const float* jitter;  // [G*G][2] offsets in the cell, or NULL (cell centres)
};

struct RadarArg {
  ff tx[SBR_MAX_TX][3];
  ff rx[SBR_MAX_RX][3];
  ff k0;  // f_c / c         [cycles per metre]
  ff kb;  // B / (c N_s)     [cycles per sample per metre]
  int ntx, nrx;
};

constexpr float kTmin = 1e-9f;
constexpr float kErr = 1.0f / 262144.0f;  // 2^-18 = 64 ulp(1): scale of the FP32 error bounds

__device__ inline ff3 ff3_arr(const ff* a) { return ff3{a[0], a[1], a[2]}; }

// Launch direction of grid ray rid in float-float: cell centre
// a = tan_half (2 (col + 1/2) / G - 1) = start + col * step, likewise b with row,
// direction = normalize(axis + a u + b v).
__device__ inline ff3 grid_dir_ff(const GridArg& g, int rid) {
  const int row = rid / g.G, col = rid - row * g.G;
  ff a, b;
  if (g.jitter) {  // a = -tan_half + (col + jx) step, col + jx exact as a float-float sum
    const float2 j = reinterpret_cast<const float2*>(g.jitter)[rid];
    a = ff_add(g.lo, ff_mul(g.step, ff_add(ff_of((float)col), ff_of(j.x))));
    b = ff_add(g.lo, ff_mul(g.step, ff_add(ff_of((float)row), ff_of(j.y))));
  } else {
    a = ff_add(g.start, ff_mulf(g.step, (float)col));
    b = ff_add(g.start, ff_mulf(g.step, (float)row));
  }
  const ff3 w = ff3_add(ff3_arr(g.ax), ff3_add(ff3_scale(ff3_arr(g.ua), a), ff3_scale(ff3_arr(g.va), b)));
  return ff3_scale(w, ff_rsqrt(ff3_dot(w, w)));
}

// The same direction in FP32 (a few ulp; the traversal's error bounds allow
// 64) and the ray's solid-angle weight cell^2 cos^3.
__device__ inline float3 grid_dir_f32(const GridArg& g, int rid, float& omega) {
  const int row = rid / g.G, col = rid - row * g.G;
  float a, b;
  if (g.jitter) {
    const float2 j = reinterpret_cast<const float2*>(g.jitter)[rid];
    a = fmaf(g.step.hi, (float)col + j.x, g.lo.hi);
    b = fmaf(g.step.hi, (float)row + j.y, g.lo.hi);
  } else {
    a = fmaf(g.step.hi, (float)col, g.start.hi);
    b = fmaf(g.step.hi, (float)row, g.start.hi);
  }
  const float3 w = f3(g.ax[0].hi + a * g.ua[0].hi + b * g.va[0].hi, g.ax[1].hi + a * g.ua[1].hi + b * g.va[1].hi,
                      g.ax[2].hi + a * g.ua[2].hi + b * g.va[2].hi);
  const float inv = rsqrtf(dot(w, w));
  omega = g.cell * g.cell * inv * inv * inv;
  return w * inv;
}

__device__ inline float3 tri_vert(const float4* __restrict__ tris, int slot, int c) {
  const float4 v = __ldg(&tris[3 * slot + c]);
  return f3(v.x, v.y, v.z);
}

__device__ inline bool ff_less(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

struct Best {
  int id, slot;
  float lo, hi;  // interval containing the exact distance
  bool exact;
  ff t;          // float-float distance when exact
};

struct Ray {
  // float-float ray (d valid once has_ff)
  ff3& o;
  ff3& d;
  __device__ Ray(ff3& o_, ff3& d_) : o(o_), d(d_) {}
  float3 of, df;  // FP32 ray driving the traversal
  float3 idir;
  int near;  // byte offsets of a 4-wide entry's near-plane rows, x | y << 8 | z << 16 (set_idir)
  int skip;
  bool has_ff;        // primary rays build d in float-float only when needed
  int rid;
  const GridArg* g;
};

__device__ inline void ensure_ff(Ray& r) {
  if (!r.has_ff) {
    r.d = grid_dir_ff(*r.g, r.rid);
    r.has_ff = true;
  }
}

// Moller-Trumbore in float-float on the float-float ray: the same two-sided
// rule as the FP64 definition (|det| < 1e-12 misses; 0 <= u, v; u + v <= 1;
// t > 1e-9), decided on signs of float-float numerators (about 1e-14 relative),
// which agree with FP64 except within rounding distance of an edge or tie.
__device__ inline bool exact_t(const float4* __restrict__ tris, Ray& r, int slot, ff& t) {
  ensure_ff(r);
  const float3 a = tri_vert(tris, slot, 0), b = tri_vert(tris, slot, 1), c = tri_vert(tris, slot, 2);
  const ff3 e1 = ff3_diff(b, a), e2 = ff3_diff(c, a);
  const ff3 p = ff3_cross(r.d, e2);
  const ff det = ff3_dot(e1, p);
  if (fabsf(det.hi) < 1e-12f) return false;
  const float sg = det.hi > 0.f ? 1.f : -1.f;
  const ff adet = ff{det.hi * sg, det.lo * sg};
  const ff3 s = ff3_sub(r.o, ff3_of(a));
  ff un = ff3_dot(s, p);
  un = ff{un.hi * sg, un.lo * sg};
  if (un.hi < 0.f || ff_sub(adet, un).hi < 0.f) return false;        // u < 0 or u > 1
  const ff3 q = ff3_cross(s, e1);
  ff vn = ff3_dot(r.d, q);
  vn = ff{vn.hi * sg, vn.lo * sg};
  if (vn.hi < 0.f || ff_sub(adet, ff_add(un, vn)).hi < 0.f) return false;  // v < 0 or u + v > 1
  t = ff_div(ff3_dot(e2, q), det);
  return ff_sub(t, ff_of(kTmin)).hi > 0.f;
}

__device__ inline void take_exact(Best& b, int id, int slot, ff t) {
  b.id = id;
  b.slot = slot;
  b.exact = true;
  b.t = t;
  b.lo = t.hi - fabsf(t.hi) * 2.4e-7f;
  b.hi = t.hi + fabsf(t.hi) * 2.4e-7f;
}

// Offer a candidate whose exact distance lies in [lo, hi] (exact: t known).
__device__ inline void consider(Best& b, const float4* __restrict__ tris, Ray& r, int id,
                                int slot, float lo, float hi, bool exact, ff t) {
  if (b.id < 0 || hi < b.lo) {
    if (exact) take_exact(b, id, slot, t);
    else {
      b.id = id; b.slot = slot; b.lo = lo; b.hi = hi; b.exact = false;
    }
    return;
  }
  if (lo > b.hi) return;
  // overlapping intervals: order in float-float, ties to the lower triangle index
  if (!exact && !exact_t(tris, r, slot, t)) return;
  if (!b.exact) {
    ff tb;
    if (!exact_t(tris, r, b.slot, tb)) {  // cannot happen with valid bounds; keep the new one
      take_exact(b, id, slot, t);
      return;
    }
    take_exact(b, b.id, b.slot, tb);
  }
  if (ff_less(t, b.t) || (t.hi == b.t.hi && t.lo == b.t.lo && id < b.id)) take_exact(b, id, slot, t);
}

__device__ inline void test_tri(Best& b, const float4* __restrict__ tris, Ray& r, int slot) {
  const float4 A = __ldg(&tris[3 * slot]);
  const int id = __float_as_int(A.w);
  if (id == r.skip) return;
  const float4 B = __ldg(&tris[3 * slot + 1]);
  const float4 C = __ldg(&tris[3 * slot + 2]);
  const float3 v0 = f3(A.x, A.y, A.z);
  const float3 e1 = f3(B.x, B.y, B.z) - v0;
  const float3 e2 = f3(C.x, C.y, C.z) - v0;
  const float3 p = cross(r.df, e2);
  const float det = dot(e1, p);
  const float3 s = r.of - v0;
  const float3 q = cross(s, e1);
  const float un = dot(s, p), vn = dot(r.df, q), tn = dot(e2, q);
  // forward error bounds of the FP32 values against FP64 arithmetic on the exact ray
  const float m1 = l1(e1), m2 = l1(e2), ms = l1(r.of) + l1(v0);
  const float edet = kErr * m1 * m2;
  const float eu = kErr * ms * m2, ev = kErr * ms * m1, et = kErr * ms * m1 * m2;
  const float adet = fabsf(det);
  bool ambiguous = adet <= edet * 1.0001f + 1.01e-12f;
  if (!ambiguous) {
    const float sg = det > 0.f ? 1.f : -1.f;
    const float su = un * sg, sv = vn * sg, st = tn * sg;
    const float sw = adet - su - sv;
    const float ew = edet + eu + ev + kErr * adet;
    if (su < -eu || sv < -ev || sw < -ew) return;  // outside in FP64 as well
    const float nlo = st - et, nhi = st + et;
    // approximate quotients (<= 2 ulp); the 6e-7 relative pad keeps the interval valid
    float lo = __fdividef(nlo, nlo >= 0.f ? adet + edet : adet - edet);
    float hi = __fdividef(nhi, nhi >= 0.f ? adet - edet : adet + edet);
    lo -= fabsf(lo) * 6e-7f;
    hi += fabsf(hi) * 6e-7f;
    if (hi <= kTmin) return;                      // behind the origin in FP64 too
    if (b.id >= 0 && lo > b.hi) return;           // farther than the current hit
    if (su > eu && sv > ev && sw > ew && lo > kTmin) {
      consider(b, tris, r, id, slot, lo, hi, false, ff_of(0.f));
      return;
    }
  }
  ff t;
  if (exact_t(tris, r, slot, t))
    consider(b, tris, r, id, slot, t.hi - fabsf(t.hi) * 2.4e-7f, t.hi + fabsf(t.hi) * 2.4e-7f, true, t);
}

// Entry and exit distances of a padded box from its planes along the ray: nx,
// ny, nz the planes entered first (per axis the lower bound when the direction
// component is positive, else the upper one), fx, fy, fz the planes left last;
// tn the largest entry, tf the smallest exit.  t = p idir - o idir, one FMA per
// plane: rounding o idir moves a plane by at most 2^-24 |o| along its axis, and
// the final rounding by 2^-24 |p - o|; both stay far inside the box pads
// (2^-18 (1 + max |coord|)) for origins within the scene's coordinate range.
// An FMA is monotone in the plane, so for lo <= hi the chosen planes give the
// min and max of each axis's pair; an unused slot is rejected by its link.
__device__ inline void slab_nf(const float3& o, const float3& idir, float nx, float fx, float ny, float fy,
                               float nz, float fz, float& tn, float& tf) {
  const float ax = -(o.x * idir.x), ay = -(o.y * idir.y), az = -(o.z * idir.z);
  tn = fmaxf(fmaxf(fmaf(nx, idir.x, ax), fmaf(ny, idir.y, ay)), fmaf(nz, idir.z, az));
  tf = fminf(fminf(fmaf(fx, idir.x, ax), fmaf(fy, idir.y, ay)), fmaf(fz, idir.z, az));
  tf = tf * 1.0000005f + 1e-30f;
}

// A 4-wide entry's boxes as the ray meets them: per axis the plane entered first
// (the lower bound when the direction component is positive, else the upper
// one) and the plane left last, one float4 over the four slots each.  Entries
// are 128-byte aligned, so a near row's byte offset (Ray::near) is OR-ed
// into the entry's address, and the far row is the near one with bit 4 flipped.
struct Planes4 {
  float4 nx, fx, ny, fy, nz, fz;
};

static_assert(offsetof(Node4, lox) == 0 && offsetof(Node4, hix) == 16 && offsetof(Node4, loy) == 32 &&
                  offsetof(Node4, hiy) == 48 && offsetof(Node4, loz) == 64 && offsetof(Node4, hiz) == 80 &&
                  alignof(Node4) == 128,
              "near/far plane rows assume this entry layout");

template <bool kGlobal>
__device__ inline float4 plane_row(const void* q, int off) {
  const float4* a = reinterpret_cast<const float4*>(reinterpret_cast<uintptr_t>(q) | (uintptr_t)(unsigned)off);
  return kGlobal ? __ldg(a) : *a;
}

template <bool kGlobal = true>
__device__ inline Planes4 load_planes(const void* q, int near) {
  const int nxo = near & 0xff, nyo = (near >> 8) & 0xff, nzo = near >> 16;
  Planes4 p;
  p.nx = plane_row<kGlobal>(q, nxo);
  p.fx = plane_row<kGlobal>(q, nxo ^ 16);
  p.ny = plane_row<kGlobal>(q, nyo);
  p.fy = plane_row<kGlobal>(q, nyo ^ 16);
  p.nz = plane_row<kGlobal>(q, nzo);
  p.fz = plane_row<kGlobal>(q, nzo ^ 16);
  return p;
}

constexpr int kStack = 192;  // 3 pending siblings per 4-wide level, 64 binary levels at most

// Order of a node's children on the stack: 2 = fully sorted by entry distance
// (a 5-exchange network), 1 = nearest child first, the other three partly ordered.
#ifndef SBR_TRACE_SORT
#define SBR_TRACE_SORT 2
#endif

// compare-exchange of (distance, child) pairs
__device__ inline void cswap(float& da, int& ca, float& db, int& cb) {
  if (db < da) {
    const float td = da;
    da = db;
    db = td;
    const int tc = ca;
    ca = cb;
    cb = tc;
  }
}

__device__ inline ff ff3_at(const ff3& v, int j) { return j == 0 ? v.x : (j == 1 ? v.y : v.z); }

// Traversals that run past kStragglerSteps entries (rays grazing a surface
// after a bounce: hundreds of node and triangle tests) would keep their whole
// CTA resident long after the other lanes finished, and decide the launch's
// length.  Such a ray is handed over, with everything needed to resume it, to
// k_trace_coop, where the 32 lanes of a warp finish it together.
constexpr int kStragglerSteps = 128;
constexpr int kDumpStack = 64;
constexpr int kDumpMax = 8192;
struct __align__(16) RayDump {
  int slot, rid, k, nh;
  int skip, has_ff, node, sp;
  float o[6], d[6];  // float-float origin and direction: (hi, lo) per axis
  int bid, bslot, bexact, pad;
  float blo, bhi, bt_hi, bt_lo;
  int stack[kDumpStack];
};

// Where a lane hands its ray over, and the ray's output slot and bounce.
struct DumpCtx {
  RayDump* dumps;
  unsigned int* n;
  int slot, k, nh;
};

constexpr int kHanded = -2;  // Best::id of a ray handed over

// Records a straggler's state; false when the hand-over area is full (the
// lane then finishes the ray itself).  Out of line: it runs for few rays.
__shared__ Node4 s_top[kTopMax];  // staged top levels (k_trace only)

// Full-tree index of a traversal entry (staged entries carry theirs in pad.y).
__device__ inline int unstage(int e) { return (kTopLevels > 0 && e >= kStaged) ? s_top[e - kStaged].pad.y : e; }

__device__ __noinline__ bool hand_over(DumpCtx dc, ff3 o, ff3 d, int rid, int skip, bool has_ff, Best b, int node,
                                       const int* stack, int sp) {
  const unsigned di = atomicAdd(dc.n, 1u);
  if (di >= (unsigned)kDumpMax) return false;
  RayDump& D = dc.dumps[di];
  D.slot = dc.slot;
  D.rid = rid;
  D.k = dc.k;
  D.nh = dc.nh;
  D.skip = skip;
  D.has_ff = has_ff;
  D.node = unstage(node);
  D.sp = sp;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const ff oj = ff3_at(o, j), dj = ff3_at(d, j);
    D.o[2 * j] = oj.hi;
    D.o[2 * j + 1] = oj.lo;
    D.d[2 * j] = has_ff ? dj.hi : 0.f;
    D.d[2 * j + 1] = has_ff ? dj.lo : 0.f;
  }
  D.bid = b.id;
  D.bslot = b.slot;
  D.bexact = b.exact;
  D.blo = b.lo;
  D.bhi = b.hi;
  D.bt_hi = b.t.hi;
  D.bt_lo = b.t.lo;
  for (int j = 0; j < sp; ++j) D.stack[j] = unstage(stack[j]);
  return true;
}

// Nearest hit through the 4-wide tree: children whose padded boxes the ray
// enters before the current hit's far bound are visited nearest first.
// kCount: also count the nodes and triangles fetched (the roofline's bytes).
template <bool kCount>
__device__ Best nearest(const float4* __restrict__ tris, const Node4* __restrict__ nodes, int nt,
                        Ray& r, int& n_nodes, int& n_tris, const DumpCtx* dc) {
  Best b;
  b.id = -1;
  b.slot = -1;
  b.lo = b.hi = INFINITY;
  b.exact = false;
  b.t = ff_of(0.f);
  if (nt <= 0) return b;
  int stack[kStack];
  int sp = 0;
  int node = nt > 1 ? (kTopLevels > 0 ? kStaged : 0) : ~0;
  // a valid tree is visited at most once per node: the cap only guards
  // against a corrupted hierarchy turning into an endless loop
  const int hand_at = 2 * nt + 64 - kStragglerSteps;  // the guard's value after kStragglerSteps entries
  for (int guard = 2 * nt + 64; guard > 0; --guard) {
    if (guard == hand_at && dc && sp <= kDumpStack &&
        hand_over(*dc, r.o, r.d, r.rid, r.skip, r.has_ff, b, node, stack, sp)) {
      b.id = kHanded;
      return b;
    }
    if (node >= 0) {
      if (kCount) ++n_nodes;
      Planes4 p;
      int4 ch;
      if (kTopLevels > 0 && node >= kStaged) {
        const Node4& q = s_top[node - kStaged];
        p = load_planes<false>(&q, r.near);
        ch = q.child;
      } else {
        const Node4* q = nodes + node;
        p = load_planes(q, r.near);
        ch = __ldg(&q->child);
      }
      const float lim = b.hi;
      float d0, d1, d2, d3, tf;
      int c0 = ch.x, c1 = ch.y, c2 = ch.z, c3 = ch.w;
      slab_nf(r.of, r.idir, p.nx.x, p.fx.x, p.ny.x, p.fy.x, p.nz.x, p.fz.x, d0, tf);
      d0 = (c0 != kEmpty && d0 <= tf && tf >= 0.f && d0 <= lim) ? d0 : INFINITY;
      slab_nf(r.of, r.idir, p.nx.y, p.fx.y, p.ny.y, p.fy.y, p.nz.y, p.fz.y, d1, tf);
      d1 = (c1 != kEmpty && d1 <= tf && tf >= 0.f && d1 <= lim) ? d1 : INFINITY;
      slab_nf(r.of, r.idir, p.nx.z, p.fx.z, p.ny.z, p.fy.z, p.nz.z, p.fz.z, d2, tf);
      d2 = (c2 != kEmpty && d2 <= tf && tf >= 0.f && d2 <= lim) ? d2 : INFINITY;
      slab_nf(r.of, r.idir, p.nx.w, p.fx.w, p.ny.w, p.fy.w, p.nz.w, p.fz.w, d3, tf);
      d3 = (c3 != kEmpty && d3 <= tf && tf >= 0.f && d3 <= lim) ? d3 : INFINITY;
      // sort the four entry distances (misses are +inf and sink to the end)
      cswap(d0, c0, d1, c1);
      cswap(d2, c2, d3, c3);
      cswap(d0, c0, d2, c2);
      if (SBR_TRACE_SORT > 1) {  // else: nearest child first, the others in a partial order
        cswap(d1, c1, d3, c3);
        cswap(d1, c1, d2, c2);
      }
      if (d0 < INFINITY) {
        if (d3 < INFINITY && sp < kStack) stack[sp++] = c3;
        if (d2 < INFINITY && sp < kStack) stack[sp++] = c2;
        if (d1 < INFINITY && sp < kStack) stack[sp++] = c1;
        node = c0;
        continue;
      }
    } else {
      if (kCount) ++n_tris;
      test_tri(b, tris, r, ~node);
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return b;
}

__device__ inline void init_best(Best& b) {
  b.id = -1;
  b.slot = -1;
  b.lo = b.hi = INFINITY;
  b.exact = false;
  b.t = ff_of(0.f);
}

// Resumable traversal for k_trace_coop: the next entry (>= 0 internal node,
// < 0 leaf ~slot) and the pending ones on `stack`.  Processes at most `budget`
// entries and returns true once the traversal is complete.  ext_lim: a far
// bound another lane holds for the same ray (pruning only).
template <bool kCount>
__device__ bool traverse(const float4* __restrict__ tris, const Node4* __restrict__ nodes, int nt, Ray& r,
                         Best& b, int* stack, int& sp, int& node, int& steps, int budget, float ext_lim,
                         int& n_nodes, int& n_tris) {
  if (nt <= 0) return true;
  const int guard = 2 * nt + 64;  // a valid tree is visited at most once per node
  for (; budget > 0; --budget) {
    if (++steps > guard) return true;
    if (node >= 0) {
      if (kCount) ++n_nodes;
      const Node4* q = nodes + node;
      const Planes4 p = load_planes(q, r.near);
      const int4 ch = __ldg(&q->child);
      const float lim = fminf(b.hi, ext_lim);
      float d0, d1, d2, d3, tf;
      int c0 = ch.x, c1 = ch.y, c2 = ch.z, c3 = ch.w;
      slab_nf(r.of, r.idir, p.nx.x, p.fx.x, p.ny.x, p.fy.x, p.nz.x, p.fz.x, d0, tf);
      d0 = (c0 != kEmpty && d0 <= tf && tf >= 0.f && d0 <= lim) ? d0 : INFINITY;
      slab_nf(r.of, r.idir, p.nx.y, p.fx.y, p.ny.y, p.fy.y, p.nz.y, p.fz.y, d1, tf);
      d1 = (c1 != kEmpty && d1 <= tf && tf >= 0.f && d1 <= lim) ? d1 : INFINITY;
      slab_nf(r.of, r.idir, p.nx.z, p.fx.z, p.ny.z, p.fy.z, p.nz.z, p.fz.z, d2, tf);
      d2 = (c2 != kEmpty && d2 <= tf && tf >= 0.f && d2 <= lim) ? d2 : INFINITY;
      slab_nf(r.of, r.idir, p.nx.w, p.fx.w, p.ny.w, p.fy.w, p.nz.w, p.fz.w, d3, tf);
      d3 = (c3 != kEmpty && d3 <= tf && tf >= 0.f && d3 <= lim) ? d3 : INFINITY;
      cswap(d0, c0, d1, c1);
      cswap(d2, c2, d3, c3);
      cswap(d0, c0, d2, c2);
      cswap(d1, c1, d3, c3);
      cswap(d1, c1, d2, c2);
      if (d0 < INFINITY) {
        if (d3 < INFINITY && sp < kStack) stack[sp++] = c3;
        if (d2 < INFINITY && sp < kStack) stack[sp++] = c2;
        if (d1 < INFINITY && sp < kStack) stack[sp++] = c1;
        node = c0;
        continue;
      }
    } else {
      if (kCount) ++n_tris;
      test_tri(b, tris, r, ~node);
    }
    if (sp == 0) return true;
    node = stack[--sp];
  }
  return false;
}

__device__ inline void set_idir(Ray& r) {
  auto inv = [](float x) { return 1.0f / (fabsf(x) < 1e-20f ? copysignf(1e-20f, x) : x); };
  r.idir = f3(inv(r.df.x), inv(r.df.y), inv(r.df.z));
  // near rows: lo (bytes 0, 32, 64 of the entry) for a positive component, hi (16, 48, 80) otherwise
  r.near = (__float_as_int(r.idir.x) < 0 ? 16 : 0) | (__float_as_int(r.idir.y) < 0 ? 48 : 32) << 8 |
           (__float_as_int(r.idir.z) < 0 ? 80 : 64) << 16;
}

__device__ inline void set_f32(Ray& r) {
  r.of = ff3_hi(r.o);
  r.df = ff3_hi(r.d);
  set_idir(r);
}

// barycentrics of the hit (reported, not used downstream), FP32
__device__ inline void bary(const Ray& r, float3 a, float3 b, float3 c, float& u, float& v) {
  const float3 e1 = b - a, e2 = c - a, p = cross(r.df, e2);
  const float inv = 1.f / dot(e1, p);
  const float3 s = r.of - a;
  u = dot(s, p) * inv;
  v = dot(r.df, cross(s, e1)) * inv;
}

#ifndef SBR_TRACE_MIN_BLOCKS
#define SBR_TRACE_MIN_BLOCKS 6  // resident 128-thread CTAs per SM the register budget targets
#endif

// Records k..K-1 of a ray that found nothing at bounce k.
__device__ inline void record_miss(sbr_hit* hits, float4* hit_pos, int slot, int k, int K) {
  for (int kk = k; kk < K; ++kk) {
    const size_t s2 = (size_t)slot * K + kk;
    hits[s2] = sbr_hit{-1, 0.f, 0.f, 0.f};
    hit_pos[2 * s2] = make_float4(0.f, 0.f, 0.f, 0.f);
    hit_pos[2 * s2 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Hit record k (written when `write`) from the ray's nearest triangle, refined
// in float-float on the plane of the exact triangle; the ray then continues
// from the hit point along d' = d - 2 (d.N) / (N.N) N.
__device__ inline void record_hit(const float4* __restrict__ tris, Ray& r, const Best& b, sbr_hit* hits,
                                  float4* hit_pos, size_t sl, bool write) {
  const float4 A = __ldg(&tris[3 * b.slot]), B = __ldg(&tris[3 * b.slot + 1]),
               C = __ldg(&tris[3 * b.slot + 2]);
  const float3 a = f3(A.x, A.y, A.z), bb = f3(B.x, B.y, B.z), c = f3(C.x, C.y, C.z);
  ensure_ff(r);
  const ff3 N = ff3_cross(ff3_diff(bb, a), ff3_diff(c, a));
  const ff den = ff3_dot(N, r.d);
  const ff t = ff_div(ff3_dot(N, ff3_sub(ff3_of(a), r.o)), den);
  const ff3 h = ff3_add(r.o, ff3_scale(r.d, t));
  const ff nn = ff3_dot(N, N);
  if (write) {
    const float cosv = fabsf(den.hi) * rsqrtf(nn.hi);
    float u, v;
    bary(r, a, bb, c, u, v);
    hits[sl] = sbr_hit{b.id, t.hi, u, v};
    hit_pos[2 * sl] = make_float4(h.x.hi, h.x.lo, h.y.hi, h.y.lo);
    hit_pos[2 * sl + 1] = make_float4(h.z.hi, h.z.lo, cosv, 0.f);
  }
  const ff f = ff_div(ff_mulf(den, 2.f), nn);
  r.d = ff3_sub(r.d, ff3_scale(N, f));
  r.o = h;
  r.skip = b.id;
  set_f32(r);
}

template <bool kCount>
__global__ void __launch_bounds__(128, SBR_TRACE_MIN_BLOCKS) k_trace(const float4* __restrict__ tris,
                                               const Node4* __restrict__ nodes, int nt, GridArg g,
                                               const int32_t* __restrict__ ray_ids, int n_rays,
                                               int K, sbr_hit* __restrict__ hits,
                                               float4* __restrict__ hit_pos,
                                               float* __restrict__ ray_w,
                                               int32_t* __restrict__ nvalid,
                                               RayDump* __restrict__ dumps, unsigned int* __restrict__ n_dumps,
                                               unsigned long long* __restrict__ counts,
                                               const Node4* __restrict__ top, const int32_t* __restrict__ top_n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int n_nodes = 0, n_tris = 0, n_trav = 0;
  if (kTopLevels > 0) {  // every thread of the CTA, before any may return
    const int n = *top_n;
    const float4* src = reinterpret_cast<const float4*>(top);
    float4* dst = reinterpret_cast<float4*>(s_top);
    for (int j = threadIdx.x; j < n * (int)(sizeof(Node4) / sizeof(float4)); j += blockDim.x) dst[j] = __ldg(&src[j]);
    __syncthreads();
  }
  if (kCount) {
    // whole warps stay to the reduction below; idle lanes count nothing
    if (i - (int)(threadIdx.x & 31) >= n_rays) return;
  } else if (i >= n_rays) {
    return;
  }
  if (i < n_rays) {
  const int rid = ray_ids ? ray_ids[i] : i;
  ff3 ray_o, ray_d;
  Ray r(ray_o, ray_d);
  float omega;
  r.g = &g;
  r.rid = rid;
  r.has_ff = false;
  r.o = ff3_arr(g.o);
  r.of = ff3_hi(r.o);
  r.df = grid_dir_f32(g, rid, omega);
  r.skip = -1;
  set_idir(r);
  ray_w[i] = omega;
  int nh = 0;
  bool handed = false;
  for (int k = 0; k < K; ++k) {
    const size_t sl = (size_t)i * K + k;
    if (kCount) ++n_trav;
    const DumpCtx dc{dumps, n_dumps, i, k, nh};
    Best b = nearest<kCount>(tris, nodes, nt, r, n_nodes, n_tris, &dc);
    if (b.id == kHanded) {  // k_trace_coop writes the rest of this ray
      handed = true;
      break;
    }
    if (b.id < 0) {
      for (int kk = k; kk < K; ++kk) {
        const size_t s2 = (size_t)i * K + kk;
        hits[s2] = sbr_hit{-1, 0.f, 0.f, 0.f};
        hit_pos[2 * s2] = make_float4(0.f, 0.f, 0.f, 0.f);
        hit_pos[2 * s2 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      break;
    }
    const float4 A = __ldg(&tris[3 * b.slot]), B = __ldg(&tris[3 * b.slot + 1]),
                 C = __ldg(&tris[3 * b.slot + 2]);
    const float3 a = f3(A.x, A.y, A.z), bb = f3(B.x, B.y, B.z), c = f3(C.x, C.y, C.z);
    // float-float refine: plane of the exact triangle, t = N.(a - o) / (N.d)
    ensure_ff(r);
    const ff3 N = ff3_cross(ff3_diff(bb, a), ff3_diff(c, a));
    const ff den = ff3_dot(N, r.d);
    const ff t = ff_div(ff3_dot(N, ff3_sub(ff3_of(a), r.o)), den);
    const ff3 h = ff3_add(r.o, ff3_scale(r.d, t));
    const ff nn = ff3_dot(N, N);
    const float cosv = fabsf(den.hi) * rsqrtf(nn.hi);
    float u, v;
    bary(r, a, bb, c, u, v);
    hits[sl] = sbr_hit{b.id, t.hi, u, v};
    hit_pos[2 * sl] = make_float4(h.x.hi, h.x.lo, h.y.hi, h.y.lo);
    hit_pos[2 * sl + 1] = make_float4(h.z.hi, h.z.lo, cosv, 0.f);
    // specular reflection d' = d - 2 (d.N) / (N.N) N, next origin = hit point
    const ff f = ff_div(ff_mulf(den, 2.f), nn);
    r.d = ff3_sub(r.d, ff3_scale(N, f));
    r.o = h;
    r.skip = b.id;
    set_f32(r);
    ++nh;
  }
  if (!handed) nvalid[i] = nh;
  }
  if (kCount) {
    for (int o = 16; o; o >>= 1) {
      n_nodes += __shfl_xor_sync(0xffffffffu, n_nodes, o);
      n_tris += __shfl_xor_sync(0xffffffffu, n_tris, o);
      n_trav += __shfl_xor_sync(0xffffffffu, n_trav, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&counts[0], (unsigned long long)n_nodes);
      atomicAdd(&counts[1], (unsigned long long)n_tris);
      atomicAdd(&counts[2], (unsigned long long)n_trav);
    }
  }
}

// ---- cooperative completion of straggler rays --------------------------------

constexpr int kCoopList = 128;  // per-warp work list: < 32 entries expanded 4-wide at most

__device__ inline float warp_min(float x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// All 32 lanes finish one ray's nearest-hit search.  The pending entries
// (list[0..cnt)) are first expanded breadth-first (an internal node is replaced
// by the children the ray enters before the current far bound) until there are
// at least 32, then dealt out to the lanes, which traverse their subtrees with
// private stacks and share the nearest far bound between rounds.  The lanes'
// candidates are merged by the rule every traversal applies (enclosing
// intervals, then float-float distance, then the lower triangle index), which
// orders candidates totally, so the result is that of one sequential traversal.
template <bool kCount>
__device__ Best coop_nearest(const float4* __restrict__ tris, const Node4* __restrict__ nodes, int nt, Ray& r,
                             Best b, int* list, int cnt, int& n_nodes, int& n_tris) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < 8 && cnt < 32; ++round) {
    const int e = lane < cnt ? list[lane] : 0;
    const bool expand = lane < cnt && e >= 0;
    int kid[4] = {0, 0, 0, 0}, nk = 0;
    if (lane < cnt && !expand) kid[nk++] = e;
    if (expand) {
      if (kCount) ++n_nodes;
      const Node4* q = nodes + e;
      const Planes4 p = load_planes(q, r.near);
      const int4 ch = __ldg(&q->child);
      float tn, tf;
      slab_nf(r.of, r.idir, p.nx.x, p.fx.x, p.ny.x, p.fy.x, p.nz.x, p.fz.x, tn, tf);
      if (ch.x != kEmpty && tn <= tf && tf >= 0.f && tn <= b.hi) kid[nk++] = ch.x;
      slab_nf(r.of, r.idir, p.nx.y, p.fx.y, p.ny.y, p.fy.y, p.nz.y, p.fz.y, tn, tf);
      if (ch.y != kEmpty && tn <= tf && tf >= 0.f && tn <= b.hi) kid[nk++] = ch.y;
      slab_nf(r.of, r.idir, p.nx.z, p.fx.z, p.ny.z, p.fy.z, p.nz.z, p.fz.z, tn, tf);
      if (ch.z != kEmpty && tn <= tf && tf >= 0.f && tn <= b.hi) kid[nk++] = ch.z;
      slab_nf(r.of, r.idir, p.nx.w, p.fx.w, p.ny.w, p.fy.w, p.nz.w, p.fz.w, tn, tf);
      if (ch.w != kEmpty && tn <= tf && tf >= 0.f && tn <= b.hi) kid[nk++] = ch.w;
    }
    if (!__any_sync(0xffffffffu, expand)) break;  // only leaves left
    int x = nk;  // inclusive scan of the entries each lane produces
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const int total = __shfl_sync(0xffffffffu, x, 31);  // <= 4 x 31 < kCoopList
    __syncwarp();  // every lane has read its entry
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < nk) list[x - nk + j] = kid[j];
    __syncwarp();
    cnt = total;
  }
  int stack[kStack];
  int sp = 0, node = 0, steps = 0;
  int mine[kCoopList / 32], nm = 0;
  for (int j = lane; j < cnt; j += 32) mine[nm++] = list[j];
  __syncwarp();  // the caller rewrites the list
  for (int m = nm - 1; m >= 1; --m) stack[sp++] = mine[m];
  bool done = nm == 0;
  if (!done) node = mine[0];
  float lim = warp_min(b.hi);
  while (__any_sync(0xffffffffu, !done)) {
    if (!done) done = traverse<kCount>(tris, nodes, nt, r, b, stack, sp, node, steps, 16, lim, n_nodes, n_tris);
    lim = warp_min(b.hi);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const int id = __shfl_xor_sync(0xffffffffu, b.id, o);
    const int slot = __shfl_xor_sync(0xffffffffu, b.slot, o);
    const float lo = __shfl_xor_sync(0xffffffffu, b.lo, o);
    const float hi = __shfl_xor_sync(0xffffffffu, b.hi, o);
    const int ex = __shfl_xor_sync(0xffffffffu, (int)b.exact, o);
    const float th = __shfl_xor_sync(0xffffffffu, b.t.hi, o);
    const float tl = __shfl_xor_sync(0xffffffffu, b.t.lo, o);
    if (id >= 0 && id != b.id) consider(b, tris, r, id, slot, lo, hi, ex != 0, ff{th, tl});
  }
  return b;
}

// One warp per handed-over ray: resumes its traversal, then makes its remaining
// bounces with cooperative traversals from the root.
template <bool kCount>
__global__ void __launch_bounds__(128) k_trace_coop(const float4* __restrict__ tris,
                                                    const Node4* __restrict__ nodes, int nt, GridArg g, int K,
                                                    const RayDump* __restrict__ dumps,
                                                    const unsigned int* __restrict__ n_dumps,
                                                    unsigned int* __restrict__ work, sbr_hit* __restrict__ hits,
                                                    float4* __restrict__ hit_pos, int32_t* __restrict__ nvalid,
                                                    unsigned long long* __restrict__ counts) {
  __shared__ int lists[4][kCoopList];
  const int lane = threadIdx.x & 31;
  int* list = lists[threadIdx.x >> 5];
  int n_nodes = 0, n_tris = 0, n_trav = 0;
  const unsigned n = min(*n_dumps, (unsigned)kDumpMax);
  for (;;) {
    unsigned idx = 0;
    if (lane == 0) idx = atomicAdd(work, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= n) break;
    const RayDump& D = dumps[idx];
    ff3 ray_o, ray_d;
    Ray r(ray_o, ray_d);
    r.g = &g;
    r.rid = D.rid;
    r.skip = D.skip;
    r.has_ff = D.has_ff != 0;
    r.o = ff3{ff{D.o[0], D.o[1]}, ff{D.o[2], D.o[3]}, ff{D.o[4], D.o[5]}};
    if (r.has_ff) {
      r.d = ff3{ff{D.d[0], D.d[1]}, ff{D.d[2], D.d[3]}, ff{D.d[4], D.d[5]}};
      set_f32(r);
    } else {  // a primary ray: the same FP32 ray as in k_trace
      float omega;
      r.of = ff3_hi(r.o);
      r.df = grid_dir_f32(g, r.rid, omega);
      set_idir(r);
    }
    Best b;
    b.id = D.bid;
    b.slot = D.bslot;
    b.exact = D.bexact != 0;
    b.lo = D.blo;
    b.hi = D.bhi;
    b.t = ff{D.bt_hi, D.bt_lo};
    int cnt = 1 + D.sp;
    for (int j = lane; j < cnt; j += 32) list[j] = j == 0 ? D.node : D.stack[j - 1];
    __syncwarp();
    const int slot = D.slot;
    int nh = D.nh, k = D.k;
    for (;;) {
      b = coop_nearest<kCount>(tris, nodes, nt, r, b, list, cnt, n_nodes, n_tris);
      if (b.id < 0) {
        if (lane == 0) {
          record_miss(hits, hit_pos, slot, k, K);
          nvalid[slot] = nh;
        }
        break;
      }
      record_hit(tris, r, b, hits, hit_pos, (size_t)slot * K + k, lane == 0);
      ++nh;
      if (++k == K) {
        if (lane == 0) nvalid[slot] = nh;
        break;
      }
      if (kCount && lane == 0) ++n_trav;
      init_best(b);
      if (lane == 0) list[0] = nt > 1 ? 0 : ~0;
      cnt = 1;
      __syncwarp();
    }
  }
  if (kCount) {
    for (int o = 16; o; o >>= 1) {
      n_nodes += __shfl_xor_sync(0xffffffffu, n_nodes, o);
      n_tris += __shfl_xor_sync(0xffffffffu, n_tris, o);
      n_trav += __shfl_xor_sync(0xffffffffu, n_trav, o);
    }
    if (lane == 0) {
      atomicAdd(&counts[0], (unsigned long long)n_nodes);
      atomicAdd(&counts[1], (unsigned long long)n_tris);
      atomicAdd(&counts[2], (unsigned long long)n_trav);
    }
  }
}

// Few rays (reconstruction steps, small requests): one warp per ray from its
// first bounce on, every nearest-hit search a cooperative traversal.  A
// thread per ray would leave most SMs idle and end when the longest ray's
// dependent node fetches end; a warp per ray fills the GPU and splits each
// search over 32 lanes.  The candidates are ordered by the same total rule as
// in k_trace, so the hits are the same.
#ifndef SBR_TRACE_WARP_MAX
#define SBR_TRACE_WARP_MAX 32768
#endif
constexpr int64_t kWarpRaysMax = SBR_TRACE_WARP_MAX;  // rays up to which k_trace_warp runs

template <bool kCount>
__global__ void __launch_bounds__(128) k_trace_warp(const float4* __restrict__ tris,
                                                    const Node4* __restrict__ nodes, int nt, GridArg g,
                                                    const int32_t* __restrict__ ray_ids, int n_rays, int K,
                                                    sbr_hit* __restrict__ hits, float4* __restrict__ hit_pos,
                                                    float* __restrict__ ray_w, int32_t* __restrict__ nvalid,
                                                    unsigned long long* __restrict__ counts) {
  __shared__ int lists[4][kCoopList];
  const int lane = threadIdx.x & 31;
  int* list = lists[threadIdx.x >> 5];
  int n_nodes = 0, n_tris = 0, n_trav = 0;
  const int slot = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (slot < n_rays) {  // the same for the whole warp
    ff3 ray_o, ray_d;
    Ray r(ray_o, ray_d);
    r.g = &g;
    r.rid = ray_ids ? ray_ids[slot] : slot;
    r.has_ff = false;
    r.skip = -1;
    r.o = ff3_arr(g.o);
    r.of = ff3_hi(r.o);
    float omega;
    r.df = grid_dir_f32(g, r.rid, omega);
    set_idir(r);
    if (lane == 0) ray_w[slot] = omega;
    int nh = 0;
    for (int k = 0; k < K; ++k) {
      Best b;
      init_best(b);
      if (nt > 0) {
        if (kCount && lane == 0) ++n_trav;
        if (lane == 0) list[0] = nt > 1 ? 0 : ~0;
        __syncwarp();
        b = coop_nearest<kCount>(tris, nodes, nt, r, b, list, 1, n_nodes, n_tris);
        __syncwarp();  // every lane is done with the list
      }
      if (b.id < 0) {
        if (lane == 0) record_miss(hits, hit_pos, slot, k, K);
        break;
      }
      record_hit(tris, r, b, hits, hit_pos, (size_t)slot * K + k, lane == 0);
      ++nh;
    }
    if (lane == 0) nvalid[slot] = nh;
  }
  if (kCount) {
    for (int o = 16; o; o >>= 1) {
      n_nodes += __shfl_xor_sync(0xffffffffu, n_nodes, o);
      n_tris += __shfl_xor_sync(0xffffffffu, n_tris, o);
      n_trav += __shfl_xor_sync(0xffffffffu, n_trav, o);
    }
    if (lane == 0) {
      atomicAdd(&counts[0], (unsigned long long)n_nodes);
      atomicAdd(&counts[1], (unsigned long long)n_tris);
      atomicAdd(&counts[2], (unsigned long long)n_trav);
    }
  }
}

__device__ inline ff3 ld_hit(const float4* __restrict__ hp, size_t sl, float& cosv) {
  const float4 p = hp[2 * sl], q = hp[2 * sl + 1];
  cosv = q.z;
  return ff3{ff{p.x, p.y}, ff{p.z, p.w}, ff{q.x, q.y}};
}

// frac(x) of a float-float value, about [-1/2, 1/2], as a float-float pair
__device__ inline ff ff_frac(ff x) {
  const float n = rintf(x.hi);
  return fast_two_sum(x.hi - n, x.lo);  // x.hi - n is exact
}

// One (ray, bounce) path per lane: the hits of a warp's 32 rays are dealt out to
// its lanes (a ray's hits are ragged, 0 to K, so one thread per ray would leave
// most lanes idle); each lane recomputes its ray's Tx legs and interior length.
// NTX > 0: that many transmitters, their path lengths held in registers;
// NTX = 0: rd.ntx of them (up to SBR_MAX_TX).
template <int NTX, bool kMotion>
__global__ void k_prep(const float4* __restrict__ hit_pos, const sbr_hit* __restrict__ hits,
                       const float* __restrict__ ray_w, const int32_t* __restrict__ first, int n_rays, int K,
                       RadarArg rd, MatArg mat, MotionArg mot, int64_t cap, float4* __restrict__ prep,
                       float2* __restrict__ plen, int32_t* __restrict__ path_ray, float* __restrict__ phase_ofs,
                       float* __restrict__ path_rate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int p0 = 0, nh = 0;
  if (i < n_rays) {
    p0 = first[i];
    nh = first[i + 1] - p0;
  }
  int x = nh;  // inclusive scan of the warp's hit counts
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  const int pre = x - nh, total = __shfl_sync(0xffffffffu, x, 31);
  for (int base = 0; base < total; base += 32) {
    const int j = base + lane;
    int s = 0;  // owner: the last lane whose first item is <= j (it has hits)
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const int pc = __shfl_sync(0xffffffffu, pre, (s + step) & 31);
      if (s + step < 32 && pc <= j) s += step;
    }
    const int ps = __shfl_sync(0xffffffffu, pre, s), p0s = __shfl_sync(0xffffffffu, p0, s);
    if (j >= total) continue;
    const int k = j - ps, ri = i - lane + s;
    const int64_t p = p0s + k;
    const float omega = ray_w[ri];
    float cosv;
    const ff3 h1 = ld_hit(hit_pos, (size_t)ri * K, cosv);
    // Fresnel factor F = prod_{j<k} r_s(j) * (-r_s(k)) of the path (materials only)
    float2 F = make_float2(1.f, 0.f);
    auto fresnel_at = [&](int j, float c) {
      const float2 e = mat.eps[material_of(mat, hits[(size_t)ri * K + j].tri)];
      float2 r = e.x <= 0.f ? make_float2(-1.f, 0.f) : fresnel_rs(c, e, nullptr);
      if (j == k) r = make_float2(-r.x, -r.y);
      F = cmul(F, r);
    };
    if (mat.n > 0) fresnel_at(0, cosv);
    // moving objects: the antenna-independent part of dL/dt (the legs between hits)
    const float3 h0f = f3(h1.x.hi, h1.y.hi, h1.z.hi);
    float3 hpf = h0f, v0 = f3(0.f, 0.f, 0.f), vp = v0;
    float rate_in = 0.f;
    if (kMotion) vp = v0 = velocity_of(mot, hits[(size_t)ri * K].tri);
    constexpr int kT = NTX > 0 ? NTX : SBR_MAX_TX;
    const int ntx = NTX > 0 ? NTX : rd.ntx;
    ff lin[kT];
#pragma unroll
    for (int t = 0; t < kT; ++t)
      if (t < ntx) lin[t] = ff3_len(ff3_sub(h1, ff3_arr(rd.tx[t])));
    ff interior = ff_of(0.f);
    ff3 h = h1;
    for (int m = 1; m <= k; ++m) {  // same order of additions as a per-ray loop
      const ff3 hm = ld_hit(hit_pos, (size_t)ri * K + m, cosv);
      interior = ff_add(interior, ff3_len(ff3_sub(hm, h)));
      h = hm;
      if (mat.n > 0) fresnel_at(m, cosv);
      if (kMotion) {  // leg m-1 -> m: arrives at hit m, leaves hit m-1
        const float3 hmf = f3(hm.x.hi, hm.y.hi, hm.z.hi);
        const float3 vm = velocity_of(mot, hits[(size_t)ri * K + m].tri);
        const float3 e = hmf - hpf;
        const float3 u = e * rsqrtf(dot(e, e));
        rate_in += dot(vm, u) - dot(vp, u);
        hpf = hmf;
        vp = vm;
      }
    }
    float rlin[kT];  // 1 / L_in
#pragma unroll
    for (int t = 0; t < kT; ++t)
      if (t < ntx) {
        lin[t] = ff_add(lin[t], interior);
        rlin[t] = 1.f / lin[t].hi;
      }
    path_ray[p] = ri;
    // perfect conductors: the sign (-1)^(k-1); materials: |F| here, arg F in the phase
    float fphase = 0.f;
    float fmag = (k & 1) ? -1.f : 1.f;
    if (mat.n > 0) {
      fmag = hypotf(F.x, F.y);
      fphase = atan2f(F.y, F.x) * (float)(0.5 / M_PI);
    }
    phase_ofs[p] = fphase;
    const float wa = omega * fmag * cosv * (float)(0.25 / M_PI);
    float rate_tx[kT];  // v_1 . unit(h_1 - Tx_t)
    if (kMotion) {
#pragma unroll
      for (int t = 0; t < kT; ++t)
        if (t < ntx) {
          const float3 e = h0f - f3(rd.tx[t][0].hi, rd.tx[t][1].hi, rd.tx[t][2].hi);
          rate_tx[t] = dot(v0, e) * rsqrtf(dot(e, e));
        }
    }
    for (int rr = 0; rr < rd.nrx; ++rr) {
      const ff lout = ff3_len(ff3_sub(ff3_arr(rd.rx[rr]), h));
      const float wo = wa / lout.hi;
      float rate_rx = 0.f;  // v_k . unit(Rx_r - h_k)
      if (kMotion) {
        const float3 e = f3(rd.rx[rr][0].hi, rd.rx[rr][1].hi, rd.rx[rr][2].hi) - hpf;
        rate_rx = dot(vp, e) * rsqrtf(dot(e, e));
      }
#pragma unroll
      for (int t = 0; t < kT; ++t) {
        if (t >= ntx) break;
        const int v = t * rd.nrx + rr;
        const ff L = ff_add(lin[t], lout);
        const ff x0 = ff_frac(ff_mul(L, rd.k0));
        float phi0 = x0.hi + x0.lo;
        phi0 -= rintf(phi0);
        if (mat.n > 0) {
          phi0 += fphase;
          phi0 -= rintf(phi0);
        }
        const ff dl = ff_frac(ff_mul(L, rd.kb));
        const float dhi = rintf(dl.hi * 4096.f) * (1.f / 4096.f);
        const float dlo = (dl.hi - dhi) + dl.lo;  // dl.hi - dhi is exact
        prep[(size_t)v * cap + p] = make_float4(phi0, dhi, dlo, wo * rlin[t]);
        plen[(size_t)v * cap + p] = make_float2(L.hi, L.lo);
        if (kMotion) path_rate[(size_t)v * cap + p] = rate_in + rate_tx[t] - rate_rx;
      }
    }
  }
}

inline int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

// k_prep for the common transmitter counts (their legs stay in registers), with or without motion
template <bool kMotion>
void launch_prep(int nb, cudaStream_t st, const float4* hp4, const sbr_paths* paths, int64_t R, int K,
                 const RadarArg& rd, const MatArg& mat, const MotionArg& mot, float4* prep, float2* plen) {
  switch (rd.ntx) {
    case 1:
      k_prep<1, kMotion><<<nb, 128, 0, st>>>(hp4, paths->hits, paths->ray_weight, paths->ray_first, (int)R, K, rd,
                                              mat, mot, paths->path_cap, prep, plen, paths->path_ray,
                                              paths->phase_ofs, paths->path_rate);
      break;
    case 2:
      k_prep<2, kMotion><<<nb, 128, 0, st>>>(hp4, paths->hits, paths->ray_weight, paths->ray_first, (int)R, K, rd,
                                              mat, mot, paths->path_cap, prep, plen, paths->path_ray,
                                              paths->phase_ofs, paths->path_rate);
      break;
    case 3:
      k_prep<3, kMotion><<<nb, 128, 0, st>>>(hp4, paths->hits, paths->ray_weight, paths->ray_first, (int)R, K, rd,
                                              mat, mot, paths->path_cap, prep, plen, paths->path_ray,
                                              paths->phase_ofs, paths->path_rate);
      break;
    case 4:
      k_prep<4, kMotion><<<nb, 128, 0, st>>>(hp4, paths->hits, paths->ray_weight, paths->ray_first, (int)R, K, rd,
                                              mat, mot, paths->path_cap, prep, plen, paths->path_ray,
                                              paths->phase_ofs, paths->path_rate);
      break;
    default:
      k_prep<0, kMotion><<<nb, 128, 0, st>>>(hp4, paths->hits, paths->ray_weight, paths->ray_first, (int)R, K, rd,
                                              mat, mot, paths->path_cap, prep, plen, paths->path_ray,
                                              paths->phase_ofs, paths->path_rate);
  }
}

// After the scan's scratch in the paths region: the straggler hand-over's two
// counters (handed over, claimed) and its records.
constexpr size_t kCtrBytes = 256;
inline size_t scan_part(int32_t R) { return (scan_scratch_bytes(R > 0 ? R : 1) + 255) / 256 * 256; }
inline unsigned int* dump_counters(const sbr_paths* p) {
  return reinterpret_cast<unsigned int*>(static_cast<char*>(p->scratch) + scan_part(p->n_rays));
}
inline RayDump* dump_records(const sbr_paths* p) {
  return reinterpret_cast<RayDump*>(static_cast<char*>(p->scratch) + scan_part(p->n_rays) + kCtrBytes);
}
// warps of the straggler kernel: 16 per SM, each takes rays until none is left
inline int coop_grid() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    sms = 152;
  return 4 * sms;
}

size_t paths_layout(sbr_paths* p, void* mem, int32_t R, int32_t K, int32_t V) {
  Carver c(mem);
  const int64_t cap = (int64_t)R * K;
  const int64_t capc = cap > 0 ? cap : 1;
  p->n_rays = R;
  p->max_bounces = K;
  p->n_virt = V;
  p->path_cap = cap;
  p->hits = c.take<sbr_hit>(capc);
  p->hit_pos = c.take<float>(8 * capc);
  p->ray_weight = c.take<float>(R > 0 ? R : 1);
  p->ray_first = c.take<int32_t>((int64_t)R + 1);
  p->path_ray = c.take<int32_t>(capc);
  p->prep = c.take<float>(4 * (int64_t)V * capc);
  p->path_len = c.take<float>(2 * (int64_t)V * capc);
  p->scratch = c.take<char>(scan_part(R) + kCtrBytes + sizeof(RayDump) * (size_t)kDumpMax);
  p->phase_ofs = c.take<float>(capc);
  p->path_rate = c.take<float>((int64_t)V * capc);
  p->count = p->ray_first ? p->ray_first + R : nullptr;
  return c.bytes();
}

}  // namespace
}  // namespace sbr

using namespace sbr;

extern "C" size_t sbr_paths_bytes(int32_t n_rays, int32_t max_bounces, int32_t n_virt) {
  sbr_paths p{};
  if (n_rays < 0 || max_bounces < 1 || n_virt < 1) return 0;
  return paths_layout(&p, nullptr, n_rays, max_bounces, n_virt);
}

extern "C" sbr_status sbr_paths_bind(void* d_mem, size_t bytes, int32_t n_rays, int32_t max_bounces,
                                     int32_t n_virt, sbr_paths* out) {
  SBR_ARG(out != nullptr, "sbr_paths_bind: out is NULL");
  SBR_ARG(n_rays >= 0 && max_bounces >= 1 && max_bounces <= 16 && n_virt >= 1 &&
              n_virt <= SBR_MAX_VIRT,
          "sbr_paths_bind: bad sizes (R=%d K=%d V=%d)", n_rays, max_bounces, n_virt);
  SBR_ARG((int64_t)n_rays * max_bounces < (1ll << 31), "sbr_paths_bind: R*K above 2^31");
  SBR_ARG(d_mem && aligned256(d_mem), "sbr_paths_bind: d_mem NULL or not 256-byte aligned");
  const size_t need = sbr_paths_bytes(n_rays, max_bounces, n_virt);
  if (bytes < need) {
    set_error("sbr_paths_bind: region of %zu bytes, %zu needed", bytes, need);
    return SBR_ERR_OOM;
  }
  paths_layout(out, d_mem, n_rays, max_bounces, n_virt);
  return SBR_OK;
}

namespace sbr {
sbr_status check_radar(const sbr_radar_cfg* r, const char* who) {
  SBR_ARG(r != nullptr, "%s: radar is NULL", who);
  SBR_ARG(r->n_tx >= 1 && r->n_tx <= SBR_MAX_TX && r->n_rx >= 1 && r->n_rx <= SBR_MAX_RX &&
              r->n_tx * r->n_rx <= SBR_MAX_VIRT,
          "%s: antenna counts n_tx=%d n_rx=%d outside the supported range", who, r->n_tx, r->n_rx);
  SBR_ARG(r->n_samples >= 32 && r->n_samples <= 4096 && (r->n_samples & (r->n_samples - 1)) == 0,
          "%s: n_samples=%d must be a power of two in [32, 4096]", who, r->n_samples);
  SBR_ARG(r->n_chirps >= 1 && r->n_chirps <= 512 && (r->n_chirps & (r->n_chirps - 1)) == 0,
          "%s: n_chirps=%d must be a power of two in [1, 512]", who, r->n_chirps);
  SBR_ARG(r->f0 > 0 && r->bandwidth > 0 && r->chirp_time > 0, "%s: non-positive chirp constants", who);
  return SBR_OK;
}

sbr_status check_grid(const sbr_ray_grid* g, const char* who) {
  SBR_ARG(g != nullptr, "%s: grid is NULL", who);
  SBR_ARG(g->G >= 1 && g->G <= 46340, "%s: grid size G=%d outside [1, 46340]", who, g->G);
  SBR_ARG(g->tan_half > 0 && g->tan_half < 1e6, "%s: tan_half must be positive", who);
  return SBR_OK;
}
}  // namespace sbr

static sbr_status trace_impl(const sbr_scene* scene, const sbr_radar_cfg* radar, const sbr_ray_grid* grid,
                             const int32_t* d_ray_ids, int32_t n_ids, int32_t max_bounces,
                             const sbr_paths* paths, sbr_stream stream, unsigned long long* d_counts);

extern "C" sbr_status sbr_trace(const sbr_scene* scene, const sbr_radar_cfg* radar,
                                const sbr_ray_grid* grid, const int32_t* d_ray_ids, int32_t n_ids,
                                int32_t max_bounces, const sbr_paths* paths, sbr_stream stream) {
  return trace_impl(scene, radar, grid, d_ray_ids, n_ids, max_bounces, paths, stream, nullptr);
}

extern "C" sbr_status sbr_trace_counts(const sbr_scene* scene, const sbr_radar_cfg* radar,
                                       const sbr_ray_grid* grid, const int32_t* d_ray_ids, int32_t n_ids,
                                       int32_t max_bounces, const sbr_paths* paths, uint64_t* d_counts,
                                       sbr_stream stream) {
  SBR_ARG(d_counts, "sbr_trace_counts: d_counts is NULL");
  return trace_impl(scene, radar, grid, d_ray_ids, n_ids, max_bounces, paths, stream,
                    reinterpret_cast<unsigned long long*>(d_counts));
}

static sbr_status trace_impl(const sbr_scene* scene, const sbr_radar_cfg* radar, const sbr_ray_grid* grid,
                             const int32_t* d_ray_ids, int32_t n_ids, int32_t max_bounces,
                             const sbr_paths* paths, sbr_stream stream, unsigned long long* d_counts) {
  SBR_ARG(scene && paths, "sbr_trace: NULL scene or paths");
  sbr_status rs = check_radar(radar, "sbr_trace");
  if (rs != SBR_OK) return rs;
  rs = check_grid(grid, "sbr_trace");
  if (rs != SBR_OK) return rs;
  const int64_t R = n_ids >= 0 ? (int64_t)n_ids : (int64_t)grid->G * grid->G;
  SBR_ARG(n_ids <= 0 || d_ray_ids, "sbr_trace: n_ids=%d rays but d_ray_ids is NULL", n_ids);
  if (n_ids < 0) d_ray_ids = nullptr;
  SBR_ARG(paths->n_rays == R && paths->max_bounces == max_bounces &&
              paths->n_virt == radar->n_tx * radar->n_rx,
          "sbr_trace: paths bound for R=%d K=%d V=%d, call needs R=%lld K=%d V=%d", paths->n_rays,
          paths->max_bounces, paths->n_virt, (long long)R, max_bounces, radar->n_tx * radar->n_rx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GridArg g;
  for (int j = 0; j < 3; ++j) {
    g.o[j] = ff_from_double(grid->origin[j]);
    g.ax[j] = ff_from_double(grid->axis[j]);
    g.ua[j] = ff_from_double(grid->u_axis[j]);
    g.va[j] = ff_from_double(grid->v_axis[j]);
  }
  g.start = ff_from_double(-grid->tan_half + grid->tan_half / grid->G);
  g.step = ff_from_double(2.0 * grid->tan_half / grid->G);
  g.lo = ff_from_double(-grid->tan_half);
  g.cell = (float)(2.0 * grid->tan_half / grid->G);
  g.G = grid->G;
  g.jitter = grid->jitter;
  RadarArg rd;
  for (int t = 0; t < SBR_MAX_TX; ++t)
    for (int j = 0; j < 3; ++j) rd.tx[t][j] = ff_from_double(radar->tx[t][j]);
  for (int r = 0; r < SBR_MAX_RX; ++r)
    for (int j = 0; j < 3; ++j) rd.rx[r][j] = ff_from_double(radar->rx[r][j]);
  rd.k0 = ff_from_double(radar->f0 / kC);
  rd.kb = ff_from_double(radar->bandwidth / (kC * radar->n_samples));
  rd.ntx = radar->n_tx;
  rd.nrx = radar->n_rx;
  if (R == 0) {
    SBR_CUDA(cudaMemsetAsync(paths->ray_first, 0, sizeof(int32_t), st));
    return SBR_OK;
  }
  RayDump* dumps = dump_records(paths);
  unsigned int* dctr = dump_counters(paths);
  SBR_CUDA(cudaMemsetAsync(dctr, 0, 2 * sizeof(unsigned int), st));
  float4* hp = reinterpret_cast<float4*>(paths->hit_pos);
  if (d_counts) SBR_CUDA(cudaMemsetAsync(d_counts, 0, 4 * sizeof(unsigned long long), st));
  if (R <= kWarpRaysMax) {  // one warp per ray (no hand-over needed)
    const int nbw = blocks(R * 32, 128);
    ::sbr::note_launch();
    if (d_counts)
      k_trace_warp<true><<<nbw, 128, 0, st>>>(scene->tris, scene->nodes4, scene->nt, g, d_ray_ids, (int)R,
                                               max_bounces, paths->hits, hp, paths->ray_weight, paths->ray_first,
                                               d_counts);
    else
      k_trace_warp<false><<<nbw, 128, 0, st>>>(scene->tris, scene->nodes4, scene->nt, g, d_ray_ids, (int)R,
                                                max_bounces, paths->hits, hp, paths->ray_weight, paths->ray_first,
                                                nullptr);
  } else if (d_counts) {
    ::sbr::note_launch();
    k_trace<true><<<blocks(R, 128), 128, 0, st>>>(scene->tris, scene->nodes4, scene->nt, g, d_ray_ids, (int)R,
                                                  max_bounces, paths->hits, hp, paths->ray_weight, paths->ray_first,
                                                  dumps, dctr, d_counts, scene->top, scene->top_n);
    ::sbr::note_launch();
    k_trace_coop<true><<<coop_grid(), 128, 0, st>>>(scene->tris, scene->nodes4, scene->nt, g, max_bounces, dumps,
                                                    dctr, dctr + 1, paths->hits, hp, paths->ray_first, d_counts);
  } else {
    ::sbr::note_launch();
    k_trace<false><<<blocks(R, 128), 128, 0, st>>>(scene->tris, scene->nodes4, scene->nt, g, d_ray_ids, (int)R,
                                                   max_bounces, paths->hits, hp, paths->ray_weight,
                                                   paths->ray_first, dumps, dctr, nullptr, scene->top, scene->top_n);
    ::sbr::note_launch();
    k_trace_coop<false><<<coop_grid(), 128, 0, st>>>(scene->tris, scene->nodes4, scene->nt, g, max_bounces, dumps,
                                                     dctr, dctr + 1, paths->hits, hp, paths->ray_first, nullptr);
  }
  SBR_CUDA(cudaGetLastError());
  SBR_CUDA(exclusive_scan(paths->ray_first, paths->ray_first, R, nullptr, paths->scratch, st));
  ::sbr::note_launch();
  {
    const float4* hp4 = reinterpret_cast<const float4*>(paths->hit_pos);
    float4* prep = reinterpret_cast<float4*>(paths->prep);
    float2* plen = reinterpret_cast<float2*>(paths->path_len);
    const int nb = blocks(R, 128);
    const MatArg mat = mat_arg(scene);
    const MotionArg mot = motion_arg(scene);
    if (mot.n > 0)
      launch_prep<true>(nb, st, hp4, paths, R, max_bounces, rd, mat, mot, prep, plen);
    else
      launch_prep<false>(nb, st, hp4, paths, R, max_bounces, rd, mat, mot, prep, plen);
  }
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}
