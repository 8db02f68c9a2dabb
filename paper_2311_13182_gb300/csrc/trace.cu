// Ray tracing with specular bounces (Section 3.2.1, Eq. 2-3) and path preparation.
//
// One thread per ray.  Each bounce runs a stack traversal of the LBVH in FP32
// (64-B nodes fetched as four float4, triangles as three float4) with the
// Moller-Trumbore (1997) test.  Every FP32 decision carries a forward error
// bound: a triangle is accepted or rejected in FP32 only when the bound says
// FP64 arithmetic on the FP64 ray would decide the same; otherwise the test is
// repeated in FP64.  Nearest-hit ordering is decided the same way (interval
// overlap -> FP64 t, exact ties -> lower triangle index).  The hit of each bounce
// is then refined in FP64 and the FP64 ray is reflected, so the chosen triangle
// sequence is that of an FP64 brute-force search for every ray not within
// rounding distance of an edge.
//
// Path preparation (FP64, O(paths x antennas)): per hit k and virtual antenna
// (t, r): L_in = |h_1 - Tx_t| + sum_{j=2..k} |h_j - h_{j-1}|, L_out = |Rx_r - h_k|,
// tau = (L_in + L_out)/c, phi0 = frac(f_c tau), delta = frac(B tau / N_s) split
// into delta_hi (a multiple of 2^-12, so n * delta_hi is exact in FP32 for
// n < 4096) and delta_lo, and A = omega (-1)^(k-1) |d_k . n_k| / (4 pi L_in L_out).
#include <math.h>

#include "scene.cuh"

namespace sbr {
namespace {

struct GridArg {
  double o[3], ax[3], ua[3], va[3];
  double th;
  int G;
};

struct RadarArg {
  double tx[SBR_MAX_TX][3];
  double rx[SBR_MAX_RX][3];
  double f0, b_over_ns;
  int ntx, nrx;
};

constexpr float kTmin = 1e-9f;
constexpr double kTmin64 = 1e-9;
constexpr float kErr = 1.0f / 262144.0f;  // 2^-18 = 64 ulp(1): scale of the FP32 error bounds

__device__ inline void grid_ray(const GridArg& g, int rid, d3& o, d3& d, float& omega) {
  const int row = rid / g.G, col = rid - row * g.G;
  const double a = g.th * (2.0 * (col + 0.5) / g.G - 1.0);
  const double b = g.th * (2.0 * (row + 0.5) / g.G - 1.0);
  d3 w = mk3(g.ax[0], g.ax[1], g.ax[2]) + (mk3(g.ua[0], g.ua[1], g.ua[2]) * a +
                                            mk3(g.va[0], g.va[1], g.va[2]) * b);
  const double len = sqrt(dot(w, w));
  d = w * (1.0 / len);
  o = mk3(g.o[0], g.o[1], g.o[2]);
  const double cell = 2.0 * g.th / g.G;
  omega = (float)(cell * cell / (len * len * len));
}

__device__ inline d3 tri_vert(const float4* __restrict__ tris, int slot, int c) {
  float4 v = __ldg(&tris[3 * slot + c]);
  return mk3(v.x, v.y, v.z);
}

// FP64 Moller-Trumbore, two-sided; the rule the brute-force definition uses.
__device__ inline bool mt64(d3 o, d3 d, d3 a, d3 b, d3 c, double& t, double& u, double& v) {
  d3 e1 = b - a, e2 = c - a;
  d3 p = cross(d, e2);
  double det = dot(e1, p);
  if (fabs(det) < 1e-12) return false;
  double inv = 1.0 / det;
  d3 s = o - a;
  u = dot(s, p) * inv;
  if (u < 0.0 || u > 1.0) return false;
  d3 q = cross(s, e1);
  v = dot(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  t = dot(e2, q) * inv;
  return t > kTmin64;
}

struct Best {
  int id, slot;
  float lo, hi;  // interval containing the FP64 distance
  bool exact;
  double t64;
};

struct Ray {
  float3 o, d, idir;
  d3 o64, d64;
  int skip;
};

__device__ inline bool exact_t(const float4* __restrict__ tris, const Ray& r, int slot, double& t) {
  double u, v;
  return mt64(r.o64, r.d64, tri_vert(tris, slot, 0), tri_vert(tris, slot, 1), tri_vert(tris, slot, 2),
              t, u, v);
}

__device__ inline void take_exact(Best& b, int id, int slot, double t) {
  b.id = id;
  b.slot = slot;
  b.exact = true;
  b.t64 = t;
  float tf = (float)t;
  b.lo = tf - fabsf(tf) * 2.4e-7f;
  b.hi = tf + fabsf(tf) * 2.4e-7f;
}

// Offer a candidate whose FP64 distance lies in [lo, hi] (exact: t64 known).
__device__ inline void consider(Best& b, const float4* __restrict__ tris, const Ray& r, int id,
                                int slot, float lo, float hi, bool exact, double t64) {
  if (b.id < 0 || hi < b.lo) {
    if (exact) take_exact(b, id, slot, t64);
    else {
      b.id = id; b.slot = slot; b.lo = lo; b.hi = hi; b.exact = false;
    }
    return;
  }
  if (lo > b.hi) return;
  // overlapping intervals: order in FP64, ties to the lower triangle index
  if (!exact && !exact_t(tris, r, slot, t64)) return;
  if (!b.exact) {
    double tb;
    if (!exact_t(tris, r, b.slot, tb)) {  // cannot happen with valid bounds; keep the new one
      take_exact(b, id, slot, t64);
      return;
    }
    take_exact(b, b.id, b.slot, tb);
  }
  if (t64 < b.t64 || (t64 == b.t64 && id < b.id)) take_exact(b, id, slot, t64);
}

__device__ inline void test_tri(Best& b, const float4* __restrict__ tris, const Ray& r, int slot) {
  const float4 A = __ldg(&tris[3 * slot]);
  const int id = __float_as_int(A.w);
  if (id == r.skip) return;
  const float4 B = __ldg(&tris[3 * slot + 1]);
  const float4 C = __ldg(&tris[3 * slot + 2]);
  const float3 v0 = f3(A.x, A.y, A.z);
  const float3 e1 = f3(B.x, B.y, B.z) - v0;
  const float3 e2 = f3(C.x, C.y, C.z) - v0;
  const float3 p = cross(r.d, e2);
  const float det = dot(e1, p);
  const float3 s = r.o - v0;
  const float3 q = cross(s, e1);
  const float un = dot(s, p), vn = dot(r.d, q), tn = dot(e2, q);
  // forward error bounds of the FP32 values against FP64 arithmetic on the FP64 ray
  const float m1 = l1(e1), m2 = l1(e2), ms = l1(r.o) + l1(v0);
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
    float lo = nlo / (nlo >= 0.f ? adet + edet : adet - edet);
    float hi = nhi / (nhi >= 0.f ? adet - edet : adet + edet);
    lo -= fabsf(lo) * 2.4e-7f;
    hi += fabsf(hi) * 2.4e-7f;
    if (hi <= kTmin) return;                      // behind the origin in FP64 too
    if (b.id >= 0 && lo > b.hi) return;           // farther than the current hit
    if (su > eu && sv > ev && sw > ew && lo > kTmin) {
      consider(b, tris, r, id, slot, lo, hi, false, 0.0);
      return;
    }
  }
  double t;
  if (exact_t(tris, r, slot, t)) {
    const float tf = (float)t;
    consider(b, tris, r, id, slot, tf - fabsf(tf) * 2.4e-7f, tf + fabsf(tf) * 2.4e-7f, true, t);
  }
}

__device__ inline void slab(const float3& o, const float3& idir, float lox, float hix, float loy,
                            float hiy, float loz, float hiz, float& tn, float& tf) {
  float tx0 = (lox - o.x) * idir.x, tx1 = (hix - o.x) * idir.x;
  float ty0 = (loy - o.y) * idir.y, ty1 = (hiy - o.y) * idir.y;
  float tz0 = (loz - o.z) * idir.z, tz1 = (hiz - o.z) * idir.z;
  tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fminf(tz0, tz1));
  tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
  tf = tf * 1.0000005f + 1e-30f;
}

__device__ Best nearest(const float4* __restrict__ tris, const Node* __restrict__ nodes, int nt,
                        const Ray& r) {
  Best b;
  b.id = -1;
  b.slot = -1;
  b.lo = b.hi = INFINITY;
  b.exact = false;
  b.t64 = 0.0;
  if (nt <= 0) return b;
  int stack[64];
  int sp = 0;
  int node = nt > 1 ? 0 : ~0;
  // a valid tree is visited at most once per node: the cap only guards
  // against a corrupted hierarchy turning into an endless loop
  for (int guard = 2 * nt + 64; guard > 0; --guard) {
    if (node >= 0) {
      const float4 a = __ldg(&nodes[node].lxy);
      const float4 c = __ldg(&nodes[node].rxy);
      const float4 z = __ldg(&nodes[node].lrz);
      const int4 ch = __ldg(&nodes[node].child);
      float ln, lf, rn, rf;
      slab(r.o, r.idir, a.x, a.y, a.z, a.w, z.x, z.y, ln, lf);
      slab(r.o, r.idir, c.x, c.y, c.z, c.w, z.z, z.w, rn, rf);
      const float lim = b.hi;
      const bool hl = ln <= lf && lf >= 0.f && ln <= lim;
      const bool hr = rn <= rf && rf >= 0.f && rn <= lim;
      if (hl && hr) {
        const bool lfirst = ln <= rn;
        if (sp < 64) stack[sp++] = lfirst ? ch.y : ch.x;
        node = lfirst ? ch.x : ch.y;
        continue;
      }
      if (hl) { node = ch.x; continue; }
      if (hr) { node = ch.y; continue; }
    } else {
      test_tri(b, tris, r, ~node);
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return b;
}

__device__ inline void set_f32(Ray& r) {
  r.o = f3((float)r.o64.x, (float)r.o64.y, (float)r.o64.z);
  r.d = f3((float)r.d64.x, (float)r.d64.y, (float)r.d64.z);
  auto inv = [](float x) { return 1.0f / (fabsf(x) < 1e-20f ? copysignf(1e-20f, x) : x); };
  r.idir = f3(inv(r.d.x), inv(r.d.y), inv(r.d.z));
}

__global__ void __launch_bounds__(128) k_trace(const float4* __restrict__ tris,
                                               const Node* __restrict__ nodes, int nt, GridArg g,
                                               const int32_t* __restrict__ ray_ids, int n_rays,
                                               int K, sbr_hit* __restrict__ hits,
                                               double4* __restrict__ hit_pos,
                                               float* __restrict__ ray_w,
                                               int32_t* __restrict__ nvalid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rays) return;
  const int rid = ray_ids ? ray_ids[i] : i;
  Ray r;
  float omega;
  grid_ray(g, rid, r.o64, r.d64, omega);
  r.skip = -1;
  set_f32(r);
  ray_w[i] = omega;
  int nh = 0;
  for (int k = 0; k < K; ++k) {
    const size_t sl = (size_t)i * K + k;
    Best b = nearest(tris, nodes, nt, r);
    if (b.id < 0) {
      for (int kk = k; kk < K; ++kk) {
        hits[(size_t)i * K + kk] = sbr_hit{-1, 0.f, 0.f, 0.f};
        hit_pos[(size_t)i * K + kk] = make_double4(0.0, 0.0, 0.0, 0.0);
      }
      break;
    }
    const d3 a = tri_vert(tris, b.slot, 0), bb = tri_vert(tris, b.slot, 1),
             c = tri_vert(tris, b.slot, 2);
    double t, u, v;
    if (!mt64(r.o64, r.d64, a, bb, c, t, u, v)) {
      // unreachable with valid bounds: fall back to the plane intersection
      d3 n0 = cross(bb - a, c - a);
      t = dot(n0, a - r.o64) / dot(n0, r.d64);
      u = v = 0.0;
    }
    const d3 h = r.o64 + r.d64 * t;
    d3 n = cross(bb - a, c - a);
    n = n * (1.0 / sqrt(dot(n, n)));
    const double dn = dot(r.d64, n);
    hits[sl] = sbr_hit{b.id, (float)t, (float)u, (float)v};
    hit_pos[sl] = make_double4(h.x, h.y, h.z, fabs(dn));
    r.d64 = r.d64 - n * (2.0 * dn);
    r.o64 = h;
    r.skip = b.id;
    set_f32(r);
    ++nh;
  }
  nvalid[i] = nh;
}

__device__ inline double dist(d3 a, d3 b) {
  d3 e = a - b;
  return sqrt(dot(e, e));
}

__global__ void k_prep(const double4* __restrict__ hit_pos, const float* __restrict__ ray_w,
                       const int32_t* __restrict__ first, int n_rays, int K, RadarArg rd,
                       int64_t cap, float4* __restrict__ prep, double* __restrict__ tau64,
                       int32_t* __restrict__ path_ray) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rays) return;
  const int p0 = first[i], nh = first[i + 1] - p0;
  const float omega = ray_w[i];
  double interior = 0.0;
  d3 h1 = mk3(0, 0, 0), hp = mk3(0, 0, 0);
  for (int k = 0; k < nh; ++k) {
    const double4 hk = hit_pos[(size_t)i * K + k];
    const d3 h = mk3(hk.x, hk.y, hk.z);
    if (k == 0) h1 = h;
    else interior += dist(h, hp);
    hp = h;
    const int64_t p = p0 + k;
    path_ray[p] = i;
    const double sign = (k & 1) ? -1.0 : 1.0;
    double lout[SBR_MAX_RX];
    for (int rr = 0; rr < rd.nrx; ++rr) lout[rr] = dist(mk3(rd.rx[rr][0], rd.rx[rr][1], rd.rx[rr][2]), h);
    for (int t = 0; t < rd.ntx; ++t) {
      const double lin = dist(h1, mk3(rd.tx[t][0], rd.tx[t][1], rd.tx[t][2])) + interior;
      for (int rr = 0; rr < rd.nrx; ++rr) {
        const int v = t * rd.nrx + rr;
        const double tau = (lin + lout[rr]) / kC;
        const double x0 = rd.f0 * tau;
        const double phi0 = x0 - rint(x0);
        double dl = rd.b_over_ns * tau;
        dl -= rint(dl);
        const double dhi = rint(dl * 4096.0) * (1.0 / 4096.0);
        const float amp = (float)(omega * sign * hk.w / (4.0 * M_PI * lin * lout[rr]));
        prep[(size_t)v * cap + p] = make_float4((float)phi0, (float)dhi, (float)(dl - dhi), amp);
        tau64[(size_t)v * cap + p] = tau;
      }
    }
  }
}

inline int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

size_t paths_layout(sbr_paths* p, void* mem, int32_t R, int32_t K, int32_t V) {
  Carver c(mem);
  const int64_t cap = (int64_t)R * K;
  const int64_t capc = cap > 0 ? cap : 1;
  p->n_rays = R;
  p->max_bounces = K;
  p->n_virt = V;
  p->path_cap = cap;
  p->hits = c.take<sbr_hit>(capc);
  p->hit_pos = c.take<double>(4 * capc);
  p->ray_weight = c.take<float>(R > 0 ? R : 1);
  p->ray_first = c.take<int32_t>((int64_t)R + 1);
  p->path_ray = c.take<int32_t>(capc);
  p->prep = c.take<float>(4 * (int64_t)V * capc);
  p->tau64 = c.take<double>((int64_t)V * capc);
  p->scratch = c.take<char>(scan_scratch_bytes(R > 0 ? R : 1));
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

extern "C" sbr_status sbr_trace(const sbr_scene* scene, const sbr_radar_cfg* radar,
                                const sbr_ray_grid* grid, const int32_t* d_ray_ids, int32_t n_ids,
                                int32_t max_bounces, const sbr_paths* paths, sbr_stream stream) {
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
    g.o[j] = grid->origin[j];
    g.ax[j] = grid->axis[j];
    g.ua[j] = grid->u_axis[j];
    g.va[j] = grid->v_axis[j];
  }
  g.th = grid->tan_half;
  g.G = grid->G;
  RadarArg rd;
  for (int t = 0; t < SBR_MAX_TX; ++t)
    for (int j = 0; j < 3; ++j) rd.tx[t][j] = radar->tx[t][j];
  for (int r = 0; r < SBR_MAX_RX; ++r)
    for (int j = 0; j < 3; ++j) rd.rx[r][j] = radar->rx[r][j];
  rd.f0 = radar->f0;
  rd.b_over_ns = radar->bandwidth / radar->n_samples;
  rd.ntx = radar->n_tx;
  rd.nrx = radar->n_rx;
  if (R == 0) {
    SBR_CUDA(cudaMemsetAsync(paths->ray_first, 0, sizeof(int32_t), st));
    return SBR_OK;
  }
  ::sbr::note_launch();
  k_trace<<<blocks(R, 128), 128, 0, st>>>(scene->tris, scene->nodes, scene->nt, g, d_ray_ids,
                                          (int)R, max_bounces, paths->hits,
                                          reinterpret_cast<double4*>(paths->hit_pos),
                                          paths->ray_weight, paths->ray_first);
  SBR_CUDA(cudaGetLastError());
  SBR_CUDA(exclusive_scan(paths->ray_first, paths->ray_first, R, nullptr, paths->scratch, st));
  ::sbr::note_launch();
  k_prep<<<blocks(R, 128), 128, 0, st>>>(reinterpret_cast<const double4*>(paths->hit_pos),
                                         paths->ray_weight, paths->ray_first, (int)R, max_bounces,
                                         rd, paths->path_cap,
                                         reinterpret_cast<float4*>(paths->prep), paths->tau64,
                                         paths->path_ray);
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}
