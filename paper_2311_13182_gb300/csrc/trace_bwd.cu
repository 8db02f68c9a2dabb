// Adjoint of the trace and path preparation (Section 3.3, Eq. 13 chain rule;
// the continuous-integrand derivative of Eq. 4-5).
//
// With the triangle sequence of every ray held fixed (visibility changes are
// the discontinuous part; see the reparameterisation below), each hit
// is a smooth function of the vertices:
//   h_k = o_k + t_k d_k,  t_k = N_k.(a_k - o_k) / (N_k.d_k),  N_k = (b_k - a_k) x (c_k - a_k)
//   d_{k+1} = d_k - 2 (d_k.n_k) n_k,  n_k = N_k / |N_k|,  o_{k+1} = h_k
// and each path (k, t, r) has length L_in + L_out and strength
//   A = omega (-1)^(k-1) |d_k.n_k| / (4 pi L_in L_out),
//   L_in = |h_1 - Tx_t| + sum_{j=2..k} |h_j - h_{j-1}|,  L_out = |Rx_r - h_k|.
// With materials each path also carries its Fresnel factor F = prod_{j<k} r_s(j)
// (-r_s(k)) (Section 3.2.2, Eq. 9-10): the strength is A |F| and the phase has
// arg F / (2 pi) added, so with G_A = sum_v dL/dA' A' and G_o = sum_v dL/d(phase
// offset) every bounce j of the path adds, through d log F = sum_j d log r_s(j),
//   dL/d cos_j += G_A Re(q) + G_o Im(q) / (2 pi),  q = d log r_s / d cos = -2 / w,
//   dL/d eps_m += the same with q = d log r_s / d eps = cos / (w (eps - 1)),
// w = sqrt(eps - 1 + cos^2), for eps = eps_re - j eps_im (d eps / d eps_im = -j).
// Reparameterised samples (Eq. 6-7, SBR_BWD_REPARAM): the first hit is attached
// to its triangle at the forward barycentrics, x = (1 - u - v) a + u b + v c,
// d_1 = (x - o) / r, r = |x - o|, and the ray's weight carries |det J_T| =
// J / J_0 with J = |s| / r^3, s = N_1.(x - o).  The sweep's adjoint of d_1 then
// flows into x, dL/dx += (I - d_1 d_1^T) dL/dd_1 / r, and with
// G_w = sum over the ray's paths of dL/dA A (A is linear in the weight),
//   dL/dx += G_w (N_1 / s - 3 (x - o) / r^2),  dL/dN_1 += G_w (x - o) / s.
// One thread per ray accumulates the adjoints of its path lengths and
// strengths onto the hit points and |d.n| terms, then sweeps the bounces in
// reverse, and adds the per-corner vertex gradients to the vertices with the
// order-independent fixed-point scatter of common.cuh (two passes over the rays:
// the largest contribution, then the integer sums), so the gradient is bitwise
// the same on every run.
#include <math.h>

#include "scene.cuh"

namespace sbr {
namespace {

constexpr int kMaxK = 8;

struct GridF {
  float o[3], ax[3], ua[3], va[3];
  float start, step;  // first cell centre -tan_half (1 - 1/G) and the cell pitch 2 tan_half / G
  float lo;           // -tan_half (jittered sampling)
  int G;
  const float* jitter;
};

struct RadarF {
  float tx[SBR_MAX_TX][3];
  float rx[SBR_MAX_RX][3];
  int ntx, nrx;
};

__device__ inline float3 ld3(const float* v, int i) { return f3(v[3 * i], v[3 * i + 1], v[3 * i + 2]); }
__device__ inline float len3(float3 a) { return sqrtf(dot(a, a)); }
__device__ inline void add3(float3& a, float3 b) { a = a + b; }

// Pass 0 records the largest |component|, pass 1 adds the fixed-point values.
template <int kPass>
__device__ inline void scatter(const FixScatter& fs, int E, float& lmax, int vi, float3 d) {
  if (kPass == 0) {
    lmax = fmaxf(lmax, fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z))));
  } else {
    fix_add(&fs.acc[3 * vi], d.x, E);
    fix_add(&fs.acc[3 * vi + 1], d.y, E);
    fix_add(&fs.acc[3 * vi + 2], d.z, E);
  }
}

// Material gradients: pass 0 records the largest magnitude, pass 1 adds.
template <int kPass>
__device__ inline void scatter_eps(const FixScatter& fe, int Ee, float& emax, int m, float dre, float dim) {
  if (kPass == 0) {
    emax = fmaxf(emax, fmaxf(fabsf(dre), fabsf(dim)));
  } else {
    fix_add(&fe.acc[2 * m], dre, Ee);
    fix_add(&fe.acc[2 * m + 1], dim, Ee);
  }
}

template <int kPass>
__device__ void ray_adjoint(int i, const float* __restrict__ verts, int nv, const int32_t* __restrict__ faces,
                            const GridF& g, const RadarF& rd, const MatArg& mat, const int32_t* __restrict__ ray_ids,
                            int K, const sbr_hit* __restrict__ hits, const float4* __restrict__ hit_pos,
                            const int32_t* __restrict__ first, const float4* __restrict__ prep, int64_t cap,
                            const float* __restrict__ glen, const float* __restrict__ gamp,
                            const float* __restrict__ gphase, bool reparam, const FixScatter& fs, int E,
                            float& lmax, const FixScatter& fe, int Ee, float& emax) {
  const int p0 = first[i], m = first[i + 1] - p0;
  if (m <= 0) return;
  // launch direction in FP32 (cell centre a = start + col step, likewise b with row)
  const int rid = ray_ids ? ray_ids[i] : i;
  const int row = rid / g.G, col = rid - row * g.G;
  float a0, b0;
  if (g.jitter) {
    const float2 jt = reinterpret_cast<const float2*>(g.jitter)[rid];
    a0 = fmaf(g.step, (float)col + jt.x, g.lo);
    b0 = fmaf(g.step, (float)row + jt.y, g.lo);
  } else {
    a0 = fmaf(g.step, (float)col, g.start);
    b0 = fmaf(g.step, (float)row, g.start);
  }
  const float wx = g.ax[0] + g.ua[0] * a0 + g.va[0] * b0, wy = g.ax[1] + g.ua[1] * a0 + g.va[1] * b0,
              wz = g.ax[2] + g.ua[2] * a0 + g.va[2] * b0;
  const float wl = rsqrtf(wx * wx + wy * wy + wz * wz);
  float3 d[kMaxK], h[kMaxK], nh[kMaxK], N[kMaxK], A[kMaxK];
  float nlen[kMaxK], t[kMaxK], cdn[kMaxK];
  int fv[kMaxK][3];
  int mj[kMaxK];        // material of bounce j (-1: perfect conductor or no materials)
  float2 wj[kMaxK];     // w = sqrt(eps - 1 + cos^2) of bounce j
  d[0] = f3(wx * wl, wy * wl, wz * wl);
  const float3 org = f3(g.o[0], g.o[1], g.o[2]);
  float3 x0 = org;
  float bu = 0.f, bv = 0.f;
  if (reparam) {  // the launch direction attached to the first hit's surface point
    const size_t s0 = (size_t)i * K;
    bu = hits[s0].u;
    bv = hits[s0].v;
    const int id = hits[s0].tri;
    int q[3];
    for (int c = 0; c < 3; ++c) {
      q[c] = faces[3 * id + c];
      q[c] = (q[c] >= 0 && q[c] < nv) ? q[c] : 0;
    }
    x0 = ld3(verts, q[0]) * (1.f - bu - bv) + ld3(verts, q[1]) * bu + ld3(verts, q[2]) * bv;
    const float3 e = x0 - org;
    d[0] = e * rsqrtf(dot(e, e));
  }
  float gw = 0.f;  // sum over the ray's paths of dL/dA A
  for (int k = 0; k < m; ++k) {
    const size_t sl = (size_t)i * K + k;
    const int id = hits[sl].tri;
    t[k] = hits[sl].t;
    const float4 hp = hit_pos[2 * sl], hq = hit_pos[2 * sl + 1];  // float-float pairs: hi parts
    h[k] = f3(hp.x, hp.z, hq.x);
    for (int c = 0; c < 3; ++c) {
      const int q = faces[3 * id + c];
      fv[k][c] = (q >= 0 && q < nv) ? q : 0;  // invalid faces were reported by the scene build
    }
    const float3 va = ld3(verts, fv[k][0]), vb = ld3(verts, fv[k][1]), vc = ld3(verts, fv[k][2]);
    A[k] = va;
    N[k] = cross(vb - va, vc - va);
    nlen[k] = len3(N[k]);
    nh[k] = N[k] * (1.f / nlen[k]);
    cdn[k] = dot(d[k], nh[k]);
    if (k + 1 < m) d[k + 1] = d[k] - nh[k] * (2.f * cdn[k]);
    mj[k] = -1;
    if (mat.n > 0) {
      const int mm = material_of(mat, id);
      if (mat.eps[mm].x > 0.f) {
        mj[k] = mm;
        fresnel_rs(fabsf(cdn[k]), mat.eps[mm], &wj[k]);
      }
    }
  }
  // adjoints of hit points and of |d.n| from every path of this ray
  float3 hb[kMaxK];
  float cb[kMaxK];
  for (int k = 0; k < m; ++k) {
    hb[k] = f3(0.f, 0.f, 0.f);
    cb[k] = 0.f;
  }
  float segb[kMaxK];  // adjoint of |h_j - h_{j-1}|
  for (int k = 0; k < m; ++k) segb[k] = 0.f;
  float interior = 0.f;
  for (int k = 0; k < m; ++k) {
    if (k > 0) interior += len3(h[k] - h[k - 1]);
    const int64_t p = p0 + k;
    float lin_sum_b = 0.f;  // sum over antennas of dL/dL_in (for the interior segments)
    float g_a = 0.f, g_o = 0.f;  // sum over antennas of dL/dA' A' and of dL/d(phase offset)
    for (int tt = 0; tt < rd.ntx; ++tt) {
      const float3 et = h[0] - f3(rd.tx[tt][0], rd.tx[tt][1], rd.tx[tt][2]);
      const float l1 = len3(et);
      const float lin = l1 + interior;
      float linb = 0.f;
      for (int rr = 0; rr < rd.nrx; ++rr) {
        const int v = tt * rd.nrx + rr;
        const float3 er = h[k] - f3(rd.rx[rr][0], rd.rx[rr][1], rd.rx[rr][2]);
        const float lout = len3(er);
        const float gl = glen[(size_t)v * cap + p], ga = gamp[(size_t)v * cap + p];
        const float amp = prep[(size_t)v * cap + p].w;
        const float ab = ga * amp;
        g_a += ab;
        if (mat.n > 0) g_o += gphase[(size_t)v * cap + p];
        linb += gl - ab / lin;
        const float loutb = gl - ab / lout;
        add3(hb[k], er * (loutb / lout));
        // A is linear in |d.n|: dA/d|d.n| = A / |d.n|
        const float ac = fabsf(cdn[k]);
        if (ac > 0.f) cb[k] += ab / ac;
      }
      add3(hb[0], et * (linb / l1));
      lin_sum_b += linb;
    }
    for (int j = 1; j <= k; ++j) segb[j] += lin_sum_b;
    gw += g_a;
    if (mat.n > 0) {  // the Fresnel factor: every bounce j <= k of this path
      const float go = g_o * (float)(0.5 / M_PI);
      for (int j = 0; j <= k; ++j) {
        if (mj[j] < 0) continue;
        const float2 w = wj[j];
        const float2 qc = cdiv(make_float2(-2.f, 0.f), w);                 // d log r_s / d cos
        cb[j] += g_a * qc.x + go * qc.y;
        const float2 e = mat.eps[mj[j]];
        const float2 qe = cdiv(make_float2(fabsf(cdn[j]), 0.f), cmul(w, make_float2(e.x - 1.f, -e.y)));
        scatter_eps<kPass>(fe, Ee, emax, mj[j], g_a * qe.x + go * qe.y, g_a * qe.y - go * qe.x);
      }
    }
  }
  for (int j = 1; j < m; ++j) {
    const float3 e = h[j] - h[j - 1];
    const float3 u = e * (segb[j] / len3(e));
    add3(hb[j], u);
    hb[j - 1] = hb[j - 1] - u;
  }
  // reverse sweep over bounces
  float3 db_next = f3(0.f, 0.f, 0.f);  // adjoint of d_{k+1}
  float3 ob_next = f3(0.f, 0.f, 0.f);  // adjoint of o_{k+1} = h_k
  for (int k = m - 1; k >= 0; --k) {
    float3 db = f3(0.f, 0.f, 0.f), nb = f3(0.f, 0.f, 0.f);
    // |d.n|
    const float cbar = cb[k] * (cdn[k] >= 0.f ? 1.f : -1.f);
    float cdb = cbar;
    // reflection d_{k+1} = d_k - 2 c n
    if (k + 1 < m) {
      add3(db, db_next);
      cdb += -2.f * dot(nh[k], db_next);
      add3(nb, db_next * (-2.f * cdn[k]));
    }
    add3(db, nh[k] * cdb);
    add3(nb, d[k] * cdb);
    // h_k = o_k + t d_k
    const float3 H = hb[k] + ob_next;
    float3 ob = H;
    const float tb = dot(H, d[k]);
    add3(db, H * t[k]);
    // t = N.(a - o) / (N.d)
    const float den = dot(N[k], d[k]);
    float3 Nb = (A[k] - h[k]) * (tb / den);
    float3 ab = N[k] * (tb / den);
    ob = ob - N[k] * (tb / den);
    db = db - N[k] * (tb * t[k] / den);
    // n = N / |N|
    add3(Nb, (nb - nh[k] * dot(nb, nh[k])) * (1.f / nlen[k]));
    // N = (b - a) x (c - a)
    const float3 vb = ld3(verts, fv[k][1]), vc = ld3(verts, fv[k][2]);
    const float3 e1 = vb - A[k], e2 = vc - A[k];
    const float3 e1b = cross(e2, Nb), e2b = cross(Nb, e1);
    ab = ab - e1b - e2b;
    scatter<kPass>(fs, E, lmax, fv[k][0], ab);
    scatter<kPass>(fs, E, lmax, fv[k][1], e1b);
    scatter<kPass>(fs, E, lmax, fv[k][2], e2b);
    db_next = db;
    ob_next = ob;
  }
  if (reparam) {  // d_1 and the weight as functions of the attached point x and of N_1
    const float3 e = x0 - org;
    const float r2 = dot(e, e), r = sqrtf(r2);
    const float3 u = e * (1.f / r);
    const float s = dot(N[0], e);
    float3 xb = (db_next - u * dot(u, db_next)) * (1.f / r);
    add3(xb, (N[0] * (1.f / s) - e * (3.f / r2)) * gw);
    const float3 Nb = e * (gw / s);
    const float3 va = A[0], vb = ld3(verts, fv[0][1]), vc = ld3(verts, fv[0][2]);
    const float3 e1b = cross(vc - va, Nb), e2b = cross(Nb, vb - va);
    scatter<kPass>(fs, E, lmax, fv[0][0], xb * (1.f - bu - bv) - e1b - e2b);
    scatter<kPass>(fs, E, lmax, fv[0][1], xb * bu + e1b);
    scatter<kPass>(fs, E, lmax, fv[0][2], xb * bv + e2b);
  }
}

template <int kPass>
__global__ void __launch_bounds__(128) k_trace_bwd(
    const float* __restrict__ verts, int nv, const int32_t* __restrict__ faces, GridF g, RadarF rd, MatArg mat,
    const int32_t* __restrict__ ray_ids, int n_rays, int K, const sbr_hit* __restrict__ hits,
    const float4* __restrict__ hit_pos, const int32_t* __restrict__ first,
    const float4* __restrict__ prep, int64_t cap, const float* __restrict__ glen,
    const float* __restrict__ gamp, const float* __restrict__ gphase, bool reparam, FixScatter fs, FixScatter fe) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int E = kPass == 0 ? 0 : fix_exp(*fs.max_bits, fs.log2n);
  const int Ee = kPass == 0 ? 0 : fix_exp(*fe.max_bits, fe.log2n);
  float lmax = 0.f, emax = 0.f;
  if (i < n_rays)
    ray_adjoint<kPass>(i, verts, nv, faces, g, rd, mat, ray_ids, K, hits, hit_pos, first, prep, cap, glen, gamp,
                       gphase, reparam, fs, E, lmax, fe, Ee, emax);
  if (kPass == 0) {  // every lane of the warp reaches this
    fix_note_warp(fs.max_bits, lmax);
    if (mat.n > 0) fix_note_warp(fe.max_bits, emax);
  }
}

// gverts[i] += acc[i] 2^-E
__global__ void k_fix_finish_add(FixScatter fs, int n, float* __restrict__ gverts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  gverts[i] += fix_get(fs.acc[i], fix_exp(*fs.max_bits, fs.log2n));
}

}  // namespace
}  // namespace sbr

using namespace sbr;

namespace {
struct BwdWs {
  FixScatter fs, fe;
};
// vertex accumulators, their max word; material accumulators, their max word
size_t bwd_ws_layout(void* base, int32_t nv, BwdWs* w) {
  Carver c(base);
  w->fs.acc = c.take<unsigned long long>(3 * (size_t)nv);
  w->fs.max_bits = c.take<unsigned int>(1);
  w->fe.acc = c.take<unsigned long long>(2 * SBR_MAX_MATERIALS);
  w->fe.max_bits = c.take<unsigned int>(1);
  return c.bytes();
}
}  // namespace

extern "C" size_t sbr_trace_bwd_ws_bytes(int32_t nv) {
  if (nv < 0) return 0;
  BwdWs w;
  return bwd_ws_layout(nullptr, nv, &w);
}

extern "C" sbr_status sbr_trace_bwd(const sbr_scene* scene, const float* d_verts, const sbr_radar_cfg* radar,
                                    const sbr_ray_grid* grid, const int32_t* d_ray_ids,
                                    const sbr_paths* paths, const float* d_glen, const float* d_gamp,
                                    const float* d_gphase, float* d_gverts, float* d_geps, int32_t flags,
                                    void* d_ws, size_t ws_bytes, sbr_stream stream) {
  SBR_ARG(scene && paths && d_verts && d_glen && d_gamp && d_gverts, "sbr_trace_bwd: NULL argument");
  SBR_ARG((flags & ~SBR_BWD_REPARAM) == 0, "sbr_trace_bwd: unknown flags 0x%x", (unsigned)flags);
  const bool reparam = (flags & SBR_BWD_REPARAM) != 0;
  SBR_ARG(scene->n_mat == 0 || d_gphase,
          "sbr_trace_bwd: the scene has materials: d_gphase (sbr_synthesize_bwd's phase gradient) is required");
  SBR_ARG(d_ws && aligned256(d_ws), "sbr_trace_bwd: workspace NULL or not 256-byte aligned");
  if (ws_bytes < sbr_trace_bwd_ws_bytes(scene->nv)) {
    set_error("sbr_trace_bwd: workspace of %zu bytes, %zu needed", ws_bytes, sbr_trace_bwd_ws_bytes(scene->nv));
    return SBR_ERR_OOM;
  }
  sbr_status rs = check_radar(radar, "sbr_trace_bwd");
  if (rs != SBR_OK) return rs;
  rs = check_grid(grid, "sbr_trace_bwd");
  if (rs != SBR_OK) return rs;
  SBR_ARG(paths->max_bounces <= kMaxK, "sbr_trace_bwd: max_bounces=%d above %d", paths->max_bounces, kMaxK);
  SBR_ARG(paths->n_virt == radar->n_tx * radar->n_rx, "sbr_trace_bwd: V mismatch");
  SBR_ARG(d_ray_ids || (int64_t)paths->n_rays == (int64_t)grid->G * grid->G,
          "sbr_trace_bwd: paths cover %d rays; the grid has %lld (pass the forward's ray list)",
          paths->n_rays, (long long)grid->G * grid->G);
  if (paths->n_rays == 0) return SBR_OK;
  GridF g;
  for (int j = 0; j < 3; ++j) {
    g.o[j] = (float)grid->origin[j];
    g.ax[j] = (float)grid->axis[j];
    g.ua[j] = (float)grid->u_axis[j];
    g.va[j] = (float)grid->v_axis[j];
  }
  g.start = (float)(grid->tan_half * (1.0 / grid->G - 1.0));
  g.step = (float)(2.0 * grid->tan_half / grid->G);
  g.lo = (float)(-grid->tan_half);
  g.G = grid->G;
  g.jitter = grid->jitter;
  RadarF rd;
  for (int t = 0; t < SBR_MAX_TX; ++t)
    for (int j = 0; j < 3; ++j) rd.tx[t][j] = (float)radar->tx[t][j];
  for (int r = 0; r < SBR_MAX_RX; ++r)
    for (int j = 0; j < 3; ++j) rd.rx[r][j] = (float)radar->rx[r][j];
  rd.ntx = radar->n_tx;
  rd.nrx = radar->n_rx;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int R = paths->n_rays;
  BwdWs w;
  bwd_ws_layout(d_ws, scene->nv, &w);
  w.fs.log2n = ceil_log2(3 * (int64_t)R * (paths->max_bounces + (reparam ? 1 : 0)));  // contributions per axis, at most
  w.fe.log2n = ceil_log2((int64_t)R * paths->max_bounces * paths->max_bounces);  // per material, at most
  const MatArg mat = mat_arg(scene);
  SBR_CUDA(cudaMemsetAsync(d_ws, 0, sbr_trace_bwd_ws_bytes(scene->nv), st));
  const float4* hp = reinterpret_cast<const float4*>(paths->hit_pos);
  const float4* pr = reinterpret_cast<const float4*>(paths->prep);
  ::sbr::note_launch();
  k_trace_bwd<0><<<(R + 127) / 128, 128, 0, st>>>(d_verts, scene->nv, scene->faces, g, rd, mat, d_ray_ids, R,
                                                   paths->max_bounces, paths->hits, hp, paths->ray_first, pr,
                                                   paths->path_cap, d_glen, d_gamp, d_gphase, reparam, w.fs, w.fe);
  ::sbr::note_launch();
  k_trace_bwd<1><<<(R + 127) / 128, 128, 0, st>>>(d_verts, scene->nv, scene->faces, g, rd, mat, d_ray_ids, R,
                                                   paths->max_bounces, paths->hits, hp, paths->ray_first, pr,
                                                   paths->path_cap, d_glen, d_gamp, d_gphase, reparam, w.fs, w.fe);
  const int n3 = 3 * scene->nv;
  if (n3 > 0) {
    ::sbr::note_launch();
    k_fix_finish_add<<<(n3 + 255) / 256, 256, 0, st>>>(w.fs, n3, d_gverts);
  }
  if (mat.n > 0 && d_geps) {
    ::sbr::note_launch();
    k_fix_finish_add<<<1, 64, 0, st>>>(w.fe, 2 * mat.n, d_geps);
  }
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}
