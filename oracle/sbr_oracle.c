/*
 * FP64 CPU oracle for the shooting-and-bouncing-rays (SBR) radar simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the bench's CPU-baseline leg may load it; the product
 * path never does.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes (every step in double precision, brute force):
 *   - the stratified ray sample set of the Monte-Carlo path integral
 *     (Section 3.2.1, Eq. 2-3) as a G x G grid of cell-centre directions, each
 *     weighted by its solid angle (cell area on the unit plane times cos^3);
 *   - for every ray, up to K specular surface interactions, each found by
 *     testing the ray against EVERY triangle with the Moller-Trumbore (1997)
 *     two-sided test, nearest hit wins, exact ties go to the lower triangle
 *     index, the previously hit triangle is skipped;
 *   - the FMCW IF signal of Eq. 8, S[v,n] = sum_p A_p exp(j 2 pi (f_c tau_p +
 *     mu tau_p t_n)), as a direct double-precision sum over every path;
 *   - the analytic derivatives of Eq. 11-12 contracted with an upstream
 *     gradient (the synthesis adjoint).
 *
 * Ray-level flags: a ray is marked "ambiguous from bounce k" when, at bounce k,
 * its hit lies within edge_eps of a triangle edge in barycentric terms
 * (min(u, v, 1-u-v) < edge_eps) or a different triangle is hit within a
 * relative distance tie_rel of the nearest one.  Such rays are excluded from
 * bit-exact triangle-index comparisons.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double x, y, z; } d3;

static inline d3 v3(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static inline d3 vsub(d3 a, d3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline d3 vadd(d3 a, d3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline d3 vmul(d3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static inline double vdot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline d3 vcross(d3 a, d3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double vlen(d3 a) { return sqrt(vdot(a, a)); }

static inline d3 vert(const float* verts, int i) {
  return v3((double)verts[3 * i], (double)verts[3 * i + 1], (double)verts[3 * i + 2]);
}

/* Moller-Trumbore ray/triangle test in FP64, two-sided.  Returns 1 on a hit. */
static int mt_hit(d3 o, d3 d, d3 a, d3 b, d3 c, double tmin,
                  double* t_out, double* u_out, double* v_out) {
  d3 e1 = vsub(b, a), e2 = vsub(c, a);
  d3 p = vcross(d, e2);
  double det = vdot(e1, p);
  if (fabs(det) < 1e-12) return 0;
  double inv = 1.0 / det;
  d3 s = vsub(o, a);
  double u = vdot(s, p) * inv;
  if (u < 0.0 || u > 1.0) return 0;
  d3 q = vcross(s, e1);
  double v = vdot(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return 0;
  double t = vdot(e2, q) * inv;
  if (t <= tmin) return 0;
  *t_out = t; *u_out = u; *v_out = v;
  return 1;
}

/* Launch direction and solid-angle weight of ray `rid` of a G x G grid.
 * grid = [origin(3), axis(3), u_axis(3), v_axis(3), tan_half]; jitter = the
 * rays' offsets (jx, jy) in their cells (stratified jittered sampling of the
 * Monte-Carlo estimate of Eq. 3), or NULL for the cell centres (1/2, 1/2). */
static void grid_ray(const double* grid, int G, const float* jitter, int rid, d3* o, d3* d, double* omega) {
  int row = rid / G, col = rid % G;
  double th = grid[12];
  double jx = jitter ? (double)jitter[2 * (size_t)rid] : 0.5;
  double jy = jitter ? (double)jitter[2 * (size_t)rid + 1] : 0.5;
  double a = th * (2.0 * (col + jx) / G - 1.0);
  double b = th * (2.0 * (row + jy) / G - 1.0);
  d3 ax = v3(grid[3], grid[4], grid[5]);
  d3 ua = v3(grid[6], grid[7], grid[8]);
  d3 va = v3(grid[9], grid[10], grid[11]);
  d3 w = vadd(ax, vadd(vmul(ua, a), vmul(va, b)));
  double len = vlen(w);
  *o = v3(grid[0], grid[1], grid[2]);
  *d = vmul(w, 1.0 / len);
  double cell = 2.0 * th / G;
  *omega = cell * cell / (len * len * len);
}

/*
 * Brute-force trace.  For n_rays rays (ray_ids[i], or i when ray_ids is NULL)
 * and up to K bounces writes, per (ray, bounce) slot i*K+k:
 *   tri[i*K+k]        nearest triangle or -1 (and -1 for every later bounce)
 *   tuv[3*(i*K+k)+]   t, u, v of that hit
 *   hit[3*(i*K+k)+]   hit point o + t d
 *   din[3*(i*K+k)+]   incident (unit) direction d_k
 *   nrm[3*(i*K+k)+]   unit geometric normal (e1 x e2)/|e1 x e2|
 * and per ray omega[i] (solid-angle weight) and flag[i] (first ambiguous
 * bounce, 1-based, or 0).
 */
int orc_trace(const float* verts, int nv, const int* faces, int nt,
              const double* grid, int G, const float* jitter, const int* ray_ids, int n_rays, int K,
              double tmin, double edge_eps, double tie_rel,
              int* tri, double* tuv, double* hit, double* din, double* nrm,
              double* omega, int* flag) {
  if (!verts || !faces || !grid || nt < 0 || nv < 0 || K < 1 || G < 1) return 1;
  for (int f = 0; f < 3 * nt; ++f)
    if (faces[f] < 0 || faces[f] >= nv) return 2;
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n_rays; ++i) {
    int rid = ray_ids ? ray_ids[i] : i;
    d3 o, d;
    grid_ray(grid, G, jitter, rid, &o, &d, &omega[i]);
    flag[i] = 0;
    int prev = -1, alive = 1;
    for (int k = 0; k < K; ++k) {
      size_t s = (size_t)i * K + k;
      tri[s] = -1;
      tuv[3 * s] = tuv[3 * s + 1] = tuv[3 * s + 2] = 0.0;
      hit[3 * s] = hit[3 * s + 1] = hit[3 * s + 2] = 0.0;
      din[3 * s] = d.x; din[3 * s + 1] = d.y; din[3 * s + 2] = d.z;
      nrm[3 * s] = nrm[3 * s + 1] = nrm[3 * s + 2] = 0.0;
      if (!alive) continue;
      int best = -1;
      double bt = INFINITY, bu = 0, bv = 0, second = INFINITY;
      for (int f = 0; f < nt; ++f) {
        if (f == prev) continue;
        double t, u, v;
        d3 a = vert(verts, faces[3 * f]), b = vert(verts, faces[3 * f + 1]),
           c = vert(verts, faces[3 * f + 2]);
        if (!mt_hit(o, d, a, b, c, tmin, &t, &u, &v)) continue;
        if (t < bt) {            /* strictly nearer: the lower index keeps exact ties */
          second = bt;
          bt = t; bu = u; bv = v; best = f;
        } else if (t < second) {
          second = t;
        }
      }
      if (best < 0) { alive = 0; continue; }
      double w = 1.0 - bu - bv;
      double mn = bu < bv ? bu : bv;
      mn = mn < w ? mn : w;
      if (!flag[i] && (mn < edge_eps || second - bt <= tie_rel * bt)) flag[i] = k + 1;
      d3 a = vert(verts, faces[3 * best]), b = vert(verts, faces[3 * best + 1]),
         c = vert(verts, faces[3 * best + 2]);
      d3 n = vcross(vsub(b, a), vsub(c, a));
      n = vmul(n, 1.0 / vlen(n));
      d3 h = vadd(o, vmul(d, bt));
      tri[s] = best;
      tuv[3 * s] = bt; tuv[3 * s + 1] = bu; tuv[3 * s + 2] = bv;
      hit[3 * s] = h.x; hit[3 * s + 1] = h.y; hit[3 * s + 2] = h.z;
      nrm[3 * s] = n.x; nrm[3 * s + 1] = n.y; nrm[3 * s + 2] = n.z;
      /* specular reflection d' = d - 2 (d.n) n, next origin = hit point */
      d = vsub(d, vmul(n, 2.0 * vdot(d, n)));
      o = h;
      prev = best;
    }
  }
  return 0;
}

/*
 * Eq. 8 as a direct FP64 sum: for every virtual antenna v and sample n,
 *   S[v,n] = sum_p amp[v*P+p] * exp(j 2 pi (f0 tau + mu tau t_n)),  t_n = n / fs,
 * with the phase reduced as x - nearbyint(x) before sin/cos.
 */
int orc_synth(const double* tau, const double* amp, long P, int V, double f0, double mu,
              double fs, int Ns, double* out_re, double* out_im) {
  if (P < 0 || V < 1 || Ns < 1) return 1;
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for collapse(2) schedule(static)
  for (int v = 0; v < V; ++v) {
    for (int n = 0; n < Ns; ++n) {
      double tn = (double)n / fs, re = 0.0, im = 0.0;
      for (long p = 0; p < P; ++p) {
        double t = tau[(size_t)v * P + p];
        double x = f0 * t + mu * t * tn;
        double fr = x - nearbyint(x);
        re += amp[(size_t)v * P + p] * cos(two_pi * fr);
        im += amp[(size_t)v * P + p] * sin(two_pi * fr);
      }
      out_re[(size_t)v * Ns + n] = re;
      out_im[(size_t)v * Ns + n] = im;
    }
  }
  return 0;
}

/*
 * Adjoint of Eq. 8 through the analytic derivatives of Eq. 11-12.  For a real
 * scalar loss with upstream gradient g[v,n] = dL/dRe S + j dL/dIm S:
 *   dL/dA_p   = sum_n Re( conj(g) * exp(j phi) )                       (Eq. 12)
 *   dL/dtau_p = sum_n Re( conj(g) * j 2 pi (mu t_n + f0) A exp(j phi) ) (Eq. 11)
 */
int orc_synth_grad(const double* tau, const double* amp, long P, int V, double f0, double mu,
                   double fs, int Ns, const double* g_re, const double* g_im,
                   double* gtau, double* gamp) {
  if (P < 0 || V < 1 || Ns < 1) return 1;
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for collapse(2) schedule(static)
  for (int v = 0; v < V; ++v) {
    for (long p = 0; p < P; ++p) {
      double t = tau[(size_t)v * P + p], a = amp[(size_t)v * P + p];
      double sa = 0.0, st = 0.0;
      for (int n = 0; n < Ns; ++n) {
        double tn = (double)n / fs;
        double x = f0 * t + mu * t * tn;
        double fr = x - nearbyint(x);
        double c = cos(two_pi * fr), s = sin(two_pi * fr);
        double gr = g_re[(size_t)v * Ns + n], gi = g_im[(size_t)v * Ns + n];
        /* Re(conj(g) e) = gr c + gi s;  Re(conj(g) j e) = gr (-s) + gi c */
        sa += gr * c + gi * s;
        st += two_pi * (mu * tn + f0) * a * (gi * c - gr * s);
      }
      gamp[(size_t)v * P + p] = sa;
      gtau[(size_t)v * P + p] = st;
    }
  }
  return 0;
}

/* Thread count of the OpenMP loops above (n >= 1; anything else leaves it); returns the count
 * in force before the call.  Used to time the oracle on one core beside all of them. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  int prev = omp_get_max_threads();
  if (n >= 1) omp_set_num_threads(n);
  return prev;
#else
  (void)n;
  return 1;
#endif
}
