// FMCW IF synthesis (Section 3.2.2, Eq. 8) and its adjoint (Eq. 11-12).
//
// cube[v, c, n] = sum_p A_{p,v} exp(j 2 pi (f_c tau_{p,v} + mu tau_{p,v} t_n)),
// t_n = n T / N_s, identical for every chirp c of a static scene.
//
// Split-phase mode, N_s <= 512 (sbr_synthesize's default path): a type-1
// non-uniform FFT.  Each (path, antenna) is spread onto a periodic grid of
// 2 N_s points with a width-8 exponential-of-semicircle kernel, one FFT per
// antenna follows, and the kernel's Fourier transform is divided out: 8 grid
// updates per (path, antenna) instead of N_s phasors, about 1e-6 from the FP64
// sum (details at k_nufft_spread).
//
// Tensor-core kernel (N_s = 256 or 512, run by the allocation-free entry
// point): with n = 16 a + b (b < 16), Eq. 8 factorises per path into
// U_p[a] W_p[b] with U_p[a] = A e^{j 2 pi (phi0 + 16 a delta)} and
// W_p[b] = e^{j 2 pi b delta}, so each antenna's samples are the complex matrix
// product sum_p U_p W_p^T, a GEMM whose contraction runs over the paths.
// Written as a real GEMM with rows (Re, Im) x a, columns b and two contraction
// entries (Re, Im) per path, it goes to mma.sync m16n8k16 with every operand
// split into two fp16 halves (hi + lo, three products hi.hi + hi.lo + lo.hi:
// ~21-bit products) and FP32 accumulation; amplitudes are scaled by a power of
// two per staged chunk so the halves stay in fp16 range (the accumulators are
// rescaled exactly when the scale drops).
//
// Direct FP32 kernel (other sample counts; persistent, one virtual antenna per
// CTA): the CTA's threads own M consecutive samples each and together cover
// all N_s samples, so the sum over paths accumulates in registers with no
// cross-thread reduction.  Paths stream through shared memory in chunks; per
// (path, thread) one split-precision anchor phase (n0 delta_hi is exact in
// FP32, frac() before the low part and phi0 are added) goes through one sincos,
// and the remaining M-1 samples follow by complex rotation with the per-path
// step e^{j 2 pi delta} (4 FP32 multiply/FMA per sample instead of two
// transcendental ops).
//
// Every evaluation writes per-CTA partial sums (or grids) that a second kernel
// adds in a fixed order, so the result is bitwise reproducible.
#include <cuda_fp16.h>
#include <limits.h>
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "fft.cuh"

namespace sbr {
namespace {

constexpr int kChunk = 512;  // paths staged per chunk (16 KB of shared memory per CTA)
constexpr float kTwoPiF = 6.28318530717958647692f;

// threads per sample group: N_s / 16 (16 samples each), at least 16, at most 256
inline int threads_for(int Ns) {
  int t = Ns / 16;
  return t < 16 ? 16 : (t > 256 ? 256 : t);
}

// Samples after the anchor follow the two-term recurrence of a sampled
// sinusoid, e_{m+1} = 2 cos(w) e_m - e_{m-1} (w = 2 pi delta), one FMA per
// component per sample; its rounding error grows at most linearly in the
// number of steps (|sin(m w) / sin(w)| <= m), so M <= 16 keeps it near 1e-6.
// A CTA has kSplitThreads threads in G = kSplitThreads / (N_s / M) sample
// groups; every group covers all N_s samples and takes every G-th path of each
// staged chunk, and the groups' sums are added through shared memory at the
// end.  (One group per CTA would cap residency at 32 CTAs x 32 threads.)
constexpr int kSplitThreads = 256;

template <int M>
__global__ void __launch_bounds__(kSplitThreads) k_synth_split(const float4* __restrict__ prep, int64_t cap,
                                                               const int32_t* __restrict__ d_P, int V,
                                                               int Q, int Ns, float2* __restrict__ partial) {
  __shared__ float4 sp[kChunk];
  __shared__ float4 sstep[kChunk];  // cos w, sin w, 2 cos w
  extern __shared__ float2 red[];   // [M][kSplitThreads] when G > 1
  const int T = Ns / M, G = kSplitThreads / T;
  const int g = threadIdx.x / T, lane = threadIdx.x - g * T;
  const int v = blockIdx.x % V, q = blockIdx.x / V;
  const int64_t P = *d_P;
  const int n0 = lane * M;
  const float fn0 = (float)n0;
  // (re, im) pairs advance with packed FP32x2 instructions: one FADD2 per
  // accumulated sample and one FFMA2 per recurrence step
  float2 acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = make_float2(0.f, 0.f);
  const float4* pv = prep + (size_t)v * cap;
  for (int64_t c0 = (int64_t)q * kChunk; c0 < P; c0 += (int64_t)Q * kChunk) {
    const int cnt = (int)min((int64_t)kChunk, P - c0);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const float4 r = pv[c0 + j];
      sp[j] = r;
      float s, c;
      sincospif(2.f * (r.y + r.z), &s, &c);
      sstep[j] = make_float4(c, s, 2.f * c, 0.f);
    }
    __syncthreads();
#pragma unroll 2
    for (int j = g; j < cnt; j += G) {
      const float4 r = sp[j];
      const float4 st = sstep[j];
      float x = fn0 * r.y;  // exact: delta_hi is a multiple of 2^-12 and n0 < 4096
      x -= rintf(x);
      x = fmaf(fn0, r.z, x) + r.x;
      x -= rintf(x);
      float s, c;
      __sincosf(kTwoPiF * x, &s, &c);
      float2 ep = __fmul2_rn(make_float2(r.w, r.w), make_float2(c, s));  // e_0
      acc[0] = __fadd2_rn(acc[0], ep);
      if (M > 1) {
        // e_1 = e_0 e^{jw}
        float2 e = __ffma2_rn(make_float2(-ep.y, ep.y), make_float2(st.y, st.x),
                              __fmul2_rn(make_float2(ep.x, ep.x), make_float2(st.x, st.y)));
        const float2 c2 = make_float2(st.z, st.z);
#pragma unroll
        for (int m = 1; m < M; ++m) {
          acc[m] = __fadd2_rn(acc[m], e);
          if (m + 1 < M) {
            const float2 en = __ffma2_rn(c2, e, make_float2(-ep.x, -ep.y));
            ep = e;
            e = en;
          }
        }
      }
    }
  }
  if (G > 1) {  // add the groups' sums (fixed order: deterministic)
    __syncthreads();
#pragma unroll
    for (int m = 0; m < M; ++m) red[m * kSplitThreads + threadIdx.x] = acc[m];
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float2 sum = make_float2(0.f, 0.f);
      for (int gg = 0; gg < G; ++gg) sum = __fadd2_rn(sum, red[m * kSplitThreads + gg * T + lane]);
      acc[m] = sum;
    }
  }
  float2* out = partial + (size_t)blockIdx.x * Ns + n0;
#pragma unroll
  for (int m = 0; m < M; ++m) out[m] = acc[m];
}

// ---- tensor-core forward kernel ---------------------------------------------

// fp16 pair (x0, x1) as hi + lo halves packed in f16x2 registers (lower index low)
__device__ inline void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// c += a b for one m16n8k16 tile (fp16 operands, FP32 accumulators)
__device__ inline void mma_f16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kMmaThreads = 256;

// MT m16 tiles of a per (Re | Im) block: N_s = 256 MT.  Warp lane (g = lane / 4,
// t = lane % 4) holds, for the 8-path group of one mma k-step, paths 2t and
// 2t + 1 (contraction columns 2t, 2t + 1 for Re and 2t + 8, 2t + 9 for Im),
// rows a = 16 m + g and 16 m + g + 8 of U, and columns b = g, g + 8 of W.
template <int MT>
__global__ void __launch_bounds__(kMmaThreads) k_synth_mma(const float4* __restrict__ prep, int64_t cap,
                                                           const int32_t* __restrict__ d_P, int V, int Q,
                                                           float2* __restrict__ partial) {
  constexpr int Ns = 256 * MT, NU = 2 * MT;  // U values per (thread, path): a = g + 8 i
  constexpr int kWarps = kMmaThreads / 32;
  // staged records and steps; at the end the warps' sums ([warp][n][Re, Im])
  constexpr int kRed = kWarps * 2 * Ns / 4, kSbuf = kRed > 2 * kChunk ? kRed : 2 * kChunk;
  __shared__ float4 sbuf[kSbuf];
  __shared__ uint32_t wmax[kWarps];
  float4* sp = sbuf;
  float4* sst = sbuf + kChunk;  // e^{j 2 pi 8 delta}, e^{j 2 pi 128 delta}
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int v = blockIdx.x % V, q = blockIdx.x / V;
  const int64_t P = *d_P;
  float acc[2][MT][2][4];  // [Re | Im][m tile][n tile][fragment]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[a][m][c][d] = 0.f;
  int s_run = 126;  // the accumulators hold the sums times 2^s_run
  const float4* pv = prep + (size_t)v * cap;
  const float fa = 16.f * (float)g, fg = (float)g;
  for (int64_t c0 = (int64_t)q * kChunk; c0 < P; c0 += (int64_t)Q * kChunk) {
    const int cnt = (int)min((int64_t)kChunk, P - c0);
    __syncthreads();
    uint32_t m = 0;
    for (int j = threadIdx.x; j < kChunk; j += blockDim.x) {
      const float4 r = j < cnt ? pv[c0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
      sp[j] = r;
      m = max(m, __float_as_uint(fabsf(r.w)));
      float x8 = 8.f * r.y;  // exact: delta_hi is a multiple of 2^-12
      x8 -= rintf(x8);
      x8 = fmaf(8.f, r.z, x8);
      float x128 = 128.f * r.y;  // exact
      x128 -= rintf(x128);
      x128 = fmaf(128.f, r.z, x128);
      x128 -= rintf(x128);
      float s8, c8, s128, c128;
      __sincosf(kTwoPiF * x8, &s8, &c8);
      __sincosf(kTwoPiF * x128, &s128, &c128);
      sst[j] = make_float4(c8, s8, c128, s128);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    m = wmax[0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) m = max(m, wmax[w]);
    if (m == 0u) continue;  // every amplitude of the chunk is zero
    // the chunk's largest |A| lands in [2^14, 2^15): in fp16 range with room for the lo halves
    const int s_c = 14 - ilogbf(__uint_as_float(m));
    if (s_c < s_run) {
      const float f = s_run > 125 ? 1.f : ldexpf(1.f, s_c - s_run);  // exact power of two
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int mm = 0; mm < MT; ++mm)
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int d = 0; d < 4; ++d) acc[a][mm][c][d] *= f;
      s_run = s_c;
    }
    const float scale = ldexpf(1.f, s_run);
    const int groups = (cnt + 7) >> 3;
    for (int gr = warp; gr < groups; gr += kWarps) {
      float ur[2][NU], ui[2][NU], wr[2][2], wi[2][2];  // [path 2t + h][a index | b = g, g + 8]
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 8 * gr + 2 * t + h;  // < kChunk; zero records beyond cnt add nothing
        const float4 r = sp[j];
        const float4 st = sst[j];
        float x = fa * r.y;  // exact: 16 g < 128
        x -= rintf(x);
        x = fmaf(fa, r.z, x) + r.x;
        x -= rintf(x);
        float su, cu;
        __sincosf(kTwoPiF * x, &su, &cu);
        const float A = r.w * scale;
        ur[h][0] = A * cu;
        ui[h][0] = A * su;
#pragma unroll
        for (int i = 1; i < NU; ++i) {  // a + 8: n + 128
          ur[h][i] = fmaf(ur[h][i - 1], st.z, -ui[h][i - 1] * st.w);
          ui[h][i] = fmaf(ur[h][i - 1], st.w, ui[h][i - 1] * st.z);
        }
        float y = fg * r.y;  // exact
        y -= rintf(y);
        y = fmaf(fg, r.z, y);
        y -= rintf(y);
        float sw, cw;
        __sincosf(kTwoPiF * y, &sw, &cw);
        wr[h][0] = cw;
        wi[h][0] = sw;
        wr[h][1] = fmaf(cw, st.x, -sw * st.y);  // b + 8
        wi[h][1] = fmaf(cw, st.y, sw * st.x);
      }
      uint32_t Bh[2][2], Bl[2][2];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        split_h2(wr[0][nt], wr[1][nt], Bh[nt][0], Bl[nt][0]);
        split_h2(wi[0][nt], wi[1][nt], Bh[nt][1], Bl[nt][1]);
      }
      constexpr uint32_t kNeg = 0x80008000u;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        uint32_t urh[2], url[2], uih[2], uil[2];
        split_h2(ur[0][2 * mt], ur[1][2 * mt], urh[0], url[0]);
        split_h2(ur[0][2 * mt + 1], ur[1][2 * mt + 1], urh[1], url[1]);
        split_h2(ui[0][2 * mt], ui[1][2 * mt], uih[0], uil[0]);
        split_h2(ui[0][2 * mt + 1], ui[1][2 * mt + 1], uih[1], uil[1]);
        // Re rows take (Re U, -Im U) against (Re W, Im W); Im rows take (Im U, Re U)
        const uint32_t Ah_re[4] = {urh[0], urh[1], uih[0] ^ kNeg, uih[1] ^ kNeg};
        const uint32_t Al_re[4] = {url[0], url[1], uil[0] ^ kNeg, uil[1] ^ kNeg};
        const uint32_t Ah_im[4] = {uih[0], uih[1], urh[0], urh[1]};
        const uint32_t Al_im[4] = {uil[0], uil[1], url[0], url[1]};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const uint32_t bh[2] = {Bh[nt][0], Bh[nt][1]}, bl[2] = {Bl[nt][0], Bl[nt][1]};
          mma_f16(acc[0][mt][nt], Ah_re, bh);
          mma_f16(acc[0][mt][nt], Ah_re, bl);
          mma_f16(acc[0][mt][nt], Al_re, bh);
          mma_f16(acc[1][mt][nt], Ah_im, bh);
          mma_f16(acc[1][mt][nt], Ah_im, bl);
          mma_f16(acc[1][mt][nt], Al_im, bh);
        }
      }
    }
  }
  // undo the scale, then add the warps' sums in a fixed order through shared memory
  const float unscale = s_run > 125 ? 0.f : ldexpf(1.f, -s_run);
  __syncthreads();
  float* red = reinterpret_cast<float*>(sbuf);  // [warp][n][Re, Im]
#pragma unroll
  for (int part = 0; part < 2; ++part)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int a = 16 * mt + g + ((e & 2) ? 8 : 0);
          const int b = 8 * nt + 2 * t + (e & 1);
          red[warp * 2 * Ns + 2 * (16 * a + b) + part] = acc[part][mt][nt][e] * unscale;
        }
  __syncthreads();
  float2* out = partial + (size_t)blockIdx.x * Ns;
  for (int n = threadIdx.x; n < Ns; n += blockDim.x) {
    float re = 0.f, im = 0.f;
    for (int w = 0; w < kWarps; ++w) {
      re += red[w * 2 * Ns + 2 * n];
      im += red[w * 2 * Ns + 2 * n + 1];
    }
    out[n] = make_float2(re, im);
  }
}

// Per-sample phase in FP64: x = f_c tau + (B / N_s) tau n, reduced mod 1.
template <int M>
__global__ void __launch_bounds__(256) k_synth_fp64(const float4* __restrict__ prep,
                                                    const float2* __restrict__ plen,
                                                    const float* __restrict__ phase_ofs, int64_t cap,
                                                    const int32_t* __restrict__ d_P, int V, int Q,
                                                    int Ns, double f0, double b_over_ns,
                                                    float2* __restrict__ partial,
                                                    const float* __restrict__ rate = nullptr,
                                                    double crep = 0.0) {
  __shared__ double2 sx[kChunk];
  __shared__ float sa[kChunk];
  const int v = blockIdx.x % V, q = blockIdx.x / V;
  const int64_t P = *d_P;
  const int n0 = threadIdx.x * M;
  float accr[M], acci[M];
#pragma unroll
  for (int m = 0; m < M; ++m) accr[m] = acci[m] = 0.f;
  for (int64_t c0 = (int64_t)q * kChunk; c0 < P; c0 += (int64_t)Q * kChunk) {
    const int cnt = (int)min((int64_t)kChunk, P - c0);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const float2 L = plen[(size_t)v * cap + c0 + j];
      double t = ((double)L.x + (double)L.y) * (1.0 / kC);
      if (rate) t += crep * (double)rate[(size_t)v * cap + c0 + j];  // this chirp's delay
      const double x0 = f0 * t;
      const double d = b_over_ns * t;
      sx[j] = make_double2(x0 - rint(x0) + (double)phase_ofs[c0 + j], d - rint(d));
      sa[j] = prep[(size_t)v * cap + c0 + j].w;
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const double2 xd = sx[j];
      const float a = sa[j];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        double x = fma((double)(n0 + m), xd.y, xd.x);
        x -= rint(x);
        float s, c;
        __sincosf(kTwoPiF * (float)x, &s, &c);
        accr[m] = fmaf(a, c, accr[m]);
        acci[m] = fmaf(a, s, acci[m]);
      }
    }
  }
  float2* out = partial + (size_t)blockIdx.x * Ns + n0;
#pragma unroll
  for (int m = 0; m < M; ++m) out[m] = make_float2(accr[m], acci[m]);
}

// Everything in FP32: tau, f_c tau and mu tau t_n (no split, no FP64).
template <int M>
__global__ void __launch_bounds__(256) k_synth_naive(const float4* __restrict__ prep,
                                                     const float2* __restrict__ plen,
                                                     const float* __restrict__ phase_ofs, int64_t cap,
                                                     const int32_t* __restrict__ d_P, int V, int Q,
                                                     int Ns, float f0, float mu, float dt,
                                                     float2* __restrict__ partial) {
  __shared__ float2 sx[kChunk];
  __shared__ float so[kChunk];
  const int v = blockIdx.x % V, q = blockIdx.x / V;
  const int64_t P = *d_P;
  const int n0 = threadIdx.x * M;
  float accr[M], acci[M];
#pragma unroll
  for (int m = 0; m < M; ++m) accr[m] = acci[m] = 0.f;
  for (int64_t c0 = (int64_t)q * kChunk; c0 < P; c0 += (int64_t)Q * kChunk) {
    const int cnt = (int)min((int64_t)kChunk, P - c0);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      sx[j] = make_float2(plen[(size_t)v * cap + c0 + j].x * (float)(1.0 / kC), prep[(size_t)v * cap + c0 + j].w);
      so[j] = phase_ofs[c0 + j];
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const float t = sx[j].x, a = sx[j].y, o = so[j];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        float x = fmaf(mu * t, (float)(n0 + m) * dt, f0 * t) + o;
        x -= rintf(x);
        float s, c;
        __sincosf(kTwoPiF * x, &s, &c);
        accr[m] = fmaf(a, c, accr[m]);
        acci[m] = fmaf(a, s, acci[m]);
      }
    }
  }
  float2* out = partial + (size_t)blockIdx.x * Ns + n0;
#pragma unroll
  for (int m = 0; m < M; ++m) out[m] = make_float2(accr[m], acci[m]);
}

// One thread per (antenna, sample) and group of kRedChirps chirps: the Q per-CTA
// partial sums added in a fixed order (bitwise reproducible), then written to
// the group's chirps (a static scene: every chirp equal).
constexpr int kRedChirps = 16;
__global__ void k_reduce(const float2* __restrict__ partial, int V, int Q, int Ns, int C,
                         float2* __restrict__ cube, int only = -1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * Ns) return;
  const int v = i / Ns, n = i - v * Ns;
  float re = 0.f, im = 0.f;
  for (int q = 0; q < Q; ++q) {
    const float2 x = partial[((size_t)q * V + v) * Ns + n];
    re += x.x;
    im += x.y;
  }
  if (only >= 0) {  // a moving scene: this chirp only
    cube[((size_t)v * C + only) * Ns + n] = make_float2(re, im);
    return;
  }
  const int c1 = min(C, (int)(blockIdx.y + 1) * kRedChirps);
  for (int c = blockIdx.y * kRedChirps; c < c1; ++c) cube[((size_t)v * C + c) * Ns + n] = make_float2(re, im);
}

inline dim3 reduce_grid(int V, int Ns, int C) {
  return dim3((V * Ns + 255) / 256, (C + kRedChirps - 1) / kRedChirps);
}

// ---- adjoint ----------------------------------------------------------------

__global__ void k_chirp_sum(const float2* __restrict__ g, int V, int C, int Ns,
                            float2* __restrict__ gs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * Ns) return;
  const int v = i / Ns, n = i - v * Ns;
  float re = 0.f, im = 0.f;
  for (int c = 0; c < C; ++c) {
    const float2 x = g[((size_t)v * C + c) * Ns + n];
    re += x.x;
    im += x.y;
  }
  gs[i] = make_float2(re, im);
}

// One thread per (path, antenna): Eq. 12 gives dL/dA = sum_n Re(conj(g_n) e_n),
// Eq. 11 gives dL/dtau = 2 pi A sum_n (f_c + mu t_n) Re(conj(g_n) j e_n); the
// phasor e_n runs by rotation and is re-anchored from the split phase every 32
// samples.  Output per metre of path: dL/dL = dL/dtau / c.
__global__ void __launch_bounds__(256) k_synth_bwd(const float4* __restrict__ prep, int64_t cap,
                                                   const int32_t* __restrict__ d_P, int Ns,
                                                   const float2* __restrict__ gs, float inv_lambda,
                                                   float b_over_cns, float* __restrict__ glen,
                                                   float* __restrict__ gamp, float* __restrict__ gphase) {
  extern __shared__ float2 sg[];
  const int v = blockIdx.y;
  for (int n = threadIdx.x; n < Ns; n += blockDim.x) sg[n] = gs[(size_t)v * Ns + n];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= *d_P) return;
  const float4 r = prep[(size_t)v * cap + p];
  float ss, cs;
  sincospif(2.f * (r.y + r.z), &ss, &cs);
  float sa = 0.f, s0 = 0.f, s1 = 0.f;
  for (int nb = 0; nb < Ns; nb += 32) {
    const float fn = (float)nb;
    float x = fn * r.y;
    x -= rintf(x);
    x = fmaf(fn, r.z, x) + r.x;
    x -= rintf(x);
    float s, c;
    __sincosf(kTwoPiF * x, &s, &c);
    float t0 = 0.f, t1 = 0.f;
#pragma unroll 8
    for (int m = 0; m < 32; ++m) {
      const float2 g = sg[nb + m];
      sa = fmaf(g.x, c, fmaf(g.y, s, sa));
      const float im = fmaf(g.y, c, -g.x * s);
      t0 += im;
      t1 = fmaf((float)m, im, t1);
      const float nc = fmaf(c, cs, -s * ss);
      const float ns = fmaf(c, ss, s * cs);
      c = nc;
      s = ns;
    }
    s0 += t0;
    s1 += fmaf(fn, t0, t1);
  }
  gamp[(size_t)v * cap + p] = sa;
  glen[(size_t)v * cap + p] = kTwoPiF * r.w * fmaf(inv_lambda, s0, b_over_cns * s1);
  // a phase offset o (cycles) enters every sample as e^{j 2 pi o}: dL/do = 2 pi A sum_n Re(conj(g_n) j e_n)
  if (gphase) gphase[(size_t)v * cap + p] = kTwoPiF * r.w * s0;
}

// ---- non-uniform FFT forward kernel -----------------------------------------
//
// For the split-phase mode with N_s <= 512 the samples are computed as a type-1
// non-uniform FFT (Dutt & Rokhlin 1993; kernel of Barnett, Magland & af Klinteberg
// 2019) instead of term by term.  With n = n' + N_s / 2 (n' in [-N_s/2, N_s/2)),
//   S[n] = sum_p c_p e^{j 2 pi n' delta_p},  c_p = A_p e^{j 2 pi (phi0_p + (N_s/2) delta_p)},
// every path is spread onto a periodic grid of M = 2 N_s points, u_p = M delta_p,
//   b[l] = sum_p c_p psi(l - u_p),  psi(x) = exp(beta (sqrt(1 - (2x/w)^2) - 1)), |x| < w/2,
// then B[k] = sum_l b[l] e^{+j 2 pi k l / M} (one M-point FFT) and, by Poisson
// summation, S[n' + N_s/2] = B[n'] / Psi(n'/M) with Psi the Fourier transform of
// psi, up to the aliasing terms Psi(n'/M - k), k != 0 (about 1e-7 relative for
// w = 8, beta = 2.3 w at upsampling 2).  Per (path, antenna) that is w = 8 kernel
// values instead of N_s phasors.
//
// The grid position keeps the split phase's precision: M delta_hi is exact in
// FP32 (delta_hi is a multiple of 2^-12, M <= 1024), so the offset of the path
// from its grid cell, t = (M delta_hi - floor(M delta_hi)) + M delta_lo, carries
// about 2^-24 of one grid step.
//
// Each warp spreads into its own grid in shared memory (no atomics): its lanes
// form four groups of w = 8, one grid point per lane; each group takes eight
// consecutive paths of the warp's batch of 32 in turn.  Neighbouring rays sit
// at nearly the same range, so consecutive paths mostly share a grid cell: a
// lane keeps the sum for its point of the current cell in registers and adds
// it to the grid only when its group's cell changes (and once after the warp's
// last batch), the flushing groups one after the other, as their cells may
// overlap.
// The warps' grids are added in a fixed order, and the CTAs' grids by the
// finishing kernel in a fixed order, so the result is bitwise reproducible.
constexpr int kNuW = 8;             // kernel width in grid points
constexpr int kNuWarps = 8;         // warps per CTA, one grid each
constexpr int kNuThreads = 32 * kNuWarps;
constexpr int kNuMaxSamples = 512;  // grids of up to 1024 points (8 KB per warp)
constexpr int kNuQuad = 32;         // Gauss-Legendre nodes for Psi

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct NufftArg {
  float half_n;    // N_s / 2
  float m;         // M = 2 N_s
  float beta_l2e;  // beta log2(e)
  int log_m;
};

// Psi(xi) = sum_i wpsi[i] cos(2 pi xi x[i]): Gauss-Legendre on [0, w/2] of 2 psi(x) cos(2 pi xi x)
struct PsiQuad {
  float x[kNuQuad];
  float wpsi[kNuQuad];
};

// CTA (v, q) spreads antenna v; the warps of the Q CTAs take contiguous ranges
// of batches of 32 paths.  Writes the CTA's grid: grids[(q V + v) M + l].
__global__ void __launch_bounds__(kNuThreads) k_nufft_spread(const float4* __restrict__ prep, int64_t cap,
                                                            const int32_t* __restrict__ d_P, int V, int Q,
                                                            NufftArg na, float2* __restrict__ grids,
                                                            unsigned int* __restrict__ fin_cnt,
                                                            const float* __restrict__ rate = nullptr,
                                                            float cnu = 0.f, float ceps = 0.f) {
  extern __shared__ float2 wgrid[];  // [warp][M]
  if (blockIdx.x == 0 && threadIdx.x < V) fin_cnt[threadIdx.x] = 0u;  // the finishing kernel's counters
  const int M = 1 << na.log_m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 3, j = lane & 7;
  float2* g = wgrid + (size_t)warp * M;
  for (int i = lane; i < M; i += 32) g[i] = make_float2(0.f, 0.f);
  __syncwarp();
  const int v = blockIdx.x % V, q = blockIdx.x / V;
  const int64_t P = *d_P;
  const float4* pv = prep + (size_t)v * cap;
  const float xo = (float)(j - (kNuW / 2 - 1));  // this lane's grid point minus floor(u), before t
  // each warp takes a contiguous range of batches of 32 paths, so that a group's
  // register sums carry over from one batch to the next (neighbouring rays)
  const int64_t nbat = (P + 31) / 32, nw = (int64_t)Q * kNuWarps, wi = (int64_t)q * kNuWarps + warp;
  const int64_t b0 = nbat * wi / nw, b1 = nbat * (wi + 1) / nw;
  float ax = 0.f, ay = 0.f;
  int cur = INT_MIN;
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t p = b * 32 + lane;  // lane prepares path p
    float cre = 0.f, cim = 0.f, t = 0.f;
    int i0 = 0;
    if (p < P) {
      float4 r = __ldg(&pv[p]);  // phi0, delta_hi, delta_lo, A
      if (rate) {
        // a moving scene's chirp: phi0 + dL/dt cnu and delta + dL/dt ceps, whole multiples of
        // 2^-12 of the delta shift moved into delta_hi (which stays exact)
        const float ld = __ldg(&rate[(size_t)v * cap + p]);
        float ph = fmaf(ld, cnu, r.x);
        r.x = ph - rintf(ph);
        const float dl = fmaf(ld, ceps, r.z);
        const float kq = rintf(dl * 4096.f);
        const float dh = r.y + kq * (1.f / 4096.f);
        r.y = dh - rintf(dh);
        r.z = dl - kq * (1.f / 4096.f);
      }
      float x = na.half_n * r.y;       // exact
      x -= rintf(x);
      x = fmaf(na.half_n, r.z, x) + r.x;
      x -= rintf(x);
      float sn, cs;
      __sincosf(kTwoPiF * x, &sn, &cs);
      cre = r.w * cs;
      cim = r.w * sn;
      const float uh = na.m * r.y;  // exact
      const float fl = floorf(uh);
      t = fmaf(na.m, r.z, uh - fl);
      i0 = (int)fl;
      if (t < 0.f) {
        t += 1.f;
        --i0;
      } else if (t >= 1.f) {
        t -= 1.f;
        ++i0;
      }
    }
    const int nb = (int)min((int64_t)32, P - b * 32);
    // group grp takes paths 8 grp .. 8 grp + 7 in turn; a lane keeps the sum for its
    // point of the current cell in registers and adds it to the grid when the cell changes
    for (int st = 0; st < 8; ++st) {
      const int src = 8 * grp + st;
      const bool live = src < nb;
      const float pr = __shfl_sync(0xffffffffu, cre, src), pi = __shfl_sync(0xffffffffu, cim, src);
      const float pt = __shfl_sync(0xffffffffu, t, src);
      const int pl = __shfl_sync(0xffffffffu, i0, src);
      const bool flush = live && pl != cur && cur != INT_MIN;
      unsigned fg = __ballot_sync(0xffffffffu, flush) & 0x01010101u;  // lane 8 g flags group g
      if (fg) {  // the flushing groups in turn: their cells may overlap
        const int lc = (cur + j - (kNuW / 2 - 1)) & (M - 1);
        do {
          const int gg = (__ffs(fg) - 1) >> 3;
          if (grp == gg) {
            float2 o = g[lc];
            o.x += ax;
            o.y += ay;
            g[lc] = o;
          }
          __syncwarp();
          fg &= fg - 1;
        } while (fg);
      }
      if (live && pl != cur) {
        ax = 0.f;
        ay = 0.f;
        cur = pl;
      }
      if (live) {
        const float z = (xo - pt) * (2.f / kNuW);
        // psi = exp(beta (sqrt(1 - z^2) - 1)); |z| <= 1 on the 8 points
        const float psi = ex2_approx(na.beta_l2e * (sqrt_approx(fmaxf(fmaf(-z, z, 1.f), 0.f)) - 1.f));
        ax = fmaf(psi, pr, ax);
        ay = fmaf(psi, pi, ay);
      }
    }
  }
  {  // the last cells
    const int lc = (cur + j - (kNuW / 2 - 1)) & (M - 1);
    for (int gg = 0; gg < 4; ++gg) {
      if (grp == gg && cur != INT_MIN) {
        float2 o = g[lc];
        o.x += ax;
        o.y += ay;
        g[lc] = o;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  float2* out = grids + ((size_t)q * V + v) * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    float2 acc = wgrid[i];
    for (int w = 1; w < kNuWarps; ++w) {
      const float2 x = wgrid[(size_t)w * M + i];
      acc.x += x.x;
      acc.y += x.y;
    }
    out[i] = acc;
  }
}

// Finishing, kNuFinSlice grid points per CTA: CTA (v, s) adds slice s of the Q
// CTAs' grids of antenna v in a fixed order (kNuFinThreads / slice threads per
// point, each over every such CTA with four interleaved sums, then the threads'
// sums in order) into bsum; the last CTA of the antenna to finish (a counter per
// antenna, zeroed by the spreading kernel) runs the M-point FFT and the division
// by Psi(n'/M) and writes S[v][n] into the cube: chirp `only` (a moving scene),
// else every chirp (a static scene's chirps are equal).
constexpr int kNuFinThreads = 1024;
constexpr int kNuFinSlice = 128;
__global__ void __launch_bounds__(kNuFinThreads) k_nufft_finish(const float2* __restrict__ grids, int V, int Q,
                                                                int Ns, int log_m, PsiQuad pq,
                                                                float2* __restrict__ bsum,
                                                                unsigned int* __restrict__ cnt,
                                                                float2* __restrict__ cube, int C, int only) {
  extern __shared__ float2 sg[];  // [M] grid, [M / 2] twiddles, [kNuFinThreads] per-thread sums
  __shared__ int s_last;
  const int M = 1 << log_m, slice = M < kNuFinSlice ? M : kNuFinSlice, S = M / slice;
  const int v = blockIdx.x / S, sl = blockIdx.x - v * S;
  float2* tw = sg + M;
  float2* part = tw + M / 2;
  const int parts = blockDim.x / slice, li = threadIdx.x % slice, k0 = threadIdx.x / slice;
  const int l = sl * slice + li;
  float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
  const float2* src = grids + (size_t)v * M + l;
  const size_t qs = (size_t)V * M;  // from one CTA's grid to the next
  int q = k0;
  for (; q + 3 * parts < Q; q += 4 * parts) {  // four loads in flight, four interleaved sums
    const float2 x0 = __ldcg(src + (size_t)q * qs), x1 = __ldcg(src + (size_t)(q + parts) * qs);
    const float2 x2 = __ldcg(src + (size_t)(q + 2 * parts) * qs), x3 = __ldcg(src + (size_t)(q + 3 * parts) * qs);
    a0.x += x0.x;
    a0.y += x0.y;
    a1.x += x1.x;
    a1.y += x1.y;
    a2.x += x2.x;
    a2.y += x2.y;
    a3.x += x3.x;
    a3.y += x3.y;
  }
  for (; q < Q; q += parts) {
    const float2 x = __ldcg(src + (size_t)q * qs);
    a0.x += x.x;
    a0.y += x.y;
  }
  part[threadIdx.x] = make_float2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
  __syncthreads();
  if (threadIdx.x < slice) {
    float2 acc = part[li];
    for (int k = 1; k < parts; ++k) {
      acc.x += part[k * slice + li].x;
      acc.y += part[k * slice + li].y;
    }
    bsum[(size_t)v * M + l] = acc;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&cnt[v], 1u) == (unsigned)(S - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  fft::fill_twiddles(tw, M, 1.f, blockDim.x, threadIdx.x);
  for (int i = threadIdx.x; i < M; i += blockDim.x) sg[fft::bitrev(i, log_m)] = __ldcg(&bsum[(size_t)v * M + i]);
  __syncthreads();
  fft::smem_fft(sg, tw, log_m, blockDim.x, threadIdx.x);
  const int h = Ns >> 1;
  for (int n = threadIdx.x; n < Ns; n += blockDim.x) {
    const float xi = (float)(n - h) / (float)M;
    float ph = 0.f;
#pragma unroll 8
    for (int i = 0; i < kNuQuad; ++i) ph = fmaf(pq.wpsi[i], cospif(2.f * xi * pq.x[i]), ph);
    const float2 B = sg[(n - h) & (M - 1)];
    const float inv = 1.f / ph;
    const float2 val = make_float2(B.x * inv, B.y * inv);
    if (only >= 0) {
      cube[((size_t)v * C + only) * Ns + n] = val;
    } else {
      for (int c = 0; c < C; ++c) cube[((size_t)v * C + c) * Ns + n] = val;
    }
  }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the three-term
// recurrence of the Legendre polynomials), mapped to Psi's quadrature.
PsiQuad make_psi_quad(double beta) {
  PsiQuad pq{};
  const int n = kNuQuad;
  const double half_w = 0.5 * kNuW;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-15) break;
    }
    const double wgt = 2.0 / ((1.0 - z * z) * dp * dp);
    // [-1, 1] -> [0, w/2]; Psi(xi) = 2 int_0^{w/2} psi(x) cos(2 pi xi x) dx
    const double x = 0.5 * half_w * (1.0 + z);
    const double zz = x / half_w;
    const double psi = exp(beta * (sqrt(1.0 - zz * zz) - 1.0));
    pq.x[i] = (float)x;
    pq.wpsi[i] = (float)(2.0 * 0.5 * half_w * wgt * psi);
  }
  return pq;
}

constexpr double kNuBeta = 2.3 * kNuW;

const PsiQuad& psi_quad() {
  static const PsiQuad pq = make_psi_quad(kNuBeta);
  return pq;
}

// Few (path, antenna) records: the direct kernels, whose one pass over the records
// costs less than the non-uniform FFT's spreading, finishing sum and FFT chain.
#ifndef SBR_NUFFT_MIN_RECORDS
#define SBR_NUFFT_MIN_RECORDS 65536
#endif
constexpr int64_t kNuMinRecords = SBR_NUFFT_MIN_RECORDS;
inline bool nufft_for(sbr_phase_mode mode, int Ns, int64_t records) {
  return mode == SBR_PHASE_SPLIT && Ns <= kNuMaxSamples && records >= kNuMinRecords;
}

// Launch-shape queries are cached per device ordinal (kernel attributes such as
// a raised shared-memory limit are per device too); ordinals at or beyond
// kDevCache are queried on every call.
constexpr int kDevCache = 64;

inline int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  return dev;
}

int sm_count() {
  static int cache[kDevCache] = {};
  const int dev = current_device();
  if (dev < kDevCache && cache[dev]) return cache[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  if (dev < kDevCache) cache[dev] = n;
  return n;
}

// Grid: V * Q CTAs, Q the largest that keeps every CTA resident at once (one
// wave), capped by the number of path chunks.
// dynamic shared memory of the split kernel: the groups' reduction buffer
inline size_t split_smem(int Ns) {
  const int T = threads_for(Ns), M = Ns / T;
  return kSplitThreads / T > 1 ? sizeof(float2) * M * kSplitThreads : 0;
}

// resident CTAs of the split kernel per SM (registers and shared memory decide)
int split_per_sm(int Ns) {
  static int cache[kDevCache][17] = {};
  const int T = threads_for(Ns), M = Ns / T;
  if (M > 16) return 1;
  const int dev = current_device();
  if (dev < kDevCache && cache[dev][M]) return cache[dev][M];
  int n = 0;
  const size_t sm = split_smem(Ns);
  switch (M) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_synth_split<1>, kSplitThreads, sm); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_synth_split<2>, kSplitThreads, sm); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_synth_split<4>, kSplitThreads, sm); break;
    case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_synth_split<8>, kSplitThreads, sm); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_synth_split<16>, kSplitThreads, sm); break;
  }
  n = n > 0 ? n : 1;
  if (dev < kDevCache) cache[dev][M] = n;
  return n;
}

// resident CTAs of the tensor-core kernel per SM (N_s = 256 or 512)
int mma_per_sm(int Ns) {
  static int cache[kDevCache][3] = {};
  const int mt = Ns / 256;
  const int dev = current_device();
  if (dev < kDevCache && cache[dev][mt]) return cache[dev][mt];
  int n = 0;
  if (mt == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_synth_mma<1>, kMmaThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_synth_mma<2>, kMmaThreads, 0);
  n = n > 0 ? n : 1;
  if (dev < kDevCache) cache[dev][mt] = n;
  return n;
}

void grid_shape(int V, int Ns, int64_t cap, int* Q) {
  int per_sm = split_per_sm(Ns);
  if (Ns == 256 || Ns == 512) {
    const int m = mma_per_sm(Ns);
    if (m < per_sm) per_sm = m;
  }
  // whole waves only: every CTA resident from the start (a CTA beyond the
  // first wave would run alone after the others and double the launch)
  int64_t q = ((int64_t)sm_count() * per_sm) / V;
  const int64_t chunks = (cap + kChunk - 1) / kChunk;
  if (q > chunks) q = chunks;
  if (q < 1) q = 1;
  *Q = (int)q;
}

// dynamic shared memory of the spreading kernel: one grid of M = 2 N_s points per warp
inline size_t nufft_smem(int Ns) { return sizeof(float2) * kNuWarps * 2 * (size_t)Ns; }

// resident spreading CTAs per SM (shared memory and registers decide); raises
// the kernel's shared-memory limit once where the grids pass 48 KB
int nufft_per_sm(int Ns) {
  static int cache[kDevCache][16] = {};
  int lg = 0;
  while ((1 << lg) < Ns) ++lg;
  const int dev = current_device();
  if (dev < kDevCache && cache[dev][lg]) return cache[dev][lg];
  const size_t sm = nufft_smem(Ns);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_nufft_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nufft_spread, kNuThreads, sm);
  n = n > 0 ? n : 1;
  if (dev < kDevCache) cache[dev][lg] = n;
  return n;
}

// CTAs per antenna of the spreading kernel: one wave, at most one per 256 paths
void nufft_shape(int V, int Ns, int64_t cap, int* Qn) {
  int64_t q = ((int64_t)sm_count() * nufft_per_sm(Ns)) / V;
  const int64_t batches = (cap + 32 * kNuWarps - 1) / (32 * kNuWarps);
  if (q > batches) q = batches;
  if (q < 1) q = 1;
  *Qn = (int)q;
}

// Workspace: per-CTA partial sums of the direct kernels, the chirp-summed
// upstream gradient of the adjoint, and, for the non-uniform FFT, the CTAs'
// grids, their sum and the finishing counters.
size_t ws_layout(const sbr_radar_cfg* radar, int64_t cap, int* Q, int* Qn = nullptr) {
  const int V = radar->n_tx * radar->n_rx, Ns = radar->n_samples;
  grid_shape(V, Ns, cap, Q);
  int qn = 0;
  if (Ns <= kNuMaxSamples) nufft_shape(V, Ns, cap, &qn);
  if (Qn) *Qn = qn;
  Carver c(nullptr);
  c.take<float2>((size_t)V * (*Q) * Ns);       // per-CTA partial sums
  c.take<float2>((size_t)V * Ns);              // chirp-summed upstream gradient
  c.take<float2>((size_t)V * qn * 2 * Ns);     // non-uniform FFT: the CTAs' grids
  c.take<float2>((size_t)V * 2 * Ns);          // non-uniform FFT: the summed grids
  c.take<unsigned int>((size_t)V);             // non-uniform FFT: finishing counters
  return c.bytes();
}

}  // namespace
}  // namespace sbr

using namespace sbr;

extern "C" size_t sbr_synth_ws_bytes(const sbr_radar_cfg* radar, int64_t path_cap) {
  if (!radar || radar->n_tx < 1 || radar->n_rx < 1 || radar->n_samples < 1) return 0;
  int Q;
  return ws_layout(radar, path_cap, &Q);
}

namespace {
struct SynthWs {
  float2* partial;
  float2* gsum;
  float2* grids;
  float2* bsum;
  unsigned int* fin_cnt;
  int Q, Qn;
};

sbr_status bind_ws(const sbr_radar_cfg* radar, int64_t cap, void* ws, size_t bytes, SynthWs* w,
                   const char* who) {
  int Q, Qn;
  const size_t need = ws_layout(radar, cap, &Q, &Qn);
  SBR_ARG(ws && aligned256(ws), "%s: workspace NULL or not 256-byte aligned", who);
  if (bytes < need) {
    set_error("%s: workspace of %zu bytes, %zu needed", who, bytes, need);
    return SBR_ERR_OOM;
  }
  const int V = radar->n_tx * radar->n_rx, Ns = radar->n_samples;
  Carver c(ws);
  w->partial = c.take<float2>((size_t)V * Q * Ns);
  w->gsum = c.take<float2>((size_t)V * Ns);
  w->grids = c.take<float2>((size_t)V * Qn * 2 * Ns);
  w->bsum = c.take<float2>((size_t)V * 2 * Ns);
  w->fin_cnt = c.take<unsigned int>((size_t)V);
  w->Q = Q;
  w->Qn = Qn;
  return SBR_OK;
}

// A moving scene: every chirp synthesised from its own delays (split phase by the
// non-uniform FFT up to 512 samples, or the FP64 phase), chirp by chirp.
sbr_status launch_moving(sbr_phase_mode mode, const sbr_paths* p, const sbr_radar_cfg* r, const SynthWs& w,
                         float2* cube, cudaStream_t st) {
  const int V = p->n_virt, Ns = r->n_samples, C = r->n_chirps;
  const double per_chirp = r->chirp_rep / kC;  // delay change per chirp per (m/s) of dL/dt
  if (mode == SBR_PHASE_SPLIT && Ns <= kNuMaxSamples) {
    int log_m = 0;
    while ((1 << log_m) < 2 * Ns) ++log_m;
    NufftArg na{0.5f * (float)Ns, 2.f * (float)Ns, (float)(kNuBeta * 1.4426950408889634), log_m};
    nufft_per_sm(Ns);
    const int M = 2 * Ns, slices = M < kNuFinSlice ? 1 : M / kNuFinSlice;
    for (int c = 0; c < C; ++c) {
      const float cnu = (float)(c * per_chirp * r->f0), ceps = (float)(c * per_chirp * r->bandwidth / Ns);
      ::sbr::note_launch();
      k_nufft_spread<<<V * w.Qn, kNuThreads, nufft_smem(Ns), st>>>(reinterpret_cast<const float4*>(p->prep),
                                                                   p->path_cap, p->count, V, w.Qn, na, w.grids,
                                                                   w.fin_cnt, p->path_rate, cnu, ceps);
      ::sbr::note_launch();
      k_nufft_finish<<<V * slices, kNuFinThreads, sizeof(float2) * (3 * (size_t)Ns + kNuFinThreads), st>>>(
          w.grids, V, w.Qn, Ns, log_m, psi_quad(), w.bsum, w.fin_cnt, cube, C, c);
    }
    return SBR_OK;
  }
  if (mode == SBR_PHASE_FP64) {
    const int T = threads_for(Ns), Mv = Ns / T;
    const int grid = V * w.Q;
    const float4* prep = reinterpret_cast<const float4*>(p->prep);
    const float2* plen = reinterpret_cast<const float2*>(p->path_len);
    for (int c = 0; c < C; ++c) {
      ::sbr::note_launch();
      switch (Mv) {
        case 1: k_synth_fp64<1><<<grid, T, 0, st>>>(prep, plen, p->phase_ofs, p->path_cap, p->count, V, w.Q, Ns, r->f0, r->bandwidth / Ns, w.partial, p->path_rate, c * per_chirp); break;
        case 2: k_synth_fp64<2><<<grid, T, 0, st>>>(prep, plen, p->phase_ofs, p->path_cap, p->count, V, w.Q, Ns, r->f0, r->bandwidth / Ns, w.partial, p->path_rate, c * per_chirp); break;
        case 4: k_synth_fp64<4><<<grid, T, 0, st>>>(prep, plen, p->phase_ofs, p->path_cap, p->count, V, w.Q, Ns, r->f0, r->bandwidth / Ns, w.partial, p->path_rate, c * per_chirp); break;
        case 8: k_synth_fp64<8><<<grid, T, 0, st>>>(prep, plen, p->phase_ofs, p->path_cap, p->count, V, w.Q, Ns, r->f0, r->bandwidth / Ns, w.partial, p->path_rate, c * per_chirp); break;
        default: k_synth_fp64<16><<<grid, T, 0, st>>>(prep, plen, p->phase_ofs, p->path_cap, p->count, V, w.Q, Ns, r->f0, r->bandwidth / Ns, w.partial, p->path_rate, c * per_chirp); break;
      }
      ::sbr::note_launch();
      k_reduce<<<dim3((V * Ns + 255) / 256, 1), 256, 0, st>>>(w.partial, V, w.Q, Ns, C, cube, c);
    }
    return SBR_OK;
  }
  set_error("sbr_synthesize: SBR_SYNTH_MOVING supports SBR_PHASE_SPLIT up to %d samples and SBR_PHASE_FP64",
            kNuMaxSamples);
  return SBR_ERR_UNSUPPORTED;
}

// Split-phase samples by the non-uniform FFT: spread, then finish (one chirp, written to all chirps).
void launch_nufft(const sbr_paths* p, const sbr_radar_cfg* r, const SynthWs& w, float2* cube, cudaStream_t st) {
  const int V = p->n_virt, Ns = r->n_samples;
  int log_m = 0;
  while ((1 << log_m) < 2 * Ns) ++log_m;
  NufftArg na{0.5f * (float)Ns, 2.f * (float)Ns, (float)(kNuBeta * 1.4426950408889634), log_m};
  nufft_per_sm(Ns);  // sets the shared-memory limit before the first launch
  ::sbr::note_launch();
  k_nufft_spread<<<V * w.Qn, kNuThreads, nufft_smem(Ns), st>>>(reinterpret_cast<const float4*>(p->prep),
                                                               p->path_cap, p->count, V, w.Qn, na, w.grids,
                                                               w.fin_cnt);
  const int M = 2 * Ns, slices = M < kNuFinSlice ? 1 : M / kNuFinSlice;
  ::sbr::note_launch();
  k_nufft_finish<<<V * slices, kNuFinThreads, sizeof(float2) * (3 * (size_t)Ns + kNuFinThreads), st>>>(
      w.grids, V, w.Qn, Ns, log_m, psi_quad(), w.bsum, w.fin_cnt, cube, r->n_chirps, -1);
}

template <int M>
void launch_fwd(sbr_phase_mode mode, const sbr_paths* p, const sbr_radar_cfg* r, const SynthWs& w,
                cudaStream_t st) {
  const int V = p->n_virt, Ns = r->n_samples, T = Ns / M;
  const int grid = V * w.Q;
  const float4* prep = reinterpret_cast<const float4*>(p->prep);
  if (mode == SBR_PHASE_SPLIT && (Ns == 256 || Ns == 512)) {
    ::sbr::note_launch();
    if (Ns == 256) k_synth_mma<1><<<grid, kMmaThreads, 0, st>>>(prep, p->path_cap, p->count, V, w.Q, w.partial);
    else k_synth_mma<2><<<grid, kMmaThreads, 0, st>>>(prep, p->path_cap, p->count, V, w.Q, w.partial);
  } else if (mode == SBR_PHASE_SPLIT) {
    ::sbr::note_launch();
    k_synth_split<M><<<grid, kSplitThreads, split_smem(Ns), st>>>(prep, p->path_cap, p->count, V, w.Q, Ns,
                                                                   w.partial);
  } else if (mode == SBR_PHASE_FP64) {
    ::sbr::note_launch();
    k_synth_fp64<M><<<grid, T, 0, st>>>(prep, reinterpret_cast<const float2*>(p->path_len), p->phase_ofs,
                                        p->path_cap, p->count, V, w.Q, Ns, r->f0, r->bandwidth / Ns, w.partial);
  } else {
    const double mu = r->bandwidth / r->chirp_time, dt = r->chirp_time / Ns;
    ::sbr::note_launch();
    k_synth_naive<M><<<grid, T, 0, st>>>(prep, reinterpret_cast<const float2*>(p->path_len), p->phase_ofs,
                                         p->path_cap, p->count, V, w.Q, Ns, (float)r->f0, (float)mu, (float)dt,
                                         w.partial);
  }
}
}  // namespace

extern "C" sbr_status sbr_synthesize(const sbr_paths* paths, const sbr_radar_cfg* radar,
                                     sbr_phase_mode mode_flags, float* d_cube, void* d_ws,
                                     size_t ws_bytes, sbr_stream stream) {
  SBR_ARG(paths && d_cube, "sbr_synthesize: NULL paths or cube");
  const bool moving = ((int)mode_flags & SBR_SYNTH_MOVING) != 0;
  const sbr_phase_mode mode = (sbr_phase_mode)((int)mode_flags & ~SBR_SYNTH_MOVING);
  sbr_status rs = check_radar(radar, "sbr_synthesize");
  if (rs != SBR_OK) return rs;
  SBR_ARG(paths->n_virt == radar->n_tx * radar->n_rx, "sbr_synthesize: paths have V=%d, radar %d",
          paths->n_virt, radar->n_tx * radar->n_rx);
  SBR_ARG(mode == SBR_PHASE_SPLIT || mode == SBR_PHASE_FP64 || mode == SBR_PHASE_NAIVE,
          "sbr_synthesize: unknown phase mode %d", (int)mode);
  SynthWs w;
  rs = bind_ws(radar, paths->path_cap, d_ws, ws_bytes, &w, "sbr_synthesize");
  if (rs != SBR_OK) return rs;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int Ns = radar->n_samples, T = threads_for(Ns), M = Ns / T;
  if (moving) {
    rs = launch_moving(mode, paths, radar, w, reinterpret_cast<float2*>(d_cube), st);
    if (rs != SBR_OK) return rs;
    SBR_CUDA(cudaGetLastError());
    return SBR_OK;
  }
  if (nufft_for(mode, Ns, paths->path_cap * paths->n_virt)) {
    launch_nufft(paths, radar, w, reinterpret_cast<float2*>(d_cube), st);
    SBR_CUDA(cudaGetLastError());
    return SBR_OK;
  }
  switch (M) {
    case 1: launch_fwd<1>(mode, paths, radar, w, st); break;
    case 2: launch_fwd<2>(mode, paths, radar, w, st); break;
    case 4: launch_fwd<4>(mode, paths, radar, w, st); break;
    case 8: launch_fwd<8>(mode, paths, radar, w, st); break;
    case 16: launch_fwd<16>(mode, paths, radar, w, st); break;
    default: set_error("sbr_synthesize: no kernel for %d samples per thread", M); return SBR_ERR_UNSUPPORTED;
  }
  SBR_CUDA(cudaGetLastError());
  const int V = paths->n_virt;
  ::sbr::note_launch();
  k_reduce<<<reduce_grid(V, Ns, radar->n_chirps), 256, 0, st>>>(w.partial, V, w.Q, Ns, radar->n_chirps,
                                                  reinterpret_cast<float2*>(d_cube));
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}

// ---- allocation-free variant ------------------------------------------------
//
// For callers that cannot call cudaMalloc (or reserve any device memory of
// their own) at the point where they synthesise: hosts that hand out no device
// allocator to plugins, real-time loops that must not risk the implicit device
// synchronisation of an allocation, or code running under a frozen memory
// budget.  The per-CTA partial sums then live in a fixed file-scope device
// array instead of a caller workspace.

namespace {
constexpr size_t kStaticPartials = 131072;  // float2 entries: 1 MiB on every device using the library
__device__ __align__(256) float2 g_static_partials[kStaticPartials];

constexpr int kMaxDevices = 64;
float2* g_static_ptr[kMaxDevices] = {};
std::mutex g_static_mu;

// Device address of the array for the current device (host code only holds a
// stand-in symbol).  Looked up once per device, on that device's first call.
sbr_status static_partials(float2** out) {
  int dev = -1;
  SBR_CUDA(cudaGetDevice(&dev));
  SBR_ARG(dev >= 0 && dev < kMaxDevices, "sbr_synthesize_noalloc: device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    SBR_CUDA(cudaGetSymbolAddress(&p, g_static_partials));
    g_static_ptr[dev] = static_cast<float2*>(p);
  }
  *out = g_static_ptr[dev];
  return SBR_OK;
}
}  // namespace

extern "C" sbr_status sbr_synthesize_noalloc(const sbr_paths* paths, const sbr_radar_cfg* radar,
                                             sbr_phase_mode mode, float* d_cube, sbr_stream stream) {
  SBR_ARG(paths && d_cube, "sbr_synthesize_noalloc: NULL paths or cube");
  sbr_status rs = check_radar(radar, "sbr_synthesize_noalloc");
  if (rs != SBR_OK) return rs;
  SBR_ARG(paths->n_virt == radar->n_tx * radar->n_rx, "sbr_synthesize_noalloc: paths have V=%d, radar %d",
          paths->n_virt, radar->n_tx * radar->n_rx);
  SBR_ARG(mode == SBR_PHASE_SPLIT || mode == SBR_PHASE_FP64 || mode == SBR_PHASE_NAIVE,
          "sbr_synthesize_noalloc: unknown phase mode %d", (int)mode);
  const int V = paths->n_virt, Ns = radar->n_samples;
  const size_t row = (size_t)V * Ns;  // one partial cube (one CTA per antenna)
  if (row > kStaticPartials) {
    set_error("sbr_synthesize_noalloc: V * N_s = %zu partial sums exceed the fixed scratch of %zu "
              "(1 MiB); use sbr_synthesize with a workspace",
              row, kStaticPartials);
    return SBR_ERR_UNSUPPORTED;
  }
  SynthWs w;
  rs = static_partials(&w.partial);
  if (rs != SBR_OK) return rs;
  w.gsum = nullptr;
  grid_shape(V, Ns, paths->path_cap, &w.Q);
  const int qmax = (int)(kStaticPartials / row);
  if (w.Q > qmax) w.Q = qmax;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int T = threads_for(Ns), M = Ns / T;
  switch (M) {
    case 1: launch_fwd<1>(mode, paths, radar, w, st); break;
    case 2: launch_fwd<2>(mode, paths, radar, w, st); break;
    case 4: launch_fwd<4>(mode, paths, radar, w, st); break;
    case 8: launch_fwd<8>(mode, paths, radar, w, st); break;
    case 16: launch_fwd<16>(mode, paths, radar, w, st); break;
    default: set_error("sbr_synthesize_noalloc: no kernel for %d samples per thread", M); return SBR_ERR_UNSUPPORTED;
  }
  SBR_CUDA(cudaGetLastError());
  ::sbr::note_launch();
  k_reduce<<<reduce_grid(V, Ns, radar->n_chirps), 256, 0, st>>>(w.partial, V, w.Q, Ns, radar->n_chirps,
                                                  reinterpret_cast<float2*>(d_cube));
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}

extern "C" sbr_status sbr_synthesize_bwd(const sbr_paths* paths, const sbr_radar_cfg* radar,
                                         const float* d_gcube, float* d_glen, float* d_gamp, float* d_gphase,
                                         void* d_ws, size_t ws_bytes, sbr_stream stream) {
  SBR_ARG(paths && d_gcube && d_glen && d_gamp, "sbr_synthesize_bwd: NULL argument");
  sbr_status rs = check_radar(radar, "sbr_synthesize_bwd");
  if (rs != SBR_OK) return rs;
  SBR_ARG(paths->n_virt == radar->n_tx * radar->n_rx, "sbr_synthesize_bwd: V mismatch");
  SynthWs w;
  rs = bind_ws(radar, paths->path_cap, d_ws, ws_bytes, &w, "sbr_synthesize_bwd");
  if (rs != SBR_OK) return rs;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int V = paths->n_virt, Ns = radar->n_samples, C = radar->n_chirps;
  // the upstream gradient summed over the (equal) chirps; one chirp needs no sum
  const float2* gs = reinterpret_cast<const float2*>(d_gcube);
  if (C > 1) {
    ::sbr::note_launch();
    k_chirp_sum<<<(V * Ns + 255) / 256, 256, 0, st>>>(gs, V, C, Ns, w.gsum);
    gs = w.gsum;
  }
  const int64_t cap = paths->path_cap;
  if (cap > 0) {
    dim3 grid((unsigned)((cap + 255) / 256), (unsigned)V);
    const double lam_inv = radar->f0 / kC;
    const double bcn = radar->bandwidth / (kC * Ns);
    ::sbr::note_launch();
    k_synth_bwd<<<grid, 256, Ns * sizeof(float2), st>>>(
        reinterpret_cast<const float4*>(paths->prep), cap, paths->count, Ns, gs,
        (float)lam_inv, (float)bcn, d_glen, d_gamp, d_gphase);
  }
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}
