// Radar point cloud from the IF cube: the signal-processing map T of Eq. 16
// (Section 3.4), and its adjoint.
//
// The paper leaves T open ("a signal processing algorithm" producing a spatial
// image; Section 4 shows radar point clouds).  This library reads it as:
//   X = FFT_chirp(FFT_sample(cube))                     range and Doppler spectra
//   Y[a,d,k] = sum_v W[a,v] X[v,d,k],  W = e^{+j 2 pi x_v u_a / lambda_c},
//              u_a = -1 + 2a/N_theta, lambda_c = c / (f_c + B/2)      angle DFT
//   Pw[a,k] = sum_d |Y[a,d,k]|^2                                     power map
//   N[a,k]  = mean of Pw over `train` cells each side beyond `guard` (range) CA-CFAR
//   w = sigmoid((ln Pw - ln(alpha N + floor_rel max Pw)) / beta)     soft detection
//   peaks: 3x3 local maxima above the floor (ties: lower cell index), w >= w_min,
//   ordered by (w desc, cell asc), at most k_max;
//   sub-bin 3-point parabola on ln Pw per axis (clamped to +-1/2 bin);
//   point = (r u, 0, r sqrt(1 - u^2)), r = (k + dk) c / (2B).
// The adjoint routes dL/d(point) and dL/dw to dPw (sparse: the peak, its
// refine neighbours, its CFAR training cells and the argmax cell), then
// dY = 2 Y dPw, dX = W^H dY, and the two inverse FFTs (unnormalised: the
// adjoint of a forward DFT).
#include <math.h>

#include <atomic>

#include "cta_sort.cuh"
#include "fft.cuh"
#include "tcgen05.cuh"

namespace sbr {
namespace {

using namespace fft;

// FFT along the contiguous last axis: one CTA per row of n points.
__global__ void k_fft_rows(const float2* __restrict__ in, float2* __restrict__ out, int n, int logn,
                           float sign) {
  extern __shared__ float2 s[];  // [n] points, [n / 2] twiddles
  float2* tw = s + n;
  const size_t row = blockIdx.x;
  fill_twiddles(tw, n, sign, blockDim.x, threadIdx.x);
  for (int i = threadIdx.x; i < n; i += blockDim.x) s[bitrev(i, logn)] = in[row * n + i];
  __syncthreads();
  smem_fft(s, tw, logn, blockDim.x, threadIdx.x);
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[row * n + i] = s[i];
}

constexpr int kColTile = 16;

// FFT along the chirp axis of [V][C][N_s]: one CTA per (v, 16 consecutive k).
// Columns sit C + 1 points apart in shared memory, so the 16 columns of one
// chirp fall in different banks.
__global__ void k_fft_cols(float2* __restrict__ x, int C, int logc, int Ns, float sign) {
  extern __shared__ float2 s[];  // [kColTile][C + 1] points, [C / 2] twiddles
  const int ld = C + 1;
  float2* tw = s + kColTile * ld;
  const int tiles = Ns / kColTile;
  const int v = blockIdx.x / tiles, k0 = (blockIdx.x - v * tiles) * kColTile;
  float2* base = x + (size_t)v * C * Ns + k0;
  fill_twiddles(tw, C, sign, blockDim.x, threadIdx.x);
  for (int i = threadIdx.x; i < C * kColTile; i += blockDim.x) {
    const int c = i / kColTile, kk = i - c * kColTile;
    s[kk * ld + bitrev(c, logc)] = base[(size_t)c * Ns + kk];
  }
  __syncthreads();
  const int hc = C >> 1;
  for (int m = 1; m <= logc; ++m) {
    const int half = 1 << (m - 1);
    for (int u = threadIdx.x; u < kColTile * hc; u += blockDim.x) {
      const int col = u >> (logc - 1), w = u & (hc - 1);
      const int j = w & (half - 1);
      float2* sc = s + col * ld;
      const int i0 = ((w >> (m - 1)) << m) + j, i1 = i0 + half;
      const float2 t = cmul(sc[i1], tw[j << (logc - m)]);
      const float2 a = sc[i0];
      sc[i0] = make_float2(a.x + t.x, a.y + t.y);
      sc[i1] = make_float2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < C * kColTile; i += blockDim.x) {
    const int c = i / kColTile, kk = i - c * kColTile;
    base[(size_t)c * Ns + kk] = s[kk * ld + c];
  }
}

// x_v / lambda_c and y_v / lambda_c per virtual antenna and the angle bins,
// passed by value (no host-to-device copy, so the entry points can be captured
// into CUDA graphs).  Angle row rho = e * A + a: azimuth cosine u_a = -1 + 2a/A,
// elevation cosine w_e = (2e + 1 - E) / E (w = 0 with one elevation bin).
struct Steer {
  float xl[SBR_MAX_VIRT];
  float yl[SBR_MAX_VIRT];
  int A, E;
};

// Phase (in half-cycles, for sincospif) of antenna v in angle row rho.
__device__ inline float steer_halfcycles(const Steer& st, int rho, int v) {
  const int e = rho / st.A, a = rho - e * st.A;
  const float u = -1.f + 2.f * (float)a / (float)st.A;
  const float w = (float)(2 * e + 1 - st.E) / (float)st.E;
  return 2.f * (st.xl[v] * u + st.yl[v] * w);
}

// Steering matrix W[rho][v] of the R = E * A angle rows into shared memory.
__device__ inline void load_w(float2* sw, const Steer& xl, int R, int V) {
  for (int i = threadIdx.x; i < R * V; i += blockDim.x) {
    const int rho = i / V, v = i - rho * V;
    float sn, cs;
    sincospif(steer_halfcycles(xl, rho, v), &sn, &cs);
    sw[i] = make_float2(cs, sn);
  }
}

constexpr int kKT = 32;  // ranges per CTA in the angle kernels

// Partial power map over one group of Doppler bins: part[g][rho][k] = sum_{d in g} |Y|^2
// for the R = 8 APT angle rows.
template <int APT>
__global__ void __launch_bounds__(256) k_angle_power(const float2* __restrict__ X,
                                                     const Steer xl, int V, int C,
                                                     int Ns, int dpg, float* __restrict__ part) {
  extern __shared__ float2 sm[];
  constexpr int R = 8 * APT;
  float2* sw = sm;                // [R][V]
  float2* sx = sm + R * V;        // [V][kKT]
  load_w(sw, xl, R, V);
  const int kk = threadIdx.x & (kKT - 1), ag = threadIdx.x >> 5;
  const int k0 = blockIdx.x * kKT, g = blockIdx.y;
  float acc[APT];
#pragma unroll
  for (int i = 0; i < APT; ++i) acc[i] = 0.f;
  for (int d = g * dpg; d < min(C, (g + 1) * dpg); ++d) {
    __syncthreads();
    for (int i = threadIdx.x; i < V * kKT; i += blockDim.x) {
      const int v = i / kKT, q = i - v * kKT;
      sx[i] = X[((size_t)v * C + d) * Ns + k0 + q];
    }
    __syncthreads();
    // antenna outer, angles inner: each x value is read once per Doppler bin
    float yr[APT], yi[APT];
#pragma unroll
    for (int i = 0; i < APT; ++i) yr[i] = yi[i] = 0.f;
    for (int v = 0; v < V; ++v) {
      const float2 x = sx[v * kKT + kk];
#pragma unroll
      for (int i = 0; i < APT; ++i) {
        const float2 w = sw[(ag * APT + i) * V + v];
        yr[i] = fmaf(w.x, x.x, fmaf(-w.y, x.y, yr[i]));
        yi[i] = fmaf(w.x, x.y, fmaf(w.y, x.x, yi[i]));
      }
    }
#pragma unroll
    for (int i = 0; i < APT; ++i) acc[i] = fmaf(yr[i], yr[i], fmaf(yi[i], yi[i], acc[i]));
  }
#pragma unroll
  for (int i = 0; i < APT; ++i) part[((size_t)g * R + ag * APT + i) * Ns + k0 + kk] = acc[i];
}

// ---- angle DFT on the tensor cores ------------------------------------------
//
// Per Doppler bin d the angle DFT of kTcM range bins is one real GEMM
//   D[k][2a + part] = sum_j A[k][j] B[2a + part][j],   j = 2v + (0: Re, 1: Im)
// with A = X^T (M = kTcM range bins, K = 2V) and B = the steering matrix of the
// R <= NR angle rows (NR = 64 or 128) as N = 2 NR real rows: row 2a = (W_re, -W_im)
// and row 2a + 1 = (W_im, W_re) at columns (2v, 2v + 1), so D[k][2a] = Re Y[a,d,k]
// and D[k][2a + 1] = Im Y[a,d,k].
// It runs as tcgen05.mma kind::tf32 from shared memory into TMEM.  Each
// operand is split as hi = tf32(x), lo = x - hi, and three products
// A_lo B_hi + A_hi B_lo + A_hi B_hi (small terms first) keep ~21 bits; the
// dropped lo.lo term is ~2^-22 relative, so Y matches the FP32 CUDA-core
// contraction to ~1e-6.  A CTA takes kTcM range bins of kTcDG Doppler bins, one
// kTcM x 2 NR FP32 accumulator per Doppler bin in TMEM; thread t of the CTA owns
// TMEM lane t (range bin k0 + t) and every angle, so |Y|^2 = D[2a]^2 + D[2a+1]^2
// needs no data exchange, and its sum over the CTA's Doppler bins stays in
// registers until one coalesced store per angle.
#ifndef SBR_ANGLE_DG
#define SBR_ANGLE_DG 2
#endif
constexpr int kTcM = 128;                      // range bins per CTA (MMA M: one TMEM lane each)
constexpr int kTcDG = SBR_ANGLE_DG;            // Doppler bins per CTA
constexpr int kTcThreads = 128;                // four warps: the four TMEM lane quadrants
constexpr int kTcK = 32;                       // K capacity: up to 16 antennas
constexpr uint32_t kTcTile = 128 * kTcK * 4;   // bytes of one 128-row operand (hi or lo)
constexpr uint32_t kTcLbo = 128;               // K-adjacent core matrices
constexpr uint32_t kTcSbo = (kTcK / 4) * 128;  // M/N-adjacent core matrices (8-row groups)
constexpr uint64_t kTcWaitNs = 200000000ull;   // bounded wait for the MMAs: 0.2 s
// NR angle rows (64 or 128): MMA N = 2 NR, TMEM columns 2 NR per Doppler bin, the
// steering operand 2 NR rows; shared memory = steering + X^T per Doppler bin (hi, lo)
template <int NR>
constexpr int tc_cols() { return 2 * NR * kTcDG; }
template <int NR>
constexpr size_t tc_smem() { return 2 * (size_t)kTcTile * (2 * NR / 128 + kTcDG) + 64; }
static_assert(tc_cols<64>() >= 32 && tc_cols<128>() <= 512, "TMEM columns");

inline int angle_tc_rows(int R) { return R <= 64 ? 64 : 128; }
inline bool angle_tc_ok(int R, int V, int Ns) { return R <= 128 && V <= 16 && Ns % kTcM == 0; }

// Byte offset of the 16-byte row chunk (row, k .. k + 3), k a multiple of 4, in
// the no-swizzle K-major layout of a K = 32 operand: 8-row x 4-element core
// matrices of 128 contiguous bytes, the 8 core matrices of a row group side by
// side along K (kTcLbo apart), row groups kTcSbo apart.
__device__ inline uint32_t tc_off(int row, int k) {
  return (uint32_t)((((row >> 3) * (kTcK / 4) + (k >> 2)) << 7) + ((row & 7) << 4));
}

// Stores hi = tf32(x) and lo = x - hi of four consecutive K entries.
__device__ inline void tc_put4(unsigned char* hi, unsigned char* lo, uint32_t off, float4 x) {
  const float4 h = make_float4(tc::to_tf32(x.x), tc::to_tf32(x.y), tc::to_tf32(x.z), tc::to_tf32(x.w));
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
}

// part[g][rho][k] = sum over the Doppler bins of group g of |Y[rho,d,k]|^2 for the R
// angle rows (R <= NR); on a timed-out wait the CTA writes NaN and sets bit 0 of *err.
template <int NR>
__global__ void __launch_bounds__(kTcThreads) k_angle_tc(const float2* __restrict__ X, const Steer xl, int R,
                                                         int V, int C, int Ns, float* __restrict__ part,
                                                         int* __restrict__ err) {
  constexpr int kN = 2 * NR;                         // MMA N
  constexpr int kCols = tc_cols<NR>();
  constexpr uint32_t kTileW = (uint32_t)kN * kTcK * 4;  // steering operand bytes (hi or lo)
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sw_hi = tsm;                  // B: steering rows
  unsigned char* sw_lo = tsm + kTileW;
  unsigned char* sx_hi = tsm + 2 * kTileW;     // A: X^T per Doppler bin, hi then lo
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sx_hi + 2 * (size_t)kTcTile * kTcDG);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int k0 = blockIdx.x * kTcM, g = blockIdx.y, d0 = g * kTcDG;
  const int nd = min(kTcDG, C - d0);  // Doppler bins of this CTA (>= 1)
  const int ks = (2 * V + 7) / 8;      // MMA K steps of 8 used
  if (warp == 0) {
    tc::tmem_alloc(tslot, kCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(mbar, 1);
  // A: thread t takes range bin k0 + t; per Doppler bin and antenna pair one 16-byte chunk
  // (Re, Im of antenna 2j, Re, Im of antenna 2j + 1); antennas >= V and bins >= nd are zero.
  // Every load is issued before the steering matrix is generated, which hides their latency.
  float2 xv[kTcDG][kTcK / 2];
#pragma unroll
  for (int dd = 0; dd < kTcDG; ++dd)
#pragma unroll
    for (int v = 0; v < kTcK / 2; ++v)
      xv[dd][v] = (dd < nd && v < V) ? X[((size_t)v * C + d0 + dd) * Ns + k0 + tid] : make_float2(0.f, 0.f);
  // B: row pair (2a, 2a + 1) of angle row a, antenna pair j: one 16-byte chunk per row
  for (int i = tid; i < NR * (kTcK / 4); i += kTcThreads) {
    const int a = i >> 3, j = i & 7;
    float c0 = 0.f, s0 = 0.f, c1 = 0.f, s1 = 0.f;
    if (a < R) {
      if (2 * j < V) sincospif(steer_halfcycles(xl, a, 2 * j), &s0, &c0);
      if (2 * j + 1 < V) sincospif(steer_halfcycles(xl, a, 2 * j + 1), &s1, &c1);
    }
    tc_put4(sw_hi, sw_lo, tc_off(2 * a, 4 * j), make_float4(c0, -s0, c1, -s1));
    tc_put4(sw_hi, sw_lo, tc_off(2 * a + 1, 4 * j), make_float4(s0, c0, s1, c1));
  }
#pragma unroll
  for (int dd = 0; dd < kTcDG; ++dd) {
    unsigned char* xh = sx_hi + 2 * (size_t)kTcTile * dd;
#pragma unroll
    for (int j = 0; j < kTcK / 4; ++j)
      tc_put4(xh, xh + kTcTile, tc_off(tid, 4 * j),
              make_float4(xv[dd][2 * j].x, xv[dd][2 * j].y, xv[dd][2 * j + 1].x, xv[dd][2 * j + 1].y));
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_tf32(kTcM, kN);
    const uint32_t wh = tc::smem_u32(sw_hi), wl = tc::smem_u32(sw_lo);
    for (int dd = 0; dd < nd; ++dd) {
      const uint32_t xh = tc::smem_u32(sx_hi + 2 * (size_t)kTcTile * dd), xlo = xh + kTcTile;
      bool acc = false;
      for (int pass = 0; pass < 3; ++pass) {  // lo.hi, hi.lo, hi.hi
        const uint32_t pa = pass == 0 ? xlo : xh, pb = pass == 1 ? wl : wh;
        for (int j = 0; j < ks; ++j) {  // K step j covers columns 8j .. 8j + 7: two core matrices
          tc::mma_tf32(tbase + (uint32_t)(dd * kN), tc::smem_desc(pa + 256u * j, kTcLbo, kTcSbo),
                       tc::smem_desc(pb + 256u * j, kTcLbo, kTcSbo), idesc, acc);
          acc = true;
        }
      }
    }
    tc::mma_commit(mbar);
  }
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait_bounded(mbar, 0, kTcWaitNs));
  tc::fence_after_sync();
  float acc[NR];
#pragma unroll
  for (int a = 0; a < NR; ++a) acc[a] = 0.f;
  if (ok) {
    const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
    for (int dd = 0; dd < nd; ++dd) {
#pragma unroll
      for (int h = 0; h < kN / 32; ++h) {
        float y[32];
        tc::tmem_ld32(lane_base + (uint32_t)(dd * kN + h * 32), y);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[h * 16 + j] = fmaf(y[2 * j], y[2 * j], fmaf(y[2 * j + 1], y[2 * j + 1], acc[h * 16 + j]));
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < NR; ++a) acc[a] = __int_as_float(0x7fc00000);
    if ((tid & 31) == 0) atomicOr(err, 1);
    if (tid == 0) tc::mbar_wait_bounded(mbar, 0, kTcWaitNs);  // the MMAs' own completion, once more
  }
  float* out = part + (size_t)g * R * Ns + k0 + tid;
#pragma unroll
  for (int a = 0; a < NR; ++a)
    if (a < R) out[(size_t)a * Ns] = acc[a];
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, kCols);
  }
}

// Pw = fixed-order sum of the Doppler-group partials; also the argmax of Pw as
// the largest key (Pw bits << 32 | ~cell): the lowest cell among equal maxima.
// amax_key must be 0 on entry.
__global__ void k_power_reduce(const float* __restrict__ part, int groups, int cells, float* __restrict__ Pw,
                               unsigned long long* __restrict__ amax_key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long key = 0ull;
  if (i < cells) {
    float s = 0.f;
    for (int g = 0; g < groups; ++g) s += part[(size_t)g * cells + i];
    Pw[i] = s;
    key = ((unsigned long long)__float_as_uint(fmaxf(s, 0.f)) << 32) | (0xffffffffu - (unsigned)i);
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
    key = y > key ? y : key;
  }
  if ((threadIdx.x & 31) == 0 && key) atomicMax(amax_key, key);
}

__device__ inline int amax_cell(const unsigned long long* key) {
  return (int)(0xffffffffu - (unsigned)(*key & 0xffffffffull));
}

struct CfarArg {
  int A, Ns, guard, train;
  float alpha, floor_rel, beta, w_min;
  int E;  // elevation bins: the map has E * A angle rows (row e * A + a) of Ns range cells
};

__device__ inline float lnp(float p) { return logf(fmaxf(p, 1e-30f)); }

__device__ inline void noise_cells(const CfarArg& c, int k, int& lo0, int& lo1, int& hi0, int& hi1) {
  lo0 = max(k - c.guard - c.train, 0);
  lo1 = k - c.guard;  // exclusive
  hi0 = k + c.guard + 1;
  hi1 = min(k + c.guard + c.train + 1, c.Ns);  // exclusive
}

__device__ inline float cfar_noise(const float* __restrict__ row, const CfarArg& c, int k, int* cnt) {
  int lo0, lo1, hi0, hi1;
  noise_cells(c, k, lo0, lo1, hi0, hi1);
  float s = 0.f;
  int n = 0;
  for (int j = lo0; j < lo1; ++j, ++n) s += row[j];
  for (int j = hi0; j < hi1; ++j, ++n) s += row[j];
  *cnt = n;
  return n ? s / (float)n : 0.f;
}

__device__ inline float soft_w(const float* __restrict__ Pw, const CfarArg& c, int a, int k, float floor_v,
                               float* zout, float* nout, int* cnt) {
  const float* row = Pw + (size_t)a * c.Ns;
  const float N = cfar_noise(row, c, k, cnt);
  const float z = (lnp(row[k]) - logf(c.alpha * N + floor_v)) / c.beta;
  if (zout) *zout = z;
  if (nout) *nout = N;
  return 1.f / (1.f + expf(-z));
}

// Detection test of cell i: a 3x3x3 (elevation, azimuth, range) local maximum
// above the floor (equal values: the lower cell wins) whose soft CFAR weight
// reaches w_min; returns the sort key (w descending), or 0xffffffff.
__device__ inline uint32_t detect_key(const float* __restrict__ Pw, const CfarArg& c, int i, float floor_v) {
  const int rho = i / c.Ns, k = i - rho * c.Ns;
  const int e = rho / c.A, a = rho - e * c.A;
  const float p = Pw[i];
  bool peak = p > floor_v;
  for (int de = -1; de <= 1 && peak; ++de)
    for (int da = -1; da <= 1 && peak; ++da)
      for (int dk = -1; dk <= 1; ++dk) {
        if (de == 0 && da == 0 && dk == 0) continue;
        const int ee = e + de, aa = a + da, kk = k + dk;
        if (ee < 0 || ee >= c.E || aa < 0 || aa >= c.A || kk < 0 || kk >= c.Ns) continue;
        const int j = ((ee * c.A) + aa) * c.Ns + kk;
        const float q = Pw[j];
        if (j < i ? !(p > q) : !(p >= q)) {
          peak = false;
          break;
        }
      }
  if (!peak) return 0xffffffffu;
  int cnt;
  const float w = soft_w(Pw, c, rho, k, floor_v, nullptr, nullptr, &cnt);
  return w >= c.w_min ? 0xffffffffu - __float_as_uint(w) : 0xffffffffu;
}

__global__ void k_detect(const float* __restrict__ Pw, CfarArg c, const unsigned long long* __restrict__ amax_key,
                         int32_t* __restrict__ amax, int32_t* __restrict__ flag, uint32_t* __restrict__ key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int am = amax_cell(amax_key);
  if (i == 0) *amax = am;
  if (i >= c.E * c.A * c.Ns) return;
  const uint32_t kk = detect_key(Pw, c, i, c.floor_rel * Pw[am]);
  if (flag) flag[i] = kk != 0xffffffffu ? 1 : 0;
  key[i] = kk;
}

__global__ void k_compact(const int32_t* __restrict__ flag, const int32_t* __restrict__ off,
                          const uint32_t* __restrict__ key, int cells, uint32_t* __restrict__ ko,
                          int32_t* __restrict__ vo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cells || !flag[i]) return;
  ko[off[i]] = key[i];
  vo[off[i]] = i;
}

// exclusive scan of one value per thread over a CTA of whole warps
__device__ inline uint32_t block_exclusive_sel(uint32_t v, uint32_t* total, uint32_t* warp_tot) {
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

__device__ inline float refine(float lm, float l0, float lp, float* dm, float* d0, float* dp) {
  const float den = lm - 2.f * l0 + lp;
  *dm = *d0 = *dp = 0.f;
  if (!(den < 0.f)) return 0.f;
  const float d = 0.5f * (lm - lp) / den;
  if (d <= -0.5f) return -0.5f;
  if (d >= 0.5f) return 0.5f;
  const float id2 = 1.f / (den * den);
  *dm = (lp - l0) * id2;
  *d0 = (lm - lp) * id2;
  *dp = (l0 - lm) * id2;
  return d;
}

struct PointArg {
  CfarArg c;
  int k_max;
  float range_bin;  // c / (2B)
};

// Point i of the cloud from detected cell `cell`: parabolic refine of ln Pw per
// axis (range, azimuth, elevation), then (r u, r v, r sqrt(1 - u^2 - v^2)) with
// its soft weight (v = 0 with one elevation bin).
__device__ inline float4 emit_point(const float* __restrict__ Pw, const PointArg& pa, float floor_v, int cell) {
  const CfarArg& c = pa.c;
  const int rho = cell / c.Ns, k = cell - rho * c.Ns;
  const int e = rho / c.A, a = rho - e * c.A;
  int cnt;
  const float w = soft_w(Pw, c, rho, k, floor_v, nullptr, nullptr, &cnt);
  const float* row = Pw + (size_t)rho * c.Ns;
  const float l0 = lnp(row[k]);
  float t0, t1, t2, dk = 0.f, da = 0.f, de = 0.f;
  if (k > 0 && k < c.Ns - 1) dk = refine(lnp(row[k - 1]), l0, lnp(row[k + 1]), &t0, &t1, &t2);
  if (a > 0 && a < c.A - 1)
    da = refine(lnp(Pw[(size_t)(rho - 1) * c.Ns + k]), l0, lnp(Pw[(size_t)(rho + 1) * c.Ns + k]), &t0, &t1, &t2);
  if (e > 0 && e < c.E - 1)
    de = refine(lnp(Pw[(size_t)(rho - c.A) * c.Ns + k]), l0, lnp(Pw[(size_t)(rho + c.A) * c.Ns + k]), &t0, &t1, &t2);
  const float r = ((float)k + dk) * pa.range_bin;
  const float u = fminf(fmaxf(-1.f + 2.f * ((float)a + da) / (float)c.A, -1.f), 1.f);
  const float v = (2.f * ((float)e + de) + 1.f - (float)c.E) / (float)c.E;
  return make_float4(r * u, r * v, r * sqrtf(fmaxf(1.f - u * u - v * v, 0.f)), w);
}

__global__ void k_points(const float* __restrict__ Pw, PointArg pa, const int32_t* __restrict__ amax,
                         const int32_t* __restrict__ cand, const int32_t* __restrict__ n_cand,
                         float4* __restrict__ pts, int32_t* __restrict__ cell_out,
                         int32_t* __restrict__ n_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = min(*n_cand, pa.k_max);
  if (i == 0) *n_out = n;
  if (i >= pa.k_max) return;
  if (i >= n) {
    pts[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    cell_out[i] = -1;
    return;
  }
  const int cell = cand[i];
  pts[i] = emit_point(Pw, pa, pa.c.floor_rel * Pw[*amax], cell);
  cell_out[i] = cell;
}

// Steps 7-9 in one CTA when the map has at most kSortOneCta cells: compaction
// of k_detect's keys in cell order (rounds of 4096 cells, four per thread, one
// block scan per round places them), the stable sort by weight, and the points.  Same
// results as scan, k_compact, the sort and k_points, in one launch instead of four.
constexpr int kSelThreads = 1024;
constexpr int kRankMax = 256;  // candidates k_select ranks directly (shared memory: 2 KB)
static_assert(2 * kRankMax <= cta::kSortSmemWords, "the rank buffers share the sort's shared memory");
__global__ void __launch_bounds__(kSelThreads) k_select(const float* __restrict__ Pw, PointArg pa,
                                                        const unsigned long long* __restrict__ amax_key,
                                                        const uint32_t* __restrict__ key,
                                                        uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1,
                                                        float4* __restrict__ pts, int32_t* __restrict__ cell_out,
                                                        int32_t* __restrict__ n_out) {
  extern __shared__ __align__(16) uint32_t sel_sm[];  // cta::kSortSmemWords
  __shared__ uint32_t wt[32];
  const CfarArg& c = pa.c;
  const int cells = c.E * c.A * c.Ns, t = threadIdx.x;
  const float floor_v = c.floor_rel * Pw[amax_cell(amax_key)];
  // rounds of 4 x kSelThreads cells (cells is a multiple of 8): thread t loads
  // cells 4t .. 4t + 3 of the round as one coalesced 16-B load, up to four
  // rounds' loads in flight before the first scan
  constexpr int kRound = 4 * kSelThreads, kBatch = 4;
  const uint4* key4 = reinterpret_cast<const uint4*>(key);
  uint32_t base = 0;
  for (int r0 = 0; r0 < cells; r0 += kBatch * kRound) {
    uint4 q[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int cell = r0 + b * kRound + 4 * t;
      q[b] = cell < cells ? __ldcg(&key4[cell >> 2]) : make_uint4(~0u, ~0u, ~0u, ~0u);
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (r0 + b * kRound >= cells) break;  // the same for every thread
      const uint32_t kq[4] = {q[b].x, q[b].y, q[b].z, q[b].w};
      uint32_t mine = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e) mine += kq[e] != 0xffffffffu;
      uint32_t total;
      uint32_t pos = base + block_exclusive_sel(mine, &total, wt);
      const int cell = r0 + b * kRound + 4 * t;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (kq[e] != 0xffffffffu) {
          k0[pos] = kq[e];
          v0[pos] = cell + e;
          ++pos;
        }
      }
      base += total;
    }
  }
  const uint32_t total = base;
  __syncthreads();  // the compacted candidates are visible to the whole CTA
  if (total <= (uint32_t)kRankMax) {
    // few candidates: each one's rank is the number of smaller keys plus the equal keys
    // before it (they are in cell order), i.e. its place in the stable sort, found with
    // two barriers instead of the sort network's dozens
    uint32_t* rk = sel_sm;
    int32_t* rv = reinterpret_cast<int32_t*>(sel_sm + kRankMax);
    for (int i = t; i < (int)total; i += kSelThreads) {
      rk[i] = k0[i];
      rv[i] = v0[i];
    }
    __syncthreads();
    if (t < (int)total) {
      const uint32_t ki = rk[t];
      int r = 0;
      for (int j = 0; j < (int)total; ++j) {
        const uint32_t kj = rk[j];
        r += (kj < ki) | ((kj == ki) & (j < t));
      }
      v0[r] = rv[t];
    }
  } else {
    cta::sort_pairs(k0, v0, k1, v1, (int64_t)total, 32, nullptr, sel_sm);
  }
  __syncthreads();
  const int n = min((int)total, pa.k_max);
  if (t == 0) *n_out = n;
  for (int i = t; i < pa.k_max; i += kSelThreads) {
    if (i >= n) {
      pts[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      cell_out[i] = -1;
    } else {
      const int cell = v0[i];
      pts[i] = emit_point(Pw, pa, floor_v, cell);
      cell_out[i] = cell;
    }
  }
}

// ---- adjoint ----------------------------------------------------------------

// dPw contributions go through the order-independent fixed-point scatter
// (common.cuh): pass 0 records the largest magnitude, pass 1 adds the integers.
template <int kPass>
struct DpwScatter {
  const FixScatter& fs;
  int E;
  float& lmax;
  __device__ void add(size_t cell, float x) const {
    if (kPass == 0) lmax = fmaxf(lmax, fabsf(x));
    else fix_add(&fs.acc[cell], x, E);
  }
};

template <int kPass>
__device__ inline void add_dl(const DpwScatter<kPass>& sc, const float* Pw, size_t cell, float dl) {
  const float p = Pw[cell];
  if (p > 1e-30f && dl != 0.f) sc.add(cell, dl / p);
}

template <int kPass>
__device__ void point_adjoint(int i, const float* __restrict__ Pw, const PointArg& pa, const int32_t* __restrict__ amax,
                              const int32_t* __restrict__ cells, const float4* __restrict__ gpts,
                              const DpwScatter<kPass>& sc) {
  const CfarArg& c = pa.c;
  const int cell = cells[i];
  const int rho = cell / c.Ns, k = cell - rho * c.Ns;
  const int e = rho / c.A, a = rho - e * c.A;
  const int am = *amax;
  const float floor_v = c.floor_rel * Pw[am];
  const float4 g = gpts[i];
  float z, N;
  int cnt;
  const float w = soft_w(Pw, c, rho, k, floor_v, &z, &N, &cnt);
  // soft weight: w = sigmoid(z), z = (l0 - ln(alpha N + F)) / beta
  const float gz = g.w * w * (1.f - w) / c.beta;
  const float den = c.alpha * N + floor_v;
  float dl0 = gz;
  const float dN = -gz * c.alpha / den;
  const float dF = -gz / den;
  sc.add((size_t)am, dF * c.floor_rel);
  if (cnt > 0) {
    int lo0, lo1, hi0, hi1;
    noise_cells(c, k, lo0, lo1, hi0, hi1);
    const float en = dN / (float)cnt;
    for (int j = lo0; j < lo1; ++j) sc.add((size_t)rho * c.Ns + j, en);
    for (int j = hi0; j < hi1; ++j) sc.add((size_t)rho * c.Ns + j, en);
  }
  // position: r = (k + dk) bin, u = -1 + 2 (a + da) / A, v = (2 (e + de) + 1 - E) / E,
  // p = (r u, r v, r sqrt(1 - u^2 - v^2))
  const float* row = Pw + (size_t)rho * c.Ns;
  const float l0 = lnp(row[k]);
  float rm = 0.f, r0 = 0.f, rp = 0.f, am_ = 0.f, a0 = 0.f, ap = 0.f, em = 0.f, e0 = 0.f, ep = 0.f;
  float dk = 0.f, da = 0.f, de = 0.f;
  const bool rk = k > 0 && k < c.Ns - 1, ra = a > 0 && a < c.A - 1, re = e > 0 && e < c.E - 1;
  const size_t up = (size_t)c.A * c.Ns;  // one elevation bin in the map
  if (rk) dk = refine(lnp(row[k - 1]), l0, lnp(row[k + 1]), &rm, &r0, &rp);
  if (ra) da = refine(lnp(Pw[(size_t)cell - c.Ns]), l0, lnp(Pw[(size_t)cell + c.Ns]), &am_, &a0, &ap);
  if (re) de = refine(lnp(Pw[(size_t)cell - up]), l0, lnp(Pw[(size_t)cell + up]), &em, &e0, &ep);
  const float r = ((float)k + dk) * pa.range_bin;
  const float ur = -1.f + 2.f * ((float)a + da) / (float)c.A;
  const float u = fminf(fmaxf(ur, -1.f), 1.f);
  const float v = (2.f * ((float)e + de) + 1.f - (float)c.E) / (float)c.E;
  const float sq = sqrtf(fmaxf(1.f - u * u - v * v, 0.f));
  const float dr = g.x * u + g.y * v + g.z * sq;
  // the clamps of u and of sqrt's argument pass no gradient
  const float du = (ur > -1.f && ur < 1.f) ? (sq > 0.f ? g.x * r - g.z * r * u / sq : g.x * r) : 0.f;
  const float dv = sq > 0.f ? g.y * r - g.z * r * v / sq : g.y * r;
  const float ddk = dr * pa.range_bin;
  const float dda = du * 2.f / (float)c.A;
  const float dde = dv * 2.f / (float)c.E;
  dl0 += ddk * r0 + dda * a0 + dde * e0;
  add_dl(sc, Pw, (size_t)cell, dl0);
  if (rk) {
    add_dl(sc, Pw, (size_t)cell - 1, ddk * rm);
    add_dl(sc, Pw, (size_t)cell + 1, ddk * rp);
  }
  if (ra) {
    add_dl(sc, Pw, (size_t)cell - c.Ns, dda * am_);
    add_dl(sc, Pw, (size_t)cell + c.Ns, dda * ap);
  }
  if (re) {
    add_dl(sc, Pw, (size_t)cell - up, dde * em);
    add_dl(sc, Pw, (size_t)cell + up, dde * ep);
  }
}

template <int kPass>
__global__ void k_points_bwd(const float* __restrict__ Pw, PointArg pa, const int32_t* __restrict__ amax,
                             const int32_t* __restrict__ cells, const int32_t* __restrict__ n_pts,
                             const float4* __restrict__ gpts, FixScatter fs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float lmax = 0.f;
  const DpwScatter<kPass> sc{fs, kPass == 0 ? 0 : fix_exp(*fs.max_bits, fs.log2n), lmax};
  if (i < *n_pts) point_adjoint<kPass>(i, Pw, pa, amax, cells, gpts, sc);
  if (kPass == 0) fix_note_warp(fs.max_bits, lmax);  // every lane of the warp reaches this
}

// dX[v,d,k] = sum_rho conj(W[rho,v]) 2 Y[rho,d,k] dPw[rho,k] over the R = 8 APT angle
// rows, Y recomputed from X.  dPw is read as floats, or, when fs.acc is set, straight
// from the point adjoint's fixed-point sums (acc 2^-E).
template <int APT>
__global__ void __launch_bounds__(256) k_angle_bwd(const float2* __restrict__ X,
                                                   const Steer xl,
                                                   const float* __restrict__ dPw, FixScatter fs, int V, int C,
                                                   int Ns, float2* __restrict__ dX) {
  extern __shared__ float2 sm[];
  constexpr int R = 8 * APT;
  float2* sw = sm;               // [R][V]
  float2* sx = sw + R * V;       // [V][kKT]
  float2* sg = sx + V * kKT;     // [R][kKT]
  load_w(sw, xl, R, V);
  const int kk = threadIdx.x & (kKT - 1), ag = threadIdx.x >> 5;
  const int k0 = blockIdx.x * kKT, d = blockIdx.y;
  for (int i = threadIdx.x; i < V * kKT; i += blockDim.x) {
    const int v = i / kKT, q = i - v * kKT;
    sx[i] = X[((size_t)v * C + d) * Ns + k0 + q];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < APT; ++i) {
    const int a = ag * APT + i;
    float yr = 0.f, yi = 0.f;
    for (int v = 0; v < V; ++v) {
      const float2 w = sw[a * V + v], x = sx[v * kKT + kk];
      yr = fmaf(w.x, x.x, fmaf(-w.y, x.y, yr));
      yi = fmaf(w.x, x.y, fmaf(w.y, x.x, yi));
    }
    const size_t cell = (size_t)a * Ns + k0 + kk;
    const float s = 2.f * (fs.acc ? fix_get(fs.acc[cell], fix_exp(*fs.max_bits, fs.log2n)) : dPw[cell]);
    sg[a * kKT + kk] = make_float2(s * yr, s * yi);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < V * kKT; i += blockDim.x) {
    const int v = i / kKT, q = i - v * kKT;
    float gr = 0.f, gi = 0.f;
    for (int a = 0; a < R; ++a) {
      const float2 w = sw[a * V + v], g = sg[a * kKT + q];  // conj(w) * g
      gr = fmaf(w.x, g.x, fmaf(w.y, g.y, gr));
      gi = fmaf(w.x, g.y, fmaf(-w.y, g.x, gi));
    }
    dX[((size_t)v * C + d) * Ns + k0 + q] = make_float2(gr, gi);
  }
}

inline int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

struct Layout {
  float2* spec;
  float* power;
  int32_t* peak_cell;
  int32_t* n_points;
  int32_t* argmax;
  unsigned long long* amax_key;
  int32_t* err;
  float* part;
  int32_t* flag;
  int32_t* off;
  uint32_t* key;
  uint32_t* skeys[2];
  int32_t* svals[2];
  void* scan_scr;
  void* sort_scr;
  float* dpw;
  unsigned long long* dpw_acc;  // fixed-point dPw of the point adjoint, then its max word
  unsigned int* dpw_max;
  int groups;
};

inline int dgroups(int C) { return C >= 2 ? C / 2 : 1; }  // 2 Doppler bins per CTA: enough CTAs to cover the SMs

// k_select's shared memory exceeds the 48 KB default: raise the limit once per device.
cudaError_t select_attr() {
  static std::atomic<uint64_t> done{0};  // bit per device ordinal below 64
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((done.load() >> dev) & 1u)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cta::kSortSmemBytes);
  if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev);
  return e;
}

// k_angle_tc's shared memory exceeds the 48 KB default: raise the limit once per device.
cudaError_t angle_tc_attr() {
  static std::atomic<uint64_t> done{0};  // bit per device ordinal below 64
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((done.load() >> dev) & 1u)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_angle_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<64>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_angle_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<128>());
  if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev);
  return e;
}

inline int n_elev(const sbr_cfar_cfg* f) { return f->n_elev > 0 ? f->n_elev : 1; }
inline int angle_rows(const sbr_cfar_cfg* f) { return n_elev(f) * f->n_theta; }

size_t pc_layout(Layout* L, void* mem, const sbr_radar_cfg* r, const sbr_cfar_cfg* f) {
  Carver c(mem);
  const int V = r->n_tx * r->n_rx, C = r->n_chirps, Ns = r->n_samples, R = angle_rows(f);
  const int64_t cells = (int64_t)R * Ns;
  L->groups = angle_tc_ok(R, V, Ns) ? (C + kTcDG - 1) / kTcDG : dgroups(C);
  L->spec = c.take<float2>((size_t)V * C * Ns);
  L->power = c.take<float>(cells);
  L->peak_cell = c.take<int32_t>(f->k_max > 0 ? f->k_max : 1);
  L->n_points = c.take<int32_t>(1);
  L->argmax = c.take<int32_t>(1);
  L->amax_key = c.take<unsigned long long>(2);  // [0] argmax key, [1] low word: bounded-wait error bits
  L->err = reinterpret_cast<int32_t*>(L->amax_key + 1);
  L->part = c.take<float>((size_t)L->groups * cells);
  L->flag = c.take<int32_t>(cells);
  L->off = c.take<int32_t>(cells + 1);
  L->key = c.take<uint32_t>(cells);
  L->skeys[0] = c.take<uint32_t>(cells);
  L->skeys[1] = c.take<uint32_t>(cells);
  L->svals[0] = c.take<int32_t>(cells);
  L->svals[1] = c.take<int32_t>(cells);
  L->scan_scr = c.take<char>(scan_scratch_bytes(cells));
  L->sort_scr = c.take<char>(sort_scratch_bytes(cells));
  L->dpw = c.take<float>(cells);
  L->dpw_acc = c.take<unsigned long long>(cells);
  L->dpw_max = c.take<unsigned int>(1);
  return c.bytes();
}

sbr_status check_cfar(const sbr_cfar_cfg* f, const sbr_radar_cfg* r, const char* who) {
  SBR_ARG(f != nullptr, "%s: cfar is NULL", who);
  const int V = r->n_tx * r->n_rx;
  SBR_ARG(f->n_theta >= 8 && f->n_theta <= 256 && (f->n_theta & (f->n_theta - 1)) == 0,
          "%s: n_theta=%d must be a power of two in [8, 256]", who, f->n_theta);
  SBR_ARG(f->n_elev >= 0 && f->n_elev <= 256 && (f->n_elev & (f->n_elev - 1)) == 0,
          "%s: n_elev=%d must be 0 or a power of two", who, f->n_elev);
  SBR_ARG(angle_rows(f) <= 256, "%s: n_elev * n_theta = %d above 256", who, angle_rows(f));
  SBR_ARG(angle_rows(f) * V <= 4096, "%s: n_elev * n_theta * V = %d above 4096", who, angle_rows(f) * V);
  SBR_ARG(f->guard >= 0 && f->train >= 0 && f->guard + f->train < 4096, "%s: bad guard/train", who);
  SBR_ARG(f->k_max >= 1 && f->k_max <= (1 << 20), "%s: k_max=%d outside [1, 2^20]", who, f->k_max);
  SBR_ARG(f->alpha > 0.f && f->beta > 0.f && f->floor_rel >= 0.f, "%s: alpha, beta > 0 needed", who);
  return SBR_OK;
}

// x_v / lambda_c and y_v / lambda_c per virtual antenna and the angle bins.
Steer steering_table(const sbr_radar_cfg* r, const sbr_cfar_cfg* f) {
  Steer s{};
  const double lam = kC / (r->f0 + 0.5 * r->bandwidth);
  for (int t = 0; t < r->n_tx; ++t)
    for (int q = 0; q < r->n_rx; ++q) {
      s.xl[t * r->n_rx + q] = (float)((r->tx[t][0] + r->rx[q][0]) / lam);
      s.yl[t * r->n_rx + q] = (float)((r->tx[t][1] + r->rx[q][1]) / lam);
    }
  s.A = f->n_theta;
  s.E = n_elev(f);
  return s;
}

inline CfarArg cfar_arg(const sbr_radar_cfg* r, const sbr_cfar_cfg* f) {
  return CfarArg{f->n_theta, r->n_samples, f->guard, f->train, f->alpha, f->floor_rel, f->beta, f->w_min, n_elev(f)};
}

template <int APT>
void launch_angle_power(const float2* X, const Steer& xl, int V, int C, int Ns, int groups, float* part,
                        cudaStream_t st) {
  const int R = 8 * APT;
  const size_t sm = sizeof(float2) * ((size_t)R * V + (size_t)V * kKT);
  dim3 grid(Ns / kKT, groups);
  ::sbr::note_launch();
  k_angle_power<APT><<<grid, 256, sm, st>>>(X, xl, V, C, Ns, (C + groups - 1) / groups, part);
}

template <int APT>
void launch_angle_bwd(const float2* X, const Steer& xl, const float* dpw, const FixScatter& fs, int V, int C, int Ns,
                      float2* dX,
                      cudaStream_t st) {
  const int R = 8 * APT;
  const size_t sm = sizeof(float2) * ((size_t)R * V + (size_t)V * kKT + (size_t)R * kKT);
  dim3 grid(Ns / kKT, C);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_angle_bwd<APT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ::sbr::note_launch();
  k_angle_bwd<APT><<<grid, 256, sm, st>>>(X, xl, dpw, fs, V, C, Ns, dX);
}

cudaError_t fft_rows(const float2* in, float2* out, int rows, int n, float sign, cudaStream_t st) {
  const int threads = n / 2 < 256 ? (n / 2 < 32 ? 32 : n / 2) : 256;
  const size_t sm = sizeof(float2) * (n + n / 2);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  ::sbr::note_launch();
  k_fft_rows<<<rows, threads, sm, st>>>(in, out, n, ilog2(n), sign);
  return cudaGetLastError();
}

cudaError_t fft_cols(float2* x, int V, int C, int Ns, float sign, cudaStream_t st) {
  if (C == 1) return cudaSuccess;
  const size_t sm = sizeof(float2) * ((size_t)(C + 1) * kColTile + C / 2);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  ::sbr::note_launch();
  k_fft_cols<<<V * (Ns / kColTile), 256, sm, st>>>(x, C, ilog2(C), Ns, sign);
  return cudaGetLastError();
}

}  // namespace
}  // namespace sbr

using namespace sbr;

extern "C" size_t sbr_pc_bytes(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar) {
  if (check_radar(radar, "sbr_pc_bytes") != SBR_OK || check_cfar(cfar, radar, "sbr_pc_bytes") != SBR_OK)
    return 0;
  Layout L;
  return pc_layout(&L, nullptr, radar, cfar);
}

extern "C" sbr_status sbr_pc_bind(void* d_mem, size_t bytes, const sbr_radar_cfg* radar,
                                  const sbr_cfar_cfg* cfar, sbr_pc_state* out) {
  SBR_ARG(out != nullptr, "sbr_pc_bind: out is NULL");
  sbr_status rs = check_radar(radar, "sbr_pc_bind");
  if (rs != SBR_OK) return rs;
  rs = check_cfar(cfar, radar, "sbr_pc_bind");
  if (rs != SBR_OK) return rs;
  SBR_ARG(d_mem && aligned256(d_mem), "sbr_pc_bind: d_mem NULL or not 256-byte aligned");
  Layout L;
  const size_t need = pc_layout(&L, nullptr, radar, cfar);
  if (bytes < need) {
    set_error("sbr_pc_bind: region of %zu bytes, %zu needed", bytes, need);
    return SBR_ERR_OOM;
  }
  pc_layout(&L, d_mem, radar, cfar);
  out->n_virt = radar->n_tx * radar->n_rx;
  out->n_chirps = radar->n_chirps;
  out->n_samples = radar->n_samples;
  out->n_theta = cfar->n_theta;
  out->k_max = cfar->k_max;
  out->n_elev = n_elev(cfar);
  out->spec = reinterpret_cast<float*>(L.spec);
  out->power = L.power;
  out->peak_cell = L.peak_cell;
  out->n_points = L.n_points;
  out->argmax = L.argmax;
  out->scratch = d_mem;
  return SBR_OK;
}

namespace {
sbr_status state_layout(const sbr_pc_state* s, const sbr_radar_cfg* r, const sbr_cfar_cfg* f, Layout* L,
                        const char* who) {
  SBR_ARG(s && s->scratch, "%s: state is NULL or unbound", who);
  SBR_ARG(s->n_virt == r->n_tx * r->n_rx && s->n_chirps == r->n_chirps && s->n_samples == r->n_samples &&
              s->n_theta == f->n_theta && s->k_max == f->k_max && s->n_elev == n_elev(f),
          "%s: state bound for another configuration", who);
  pc_layout(L, s->scratch, r, f);
  return SBR_OK;
}
}  // namespace

namespace sbr {
namespace {
// Steps 1-4 of T: range FFT, Doppler FFT, angle DFT, power map Pw (and its argmax key).
sbr_status power_map_impl(const float* d_cube, const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, const Layout& L,
                          cudaStream_t st) {
  const int V = radar->n_tx * radar->n_rx, C = radar->n_chirps, Ns = radar->n_samples, R = angle_rows(cfar);
  const int cells = R * Ns;
  const Steer xl = steering_table(radar, cfar);
  // 1-2: range FFT over samples, Doppler FFT over chirps
  SBR_CUDA(fft_rows(reinterpret_cast<const float2*>(d_cube), L.spec, V * C, Ns, -1.f, st));
  SBR_CUDA(fft_cols(L.spec, V, C, Ns, -1.f, st));
  // 3-4: angle DFT and power map (partials per Doppler group, fixed-order sum)
  SBR_CUDA(cudaMemsetAsync(L.amax_key, 0, 2 * sizeof(unsigned long long), st));
  if (angle_tc_ok(R, V, Ns)) {
    SBR_CUDA(angle_tc_attr());
    ::sbr::note_launch();
    const dim3 grid(Ns / kTcM, L.groups);
    if (angle_tc_rows(R) == 64)
      k_angle_tc<64><<<grid, kTcThreads, tc_smem<64>(), st>>>(L.spec, xl, R, V, C, Ns, L.part, L.err);
    else
      k_angle_tc<128><<<grid, kTcThreads, tc_smem<128>(), st>>>(L.spec, xl, R, V, C, Ns, L.part, L.err);
  } else switch (R / 8) {
    case 1: launch_angle_power<1>(L.spec, xl, V, C, Ns, L.groups, L.part, st); break;
    case 2: launch_angle_power<2>(L.spec, xl, V, C, Ns, L.groups, L.part, st); break;
    case 4: launch_angle_power<4>(L.spec, xl, V, C, Ns, L.groups, L.part, st); break;
    case 8: launch_angle_power<8>(L.spec, xl, V, C, Ns, L.groups, L.part, st); break;
    case 16: launch_angle_power<16>(L.spec, xl, V, C, Ns, L.groups, L.part, st); break;
    case 32: launch_angle_power<32>(L.spec, xl, V, C, Ns, L.groups, L.part, st); break;
    default: set_error("sbr_pointcloud: %d angle rows unsupported", R); return SBR_ERR_UNSUPPORTED;
  }
  SBR_CUDA(cudaGetLastError());
  ::sbr::note_launch();
  k_power_reduce<<<(cells + 255) / 256, 256, 0, st>>>(L.part, L.groups, cells, L.power, L.amax_key);
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}
}  // namespace
}  // namespace sbr

extern "C" sbr_status sbr_power_map(const float* d_cube, const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar,
                                    sbr_pc_state* state, sbr_stream stream) {
  SBR_ARG(d_cube, "sbr_power_map: NULL cube");
  sbr_status rs = check_radar(radar, "sbr_power_map");
  if (rs != SBR_OK) return rs;
  rs = check_cfar(cfar, radar, "sbr_power_map");
  if (rs != SBR_OK) return rs;
  Layout L;
  rs = state_layout(state, radar, cfar, &L, "sbr_power_map");
  if (rs != SBR_OK) return rs;
  return power_map_impl(d_cube, radar, cfar, L, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" sbr_status sbr_pointcloud(const float* d_cube, const sbr_radar_cfg* radar,
                                     const sbr_cfar_cfg* cfar, float* d_points, sbr_pc_state* state,
                                     sbr_stream stream) {
  SBR_ARG(d_cube && d_points, "sbr_pointcloud: NULL cube or points");
  sbr_status rs = check_radar(radar, "sbr_pointcloud");
  if (rs != SBR_OK) return rs;
  rs = check_cfar(cfar, radar, "sbr_pointcloud");
  if (rs != SBR_OK) return rs;
  Layout L;
  rs = state_layout(state, radar, cfar, &L, "sbr_pointcloud");
  if (rs != SBR_OK) return rs;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int Ns = radar->n_samples;
  const int cells = angle_rows(cfar) * Ns;
  rs = power_map_impl(d_cube, radar, cfar, L, st);
  if (rs != SBR_OK) return rs;
  // 5-9: soft CFAR, peaks, compaction in cell order, stable sort by weight, points
  const CfarArg ca = cfar_arg(radar, cfar);
  PointArg pa{ca, cfar->k_max, (float)(kC / (2.0 * radar->bandwidth))};
  if (cells <= kSortOneCta) {
    SBR_CUDA(select_attr());
    ::sbr::note_launch();
    k_detect<<<(cells + 255) / 256, 256, 0, st>>>(L.power, ca, L.amax_key, L.argmax, nullptr, L.key);
    ::sbr::note_launch();
    k_select<<<1, kSelThreads, cta::kSortSmemBytes, st>>>(L.power, pa, L.amax_key, L.key, L.skeys[0],
                                                           L.svals[0], L.skeys[1], L.svals[1],
                                                           reinterpret_cast<float4*>(d_points), L.peak_cell,
                                                           L.n_points);
    SBR_CUDA(cudaGetLastError());
    return SBR_OK;
  }
  ::sbr::note_launch();
  k_detect<<<(cells + 255) / 256, 256, 0, st>>>(L.power, ca, L.amax_key, L.argmax, L.flag, L.key);
  SBR_CUDA(exclusive_scan(L.flag, L.off, cells, nullptr, L.scan_scr, st));
  ::sbr::note_launch();
  k_compact<<<(cells + 255) / 256, 256, 0, st>>>(L.flag, L.off, L.key, cells, L.skeys[0], L.svals[0]);
  SBR_CUDA(radix_sort_pairs(L.skeys, L.svals, cells, L.off + cells, 32, L.sort_scr, st));
  // 8-9: refine and emit points
  ::sbr::note_launch();
  k_points<<<(cfar->k_max + 255) / 256, 256, 0, st>>>(L.power, pa, L.argmax, L.svals[0], L.off + cells,
                                                       reinterpret_cast<float4*>(d_points), L.peak_cell,
                                                       L.n_points);
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}

extern "C" sbr_status sbr_pc_check(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar,
                                   const sbr_pc_state* state, sbr_stream stream) {
  sbr_status rs = check_radar(radar, "sbr_pc_check");
  if (rs != SBR_OK) return rs;
  rs = check_cfar(cfar, radar, "sbr_pc_check");
  if (rs != SBR_OK) return rs;
  Layout L;
  rs = state_layout(state, radar, cfar, &L, "sbr_pc_check");
  if (rs != SBR_OK) return rs;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SBR_CUDA(cudaStreamSynchronize(st));
  int32_t err = 0;
  SBR_CUDA(cudaMemcpy(&err, L.err, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) {
    set_error("sbr_pc_check: the tensor-core angle kernel gave up waiting for its matrix products "
              "(status 0x%x); the power map holds NaN",
              (unsigned)err);
    return SBR_ERR_TIMEOUT;
  }
  return SBR_OK;
}

namespace sbr {
namespace {
// dL/dcube from dL/dPw (L.dpw, or the fixed-point sums in fs when fs.acc is set):
// dY = 2 Y dPw, dX = W^H dY, then the adjoints of the forward DFTs (unnormalised
// inverse transforms, in place).
sbr_status cube_adjoint(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, const Layout& L, const FixScatter& fs,
                        float* d_gcube, cudaStream_t st) {
  const int V = radar->n_tx * radar->n_rx, C = radar->n_chirps, Ns = radar->n_samples, R = angle_rows(cfar);
  const Steer xl = steering_table(radar, cfar);
  float2* g = reinterpret_cast<float2*>(d_gcube);
  switch (R / 8) {
    case 1: launch_angle_bwd<1>(L.spec, xl, L.dpw, fs, V, C, Ns, g, st); break;
    case 2: launch_angle_bwd<2>(L.spec, xl, L.dpw, fs, V, C, Ns, g, st); break;
    case 4: launch_angle_bwd<4>(L.spec, xl, L.dpw, fs, V, C, Ns, g, st); break;
    case 8: launch_angle_bwd<8>(L.spec, xl, L.dpw, fs, V, C, Ns, g, st); break;
    case 16: launch_angle_bwd<16>(L.spec, xl, L.dpw, fs, V, C, Ns, g, st); break;
    case 32: launch_angle_bwd<32>(L.spec, xl, L.dpw, fs, V, C, Ns, g, st); break;
    default: set_error("%d angle rows unsupported", R); return SBR_ERR_UNSUPPORTED;
  }
  SBR_CUDA(cudaGetLastError());
  SBR_CUDA(fft_cols(g, V, C, Ns, +1.f, st));
  SBR_CUDA(fft_rows(g, g, V * C, Ns, +1.f, st));
  return SBR_OK;
}

constexpr int kMseThreads = 1024;

// Eq. 16 on the power map: loss = (1/N) sum_i (Pw_i - T_i)^2 and dL/dPw_i = 2 (Pw_i - T_i) / N;
// one CTA, each thread over a fixed stride of cells, then a fixed-order block sum.
__global__ void __launch_bounds__(kMseThreads) k_image_mse(const float* __restrict__ Pw, const float* __restrict__ T,
                                                           int cells, float* __restrict__ loss,
                                                           float* __restrict__ dpw) {
  __shared__ float red[kMseThreads / 32];
  const float inv_n = 1.f / (float)cells;
  float s = 0.f;
  for (int i = threadIdx.x; i < cells; i += kMseThreads) {
    const float d = Pw[i] - T[i];
    s = fmaf(d, d, s);
    if (dpw) dpw[i] = 2.f * d * inv_n;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = red[threadIdx.x];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *loss = t * inv_n;
  }
}
}  // namespace
}  // namespace sbr

extern "C" sbr_status sbr_image_loss(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, const sbr_pc_state* state,
                                     const float* d_target, float* d_loss, float* d_gcube, sbr_stream stream) {
  SBR_ARG(d_target && d_loss, "sbr_image_loss: NULL target or loss");
  sbr_status rs = check_radar(radar, "sbr_image_loss");
  if (rs != SBR_OK) return rs;
  rs = check_cfar(cfar, radar, "sbr_image_loss");
  if (rs != SBR_OK) return rs;
  Layout L;
  rs = state_layout(state, radar, cfar, &L, "sbr_image_loss");
  if (rs != SBR_OK) return rs;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int cells = angle_rows(cfar) * radar->n_samples;
  ::sbr::note_launch();
  k_image_mse<<<1, kMseThreads, 0, st>>>(L.power, d_target, cells, d_loss, d_gcube ? L.dpw : nullptr);
  SBR_CUDA(cudaGetLastError());
  if (!d_gcube) return SBR_OK;
  return cube_adjoint(radar, cfar, L, FixScatter{nullptr, nullptr, 0}, d_gcube, st);
}

extern "C" sbr_status sbr_pointcloud_bwd(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar,
                                         const sbr_pc_state* state, const float* d_gpoints,
                                         float* d_gcube, sbr_stream stream) {
  SBR_ARG(d_gpoints && d_gcube, "sbr_pointcloud_bwd: NULL gradient");
  sbr_status rs = check_radar(radar, "sbr_pointcloud_bwd");
  if (rs != SBR_OK) return rs;
  rs = check_cfar(cfar, radar, "sbr_pointcloud_bwd");
  if (rs != SBR_OK) return rs;
  Layout L;
  rs = state_layout(state, radar, cfar, &L, "sbr_pointcloud_bwd");
  if (rs != SBR_OK) return rs;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int cells = angle_rows(cfar) * radar->n_samples;
  // accumulator and max word are adjacent: one memset clears both
  SBR_CUDA(cudaMemsetAsync(L.dpw_acc, 0,
                           reinterpret_cast<char*>(L.dpw_max + 1) - reinterpret_cast<char*>(L.dpw_acc), st));
  const CfarArg ca = cfar_arg(radar, cfar);
  PointArg pa{ca, cfar->k_max, (float)(kC / (2.0 * radar->bandwidth))};
  // adds per point: floor, 2 train windows, the cell, 2 neighbours per refined axis
  const int64_t per_point = 6 + 2 * (int64_t)cfar->train + (ca.E > 1 ? 2 : 0);
  FixScatter fs{L.dpw_acc, L.dpw_max, ceil_log2((int64_t)cfar->k_max * per_point)};
  const float4* gp = reinterpret_cast<const float4*>(d_gpoints);
  const int nb = (cfar->k_max + 255) / 256;
  ::sbr::note_launch();
  k_points_bwd<0><<<nb, 256, 0, st>>>(L.power, pa, L.argmax, L.peak_cell, L.n_points, gp, fs);
  ::sbr::note_launch();
  k_points_bwd<1><<<nb, 256, 0, st>>>(L.power, pa, L.argmax, L.peak_cell, L.n_points, gp, fs);
  return cube_adjoint(radar, cfar, L, fs, d_gcube, st);
}
