// Radix-2 FFT pieces shared by the point-cloud transforms and the synthesis:
// complex product, bit reversal, a per-CTA twiddle table and the in-place
// shared-memory transform.
#pragma once

#include <cuda_runtime.h>

namespace sbr {
namespace fft {

__device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ inline int bitrev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// Twiddles tw[j] = e^{sign 2 pi i j / n}, j < n / 2, into shared memory; the
// stage of length len = 2^m takes tw[j << (logn - m)] (the same float argument
// 2 j / len as a direct evaluation: both quotients are exact).
__device__ inline void fill_twiddles(float2* tw, int n, float sign, int lanes, int lane) {
  for (int j = lane; j < (n >> 1); j += lanes) {
    float sn, cs;
    sincospif(sign * 2.f * (float)j / (float)n, &sn, &cs);
    tw[j] = make_float2(cs, sn);
  }
}

// In-place radix-2 DIT FFT of n points held in shared memory (already in
// bit-reversed order) with the twiddles of fill_twiddles, all threads of the
// block cooperating.
__device__ inline void smem_fft(float2* s, const float2* tw, int logn, int lanes, int lane) {
  const int n = 1 << logn;
  for (int m = 1; m <= logn; ++m) {
    const int half = 1 << (m - 1);
    for (int u = lane; u < (n >> 1); u += lanes) {
      const int j = u & (half - 1);
      const int i0 = ((u >> (m - 1)) << m) + j, i1 = i0 + half;
      const float2 t = cmul(s[i1], tw[j << (logn - m)]);
      const float2 a = s[i0];
      s[i0] = make_float2(a.x + t.x, a.y + t.y);
      s[i1] = make_float2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

}  // namespace fft
}  // namespace sbr
