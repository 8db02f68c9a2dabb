// Device-wide exclusive scan and stable LSD radix sort (4-bit digits).
//
// Used for path compaction (ray -> first path index), the LBVH's Morton-code
// sort and the point-cloud candidate ordering.  Both are three-phase (tile
// totals, scan of totals, tile-local scan/scatter): no inter-CTA waiting, so no
// kernel here can spin.
#include <stdio.h>

#include <atomic>

#include "cta_sort.cuh"

namespace sbr {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__device__ inline int64_t clamp_n(int64_t cap, const int32_t* d_n) {
  if (!d_n) return cap;
  int64_t n = *d_n;
  return n < 0 ? 0 : (n > cap ? cap : n);
}

// Exclusive scan of one uint32 per thread across the block (blockDim multiple of 32).
// Lanes of packed 16-bit counters scan independently as long as no half overflows.
__device__ inline uint32_t block_exclusive(uint32_t v, uint32_t* total, uint32_t* warp_tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;
  }
  __syncthreads();
  uint32_t res = (w ? warp_tot[w - 1] : 0u) + x - v;
  *total = warp_tot[nw - 1];
  __syncthreads();
  return res;
}

__global__ void k_tile_sums(const int32_t* __restrict__ in, int64_t cap, const int32_t* d_n,
                            int32_t* __restrict__ sums) {
  __shared__ uint32_t wt[32];
  const int64_t n = clamp_n(cap, d_n);
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i)
    if (base + i < n) s += (uint32_t)in[base + i];
  uint32_t tot;
  block_exclusive(s, &tot, wt);
  if (threadIdx.x == 0) sums[blockIdx.x] = (int32_t)tot;
}

// In-place exclusive scan of m values with one CTA (m up to a few million).
__global__ void k_scan_single(int32_t* __restrict__ a, int64_t m) {
  __shared__ uint32_t wt[32];
  uint32_t carry = 0;
  for (int64_t base = 0; base < m; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < m ? (uint32_t)a[i] : 0u;
    uint32_t tot;
    uint32_t ex = block_exclusive(v, &tot, wt);
    if (i < m) a[i] = (int32_t)(carry + ex);
    carry += tot;
  }
}

__global__ void k_tile_scan(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t cap,
                            const int32_t* d_n, const int32_t* __restrict__ sums) {
  __shared__ uint32_t wt[32];
  const int64_t n = clamp_n(cap, d_n);
  if (n == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
    return;
  }
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  int32_t v[kItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += (uint32_t)v[i];
  }
  uint32_t tot;
  uint32_t run = block_exclusive(s, &tot, wt) + (uint32_t)sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (base + i < n) out[base + i] = (int32_t)run;
    run += (uint32_t)v[i];
    if (base + i == n - 1) out[n] = (int32_t)run;
  }
}

// ---- radix sort -------------------------------------------------------------

__global__ void k_digit_hist(const uint32_t* __restrict__ keys, int64_t cap, const int32_t* d_n,
                             int shift, int32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t cnt[16];
  if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t n = clamp_n(cap, d_n);
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
#pragma unroll
  for (int i = 0; i < kItems; ++i)
    if (base + i < n) atomicAdd(&cnt[(keys[base + i] >> shift) & 15u], 1u);
  __syncthreads();
  if (threadIdx.x < 16) hist[threadIdx.x * ntiles + blockIdx.x] = (int32_t)cnt[threadIdx.x];
}

// Stable scatter: each thread owns kItems consecutive items, so item order is
// (thread, slot) order; per-digit offsets come from a block scan of packed
// 16-bit per-thread digit counts (two digits per 32-bit word).
__global__ void k_digit_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                                int64_t cap, const int32_t* d_n, int shift,
                                const int32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t wt[32];
  __shared__ int32_t tile_off[16];
  if (threadIdx.x < 16) tile_off[threadIdx.x] = hist[threadIdx.x * ntiles + blockIdx.x];
  const int64_t n = clamp_n(cap, d_n);
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  uint32_t key[kItems];
  int32_t val[kItems];
  int dig[kItems];
  uint32_t cnt[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) cnt[j] = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    bool ok = base + i < n;
    key[i] = ok ? kin[base + i] : 0u;
    val[i] = ok ? vin[base + i] : 0;
    dig[i] = ok ? (int)((key[i] >> shift) & 15u) : -1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (ok && (dig[i] >> 1) == j) cnt[j] += 1u << (16 * (dig[i] & 1));
  }
  uint32_t pre[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint32_t tot;
    pre[j] = block_exclusive(cnt[j], &tot, wt);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (dig[i] < 0) continue;
    const int d = dig[i];
    uint32_t p = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if ((d >> 1) == j) p = pre[j];
    const uint32_t rank = (p >> (16 * (d & 1))) & 0xffffu;
    const int64_t pos = (int64_t)tile_off[d] + rank;
    kout[pos] = key[i];
    vout[pos] = val[i];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if ((d >> 1) == j) pre[j] += 1u << (16 * (d & 1));
  }
}

inline int tiles_for(int64_t n) { return (int)((n + kTile - 1) / kTile); }

// ---- single-CTA variants for small inputs -----------------------------------
//
// Below kSmall elements a scan runs in one CTA (one launch instead of three),
// and so does a sort of up to kSmall keys: the LBVH's Morton codes (tens of
// thousands of triangles) and the point cloud's detected peaks.  The sort uses
// 8-bit digits (four passes for 32-bit keys, against eight 4-bit passes of
// three launches each on the multi-CTA path).

constexpr int kSmall = (int)kSortOneCta;
using cta::kSmallThreads;
using cta::kBitonicMax;
using cta::kSortSmemBytes;

__global__ void __launch_bounds__(kSmallThreads) k_scan_small(const int32_t* __restrict__ in,
                                                              int32_t* __restrict__ out, int64_t cap,
                                                              const int32_t* d_n) {
  __shared__ uint32_t wt[32];
  const int64_t n = clamp_n(cap, d_n);
  uint32_t carry = 0;
  for (int64_t base = 0; base < n; base += (int64_t)kSmallThreads * kItems) {
    const int64_t b = base + (int64_t)threadIdx.x * kItems;
    int32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      v[i] = b + i < n ? in[b + i] : 0;
      s += (uint32_t)v[i];
    }
    uint32_t tot;
    uint32_t run = carry + block_exclusive(s, &tot, wt);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      if (b + i < n) out[b + i] = (int32_t)run;
      run += (uint32_t)v[i];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = (int32_t)carry;
}

__global__ void __launch_bounds__(kSmallThreads) k_sort_small(uint32_t* k0, int32_t* v0, uint32_t* k1,
                                                              int32_t* v1, int64_t cap, const int32_t* d_n,
                                                              int bits, const uint32_t* __restrict__ d_hist) {
  extern __shared__ __align__(16) uint32_t sm[];  // kSortSmemWords
  cta::sort_pairs(k0, v0, k1, v1, clamp_n(cap, d_n), bits, d_hist, sm);
}

// The sort's shared memory exceeds the 48 KB default: raise the limit once per device.
cudaError_t sort_small_attr() {
  static std::atomic<uint64_t> done{0};  // bit per device ordinal below 64
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((done.load() >> dev) & 1u)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmemBytes);
  if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev);
  return e;
}

}  // namespace

size_t scan_scratch_bytes(int64_t capacity) {
  return (size_t)(tiles_for(capacity) + 1) * sizeof(int32_t);
}

cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t n, const int32_t* d_n,
                           void* scratch, cudaStream_t s) {
  if (n <= kSmall) {
    ::sbr::note_launch();
    k_scan_small<<<1, kSmallThreads, 0, s>>>(in, out, n, d_n);
    return cudaGetLastError();
  }
  const int nt = tiles_for(n < 1 ? 1 : n);
  int32_t* sums = static_cast<int32_t*>(scratch);
  ::sbr::note_launch();
  k_tile_sums<<<nt, kThreads, 0, s>>>(in, n, d_n, sums);
  ::sbr::note_launch();
  k_scan_single<<<1, 1024, 0, s>>>(sums, nt);
  ::sbr::note_launch();
  k_tile_scan<<<nt, kThreads, 0, s>>>(in, out, n, d_n, sums);
  return cudaGetLastError();
}

size_t sort_scratch_bytes(int64_t capacity) {
  return (size_t)16 * tiles_for(capacity < 1 ? 1 : capacity) * sizeof(int32_t);
}

cudaError_t radix_sort_pairs(uint32_t* keys[2], int32_t* vals[2], int64_t n, const int32_t* d_n,
                             int bits, void* scratch, cudaStream_t s, const uint32_t* d_hist) {
  if (n <= kSmall) {  // one launch in place of 3 per 4-bit pass
    cudaError_t e = sort_small_attr();
    if (e != cudaSuccess) return e;
    ::sbr::note_launch();
    k_sort_small<<<1, kSmallThreads, kSortSmemBytes, s>>>(keys[0], vals[0], keys[1], vals[1], n, d_n, bits,
                                                          d_hist);
    return cudaGetLastError();
  }
  const int passes = (bits + 3) / 4;
  const int nt = tiles_for(n < 1 ? 1 : n);
  int32_t* hist = static_cast<int32_t*>(scratch);
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = 4 * p;
    ::sbr::note_launch();
    k_digit_hist<<<nt, kThreads, 0, s>>>(keys[cur], n, d_n, shift, hist, nt);
    ::sbr::note_launch();
    k_scan_single<<<1, 1024, 0, s>>>(hist, (int64_t)16 * nt);
    ::sbr::note_launch();
    k_digit_scatter<<<nt, kThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n,
                                            d_n, shift, hist, nt);
    cur ^= 1;
  }
  if (cur == 1) {  // odd number of passes: copy back so the result is in buffer 0
    cudaMemcpyAsync(keys[0], keys[1], (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(vals[0], vals[1], (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

}  // namespace sbr
