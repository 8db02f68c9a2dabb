// Device-wide exclusive scan and stable LSD radix sort (4-bit digits).
//
// Used for path compaction (ray -> first path index), the LBVH's Morton-code
// sort and the point-cloud candidate ordering.  Both are three-phase (tile
// totals, scan of totals, tile-local scan/scatter): no inter-CTA waiting, so no
// kernel here can spin.
#include <stdio.h>

#include <atomic>

#include "common.cuh"

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
constexpr int kSmallThreads = 1024;
constexpr int kBitonicMax = 2048;  // keys sorted in shared memory by one bitonic network
constexpr int kWarps = kSmallThreads / 32;
constexpr int kRankItems = 8;                                // items per thread per round
constexpr int kRankRound = kSmallThreads * kRankItems;       // 8192 items per round
constexpr int kCntStride = 257;                              // padded per-warp row of 256 counters
// dynamic shared memory (words): per-warp counters, per-pass digit offsets,
// round digit totals and starts, and the round's items regrouped by digit
constexpr int kSortSmemWords = kWarps * kCntStride + 4 * 256 + 2 * 256 + 2 * kRankRound;
constexpr size_t kSortSmemBytes = (size_t)kSortSmemWords * 4;
static_assert(kWarps * kCntStride * 4 >= kBitonicMax * 8, "bitonic buffer shares the counter storage");

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

// Stable LSD sort of (key, value) pairs by one CTA.  All digit histograms come
// from one sweep up front; then each pass moves the array in rounds of 8192
// items.  A round ranks items inside each warp by digit (warp-level multisplit:
// the lanes holding equal digits find each other with one ballot per digit bit,
// and rank by their lane order after the warp's running count of that digit), turns the
// per-(digit, warp) counts into output offsets with one scan per digit across
// warps, and scatters.  Item order within a round is (warp, slot, lane), which
// is input order, so equal keys keep their order.
__global__ void __launch_bounds__(kSmallThreads) k_sort_small(uint32_t* k0, int32_t* v0, uint32_t* k1,
                                                              int32_t* v1, int64_t cap, const int32_t* d_n,
                                                              int bits, const uint32_t* __restrict__ d_hist) {
  extern __shared__ __align__(16) uint32_t sm[];  // kSortSmemWords
  const int64_t n = clamp_n(cap, d_n);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (n <= kBitonicMax) {
    // few live keys: bitonic sort of (key, value) pairs in shared memory; the
    // values are distinct and already ascending in input order for equal keys
    // (cell order), so the lexicographic order equals the stable radix order
    unsigned long long* bsort = reinterpret_cast<unsigned long long*>(sm);
    int N = 1;
    while (N < n) N <<= 1;
    for (int i = threadIdx.x; i < N; i += kSmallThreads)
      bsort[i] = i < n ? ((unsigned long long)k0[i] << 32) | (uint32_t)v0[i] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < N; i += kSmallThreads) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long a = bsort[i], b = bsort[ixj];
            if ((a > b) == ((i & k) == 0)) {
              bsort[i] = b;
              bsort[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
      k0[i] = (uint32_t)(bsort[i] >> 32);
      v0[i] = (int32_t)(uint32_t)bsort[i];
    }
    return;
  }
  const int passes = (bits + 7) / 8;  // <= 4
  uint32_t* cnt = sm;                      // [warp][digit], row stride kCntStride
  uint32_t* off = sm + kWarps * kCntStride;  // [pass][digit]: running output offset
  uint32_t* tot = off + 4 * 256;             // [digit]: items of the round
  uint32_t* lstart = tot + 256;              // [digit]: start of the digit in the round's staging
  uint32_t* stage_k = lstart + 256;          // [kRankRound] the round's items grouped by digit
  int32_t* stage_v = reinterpret_cast<int32_t*>(stage_k + kRankRound);
  // 1. histograms of every digit place (given, or counted here)
  if (d_hist) {
    for (int i = threadIdx.x; i < 4 * 256; i += kSmallThreads) off[i] = d_hist[i];
  } else {
    for (int i = threadIdx.x; i < 4 * 256; i += kSmallThreads) off[i] = 0u;
    __syncthreads();
    for (int64_t base = 0; base < n; base += kRankRound) {
      uint32_t key[kRankItems];
#pragma unroll
      for (int j = 0; j < kRankItems; ++j) {  // all loads in flight before the first ballot
        const int64_t i = base + (int64_t)j * kSmallThreads + threadIdx.x;
        key[j] = i < n ? k0[i] : 0u;
      }
#pragma unroll
      for (int j = 0; j < kRankItems; ++j) {
        const bool ok = base + (int64_t)j * kSmallThreads + threadIdx.x < n;
        for (int p = 0; p < passes; ++p) {
          const uint32_t d = (key[j] >> (8 * p)) & 255u;
          const uint32_t peers = warp_peers8(d, ok);
          if (ok && lane == __ffs(peers) - 1) atomicAdd(&off[256 * p + d], (uint32_t)__popc(peers));
        }
      }
    }
  }
  __syncthreads();
  // exclusive scan of each place's 256 counts: warp p, 8 digits per lane
  if (w < passes) {
    uint32_t c[8], s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = off[256 * w + 8 * lane + j];
      s += c[j];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    uint32_t run = x - s;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      off[256 * w + 8 * lane + j] = run;
      run += c[j];
    }
  }
  __syncthreads();
  // 2. passes
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t* kin = k0;
  int32_t* vin = v0;
  uint32_t* kout = k1;
  int32_t* vout = v1;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    uint32_t* run = off + 256 * p;
    for (int64_t base = 0; base < n; base += kRankRound) {
      uint32_t* row = cnt + w * kCntStride;
      uint32_t key[kRankItems], rank[kRankItems];
      int32_t val[kRankItems];
#pragma unroll
      for (int j = 0; j < kRankItems; ++j) {  // all loads in flight before the ranking
        const int64_t i = base + (int64_t)w * (32 * kRankItems) + 32 * j + lane;
        key[j] = i < n ? kin[i] : 0u;
        val[j] = i < n ? vin[i] : 0;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) row[lane + 32 * j] = 0u;
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kRankItems; ++j) {
        const bool ok = base + (int64_t)w * (32 * kRankItems) + 32 * j + lane < n;
        const uint32_t d = (key[j] >> shift) & 255u;
        const uint32_t peers = warp_peers8(d, ok);
        const uint32_t before = ok ? row[d] : 0u;
        rank[j] = ok ? before + __popc(peers & lt) : 0xffffffffu;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) row[d] = before + __popc(peers);
        __syncwarp();
      }
      __syncthreads();
      // per digit: exclusive scan of the warps' counts; warp w handles digits
      // w, w+32, ...
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int d = w + 32 * j;
        const uint32_t c = cnt[lane * kCntStride + d];
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        cnt[lane * kCntStride + d] = x - c;
        if (lane == 31) tot[d] = x;
      }
      __syncthreads();
      if (w == 0) {  // digit starts within the round
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          c[j] = tot[8 * lane + j];
          sum += c[j];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        uint32_t r = x - sum;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          lstart[8 * lane + j] = r;
          r += c[j];
        }
      }
      __syncthreads();
      // regroup the round by digit in shared memory ...
#pragma unroll
      for (int j = 0; j < kRankItems; ++j) {
        if (rank[j] == 0xffffffffu) continue;
        const uint32_t d = (key[j] >> shift) & 255u;
        const uint32_t q = lstart[d] + row[d] + rank[j];
        stage_k[q] = key[j];
        stage_v[q] = val[j];
      }
      __syncthreads();
      // ... and write it out in runs of equal digits (coalesced stores)
      const int rn = n - base < kRankRound ? (int)(n - base) : kRankRound;
      for (int q = threadIdx.x; q < rn; q += kSmallThreads) {
        const uint32_t key = stage_k[q];
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t pos = run[d] + (uint32_t)q - lstart[d];
        if (pos < (uint32_t)n) {  // always true when the histogram matches the keys
          kout[pos] = key;
          vout[pos] = stage_v[q];
        }
      }
      __syncthreads();
      if (threadIdx.x < 256) run[threadIdx.x] += tot[threadIdx.x];
      // the next round's first barrier orders this update before any use
    }
    __syncthreads();  // the pass's output is visible to the whole CTA
    uint32_t* tk = kin;
    kin = kout;
    kout = tk;
    int32_t* tv = vin;
    vin = vout;
    vout = tv;
  }
  if (kin != k0) {  // odd number of passes: the result is in buffer 1
    for (int64_t i = threadIdx.x; i < n; i += kSmallThreads) {
      k0[i] = k1[i];
      v0[i] = v1[i];
    }
  }
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
