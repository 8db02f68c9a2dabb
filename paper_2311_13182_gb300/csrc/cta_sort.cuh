// One-CTA stable radix sort of (key, value) pairs, callable from any kernel
// running 1024 threads with kSortSmemBytes of dynamic shared memory: the
// single-launch sort of scan_sort.cu and the point cloud's fused selection.
#pragma once

#include "common.cuh"

namespace sbr {
namespace cta {

constexpr int kSmallThreads = 1024;  // threads of the calling CTA
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

// Stable LSD sort of (key, value) pairs by one CTA.  All digit histograms come
// from one sweep up front; then each pass moves the array in rounds of 8192
// items.  A round ranks items inside each warp by digit (warp-level multisplit:
// the lanes holding equal digits find each other with one ballot per digit bit,
// and rank by their lane order after the warp's running count of that digit), turns the
// per-(digit, warp) counts into output offsets with one scan per digit across
// warps, and scatters.  Item order within a round is (warp, slot, lane), which
// is input order, so equal keys keep their order.
// n live keys (already clamped); sm: kSortSmemWords of shared memory.
__device__ inline void sort_pairs(uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int64_t n, int bits,
                                  const uint32_t* __restrict__ d_hist, uint32_t* sm) {
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

}  // namespace cta
}  // namespace sbr
