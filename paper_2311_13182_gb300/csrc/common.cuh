// Shared helpers of libsbr: status/error plumbing, region carving, small vector math.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "sbr.h"

namespace sbr {

void set_error(const char* fmt, ...);

// Host-side count of kernel launches issued by the library (sbr_launch_count).
void note_launch();

constexpr double kC = 299792458.0;  // m/s
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kAlign = 256;

// Carves sub-regions out of one caller-provided device allocation.  Used twice:
// once with base = nullptr to size the region, once to bind pointers.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t bytes() const { return (off + kAlign - 1) / kAlign * kAlign; }
};

inline bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

// ---- device scan / sort utilities (scan_sort.cu) --------------------------

// Exclusive scan of n int32 (n from host, or from *d_n when d_n != nullptr with
// n as the capacity).  out[n_actual] receives the total.  scratch needs
// scan_scratch_bytes(capacity).
size_t scan_scratch_bytes(int64_t capacity);
cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t n, const int32_t* d_n,
                           void* scratch, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys.  Ping-pongs between the two buffers; the sorted result ends in
// keys[0]/vals[0].  n from host, or from *d_n (n = capacity).  Up to
// kSortOneCta keys sort in one CTA with 8-bit digits; d_hist, when not NULL,
// then holds the caller's counts of every digit place (place p's 256 counts at
// [256p, 256p + 256), for the live keys), which spares the CTA its counting
// sweep.  Larger inputs take the multi-CTA path (4-bit digits) and ignore it.
constexpr int64_t kSortOneCta = 65536;
size_t sort_scratch_bytes(int64_t capacity);
cudaError_t radix_sort_pairs(uint32_t* keys[2], int32_t* vals[2], int64_t n, const int32_t* d_n,
                             int bits, void* scratch, cudaStream_t s, const uint32_t* d_hist = nullptr);

// Lanes of the calling warp (all 32 active) whose 8-bit value d equals this
// lane's, restricted to lanes with ok set: one ballot per bit.
__device__ inline uint32_t warp_peers8(uint32_t d, bool ok) {
  uint32_t m = __ballot_sync(0xffffffffu, ok);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const uint32_t bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bal : ~bal;
  }
  return m;
}

// ---- order-independent (bitwise deterministic) scatter-add -------------------
//
// Float atomics add in whatever order threads arrive, so such sums change in
// their last bits from run to run.  This scatter adds integers instead, whose sum
// does not depend on the order: pass 1 finds the largest magnitude m among the
// contributions (atomicMax on the float bits), pass 2 adds each contribution x as
// round(x 2^E) to a 64-bit accumulator, E chosen so that 2^log2n contributions of
// magnitude <= m stay below 2^62, and a finishing pass converts acc 2^-E back to
// float.  The resolution 2^-E is about m 2^(log2n - 61), ~1e-12 m for a million
// contributions: far finer than the FP32 sum it replaces.
struct FixScatter {
  unsigned long long* acc;  // zeroed before pass 2
  unsigned int* max_bits;   // zeroed before pass 1
  int log2n;                // ceil(log2(a bound on the number of contributions))
};

__host__ inline int ceil_log2(int64_t n) {
  int l = 0;
  while (l < 62 && ((int64_t)1 << l) < n) ++l;
  return l;
}

// Exponent E for the largest magnitude recorded: m < 2^e with e = biased exponent - 126.
__device__ inline int fix_exp(unsigned int max_bits, int log2n) {
  return 62 - log2n - ((int)((max_bits >> 23) & 0xffu) - 126);
}
__device__ inline void fix_add(unsigned long long* acc, float x, int E) {
  atomicAdd(acc, (unsigned long long)__double2ll_rn(ldexp((double)x, E)));
}
__device__ inline float fix_get(unsigned long long a, int E) { return (float)ldexp((double)(long long)a, -E); }
// Warp-reduced max of |x| over the calling warp's lanes (all 32 must call), one atomic per warp.
__device__ inline void fix_note_warp(unsigned int* max_bits, float local_max_abs) {
  const unsigned int b = __reduce_max_sync(0xffffffffu, __float_as_uint(local_max_abs));
  if ((threadIdx.x & 31) == 0 && b) atomicMax(max_bits, b);
}

// Argument validation shared by the entry points (trace.cu).
sbr_status check_radar(const sbr_radar_cfg* r, const char* who);
sbr_status check_grid(const sbr_ray_grid* g, const char* who);

}  // namespace sbr

#define SBR_ARG(cond, ...)                          \
  do {                                              \
    if (!(cond)) {                                  \
      ::sbr::set_error(__VA_ARGS__);                \
      return SBR_ERR_INVALID_ARG;                   \
    }                                               \
  } while (0)

#define SBR_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::sbr::set_error("%s failed: %s", #call, cudaGetErrorString(e_));      \
      return SBR_ERR_CUDA;                                                    \
    }                                                                         \
  } while (0)

// ---- small vector math ------------------------------------------------------

struct d3 {
  double x, y, z;
};
__host__ __device__ inline d3 mk3(double x, double y, double z) { return d3{x, y, z}; }
__host__ __device__ inline d3 operator-(d3 a, d3 b) { return d3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ inline d3 operator+(d3 a, d3 b) { return d3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ inline d3 operator*(d3 a, double s) { return d3{a.x * s, a.y * s, a.z * s}; }
__host__ __device__ inline double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline d3 cross(d3 a, d3 b) {
  return d3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

__host__ __device__ inline float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ inline float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ inline float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ inline float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ inline float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline float3 cross(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline float l1(float3 a) { return fabsf(a.x) + fabsf(a.y) + fabsf(a.z); }
