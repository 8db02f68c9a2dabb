// Reconstruction loss and optimiser (Section 3.4: Eq. 14 objective, Eq. 15
// gradient update).
//
// The paper minimises a loss between simulated and observed radar data with
// SGD.  The reconstruction loop here compares radar point clouds with a
// weighted squared Chamfer distance plus a uniform-Laplacian smoothness term on
// the mesh, and updates the vertices with Adam (Kingma & Ba 2015).  All three
// have hand-written gradients; the Chamfer kernel is deterministic (no atomics).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sbr {
namespace {

constexpr int kChamferMax = 2048;  // points per side (static shared memory: 32 KB)

__device__ inline float block_sum(float v, float* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// One CTA: nearest neighbours both ways, the two weighted means, gradients.
//   L = sum_i w_i |p_i - q_nn(i)|^2 / sum_i w_i + sum_j u_j |q_j - p_nn(j)|^2 / sum_j u_j
__global__ void __launch_bounds__(1024) k_chamfer(const float4* __restrict__ P, const int32_t* __restrict__ d_n,
                                                  int cap, const float4* __restrict__ Q, int m,
                                                  float* __restrict__ loss, float4* __restrict__ gP) {
  __shared__ int nn_p[kChamferMax], nn_q[kChamferMax];
  __shared__ float d2_p[kChamferMax], d2_q[kChamferMax];
  __shared__ float red[32];
  const int n = min(max(*d_n, 0), cap);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float4 p = P[i];
    float best = INFINITY;
    int bj = 0;
    for (int j = 0; j < m; ++j) {
      const float4 q = Q[j];
      const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
      const float d = dx * dx + dy * dy + dz * dz;
      if (d < best) { best = d; bj = j; }
    }
    nn_p[i] = bj;
    d2_p[i] = best;
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const float4 q = Q[j];
    float best = INFINITY;
    int bi = 0;
    for (int i = 0; i < n; ++i) {
      const float4 p = P[i];
      const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
      const float d = dx * dx + dy * dy + dz * dz;
      if (d < best) { best = d; bi = i; }
    }
    nn_q[j] = bi;
    d2_q[j] = best;
  }
  __syncthreads();
  float sw = 0.f, swd = 0.f, su = 0.f, sud = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sw += P[i].w;
    swd += P[i].w * d2_p[i];
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    su += Q[j].w;
    sud += Q[j].w * d2_q[j];
  }
  sw = block_sum(sw, red);
  swd = block_sum(swd, red);
  su = block_sum(su, red);
  sud = block_sum(sud, red);
  const bool ok = n > 0 && m > 0 && sw > 0.f && su > 0.f;
  const float l1 = ok ? swd / sw : 0.f, l2 = ok ? sud / su : 0.f;
  if (threadIdx.x == 0) *loss = l1 + l2;
  for (int i = threadIdx.x; i < cap; i += blockDim.x) {
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ok && i < n) {
      const float4 p = P[i], q = Q[nn_p[i]];
      const float s = 2.f * p.w / sw;
      g.x = s * (p.x - q.x);
      g.y = s * (p.y - q.y);
      g.z = s * (p.z - q.z);
      g.w = (d2_p[i] - l1) / sw;
      for (int j = 0; j < m; ++j) {
        if (nn_q[j] != i) continue;
        const float4 qj = Q[j];
        const float t = 2.f * qj.w / su;
        g.x += t * (p.x - qj.x);
        g.y += t * (p.y - qj.y);
        g.z += t * (p.z - qj.z);
      }
    }
    gP[i] = g;
  }
}

constexpr int kLapThreads = 256;
constexpr int kLapFirst = 8;  // neighbour indices loaded together before their values

// delta_i = v_i - mean_{j in N(i)} v_j; partial[blockIdx] = the CTA's sum of
// |delta_i|^2 (fixed order).  The first kLapFirst neighbour indices are loaded
// before any of their positions, so that the position loads overlap; the sums
// run in neighbour order either way.
__global__ void __launch_bounds__(kLapThreads) k_lap_delta(const float* __restrict__ v, int nv,
                                                           const int32_t* __restrict__ off,
                                                           const int32_t* __restrict__ adj, float* __restrict__ delta,
                                                           float* __restrict__ partial) {
  __shared__ float red[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.f;
  if (i < nv) {
    const int b = __ldg(&off[i]), e = __ldg(&off[i + 1]);
    int nb[kLapFirst];
#pragma unroll
    for (int u = 0; u < kLapFirst; ++u) nb[u] = b + u < e ? __ldg(&adj[b + u]) : -1;
    float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
    for (int u = 0; u < kLapFirst; ++u)
      if (nb[u] >= 0) {
        mx += __ldg(&v[3 * nb[u]]);
        my += __ldg(&v[3 * nb[u] + 1]);
        mz += __ldg(&v[3 * nb[u] + 2]);
      }
    for (int q = b + kLapFirst; q < e; ++q) {
      const int j = __ldg(&adj[q]);
      mx += __ldg(&v[3 * j]);
      my += __ldg(&v[3 * j + 1]);
      mz += __ldg(&v[3 * j + 2]);
    }
    const float inv = e > b ? 1.f / (float)(e - b) : 0.f;
    const float dx = e > b ? v[3 * i] - mx * inv : 0.f, dy = e > b ? v[3 * i + 1] - my * inv : 0.f,
                dz = e > b ? v[3 * i + 2] - mz * inv : 0.f;
    delta[3 * i] = dx;
    delta[3 * i + 1] = dy;
    delta[3 * i + 2] = dz;
    sq = dx * dx + dy * dy + dz * dz;
  }
  sq = block_sum(sq, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = sq;
}

// dL/dv_k = weight (2 / nv) (delta_k - sum_{i in N(k)} delta_i / deg_i); the first
// CTA also adds lscale * (the sum of the nb CTA partials, fixed order) to *loss.
__global__ void __launch_bounds__(kLapThreads) k_lap_grad(const float* __restrict__ delta, int nv,
                                                          const int32_t* __restrict__ off,
                                                          const int32_t* __restrict__ adj, float scale,
                                                          float* __restrict__ g, const float* __restrict__ partial,
                                                          int nb, float lscale, float* __restrict__ loss) {
  __shared__ float red[32];
  if (blockIdx.x == 0) {
    float s = 0.f;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *loss += lscale * s;
  }
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nv) return;
  float gx = delta[3 * k], gy = delta[3 * k + 1], gz = delta[3 * k + 2];
  const int b = __ldg(&off[k]), e = __ldg(&off[k + 1]);
  int nbr[kLapFirst];
#pragma unroll
  for (int u = 0; u < kLapFirst; ++u) nbr[u] = b + u < e ? __ldg(&adj[b + u]) : -1;
#pragma unroll
  for (int u = 0; u < kLapFirst; ++u)
    if (nbr[u] >= 0) {
      const int i = nbr[u];
      const float inv = 1.f / (float)(__ldg(&off[i + 1]) - __ldg(&off[i]));
      gx -= delta[3 * i] * inv;
      gy -= delta[3 * i + 1] * inv;
      gz -= delta[3 * i + 2] * inv;
    }
  for (int q = b + kLapFirst; q < e; ++q) {
    const int i = __ldg(&adj[q]);
    const float inv = 1.f / (float)(__ldg(&off[i + 1]) - __ldg(&off[i]));
    gx -= delta[3 * i] * inv;
    gy -= delta[3 * i + 1] * inv;
    gz -= delta[3 * i + 2] * inv;
  }
  g[3 * k] += scale * gx;
  g[3 * k + 1] += scale * gy;
  g[3 * k + 2] += scale * gz;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, const int32_t* __restrict__ step, float lr, float b1,
                       float b2, float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float t = (float)(*step + 1);
  const float c1 = 1.f / (1.f - powf(b1, t)), c2 = 1.f / (1.f - powf(b2, t));
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void k_step_inc(int32_t* step) { *step += 1; }

}  // namespace
}  // namespace sbr

using namespace sbr;

extern "C" sbr_status sbr_chamfer(const float* d_pred, const int32_t* d_n_pred, int32_t pred_cap,
                                  const float* d_target, int32_t n_target, float* d_loss, float* d_gpred,
                                  sbr_stream stream) {
  SBR_ARG(d_pred && d_n_pred && d_loss && d_gpred, "sbr_chamfer: NULL argument");
  SBR_ARG(pred_cap >= 1 && pred_cap <= kChamferMax, "sbr_chamfer: pred_cap=%d outside [1, %d]", pred_cap,
          kChamferMax);
  SBR_ARG(n_target >= 0 && n_target <= kChamferMax && (n_target == 0 || d_target),
          "sbr_chamfer: n_target=%d outside [0, %d]", n_target, kChamferMax);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ::sbr::note_launch();
  k_chamfer<<<1, 1024, 0, st>>>(reinterpret_cast<const float4*>(d_pred), d_n_pred, pred_cap,
                                reinterpret_cast<const float4*>(d_target), n_target, d_loss,
                                reinterpret_cast<float4*>(d_gpred));
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}

extern "C" sbr_status sbr_mesh_adjacency(const int32_t* h_faces, int32_t nt, int32_t nv, int32_t* h_off,
                                         int32_t* h_adj, int32_t adj_cap, int32_t* n_adj) {
  SBR_ARG(h_faces && h_off && n_adj && nt >= 0 && nv >= 1, "sbr_mesh_adjacency: bad argument");
  std::vector<std::pair<int32_t, int32_t>> e;
  e.reserve((size_t)nt * 6);
  for (int32_t f = 0; f < nt; ++f) {
    for (int c = 0; c < 3; ++c) {
      const int32_t a = h_faces[3 * f + c], b = h_faces[3 * f + (c + 1) % 3];
      SBR_ARG(a >= 0 && a < nv && b >= 0 && b < nv, "sbr_mesh_adjacency: face %d index outside [0, nv)", f);
      if (a == b) continue;
      e.emplace_back(a, b);
      e.emplace_back(b, a);
    }
  }
  std::sort(e.begin(), e.end());
  e.erase(std::unique(e.begin(), e.end()), e.end());
  *n_adj = (int32_t)e.size();
  if (!h_adj) return SBR_OK;  // size query
  if ((int64_t)e.size() > adj_cap) {
    set_error("sbr_mesh_adjacency: %zu entries, capacity %d", e.size(), adj_cap);
    return SBR_ERR_OOM;
  }
  memset(h_off, 0, sizeof(int32_t) * (nv + 1));
  for (auto& x : e) h_off[x.first + 1]++;
  for (int32_t i = 0; i < nv; ++i) h_off[i + 1] += h_off[i];
  for (size_t q = 0; q < e.size(); ++q) h_adj[q] = e[q].second;
  return SBR_OK;
}

extern "C" size_t sbr_laplacian_ws_bytes(int32_t nv) {
  Carver c(nullptr);
  c.take<float>(3 * (size_t)(nv > 0 ? nv : 1));
  c.take<float>(nv > 0 ? nv : 1);
  return c.bytes();
}

extern "C" sbr_status sbr_laplacian(const float* d_verts, int32_t nv, const int32_t* d_off, const int32_t* d_adj,
                                    float weight, float* d_loss, float* d_gverts, void* d_ws, size_t ws_bytes,
                                    sbr_stream stream) {
  SBR_ARG(d_verts && d_off && d_adj && d_loss && d_gverts && d_ws, "sbr_laplacian: NULL argument");
  SBR_ARG(nv >= 1, "sbr_laplacian: nv=%d", nv);
  SBR_ARG(aligned256(d_ws), "sbr_laplacian: workspace not 256-byte aligned");
  if (ws_bytes < sbr_laplacian_ws_bytes(nv)) {
    set_error("sbr_laplacian: workspace of %zu bytes, %zu needed", ws_bytes, sbr_laplacian_ws_bytes(nv));
    return SBR_ERR_OOM;
  }
  Carver c(d_ws);
  float* delta = c.take<float>(3 * (size_t)nv);
  float* partial = c.take<float>(nv);  // one per CTA (nb <= nv)
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int b = (nv + kLapThreads - 1) / kLapThreads;
  ::sbr::note_launch();
  k_lap_delta<<<b, kLapThreads, 0, st>>>(d_verts, nv, d_off, d_adj, delta, partial);
  ::sbr::note_launch();
  k_lap_grad<<<b, kLapThreads, 0, st>>>(delta, nv, d_off, d_adj, 2.f * weight / (float)nv, d_gverts, partial, b,
                                        weight / (float)nv, d_loss);
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}

extern "C" sbr_status sbr_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t n,
                                    int32_t* d_step, float lr, float beta1, float beta2, float eps,
                                    sbr_stream stream) {
  SBR_ARG(d_params && d_grad && d_m && d_v && d_step && n >= 0, "sbr_adam_step: bad argument");
  SBR_ARG(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f, "sbr_adam_step: bad betas");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n > 0) {
    ::sbr::note_launch();
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_params, d_grad, d_m, d_v, n, d_step, lr, beta1, beta2,
                                                         eps);
  }
  ::sbr::note_launch();
  k_step_inc<<<1, 1, 0, st>>>(d_step);
  SBR_CUDA(cudaGetLastError());
  return SBR_OK;
}
