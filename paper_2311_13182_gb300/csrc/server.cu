// Serving: continuous batching of simulation and reconstruction requests.
//
// The paper has no serving layer; this is the deployment form of the
// simulator.  Requests of uneven mesh and ray budgets arrive over time; the
// server admits them as slots (one CUDA stream each) and device memory free
// up, sizing every request by its exact footprint (the *_bytes queries of the
// library) inside the caller's device arena; their kernels overlap on the
// GPU.  BVHs of meshes that callers identify (mesh_id) stay resident after
// their request finishes, and so do the IF cubes of forward requests, so a
// repeated mesh skips the build and a repeated (mesh, grid) skips trace and
// synthesis; resident entries are evicted least-recently-used when a waiting
// request needs the memory.  The loop is driven by the caller (poll), with no
// thread of its own: each turn collects finished requests (CUDA events) and
// admits new ones.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "scene.cuh"

// ---- arena -------------------------------------------------------------------

struct sbr_arena {
  static constexpr size_t kGranule = 256;
  size_t size = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> length, disjoint, non-adjacent

  explicit sbr_arena(size_t n) : size(n / kGranule * kGranule) {
    if (size) free_[0] = size;
  }
  static size_t round(size_t n) { return ((n ? n : 1) + kGranule - 1) / kGranule * kGranule; }

  int64_t alloc(size_t n) {
    n = round(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, rem = it->second - n;
      free_.erase(it);
      if (rem) free_[off + n] = rem;
      used += n;
      peak = std::max(peak, used);
      return (int64_t)off;
    }
    return -1;
  }

  void release(size_t off, size_t n) {
    n = round(n);
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

  size_t largest() const {
    size_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
};

extern "C" sbr_arena* sbr_arena_create(size_t bytes) { return new (std::nothrow) sbr_arena(bytes); }
extern "C" int64_t sbr_arena_alloc(sbr_arena* a, size_t bytes) { return a ? a->alloc(bytes) : -1; }
extern "C" void sbr_arena_free(sbr_arena* a, int64_t offset, size_t bytes) {
  if (a && offset >= 0) a->release((size_t)offset, bytes);
}
extern "C" size_t sbr_arena_used(const sbr_arena* a) { return a ? a->used : 0; }
extern "C" size_t sbr_arena_peak(const sbr_arena* a) { return a ? a->peak : 0; }
extern "C" size_t sbr_arena_largest_free(const sbr_arena* a) { return a ? a->largest() : 0; }
extern "C" void sbr_arena_destroy(sbr_arena* a) { delete a; }

// ---- server ------------------------------------------------------------------

namespace sbr {
namespace {

double now_us(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
}

uint64_t grid_key(const sbr_ray_grid& g, int K) {
  // FNV-1a over the descriptor's bytes and the bounce count
  uint64_t h = 1469598103934665603ull;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&g);
  for (size_t i = 0; i < sizeof(g); ++i) h = (h ^ p[i]) * 1099511628211ull;
  return (h ^ (uint64_t)K) * 1099511628211ull;
}

struct SceneEntry {
  uint64_t mesh_id = 0;
  int64_t off = -1;
  size_t bytes = 0;
  sbr_scene* scene = nullptr;
  int refs = 0;
  uint64_t last = 0;
  cudaEvent_t built = nullptr;
};

struct CubeEntry {
  uint64_t mesh_id = 0, key = 0;
  int64_t off = -1;
  size_t bytes = 0;
  int refs = 0;
  uint64_t last = 0;
  cudaEvent_t ready = nullptr;
};

struct Sizes {  // device bytes of each part of a request
  size_t mesh, scene, paths, ws, cube, pc, points, recon;
};

struct Req {
  int64_t ticket = 0;
  sbr_request r{};
  std::vector<float> verts, target;
  std::vector<int32_t> faces, adj_off, adj;
  double t_submit = 0, t_admit = 0;
  Sizes sz{};
  int64_t off = -1;  // private block
  size_t bytes = 0;
  int slot = -1;
  SceneEntry* scene_ref = nullptr;
  CubeEntry* cube_ref = nullptr;
  bool scene_hit = false, cube_hit = false;
  bool created_scene = false, created_cube = false;  // resident entries this request fills
  sbr_scene* own_scene = nullptr;
  sbr_status status = SBR_OK;
};

struct Slot {
  cudaStream_t stream = nullptr;
  // the slot's tree builds run on a stream of the greatest priority, joined to `stream` by
  // events: a cooperative build needs all its CTAs resident at once, and beside another
  // slot's trace it would otherwise find them only when that trace drains
  cudaStream_t build_stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  Req* req = nullptr;
  char* pinned = nullptr;  // page-locked staging: the request's results, then its inputs
  size_t pinned_bytes = 0;
};

}  // namespace
}  // namespace sbr

struct sbr_server {
  char* base = nullptr;
  std::unique_ptr<sbr_arena> arena;
  sbr_radar_cfg radar{};
  sbr_cfar_cfg cfar{};
  std::vector<sbr::Slot> slots;
  std::deque<sbr::Req*> waiting;
  std::vector<sbr_completion> done;
  std::map<uint64_t, std::unique_ptr<sbr::SceneEntry>> scenes;
  std::map<std::pair<uint64_t, uint64_t>, std::unique_ptr<sbr::CubeEntry>> cubes;
  std::chrono::steady_clock::time_point t0;
  cudaEvent_t t0_event = nullptr;  // device-clock origin of the completions' gpu_t0_ms / gpu_t1_ms
  int64_t next_ticket = 1, submitted = 0, completed = 0, cache_hits = 0;
  uint64_t clock = 0;
};

namespace sbr {
namespace {

// Reconstruction requests refit the scene's tree to the moved vertices each
// iteration and rebuild it every kRebuildEvery iterations (the hits are the same).
constexpr int kRebuildEvery = 50;

Sizes request_sizes(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, const sbr_request* q) {
  Sizes s{};
  const int V = radar->n_tx * radar->n_rx;
  const int64_t R = (int64_t)q->grid.G * q->grid.G;
  s.mesh = sbr_arena::round(sizeof(float) * 3 * (size_t)q->nv) + sbr_arena::round(sizeof(int32_t) * 3 * (size_t)q->nt);
  s.scene = sbr_arena::round(sbr_scene_bytes(q->nt));
  s.paths = sbr_arena::round(sbr_paths_bytes((int32_t)R, q->max_bounces, V));
  s.ws = sbr_arena::round(sbr_synth_ws_bytes(radar, R * q->max_bounces));
  s.cube = sbr_arena::round(sizeof(float) * 2 * (size_t)V * radar->n_chirps * radar->n_samples);
  s.pc = sbr_arena::round(sbr_pc_bytes(radar, cfar));
  s.points = sbr_arena::round(sizeof(float) * 4 * (size_t)cfar->k_max) + kAlign;
  s.recon = 0;
  if (q->kind == SBR_REQ_RECON) {
    const size_t nv3 = sbr_arena::round(sizeof(float) * 3 * (size_t)q->nv);
    const size_t cap = (size_t)R * q->max_bounces;
    s.recon = 4 * nv3                                            // working verts, grad, m, v
              + sbr_arena::round(sizeof(float) * 4 * (size_t)q->n_target)  // target
              + 2 * sbr_arena::round(sizeof(float) * 4 * (size_t)cfar->k_max)  // gpoints
              + 2 * sbr_arena::round(sizeof(float) * V * cap)       // glen, gamp
              + s.cube                                              // gcube
              + sbr_arena::round(sizeof(int32_t) * ((size_t)q->nv + 1)) +
              sbr_arena::round(sizeof(int32_t) * 6 * (size_t)q->nt)  // adjacency (<= 6 per face)
              + sbr_arena::round(sbr_laplacian_ws_bytes(q->nv))
              + sbr_arena::round(sbr_trace_bwd_ws_bytes(q->nv)) + 2 * kAlign;  // step, loss
  }
  return s;
}

size_t total_bytes(const Sizes& s) { return s.mesh + s.scene + s.paths + s.ws + s.cube + s.pc + s.points + s.recon; }

sbr_status check_request(const sbr_radar_cfg* radar, const sbr_request* q) {
  SBR_ARG(q != nullptr, "sbr_server_submit: request is NULL");
  SBR_ARG(q->kind == SBR_REQ_FORWARD || q->kind == SBR_REQ_RECON, "sbr_server_submit: unknown kind %d", q->kind);
  SBR_ARG(q->nv >= 1 && q->nt >= 1 && q->verts && q->faces, "sbr_server_submit: empty or NULL mesh");
  SBR_ARG(q->max_bounces >= 1 && q->max_bounces <= 8, "sbr_server_submit: max_bounces=%d outside [1, 8]",
          q->max_bounces);
  SBR_ARG(q->out_points, "sbr_server_submit: out_points is NULL");
  sbr_status rs = check_grid(&q->grid, "sbr_server_submit");
  if (rs != SBR_OK) return rs;
  SBR_ARG((int64_t)q->grid.G * q->grid.G * q->max_bounces < (1ll << 31), "sbr_server_submit: ray budget too large");
  for (int64_t i = 0; i < 3 * (int64_t)q->nt; ++i)
    SBR_ARG(q->faces[i] >= 0 && q->faces[i] < q->nv, "sbr_server_submit: face %lld references vertex %d of %d",
            (long long)(i / 3), q->faces[i], q->nv);
  for (int64_t i = 0; i < 3 * (int64_t)q->nv; ++i)
    SBR_ARG(isfinite(q->verts[i]), "sbr_server_submit: vertex %lld is not finite", (long long)(i / 3));
  if (q->kind == SBR_REQ_RECON) {
    SBR_ARG(q->iterations >= 1 && q->n_target >= 1 && q->n_target <= 2048 && q->target,
            "sbr_server_submit: reconstruction needs iterations >= 1 and 1..2048 target points");
    SBR_ARG(q->lr > 0.f, "sbr_server_submit: lr must be positive");
  }
  (void)radar;
  return SBR_OK;
}

void touch(sbr_server* s, SceneEntry* e) { e->last = ++s->clock; }
void touch(sbr_server* s, CubeEntry* e) { e->last = ++s->clock; }

// Evicts the least-recently-used idle resident scene or cube; false when none.
bool evict_one(sbr_server* s) {
  SceneEntry* bs = nullptr;
  CubeEntry* bc = nullptr;
  for (auto& kv : s->scenes)
    if (kv.second->refs == 0 && (!bs || kv.second->last < bs->last)) bs = kv.second.get();
  for (auto& kv : s->cubes)
    if (kv.second->refs == 0 && (!bc || kv.second->last < bc->last)) bc = kv.second.get();
  if (!bs && !bc) return false;
  if (bs && (!bc || bs->last <= bc->last)) {
    cudaEventSynchronize(bs->built);
    sbr_scene_destroy(bs->scene);
    cudaEventDestroy(bs->built);
    s->arena->release((size_t)bs->off, bs->bytes);
    s->scenes.erase(bs->mesh_id);
  } else {
    cudaEventSynchronize(bc->ready);
    cudaEventDestroy(bc->ready);
    s->arena->release((size_t)bc->off, bc->bytes);
    s->cubes.erase({bc->mesh_id, bc->key});
  }
  return true;
}

int64_t alloc_evicting(sbr_server* s, size_t bytes) {
  for (;;) {
    const int64_t off = s->arena->alloc(bytes);
    if (off >= 0) return off;
    if (!evict_one(s)) return -1;
  }
}

bool ensure_pinned(Slot& sl, size_t bytes) {
  if (sl.pinned_bytes >= bytes) return true;
  if (sl.pinned) cudaFreeHost(sl.pinned);
  sl.pinned = nullptr;
  sl.pinned_bytes = 0;
  if (cudaMallocHost(&sl.pinned, bytes) != cudaSuccess) return false;
  sl.pinned_bytes = bytes;
  return true;
}

inline size_t round256(size_t n) { return (n + 255) / 256 * 256; }

// Results area of a slot's pinned buffer: points, status words, final vertices.
size_t pinned_out(const sbr_server* s, const Req* q) {
  return round256(sizeof(float) * 4 * (size_t)s->cfar.k_max + 64 +
                  (q->r.out_verts ? sizeof(float) * 3 * (size_t)q->r.nv : 0));
}

// Inputs area after it: the host arrays the request's device work reads.
size_t pinned_in(const Req* q) {
  size_t n = round256(q->verts.size() * sizeof(float)) + round256(q->faces.size() * sizeof(int32_t));
  if (q->r.kind == SBR_REQ_RECON)
    n += round256(q->target.size() * sizeof(float)) + round256(q->adj_off.size() * sizeof(int32_t)) +
         round256(q->adj.size() * sizeof(int32_t));
  return n;
}

size_t pinned_need(const sbr_server* s, const Req* q) { return pinned_out(s, q) + pinned_in(q); }

// Copies a request's host arrays into the inputs area of its slot's pinned buffer,
// so the host-to-device copies from there run asynchronously on the slot's stream
// (a copy from pageable memory is staged through a driver buffer by the calling
// thread, which would hold up the poll loop while other slots run).
struct Staging {
  char* at;
  template <class T>
  const T* put(const std::vector<T>& v) {
    T* p = reinterpret_cast<T*>(at);
    if (!v.empty()) memcpy(p, v.data(), v.size() * sizeof(T));
    at += round256(v.size() * sizeof(T));
    return p;
  }
};

#define ENQ(call)                        \
  do {                                   \
    sbr_status st_ = (call);             \
    if (st_ != SBR_OK) return st_;       \
  } while (0)

#define ENQ_CUDA(call)                                                       \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error("server: %s failed: %s", #call, cudaGetErrorString(e_));     \
      return SBR_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

// Runs build(stream) on the slot's build stream, ordered after the slot stream's work so far
// and before its next work.
template <class F>
sbr_status on_build_stream(Slot& sl, F build) {
  if (cudaEventRecord(sl.fork, sl.stream) != cudaSuccess ||
      cudaStreamWaitEvent(sl.build_stream, sl.fork, 0) != cudaSuccess) {
    set_error("server: fork to the build stream failed");
    return SBR_ERR_CUDA;
  }
  const sbr_status rs = build(reinterpret_cast<sbr_stream>(sl.build_stream));
  if (rs != SBR_OK) return rs;
  if (cudaEventRecord(sl.join, sl.build_stream) != cudaSuccess ||
      cudaStreamWaitEvent(sl.stream, sl.join, 0) != cudaSuccess) {
    set_error("server: join from the build stream failed");
    return SBR_ERR_CUDA;
  }
  return SBR_OK;
}

// Enqueues a forward request's work on its slot stream.
sbr_status enqueue_forward(sbr_server* s, Req* q, Slot& sl) {
  cudaStream_t st = sl.stream;
  const sbr_request& r = q->r;
  char* priv = s->base + q->off;
  Carver c(priv);
  sbr_scene* scene = nullptr;
  if (q->scene_hit) {
    scene = q->scene_ref->scene;
    ENQ_CUDA(cudaStreamWaitEvent(st, q->scene_ref->built, 0));
  } else {
    Carver m(q->scene_ref ? s->base + q->scene_ref->off : c.take<char>(q->sz.mesh + q->sz.scene));
    float* dv = m.take<float>(3 * (size_t)r.nv);
    int32_t* df = m.take<int32_t>(3 * (size_t)r.nt);
    void* dmem = m.take<char>(q->sz.scene);
    Staging in{sl.pinned + pinned_out(s, q)};
    const float* hv = in.put(q->verts);
    const int32_t* hf = in.put(q->faces);
    ENQ_CUDA(cudaMemcpyAsync(dv, hv, sizeof(float) * 3 * r.nv, cudaMemcpyHostToDevice, st));
    ENQ_CUDA(cudaMemcpyAsync(df, hf, sizeof(int32_t) * 3 * r.nt, cudaMemcpyHostToDevice, st));
    ENQ(on_build_stream(sl, [&](sbr_stream bs) {
      return sbr_scene_create(dv, r.nv, df, r.nt, dmem, q->sz.scene, bs, &scene);
    }));
    if (q->scene_ref) {
      q->scene_ref->scene = scene;
      ENQ_CUDA(cudaEventRecord(q->scene_ref->built, st));
    } else {
      q->own_scene = scene;
    }
  }
  float* cube;
  if (q->cube_hit) {
    cube = reinterpret_cast<float*>(s->base + q->cube_ref->off);
    ENQ_CUDA(cudaStreamWaitEvent(st, q->cube_ref->ready, 0));
  } else {
    const int V = s->radar.n_tx * s->radar.n_rx;
    const int64_t R = (int64_t)r.grid.G * r.grid.G;
    sbr_paths paths;
    ENQ(sbr_paths_bind(c.take<char>(q->sz.paths), q->sz.paths, (int32_t)R, r.max_bounces, V, &paths));
    void* ws = c.take<char>(q->sz.ws);
    cube = q->cube_ref ? reinterpret_cast<float*>(s->base + q->cube_ref->off) : c.take<float>(q->sz.cube / 4);
    ENQ(sbr_trace(scene, &s->radar, &r.grid, nullptr, -1, r.max_bounces, &paths, reinterpret_cast<sbr_stream>(st)));
    ENQ(sbr_synthesize(&paths, &s->radar, SBR_PHASE_SPLIT, cube, ws, q->sz.ws, reinterpret_cast<sbr_stream>(st)));
    if (q->cube_ref) ENQ_CUDA(cudaEventRecord(q->cube_ref->ready, st));
  }
  sbr_pc_state pc;
  ENQ(sbr_pc_bind(c.take<char>(q->sz.pc), q->sz.pc, &s->radar, &s->cfar, &pc));
  float* pts = c.take<float>(4 * (size_t)s->cfar.k_max);
  ENQ(sbr_pointcloud(cube, &s->radar, &s->cfar, pts, &pc, reinterpret_cast<sbr_stream>(st)));
  float* hp = reinterpret_cast<float*>(sl.pinned);
  int32_t* hm = reinterpret_cast<int32_t*>(sl.pinned + sizeof(float) * 4 * (size_t)s->cfar.k_max);
  ENQ_CUDA(cudaMemcpyAsync(hp, pts, sizeof(float) * 4 * s->cfar.k_max, cudaMemcpyDeviceToHost, st));
  ENQ_CUDA(cudaMemcpyAsync(hm, pc.n_points, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  ENQ_CUDA(cudaMemcpyAsync(hm + 1, scene->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  return SBR_OK;
}

// Enqueues a reconstruction: iterations of forward + Chamfer/Laplacian loss +
// adjoints + Adam on the request's own copy of the vertices.
sbr_status enqueue_recon(sbr_server* s, Req* q, Slot& sl) {
  cudaStream_t st = sl.stream;
  sbr_stream ss = reinterpret_cast<sbr_stream>(st);
  const sbr_request& r = q->r;
  const int V = s->radar.n_tx * s->radar.n_rx;
  const int64_t R = (int64_t)r.grid.G * r.grid.G;
  const size_t cap = (size_t)R * r.max_bounces;
  Carver c(s->base + q->off);
  float* dv = c.take<float>(3 * (size_t)r.nv);
  int32_t* df = c.take<int32_t>(3 * (size_t)r.nt);
  void* dscene = c.take<char>(q->sz.scene);
  sbr_paths paths;
  ENQ(sbr_paths_bind(c.take<char>(q->sz.paths), q->sz.paths, (int32_t)R, r.max_bounces, V, &paths));
  void* ws = c.take<char>(q->sz.ws);
  float* cube = c.take<float>(q->sz.cube / 4);
  sbr_pc_state pc;
  ENQ(sbr_pc_bind(c.take<char>(q->sz.pc), q->sz.pc, &s->radar, &s->cfar, &pc));
  float* pts = c.take<float>(4 * (size_t)s->cfar.k_max);
  float* grad = c.take<float>(3 * (size_t)r.nv);
  float* m1 = c.take<float>(3 * (size_t)r.nv);
  float* m2 = c.take<float>(3 * (size_t)r.nv);
  float* tgt = c.take<float>(4 * (size_t)r.n_target);
  float* gpts = c.take<float>(4 * (size_t)s->cfar.k_max);
  float* glen = c.take<float>((size_t)V * cap);
  float* gamp = c.take<float>((size_t)V * cap);
  float* gcube = c.take<float>(q->sz.cube / 4);
  int32_t* aoff = c.take<int32_t>((size_t)r.nv + 1);
  int32_t* adj = c.take<int32_t>(q->adj.size() ? q->adj.size() : 1);
  const size_t lws = sbr_laplacian_ws_bytes(r.nv);
  void* lap = c.take<char>(lws);
  const size_t bws = sbr_trace_bwd_ws_bytes(r.nv);
  void* bwd = c.take<char>(bws);
  int32_t* step = c.take<int32_t>(1);
  float* loss = c.take<float>(1);
  Staging in{sl.pinned + pinned_out(s, q)};
  const float* hv = in.put(q->verts);
  const int32_t* hf = in.put(q->faces);
  const float* ht = in.put(q->target);
  const int32_t* ho = in.put(q->adj_off);
  const int32_t* ha = in.put(q->adj);
  ENQ_CUDA(cudaMemcpyAsync(dv, hv, sizeof(float) * 3 * r.nv, cudaMemcpyHostToDevice, st));
  ENQ_CUDA(cudaMemcpyAsync(df, hf, sizeof(int32_t) * 3 * r.nt, cudaMemcpyHostToDevice, st));
  ENQ_CUDA(cudaMemcpyAsync(tgt, ht, sizeof(float) * 4 * r.n_target, cudaMemcpyHostToDevice, st));
  ENQ_CUDA(cudaMemcpyAsync(aoff, ho, sizeof(int32_t) * (r.nv + 1), cudaMemcpyHostToDevice, st));
  if (!q->adj.empty())
    ENQ_CUDA(cudaMemcpyAsync(adj, ha, sizeof(int32_t) * q->adj.size(), cudaMemcpyHostToDevice, st));
  ENQ_CUDA(cudaMemsetAsync(m1, 0, sizeof(float) * 3 * r.nv, st));
  ENQ_CUDA(cudaMemsetAsync(m2, 0, sizeof(float) * 3 * r.nv, st));
  ENQ_CUDA(cudaMemsetAsync(step, 0, sizeof(int32_t), st));
  sbr_scene* scene = nullptr;
  ENQ(on_build_stream(sl, [&](sbr_stream bs) {
    return sbr_scene_create(dv, r.nv, df, r.nt, dscene, q->sz.scene, bs, &scene);
  }));
  q->own_scene = scene;
  for (int it = 0; it < r.iterations; ++it) {
    // the moved vertices into the tree: refitted, rebuilt every kRebuildEvery iterations
    if (it > 0)
      ENQ(on_build_stream(sl, [&](sbr_stream bs) {
        return it % kRebuildEvery == 0 ? sbr_scene_update(scene, dv, bs) : sbr_scene_refit(scene, dv, bs);
      }));
    ENQ(sbr_trace(scene, &s->radar, &r.grid, nullptr, -1, r.max_bounces, &paths, ss));
    ENQ(sbr_synthesize(&paths, &s->radar, SBR_PHASE_SPLIT, cube, ws, q->sz.ws, ss));
    ENQ(sbr_pointcloud(cube, &s->radar, &s->cfar, pts, &pc, ss));
    ENQ(sbr_chamfer(pts, pc.n_points, s->cfar.k_max, tgt, r.n_target, loss, gpts, ss));
    ENQ_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * 3 * r.nv, st));
    ENQ(sbr_laplacian(dv, r.nv, aoff, adj, r.lap_weight, loss, grad, lap, lws, ss));
    ENQ(sbr_pointcloud_bwd(&s->radar, &s->cfar, &pc, gpts, gcube, ss));
    ENQ(sbr_synthesize_bwd(&paths, &s->radar, gcube, glen, gamp, nullptr, ws, q->sz.ws, ss));
    ENQ(sbr_trace_bwd(scene, dv, &s->radar, &r.grid, nullptr, &paths, glen, gamp, nullptr, grad, nullptr, 0, bwd,
                      bws, ss));
    ENQ(sbr_adam_step(dv, grad, m1, m2, 3 * (int64_t)r.nv, step, r.lr, 0.9f, 0.999f, 1e-8f, ss));
  }
  float* hp = reinterpret_cast<float*>(sl.pinned);
  char* hm = sl.pinned + sizeof(float) * 4 * (size_t)s->cfar.k_max;
  ENQ_CUDA(cudaMemcpyAsync(hp, pts, sizeof(float) * 4 * s->cfar.k_max, cudaMemcpyDeviceToHost, st));
  ENQ_CUDA(cudaMemcpyAsync(hm, pc.n_points, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  ENQ_CUDA(cudaMemcpyAsync(hm + 4, scene->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  ENQ_CUDA(cudaMemcpyAsync(hm + 8, loss, sizeof(float), cudaMemcpyDeviceToHost, st));
  if (r.out_verts)
    ENQ_CUDA(cudaMemcpyAsync(sl.pinned + sizeof(float) * 4 * (size_t)s->cfar.k_max + 64, dv,
                             sizeof(float) * 3 * r.nv, cudaMemcpyDeviceToHost, st));
  return SBR_OK;
}

// A failed request must not leave half-built resident entries behind.
void drop_created(sbr_server* s, Req* q) {
  if (q->created_scene && q->scene_ref && q->scene_ref->refs == 1) {
    SceneEntry* e = q->scene_ref;
    if (e->scene) sbr_scene_destroy(e->scene);
    cudaEventDestroy(e->built);
    s->arena->release((size_t)e->off, e->bytes);
    q->scene_ref = nullptr;
    s->scenes.erase(q->r.mesh_id);
  }
  if (q->created_cube && q->cube_ref && q->cube_ref->refs == 1) {
    CubeEntry* e = q->cube_ref;
    cudaEventDestroy(e->ready);
    s->arena->release((size_t)e->off, e->bytes);
    q->cube_ref = nullptr;
    s->cubes.erase({e->mesh_id, e->key});
  }
}

void release_request(sbr_server* s, Req* q) {
  if (q->own_scene) {
    sbr_scene_destroy(q->own_scene);
    q->own_scene = nullptr;
  }
  if (q->off >= 0) s->arena->release((size_t)q->off, q->bytes);
  q->off = -1;
  if (q->scene_ref) q->scene_ref->refs--;
  if (q->cube_ref) q->cube_ref->refs--;
}

void complete(sbr_server* s, Req* q, sbr_status status, Slot* sl) {
  sbr_completion cpl{};
  cpl.ticket = q->ticket;
  cpl.status = status;
  cpl.t_submit_us = q->t_submit;
  cpl.t_admit_us = q->t_admit;
  cpl.t_done_us = now_us(s->t0);
  cpl.scene_cached = q->scene_hit;
  cpl.cube_cached = q->cube_hit;
  cpl.footprint = q->bytes;
  if (sl && status == SBR_OK) {
    const char* hm = sl->pinned + sizeof(float) * 4 * (size_t)s->cfar.k_max;
    int32_t n = 0, err = 0;
    memcpy(&n, hm, 4);
    memcpy(&err, hm + 4, 4);
    if (q->r.kind == SBR_REQ_RECON) memcpy(&cpl.loss, hm + 8, 4);
    cpl.n_points = n;
    memcpy(q->r.out_points, sl->pinned, sizeof(float) * 4 * (size_t)s->cfar.k_max);
    if (q->r.kind == SBR_REQ_RECON && q->r.out_verts)
      memcpy(q->r.out_verts, sl->pinned + sizeof(float) * 4 * (size_t)s->cfar.k_max + 64,
             sizeof(float) * 3 * q->r.nv);
    if (err) cpl.status = SBR_ERR_INVALID_ARG;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sl->start, sl->done) == cudaSuccess) cpl.gpu_ms = ms;
    if (cudaEventElapsedTime(&ms, s->t0_event, sl->start) == cudaSuccess) cpl.gpu_t0_ms = ms;
    if (cudaEventElapsedTime(&ms, s->t0_event, sl->done) == cudaSuccess) cpl.gpu_t1_ms = ms;
  }
  s->done.push_back(cpl);
  s->completed++;
}

// Tries to admit q into slot sl; false (nothing changed) when memory is short.
bool admit(sbr_server* s, Req* q, Slot& sl) {
  const sbr_request& r = q->r;
  SceneEntry* se = nullptr;
  CubeEntry* ce = nullptr;
  bool scene_hit = false, cube_hit = false;
  if (r.kind == SBR_REQ_FORWARD && r.mesh_id) {
    auto it = s->scenes.find(r.mesh_id);
    if (it != s->scenes.end()) {
      se = it->second.get();
      scene_hit = true;
    }
    auto ic = s->cubes.find({r.mesh_id, grid_key(r.grid, r.max_bounces)});
    if (ic != s->cubes.end()) {
      ce = ic->second.get();
      cube_hit = true;
    }
  }
  // pin reused entries so eviction below cannot take them
  if (se) se->refs++;
  if (ce) ce->refs++;
  const Sizes& z = q->sz;
  size_t priv = z.pc + z.points + z.recon;
  if (!cube_hit) priv += z.paths + z.ws + ((r.kind == SBR_REQ_FORWARD && r.mesh_id) ? 0 : z.cube);
  if (!scene_hit && !(r.kind == SBR_REQ_FORWARD && r.mesh_id)) priv += z.mesh + z.scene;
  int64_t off_scene = -1, off_cube = -1;
  const int64_t off = alloc_evicting(s, priv);
  bool ok = off >= 0;
  if (ok && !scene_hit && r.kind == SBR_REQ_FORWARD && r.mesh_id) {
    off_scene = alloc_evicting(s, z.mesh + z.scene);
    ok = off_scene >= 0;
  }
  if (ok && !cube_hit && r.kind == SBR_REQ_FORWARD && r.mesh_id) {
    off_cube = alloc_evicting(s, z.cube);
    ok = off_cube >= 0;
  }
  if (!ok) {
    if (off >= 0) s->arena->release((size_t)off, priv);
    if (off_scene >= 0) s->arena->release((size_t)off_scene, z.mesh + z.scene);
    if (se) se->refs--;
    if (ce) ce->refs--;
    return false;
  }
  if (off_scene >= 0) {
    auto e = std::make_unique<SceneEntry>();
    e->mesh_id = r.mesh_id;
    e->off = off_scene;
    e->bytes = z.mesh + z.scene;
    cudaEventCreateWithFlags(&e->built, cudaEventDisableTiming);
    se = e.get();
    se->refs = 1;
    s->scenes[r.mesh_id] = std::move(e);
  }
  if (off_cube >= 0) {
    auto e = std::make_unique<CubeEntry>();
    e->mesh_id = r.mesh_id;
    e->key = grid_key(r.grid, r.max_bounces);
    e->off = off_cube;
    e->bytes = z.cube;
    cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming);
    ce = e.get();
    ce->refs = 1;
    s->cubes[{e->mesh_id, e->key}] = std::move(e);
  }
  if (se) touch(s, se);
  if (ce) touch(s, ce);
  if (scene_hit || cube_hit) s->cache_hits++;
  q->off = off;
  q->bytes = priv;
  q->scene_ref = se;
  q->cube_ref = ce;
  q->scene_hit = scene_hit;
  q->cube_hit = cube_hit;
  q->created_scene = off_scene >= 0;
  q->created_cube = off_cube >= 0;
  q->t_admit = now_us(s->t0);
  sl.req = q;
  if (!ensure_pinned(sl, pinned_need(s, q))) {
    q->status = SBR_ERR_OOM;
    return true;
  }
  cudaEventRecord(sl.start, sl.stream);
  q->status = r.kind == SBR_REQ_FORWARD ? enqueue_forward(s, q, sl) : enqueue_recon(s, q, sl);
  cudaEventRecord(sl.done, sl.stream);
  return true;
}

}  // namespace
}  // namespace sbr

using namespace sbr;

extern "C" size_t sbr_server_request_bytes(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar,
                                           const sbr_request* req) {
  if (!radar || !cfar || !req || check_radar(radar, "sbr_server_request_bytes") != SBR_OK) return 0;
  if (sbr_pc_bytes(radar, cfar) == 0) return 0;
  return total_bytes(request_sizes(radar, cfar, req));
}

extern "C" sbr_status sbr_server_create(void* d_arena, size_t arena_bytes, int32_t n_slots,
                                        const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, sbr_server** out) {
  SBR_ARG(out, "sbr_server_create: out is NULL");
  *out = nullptr;
  SBR_ARG(d_arena && aligned256(d_arena) && arena_bytes >= 4096, "sbr_server_create: arena NULL, misaligned or tiny");
  SBR_ARG(n_slots >= 1 && n_slots <= 64, "sbr_server_create: n_slots=%d outside [1, 64]", n_slots);
  sbr_status rs = check_radar(radar, "sbr_server_create");
  if (rs != SBR_OK) return rs;
  SBR_ARG(cfar && sbr_pc_bytes(radar, cfar) > 0, "sbr_server_create: invalid point-cloud configuration");
  auto s = std::make_unique<sbr_server>();
  s->base = static_cast<char*>(d_arena);
  s->arena.reset(new sbr_arena(arena_bytes));
  s->radar = *radar;
  s->cfar = *cfar;
  s->t0 = std::chrono::steady_clock::now();
  s->slots.resize(n_slots);
  for (auto& sl : s->slots) {
    SBR_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
    int least = 0, greatest = 0;
    SBR_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    SBR_CUDA(cudaStreamCreateWithPriority(&sl.build_stream, cudaStreamNonBlocking, greatest));
    SBR_CUDA(cudaEventCreateWithFlags(&sl.fork, cudaEventDisableTiming));
    SBR_CUDA(cudaEventCreateWithFlags(&sl.join, cudaEventDisableTiming));
    SBR_CUDA(cudaEventCreate(&sl.start));
    SBR_CUDA(cudaEventCreate(&sl.done));
  }
  SBR_CUDA(cudaEventCreate(&s->t0_event));
  SBR_CUDA(cudaEventRecord(s->t0_event, s->slots[0].stream));
  *out = s.release();
  return SBR_OK;
}

extern "C" sbr_status sbr_server_submit(sbr_server* s, const sbr_request* req, int64_t* ticket) {
  SBR_ARG(s && ticket, "sbr_server_submit: NULL server or ticket");
  sbr_status rs = check_request(&s->radar, req);
  if (rs != SBR_OK) return rs;
  const Sizes z = request_sizes(&s->radar, &s->cfar, req);
  if (total_bytes(z) > s->arena->size) {
    set_error("sbr_server_submit: request needs %zu bytes, arena holds %zu", total_bytes(z), s->arena->size);
    return SBR_ERR_OOM;
  }
  auto q = new Req();
  q->ticket = s->next_ticket++;
  q->r = *req;
  q->sz = z;
  q->verts.assign(req->verts, req->verts + 3 * (size_t)req->nv);
  q->faces.assign(req->faces, req->faces + 3 * (size_t)req->nt);
  if (req->kind == SBR_REQ_RECON) {
    q->target.assign(req->target, req->target + 4 * (size_t)req->n_target);
    q->adj_off.resize((size_t)req->nv + 1);
    int32_t n = 0;
    rs = sbr_mesh_adjacency(q->faces.data(), req->nt, req->nv, q->adj_off.data(), nullptr, 0, &n);
    if (rs == SBR_OK) {
      q->adj.resize(n > 0 ? n : 1);
      rs = sbr_mesh_adjacency(q->faces.data(), req->nt, req->nv, q->adj_off.data(), q->adj.data(),
                              (int32_t)q->adj.size(), &n);
    }
    if (rs != SBR_OK) {
      delete q;
      return rs;
    }
  }
  q->r.verts = q->verts.data();
  q->r.faces = q->faces.data();
  q->r.target = q->target.empty() ? nullptr : q->target.data();
  q->t_submit = now_us(s->t0);
  s->waiting.push_back(q);
  s->submitted++;
  *ticket = q->ticket;
  return SBR_OK;
}

extern "C" sbr_status sbr_server_cancel(sbr_server* s, int64_t ticket) {
  SBR_ARG(s, "sbr_server_cancel: NULL server");
  for (auto it = s->waiting.begin(); it != s->waiting.end(); ++it) {
    if ((*it)->ticket != ticket) continue;
    Req* q = *it;
    s->waiting.erase(it);
    complete(s, q, SBR_ERR_CANCELLED, nullptr);
    delete q;
    return SBR_OK;
  }
  set_error("sbr_server_cancel: ticket %lld is not waiting", (long long)ticket);
  return SBR_ERR_INVALID_ARG;
}

extern "C" sbr_status sbr_server_poll(sbr_server* s, sbr_completion* out, int32_t cap, int32_t* n_out) {
  SBR_ARG(s && n_out && (cap == 0 || out), "sbr_server_poll: bad argument");
  // 1. finished requests release their slots and memory
  for (auto& sl : s->slots) {
    if (!sl.req) continue;
    const cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady) continue;
    Req* q = sl.req;
    sbr_status st = q->status;
    if (e != cudaSuccess && st == SBR_OK) {
      set_error("server: request %lld failed on the device: %s", (long long)q->ticket, cudaGetErrorString(e));
      st = SBR_ERR_CUDA;
    }
    if (st != SBR_OK) cudaStreamSynchronize(sl.stream);  // partially enqueued work may still read the block
    complete(s, q, st, &sl);
    if (s->done.back().status != SBR_OK) drop_created(s, q);
    release_request(s, q);
    sl.req = nullptr;
    delete q;
  }
  // 2. admission: FIFO, a request may pass at most 8 that do not fit
  int skipped = 0;
  for (auto it = s->waiting.begin(); it != s->waiting.end() && skipped <= 8;) {
    Slot* free_slot = nullptr;
    for (auto& sl : s->slots)
      if (!sl.req) {
        free_slot = &sl;
        break;
      }
    if (!free_slot) break;
    if (admit(s, *it, *free_slot)) {
      it = s->waiting.erase(it);
    } else {
      ++skipped;
      ++it;
    }
  }
  // 3. hand out completions
  const int32_t n = (int32_t)std::min<size_t>(s->done.size(), (size_t)cap);
  for (int32_t i = 0; i < n; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + n);
  *n_out = n;
  return SBR_OK;
}

extern "C" sbr_status sbr_server_get_stats(const sbr_server* s, sbr_server_stats* o) {
  SBR_ARG(s && o, "sbr_server_get_stats: NULL argument");
  *o = sbr_server_stats{};
  o->arena_bytes = s->arena->size;
  o->used_bytes = s->arena->used;
  o->peak_bytes = s->arena->peak;
  for (auto& kv : s->scenes) o->cached_bytes += kv.second->bytes;
  for (auto& kv : s->cubes) o->cached_bytes += kv.second->bytes;
  o->waiting = (int32_t)s->waiting.size();
  for (auto& sl : s->slots) o->running += sl.req ? 1 : 0;
  o->cached_scenes = (int32_t)s->scenes.size();
  o->cached_cubes = (int32_t)s->cubes.size();
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->cache_hits = s->cache_hits;
  return SBR_OK;
}

extern "C" void sbr_server_destroy(sbr_server* s) {
  if (!s) return;
  for (auto& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.req) {
      release_request(s, sl.req);
      delete sl.req;
    }
    if (sl.pinned) cudaFreeHost(sl.pinned);
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.build_stream) cudaStreamDestroy(sl.build_stream);
    if (sl.fork) cudaEventDestroy(sl.fork);
    if (sl.join) cudaEventDestroy(sl.join);
  }
  for (auto& kv : s->scenes) {
    sbr_scene_destroy(kv.second->scene);
    cudaEventDestroy(kv.second->built);
  }
  for (auto& kv : s->cubes) cudaEventDestroy(kv.second->ready);
  for (auto* q : s->waiting) delete q;
  if (s->t0_event) cudaEventDestroy(s->t0_event);
  delete s;
}
