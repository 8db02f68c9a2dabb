/*
 * sbr.h -- C ABI of libsbr, a GB300 (sm_103a) shooting-and-bouncing-rays (SBR)
 * FMCW radar simulator with hand-written adjoints.
 *
 * The library follows the paper's statement of the problem (Section 3.4,
 * Eq. 14: a simulator S : Theta -> Y) split into its three stages:
 *
 *   sbr_trace       mesh, radar, ray grid -> paths      (Section 3.2.1, Eq. 2-3:
 *                   Monte-Carlo ray tracing; the path records are the time of
 *                   flight I^t and signal strength I^s named there)
 *   sbr_synthesize  paths -> IF cube [V, C, N_s]        (Section 3.2.2, Eq. 8)
 *   sbr_pointcloud  IF cube -> radar point cloud        (Section 3.4, Eq. 16: the
 *                   signal-processing map T; range FFT, Doppler FFT, angle DFT,
 *                   soft CA-CFAR, sub-bin refine)
 *
 * plus the adjoint of each stage (Section 3.3, Eq. 13 chain rule; Eq. 11-12
 * for synthesis) and the loss / optimiser kernels of the reconstruction loop
 * (Section 3.4, Eq. 14-15).
 *
 * Conventions (every entry point):
 *  - Returns sbr_status; SBR_OK = 0.  Nothing aborts, throws across the ABI or
 *    traps on the device.  sbr_last_error() gives a message for the calling
 *    thread's last failure.
 *  - Work is enqueued asynchronously on the given stream (NULL = legacy default
 *    stream); argument checks that need no device data happen before anything
 *    is enqueued and fail without side effects.
 *  - Every device pointer is owned by the caller, must stay valid until the
 *    enqueued work completes, and must be 256-byte aligned when it is the base
 *    of a region carved by a *_bind function.  The library performs no device
 *    allocation of its own; *_bytes functions give the sizes to allocate.
 *  - Frame: metres, seconds, Hz.  Radar frame origin at the ray origin,
 *    boresight +z, array along +x.
 *  - Sizes are device-side where they depend on data (e.g. the number of valid
 *    paths P, the number of detected points): kernels read them from device
 *    memory, so no call synchronises the host.
 */
#ifndef SBR_H_
#define SBR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sbr_stream; /* identical to cudaStream_t */

typedef enum {
  SBR_OK = 0,
  SBR_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or configuration */
  SBR_ERR_OOM = 2,         /* caller-provided region smaller than *_bytes() */
  SBR_ERR_TIMEOUT = 3,     /* a bounded device wait gave up (status word) */
  SBR_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the name) */
  SBR_ERR_UNSUPPORTED = 5, /* configuration outside the compiled kernels' range */
  SBR_ERR_CANCELLED = 6    /* serving: the request was cancelled before admission */
} sbr_status;

#define SBR_MAX_TX 16
#define SBR_MAX_RX 16
#define SBR_MAX_VIRT 64
#define SBR_MAX_MATERIALS 16
#define SBR_MAX_OBJECTS 16

/* FMCW radar (Section 3.2.2, Eq. 8: carrier f_c, sweep B over chirp time T,
 * mu = B / T).  Samples t_n = n T / N_s, n = 0..N_s-1.  Virtual antenna
 * v = t * n_rx + r pairs Tx t with Rx r. */
typedef struct {
  double f0;          /* carrier f_c [Hz] */
  double bandwidth;   /* sweep B [Hz] */
  double chirp_time;  /* chirp duration T [s] */
  double chirp_rep;   /* chirp repetition interval [s] (static scene: unused) */
  int32_t n_samples;  /* N_s, power of two in [32, 4096] */
  int32_t n_chirps;   /* C, power of two in [1, 512] */
  int32_t n_tx, n_rx; /* n_tx * n_rx <= SBR_MAX_VIRT */
  double tx[SBR_MAX_TX][3];
  double rx[SBR_MAX_RX][3];
} sbr_radar_cfg;

/* Stratified G x G ray grid: the Monte-Carlo sample set of Eq. 3.  Ray
 * index = row * G + col; direction = normalize(axis + a u_axis + b v_axis),
 * a = tan_half (2 (col + jx) / G - 1), b = tan_half (2 (row + jy) / G - 1) with
 * (jx, jy) = (1/2, 1/2) (cell centres) or, with `jitter`, the ray's own offsets
 * in its cell (stratified jittered sampling); weight = (2 tan_half / G)^2 cos^3
 * of the direction's angle to axis (the cell's solid angle at the sample). */
typedef struct {
  int32_t G;
  int32_t _pad;
  double origin[3];
  double axis[3];   /* unit */
  double u_axis[3]; /* unit, orthogonal to axis */
  double v_axis[3]; /* unit, orthogonal to axis and u_axis */
  double tan_half;
  const float* jitter; /* device [G*G][2] offsets (jx, jy) in [0, 1) per ray, or NULL (cell centres);
                          borrowed: must stay valid while traces and adjoints of the grid run */
} sbr_ray_grid;

/* Soft CA-CFAR and point extraction (the map T of Eq. 16; parameters are
 * this library's reading: the paper names T only as "a signal processing
 * algorithm").  Angle rows rho = e * n_theta + a, R = n_elev * n_theta of them:
 * azimuth cosine u_a = -1 + 2a / n_theta, elevation cosine
 * w_e = (2e + 1 - n_elev) / n_elev (w = 0 with one elevation bin); the steering
 * phase of virtual element v is 2 pi (x_v u + y_v w) / lambda_c with x_v, y_v
 * the sums of its Tx and Rx x and y coordinates. */
typedef struct {
  int32_t n_theta; /* azimuth bins, power of two in [8, 256] */
  int32_t guard;   /* CFAR guard cells each side along range */
  int32_t train;   /* CFAR training cells each side beyond the guard */
  int32_t k_max;   /* maximum points returned */
  float alpha;     /* CFAR scale (linear power) */
  float floor_rel; /* absolute floor as a fraction of the map's maximum power */
  float beta;      /* sigmoid temperature in natural-log power units */
  float w_min;     /* minimum soft weight for a point to be kept */
  int32_t n_elev;  /* elevation bins (0 reads as 1), power of two; R = n_elev * n_theta <= 256
                      and R * V <= 4096 */
  int32_t _pad;
} sbr_cfar_cfg;

typedef enum {
  SBR_PHASE_SPLIT = 0, /* tau in float-float, phase anchors in hi/lo FP32, FP32 rotation */
  SBR_PHASE_FP64 = 1,  /* per-sample carrier phase f_c tau + mu tau t_n in FP64 */
  SBR_PHASE_NAIVE = 2  /* tau, f_c tau and mu tau t_n all in FP32 */
} sbr_phase_mode;

/* OR'ed into sbr_synthesize's mode: synthesise every chirp from the paths'
 * dL/dt (a trace of a scene with motion) instead of one chirp broadcast to all;
 * SBR_PHASE_SPLIT (N_s <= 512) and SBR_PHASE_FP64 only. */
#define SBR_SYNTH_MOVING 0x100

/* One surface interaction of a ray (16 B).  tri = original triangle index or
 * -1 (no hit; every later bounce of that ray is -1 too). */
typedef struct {
  int32_t tri;
  float t, u, v;
} sbr_hit;

const char* sbr_version(void);
/* Copies the calling thread's last error message (NUL-terminated, truncated to n). */
void sbr_last_error(char* buf, size_t n);
/* Number of CUDA kernel launches the library has issued in this process. */
uint64_t sbr_launch_count(void);

/* ------------------------------------------------------------------------ */
/* Scene: triangle mesh + LBVH (Section 3.1: the mesh is the scene          */
/* representation whose vertices are the optimised parameters).             */
/* ------------------------------------------------------------------------ */

typedef struct sbr_scene sbr_scene; /* opaque host-side handle */

/* Device bytes a scene of nt triangles needs (triangle records, BVH nodes,
 * sort and refit scratch). */
size_t sbr_scene_bytes(int32_t nt);

/* Packs the mesh and builds its LBVH (Morton codes of centroids, radix sort,
 * binary radix tree, bottom-up AABB refit, then the 4-wide tree the traversal
 * walks) in d_mem; up to 65,536 triangles the build is one cooperative launch
 * (all its CTAs resident; a device that cannot host them gets the multi-kernel
 * build, same tree).  The paper (Section 3.2.1) names no acceleration
 * structure: this one only speeds up the nearest-hit search of Eq. 2-3.
 * d_verts [nv][3] float32, d_faces [nt][3] int32 stay owned by the caller and
 * are read, not kept.
 * Face indices must lie in [0, nv): out-of-range faces make the build set an
 * error word that the next sbr_scene_check() reports; d_mem must hold
 * sbr_scene_bytes(nt) bytes.  *out is a host handle released by
 * sbr_scene_destroy (which does not touch d_mem). */
sbr_status sbr_scene_create(const float* d_verts, int32_t nv, const int32_t* d_faces,
                            int32_t nt, void* d_mem, size_t mem_bytes, sbr_stream stream,
                            sbr_scene** out);
/* Rebuilds the scene for new vertex positions of the same topology (Morton
 * order, tree and boxes from the new positions).  sbr_scene_refit below keeps
 * the tree and costs less; a rebuild keeps the boxes tight after large vertex
 * moves (the reconstruction loop refits each iteration and rebuilds now and then). */
sbr_status sbr_scene_update(sbr_scene* scene, const float* d_verts, sbr_stream stream);
/* New vertex positions of the same mesh into the tree of the last create or
 * update: the triangles are re-packed in that build's order and every box is
 * recomputed bottom-up, the topology (Morton order, children) kept.  The trace
 * of a refitted scene finds the same hits as that of a rebuilt one (the nearest
 * hit does not depend on the tree); it only slows down as the positions drift
 * from those the tree was built for, so callers moving vertices far rebuild
 * now and then.  Cheaper than sbr_scene_update (no Morton codes, sort or tree
 * construction).  Same errors as sbr_scene_update. */
sbr_status sbr_scene_refit(sbr_scene* scene, const float* d_verts, sbr_stream stream);
/* Synchronises the stream and reports a device-side error word set by the
 * build: bit 0 (a face index outside [0, nv)) gives SBR_ERR_INVALID_ARG; bit 1
 * (the crossing-node bound of the tiled refit exceeded, which a radix tree
 * cannot do) and bit 2 (a grid barrier of the cooperative build gave up after
 * its bounded wait) give SBR_ERR_CUDA, and the scene must be recreated. */
sbr_status sbr_scene_check(const sbr_scene* scene, sbr_stream stream);
void sbr_scene_destroy(sbr_scene* scene);

/* Surface materials (Section 3.2.2, Eq. 9-10: Fresnel reflection with a complex
 * relative permittivity per material).  Material m has eps_m = eps_re[m] -
 * j eps_im[m] (eps_im = sigma / (omega eps_0) >= 0); eps_re[m] <= 0 marks a
 * perfect conductor.  Reading of the paper (whose Eq. 10 inverts Snell's law
 * and calls the index ratio an impedance): cos d_i = |d . n|, sin d_t =
 * sin d_i / sqrt(eps), eta = sqrt(eps), so that Eq. 9 is the textbook pair
 *   r_s = (cos d_i - w) / (cos d_i + w),  r_p = (eps cos d_i - w) / (eps cos d_i + w),
 *   w = eta cos d_t = sqrt(eps - sin^2 d_i)   (principal root, Re w >= 0);
 * the radar's polarisation is taken perpendicular to each plane of incidence,
 * so every interaction applies r_s: a path scattering back at its k-th hit
 * carries F = prod_{j<k} r_s(j) * (-r_s(k)), and with perfect conductors
 * everywhere F = (-1)^(k-1), the conductor model used without materials. */
typedef struct {
  int32_t n_materials;           /* 0: every surface a perfect conductor (the rest unread) */
  int32_t _pad;
  const int32_t* tri_material;   /* device [nt], material of each triangle in the caller's face order;
                                    NULL: every triangle material 0.  Borrowed: must stay valid while
                                    the scene is traced or differentiated. */
  float eps_re[SBR_MAX_MATERIALS];
  float eps_im[SBR_MAX_MATERIALS];
} sbr_materials;

/* Attaches (or, with NULL or n_materials = 0, removes) materials: the scene's
 * later sbr_trace calls fold each path's Fresnel factor F into its strength
 * and phase, and sbr_trace_bwd can return dL/d eps.  Host-side only (the table
 * is copied); SBR_ERR_INVALID_ARG for more than SBR_MAX_MATERIALS materials,
 * eps_im < 0, or |eps - 1| < 1e-6 (a surface that does not reflect).
 * Material indices outside [0, n_materials) are clamped to the last material. */
sbr_status sbr_scene_set_materials(sbr_scene* scene, const sbr_materials* materials);

/* Moving objects (the scene dynamics of Section 3.1).  Each triangle belongs to
 * an object that translates with a constant velocity (m/s, radar frame) over the
 * frame of chirps; every hit point moves with its object, so a path's length
 * changes at dL/dt = sum_j v_j . (u_in,j - u_out,j) (u_in,j and u_out,j the unit
 * vectors of the legs arriving at and leaving hit j; the first leg from Tx, the
 * last towards Rx), and chirp c, starting c chirp_rep after the first, sees the
 * delay tau + c chirp_rep (dL/dt) / c_0.  Amplitudes are held over the frame. */
typedef struct {
  int32_t n_objects;            /* 0: a static scene (the rest unread) */
  int32_t _pad;
  const int32_t* tri_object;    /* device [nt], object of each triangle in the caller's face order; NULL:
                                   all object 0.  Borrowed: must stay valid while the scene is traced. */
  float velocity[SBR_MAX_OBJECTS][3];
} sbr_motion;

/* Attaches (or, with NULL or n_objects = 0, removes) object motion: later
 * sbr_trace calls write every path's dL/dt to paths->path_rate, which
 * sbr_synthesize reads in SBR_SYNTH_MOVING mode.  Host-side only;
 * SBR_ERR_INVALID_ARG for more than SBR_MAX_OBJECTS objects or non-finite
 * velocities.  Object indices outside [0, n_objects) are clamped. */
sbr_status sbr_scene_set_motion(sbr_scene* scene, const sbr_motion* motion);

/* ------------------------------------------------------------------------ */
/* Trace (Section 3.2.1, Eq. 2-3) and path preparation                      */
/* ------------------------------------------------------------------------ */

/* Caller-owned path records, carved from one region by sbr_paths_bind.
 * R rays x K bounces slots; P <= R*K valid paths are compacted ray-major,
 * bounce-minor; per path and virtual antenna v the synthesis record is at
 * prep[v * path_cap + p]. */
typedef struct {
  int32_t n_rays, max_bounces, n_virt, _pad;
  int64_t path_cap;   /* = n_rays * max_bounces */
  sbr_hit* hits;      /* [R*K] nearest hits */
  float* hit_pos;     /* [R*K*8] hit point as float-float pairs: x = [0] + [1],
                         y = [2] + [3], z = [4] + [5] (about 48 bits); [6] = |d_k . n_k| */
  float* ray_weight;  /* [R] solid-angle weight omega */
  int32_t* ray_first; /* [R+1] first path of each ray (exclusive scan); [R] = P */
  int32_t* path_ray;  /* [path_cap] ray of path p */
  float* prep;        /* [V*path_cap*4] {phi0, delta_hi, delta_lo, A} per (v, p) */
  float* path_len;    /* [V*path_cap*2] path length L_in + L_out [m] per (v, p) as a
                         float-float pair (hi, lo); tau = L / c */
  int32_t* count;     /* [1] P (device) */
  void* scratch;      /* scan scratch */
  float* phase_ofs;   /* [path_cap] phase of the path's Fresnel factor F in cycles (0 without
                         materials); folded into phi0 of prep, read by the FP64 and naive
                         synthesis modes, which form the carrier phase from path_len */
  float* path_rate;   /* [V*path_cap] dL/dt [m/s] per (v, p), written only when the scene has motion */
} sbr_paths;

size_t sbr_paths_bytes(int32_t n_rays, int32_t max_bounces, int32_t n_virt);
sbr_status sbr_paths_bind(void* d_mem, size_t bytes, int32_t n_rays, int32_t max_bounces,
                          int32_t n_virt, sbr_paths* out);

/* Traces the grid's rays (all G*G when n_ids < 0; otherwise the n_ids ray
 * indices in d_ray_ids, each in [0, G*G), any order, n_ids = 0 allowed) through up to max_bounces specular interactions with
 * nearest-hit Moller-Trumbore tests (FP32 with a guarded float-float fallback,
 * about 48 significant bits, that makes the chosen triangle that of an FP64
 * brute-force search except within rounding distance of an edge or tie),
 * skipping the previously hit triangle; refines every hit in float-float
 * (Section 3.2.1, Eq. 2-3), and writes per path and virtual antenna the
 * float-float delay tau = (|h_1 - Tx_t| + sum |h_j - h_{j-1}| +
 * |Rx_r - h_k|) / c, its phase terms frac(f_c tau), frac(mu tau T / N_s) split
 * hi/lo, and the strength A = omega (-1)^(k-1) |d_k . n_k| / (4 pi L_in L_out).
 * With materials attached to the scene (sbr_scene_set_materials) the factor
 * (-1)^(k-1) becomes the path's Fresnel factor F: prep holds A |F| and
 * phi0 + arg(F) / (2 pi), phase_ofs[p] = arg(F) / (2 pi).
 * paths must come from sbr_paths_bind with n_rays = (n_ids < 0 ? G*G : n_ids). */
sbr_status sbr_trace(const sbr_scene* scene, const sbr_radar_cfg* radar,
                     const sbr_ray_grid* grid, const int32_t* d_ray_ids, int32_t n_ids,
                     int32_t max_bounces, const sbr_paths* paths, sbr_stream stream);

/* sbr_trace plus work counters for roofline accounting: d_counts[0] = 4-wide
 * BVH nodes fetched (112 B each), [1] = triangles tested (48 B each), [2] = ray
 * traversals (one per bounce attempted), [3] = 0.  d_counts (device, 4 x
 * uint64) is zeroed by the call.  Same results as sbr_trace; slower (the
 * counting kernel variant), so not for timed runs. */
sbr_status sbr_trace_counts(const sbr_scene* scene, const sbr_radar_cfg* radar,
                            const sbr_ray_grid* grid, const int32_t* d_ray_ids, int32_t n_ids,
                            int32_t max_bounces, const sbr_paths* paths, uint64_t* d_counts,
                            sbr_stream stream);

/* ------------------------------------------------------------------------ */
/* Synthesis (Section 3.2.2, Eq. 8)                                         */
/* ------------------------------------------------------------------------ */

/* Scratch bytes for sbr_synthesize / sbr_synthesize_bwd. */
size_t sbr_synth_ws_bytes(const sbr_radar_cfg* radar, int64_t path_cap);

/* d_cube [V][C][N_s] complex64 (interleaved re, im) =
 *   sum_p A_{p,v} exp(j 2 pi (f_c tau_{p,v} + mu tau_{p,v} t_n)),
 * broadcast over the C chirps of a static scene.  Deterministic: partial sums
 * per CTA are reduced in a fixed order.  SBR_PHASE_SPLIT with N_s <= 512 and
 * at least 65536 record slots (path_cap * n_virt) is evaluated as a type-1
 * non-uniform FFT (spreading onto 2 N_s grid points with a width-8
 * exponential-of-semicircle kernel, one FFT, deconvolution; ~1e-6 relative to
 * the FP64 sum), term by term otherwise.  SBR_PHASE_FP64 forms each
 * sample's phase in FP64 from paths->path_len; SBR_PHASE_NAIVE rounds the delay
 * to FP32.  With SBR_SYNTH_MOVING OR'ed into mode (paths traced on a scene with
 * motion) every chirp c is synthesised from the delays tau + c chirp_rep
 * (dL/dt) / c_0, chirp by chirp; the adjoint below is the static model's. */
sbr_status sbr_synthesize(const sbr_paths* paths, const sbr_radar_cfg* radar,
                          sbr_phase_mode mode, float* d_cube, void* d_ws, size_t ws_bytes,
                          sbr_stream stream);

/* Allocation-free variant of sbr_synthesize (the paper has no counterpart;
 * this is a deployment convenience).  Some callers cannot allocate device
 * memory where they synthesise: plugin hosts that own every device
 * allocation and hand none to their plugins, real-time loops that must not
 * risk the device-wide synchronisation an allocation can cause, or code under
 * a fixed memory budget.  This entry point takes no workspace: its per-CTA
 * partial sums live in one file-scope device array of 1 MiB (131072 complex
 * FP32 values) that every GPU which loads the library keeps until the process
 * exits.  Same inputs and outputs as sbr_synthesize; it always sums Eq. 8 term
 * by term (for SBR_PHASE_SPLIT with 256 or 512 samples as an fp16x3 tensor-core
 * GEMM over the paths), where sbr_synthesize evaluates the split mode up to 512
 * samples as a non-uniform FFT: the two agree to about 1e-6 relative.  Limits:
 *  - n_virt * n_samples must not exceed 131072, otherwise SBR_ERR_UNSUPPORTED
 *    is returned before anything is enqueued;
 *  - the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    life of the process; make that first call before any stream capture on
 *    the device.  A cudaDeviceReset of that device leaves the kept address
 *    stale: do not call this entry point on the device again in that process;
 *  - every call shares the one array: calls whose work overlaps on the GPU
 *    (different streams, concurrent host threads) race on it and must be
 *    serialised by the caller.  Each call overwrites every partial sum it
 *    later reads, so no state carries over between calls.
 * It calls no cudaMalloc/cudaFree or other allocating routine. */
sbr_status sbr_synthesize_noalloc(const sbr_paths* paths, const sbr_radar_cfg* radar,
                                  sbr_phase_mode mode, float* d_cube, sbr_stream stream);

/* Adjoint through Eq. 11-12: for upstream d_gcube = dL/dRe + j dL/dIm of the
 * cube, writes d_gtau [V*path_cap] = dL/dtau (per metre of path length, i.e.
 * dL/dtau / c), d_gamp [V*path_cap] = dL/dA and, when d_gphase is not NULL,
 * d_gphase [V*path_cap] = dL/d(phase offset in cycles) (the path's Fresnel
 * phase; needed by sbr_trace_bwd when the scene has materials). */
sbr_status sbr_synthesize_bwd(const sbr_paths* paths, const sbr_radar_cfg* radar,
                              const float* d_gcube, float* d_glen, float* d_gamp, float* d_gphase,
                              void* d_ws, size_t ws_bytes, sbr_stream stream);

/* ------------------------------------------------------------------------ */
/* Point cloud (the map T of Eq. 16)                                        */
/* ------------------------------------------------------------------------ */

/* Saved state of one point-cloud evaluation (needed by its adjoint) and its
 * scratch, carved from one region by sbr_pc_bind. */
typedef struct {
  int32_t n_virt, n_chirps, n_samples, n_theta, k_max, n_elev;
  float* spec;        /* [V*C*N_s*2] range+Doppler spectrum X */
  float* power;       /* [n_elev*n_theta*N_s] power map Pw, row e*n_theta+a */
  int32_t* peak_cell; /* [k_max] linear cell rho*N_s+k of each output point */
  int32_t* n_points;  /* [1] number of points written (device) */
  int32_t* argmax;    /* [1] cell of max Pw */
  void* scratch;
} sbr_pc_state;

size_t sbr_pc_bytes(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar);
sbr_status sbr_pc_bind(void* d_mem, size_t bytes, const sbr_radar_cfg* radar,
                       const sbr_cfar_cfg* cfar, sbr_pc_state* out);

/* d_points [k_max][4] = (x, y, z, w) ordered by (w desc, cell asc); rows at
 * and beyond *n_points are zero.  Detection: 3x3x3 (elevation, azimuth, range)
 * local maxima; each point is (r u, r w, r sqrt(1 - u^2 - w^2)) after a
 * parabolic refine of ln Pw along each axis.  The angle DFT runs on the tensor
 * cores (tcgen05, TF32 with a hi/lo operand split: ~1e-6 relative to FP32) when
 * R <= 128, V <= 16 and N_s is a multiple of 128, on CUDA cores otherwise. */
sbr_status sbr_pointcloud(const float* d_cube, const sbr_radar_cfg* radar,
                          const sbr_cfar_cfg* cfar, float* d_points, sbr_pc_state* state,
                          sbr_stream stream);

/* Steps 1-4 of sbr_pointcloud only: range FFT, Doppler FFT, angle DFT and the
 * range-angle power map Pw [R][N_s] = sum over Doppler bins of |Y|^2, left
 * in state->power (and the spectrum in state->spec, for the adjoint); no
 * detection, no points.  This is the image T(y) of the spatial loss below. */
sbr_status sbr_power_map(const float* d_cube, const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar,
                         sbr_pc_state* state, sbr_stream stream);

/* Spatial multi-antenna loss (Section 3.4, Eq. 16):
 *   loss = (1/N) sum_i (T(y)_i - T(ybar)_i)^2,  N = R x N_s,
 * with T(y) the power map Pw of the last sbr_power_map or sbr_pointcloud on
 * `state` (the paper names T only as a signal-processing map to a spatial
 * image; this library's image is the range-angle power map) and d_target
 * [R][N_s] the target image T(ybar).  Writes *d_loss (device float) and,
 * when d_gcube is not NULL, dloss/dcube [V][C][N_s] complex (overwritten)
 * through the adjoints of the power map, the angle DFT and the two FFTs.
 * Deterministic (fixed-order sums). */
sbr_status sbr_image_loss(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, const sbr_pc_state* state,
                          const float* d_target, float* d_loss, float* d_gcube, sbr_stream stream);

/* Synchronises the stream and reports the device-side status of the last
 * sbr_pointcloud on `state` (each call clears it on entry): SBR_ERR_TIMEOUT
 * when the tensor-core angle DFT (used for R <= 128, at most 16 virtual
 * antennas and N_s a multiple of 128) gave up its bounded wait for its matrix
 * products, in which case the power map holds NaN. */
sbr_status sbr_pc_check(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, const sbr_pc_state* state,
                        sbr_stream stream);

/* Adjoint: d_gpoints [k_max][4] -> d_gcube [V][C][N_s] complex (overwritten).
 * Bitwise reproducible: the gradients of overlapping point neighbourhoods are
 * summed per power-map cell as fixed-point integers, the rest in fixed orders. */
sbr_status sbr_pointcloud_bwd(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar,
                              const sbr_pc_state* state, const float* d_gpoints,
                              float* d_gcube, sbr_stream stream);

/* ------------------------------------------------------------------------ */
/* Trace adjoint (Section 3.3, Eq. 13; interior derivative, Eq. 4-5; the    */
/* reparameterised samples of Eq. 6-7 with SBR_BWD_REPARAM)                 */
/* ------------------------------------------------------------------------ */

/* sbr_trace_bwd flags.  SBR_BWD_REPARAM: differentiate under the change of
 * variables of Eq. 6-7 instead of with fixed launch directions.  T attaches each
 * ray's first hit to its triangle at the forward hit's barycentrics (u, v), so
 * the launch direction follows the surface, d_1 = (x - o)/|x - o| with
 * x = (1 - u - v) a + u b + v c, and the ray's solid-angle weight takes the
 * factor |det J_T| = J / J_0, J = |N.(x - o)| / |x - o|^3 (N = (b - a) x (c - a)):
 * the gradient gains the motion of the sample with the surface and the term
 * f dlog|det J_T| of Eq. 7.  This carries the silhouette (boundary) term of a
 * surface seen against empty space, which fixed directions miss; occlusion
 * edges between two surfaces are not reparameterised. */
#define SBR_BWD_REPARAM 0x1

/* Scratch bytes of sbr_trace_bwd for a scene of nv vertices (a 64-bit
 * accumulator per vertex coordinate and per material parameter, status words). */
size_t sbr_trace_bwd_ws_bytes(int32_t nv);

/* Accumulates dL/dverts [nv][3] (added to d_gverts) from per-path gradients
 * d_glen (dL/d path length, [V*path_cap]) and d_gamp (dL/dA) through the
 * hit points, reflection directions and |d.n| of every bounce; triangle
 * indices stay those of the forward trace (visibility is held fixed).
 * d_verts are the vertices the scene was built from; d_ray_ids is the
 * forward call's ray list (NULL when it traced the whole grid).  The per-corner
 * contributions are summed per vertex as 64-bit fixed-point integers (scaled by
 * a power of two set from the largest contribution; resolution ~1e-12 of it),
 * so the gradient is bitwise reproducible whatever order threads run in.
 * With materials on the scene, d_gphase (sbr_synthesize_bwd's dL/d phase
 * offset) is required: the Fresnel factors depend on every bounce's incidence
 * angle, and d_geps, when not NULL, receives (added) dL/d eps_re[m] and
 * dL/d eps_im[m] at [2m], [2m + 1] for m < n_materials (eps = eps_re - j eps_im),
 * summed the same deterministic way.
 * flags: 0 or SBR_BWD_REPARAM (above); other bits SBR_ERR_INVALID_ARG.
 * d_ws (256-byte aligned) holds sbr_trace_bwd_ws_bytes(nv) bytes, else
 * SBR_ERR_OOM.  max_bounces <= 8. */
sbr_status sbr_trace_bwd(const sbr_scene* scene, const float* d_verts, const sbr_radar_cfg* radar,
                         const sbr_ray_grid* grid, const int32_t* d_ray_ids,
                         const sbr_paths* paths, const float* d_glen, const float* d_gamp,
                         const float* d_gphase, float* d_gverts, float* d_geps, int32_t flags, void* d_ws,
                         size_t ws_bytes, sbr_stream stream);

/* ------------------------------------------------------------------------ */
/* Reconstruction loss and optimiser (Section 3.4: Eq. 14 objective and the */
/* Eq. 15 gradient step; the loss terms and Adam are this library's choice) */
/* ------------------------------------------------------------------------ */

/* Weighted squared Chamfer distance between predicted points d_pred
 * [pred_cap][4] (x, y, z, w; the first *d_n_pred rows valid) and target
 * points d_target [n_target][4]:
 *   L = sum_i w_i |p_i - q_nn(i)|^2 / sum_i w_i + sum_j u_j |q_j - p_nn(j)|^2 / sum_j u_j.
 * Writes *d_loss and d_gpred [pred_cap][4] = dL/d(x, y, z, w) (zero rows past
 * the valid count).  Both sides at most 2048 points; deterministic. */
sbr_status sbr_chamfer(const float* d_pred, const int32_t* d_n_pred, int32_t pred_cap,
                       const float* d_target, int32_t n_target, float* d_loss, float* d_gpred,
                       sbr_stream stream);

/* Host helper: CSR vertex adjacency (unique undirected mesh edges) of a host
 * face array.  With h_adj == NULL only *n_adj is computed (size query);
 * h_off has nv + 1 entries. */
sbr_status sbr_mesh_adjacency(const int32_t* h_faces, int32_t nt, int32_t nv, int32_t* h_off,
                              int32_t* h_adj, int32_t adj_cap, int32_t* n_adj);

size_t sbr_laplacian_ws_bytes(int32_t nv);
/* Uniform Laplacian smoothness, weight * mean_i |v_i - mean_{j in N(i)} v_j|^2:
 * ADDS the term to *d_loss and its gradient to d_gverts [nv][3]. */
sbr_status sbr_laplacian(const float* d_verts, int32_t nv, const int32_t* d_off, const int32_t* d_adj,
                         float weight, float* d_loss, float* d_gverts, void* d_ws, size_t ws_bytes,
                         sbr_stream stream);

/* One bias-corrected Adam step on n parameters in place.  *d_step (device)
 * counts completed steps: the update uses t = *d_step + 1 and the call then
 * increments it, so a captured CUDA graph of the loop stays correct. */
sbr_status sbr_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t n,
                         int32_t* d_step, float lr, float beta1, float beta2, float eps, sbr_stream stream);

/* ------------------------------------------------------------------------ */
/* Serving (the deployment form of the simulator; the paper has no serving   */
/* layer): continuous batching of forward-simulation and reconstruction     */
/* requests of uneven mesh and ray budgets on one GPU.                      */
/* ------------------------------------------------------------------------ */

/* Offset allocator over a byte range (first fit, 256-byte granules, adjacent
 * free blocks merged).  Host bookkeeping only: it never touches device memory;
 * the server places every request's device buffers with it. */
typedef struct sbr_arena sbr_arena;
sbr_arena* sbr_arena_create(size_t bytes);
int64_t sbr_arena_alloc(sbr_arena* a, size_t bytes);   /* offset, or -1 when no block fits */
void sbr_arena_free(sbr_arena* a, int64_t offset, size_t bytes);
size_t sbr_arena_used(const sbr_arena* a);
size_t sbr_arena_peak(const sbr_arena* a);
size_t sbr_arena_largest_free(const sbr_arena* a);
void sbr_arena_destroy(sbr_arena* a);

typedef enum { SBR_REQ_FORWARD = 0, SBR_REQ_RECON = 1 } sbr_request_kind;

/* A request.  Host arrays are copied at submission (and, at admission, into the
 * slot's page-locked staging buffer, from which the device copies run
 * asynchronously); out_* must stay valid until the request's completion is
 * returned by sbr_server_poll. */
typedef struct {
  int32_t kind;         /* sbr_request_kind */
  int32_t max_bounces;
  uint64_t mesh_id;     /* caller identity of (verts, faces); equal ids = equal meshes; 0 = not cached */
  const float* verts;   /* host [nv][3] */
  const int32_t* faces; /* host [nt][3] */
  int32_t nv, nt;
  sbr_ray_grid grid;
  /* reconstruction: iterations of forward + loss + adjoints + Adam from verts (the
     tree refitted to the moved vertices each iteration, rebuilt every 50) */
  int32_t iterations;
  int32_t n_target;
  const float* target;  /* host [n_target][4] target points (x, y, z, w) */
  float lr, lap_weight;
  /* results */
  float* out_points;    /* host [k_max][4] point cloud (recon: of the last iteration) */
  float* out_verts;     /* host [nv][3] final vertices of a reconstruction, or NULL */
} sbr_request;

typedef struct {
  int64_t ticket;
  int32_t status;       /* sbr_status of this request */
  int32_t n_points;
  int32_t scene_cached; /* 1: a resident BVH was reused (no build) */
  int32_t cube_cached;  /* 1: a resident IF cube was reused (no trace, no synthesis) */
  float loss;           /* reconstruction: loss of the last iteration */
  float gpu_ms;         /* device time from admission to completion (CUDA events) */
  double t_submit_us, t_admit_us, t_done_us; /* host clock, microseconds since sbr_server_create */
  uint64_t footprint;   /* device bytes the request held while running */
  double gpu_t0_ms, gpu_t1_ms; /* device clock (CUDA events), ms since sbr_server_create: start and end of
                                  the request's work on its slot stream; intervals of different requests
                                  that overlap ran concurrently on the device */
} sbr_completion;

typedef struct {
  uint64_t arena_bytes, used_bytes, peak_bytes, cached_bytes;
  int32_t waiting, running, cached_scenes, cached_cubes;
  int64_t submitted, completed, cache_hits;
} sbr_server_stats;

typedef struct sbr_server sbr_server;

/* Device bytes a request holds while it runs (its admission footprint),
 * excluding a resident scene or cube it may reuse. */
size_t sbr_server_request_bytes(const sbr_radar_cfg* radar, const sbr_cfar_cfg* cfar, const sbr_request* req);
/* d_arena / arena_bytes: the caller's device memory the server may use (the
 * HBM budget).  n_slots requests run concurrently, each on its own stream. */
sbr_status sbr_server_create(void* d_arena, size_t arena_bytes, int32_t n_slots, const sbr_radar_cfg* radar,
                             const sbr_cfar_cfg* cfar, sbr_server** out);
/* Queues a request (FIFO).  SBR_ERR_OOM when its footprint exceeds the whole
 * arena, SBR_ERR_INVALID_ARG for malformed sizes; nothing runs until polled. */
sbr_status sbr_server_submit(sbr_server* s, const sbr_request* req, int64_t* ticket);
/* Cancels a request that has not been admitted (its completion then reports
 * SBR_ERR_CANCELLED); SBR_ERR_INVALID_ARG for unknown or admitted tickets. */
sbr_status sbr_server_cancel(sbr_server* s, int64_t ticket);
/* One turn of the loop: collects requests whose device work has finished
 * (their memory and slots return to the pool), admits waiting requests while a
 * slot is free and their footprint fits (evicting least-recently-used
 * resident scenes and cubes when needed; a request may overtake at most 8
 * larger ones ahead of it), enqueues their work, and copies up to cap
 * completions into out. */
sbr_status sbr_server_poll(sbr_server* s, sbr_completion* out, int32_t cap, int32_t* n_out);
sbr_status sbr_server_get_stats(const sbr_server* s, sbr_server_stats* out);
/* Waits for the device work of every running request, then frees the host state. */
void sbr_server_destroy(sbr_server* s);

#ifdef __cplusplus
}
#endif
#endif /* SBR_H_ */
