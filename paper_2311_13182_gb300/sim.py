"""Torch-facing wrappers of the libsbr C ABI (device memory and streams only).

Every function here marshals arguments and calls one ``sbr_*`` entry point;
all arithmetic of the simulator runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

PHASE_SPLIT, PHASE_FP64, PHASE_NAIVE = L.PHASE_SPLIT, L.PHASE_FP64, L.PHASE_NAIVE
SYNTH_MOVING = L.SYNTH_MOVING  # OR into a phase mode: every chirp from the paths' dL/dt
BWD_REPARAM = L.BWD_REPARAM    # sbr_trace_bwd: reparameterised samples (Eq. 6-7)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(t: torch.Tensor, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")


def radar_struct(radar) -> L.RadarCfg:
    r = L.RadarCfg()
    r.f0, r.bandwidth, r.chirp_time, r.chirp_rep = radar.f0, radar.bandwidth, radar.chirp_time, radar.chirp_rep
    r.n_samples, r.n_chirps = radar.n_samples, radar.n_chirps
    r.n_tx, r.n_rx = radar.n_tx, radar.n_rx
    if radar.n_tx > L.MAX_TX or radar.n_rx > L.MAX_RX:
        raise ValueError("too many antennas for the C ABI")
    for t in range(radar.n_tx):
        for j in range(3):
            r.tx[t][j] = float(radar.tx[t][j])
    for q in range(radar.n_rx):
        for j in range(3):
            r.rx[q][j] = float(radar.rx[q][j])
    return r


_JITTER = {}  # id(grid offsets array) -> (array, device copy): the library borrows the device pointer


def jitter_device(grid, device="cuda"):
    """Device copy of a grid's jitter offsets [G*G, 2] (cached per offsets array), or None."""
    jit = getattr(grid, "jitter", None)
    if jit is None:
        return None
    key = id(jit)
    hit = _JITTER.get(key)
    if hit is None or hit[0] is not jit:
        arr = np.ascontiguousarray(jit, dtype=np.float32).reshape(-1, 2)
        if arr.shape[0] != grid.G * grid.G:
            raise ValueError("jitter must hold G*G offset pairs")
        hit = (jit, torch.from_numpy(arr).to(device))
        _JITTER[key] = hit
    return hit[1]


def grid_struct(grid) -> L.RayGrid:
    g = L.RayGrid()
    g.G = grid.G
    for j in range(3):
        g.origin[j] = float(grid.origin[j])
        g.axis[j] = float(grid.axis[j])
        g.u_axis[j] = float(grid.u_axis[j])
        g.v_axis[j] = float(grid.v_axis[j])
    g.tan_half = float(grid.tan_half)
    jd = jitter_device(grid)
    g.jitter = jd.data_ptr() if jd is not None else None
    return g


def cfar_struct(cfg) -> L.CfarCfg:
    c = L.CfarCfg()
    c.n_theta, c.guard, c.train, c.k_max = cfg.n_theta, cfg.guard, cfg.train, cfg.k_max
    c.alpha, c.floor_rel, c.beta, c.w_min = cfg.alpha, cfg.floor_rel, cfg.beta, cfg.w_min
    c.n_elev = int(getattr(cfg, "n_elev", 1))
    return c


def _region(mem: torch.Tensor, ptr: int, dtype, shape):
    """Typed view of a sub-region of ``mem`` starting at device address ``ptr``."""
    off = ptr - mem.data_ptr()
    n = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
    return mem[off:off + n].view(dtype).view(*shape)


class Scene:
    """Triangle mesh + LBVH resident in device memory (sbr_scene_create)."""

    def __init__(self, verts: torch.Tensor, faces: torch.Tensor, stream=None):
        _need_cuda(verts, torch.float32, "verts")
        _need_cuda(faces, torch.int32, "faces")
        self.nv, self.nt = int(verts.shape[0]), int(faces.shape[0])
        nbytes = int(L.load().sbr_scene_bytes(self.nt))
        self.mem = torch.empty(nbytes, dtype=torch.uint8, device=verts.device)
        h = ctypes.c_void_p()
        L.call("sbr_scene_create", _vp(verts), self.nv, _vp(faces), self.nt, _vp(self.mem), nbytes,
               _stream(stream), ctypes.byref(h))
        self.handle = h
        self.device = verts.device

    @staticmethod
    def bytes_for(nt: int) -> int:
        return int(L.load().sbr_scene_bytes(nt))

    def update(self, verts: torch.Tensor, stream=None):
        _need_cuda(verts, torch.float32, "verts")
        L.call("sbr_scene_update", self.handle, _vp(verts), _stream(stream))

    def refit(self, verts: torch.Tensor, stream=None):
        """sbr_scene_refit: new positions into the last build's tree (same hits, no rebuild)."""
        _need_cuda(verts, torch.float32, "verts")
        L.call("sbr_scene_refit", self.handle, _vp(verts), _stream(stream))

    def check(self, stream=None):
        L.call("sbr_scene_check", self.handle, _stream(stream))

    def set_materials(self, eps, tri_material: torch.Tensor | None = None):
        """sbr_scene_set_materials: complex relative permittivities ``eps`` (eps_re - j eps_im, a
        material with eps_re <= 0 is a perfect conductor) and the material of each triangle
        (device int32 [nt], None: all material 0); ``eps`` empty or None removes them."""
        m = L.Materials()
        eps = [] if eps is None else [complex(e) for e in eps]
        if len(eps) > L.MAX_MATERIALS:
            raise ValueError(f"at most {L.MAX_MATERIALS} materials")
        m.n_materials = len(eps)
        for i, e in enumerate(eps):
            m.eps_re[i], m.eps_im[i] = e.real, -e.imag
        if tri_material is not None:
            _need_cuda(tri_material, torch.int32, "tri_material")
        self._tri_material = tri_material          # borrowed by the library: keep it alive
        m.tri_material = tri_material.data_ptr() if tri_material is not None else None
        L.call("sbr_scene_set_materials", self.handle, ctypes.byref(m))
        self.n_materials = len(eps)

    def set_motion(self, velocities, tri_object: torch.Tensor | None = None):
        """sbr_scene_set_motion: a velocity [m/s] per object and the object of each triangle
        (device int32 [nt], None: all object 0); empty or None makes the scene static."""
        m = L.Motion()
        vel = [] if velocities is None else [tuple(float(x) for x in v) for v in velocities]
        if len(vel) > L.MAX_OBJECTS:
            raise ValueError(f"at most {L.MAX_OBJECTS} objects")
        m.n_objects = len(vel)
        for i, v in enumerate(vel):
            for j in range(3):
                m.velocity[i][j] = v[j]
        if tri_object is not None:
            _need_cuda(tri_object, torch.int32, "tri_object")
        self._tri_object = tri_object              # borrowed by the library: keep it alive
        m.tri_object = tri_object.data_ptr() if tri_object is not None else None
        L.call("sbr_scene_set_motion", self.handle, ctypes.byref(m))
        self.n_objects = len(vel)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and L._LIB is not None:
            L._LIB.sbr_scene_destroy(h)
            self.handle = None


class PathBuffers:
    """Caller-owned path records of one trace (sbr_paths_bind)."""

    def __init__(self, n_rays: int, max_bounces: int, n_virt: int, device="cuda"):
        nbytes = int(L.load().sbr_paths_bytes(n_rays, max_bounces, n_virt))
        if nbytes == 0:
            raise ValueError("invalid path buffer sizes")
        self.mem = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.s = L.Paths()
        L.call("sbr_paths_bind", _vp(self.mem), nbytes, n_rays, max_bounces, n_virt, ctypes.byref(self.s))
        self.R, self.K, self.V, self.cap = n_rays, max_bounces, n_virt, int(self.s.path_cap)

    @staticmethod
    def bytes_for(n_rays, max_bounces, n_virt) -> int:
        return int(L.load().sbr_paths_bytes(n_rays, max_bounces, n_virt))

    def hits(self):
        raw = _region(self.mem, self.s.hits, torch.int32, (self.R, self.K, 4))
        return raw[..., 0], raw[..., 1:].view(torch.float32)

    def hit_pos(self):
        """Raw hit records [R, K, 8]: float-float x, y, z pairs and |d.n| (see sbr.h)."""
        return _region(self.mem, self.s.hit_pos, torch.float32, (self.R, self.K, 8))

    def hit_points(self):
        """Hit points [R, K, 3] in float64 (hi + lo of the stored float-float pairs)."""
        raw = self.hit_pos().double()
        return raw[..., 0:6:2] + raw[..., 1:6:2]

    def ray_weight(self):
        return _region(self.mem, self.s.ray_weight, torch.float32, (self.R,))

    def ray_first(self):
        return _region(self.mem, self.s.ray_first, torch.int32, (self.R + 1,))

    def path_ray(self):
        return _region(self.mem, self.s.path_ray, torch.int32, (max(self.cap, 1),))

    def prep(self):
        return _region(self.mem, self.s.prep, torch.float32, (self.V, max(self.cap, 1), 4))

    def path_len(self):
        """Path lengths L_in + L_out [V, path_cap] in float64 (hi + lo of the stored pairs)."""
        raw = _region(self.mem, self.s.path_len, torch.float32, (self.V, max(self.cap, 1), 2)).double()
        return raw[..., 0] + raw[..., 1]

    def path_rate(self):
        """dL/dt [V, path_cap] in m/s (written by a trace of a scene with motion)."""
        return _region(self.mem, self.s.path_rate, torch.float32, (self.V, max(self.cap, 1)))

    def phase_ofs(self):
        """Per-path Fresnel phase [path_cap] in cycles (0 without materials)."""
        return _region(self.mem, self.s.phase_ofs, torch.float32, (max(self.cap, 1),))

    def count_tensor(self):
        return _region(self.mem, self.s.count, torch.int32, (1,))

    def count(self) -> int:
        return int(self.count_tensor().item())


def trace(scene: Scene, radar, grid, max_bounces: int, ray_ids: torch.Tensor | None = None,
          out: PathBuffers | None = None, stream=None) -> PathBuffers:
    """sbr_trace: nearest-hit specular trace of the grid (or of ``ray_ids``) + path prep."""
    n = int(ray_ids.shape[0]) if ray_ids is not None else grid.G * grid.G
    if ray_ids is not None:
        _need_cuda(ray_ids, torch.int32, "ray_ids")
    V = radar.n_tx * radar.n_rx
    if out is None:
        out = PathBuffers(n, max_bounces, V, device=scene.device)
    r, g = radar_struct(radar), grid_struct(grid)
    L.call("sbr_trace", scene.handle, ctypes.byref(r), ctypes.byref(g), _vp(ray_ids),
           n if ray_ids is not None else -1, max_bounces, ctypes.byref(out.s), _stream(stream))
    return out


def trace_counts(scene: Scene, radar, grid, max_bounces: int, out: PathBuffers, ray_ids=None, stream=None):
    """sbr_trace_counts: the trace of ``trace`` plus (nodes fetched, triangles tested, traversals)."""
    counts = torch.zeros(4, dtype=torch.int64, device=scene.device)
    r, g = radar_struct(radar), grid_struct(grid)
    n = int(ray_ids.shape[0]) if ray_ids is not None else -1
    L.call("sbr_trace_counts", scene.handle, ctypes.byref(r), ctypes.byref(g), _vp(ray_ids), n, max_bounces,
           ctypes.byref(out.s), _vp(counts), _stream(stream))
    c = counts.cpu().tolist()
    return c[0], c[1], c[2]


def synth_ws_bytes(radar, path_cap: int) -> int:
    return int(L.load().sbr_synth_ws_bytes(ctypes.byref(radar_struct(radar)), path_cap))


def synthesize(paths: PathBuffers, radar, mode: int = PHASE_SPLIT, out: torch.Tensor | None = None,
               ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """sbr_synthesize: IF cube [V, C, N_s, 2] float32 (re, im) of Eq. 8."""
    r = radar_struct(radar)
    V, C, Ns = radar.n_virt, radar.n_chirps, radar.n_samples
    if out is None:
        out = torch.empty((V, C, Ns, 2), dtype=torch.float32, device=paths.mem.device)
    nb = synth_ws_bytes(radar, paths.cap)
    if ws is None or ws.numel() < nb:
        ws = torch.empty(nb, dtype=torch.uint8, device=paths.mem.device)
    L.call("sbr_synthesize", ctypes.byref(paths.s), ctypes.byref(r), int(mode), _vp(out), _vp(ws), nb,
           _stream(stream))
    return out


def synthesize_bwd(paths: PathBuffers, radar, gcube: torch.Tensor, ws: torch.Tensor | None = None,
                   phase: bool = False, stream=None):
    """sbr_synthesize_bwd: (dL/d path length, dL/dA), each [V, path_cap] float32, and with
    ``phase`` also dL/d(phase offset in cycles) as a third array."""
    _need_cuda(gcube, torch.float32, "gcube")
    r = radar_struct(radar)
    glen = torch.empty((paths.V, max(paths.cap, 1)), dtype=torch.float32, device=gcube.device)
    gamp = torch.empty_like(glen)
    gph = torch.empty_like(glen) if phase else None
    nb = synth_ws_bytes(radar, paths.cap)
    if ws is None or ws.numel() < nb:
        ws = torch.empty(nb, dtype=torch.uint8, device=gcube.device)
    L.call("sbr_synthesize_bwd", ctypes.byref(paths.s), ctypes.byref(r), _vp(gcube), _vp(glen), _vp(gamp),
           _vp(gph), _vp(ws), nb, _stream(stream))
    return (glen, gamp, gph) if phase else (glen, gamp)


class PcState:
    """Saved state + scratch of one point-cloud evaluation (sbr_pc_bind)."""

    def __init__(self, radar, cfar, device="cuda"):
        self.r, self.c = radar_struct(radar), cfar_struct(cfar)
        nbytes = int(L.load().sbr_pc_bytes(ctypes.byref(self.r), ctypes.byref(self.c)))
        if nbytes == 0:
            raise ValueError(f"unsupported point-cloud configuration: {L.last_error()}")
        self.mem = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.s = L.PcState()
        L.call("sbr_pc_bind", _vp(self.mem), nbytes, ctypes.byref(self.r), ctypes.byref(self.c),
               ctypes.byref(self.s))
        self.k_max = cfar.k_max
        self.shape = (radar.n_virt, radar.n_chirps, radar.n_samples)
        self.rows = max(1, int(getattr(cfar, "n_elev", 1))) * cfar.n_theta  # angle rows e * n_theta + a

    def n_points_tensor(self):
        return _region(self.mem, self.s.n_points, torch.int32, (1,))

    def n_points(self) -> int:
        return int(self.n_points_tensor().item())

    def power(self):
        return _region(self.mem, self.s.power, torch.float32, (self.rows, self.shape[2]))

    def spectrum(self):
        return _region(self.mem, self.s.spec, torch.float32, (*self.shape, 2))

    def peak_cells(self):
        return _region(self.mem, self.s.peak_cell, torch.int32, (self.k_max,))

    def check(self, stream=None):
        """sbr_pc_check: raises if the last point-cloud call's bounded device wait gave up."""
        L.call("sbr_pc_check", ctypes.byref(self.r), ctypes.byref(self.c), ctypes.byref(self.s), _stream(stream))


def pointcloud(cube: torch.Tensor, radar, cfar, state: PcState | None = None, out: torch.Tensor | None = None,
               stream=None):
    """sbr_pointcloud: points [k_max, 4] (x, y, z, w) and the state holding the count."""
    _need_cuda(cube, torch.float32, "cube")
    if state is None:
        state = PcState(radar, cfar, device=cube.device)
    if out is None:
        out = torch.empty((cfar.k_max, 4), dtype=torch.float32, device=cube.device)
    L.call("sbr_pointcloud", _vp(cube), ctypes.byref(state.r), ctypes.byref(state.c), _vp(out),
           ctypes.byref(state.s), _stream(stream))
    return out, state


def power_map(cube: torch.Tensor, radar, cfar, state: PcState | None = None, stream=None) -> PcState:
    """sbr_power_map: the range-angle power map [n_elev * n_theta, N_s] of the cube (row
    e * n_theta + a), left in ``state.power()``."""
    _need_cuda(cube, torch.float32, "cube")
    if state is None:
        state = PcState(radar, cfar, device=cube.device)
    L.call("sbr_power_map", _vp(cube), ctypes.byref(state.r), ctypes.byref(state.c), ctypes.byref(state.s),
           _stream(stream))
    return state


def image_loss(state: PcState, target: torch.Tensor, loss: torch.Tensor | None = None,
               gcube: torch.Tensor | None = None, want_grad: bool = True, stream=None):
    """sbr_image_loss (Eq. 16): loss [1] = mean (Pw - target)^2 over the power map of ``state``,
    and dloss/dcube [V, C, N_s, 2] when ``want_grad``."""
    _need_cuda(target, torch.float32, "target")
    if target.numel() != state.rows * state.shape[2]:
        raise ValueError(f"target of {target.numel()} cells, the power map has {state.rows * state.shape[2]}")
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=target.device)
    if want_grad and gcube is None:
        gcube = torch.empty((*state.shape, 2), dtype=torch.float32, device=target.device)
    L.call("sbr_image_loss", ctypes.byref(state.r), ctypes.byref(state.c), ctypes.byref(state.s), _vp(target),
           _vp(loss), _vp(gcube if want_grad else None), _stream(stream))
    return loss, gcube


def pointcloud_bwd(state: PcState, gpoints: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """sbr_pointcloud_bwd: dL/dcube [V, C, N_s, 2] from dL/dpoints [k_max, 4]."""
    _need_cuda(gpoints, torch.float32, "gpoints")
    if out is None:
        out = torch.empty((*state.shape, 2), dtype=torch.float32, device=gpoints.device)
    L.call("sbr_pointcloud_bwd", ctypes.byref(state.r), ctypes.byref(state.c), ctypes.byref(state.s),
           _vp(gpoints), _vp(out), _stream(stream))
    return out


def trace_bwd_ws_bytes(nv: int) -> int:
    return int(L.load().sbr_trace_bwd_ws_bytes(nv))


def trace_bwd(scene: Scene, verts: torch.Tensor, radar, grid, paths: PathBuffers, glen: torch.Tensor,
              gamp: torch.Tensor, ray_ids: torch.Tensor | None = None, gverts: torch.Tensor | None = None,
              ws: torch.Tensor | None = None, gphase: torch.Tensor | None = None, geps: torch.Tensor | None = None,
              reparam: bool = False, stream=None):
    """sbr_trace_bwd: adds dL/dverts [nv, 3] from per-path (dL/dlength, dL/dA) and, on a scene
    with materials, the Fresnel terms from dL/d(phase offset) ``gphase``; adds dL/d eps
    [n_materials, 2] (d eps_re, d eps_im) to ``geps`` when given.  ``reparam``: the
    reparameterised samples of Eq. 6-7 (SBR_BWD_REPARAM) instead of fixed launch directions."""
    _need_cuda(verts, torch.float32, "verts")
    if gverts is None:
        gverts = torch.zeros_like(verts)
    nb = trace_bwd_ws_bytes(scene.nv)
    if ws is None or ws.numel() < nb:
        ws = torch.empty(nb, dtype=torch.uint8, device=verts.device)
    r, g = radar_struct(radar), grid_struct(grid)
    L.call("sbr_trace_bwd", scene.handle, _vp(verts), ctypes.byref(r), ctypes.byref(g), _vp(ray_ids),
           ctypes.byref(paths.s), _vp(glen), _vp(gamp), _vp(gphase), _vp(gverts), _vp(geps),
           BWD_REPARAM if reparam else 0, _vp(ws), nb, _stream(stream))
    return gverts


def chamfer(pred: torch.Tensor, n_pred: torch.Tensor, target: torch.Tensor, loss: torch.Tensor | None = None,
            gpred: torch.Tensor | None = None, stream=None):
    """sbr_chamfer: weighted squared Chamfer loss [1] and dL/dpred [cap, 4]."""
    _need_cuda(pred, torch.float32, "pred")
    _need_cuda(target, torch.float32, "target")
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=pred.device)
    if gpred is None:
        gpred = torch.empty_like(pred)
    L.call("sbr_chamfer", _vp(pred), _vp(n_pred), int(pred.shape[0]), _vp(target), int(target.shape[0]),
           _vp(loss), _vp(gpred), _stream(stream))
    return loss, gpred


class Adjacency:
    """CSR vertex adjacency of a mesh topology, resident on the device."""

    def __init__(self, faces: np.ndarray, nv: int, device="cuda"):
        f = np.ascontiguousarray(faces, dtype=np.int32)
        n = ctypes.c_int32()
        off = np.zeros(nv + 1, np.int32)
        L.call("sbr_mesh_adjacency", f.ctypes.data_as(ctypes.c_void_p), f.shape[0], nv,
               off.ctypes.data_as(ctypes.c_void_p), None, 0, ctypes.byref(n))
        adj = np.zeros(max(n.value, 1), np.int32)
        L.call("sbr_mesh_adjacency", f.ctypes.data_as(ctypes.c_void_p), f.shape[0], nv,
               off.ctypes.data_as(ctypes.c_void_p), adj.ctypes.data_as(ctypes.c_void_p), adj.shape[0],
               ctypes.byref(n))
        self.nv = nv
        self.off = torch.from_numpy(off).to(device)
        self.adj = torch.from_numpy(adj).to(device)
        nb = int(L.load().sbr_laplacian_ws_bytes(nv))
        self.ws = torch.empty(nb, dtype=torch.uint8, device=device)


def laplacian(verts: torch.Tensor, adj: Adjacency, weight: float, loss: torch.Tensor, gverts: torch.Tensor,
              stream=None):
    """sbr_laplacian: adds weight * uniform-Laplacian term to loss and its gradient to gverts."""
    L.call("sbr_laplacian", _vp(verts), adj.nv, _vp(adj.off), _vp(adj.adj), float(weight), _vp(loss),
           _vp(gverts), _vp(adj.ws), int(adj.ws.numel()), _stream(stream))


def adam_step(params: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: torch.Tensor,
              lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """sbr_adam_step: in-place Adam update; ``step`` is a device int32 counter it increments."""
    L.call("sbr_adam_step", _vp(params), _vp(grad), _vp(m), _vp(v), params.numel(), _vp(step), float(lr),
           float(beta1), float(beta2), float(eps), _stream(stream))
