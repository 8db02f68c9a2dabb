"""Differentiable simulator: vertices -> radar point cloud with hand-written backward.

``Simulator`` owns the device buffers of one scene/radar/grid configuration and
chains the library calls (Section 3.3, Eq. 13):

  forward   scene update -> sbr_trace -> sbr_synthesize -> sbr_pointcloud
  backward  sbr_pointcloud_bwd -> sbr_synthesize_bwd -> sbr_trace_bwd

With ``recompute=True`` the path records of the forward trace are not kept:
their buffer is released after synthesis and the backward re-traces the same
vertices (triangle sequences are a deterministic function of the vertices),
trading one trace for the path memory (R x K x (48 + 24 V) bytes).
``SimulateFn`` exposes it as a torch.autograd.Function.  A Simulator holds the
state of its latest forward pass only, so each backward must follow its own
forward with no other forward on the same Simulator in between (checked).
"""
from __future__ import annotations

import numpy as np
import torch

from . import sim


class Simulator:
    def __init__(self, faces: np.ndarray, nv: int, radar, grid, max_bounces: int, cfar, ray_ids=None,
                 phase_mode: int = sim.PHASE_SPLIT, recompute: bool = False, materials=None, motion=None,
                 reparam: bool = False, device="cuda"):
        """materials: None (perfect conductors) or (eps, tri_material): complex relative
        permittivities (eps_re - j eps_im; eps_re <= 0 a perfect conductor) and each triangle's
        material index (None: all material 0), Section 3.2.2 Eq. 9-10.
        motion: None (a static scene) or (velocities, tri_object): a velocity [m/s] per object
        and each triangle's object; the forward pass then synthesises every chirp from the
        moving delays (no gradients through the motion).
        reparam: differentiate the trace under the reparameterised samples of Eq. 6-7 (first
        hits attached to their surfaces) instead of with fixed launch directions."""
        self.reparam = reparam
        self.velocities = None
        self.tri_object = None
        if motion is not None:
            vel, tri_obj = motion
            self.velocities = [tuple(float(x) for x in v) for v in vel]
            if tri_obj is not None:
                self.tri_object = torch.as_tensor(np.asarray(tri_obj, np.int32)).to(device)
            phase_mode = phase_mode | sim.SYNTH_MOVING
        self.eps = None
        self.tri_material = None
        if materials is not None:
            eps, tri_mat = materials
            self.eps = [complex(e) for e in eps]
            if tri_mat is not None:
                self.tri_material = torch.as_tensor(np.asarray(tri_mat, np.int32)).to(device)
        self.faces_np = np.ascontiguousarray(faces, dtype=np.int32)
        self.faces = torch.from_numpy(self.faces_np).to(device)
        self.nv, self.radar, self.grid, self.K, self.cfar = nv, radar, grid, max_bounces, cfar
        self.ray_ids = None if ray_ids is None else torch.as_tensor(np.asarray(ray_ids, np.int32)).to(device)
        self.n_rays = grid.G * grid.G if ray_ids is None else int(self.ray_ids.shape[0])
        self.mode, self.recompute, self.device = phase_mode, recompute, device
        self.scene = None
        # after the first build: True refits the tree for new vertex positions
        # (sbr_scene_refit: same hits, no rebuild), False rebuilds it (sbr_scene_update)
        self.bvh_refit = False
        self.paths = None if recompute else sim.PathBuffers(self.n_rays, max_bounces, radar.n_virt, device)
        cap = self.n_rays * max_bounces
        self.synth_ws = torch.empty(sim.synth_ws_bytes(radar, cap), dtype=torch.uint8, device=device)
        self.cube = torch.empty((radar.n_virt, radar.n_chirps, radar.n_samples, 2), dtype=torch.float32,
                                device=device)
        self.points = torch.empty((cfar.k_max, 4), dtype=torch.float32, device=device)
        self.state = sim.PcState(radar, cfar, device)
        self.gcube = torch.empty_like(self.cube)
        self.bwd_ws = torch.empty(sim.trace_bwd_ws_bytes(nv), dtype=torch.uint8, device=device)
        # forward passes so far: the backward reads the state of the latest one only
        self.generation = 0

    def _trace(self, verts):
        if self.scene is None:
            self.scene = sim.Scene(verts, self.faces)
            if self.eps:
                self.scene.set_materials(self.eps, self.tri_material)
            if self.velocities:
                self.scene.set_motion(self.velocities, self.tri_object)
        elif self.bvh_refit:
            self.scene.refit(verts)
        else:
            self.scene.update(verts)
        paths = self.paths if self.paths is not None else sim.PathBuffers(self.n_rays, self.K, self.radar.n_virt,
                                                                        self.device)
        sim.trace(self.scene, self.radar, self.grid, self.K, self.ray_ids, out=paths)
        return paths

    def forward(self, verts: torch.Tensor):
        self.generation += 1
        paths = self._trace(verts)
        sim.synthesize(paths, self.radar, self.mode, out=self.cube, ws=self.synth_ws)
        sim.pointcloud(self.cube, self.radar, self.cfar, state=self.state, out=self.points)
        return self.points, self.state.n_points_tensor()

    def forward_image(self, verts: torch.Tensor):
        """vertices -> range-angle power map [n_theta, N_s] (the image T(y) of Eq. 16)."""
        self.generation += 1
        paths = self._trace(verts)
        sim.synthesize(paths, self.radar, self.mode, out=self.cube, ws=self.synth_ws)
        sim.power_map(self.cube, self.radar, self.cfar, state=self.state)
        return self.state.power()

    def backward(self, verts: torch.Tensor, gpoints: torch.Tensor, gverts: torch.Tensor):
        """Adds dL/dverts to gverts for upstream dL/dpoints [k_max, 4]."""
        sim.pointcloud_bwd(self.state, gpoints.contiguous(), out=self.gcube)
        return self.backward_cube(verts, self.gcube, gverts)

    def backward_cube(self, verts: torch.Tensor, gcube: torch.Tensor, gverts: torch.Tensor,
                      geps: torch.Tensor | None = None):
        """Adds dL/dverts to gverts for upstream dL/dcube [V, C, N_s, 2]; with materials also
        dL/d eps [n_materials, 2] (d eps_re, d eps_im) to ``geps`` when given."""
        if self.velocities:
            raise NotImplementedError("gradients through moving objects are not built (static model only)")
        paths = self.paths if self.paths is not None else self._trace(verts)
        gph = None
        if self.eps:
            glen, gamp, gph = sim.synthesize_bwd(paths, self.radar, gcube, ws=self.synth_ws, phase=True)
        else:
            glen, gamp = sim.synthesize_bwd(paths, self.radar, gcube, ws=self.synth_ws)
        sim.trace_bwd(self.scene, verts, self.radar, self.grid, paths, glen, gamp, self.ray_ids, gverts=gverts,
                      ws=self.bwd_ws, gphase=gph, geps=geps, reparam=self.reparam)
        return gverts


class SimulateFn(torch.autograd.Function):
    """points = SimulateFn.apply(verts, simulator); rows past n_points are zero."""

    @staticmethod
    def forward(ctx, verts, simulator):
        v = verts.detach().contiguous()
        pts, _ = simulator.forward(v)
        ctx.sim = simulator
        ctx.generation = simulator.generation
        ctx.save_for_backward(v)
        return pts.clone()

    @staticmethod
    def backward(ctx, gpoints):
        # the simulator keeps one forward's point-cloud state (and path records):
        # a backward through an older forward would silently use the newer one's
        if ctx.generation != ctx.sim.generation:
            raise RuntimeError("SimulateFn.backward: the Simulator ran another forward pass since this one; "
                               "run one forward per backward, or one Simulator per pending graph")
        (v,) = ctx.saved_tensors
        g = torch.zeros_like(v)
        ctx.sim.backward(v, gpoints.float(), g)
        return g, None
