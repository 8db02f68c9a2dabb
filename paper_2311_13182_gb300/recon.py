"""Gradient-based mesh reconstruction against a target radar observation (Section 3.4).

One iteration (Eq. 14 objective, Eq. 15 update; Adam in place of plain SGD):
  scene update -> trace -> synthesize -> point cloud            (forward, Eq. 8, Eq. 16's T)
  loss = weighted squared Chamfer(points, target) + w_lap * uniform Laplacian
  point-cloud adjoint -> synthesis adjoint (Eq. 11-12) -> trace adjoint (Eq. 13)
  Adam step on the vertex positions
(reparam=True: the trace adjoint under the reparameterised samples of Eq. 6-7)
or, with loss="image", the paper's spatial multi-antenna loss (Eq. 16): the
target is a range-angle power map [n_theta, N_s], the forward stops at the power
map, and loss = mean squared image difference + w_lap * Laplacian, whose adjoint
enters the synthesis adjoint directly.
Every step is a library kernel with no host synchronisation (the Laplacian term
on a second stream beside the forward pass), so the whole iteration is captured
into a CUDA graph and replayed.  The scene's tree
is refitted to the new vertices each iteration (sbr_scene_refit: the same hits as
a rebuild) and rebuilt every ``rebuild_every`` iterations (two captured graphs), so
that its boxes stay tight as the mesh moves.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sim
from .autograd import Simulator


class Reconstruction:
    def __init__(self, verts0: np.ndarray, faces: np.ndarray, target: torch.Tensor, radar, grid, max_bounces,
                 cfar, lr=1e-3, lap_weight=0.1, ray_ids=None, recompute=False, loss="chamfer", reparam=False,
                 rebuild_every: int = 50, device="cuda"):
        if loss not in ("chamfer", "image"):
            raise ValueError(f"loss must be 'chamfer' or 'image', not {loss!r}")
        if rebuild_every < 1:
            raise ValueError("rebuild_every must be at least 1 (1: rebuild the tree every iteration)")
        self.rebuild_every = int(rebuild_every)
        self.iters = 0  # iterations run (eager or replayed): every rebuild_every-th rebuilds the tree
        self.kind = loss
        self.verts = torch.from_numpy(np.ascontiguousarray(verts0, np.float32)).to(device)
        self.nv = self.verts.shape[0]
        self.sim = Simulator(faces, self.nv, radar, grid, max_bounces, cfar, ray_ids=ray_ids,
                             recompute=recompute, reparam=reparam, device=device)
        self.adj = sim.Adjacency(faces, self.nv, device)
        self.target = target.contiguous().float().to(device)
        self.lr, self.lap_weight = lr, lap_weight
        self.grad = torch.zeros_like(self.verts)
        self.m = torch.zeros_like(self.verts)
        self.v = torch.zeros_like(self.verts)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.loss_lap = torch.zeros(1, dtype=torch.float32, device=device)
        self.lap_stream = torch.cuda.Stream(device=device)
        self.gpoints = torch.zeros((cfar.k_max, 4), dtype=torch.float32, device=device)
        self.graph = None
        self.graph_rebuild = None

    def _iteration(self, rebuild: bool = True):
        self.sim.bvh_refit = not rebuild
        main = torch.cuda.current_stream()
        # The smoothness term depends on the vertices alone, so it runs on a second stream
        # beside the forward pass: it zeroes the gradient and adds its own term, which the
        # adjoint of the data term then adds to (the same order as one stream), and keeps its
        # loss term apart until the data term has written the loss (the same sum).
        lap_done = torch.cuda.Event()
        self.lap_stream.wait_stream(main)
        with torch.cuda.stream(self.lap_stream):
            self.grad.zero_()
            self.loss_lap.zero_()
            sim.laplacian(self.verts, self.adj, self.lap_weight, self.loss_lap, self.grad)
            lap_done.record()
        if self.kind == "image":
            self.sim.forward_image(self.verts)
            sim.image_loss(self.sim.state, self.target, loss=self.loss, gcube=self.sim.gcube)
        else:
            pts, n = self.sim.forward(self.verts)
            sim.chamfer(pts, n, self.target, loss=self.loss, gpred=self.gpoints)
        self.lap_stream.wait_stream(main)  # the data term has written the loss
        with torch.cuda.stream(self.lap_stream):
            self.loss.add_(self.loss_lap)
        main.wait_event(lap_done)
        if self.kind == "image":
            self.sim.backward_cube(self.verts, self.sim.gcube, self.grad)
        else:
            self.sim.backward(self.verts, self.gpoints, self.grad)
        sim.adam_step(self.verts, self.grad, self.m, self.v, self.step_count, lr=self.lr)
        main.wait_stream(self.lap_stream)

    def _rebuild_now(self) -> bool:
        return self.iters % self.rebuild_every == 0

    def step(self):
        """One eager iteration (the first call also builds the scene)."""
        self._iteration(self._rebuild_now())
        self.iters += 1

    def capture(self):
        """Capture the iteration into CUDA graphs (after at least one eager step): one with
        the tree refitted, one with it rebuilt.  Capturing runs no iteration."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        state = [t.clone() for t in (self.verts, self.m, self.v, self.step_count, self.loss)]
        with torch.cuda.stream(s):
            self._iteration(False)  # warm the stream-local allocator state before capture
            self._iteration(True)
        torch.cuda.current_stream().wait_stream(s)
        for t, t0 in zip((self.verts, self.m, self.v, self.step_count, self.loss), state):
            t.copy_(t0)  # the warm-up iterations leave no trace
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._iteration(False)
        self.graph_rebuild = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph_rebuild):
            self._iteration(True)

    def replay(self, n: int = 1):
        for _ in range(n):
            (self.graph_rebuild if self._rebuild_now() else self.graph).replay()
            self.iters += 1
