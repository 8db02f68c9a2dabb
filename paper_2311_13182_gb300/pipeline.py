"""The forward simulation as one CUDA graph.

A forward step (LBVH build of the current vertices, trace and path preparation
(Section 3.2.1, Eq. 2-3), synthesis (Section 3.2.2, Eq. 8), point cloud (the map
T of Section 3.4)) is about twenty kernel launches and memsets on fixed
buffers.  ``Forward`` captures the sequence once and replays it, so a step costs
one graph launch on the host and no gaps between dependent kernels on the GPU.
New vertex positions of the same topology are written into ``verts`` between
replays (``set_vertices``); everything else (radar, grid, bounce count, CFAR
settings) is fixed at construction.  With ``host_io`` the graph also holds the
step's host traffic: the copy of the vertex positions from a page-locked host
buffer at its start, and the copies of the points and their count into
page-locked host buffers at its end (``run_host``).

``PipelinedForward`` keeps several batches in flight for throughput: the build
of the next batch and the point cloud of an earlier one (and optionally the
synthesis of the previous one) run on more streams beside the current batch's
trace.
"""
from __future__ import annotations

import torch

from . import sim


class Forward:
    def __init__(self, verts: torch.Tensor, faces: torch.Tensor, radar, grid, max_bounces: int, cfar,
                 mode: int = sim.PHASE_SPLIT, graph: bool = True, host_io: bool = False):
        self.radar, self.grid, self.max_bounces, self.cfar, self.mode = radar, grid, max_bounces, cfar, mode
        self.verts = verts.detach().clone().contiguous()
        self.faces = faces.detach().contiguous()
        self.scene = sim.Scene(self.verts, self.faces)
        self.paths = sim.PathBuffers(grid.n_rays, max_bounces, radar.n_virt)
        self.ws = torch.empty(sim.synth_ws_bytes(radar, self.paths.cap), dtype=torch.uint8, device=self.verts.device)
        self.cube = torch.empty((radar.n_virt, radar.n_chirps, radar.n_samples, 2), device=self.verts.device)
        self.state = sim.PcState(radar, cfar)
        self.points = torch.empty((cfar.k_max, 4), device=self.verts.device)
        self.host_io = host_io
        if host_io:
            self.h_verts = torch.empty(self.verts.shape, dtype=torch.float32).pin_memory()
            self.h_verts.copy_(self.verts)
            self.h_points = torch.empty((cfar.k_max, 4), dtype=torch.float32).pin_memory()
            self.h_n = torch.empty(1, dtype=torch.int32).pin_memory()
            self.done = torch.cuda.Event()
        self.graph = None
        if graph:
            # first calls outside the capture: they set per-device kernel attributes
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(2):
                    self.run_eager()
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                if host_io:
                    self.verts.copy_(self.h_verts, non_blocking=True)
                self.run_eager()
                if host_io:
                    self.h_points.copy_(self.points, non_blocking=True)
                    self.h_n.copy_(self.state.n_points_tensor(), non_blocking=True)
            torch.cuda.synchronize()

    def set_vertices(self, verts: torch.Tensor):
        """New positions for the same topology (read by the next run)."""
        self.verts.copy_(verts, non_blocking=True)

    def run_eager(self, events=None):
        """The step as separate launches; events[0..4] (optional) bracket its four stages."""
        def mark(i):
            if events is not None:
                events[i].record()
        mark(0)
        self.scene.update(self.verts)
        mark(1)
        sim.trace(self.scene, self.radar, self.grid, self.max_bounces, out=self.paths)
        mark(2)
        sim.synthesize(self.paths, self.radar, self.mode, out=self.cube, ws=self.ws)
        mark(3)
        sim.pointcloud(self.cube, self.radar, self.cfar, state=self.state, out=self.points)
        mark(4)

    def run(self):
        """One forward step: a graph replay (or the eager launches when built with graph=False)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self.run_eager()

    def run_host(self, verts=None):
        """One step from host memory (requires host_io and the graph): ``verts`` (array-like
        [nv, 3], or None to keep the page-locked buffer's contents) go into the page-locked input
        buffer once the previous step has finished with it, then the graph replays; the points
        and their count land in ``h_points`` / ``h_n`` when ``done`` (an event) completes."""
        if not self.host_io or self.graph is None:
            raise RuntimeError("run_host needs Forward(..., graph=True, host_io=True)")
        if verts is not None:
            self.done.synchronize()  # the previous replay has read the buffer
            self.h_verts.copy_(torch.as_tensor(verts, dtype=torch.float32))
        self.graph.replay()
        self.done.record()

    def n_points(self) -> int:
        return self.state.n_points()


class PipelinedForward:
    """The forward step several batches deep, for throughput.

    A step j (one graph replay; the parity of j picks one of two captured graphs) runs
    independent branches on separate streams, each on buffers of its own parity:

      * the trace of batch j from tree ``scenes[j % 2]``;
      * the LBVH build of batch j+1 from ``verts`` into ``scenes[(j + 1) % 2]``, the tree the
        next step traces (highest priority: its cooperative launch needs all its CTAs resident
        at once, and once the trace's CTAs are being placed it would wait for the trace to
        drain);
      * ``depth`` 4 (the default): the synthesis of batch j-1 from the other of two path
        buffers (lowest priority) and the point cloud of batch j-2 (highest priority);
        ``depth`` 3: the synthesis of batch j after its trace, and the point cloud of batch j-1.

    The branches share no buffer, so the build's few dozen CTAs, the point cloud's small kernels
    and (depth 4) the synthesis fill SMs beside the trace instead of running alone after it;
    every step still builds, traces, synthesizes and images one batch each.  The synthesis call
    starts with its one-wave spreading kernel while the trace's first kernel follows a memset;
    three tiny ops at the head of the synthesis branch let the trace's CTAs be placed first, so
    that the synthesis takes the SMs the trace's last CTAs leave idle rather than holding every
    SM for a wave before the trace starts.  The points after step j are those of the vertices
    set before step j - ``lag`` (``lag`` = depth - 1; earlier steps: the constructor's vertices,
    whose paths and cube the constructor computes).  With ``host_io`` the graph also copies the vertices from
    the page-locked ``h_verts`` at its start, and the points and their count into ``h_points`` /
    ``h_n`` at the point-cloud branch's end (``run_host``).
    """

    SYNTH_DELAY = 3  # tiny ops ahead of the synthesis in its branch

    def __init__(self, verts: torch.Tensor, faces: torch.Tensor, radar, grid, max_bounces: int, cfar,
                 mode: int = sim.PHASE_SPLIT, graph: bool = True, host_io: bool = False, depth: int = 4):
        if depth not in (3, 4):
            raise ValueError("depth must be 3 or 4")
        dev = verts.device
        self.depth, self.lag = depth, depth - 1
        self.radar, self.grid, self.max_bounces, self.cfar, self.mode = radar, grid, max_bounces, cfar, mode
        self.verts = verts.detach().clone().contiguous()
        self.faces = faces.detach().contiguous()
        self.scenes = [sim.Scene(self.verts, self.faces), sim.Scene(self.verts, self.faces)]
        self.paths = [sim.PathBuffers(grid.n_rays, max_bounces, radar.n_virt) for _ in range(depth - 2)]
        self.ws = torch.empty(sim.synth_ws_bytes(radar, self.paths[0].cap), dtype=torch.uint8, device=dev)
        self.cubes = [torch.zeros((radar.n_virt, radar.n_chirps, radar.n_samples, 2), device=dev) for _ in range(2)]
        self.state = sim.PcState(radar, cfar)
        self.points = torch.empty((cfar.k_max, 4), device=dev)
        lo, hi = torch.cuda.Stream.priority_range()  # (lowest, highest): larger numbers run later
        self.build_stream = torch.cuda.Stream(device=dev, priority=hi)
        self.pc_stream = torch.cuda.Stream(device=dev, priority=hi)
        if depth == 4:
            self.trace_stream = torch.cuda.Stream(device=dev, priority=(lo + hi) // 2)
            self.synth_stream = torch.cuda.Stream(device=dev, priority=lo)
            self.delay = torch.zeros(1, dtype=torch.int32, device=dev)
        self.host_io = host_io
        if host_io:
            self.h_verts = torch.empty(self.verts.shape, dtype=torch.float32).pin_memory()
            self.h_verts.copy_(self.verts)
            self.h_points = torch.empty((cfar.k_max, 4), dtype=torch.float32).pin_memory()
            self.h_n = torch.empty(1, dtype=torch.int32).pin_memory()
            self.done = torch.cuda.Event()
        self.graphs = None
        self._prime()  # the first point cloud images a real cube
        if graph:
            # first calls outside the capture: they set per-device kernel attributes
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for j in range(2):
                    self._step(j, copies=False)
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            self.graphs = []
            for p in range(2):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self._step(p, copies=host_io)
                self.graphs.append(g)
            torch.cuda.synchronize()
        self._prime()

    def _prime(self):
        """Step 0's state from the current vertices: tree 0, and the paths and cube the first
        step's synthesis and point cloud take (depth 3: cube 1; depth 4: paths 1 and cube 0)."""
        self.scenes[0].update(self.verts)
        sim.trace(self.scenes[0], self.radar, self.grid, self.max_bounces, out=self.paths[-1])
        sim.synthesize(self.paths[-1], self.radar, self.mode, out=self.cubes[1 if self.depth == 3 else 0], ws=self.ws)
        self.j = 0

    def _step(self, p: int, copies: bool):
        main = torch.cuda.current_stream()
        if copies:  # ahead of every branch, so that the build is not held behind it
            self.verts.copy_(self.h_verts, non_blocking=True)
        side = [self.build_stream, self.pc_stream]
        if self.depth == 4:
            side += [self.trace_stream, self.synth_stream]
        for st in side:
            st.wait_stream(main)
        with torch.cuda.stream(self.build_stream):
            self.scenes[1 - p].update(self.verts)
        with torch.cuda.stream(self.pc_stream):
            sim.pointcloud(self.cubes[1 - p if self.depth == 3 else p], self.radar, self.cfar, state=self.state,
                           out=self.points)
            if copies:
                self.h_points.copy_(self.points, non_blocking=True)
                self.h_n.copy_(self.state.n_points_tensor(), non_blocking=True)
        if self.depth == 3:
            sim.trace(self.scenes[p], self.radar, self.grid, self.max_bounces, out=self.paths[0])
            sim.synthesize(self.paths[0], self.radar, self.mode, out=self.cubes[p], ws=self.ws)
        else:
            with torch.cuda.stream(self.trace_stream):
                sim.trace(self.scenes[p], self.radar, self.grid, self.max_bounces, out=self.paths[p])
            with torch.cuda.stream(self.synth_stream):
                for _ in range(self.SYNTH_DELAY):
                    self.delay.zero_()
                sim.synthesize(self.paths[1 - p], self.radar, self.mode, out=self.cubes[1 - p], ws=self.ws)
        for st in side:
            main.wait_stream(st)

    def synthesized(self):
        """The cube the last step synthesized (that of the vertices set before step j - depth + 2)."""
        q = (self.j - 1) % 2
        return self.cubes[q if self.depth == 3 else 1 - q]

    def set_vertices(self, verts: torch.Tensor):
        """New positions for the same topology: the next step builds their tree and the points
        of the step ``depth`` - 1 steps after it are theirs."""
        self.verts.copy_(verts, non_blocking=True)

    def run(self):
        """One step: a graph replay (or the launches themselves when built with graph=False)."""
        if self.graphs is not None:
            self.graphs[self.j % 2].replay()
        else:
            self._step(self.j % 2, copies=False)
        self.j += 1

    def run_host(self, verts=None):
        """One step from host memory (requires host_io and the graphs): ``verts`` (array-like
        [nv, 3], or None to keep the page-locked buffer's contents) go into the page-locked input
        buffer once the previous step has finished with it, then the graph replays; ``h_points`` /
        ``h_n`` hold the points of the vertices of ``depth`` - 1 calls earlier when ``done``
        completes."""
        if not self.host_io or self.graphs is None:
            raise RuntimeError("run_host needs PipelinedForward(..., graph=True, host_io=True)")
        if verts is not None:
            self.done.synchronize()  # the previous replay has read the buffer
            self.h_verts.copy_(torch.as_tensor(verts, dtype=torch.float32))
        self.run()
        self.done.record()

    def n_points(self) -> int:
        return self.state.n_points()
