"""Serving front end: submits requests to the native continuous-batching server
(sbr_server_* in libsbr) and drives its loop.

The scheduler, admission by HBM footprint, the resident BVH / IF-cube caches and
the per-request pipelines are C++ in the library; this module marshals
requests, paces a request stream in real time and collects completions.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from . import _lib as L
from . import sim

c_i32, c_i64, c_u64, c_f32, c_f64, c_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float,
                                          ctypes.c_double, ctypes.c_void_p)
FORWARD, RECON = 0, 1


Request, Completion, Stats = L.Request, L.Completion, L.ServerStats


def _declare():
    return L.load()


class Arena:
    """Host-side offset allocator of the server (testable without a GPU)."""

    def __init__(self, nbytes: int):
        self.lib = _declare()
        self.h = self.lib.sbr_arena_create(nbytes)

    def alloc(self, n: int) -> int:
        return int(self.lib.sbr_arena_alloc(self.h, n))

    def free(self, off: int, n: int):
        self.lib.sbr_arena_free(self.h, off, n)

    def used(self) -> int:
        return int(self.lib.sbr_arena_used(self.h))

    def peak(self) -> int:
        return int(self.lib.sbr_arena_peak(self.h))

    def largest_free(self) -> int:
        return int(self.lib.sbr_arena_largest_free(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.sbr_arena_destroy(self.h)
            self.h = None


class Server:
    """Continuous-batching server over a device arena of ``arena_bytes``."""

    def __init__(self, radar, cfar, arena_bytes: int, n_slots: int = 8, device="cuda"):
        self.lib = _declare()
        self.radar, self.cfar = radar, cfar
        self.r, self.c = sim.radar_struct(radar), sim.cfar_struct(cfar)
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=device)
        h = c_p()
        L.check(self.lib.sbr_server_create(c_p(self.arena.data_ptr()), arena_bytes, n_slots, ctypes.byref(self.r),
                                           ctypes.byref(self.c), ctypes.byref(h)), "sbr_server_create")
        self.h = h
        self.live = {}  # ticket -> output buffers kept alive until completion

    def _request(self, kind, verts, faces, grid, max_bounces, mesh_id=0, iterations=0, target=None, lr=1e-3,
                 lap_weight=0.1, want_verts=False):
        v = np.ascontiguousarray(verts, dtype=np.float32)
        f = np.ascontiguousarray(faces, dtype=np.int32)
        q = Request()
        q.kind, q.max_bounces, q.mesh_id = kind, max_bounces, mesh_id
        q.verts, q.faces = v.ctypes.data, f.ctypes.data
        q.nv, q.nt = v.shape[0], f.shape[0]
        q.grid = sim.grid_struct(grid)
        pts = np.zeros((self.cfar.k_max, 4), np.float32)
        q.out_points = pts.ctypes.data
        outv = None
        if kind == RECON:
            t = np.ascontiguousarray(target, dtype=np.float32)
            q.iterations, q.n_target, q.target = iterations, t.shape[0], t.ctypes.data
            q.lr, q.lap_weight = lr, lap_weight
            if want_verts:
                outv = np.zeros_like(v)
                q.out_verts = outv.ctypes.data
            keep = (v, f, t)
        else:
            keep = (v, f)
        return q, pts, outv, keep

    def request_bytes(self, **kw) -> int:
        q, _, _, _keep = self._request(**kw)
        return int(self.lib.sbr_server_request_bytes(ctypes.byref(self.r), ctypes.byref(self.c), ctypes.byref(q)))

    def submit(self, **kw) -> int:
        q, pts, outv, keep = self._request(**kw)
        t = c_i64()
        L.check(self.lib.sbr_server_submit(self.h, ctypes.byref(q), ctypes.byref(t)), "sbr_server_submit")
        self.live[t.value] = (pts, outv)
        return t.value

    def cancel(self, ticket: int):
        L.check(self.lib.sbr_server_cancel(self.h, ticket), "sbr_server_cancel")

    def poll(self, cap: int = 64):
        buf = (Completion * cap)()
        n = c_i32()
        L.check(self.lib.sbr_server_poll(self.h, buf, cap, ctypes.byref(n)), "sbr_server_poll")
        out = []
        for i in range(n.value):
            c = buf[i]
            pts, outv = self.live.pop(c.ticket, (None, None))
            out.append(dict(ticket=c.ticket, status=c.status, n_points=c.n_points,
                            points=None if pts is None else pts[: c.n_points], verts=outv, loss=c.loss,
                            gpu_ms=c.gpu_ms, scene_cached=bool(c.scene_cached), cube_cached=bool(c.cube_cached),
                            t_submit_us=c.t_submit_us, t_admit_us=c.t_admit_us, t_done_us=c.t_done_us,
                            footprint=int(c.footprint), gpu_t0_ms=c.gpu_t0_ms, gpu_t1_ms=c.gpu_t1_ms))
        return out

    def stats(self) -> dict:
        s = Stats()
        L.check(self.lib.sbr_server_get_stats(self.h, ctypes.byref(s)), "sbr_server_get_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def drain(self, timeout_s: float = 600.0):
        res = []
        t_end = time.perf_counter() + timeout_s
        while self.live and time.perf_counter() < t_end:
            res += self.poll()
        return res

    def close(self):
        if getattr(self, "h", None):
            self.lib.sbr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def run_stream(server: Server, items, rate_hz: float, seed: int = 0):
    """Submits ``items`` (dicts of Server.submit keywords) at Poisson arrival times of mean rate
    ``rate_hz`` (seeded), polling the server continuously; returns completions and wall time."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=len(items))
    arrivals = np.cumsum(gaps)
    done, tickets = [], []
    t0 = time.perf_counter()
    i = 0
    while i < len(items) or server.live:
        now = time.perf_counter() - t0
        while i < len(items) and arrivals[i] <= now:
            tickets.append(server.submit(**items[i]))
            i += 1
        done += server.poll()
    wall = time.perf_counter() - t0
    return done, wall, tickets


def device_overlap(done):
    """From the completions' device-clock intervals [gpu_t0_ms, gpu_t1_ms]: the time the device
    had at least one request in flight, and the fraction of it with two or more at once."""
    ev = []
    for d in done:
        if d["status"] == 0 and d["gpu_t1_ms"] > d["gpu_t0_ms"]:
            ev += [(d["gpu_t0_ms"], 1), (d["gpu_t1_ms"], -1)]
    ev.sort()
    busy = multi = 0.0
    depth, last = 0, None
    for t, step in ev:
        if last is not None and depth >= 1:
            busy += t - last
            if depth >= 2:
                multi += t - last
        depth += step
        last = t
    return {"busy_ms": busy, "two_or_more_frac": multi / busy if busy > 0 else 0.0}


def percentiles(ms):
    ms = np.asarray(ms, dtype=np.float64)
    return {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "mean_ms": float(ms.mean())}


def build_items(meshes, reqs, radar, cfar, max_bounces=2):
    """Materialises a serving workload: pool meshes, per-request ray grids over the mesh's
    bounding cone, and for reconstructions a template (the mesh shrunk by 10 % about its
    centre) and a target point cloud (the plain simulator's points of the mesh itself)."""
    from sbr_inputs import bounding_sphere, ray_grid_for_sphere, request_mesh
    pool = {}
    for m in meshes:
        v, f = request_mesh(dict(seed=m["seed"], mesh=m["mesh"], n_tris=m["n_tris"]))
        c, r = bounding_sphere(v)
        pool[m["id"]] = (v, f, c, r)
    items = []
    for q in reqs:
        v, f, c, r = pool[q["mesh"] + 1]
        grid = ray_grid_for_sphere(c, r, q["G"])
        if q["kind"] == "forward":
            items.append(dict(kind=FORWARD, verts=v, faces=f, grid=grid, max_bounces=max_bounces,
                              mesh_id=q["mesh"] + 1))
        else:
            target = plain_forward(v, f, radar, cfar, grid, max_bounces)
            tmpl = (c + 0.9 * (v.astype(np.float64) - c)).astype(np.float32)
            items.append(dict(kind=RECON, verts=tmpl, faces=f, grid=grid, max_bounces=max_bounces,
                              iterations=q["iterations"], target=target[: min(len(target), 2048)],
                              lr=1e-3, lap_weight=0.1))
    return items


def plain_forward(verts, faces, radar, cfar, grid, max_bounces):
    """One forward simulation through the plain (non-served) path; returns the points."""
    v = torch.from_numpy(np.ascontiguousarray(verts, np.float32)).cuda()
    f = torch.from_numpy(np.ascontiguousarray(faces, np.int32)).cuda()
    scene = sim.Scene(v, f)
    paths = sim.trace(scene, radar, grid, max_bounces)
    cube = sim.synthesize(paths, radar)
    pts, st = sim.pointcloud(cube, radar, cfar)
    n = st.n_points()
    out = pts[: max(n, 1)].cpu().numpy()
    if n == 0:
        out = np.zeros((1, 4), np.float32)
        out[0, 2], out[0, 3] = 1.0, 1.0
    return out


def run_sequential(items, radar, cfar):
    """The same requests one at a time through the plain simulator (no batching, no
    caches, synchronous); returns per-request service times [ms]."""
    from .recon import Reconstruction
    times = []
    for it in items:
        torch.cuda.synchronize()
        t = time.perf_counter()
        if it["kind"] == FORWARD:
            plain_forward(it["verts"], it["faces"], radar, cfar, it["grid"], it["max_bounces"])
        else:
            tgt = torch.from_numpy(np.ascontiguousarray(it["target"], np.float32)).cuda()
            rec = Reconstruction(it["verts"], it["faces"], tgt, radar, it["grid"], it["max_bounces"], cfar,
                                 lr=it["lr"], lap_weight=it["lap_weight"])
            for _ in range(it["iterations"]):
                rec.step()
            rec.loss.item()
        torch.cuda.synchronize()
        times.append(1e3 * (time.perf_counter() - t))
    return times
