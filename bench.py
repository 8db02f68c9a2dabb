#!/usr/bin/env python3
"""Benchmark of the SBR radar simulator hot path on GB300.

One step = one pass of the forward hot path over the 3 Tx x 4 Rx MIMO workload:
mesh pack + LBVH build of a 20,002-triangle scene (seeded superquadric over a
ground plane), the trace of 1024 x 1024 rays with up to 3 specular bounces and
float-float path preparation, the synthesis of the [12, 128, 256] IF cube (Eq. 8),
and the point cloud (range FFT, Doppler FFT, angle DFT, soft CFAR, refine).
Steps are timed four batches deep (sbr.PipelinedForward: the next batch's
build, the previous batch's synthesis and an earlier batch's point cloud beside
this batch's trace, every stage once per step); the serial step (one batch end
to end per replay) is timed and printed beside it.

Printed (rank 0, one JSON line): traced rays/s over all ranks (device-timed,
inputs resident), the same end to end through the public API with host
buffers (`e2e`), path-samples/s, reconstruction iterations/s (2562-vertex
template against a superquadric's point cloud, one CUDA-graph replay per
iteration), the roofline of the dominant kernel against MEASURED_PEAKS.json,
SM clocks sampled during the timed region, and the FP64 CPU oracle timed on a
bounded sample on this host (`cpu_baseline`).

``--impl reference`` times the FP64 CPU oracle itself (the only reference this
method has) on the same workload and prints its line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "traced rays/s & path-samples/s; recon iters/s; p50/p99 request ms"
WORKLOAD = ("superquadric 20,000 tris + 4x4 m ground (2 tris), seed 0; 1024x1024 rays, <=3 specular bounces; "
            "77 GHz 3Tx x 4Rx (12 virtual), 128 chirps x 256 samples; range FFT, Doppler FFT, 64-bin angle DFT, "
            "soft CA-CFAR -> <=2000 points")
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-recon", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the long-range precision sweep")
    ap.add_argument("--no-moving", action="store_true", help="skip the moving-scene (per-chirp) measurement")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--write-counters", metavar="NCU_CSV", nargs="+",
                    help="write profiles/counters.json from ncu --csv logs (one capture per kernel) of "
                         "dram__bytes_read.sum, dram__bytes_write.sum and smsp__inst_executed.sum, then exit")
    return ap.parse_args()


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend, init_method="env://")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.15)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def gpu_arm(args, rank, world, local):
    import torch
    import paper_2311_13182_gb300 as sbr
    from sbr_inputs import CfarParams, superquadric_scene

    sbr.build.build()
    L = sbr.load()
    torch.cuda.set_device(local)
    wl = superquadric_scene(seed=args.seed + rank, G=1024)
    cfg = CfarParams()
    # the step as one CUDA graph (sbr.Forward): capture, then replays
    fw = sbr.Forward(torch.from_numpy(wl.verts).cuda(), torch.from_numpy(wl.faces).cuda(), wl.radar, wl.grid,
                     wl.max_bounces, cfg)
    b = {"scene": fw.scene, "paths": fw.paths, "state": fw.state}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    mk = lambda: torch.cuda.Event(enable_timing=True)
    # per-stage breakdown: the same step as separate launches, events between the stages
    evs = [[mk() for _ in range(5)] for _ in range(args.steps)]
    for _ in range(3):
        fw.run_eager()
    launches0 = int(L.sbr_launch_count())
    fw.run_eager()
    per_step_launches = int(L.sbr_launch_count()) - launches0  # = the kernels in the graph
    for i in range(args.steps):
        flush.fill_(float(i))
        fw.run_eager(evs[i])
    torch.cuda.synchronize()
    stage = np.array([[evs[i][j].elapsed_time(evs[i][j + 1]) for j in range(4)] for i in range(args.steps)])
    for _ in range(max(args.warmup, 3)):
        fw.run()
    torch.cuda.synchronize()
    P = b["paths"].count()
    n_points = b["state"].n_points()
    # one batch end to end per replay (the serial step's latency), L2 flushed between steps
    ev = [(mk(), mk()) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        fw.run()
        ev[i][1].record()
    torch.cuda.synchronize()
    ms_serial = reduce_max(float(np.mean([a.elapsed_time(e) for a, e in ev])), world)
    # the step four batches deep (sbr.PipelinedForward): the next batch's build, the previous
    # batch's synthesis and an earlier batch's point cloud beside this batch's trace
    pf = sbr.PipelinedForward(torch.from_numpy(wl.verts).cuda(), torch.from_numpy(wl.faces).cuda(), wl.radar,
                              wl.grid, wl.max_bounces, cfg)
    for _ in range(max(args.warmup, 3)):
        pf.run()
    torch.cuda.synchronize()

    # ---- device-timed region: graph replays, inputs resident, L2 flushed between steps
    ev = [(mk(), mk()) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        pf.run()
        ev[i][1].record()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = per_step_launches * args.steps
    barrier(world)
    clk = clocks.stop()
    ms_step = float(np.mean([a.elapsed_time(e) for a, e in ev]))
    ms_step_all = reduce_max(ms_step, world)
    if pf.n_points() != n_points:
        raise RuntimeError(f"pipelined step found {pf.n_points()} points, the serial step {n_points}")
    del pf
    rays = wl.grid.n_rays
    value = reduce_sum(rays, world) / (ms_step_all * 1e-3)
    samples = P * wl.radar.n_virt * wl.radar.n_samples
    path_samples = reduce_sum(samples, world) / (ms_step_all * 1e-3)
    stage_ms = dict(zip(["scene_build", "trace", "synthesize", "pointcloud"], stage.mean(0).round(4).tolist()))

    # ---- end to end through the public API with host buffers
    e2e = e2e_arm(sbr, torch, wl, cfg, args, world, flush)

    # ---- rooflines (work counters from one counting trace, outside the timed region)
    from paper_2311_13182_gb300 import sim as _sim
    counts = _sim.trace_counts(b["scene"], wl.radar, wl.grid, wl.max_bounces, out=b["paths"])
    peaks, src = measured_peaks()
    roof, roofs = rooflines(stage_ms, wl, P, counts, peaks, src)

    recon = None if args.no_recon else recon_arm(sbr, torch, args)
    sweep = None if args.no_sweep else precision_sweep_arm(sbr, torch, args)
    moving = None if args.no_moving else moving_arm(sbr, torch, args)
    serve = None if args.no_serve else serve_arm(sbr, torch, args)
    out = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_step_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (float-float ray refine, delays and phase reduction)",
        "data": "synthetic (seeded superquadric + ground; no datasets)",
        "config": {"workload": WORKLOAD, "rays_per_step": rays, "paths_per_step": P, "points": n_points,
                   "parallelism": f"replicas x{world} (independent scenes per GPU, no collective)",
                   "l2": f"{L2_FLUSH_BYTES >> 20} MiB buffer written between steps, outside the per-step events",
                   "timing": "each step one CUDA-graph replay of sbr.PipelinedForward (depth 4): this batch's "
                             "trace, the previous batch's synthesis, the next batch's LBVH build and the point "
                             "cloud of the batch before the previous on four streams (every stage once per "
                             "step); serial = one batch end to end per replay (sbr.Forward); stage_ms from the "
                             "serial step as separate launches with events between the stages"},
        "serial": {"ms_per_step": ms_serial, "rays_per_s": reduce_sum(rays, world) / (ms_serial * 1e-3)},
        "path_samples_per_s": path_samples,
        "stage_ms": stage_ms,
        "recon_iters_per_s": None if recon is None else recon["iters_per_s"],
        "recon": recon,
        "serving": serve,
        "precision_sweep": sweep,
        "moving": moving,
        "e2e": e2e,
        "gpu_launches": launches,
        "wall_s_timed_region": t_wall,
        "roofline": roof,
        "rooflines": roofs,
        "clocks": clk,
    }
    return out


def e2e_arm(sbr, torch, wl, cfg, args, world, flush):
    """Same step through the public API from page-locked host buffers: sbr.PipelinedForward with
    host_io, whose graphs copy the vertex positions host-to-device for the batch they build (the
    topology fixed at construction), build, trace, synthesise and extract points (four batches in
    flight), and copy the points and their count device-to-host; one run_host call per step, L2
    flushed between steps outside the per-step events as in the device-timed arm."""
    fwd = sbr.PipelinedForward(torch.from_numpy(wl.verts).cuda(), torch.from_numpy(wl.faces).cuda(), wl.radar,
                               wl.grid, wl.max_bounces, cfg, host_io=True)
    for _ in range(3):
        fwd.run_host(wl.verts)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        fwd.run_host()
        ev[i][1].record()
    torch.cuda.synchronize()
    ms = reduce_max(float(np.mean([a.elapsed_time(b) for a, b in ev])), world)
    bi = fwd.h_verts.numel() * 4
    bo = fwd.h_points.numel() * 4 + 4
    return {"value": reduce_sum(wl.grid.n_rays, world) / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms,
            "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "path": "sbr.PipelinedForward(host_io=True).run_host: H2D of the vertices, the step, D2H of the "
                    "points, one CUDA graph per step"}


# Counters per launch of each roofline stage (DRAM bytes, warp instructions), from ncu captures
# of one kernel each (profiles/counters.json); used only while the library sources still hash to
# what was captured.  Each kernel runs once per stage call.
COUNTER_STAGES = {
    "trace": ("k_trace", "k_trace_coop", "k_tile_sums", "k_scan_single", "k_tile_scan", "k_scan_small", "k_prep"),
    "synthesize": ("k_nufft_spread", "k_nufft_finish", "k_reduce"),
    "pointcloud": ("k_fft_rows", "k_fft_cols", "k_angle_power", "k_angle_tc", "k_power_reduce", "k_detect",
                   "k_select"),
}

# the sources each stage's kernels are compiled from
COUNTER_SOURCES = {
    "trace": ("trace.cu", "scan_sort.cu", "cta_sort.cuh", "scene.cuh", "ff.cuh", "common.cuh"),
    "synthesize": ("synth.cu", "fft.cuh", "common.cuh"),
    "pointcloud": ("pointcloud.cu", "tcgen05.cuh", "fft.cuh", "cta_sort.cuh", "common.cuh"),
}
COUNTERS_FILE = os.path.join("profiles", "counters.json")
COUNTER_METRICS = {"dram__bytes_read.sum": "dram", "dram__bytes_write.sum": "dram", "smsp__inst_executed.sum": "inst"}


def sources_sha1(stage: str) -> str:
    """SHA-1 of the stage's kernel sources and of the C header without its comments (the
    header's declarations and constants reach the kernels; its documentation does not)."""
    import hashlib
    import re
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2311_13182_gb300", "csrc")
    for f in [os.path.join(csrc, n) for n in COUNTER_SOURCES[stage]] + [os.path.join(ROOT, "include", "sbr.h")]:
        if os.path.exists(f):
            with open(f, "rb") as fh:
                data = fh.read()
            if f.endswith(".h"):
                data = re.sub(rb"/\*.*?\*/", b"", data, flags=re.S)
            h.update(os.path.basename(f).encode() + data)
    return h.hexdigest()


def _kernel_name(raw: str) -> str:
    return raw.split("(")[0].split("::")[-1].split("<")[0].replace("void ", "").strip()


def write_counters(csv_paths):
    """Per-launch DRAM bytes and warp instructions of each stage from ncu --csv logs (one capture per
    kernel): per kernel the mean over its captured launches, per stage the sum over its kernels."""
    import csv
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "inst": 1.0, "Kinst": 1e3, "Minst": 1e6,
             "": 1.0}
    per = {}  # kernel -> {launch id -> {"dram": x, "inst": y}}
    for path in csv_paths:
        with open(path) as fh:
            rows = list(csv.reader(fh))
        head = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
        hdr = rows[head]
        ii, ki, mi, vi, ui = (hdr.index("ID"), hdr.index("Kernel Name"), hdr.index("Metric Name"),
                              hdr.index("Metric Value"), hdr.index("Metric Unit"))
        for r in rows[head + 1:]:
            if len(r) <= vi or r[mi] not in COUNTER_METRICS:
                continue
            k = _kernel_name(r[ki])
            launch = per.setdefault(k, {}).setdefault((path, r[ii]), {"dram": 0.0, "inst": 0.0})
            launch[COUNTER_METRICS[r[mi]]] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
    kernels = {k: {"launches": len(v), "dram_bytes": sum(x["dram"] for x in v.values()) / len(v),
                   "inst": sum(x["inst"] for x in v.values()) / len(v)} for k, v in per.items()}
    stages = {}
    for st, names in COUNTER_STAGES.items():
        got = [k for k in names if k in kernels]
        if not got:
            continue
        stages[st] = {"dram_bytes_per_launch": sum(kernels[k]["dram_bytes"] for k in got),
                      "inst_per_launch": sum(kernels[k]["inst"] for k in got),
                      "kernels": got, "sources_sha1": sources_sha1(st)}
    out = {"stages": stages, "kernels": kernels, "from": [os.path.basename(p) for p in csv_paths]}
    with open(os.path.join(ROOT, COUNTERS_FILE), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


def measured_counters() -> dict:
    try:
        with open(os.path.join(ROOT, COUNTERS_FILE)) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return {}
    return {st: v for st, v in d.get("stages", {}).items()
            if st in COUNTER_SOURCES and v.get("sources_sha1") == sources_sha1(st)}


def rooflines(stage_ms, wl, P, counts, peaks, src):
    """Rooflines of the step's two large stages, each against the bound that limits it.

    Both stages are issue-bound (ncu: profiles/k_trace_*, profiles/k_nufft_spread_*), so `frac` is
    issue slots used: warp instructions per call (smsp__inst_executed.sum, profiles/counters.json)
    / (CUDA-event time x 152 SMs x 4 schedulers x f_max).  Beside it:
    trace (sbr_trace = k_trace + k_trace_coop + scan + k_prep, timed together):
      served: the algorithmic bytes of a call (4-wide nodes fetched x 112 B + triangles tested x 48 B,
      both counted by sbr_trace_counts, + 48 B per ray-bounce slot + 8 B per ray + 24 B per (path,
      antenna) + 4 B per path) per second against the HBM copy rate: the working set is L2-resident,
      so these bytes are served mostly by L1/L2 (a bytes-served rate, not DRAM);
      dram: the call's DRAM bytes (ncu) per second against the HBM copy rate.
    synthesis (k_nufft_spread + k_nufft_finish; Eq. 8 as a type-1 non-uniform FFT):
      dram as above; speedup_vs_direct_sum: Eq. 8 terms (path, antenna, sample) per second over the
      FP32-pipe bound of a term-by-term kernel (152 SMs x 128 lanes x f_max / 4 lane-ops per term)."""
    V, Ns = wl.radar.n_virt, wl.radar.n_samples
    R, K = wl.grid.n_rays, wl.max_bounces
    ctr = measured_counters()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    issue_peak = 152 * 4 * mhz * 1e6
    hbm = float(peaks["hbm_gbs"])
    issue_src = f"152 SMs x 4 schedulers x {mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json, {src})"

    def issue(stage, t):
        inst = ctr.get(stage, {}).get("inst_per_launch")
        return (None, None) if inst is None else (inst / t, inst / t / issue_peak)

    def dram(stage, t):
        b = ctr.get(stage, {}).get("dram_bytes_per_launch")
        return {"bytes_per_launch": b, "achieved_gbs": None if b is None else b / t / 1e9,
                "frac_of_hbm": None if b is None else b / t / 1e9 / hbm}

    nodes, tris, trav = counts
    tb = nodes * 112 + tris * 48 + R * K * 48 + R * 8 + P * V * 24 + P * 4
    t_tr = stage_ms["trace"] * 1e-3
    ach, frac = issue("trace", t_tr)
    trace = {"kernel": "k_trace (+ k_trace_coop, scan, k_prep)", "bound": "alu", "limiter": "issue slots",
             "achieved": ach, "peak": issue_peak, "unit": "warp-inst/s", "frac": frac,
             "inst_per_launch": ctr.get("trace", {}).get("inst_per_launch"),
             "traffic": ctr.get("trace", {}).get("dram_bytes_per_launch"),
             "dram": dram("trace", t_tr),
             "served": {"bytes_per_launch": tb, "achieved_gbs": tb / t_tr / 1e9, "frac_of_hbm": tb / t_tr / 1e9 / hbm,
                        "note": "algorithmic bytes (nodes, triangles, records) per second: mostly L1/L2 hits"},
             "units": {"rays": R, "traversals": trav, "nodes": nodes, "triangles": tris, "paths": P},
             "peak_source": issue_src, "hbm_peak_gbs": hbm}
    terms = P * V * Ns
    t_sy = stage_ms["synthesize"] * 1e-3
    ach, frac = issue("synthesize", t_sy)
    fp32_terms = 152 * 128 * mhz * 1e6 / 4
    rec = P * V * 16
    synth = {"kernel": "k_nufft_spread (+ k_nufft_finish)", "bound": "alu", "limiter": "issue slots",
             "achieved": ach, "peak": issue_peak, "unit": "warp-inst/s", "frac": frac,
             "inst_per_launch": ctr.get("synthesize", {}).get("inst_per_launch"),
             "traffic": ctr.get("synthesize", {}).get("dram_bytes_per_launch"),
             "dram": dram("synthesize", t_sy),
             "terms_per_launch": terms, "grid_updates_per_launch": P * V * 8,
             "speedup_vs_direct_sum": {"terms_per_s": terms / t_sy, "direct_sum_bound_terms_per_s": fp32_terms,
                                       "ratio": terms / t_sy / fp32_terms},
             "records": {"bytes_per_launch": rec, "achieved_gbs": rec / t_sy / 1e9, "frac_of_hbm": rec / t_sy / 1e9 / hbm},
             "peak_source": issue_src}
    for r in (trace, synth):
        if r["achieved"] is None:
            # no instruction counts for these sources: report the bytes-served figure in their place
            r.update(bound="hbm", limiter="bytes served (issue counters absent for these sources)",
                     unit="GB/s", peak=hbm, peak_source=f"hbm_gbs of MEASURED_PEAKS.json ({src}, burst copy)")
            if "served" in r:
                r.update(achieved=r["served"]["achieved_gbs"], frac=r["served"]["frac_of_hbm"])
            else:
                r.update(achieved=r["records"]["achieved_gbs"], frac=r["records"]["frac_of_hbm"])
    dom = trace if stage_ms["trace"] >= stage_ms["synthesize"] else synth
    return dom, [trace, synth]


def _chamfer_mm(P, Q):
    """Weighted mean nearest-neighbour distance of point sets (x, y, z, w), both ways, averaged [mm]."""
    if len(P) == 0 or len(Q) == 0:
        return 0.0 if len(P) == len(Q) else float("inf")
    d = np.sqrt(((P[:, None, :3] - Q[None, :, :3]) ** 2).sum(-1))
    a = (P[:, 3] * d.min(1)).sum() / P[:, 3].sum()
    b = (Q[:, 3] * d.min(0)).sum() / Q[:, 3].sum()
    return float(500.0 * (a + b))


def precision_sweep_arm(sbr, torch, args):
    """Long-range precision sweep: the 320-triangle sphere (radius 0.2 m) centred 5, 10 and 20 m
    out, 1024, 2048 and 4096 samples per chirp, 2048 x 2048 rays (4,194,304), up to 2 bounces,
    1 Tx / 4 Rx.  Per (distance, samples) the full trace is timed (rays/s), then the synthesis in
    each carrier-phase mode (path-samples/s = P x V x N_s per call).  Beside each mode: IF-cube
    relative L2 and point-cloud Chamfer against the FP64 oracle on a seeded 4096-ray subset of the
    same grid, the oracle's values read from tests/golden/precision_sweep_subset4096.npz (written
    from the oracle alone by tests/golden/make_golden.py)."""
    from sbr_inputs import CfarParams, ray_subset, sphere_scene
    gold = np.load(os.path.join(ROOT, "tests", "golden", "precision_sweep_subset4096.npz"))
    cfg = CfarParams()
    modes = (("split", sbr.PHASE_SPLIT), ("fp64", sbr.PHASE_FP64), ("naive", sbr.PHASE_NAIVE))
    reps = 3
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    rows = []
    for dist in (5.0, 10.0, 20.0):
        wl0 = sphere_scene(G=2048, distance=dist, n_samples=1024)
        v = torch.from_numpy(wl0.verts).cuda()
        f = torch.from_numpy(wl0.faces).cuda()
        scene = sbr.Scene(v, f)
        paths = sbr.PathBuffers(wl0.grid.n_rays, wl0.max_bounces, wl0.radar.n_virt)
        ids = torch.from_numpy(ray_subset(11, wl0.grid.n_rays, 4096)).cuda()
        sub = sbr.PathBuffers(4096, wl0.max_bounces, wl0.radar.n_virt)
        for ns in (1024, 2048, 4096):
            wl = sphere_scene(G=2048, distance=dist, n_samples=ns)
            t_tr = timed(lambda: sbr.trace(scene, wl.radar, wl.grid, wl.max_bounces, out=paths))
            P = paths.count()
            sbr.trace(scene, wl.radar, wl.grid, wl.max_bounces, ray_ids=ids, out=sub)
            key = f"d{int(dist)}_ns{ns}"
            ref = gold["cube_" + key]
            ref_pts = gold["points_" + key]
            cube = torch.empty((wl.radar.n_virt, 1, ns, 2), device="cuda")
            ws = torch.empty(sbr.synth_ws_bytes(wl.radar, paths.cap), dtype=torch.uint8, device="cuda")
            row = {"distance_m": dist, "n_samples": ns, "rays": wl.grid.n_rays, "paths": P,
                   "trace_ms": t_tr, "rays_per_s": wl.grid.n_rays / (t_tr * 1e-3), "modes": {}}
            for name, m in modes:
                t_sy = timed(lambda: sbr.synthesize(paths, wl.radar, m, out=cube, ws=ws))
                c_sub = sbr.synthesize(sub, wl.radar, m)
                pts, st = sbr.pointcloud(c_sub, wl.radar, cfg)
                got = c_sub.double().cpu().numpy()
                got = got[:, 0, :, 0] + 1j * got[:, 0, :, 1]
                err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
                n = st.n_points()
                ch = _chamfer_mm(pts[:n].cpu().numpy().astype(np.float64), ref_pts)
                row["modes"][name] = {"synth_ms": t_sy,
                                      "path_samples_per_s": P * wl.radar.n_virt * ns / (t_sy * 1e-3),
                                      "cube_rel_l2_vs_oracle": err, "chamfer_mm_vs_oracle": ch}
            rows.append(row)
            del ws
        del paths, sub, scene
        torch.cuda.empty_cache()
    return {"workload": "icosphere 320 tris r 0.2 m at 5/10/20 m; 2048x2048 rays, <=2 bounces; 1 Tx x 4 Rx; "
                        "1024/2048/4096 samples, 1 chirp",
            "timing": f"CUDA events, mean of {reps} calls after one warm-up call, inputs resident",
            "accuracy": "4096 seeded rays of the same grid vs the FP64 oracle's stored cube and points "
                        "(tests/golden/precision_sweep_subset4096.npz)",
            "rows": rows}


def moving_arm(sbr, torch, args):
    """Moving scene: the bench's superquadric (20,000 triangles) receding at 2 m/s along
    boresight and drifting 0.5 m/s sideways over its static ground plane, 1024 x 1024 rays,
    3 Tx x 4 Rx, 128 chirps 40 us apart x 256 samples; every path's dL/dt from the trace,
    then all 128 chirps synthesised from their own delays (split phase).  Path-samples count
    the chirps: P x V x N_s x C per call."""
    from sbr_inputs import superquadric_scene
    wl = superquadric_scene(seed=args.seed, G=1024)
    nt = wl.faces.shape[0]
    tri_obj = np.zeros(nt, np.int32)
    tri_obj[-2:] = 1                                # the ground plane's two triangles
    v = torch.from_numpy(wl.verts).cuda()
    scene = sbr.Scene(v, torch.from_numpy(wl.faces).cuda())
    to = torch.from_numpy(tri_obj).cuda()
    scene.set_motion([(0.5, 0.0, 2.0), (0.0, 0.0, 0.0)], to)
    paths = sbr.PathBuffers(wl.grid.n_rays, wl.max_bounces, wl.radar.n_virt)
    cube = torch.empty((wl.radar.n_virt, wl.radar.n_chirps, wl.radar.n_samples, 2), device="cuda")
    ws = torch.empty(sbr.synth_ws_bytes(wl.radar, paths.cap), dtype=torch.uint8, device="cuda")
    mode = sbr.PHASE_SPLIT | sbr.SYNTH_MOVING
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        sbr.trace(scene, wl.radar, wl.grid, wl.max_bounces, out=paths)
        sbr.synthesize(paths, wl.radar, mode, out=cube, ws=ws)
    torch.cuda.synchronize()
    reps = 5
    a, b, c = ev(), ev(), ev()
    a.record()
    for _ in range(reps):
        sbr.trace(scene, wl.radar, wl.grid, wl.max_bounces, out=paths)
    b.record()
    for _ in range(reps):
        sbr.synthesize(paths, wl.radar, mode, out=cube, ws=ws)
    c.record()
    torch.cuda.synchronize()
    t_tr, t_sy = a.elapsed_time(b) / reps, b.elapsed_time(c) / reps
    P = paths.count()
    C = wl.radar.n_chirps
    samples = P * wl.radar.n_virt * wl.radar.n_samples * C
    return {"workload": "superquadric 20k tris moving (0.5, 0, 2) m/s over a static ground; 1024x1024 rays, "
                        "<=3 bounces; 3Tx x 4Rx, 128 chirps x 256 samples, every chirp synthesised",
            "paths": P, "trace_ms": t_tr, "synth_ms": t_sy, "rays_per_s": wl.grid.n_rays / (t_tr * 1e-3),
            "path_samples_per_s": samples / (t_sy * 1e-3), "synth_ms_per_chirp": t_sy / C,
            "timing": f"CUDA events, mean of {reps} calls after two warm-up calls, inputs resident"}


def recon_arm(sbr, torch, args):
    """Reconstruction iterations/s: 2562-vertex icosphere template fitted to the point cloud of a
    seeded superquadric seen by the 1 Tx / 4 Rx radar (64 x 64 rays, 2 bounces)."""
    from paper_2311_13182_gb300.autograd import Simulator
    from paper_2311_13182_gb300.recon import Reconstruction
    from sbr_inputs import CfarParams, icosphere, radar_single_tx, ray_grid_for_sphere, superquadric

    sv, sf, params = superquadric(seed=5)
    c = np.array(params["center"])
    radar = radar_single_tx(256, 1)
    grid = ray_grid_for_sphere(c, 0.6, 64)
    cfg = CfarParams()
    tsim = Simulator(sf, sv.shape[0], radar, grid, 2, cfg)
    tpts, tn = tsim.forward(torch.from_numpy(sv).cuda())
    target = tpts[: int(tn.item())].clone()
    tv, tf = icosphere(4, 0.2, c)
    rec = Reconstruction(tv, tf, target, radar, grid, 2, cfg, lr=1e-3, lap_weight=0.1)
    for _ in range(3):
        rec.step()
    loss0 = float(rec.loss.item())
    rec.capture()
    torch.cuda.synchronize()
    n = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rec.replay(n)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    return {"iters_per_s": 1e3 / ms, "ms_per_iter": ms, "iterations": n + 4, "loss_first": loss0,
            "loss_last": float(rec.loss.item()), "vertices": int(tv.shape[0]), "rays": grid.n_rays,
            "mode": "CUDA graph of one full iteration (forward, loss, adjoints, Adam); the tree refitted each "
                    "iteration and rebuilt every 50 (rec.rebuild_every)"}


def serve_arm(sbr, torch, args):
    """Serving: a seeded Poisson stream of requests over a pool of 64 meshes (superquadrics and
    perturbed icospheres, 1k-200k triangles log-uniform), ray budgets 64k-4M (log-uniform),
    half forward-only and half 50-iteration reconstructions, 1 Tx / 4 Rx radar, 2 bounces.
    First the same requests run one at a time through the plain simulator (synchronous, no
    caches); the stream rate is then 0.8 x that single-stream capacity.  Latency = completion
    time - arrival time of each request."""
    from paper_2311_13182_gb300 import serving as S
    from sbr_inputs import CfarParams, radar_single_tx, serving_workload
    radar, cfg = radar_single_tx(256, 1), CfarParams()
    meshes, reqs = serving_workload(args.seed + 7, n=args.serve_requests, pool=64)
    items = S.build_items(meshes, reqs, radar, cfg)
    rays = [it["grid"].G ** 2 * (it["iterations"] if it["kind"] == S.RECON else 1) for it in items]
    seq = S.run_sequential(items, radar, cfg)
    capacity = len(items) / (sum(seq) * 1e-3)
    rate = 0.8 * capacity
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(64 << 30, 0.5 * free))
    srv = S.Server(radar, cfg, arena, n_slots=16)
    done, wall, tickets = S.run_stream(srv, items, rate, seed=args.seed + 11)
    stats = srv.stats()
    srv.close()
    ok = [d for d in done if d["status"] == 0]
    lat = [(d["t_done_us"] - d["t_submit_us"]) * 1e-3 for d in ok]
    # one at a time under the same arrivals: a single FIFO server with the measured service times
    arrivals = np.cumsum(np.random.default_rng(args.seed + 11).exponential(1.0 / rate, size=len(items))) * 1e3
    t_free, seq_lat = 0.0, []
    for a, st in zip(arrivals, seq):
        start = max(a, t_free)
        t_free = start + st
        seq_lat.append(t_free - a)
    # capacity of the served system: every request submitted at once
    srv = S.Server(radar, cfg, arena, n_slots=16)
    t0 = time.perf_counter()
    for it in items:
        srv.submit(**it)
    sat = srv.drain(600)
    sat_wall = time.perf_counter() - t0
    srv.close()
    gpu = [d["gpu_ms"] for d in ok]
    out = {"requests": len(items), "completed_ok": len(ok), "rate_hz": rate,
           "rate_rule": "0.8 x one-at-a-time capacity", "capacity_one_at_a_time_hz": capacity,
           "paced": {"wall_s": wall, **S.percentiles(lat),
                     "gpu_ms": {k.replace("_ms", ""): v for k, v in S.percentiles(gpu).items()},
                     "device": S.device_overlap(ok)},
           "one_at_a_time_same_arrivals": S.percentiles(seq_lat),
           "saturated": {"rays_per_s": sum(rays) / sat_wall, "wall_s": sat_wall,
                         "completed_ok": sum(1 for d in sat if d["status"] == 0),
                         "device": S.device_overlap(sat)},
           "one_at_a_time": {"rays_per_s": sum(rays) / (sum(seq) * 1e-3), "wall_s": sum(seq) * 1e-3,
                             "service_p50_ms": float(np.percentile(seq, 50)),
                             "service_p99_ms": float(np.percentile(seq, 99))},
           "cache_hits": stats["cache_hits"], "peak_bytes": stats["peak_bytes"], "arena_bytes": arena,
           "slots": 16, "recon_iterations": 50, "rays_counted": "rays per forward pass x passes"}
    out["p50_ms"], out["p99_ms"] = out["paced"]["p50_ms"], out["paced"]["p99_ms"]
    return out


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(n_rays: int, seed: int):
    """FP64 oracle on a seeded sample of the workload's rays: brute-force trace, paths,
    direct-sum synthesis of the sampled paths, point cloud of that partial cube."""
    import oracle
    from oracle import pointcloud as opc
    from sbr_inputs import superquadric_scene, ray_subset
    wl = superquadric_scene(seed=seed, G=1024)
    ids = ray_subset(1234, wl.grid.n_rays, n_rays)
    t0 = time.perf_counter()
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, wl.max_bounces, ray_ids=ids)
    pa = oracle.paths(tr, wl.radar)
    cube = oracle.synthesize(pa["tau"], pa["amp"], wl.radar)
    opc.pointcloud(cube, wl.radar)
    return time.perf_counter() - t0, pa["P"]


def cpu_baseline(seed: int, budget_s: float = 20.0, single_s: float = 6.0):
    """The oracle on every host core over a ~budget_s sample, and on one core over a ~single_s one."""
    import oracle
    n = 2048
    dt, _ = oracle_sample(n, seed)
    n2 = int(min(1 << 20, max(n, n * budget_s / max(dt, 1e-3))))
    dt2, P = oracle_sample(n2, seed)
    out = {"value": n2 / dt2, "unit": "rays/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{n2} of 1,048,576 rays (seeded subset): brute-force FP64 trace, paths, direct-sum "
                     f"synthesis of their {P} paths x 12 antennas x 256 samples, point cloud; {dt2:.1f} s"}
    prev = oracle.set_threads(1)
    try:
        m = 256
        dt1, _ = oracle_sample(m, seed)
        m2 = int(min(n2, max(m, m * single_s / max(dt1, 1e-3))))
        dt12, P1 = oracle_sample(m2, seed)
    finally:
        oracle.set_threads(prev)
    out["single_thread"] = {"value": m2 / dt12, "unit": "rays/s", "cores": 1,
                            "sample": f"{m2} rays of the same seeded subset order ({P1} paths); {dt12:.1f} s"}
    return out


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    per_step = 1024
    for _ in range(max(args.warmup, 3)):
        oracle_sample(256, args.seed)
    times = []
    for _ in range(args.steps):
        dt, _ = oracle_sample(per_step, args.seed)
        times.append(dt)
    ms = 1e3 * float(np.mean(times))
    val = per_step / (ms * 1e-3)
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "rays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_rays_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": "rays/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{per_step} seeded rays of the 1024x1024 grid per step"},
            "e2e": {"value": val, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.write_counters:
        write_counters(args.write_counters)
        return
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        out = reference_arm(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    # CPU baseline first (forking a pool after CUDA init is unsafe; the oracle uses OpenMP threads)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu = cpu_baseline(args.seed)
    out = gpu_arm(args, rank, world, local)
    if rank == 0:
        out["cpu_baseline"] = cpu
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
