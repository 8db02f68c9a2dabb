"""ctypes binding of libsbr (include/sbr.h): structs, signatures, status checks.

Argument marshalling only.  Loading fails loudly when the compiled library is
missing; there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_i32, c_i64, c_f32, c_f64, c_sz, c_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double,
                                          ctypes.c_size_t, ctypes.c_void_p)

MAX_TX = 16
MAX_RX = 16
MAX_VIRT = 64

PHASE_SPLIT, PHASE_FP64, PHASE_NAIVE = 0, 1, 2
STATUS = {0: "SBR_OK", 1: "SBR_ERR_INVALID_ARG", 2: "SBR_ERR_OOM", 3: "SBR_ERR_TIMEOUT", 4: "SBR_ERR_CUDA",
          5: "SBR_ERR_UNSUPPORTED", 6: "SBR_ERR_CANCELLED"}


class SbrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class RadarCfg(ctypes.Structure):
    _fields_ = [("f0", c_f64), ("bandwidth", c_f64), ("chirp_time", c_f64), ("chirp_rep", c_f64),
                ("n_samples", c_i32), ("n_chirps", c_i32), ("n_tx", c_i32), ("n_rx", c_i32),
                ("tx", (c_f64 * 3) * MAX_TX), ("rx", (c_f64 * 3) * MAX_RX)]


class RayGrid(ctypes.Structure):
    _fields_ = [("G", c_i32), ("_pad", c_i32), ("origin", c_f64 * 3), ("axis", c_f64 * 3),
                ("u_axis", c_f64 * 3), ("v_axis", c_f64 * 3), ("tan_half", c_f64), ("jitter", c_p)]


class CfarCfg(ctypes.Structure):
    _fields_ = [("n_theta", c_i32), ("guard", c_i32), ("train", c_i32), ("k_max", c_i32),
                ("alpha", c_f32), ("floor_rel", c_f32), ("beta", c_f32), ("w_min", c_f32),
                ("n_elev", c_i32), ("_pad", c_i32)]


class Paths(ctypes.Structure):
    _fields_ = [("n_rays", c_i32), ("max_bounces", c_i32), ("n_virt", c_i32), ("_pad", c_i32),
                ("path_cap", c_i64), ("hits", c_p), ("hit_pos", c_p), ("ray_weight", c_p),
                ("ray_first", c_p), ("path_ray", c_p), ("prep", c_p), ("path_len", c_p), ("count", c_p),
                ("scratch", c_p), ("phase_ofs", c_p), ("path_rate", c_p)]


MAX_MATERIALS = 16
MAX_OBJECTS = 16
SYNTH_MOVING = 0x100
BWD_REPARAM = 0x1


class Motion(ctypes.Structure):
    _fields_ = [("n_objects", c_i32), ("_pad", c_i32), ("tri_object", c_p), ("velocity", (c_f32 * 3) * MAX_OBJECTS)]


class Materials(ctypes.Structure):
    _fields_ = [("n_materials", c_i32), ("_pad", c_i32), ("tri_material", c_p),
                ("eps_re", c_f32 * MAX_MATERIALS), ("eps_im", c_f32 * MAX_MATERIALS)]


class PcState(ctypes.Structure):
    _fields_ = [("n_virt", c_i32), ("n_chirps", c_i32), ("n_samples", c_i32), ("n_theta", c_i32),
                ("k_max", c_i32), ("n_elev", c_i32), ("spec", c_p), ("power", c_p), ("peak_cell", c_p),
                ("n_points", c_p), ("argmax", c_p), ("scratch", c_p)]


class Request(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("max_bounces", c_i32), ("mesh_id", ctypes.c_uint64), ("verts", c_p),
                ("faces", c_p), ("nv", c_i32), ("nt", c_i32), ("grid", RayGrid), ("iterations", c_i32),
                ("n_target", c_i32), ("target", c_p), ("lr", c_f32), ("lap_weight", c_f32), ("out_points", c_p),
                ("out_verts", c_p)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", c_i64), ("status", c_i32), ("n_points", c_i32), ("scene_cached", c_i32),
                ("cube_cached", c_i32), ("loss", c_f32), ("gpu_ms", c_f32), ("t_submit_us", c_f64),
                ("t_admit_us", c_f64), ("t_done_us", c_f64), ("footprint", ctypes.c_uint64),
                ("gpu_t0_ms", c_f64), ("gpu_t1_ms", c_f64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("used_bytes", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("cached_bytes", ctypes.c_uint64), ("waiting", c_i32), ("running", c_i32),
                ("cached_scenes", c_i32), ("cached_cubes", c_i32), ("submitted", c_i64), ("completed", c_i64),
                ("cache_hits", c_i64)]


P = ctypes.POINTER
_SIGS = {
    "sbr_server_request_bytes": (c_sz, [P(RadarCfg), P(CfarCfg), P(Request)]),
    "sbr_server_create": (c_i32, [c_p, c_sz, c_i32, P(RadarCfg), P(CfarCfg), P(c_p)]),
    "sbr_server_submit": (c_i32, [c_p, P(Request), P(c_i64)]),
    "sbr_server_cancel": (c_i32, [c_p, c_i64]),
    "sbr_server_poll": (c_i32, [c_p, P(Completion), c_i32, P(c_i32)]),
    "sbr_server_get_stats": (c_i32, [c_p, P(ServerStats)]),
    "sbr_server_destroy": (None, [c_p]),
    "sbr_arena_create": (c_p, [c_sz]),
    "sbr_arena_alloc": (c_i64, [c_p, c_sz]),
    "sbr_arena_free": (None, [c_p, c_i64, c_sz]),
    "sbr_arena_used": (c_sz, [c_p]),
    "sbr_arena_peak": (c_sz, [c_p]),
    "sbr_arena_largest_free": (c_sz, [c_p]),
    "sbr_arena_destroy": (None, [c_p]),
    "sbr_version": (ctypes.c_char_p, []),
    "sbr_last_error": (None, [ctypes.c_char_p, c_sz]),
    "sbr_launch_count": (ctypes.c_uint64, []),
    "sbr_scene_bytes": (c_sz, [c_i32]),
    "sbr_scene_create": (c_i32, [c_p, c_i32, c_p, c_i32, c_p, c_sz, c_p, P(c_p)]),
    "sbr_scene_update": (c_i32, [c_p, c_p, c_p]),
    "sbr_scene_refit": (c_i32, [c_p, c_p, c_p]),
    "sbr_scene_check": (c_i32, [c_p, c_p]),
    "sbr_scene_destroy": (None, [c_p]),
    "sbr_paths_bytes": (c_sz, [c_i32, c_i32, c_i32]),
    "sbr_paths_bind": (c_i32, [c_p, c_sz, c_i32, c_i32, c_i32, P(Paths)]),
    "sbr_trace": (c_i32, [c_p, P(RadarCfg), P(RayGrid), c_p, c_i32, c_i32, P(Paths), c_p]),
    "sbr_trace_counts": (c_i32, [c_p, P(RadarCfg), P(RayGrid), c_p, c_i32, c_i32, P(Paths), c_p, c_p]),
    "sbr_synth_ws_bytes": (c_sz, [P(RadarCfg), c_i64]),
    "sbr_synthesize": (c_i32, [P(Paths), P(RadarCfg), c_i32, c_p, c_p, c_sz, c_p]),
    "sbr_synthesize_bwd": (c_i32, [P(Paths), P(RadarCfg), c_p, c_p, c_p, c_p, c_p, c_sz, c_p]),
    "sbr_scene_set_materials": (c_i32, [c_p, P(Materials)]),
    "sbr_scene_set_motion": (c_i32, [c_p, P(Motion)]),
    "sbr_synthesize_noalloc": (c_i32, [P(Paths), P(RadarCfg), c_i32, c_p, c_p]),
    "sbr_pc_bytes": (c_sz, [P(RadarCfg), P(CfarCfg)]),
    "sbr_pc_bind": (c_i32, [c_p, c_sz, P(RadarCfg), P(CfarCfg), P(PcState)]),
    "sbr_pointcloud": (c_i32, [c_p, P(RadarCfg), P(CfarCfg), c_p, P(PcState), c_p]),
    "sbr_pointcloud_bwd": (c_i32, [P(RadarCfg), P(CfarCfg), P(PcState), c_p, c_p, c_p]),
    "sbr_pc_check": (c_i32, [P(RadarCfg), P(CfarCfg), P(PcState), c_p]),
    "sbr_power_map": (c_i32, [c_p, P(RadarCfg), P(CfarCfg), P(PcState), c_p]),
    "sbr_image_loss": (c_i32, [P(RadarCfg), P(CfarCfg), P(PcState), c_p, c_p, c_p, c_p]),
    "sbr_trace_bwd_ws_bytes": (c_sz, [c_i32]),
    "sbr_trace_bwd": (c_i32, [c_p, c_p, P(RadarCfg), P(RayGrid), c_p, P(Paths), c_p, c_p, c_p, c_p, c_p, c_i32, c_p,
                              c_sz, c_p]),
    "sbr_chamfer": (c_i32, [c_p, c_p, c_i32, c_p, c_i32, c_p, c_p, c_p]),
    "sbr_mesh_adjacency": (c_i32, [c_p, c_i32, c_i32, c_p, c_p, c_i32, P(c_i32)]),
    "sbr_laplacian_ws_bytes": (c_sz, [c_i32]),
    "sbr_laplacian": (c_i32, [c_p, c_i32, c_p, c_p, c_f32, c_p, c_p, c_p, c_sz, c_p]),
    "sbr_adam_step": (c_i32, [c_p, c_p, c_p, c_p, c_i64, c_p, c_f32, c_f32, c_f32, c_f32, c_p]),
}

_LIB = None
_LOCK = threading.Lock()


def declared_symbols():
    return list(_SIGS)


def load(path: str | None = None):
    """Load the compiled library (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = path or _build.lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libsbr is not built ({path} missing): run paper_2311_13182_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
        return lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    load().sbr_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(status: int, what: str = ""):
    if status != 0:
        raise SbrError(status, f"{what}: {last_error()}" if what else last_error())


def call(name: str, *args):
    fn = getattr(load(), name)
    st = fn(*args)
    if fn.restype is c_i32:
        check(st, name)
    return st
