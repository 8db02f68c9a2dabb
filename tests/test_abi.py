"""CPU checks of the C ABI: the library builds, loads and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "sbr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sbr_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_13182_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = header_symbols()
    for s in ("sbr_trace", "sbr_synthesize", "sbr_pointcloud", "sbr_synthesize_bwd", "sbr_pointcloud_bwd",
              "sbr_trace_bwd", "sbr_scene_create"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in header_symbols() if not hasattr(lib, s)]
    assert not missing, f"declared in sbr.h but not exported: {missing}"


def test_binding_signatures_cover_header(lib):
    from paper_2311_13182_gb300 import _lib
    assert set(header_symbols()) <= set(_lib.declared_symbols())


def test_size_queries_and_host_side_errors(lib):
    from paper_2311_13182_gb300 import _lib
    L = _lib.load()
    assert L.sbr_scene_bytes(320) > 320 * 48
    assert L.sbr_paths_bytes(4096, 2, 4) > 4096 * 2 * 4 * 16
    assert L.sbr_paths_bytes(10, 0, 4) == 0
    assert L.sbr_version().startswith(b"libsbr")
    # argument errors are reported before any device work: no GPU needed
    st = L.sbr_scene_create(None, 0, None, 5, None, 0, None, ctypes.byref(ctypes.c_void_p()))
    assert st == 1 and "NULL" in _lib.last_error()
    p = _lib.Paths()
    st = L.sbr_paths_bind(ctypes.c_void_p(256), 10, 16, 2, 4, ctypes.byref(p))
    assert st == 2          # region too small -> SBR_ERR_OOM
    st = L.sbr_paths_bind(ctypes.c_void_p(100), 1 << 30, 16, 2, 4, ctypes.byref(p))
    assert st == 1          # misaligned
    r = _lib.RadarCfg()
    r.n_tx, r.n_rx, r.n_samples, r.n_chirps, r.f0, r.bandwidth, r.chirp_time = 1, 4, 100, 1, 77e9, 4e9, 4e-5
    st = L.sbr_trace(ctypes.c_void_p(8), ctypes.byref(r), ctypes.byref(_lib.RayGrid()), None, 0, 2,
                     ctypes.byref(p), None)
    assert st == 1 and "n_samples" in _lib.last_error()


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2311_13182_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_every_status_code_has_a_name():
    """Each sbr_status value the header declares has a name in the binding's error messages."""
    from paper_2311_13182_gb300 import _lib
    txt = open(os.path.join(ROOT, "include", "sbr.h")).read()
    codes = {int(v): n for n, v in re.findall(r"\b(SBR_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", txt)}
    assert codes and all(_lib.STATUS.get(v) == n for v, n in codes.items()), (codes, _lib.STATUS)


def test_pointcloud_config_validation(lib):
    """Angle-row limits of the point-cloud configuration are checked on the host: n_elev a power of
    two (0 reads as 1), n_elev * n_theta <= 256 and n_elev * n_theta * V <= 4096."""
    from paper_2311_13182_gb300 import _lib
    L = _lib.load()
    r = _lib.RadarCfg()
    r.n_tx, r.n_rx, r.n_samples, r.n_chirps, r.f0, r.bandwidth, r.chirp_time = 3, 4, 256, 4, 77e9, 4e9, 4e-5
    r.chirp_rep = 4e-5

    def size(n_theta, n_elev):
        c = _lib.CfarCfg()
        c.n_theta, c.guard, c.train, c.k_max, c.alpha, c.floor_rel, c.beta, c.w_min = n_theta, 2, 8, 100, 16., 1e-4, .5, .01
        c.n_elev = n_elev
        return L.sbr_pc_bytes(ctypes.byref(r), ctypes.byref(c))

    base = size(64, 0)
    assert base > 0 and size(64, 1) == base
    assert size(64, 4) > size(64, 2) > base          # the map and its scratch grow with the rows
    assert size(64, 3) == 0 and "n_elev" in _lib.last_error()
    assert size(64, 8) == 0 and "256" in _lib.last_error()   # 512 rows
    assert size(256, 2) == 0                                  # 512 rows
    r.n_tx, r.n_rx = 4, 8                                     # V = 32: 256 rows x 32 > 4096
    assert size(32, 8) == 0 and "4096" in _lib.last_error()
