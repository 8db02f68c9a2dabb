"""sbr_synthesize_noalloc: the synthesis entry point for callers that cannot allocate device
memory (its partial sums live in a fixed 1 MiB device array instead of a caller workspace).

Collected last on purpose, so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from sbr_inputs import radar_mimo_3x4, ray_subset, sphere_scene, superquadric_scene
from tests._util import cube_complex, gpu_trace, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the IF-cube tolerance of the synthesis parity tests


def noalloc(sbr, paths, radar, mode, out):
    from paper_2311_13182_gb300 import _lib, sim
    r = sim.radar_struct(radar)
    st = _lib.load().sbr_synthesize_noalloc(ctypes.byref(paths.s), ctypes.byref(r), int(mode),
                                            ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("scene", ["sphere", "superquadric"])
def test_noalloc_matches_workspace_entry_point_twice(sbr, scene):
    if scene == "sphere":
        wl, ids = sphere_scene(), None
    else:
        wl = superquadric_scene(seed=6, G=1024)
        ids = ray_subset(8, wl.grid.n_rays, 65536)
    _, paths = gpu_trace(sbr, wl, ray_ids=ids)
    for mode in (sbr.PHASE_SPLIT, sbr.PHASE_FP64):
        ref = cube_complex(sbr.synthesize(paths, wl.radar, mode))
        out = torch.empty((wl.radar.n_virt, wl.radar.n_chirps, wl.radar.n_samples, 2), device="cuda")
        for call in range(2):            # the shared scratch keeps the previous call's contents
            out.fill_(float("nan"))
            assert noalloc(sbr, paths, wl.radar, mode, out) == 0
            torch.cuda.synchronize()
            got = cube_complex(out)
            assert np.isfinite(got).all()
            assert rel_l2(got, ref) <= TOL, (scene, mode, call)


def test_noalloc_rejects_oversized_cube(sbr):
    from paper_2311_13182_gb300 import _lib
    radar = radar_mimo_3x4(4096, 1)
    radar.tx = np.zeros((8, 3))
    radar.rx = np.zeros((8, 3))              # 64 virtual antennas x 4096 samples > 131072
    wl = sphere_scene(G=4)
    paths = sbr.PathBuffers(16, 1, 64)
    out = torch.empty((64, 1, 4096, 2), device="cuda")
    st = noalloc(sbr, paths, radar, sbr.PHASE_SPLIT, out)
    assert st == 5 and "131072" in _lib.last_error()


@pytest.mark.parametrize("mode", ["split", "fp64", "naive"])
def test_noalloc_partial_cap_all_modes(sbr, mode):
    """12 virtual antennas x 1024 samples: one partial cube is 12288 values, so the fixed
    array holds at most 10 CTAs per antenna, while the workspace entry point launches at
    least one CTA per SM over the 12 antennas (152 / 12 > 10) whenever the paths fill more
    than 10 chunks of 512: the allocation-free call runs with its grid cut to the array's
    size, its CTAs looping over more path chunks each, in every phase mode."""
    wl = superquadric_scene(seed=3, G=512, n_chirps=1, n_samples=1024)
    _, paths = gpu_trace(sbr, wl)
    V, Ns = wl.radar.n_virt, wl.radar.n_samples
    qmax = 131072 // (V * Ns)
    assert qmax == 10 and 152 // V > qmax
    assert paths.count() > 4 * qmax * 512            # several chunks per capped CTA
    m = dict(split=sbr.PHASE_SPLIT, fp64=sbr.PHASE_FP64, naive=sbr.PHASE_NAIVE)[mode]
    ref = cube_complex(sbr.synthesize(paths, wl.radar, m))
    out = torch.empty((V, 1, Ns, 2), device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        assert noalloc(sbr, paths, wl.radar, m, out) == 0
        torch.cuda.synchronize()
        got = cube_complex(out)
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL, (mode, call)
