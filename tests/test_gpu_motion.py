"""Moving objects on the GPU (the scene dynamics of Section 3.1): every path's dL/dt, the
per-chirp IF cube and its Doppler spectrum against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from oracle import pointcloud as opc
from sbr_inputs import C_LIGHT, CfarParams, radar_mimo_3x4, sphere_scene
from tests._util import cube_complex, rel_l2

pytestmark = pytest.mark.gpu


def moving_workload(n_chirps=8, v_los=None):
    """The 320-triangle sphere seen by the 3 Tx x 4 Rx radar, its two halves (alternate
    triangles) moving differently; chirps 50 us apart."""
    wl = sphere_scene(G=48)
    radar = radar_mimo_3x4(256, n_chirps)
    radar.chirp_rep = 50e-6
    wl = dataclasses.replace(wl, radar=radar)
    tri_obj = (np.arange(wl.faces.shape[0]) % 2).astype(np.int32)
    if v_los is None:
        vel = np.array([[0.4, -0.3, 2.5], [-0.2, 0.1, -1.5]])
    else:
        vel = np.array([[0.0, 0.0, v_los], [0.0, 0.0, v_los]])
    return wl, tri_obj, vel


def gpu_moving_paths(sbr, wl, tri_obj, vel):
    v = torch.from_numpy(wl.verts).cuda()
    f = torch.from_numpy(wl.faces).cuda()
    scene = sbr.Scene(v, f)
    to = torch.from_numpy(tri_obj).cuda()
    scene.set_motion(vel, to)
    paths = sbr.trace(scene, wl.radar, wl.grid, wl.max_bounces)
    torch.cuda.synchronize()
    return scene, paths, to


def test_path_rates_and_moving_cube(sbr):
    wl, tri_obj, vel = moving_workload()
    ref, tr, pa = oracle.simulate_cube(wl, motion=(tri_obj, vel))
    scene, paths, _ = gpu_moving_paths(sbr, wl, tri_obj, vel)
    P = paths.count()
    assert P == pa["P"] and (paths.hits()[0].cpu().numpy() == tr["tri"]).all()
    rate = paths.path_rate().cpu().numpy()[:, :P].astype(np.float64)
    np.testing.assert_allclose(rate, pa["rate"], rtol=0, atol=2e-6 * np.abs(pa["rate"]).max())
    for name, mode in (("split", sbr.PHASE_SPLIT), ("fp64", sbr.PHASE_FP64)):
        cube = cube_complex(sbr.synthesize(paths, wl.radar, mode | sbr.SYNTH_MOVING))
        assert cube.shape == ref.shape
        assert rel_l2(cube, ref) <= 1e-4, name
    # the chirps really differ (path lengths change by up to ~0.25 mm per chirp, 0.06 wavelength)
    assert rel_l2(ref[:, -1], ref[:, 0]) > 0.1
    with pytest.raises(sbr.SbrError):
        sbr.synthesize(paths, wl.radar, sbr.PHASE_NAIVE | sbr.SYNTH_MOVING)


def test_moving_doppler_spectrum(sbr):
    """A sphere receding along boresight: the Doppler spectrum of its strongest range bin peaks
    in the same bin as the oracle's (near 2 v (f_c + B/2) T_rep C / c = 5)."""
    radar_probe = radar_mimo_3x4(256, 32)
    v = 5 * C_LIGHT / (2 * (radar_probe.f0 + radar_probe.bandwidth / 2) * 50e-6 * 32)
    wl, tri_obj, vel = moving_workload(n_chirps=32, v_los=v)
    ref, _, _ = oracle.simulate_cube(wl, motion=(tri_obj, vel))
    _, paths, _ = gpu_moving_paths(sbr, wl, tri_obj, vel)
    cube = sbr.synthesize(paths, wl.radar, sbr.PHASE_SPLIT | sbr.SYNTH_MOVING)
    st = sbr.power_map(cube, wl.radar, CfarParams())
    X = st.spectrum().double().cpu().numpy()
    X = X[..., 0] + 1j * X[..., 1]                    # [V, C, N_s] after range and Doppler FFTs
    Xo = opc.dft(opc.dft(ref, axis=2), axis=1)
    k = int(np.argmax(np.abs(Xo).sum(axis=(0, 1))))
    dop_gpu = int(np.argmax(np.abs(X[:, :, k]).sum(axis=0)))
    dop_ref = int(np.argmax(np.abs(Xo[:, :, k]).sum(axis=0)))
    assert dop_gpu == dop_ref and abs(dop_ref - 5) <= 1
    assert rel_l2(X, Xo) <= 1e-4


def test_zero_velocity_equals_static(sbr):
    wl, tri_obj, _ = moving_workload()
    _, paths, _ = gpu_moving_paths(sbr, wl, tri_obj, np.zeros((2, 3)))
    moving = sbr.synthesize(paths, wl.radar, sbr.PHASE_SPLIT | sbr.SYNTH_MOVING)
    static = sbr.synthesize(paths, wl.radar, sbr.PHASE_SPLIT)
    assert rel_l2(cube_complex(moving), cube_complex(static)) <= 1e-6
