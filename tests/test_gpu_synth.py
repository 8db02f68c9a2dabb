"""GPU synthesis parity: IF cube relative L2 <= 1e-4 against the FP64 oracle (Eq. 8), and the
Eq. 11-12 adjoint against the oracle's FP64 adjoint."""
import numpy as np
import pytest
import torch

import oracle
from sbr_inputs import C_LIGHT, ray_subset, sphere_scene, superquadric_scene
from tests._util import cube_complex, gpu_trace, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-4


def oracle_cube(wl, ids=None):
    cube, tr, pa = oracle.simulate_cube(wl, ids)
    return cube, tr, pa


@pytest.mark.parametrize("mode", ["split", "fp64"])
def test_sphere_cube(sbr, mode):
    wl = sphere_scene()
    ref, _, _ = oracle_cube(wl)
    _, paths = gpu_trace(sbr, wl)
    m = dict(split=sbr.PHASE_SPLIT, fp64=sbr.PHASE_FP64)[mode]
    cube = cube_complex(sbr.synthesize(paths, wl.radar, m))
    assert rel_l2(cube, ref) <= TOL


def test_superquadric_mimo_cube_subset(sbr):
    """12 virtual antennas x 128 chirps x 256 samples on a seeded 1/64 ray subset of G=1024."""
    wl = superquadric_scene(seed=2, G=1024)
    ids = ray_subset(7, wl.grid.n_rays, wl.grid.n_rays // 64)
    ref, _, _ = oracle_cube(wl, ids)
    _, paths = gpu_trace(sbr, wl, ray_ids=ids)
    cube = cube_complex(sbr.synthesize(paths, wl.radar))
    assert cube.shape == (12, 128, 256)
    assert rel_l2(cube, ref) <= TOL
    # static scene: every chirp identical, bitwise
    assert (cube == cube[:, :1]).all()


@pytest.mark.parametrize("ns", [1024, 2048, 4096])
@pytest.mark.parametrize("dist", [5.0, 10.0, 20.0])
def test_precision_sweep_cube_and_points(sbr, dist, ns):
    """The long-range sweep: the sphere at 5-20 m, 1024-4096 samples, a seeded 4096-ray subset
    of the 2048 x 2048 grid.  Against the FP64 oracle, the split and FP64 phase modes keep the
    IF cube within relative L2 1e-4 and the point cloud within 1 mm Chamfer; naive FP32 phase
    (f_c tau spans ~10^4 cycles at 20 m) is reported and must be the worst of the three."""
    from oracle import pointcloud as opc
    from sbr_inputs import CfarParams
    wl = sphere_scene(G=2048, distance=dist, n_samples=ns)
    ids = ray_subset(11, wl.grid.n_rays, 4096)
    ref, _, _ = oracle_cube(wl, ids)
    ref_pts = opc.pointcloud(ref, wl.radar, CfarParams())["points"]
    _, paths = gpu_trace(sbr, wl, ray_ids=ids)
    errs, cham = {}, {}
    for name, m in (("split", sbr.PHASE_SPLIT), ("fp64", sbr.PHASE_FP64), ("naive", sbr.PHASE_NAIVE)):
        cube_t = sbr.synthesize(paths, wl.radar, m)
        errs[name] = rel_l2(cube_complex(cube_t), ref)
        pts, st = sbr.pointcloud(cube_t, wl.radar, CfarParams())
        n = st.n_points()
        cham[name] = opc.chamfer_parity(pts[:n].cpu().numpy().astype(np.float64), ref_pts)
    print(f"\nsweep {dist:g} m, {ns} samples: cube rel L2 {errs}, Chamfer [m] {cham}")
    assert errs["split"] <= TOL and errs["fp64"] <= TOL, errs
    assert cham["split"] <= 1e-3 and cham["fp64"] <= 1e-3, cham
    assert errs["naive"] > max(errs["split"], errs["fp64"]), errs


def test_deterministic(sbr):
    wl = sphere_scene()
    _, paths = gpu_trace(sbr, wl)
    a = sbr.synthesize(paths, wl.radar).clone()
    b = sbr.synthesize(paths, wl.radar)
    assert torch.equal(a, b)


def test_synthesis_adjoint_matches_oracle(sbr):
    wl = sphere_scene(G=32)
    cube, tr, pa = oracle_cube(wl)
    _, paths = gpu_trace(sbr, wl)
    rng = np.random.default_rng(4)
    g = rng.normal(size=cube.shape) + 1j * rng.normal(size=cube.shape)
    gt, ga = oracle.synthesize_grad(pa["tau"], pa["amp"], wl.radar, g)
    gcube = torch.from_numpy(np.stack([g.real, g.imag], -1).astype(np.float32)).cuda()
    glen, gamp = sbr.synthesize_bwd(paths, wl.radar, gcube)
    P = paths.count()
    glen = glen.cpu().numpy()[:, :P].astype(np.float64)
    gamp = gamp.cpu().numpy()[:, :P].astype(np.float64)
    # GPU reports dL/d(path length) = dL/dtau / c
    np.testing.assert_allclose(glen * C_LIGHT, gt, rtol=0, atol=1e-3 * np.abs(gt).max())
    np.testing.assert_allclose(gamp, ga, rtol=0, atol=1e-4 * np.abs(ga).max())


@pytest.mark.parametrize("ns", [32, 64, 128, 256, 512, 1024])
def test_split_sample_counts(sbr, ns):
    """The split mode: a type-1 non-uniform FFT of Eq. 8 up to 512 samples (grid of 2 N_s
    points, width-8 kernel), the direct FP32 recurrence kernel above; both far inside 1e-4."""
    wl = sphere_scene(G=64, distance=2.0, n_samples=ns)
    ref, _, _ = oracle_cube(wl)
    _, paths = gpu_trace(sbr, wl)
    cube = cube_complex(sbr.synthesize(paths, wl.radar, sbr.PHASE_SPLIT))
    e_split = rel_l2(cube, ref)
    e_fp64 = rel_l2(cube_complex(sbr.synthesize(paths, wl.radar, sbr.PHASE_FP64)), ref)
    assert e_split <= 1e-5 and e_fp64 <= 1e-5, (e_split, e_fp64)


@pytest.mark.parametrize("ns", [256, 512])
def test_direct_tensor_core_path(sbr, ns):
    """The term-by-term tensor-core evaluation (fp16x3 mma.sync on n = 16 a + b), which the
    allocation-free entry point runs for 256 and 512 samples, against the oracle."""
    import ctypes
    from paper_2311_13182_gb300 import _lib, sim
    wl = sphere_scene(G=64, distance=2.0, n_samples=ns)
    ref, _, _ = oracle_cube(wl)
    _, paths = gpu_trace(sbr, wl)
    out = torch.empty((wl.radar.n_virt, wl.radar.n_chirps, ns, 2), device="cuda")
    r = sim.radar_struct(wl.radar)
    st = _lib.load().sbr_synthesize_noalloc(ctypes.byref(paths.s), ctypes.byref(r), int(sbr.PHASE_SPLIT),
                                            ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert rel_l2(cube_complex(out), ref) <= 1e-5


def test_no_paths_gives_zero_cube(sbr):
    wl = sphere_scene(G=8)
    from sbr_inputs import Workload
    far = Workload("miss", wl.verts + np.float32([50, 0, 0]), wl.faces, wl.radar, wl.grid, 2, {})
    _, paths = gpu_trace(sbr, far)
    assert paths.count() == 0
    cube = sbr.synthesize(paths, far.radar)
    assert torch.count_nonzero(cube).item() == 0
