"""Fresnel materials on the GPU (Section 3.2.2, Eq. 9-10): per-path Fresnel factors, the IF
cube and the point cloud against the FP64 oracle, the perfect-conductor limit, and the
adjoint's dL/d eps and dL/dverts against FP64 central differences of the oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import pointcloud as opc
from sbr_inputs import C_LIGHT, CfarParams, Workload, merge_meshes, radar_single_tx, sphere_scene
from tests._util import cube_complex, rel_l2

pytestmark = pytest.mark.gpu

EPS = np.array([4.0 - 0.5j, -1.0 + 0j, 9.0 - 2.0j])   # a lossy dielectric, a conductor, a lossier one


def wedge_workload():
    from tests.test_oracle_pins import axis_grid, square
    E = np.array([0.0, -1.0, 2.0])
    a = square(E, (0, 2.0, 0), (-0.5, 0.0, -0.875))
    b = square(E, (0, 2.0, 0), (0.5, 0.0, -0.875))
    v, f = merge_meshes(a, b)
    return Workload("wedge", v, f, radar_single_tx(), axis_grid(48, 0.3), 2, {}), np.array([0, 0, 2, 2], np.int32)


def sphere_workload():
    wl = sphere_scene(G=32)
    return wl, (np.arange(wl.faces.shape[0]) % 3).astype(np.int32)


def gpu_paths(sbr, wl, tri_mat, eps=EPS):
    v = torch.from_numpy(wl.verts).cuda()
    f = torch.from_numpy(wl.faces).cuda()
    scene = sbr.Scene(v, f)
    tm = torch.from_numpy(tri_mat).cuda()
    scene.set_materials(eps, tm)
    paths = sbr.trace(scene, wl.radar, wl.grid, wl.max_bounces)
    torch.cuda.synchronize()
    return scene, paths, v, tm


@pytest.mark.parametrize("which", ["wedge", "sphere"])
def test_material_paths_cube_and_points(sbr, which):
    wl, tri_mat = wedge_workload() if which == "wedge" else sphere_workload()
    ref, tr, pa = oracle.simulate_cube(wl, materials=(tri_mat, EPS))
    scene, paths, _, _ = gpu_paths(sbr, wl, tri_mat)
    P = paths.count()
    assert P == pa["P"] and (paths.hits()[0].cpu().numpy() == tr["tri"]).all()
    # strength A |F| and phase arg F / (2 pi) of every path against the oracle's complex strength
    amp = paths.prep().cpu().numpy()[:, :P, 3].astype(np.float64)
    ph = paths.phase_ofs().cpu().numpy()[:P].astype(np.float64)
    gpu_c = amp * np.exp(2j * np.pi * ph)[None, :]
    np.testing.assert_allclose(gpu_c, pa["amp_c"], rtol=0, atol=3e-6 * np.abs(pa["amp_c"]).max())
    assert (np.abs(pa["fresnel"]) < 0.999).any()        # the dielectrics do attenuate
    for name, mode in (("split", sbr.PHASE_SPLIT), ("fp64", sbr.PHASE_FP64)):
        cube = cube_complex(sbr.synthesize(paths, wl.radar, mode))
        assert rel_l2(cube, ref) <= 1e-4, name
    pts, st = sbr.pointcloud(sbr.synthesize(paths, wl.radar), wl.radar, CfarParams())
    n = st.n_points()
    ref_pts = opc.pointcloud(ref, wl.radar)["points"]
    assert n > 0 and opc.chamfer_parity(pts[:n].cpu().numpy().astype(np.float64), ref_pts) <= 1e-3


def test_conductor_materials_equal_no_materials(sbr):
    """Every material a perfect conductor: the cube is the conductor model's, within rounding
    (the sign moves from the strength into the phase)."""
    wl, tri_mat = sphere_workload()
    _, paths, _, _ = gpu_paths(sbr, wl, tri_mat, eps=[-1.0, -1.0, -1.0])
    c_mat = cube_complex(sbr.synthesize(paths, wl.radar))
    v = torch.from_numpy(wl.verts).cuda()
    plain = sbr.trace(sbr.Scene(v, torch.from_numpy(wl.faces).cuda()), wl.radar, wl.grid, wl.max_bounces)
    c_pec = cube_complex(sbr.synthesize(plain, wl.radar))
    assert rel_l2(c_mat, c_pec) <= 1e-6


def test_material_adjoint_fd(sbr):
    """L = Re sum conj(g) S for a random upstream g: dL/d eps (per material, real and
    imaginary part) and dL/dverts through the Fresnel factors' incidence angles, against FP64
    central differences of the oracle with the triangle sequences held fixed."""
    wl, tri_mat = wedge_workload()
    scene, paths, v, tm = gpu_paths(sbr, wl, tri_mat)
    rng = np.random.default_rng(5)
    shape = (wl.radar.n_virt, 1, wl.radar.n_samples)
    g = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    gcube = torch.from_numpy(np.stack([g.real, g.imag], -1).astype(np.float32)).cuda()
    glen, gamp, gph = sbr.synthesize_bwd(paths, wl.radar, gcube, phase=True)
    gv = torch.zeros_like(v)
    geps = torch.zeros((len(EPS), 2), device="cuda")
    sbr.trace_bwd(scene, v, wl.radar, wl.grid, paths, glen, gamp, gverts=gv, gphase=gph, geps=geps)
    gv, geps = gv.cpu().numpy().astype(np.float64), geps.cpu().numpy().astype(np.float64)
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, wl.max_bounces)

    def L(verts, eps):
        t2 = oracle.trace_frozen(verts, wl.faces, tr, wl.grid)
        pa = oracle.paths(t2, wl.radar)
        F = oracle.path_fresnel(t2, pa, tri_mat, eps)
        sign = np.where(pa["bounce"] % 2 == 0, 1.0, -1.0)
        S = oracle.synthesize(pa["tau"], pa["amp"] * sign[None, :] * F[None, :], wl.radar)
        return float(np.real(np.conj(g) * S).sum())

    v64 = wl.verts.astype(np.float64)
    h = 1e-4
    for m in (0, 2):                       # the conductor (material 1) has no parameter
        for part, dz in ((0, 1.0), (1, -1j)):   # eps = eps_re - j eps_im
            ep, em = EPS.copy(), EPS.copy()
            ep[m] += h * dz
            em[m] -= h * dz
            fd = (L(v64, ep) - L(v64, em)) / (2 * h)
            assert abs(geps[m, part] - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.abs(geps).max()), (m, part, geps, fd)
    assert geps[1].tolist() == [0.0, 0.0]
    hv = 1e-6
    fd = np.zeros((4, 3))
    for vi in range(4):
        for ax in range(3):
            vp, vm = v64.copy(), v64.copy()
            vp[vi, ax] += hv
            vm[vi, ax] -= hv
            fd[vi, ax] = (L(vp, EPS) - L(vm, EPS)) / (2 * hv)
    den = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert (np.abs(gv[:4] - fd) / den).max() <= 1e-3, (gv[:4], fd)
