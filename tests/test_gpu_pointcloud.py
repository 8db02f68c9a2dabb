"""GPU point cloud parity (Chamfer <= 1 mm against the FP64 oracle's chain) and its adjoint
against FP64 central differences with the peak set held fixed."""
import numpy as np
import pytest
import torch

import oracle
from oracle import pointcloud as opc
from sbr_inputs import CfarParams, ray_subset, sphere_scene, superquadric_scene
from tests._util import cube_complex, gpu_trace, rel_l2

pytestmark = pytest.mark.gpu

CHAMFER_TOL = 1e-3  # m


def to_cube_t(cube):
    return torch.from_numpy(np.stack([cube.real, cube.imag], -1).astype(np.float32)).cuda().contiguous()


def gpu_points(sbr, cube_t, radar, cfg):
    pts, st = sbr.pointcloud(cube_t, radar, cfg)
    n = st.n_points()
    return pts.cpu().numpy()[:n].astype(np.float64), st, n


@pytest.mark.parametrize("scene", ["sphere", "superquadric"])
def test_pointcloud_from_oracle_cube(sbr, scene):
    """Same IF cube into both chains: power map, peak cells and points agree."""
    if scene == "sphere":
        wl, ids = sphere_scene(), None
    else:
        wl = superquadric_scene(seed=3, G=1024)
        ids = ray_subset(5, wl.grid.n_rays, wl.grid.n_rays // 64)
    cube, _, _ = oracle.simulate_cube(wl, ids)
    cfg = CfarParams()
    ref = opc.pointcloud(cube, wl.radar, cfg)
    pts, st, n = gpu_points(sbr, to_cube_t(cube), wl.radar, cfg)
    assert rel_l2(st.power().double().cpu().numpy(), ref["Pw"]) < 1e-5
    assert n > 0 and abs(n - ref["points"].shape[0]) <= max(2, n // 50)
    assert opc.chamfer_parity(pts, ref["points"]) <= CHAMFER_TOL
    # strong detections: identical cells
    strong = ref["points"][:, 3] > 0.5
    cells_ref = set((ref["a"][strong] * wl.radar.n_samples + ref["k"][strong]).tolist())
    cells_gpu = set(st.peak_cells().cpu().numpy()[:n].tolist())
    assert cells_ref <= cells_gpu
    # rows past the count are zero
    assert (sbr.pointcloud(to_cube_t(cube), wl.radar, cfg, state=st)[0][n:] == 0).all()


@pytest.mark.parametrize("cube_kind", ["sphere", "noise"])
def test_point_order(sbr, cube_kind):
    """The emitted points run in the selection's order: weights non-increasing, equal weights in
    ascending cell order, for a cube with few candidates (the sphere: ranked directly) and for a
    seeded noise cube whose local maxima give hundreds (the sort network); the count is the
    oracle chain's within 2 % and the weighted point sets agree within 1 mm."""
    import dataclasses
    wl = sphere_scene()
    cfg = CfarParams()
    if cube_kind == "sphere":
        cube, _, _ = oracle.simulate_cube(wl)
    else:
        cfg = dataclasses.replace(cfg, alpha_db=6.0)  # ~400 candidates
        rng = np.random.default_rng(17)
        shape = (wl.radar.n_virt, wl.radar.n_chirps, wl.radar.n_samples)
        cube = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 1e-3
    ref = opc.pointcloud(cube, wl.radar, cfg)
    pts, st, n = gpu_points(sbr, to_cube_t(cube), wl.radar, cfg)
    cells = st.peak_cells().cpu().numpy()[:n]
    if cube_kind == "noise":
        assert n > 256  # past the directly ranked sizes
    else:
        assert 0 < n <= 256
    w = pts[:, 3]
    assert (np.diff(w) <= 0).all()
    tie = np.diff(w) == 0
    assert (np.diff(cells)[tie] > 0).all()
    assert abs(n - ref["points"].shape[0]) <= max(2, n // 50)
    assert opc.chamfer_parity(pts, ref["points"]) <= CHAMFER_TOL


def test_end_to_end_sphere_chamfer(sbr):
    wl = sphere_scene()
    cube, _, _ = oracle.simulate_cube(wl)
    ref = opc.pointcloud(cube, wl.radar)
    _, paths = gpu_trace(sbr, wl)
    gcube = sbr.synthesize(paths, wl.radar)
    pts, st, n = gpu_points(sbr, gcube, wl.radar, CfarParams())
    assert opc.chamfer_parity(pts, ref["points"]) <= CHAMFER_TOL


def test_end_to_end_superquadric_subset_chamfer(sbr):
    wl = superquadric_scene(seed=4, G=1024)
    ids = ray_subset(9, wl.grid.n_rays, wl.grid.n_rays // 64)
    cube, _, _ = oracle.simulate_cube(wl, ids)
    ref = opc.pointcloud(cube, wl.radar)
    _, paths = gpu_trace(sbr, wl, ray_ids=ids)
    pts, _, n = gpu_points(sbr, sbr.synthesize(paths, wl.radar), wl.radar, CfarParams())
    assert opc.chamfer_parity(pts, ref["points"]) <= CHAMFER_TOL


def test_empty_cube_no_points(sbr):
    wl = sphere_scene()
    z = torch.zeros((4, 1, 256, 2), device="cuda")
    pts, st = sbr.pointcloud(z, wl.radar, CfarParams())
    assert st.n_points() == 0 and (pts == 0).all()


def test_pointcloud_adjoint_directional_fd(sbr):
    """dL/dcube from sbr_pointcloud_bwd vs FP64 central differences of the oracle chain with
    its own peak cells held fixed; L = sum_i g_i . point_i."""
    wl = sphere_scene()
    cube, _, _ = oracle.simulate_cube(wl)
    cfg = CfarParams()
    ref = opc.pointcloud(cube, wl.radar, cfg)
    a, k = ref["a"], ref["k"]
    pts, st, n = gpu_points(sbr, to_cube_t(cube), wl.radar, cfg)
    cells_gpu = st.peak_cells().cpu().numpy()[:n]
    assert sorted(cells_gpu.tolist()) == sorted((a * 256 + k).tolist())
    rng = np.random.default_rng(21)
    g_by_cell = {int(c): rng.normal(size=4) for c in sorted(cells_gpu.tolist())}
    g_gpu = np.zeros((cfg.k_max, 4), np.float32)
    for i, c in enumerate(cells_gpu):
        g_gpu[i] = g_by_cell[int(c)]
    g_ref = np.array([g_by_cell[int(c)] for c in (a * 256 + k)])
    gcube = sbr.pointcloud_bwd(st, torch.from_numpy(g_gpu).cuda())
    gc = cube_complex(gcube)

    def L(c):
        _, _, Pw = opc.power_map(c, wl.radar, cfg)
        return float((opc.points_at(Pw, wl.radar, cfg, a, k) * g_ref).sum())

    scale = np.abs(cube).max()
    for trial in range(3):
        D = rng.normal(size=cube.shape) + 1j * rng.normal(size=cube.shape)
        h = 1e-6 * scale
        fd = (L(cube + h * D) - L(cube - h * D)) / (2 * h)
        an = float((gc.real * D.real + gc.imag * D.imag).sum())
        assert abs(an - fd) <= 1e-3 * abs(fd), (trial, an, fd)


@pytest.mark.parametrize("n_tx,n_rx,C,Ns,A", [
    (1, 4, 1, 256, 64),     # the 1 Tx x 4 Rx radar, one chirp
    (3, 4, 128, 256, 64),   # the 3 Tx x 4 Rx radar of the bench step
    (1, 5, 1, 128, 64),     # odd antenna count, one range tile, a Doppler group of one bin
    (3, 4, 8, 128, 64),     # several Doppler groups
    (4, 4, 8, 128, 32),     # 16 antennas (the full K of the tensor path), 32 angle bins
    (2, 3, 4, 4096, 16),    # 4096 samples per chirp, 16 angle bins
    (4, 5, 2, 128, 64),     # 20 antennas: beyond the tensor path, CUDA cores
    (1, 4, 2, 64, 64),      # 64 samples: below one 128-bin tile, CUDA cores
    (1, 4, 1, 256, 128),    # 128 angle bins: tensor cores with N = 256
    (2, 4, 2, 128, 256),    # 256 angle bins: CUDA cores
])
def test_power_map_shapes(sbr, n_tx, n_rx, C, Ns, A):
    """Angle DFT + power map (the tensor-core kernel where the shape allows, CUDA cores
    otherwise) against the oracle's direct FP64 chain on a random cube: relative L2 < 1e-5,
    and the device status word clean."""
    from sbr_inputs import _radar
    radar = _radar(77e9, 4e9, 40e-6, Ns, C, n_tx, 0.5 * n_rx, n_rx=n_rx)
    rng = np.random.default_rng(n_tx * 1000 + n_rx * 100 + C + Ns + A)
    V = n_tx * n_rx
    cube = rng.normal(size=(V, C, Ns)) + 1j * rng.normal(size=(V, C, Ns))
    cfg = CfarParams(n_theta=A)
    _, _, Pw = opc.power_map(cube, radar, cfg)
    _, st = sbr.pointcloud(to_cube_t(cube), radar, cfg)
    st.check()
    assert rel_l2(st.power().double().cpu().numpy(), Pw) < 1e-5


def test_image_loss_value_and_cube_gradient(sbr):
    """Eq. 16 image loss of a random 4-antenna, 2-chirp cube against a perturbed copy of its own
    power map: the value against the oracle's FP64 chain, dloss/dcube against FP64 central
    differences of the oracle along random directions."""
    from sbr_inputs import _radar
    radar = _radar(77e9, 4e9, 40e-6, 128, 2, 1, 2.0, n_rx=4)
    rng = np.random.default_rng(21)
    cube = rng.normal(size=(4, 2, 128)) + 1j * rng.normal(size=(4, 2, 128))
    cfg = CfarParams()
    _, _, Pw = opc.power_map(cube, radar, cfg)
    target = Pw * rng.uniform(0.5, 1.5, size=Pw.shape)
    st = sbr.power_map(to_cube_t(cube), radar, cfg)
    st.check()
    loss, gcube = sbr.image_loss(st, torch.from_numpy(target.astype(np.float32)).cuda())
    ref = opc.image_loss(cube, target, radar, cfg)
    assert abs(float(loss.item()) - ref) <= 1e-5 * abs(ref)
    g = gcube.double().cpu().numpy()
    g = g[..., 0] + 1j * g[..., 1]
    h = 1e-5
    for _ in range(3):
        u = rng.normal(size=cube.shape) + 1j * rng.normal(size=cube.shape)
        fd = (opc.image_loss(cube + h * u, target, radar, cfg) - opc.image_loss(cube - h * u, target, radar, cfg)) / (2 * h)
        an = float(np.sum(g.real * u.real + g.imag * u.imag))
        assert abs(an - fd) <= 1e-3 * abs(fd), (an, fd)
    # the loss alone (no gradient requested) gives the same value
    loss2, _ = sbr.image_loss(st, torch.from_numpy(target.astype(np.float32)).cuda(), want_grad=False)
    assert float(loss2.item()) == float(loss.item())


def point_cube(radar, targets):
    """IF cube of ideal point targets [(position, amplitude)] through the oracle's Eq. 8."""
    from sbr_inputs import C_LIGHT
    tau = np.zeros((radar.n_virt, len(targets)))
    amp = np.zeros_like(tau)
    for j, (p, a) in enumerate(targets):
        p = np.asarray(p, float)
        for t in range(radar.n_tx):
            for r in range(radar.n_rx):
                tau[t * radar.n_rx + r, j] = (np.linalg.norm(p - radar.tx[t]) + np.linalg.norm(p - radar.rx[r])) / C_LIGHT
                amp[t * radar.n_rx + r, j] = a
    return oracle.synthesize(tau, amp, radar)


def elevated_targets():
    out = []
    for u0, w0, r0, a in ((0.3, 0.2, 2.1, 1.0), (-0.4, -0.5, 3.3, 0.7), (0.05, 0.6, 1.6, 0.5), (-0.1, 0.0, 4.2, 0.8)):
        out.append(((r0 * u0, r0 * w0, r0 * np.sqrt(1 - u0 * u0 - w0 * w0)), a))
    return out


@pytest.mark.parametrize("C,E,A", [
    (4, 2, 64),    # 128 rows: tensor cores with N = 256
    (4, 4, 16),    # 64 rows: tensor cores with N = 128
    (2, 8, 32),    # 256 rows: CUDA cores
    (1, 4, 64),    # 256 rows, one chirp: CUDA cores
])
def test_power_map_elevation_rows(sbr, C, E, A):
    """The 2D virtual array of the AWR1843-like radar (middle Tx raised by lambda/2): the power map
    over E x A angle rows (row e * A + a, steering with x and y of every element) against the
    oracle's FP64 chain on a random cube: relative L2 < 1e-5, the status word clean."""
    from sbr_inputs import radar_awr1843
    radar = radar_awr1843(256, C)
    rng = np.random.default_rng(100 * E + A + C)
    cube = rng.normal(size=(12, C, 256)) + 1j * rng.normal(size=(12, C, 256))
    cfg = CfarParams(n_theta=A, n_elev=E)
    _, _, Pw = opc.power_map(cube, radar, cfg)
    assert Pw.shape == (E * A, 256)
    st = sbr.power_map(to_cube_t(cube), radar, cfg)
    st.check()
    assert tuple(st.power().shape) == (E * A, 256)
    assert rel_l2(st.power().double().cpu().numpy(), Pw) < 1e-5


@pytest.mark.parametrize("E", [1, 4, 8])
def test_pointcloud_elevation_point_targets(sbr, E):
    """Point targets at four (azimuth, elevation, range) through the oracle's Eq. 8 into both point
    clouds with E elevation bins: the peak cells of every strong detection identical, the points
    within 1 mm (Chamfer) and the strongest point of each target within 0.02 of its direction
    cosines for E = 8; with E = 1 every point has y = 0."""
    from sbr_inputs import radar_awr1843
    radar = radar_awr1843(256, 2)
    cube = point_cube(radar, elevated_targets())
    cfg = CfarParams(n_theta=64 if E < 8 else 32, n_elev=E)  # at most 256 angle rows
    ref = opc.pointcloud(cube, radar, cfg)
    pts, st, n = gpu_points(sbr, to_cube_t(cube), radar, cfg)
    st.check()
    assert rel_l2(st.power().double().cpu().numpy(), ref["Pw"]) < 1e-5
    assert n > 0 and abs(n - ref["points"].shape[0]) <= max(2, n // 50)
    assert opc.chamfer_parity(pts, ref["points"]) <= CHAMFER_TOL
    strong = ref["points"][:, 3] > 0.5
    cells_ref = set((ref["a"][strong] * 256 + ref["k"][strong]).tolist())
    assert cells_ref <= set(st.peak_cells().cpu().numpy()[:n].tolist())
    if E == 1:
        assert (pts[:, 1] == 0).all()
    if E == 8:
        cells = st.peak_cells().cpu().numpy()[:n]
        Pw = st.power().double().cpu().numpy().ravel()
        for p, _ in elevated_targets():
            p = np.asarray(p)
            r0 = np.linalg.norm(p)
            near = np.flatnonzero(np.abs(np.linalg.norm(pts[:, :3], axis=1) - r0) < 0.05)
            assert near.size
            top = pts[near[np.argmax(Pw[cells[near]])]]  # the target's strongest cell
            rr = np.linalg.norm(top[:3])
            assert abs(top[0] / rr - p[0] / r0) < 0.02 and abs(top[1] / rr - p[1] / r0) < 0.02, (top, p)


def test_pointcloud_adjoint_elevation_fd(sbr):
    """sbr_pointcloud_bwd with 4 elevation bins (elevation refine on the two inner bins) against FP64
    central differences of the oracle chain with its peak cells held fixed."""
    from sbr_inputs import radar_awr1843
    radar = radar_awr1843(256, 1)
    cube = point_cube(radar, elevated_targets())
    cfg = CfarParams(n_elev=4)
    ref = opc.pointcloud(cube, radar, cfg)
    a, k = ref["a"], ref["k"]
    assert ((a // cfg.n_theta > 0) & (a // cfg.n_theta < 3)).any()  # some points refine in elevation
    pts, st, n = gpu_points(sbr, to_cube_t(cube), radar, cfg)
    cells_gpu = st.peak_cells().cpu().numpy()[:n]
    assert sorted(cells_gpu.tolist()) == sorted((a * 256 + k).tolist())
    rng = np.random.default_rng(33)
    g_by_cell = {int(c): rng.normal(size=4) for c in sorted(cells_gpu.tolist())}
    g_gpu = np.zeros((cfg.k_max, 4), np.float32)
    for i, c in enumerate(cells_gpu):
        g_gpu[i] = g_by_cell[int(c)]
    g_ref = np.array([g_by_cell[int(c)] for c in (a * 256 + k)])
    gc = cube_complex(sbr.pointcloud_bwd(st, torch.from_numpy(g_gpu).cuda()))

    def L(c):
        _, _, Pw = opc.power_map(c, radar, cfg)
        return float((opc.points_at(Pw, radar, cfg, a, k) * g_ref).sum())

    scale = np.abs(cube).max()
    for trial in range(3):
        D = rng.normal(size=cube.shape) + 1j * rng.normal(size=cube.shape)
        h = 1e-6 * scale
        fd = (L(cube + h * D) - L(cube - h * D)) / (2 * h)
        an = float((gc.real * D.real + gc.imag * D.imag).sum())
        assert abs(an - fd) <= 1e-3 * abs(fd), (trial, an, fd)


def test_image_loss_elevation(sbr):
    """Eq. 16 image loss over the E x A map of the 2D array: value and dloss/dcube against the oracle."""
    from sbr_inputs import radar_awr1843
    radar = radar_awr1843(128, 2)
    rng = np.random.default_rng(44)
    cube = rng.normal(size=(12, 2, 128)) + 1j * rng.normal(size=(12, 2, 128))
    cfg = CfarParams(n_theta=32, n_elev=2)
    _, _, Pw = opc.power_map(cube, radar, cfg)
    target = Pw * rng.uniform(0.5, 1.5, size=Pw.shape)
    st = sbr.power_map(to_cube_t(cube), radar, cfg)
    tt = torch.from_numpy(target.astype(np.float32)).cuda()
    loss, gcube = sbr.image_loss(st, tt)
    ref = opc.image_loss(cube, target, radar, cfg)
    assert abs(float(loss.item()) - ref) <= 1e-5 * abs(ref)
    g = cube_complex(gcube)
    h = 1e-5
    for _ in range(2):
        u = rng.normal(size=cube.shape) + 1j * rng.normal(size=cube.shape)
        fd = (opc.image_loss(cube + h * u, target, radar, cfg) - opc.image_loss(cube - h * u, target, radar, cfg)) / (2 * h)
        an = float(np.sum(g.real * u.real + g.imag * u.imag))
        assert abs(an - fd) <= 1e-3 * abs(fd), (an, fd)
    with pytest.raises(ValueError):
        sbr.image_loss(st, tt[: 32])
