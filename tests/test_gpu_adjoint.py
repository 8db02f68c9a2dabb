"""Trace adjoint and the end-to-end reconstruction gradient against FP64 central finite
differences of the oracle with the discrete structure (triangle sequences, peak cells,
nearest-neighbour pairs) held at the oracle's own unperturbed values.
Relative error |g - g_fd| / max(|g_fd|, 1e-3 max|g_fd|) <= 1e-3."""
import numpy as np
import pytest
import torch

import oracle
from oracle import pointcloud as opc
from sbr_inputs import (C_LIGHT, CfarParams, Workload, icosphere, radar_single_tx, ray_grid_for_sphere,
                        sphere_scene, superquadric)
from tests._util import gpu_trace

pytestmark = pytest.mark.gpu
H = 1e-6  # m


def weights(ray, k, v):
    """Deterministic upstream gradients per (ray, bounce, antenna) for both sides."""
    return np.sin(1.3 * ray + 0.7 * k + 2.1 * v), np.cos(0.9 * ray - 1.1 * k + 0.5 * v) * 1e4


def oracle_L(verts, wl, tr_ref, gl, ga, reparam=False):
    if reparam:
        tr = oracle.trace_reparam(verts, wl.faces, tr_ref, wl.grid, wl.verts)
    else:
        tr = oracle.trace_frozen(verts, wl.faces, tr_ref, wl.grid)
    pa = oracle.paths(tr, wl.radar)
    return float((gl * pa["tau"] * C_LIGHT).sum() + (ga * pa["amp"]).sum())


def rel_err(g, fd):
    return np.abs(g - fd) / np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())


def check_trace_adjoint(sbr, wl, ids=None, n_vert_checks=12, reparam=False):
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, wl.max_bounces, ray_ids=ids)
    scene, paths = gpu_trace(sbr, wl, ray_ids=ids)
    P = paths.count()
    ray_g = paths.path_ray().cpu().numpy()[:P]
    first = paths.ray_first().cpu().numpy()
    k_g = np.arange(P) - first[ray_g]
    V = wl.radar.n_virt
    gl = np.zeros((V, paths.cap), np.float32)
    ga = np.zeros((V, paths.cap), np.float32)
    for v in range(V):
        gl[v, :P], ga[v, :P] = weights(ray_g, k_g, v)
    vt = torch.from_numpy(wl.verts).cuda()
    ids_t = None if ids is None else torch.from_numpy(ids).cuda()
    g = sbr.trace_bwd(scene, vt, wl.radar, wl.grid, paths, torch.from_numpy(gl).cuda(),
                      torch.from_numpy(ga).cuda(), ray_ids=ids_t, reparam=reparam).cpu().numpy().astype(np.float64)
    pa = oracle.paths(tr, wl.radar)
    glo = np.stack([weights(pa["ray"], pa["bounce"], v)[0] for v in range(V)])
    gao = np.stack([weights(pa["ray"], pa["bounce"], v)[1] for v in range(V)])
    # the GPU trace must have the same triangle sequences (checked elsewhere); require it here
    assert (paths.hits()[0].cpu().numpy() == tr["tri"]).all()
    v64 = wl.verts.astype(np.float64)
    used = np.unique(wl.faces[tr["tri"][tr["tri"] >= 0]])
    rng = np.random.default_rng(3)
    for vi in rng.choice(used, size=min(n_vert_checks, used.size), replace=False):
        for ax in range(3):
            vp, vm = v64.copy(), v64.copy()
            vp[vi, ax] += H
            vm[vi, ax] -= H
            fd = (oracle_L(vp, wl, tr, glo, gao, reparam) - oracle_L(vm, wl, tr, glo, gao, reparam)) / (2 * H)
            scale = max(abs(fd), 1e-3 * np.abs(g).max())
            assert abs(g[vi, ax] - fd) <= 1e-3 * scale, (vi, ax, g[vi, ax], fd)
    # a random direction over all vertices
    D = rng.normal(size=v64.shape)
    fd = (oracle_L(v64 + H * D, wl, tr, glo, gao, reparam) - oracle_L(v64 - H * D, wl, tr, glo, gao, reparam)) / (2 * H)
    assert abs((g * D).sum() - fd) <= 1e-3 * abs(fd)
    return g


def test_trace_adjoint_sphere(sbr):
    check_trace_adjoint(sbr, sphere_scene(G=48))


def test_trace_adjoint_reparam_sphere(sbr):
    """SBR_BWD_REPARAM (Eq. 6-7: first hits attached to the surface, weights with |det J_T|) against
    FP64 central differences of the oracle's reparameterised samples; differs from the interior one."""
    wl = sphere_scene(G=48)
    g = check_trace_adjoint(sbr, wl, reparam=True)
    g0 = check_trace_adjoint(sbr, wl, n_vert_checks=2)
    assert np.abs(g - g0).max() > 1e-3 * np.abs(g0).max()


def test_trace_adjoint_reparam_corner_three_bounces(sbr):
    from tests.test_oracle_pins import axis_grid, corner_reflector
    C = np.array([0.25, 0.125, 2.0])
    v, f = corner_reflector(C, 0.75)
    wl = Workload("corner", v, f, radar_single_tx(), axis_grid(24, 0.12, axis=C), 3, {})
    check_trace_adjoint(sbr, wl, n_vert_checks=8, reparam=True)


def test_trace_adjoint_reparam_plate_integral(sbr):
    """With dL/dA = 1 on one antenna's paths the trace adjoint is the gradient of the
    Monte-Carlo estimate of the plate's integral of Eq. 1's strength.  Under the
    reparameterised samples its derivative along random vertex motions follows the derivative
    of the exact integral (quadrature) within 0.5 %, silhouette motion included; with fixed
    launch directions it does not (the boundary term is missing)."""
    from tests.test_oracle_pins import axis_grid, plate_integral, square
    v, f = square((-0.35, -0.25, 1.2), (0.7, 0.05, 0.15), (-0.05, 0.6, 0.1))
    wl = Workload("plate", v, f, radar_single_tx(), axis_grid(256, 0.5), 1, {})
    scene, paths = gpu_trace(sbr, wl)
    P = paths.count()
    V = wl.radar.n_virt
    gl = torch.zeros((V, paths.cap), device="cuda")
    ga = torch.zeros((V, paths.cap), device="cuda")
    ga[0, :P] = 1.0
    vt = torch.from_numpy(v).cuda()
    g = sbr.trace_bwd(scene, vt, wl.radar, wl.grid, paths, gl, ga, reparam=True).cpu().numpy().astype(np.float64)
    g0 = sbr.trace_bwd(scene, vt, wl.radar, wl.grid, paths, gl, ga).cpu().numpy().astype(np.float64)
    v64 = v.astype(np.float64)
    est = float(paths.prep()[0, :P, 3].double().sum())
    assert abs(est - plate_integral(v64, f, wl.radar)) < 0.01 * est
    rng = np.random.default_rng(7)
    miss = 0.0
    for _ in range(3):
        D = rng.normal(size=v64.shape)
        h = 1e-6
        ex = (plate_integral(v64 + h * D, f, wl.radar) - plate_integral(v64 - h * D, f, wl.radar)) / (2 * h)
        assert abs((g * D).sum() - ex) < 0.005 * abs(ex), ((g * D).sum(), ex)
        miss = max(miss, abs((g0 * D).sum() - ex) / abs(ex))
    assert miss > 0.05  # the fixed-direction gradient misses the boundary term


def test_trace_adjoint_corner_three_bounces(sbr):
    from tests.test_oracle_pins import axis_grid, corner_reflector
    C = np.array([0.25, 0.125, 2.0])
    v, f = corner_reflector(C, 0.75)
    wl = Workload("corner", v, f, radar_single_tx(), axis_grid(24, 0.12, axis=C), 3, {})
    check_trace_adjoint(sbr, wl, n_vert_checks=12)


def recon_setup(n_rays_side=64):
    """Reconstruction workload: superquadric target (20,000 tris) seen by the 1 Tx / 4 Rx radar,
    icosphere template (2562 vertices) at the target's centre."""
    sv, sf, params = superquadric(seed=5)
    c = np.array(params["center"])
    radar = radar_single_tx(256, 1)
    grid = ray_grid_for_sphere(c, 0.6, n_rays_side)
    tv, tf = icosphere(4, 0.2, c)
    return sv, sf, tv, tf, radar, grid


def test_reconstruction_gradient_fd(sbr):
    """End-to-end dLoss/dverts (Chamfer + 0.1 Laplacian) vs FP64 FD on 26 seeded vertices."""
    from paper_2311_13182_gb300.autograd import Simulator
    sv, sf, tv, tf, radar, grid = recon_setup()
    cfg = CfarParams()
    K = 2
    # target: the oracle's point cloud of the superquadric
    twl = Workload("target", sv, sf, radar, grid, K, {})
    tcube, _, _ = oracle.simulate_cube(twl)
    target = opc.pointcloud(tcube, radar, cfg)["points"]
    # oracle structure at the template
    wl = Workload("tmpl", tv, tf, radar, grid, K, {})
    tr = oracle.trace(tv, tf, grid, K)
    pa = oracle.paths(tr, radar)
    cube = oracle.synthesize(pa["tau"], pa["amp"], radar)
    pc = opc.pointcloud(cube, radar, cfg)
    a, k = pc["a"], pc["k"]
    P = pc["points"]
    nn_pq = opc._nn(P, target)[0]
    nn_qp = opc._nn(target, P)[0]

    def loss(v):
        trf = oracle.trace_frozen(v, tf, tr, grid)
        p = oracle.paths(trf, radar)
        c = oracle.synthesize(p["tau"], p["amp"], radar)
        _, _, Pw = opc.power_map(c, radar, cfg)
        pts = opc.points_at(Pw, radar, cfg, a, k)
        return opc.chamfer_loss(pts, target, nn_pq, nn_qp) + 0.1 * opc.laplacian(v, tf)

    # GPU gradient
    simr = Simulator(tf, tv.shape[0], radar, grid, K, cfg)
    vt = torch.from_numpy(tv).cuda()
    pts, n = simr.forward(vt)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    l_gpu, gpts = sbr.chamfer(pts, n, tgt)
    g = torch.zeros_like(vt)
    adj = sbr.Adjacency(tf, tv.shape[0])
    sbr.laplacian(vt, adj, 0.1, l_gpu, g)
    simr.backward(vt, gpts, g)
    g = g.cpu().numpy().astype(np.float64)
    n = int(n.item())
    assert sorted(simr.state.peak_cells().cpu().numpy()[:n].tolist()) == sorted((a * 256 + k).tolist())
    v64 = tv.astype(np.float64)
    assert abs(float(l_gpu.item()) - loss(v64)) <= 1e-3 * abs(loss(v64))
    rng = np.random.default_rng(26)
    seen = np.unique(tf[tr["tri"][tr["tri"] >= 0]])
    chosen = rng.choice(seen, size=min(26, seen.size), replace=False)
    fd = np.zeros((len(chosen), 3))
    for i, vi in enumerate(chosen):
        for ax in range(3):
            vp, vm = v64.copy(), v64.copy()
            vp[vi, ax] += H
            vm[vi, ax] -= H
            fd[i, ax] = (loss(vp) - loss(vm)) / (2 * H)
    err = rel_err(g[chosen], fd)
    assert (err <= 1e-3).all(), err.max()


@pytest.mark.parametrize("reparam", [False, True])
def test_image_loss_gradient_fd(sbr, reparam):
    """The paper's spatial loss (Eq. 16) end to end: dloss/dverts of the mean squared
    range-angle power-map difference (no Laplacian) against FP64 central differences of the
    oracle chain (frozen triangle sequences, paths, Eq. 8, direct DFTs, power map) on 12
    seeded template vertices x 3 axes; with reparam, the oracle chain samples under the
    change of variables of Eq. 6-7 (trace_reparam) and the simulator differentiates the same."""
    from paper_2311_13182_gb300.autograd import Simulator
    sv, sf, tv, tf, radar, grid = recon_setup()
    cfg = CfarParams()
    K = 2
    tcube, _, _ = oracle.simulate_cube(Workload("t", sv, sf, radar, grid, K, {}))
    _, _, target = opc.power_map(tcube, radar, cfg)
    s = Simulator(tf, tv.shape[0], radar, grid, K, cfg, reparam=reparam)
    vt = torch.from_numpy(tv).cuda()
    s.forward_image(vt)
    loss, gcube = sbr.image_loss(s.state, torch.from_numpy(target.astype(np.float32)).cuda())
    g = torch.zeros_like(vt)
    s.backward_cube(vt, gcube, g)
    g = g.cpu().numpy().astype(np.float64)
    wl = Workload("tmpl", tv, tf, radar, grid, K, {})
    tr = oracle.trace(tv, tf, grid, K)

    def L(verts):
        trv = oracle.trace_reparam(verts, tf, tr, grid, tv) if reparam else oracle.trace_frozen(verts, tf, tr, grid)
        pa = oracle.paths(trv, radar)
        return opc.image_loss(oracle.synthesize(pa["tau"], pa["amp"], radar), target, radar, cfg)

    v64 = tv.astype(np.float64)
    assert abs(float(loss.item()) - L(v64)) <= 1e-4 * L(v64)
    used = np.unique(tf[tr["tri"][(tr["tri"] >= 0) & (tr["flag"][:, None] == 0)]])
    rng = np.random.default_rng(17)
    picks = rng.choice(used, size=12, replace=False)
    fd = np.zeros((12, 3))
    for i, vi in enumerate(picks):
        for ax in range(3):
            vp, vm = v64.copy(), v64.copy()
            vp[vi, ax] += H
            vm[vi, ax] -= H
            fd[i, ax] = (L(vp) - L(vm)) / (2 * H)
    err = rel_err(g[picks], fd)
    assert err.max() <= 1e-3, (err.max(), g[picks], fd)


def test_image_loss_reconstruction_descends(sbr):
    """Reconstruction with the paper's spatial loss (Eq. 16) against the target's power map:
    30 Adam iterations, replayed as a CUDA graph, lower the loss."""
    from paper_2311_13182_gb300.recon import Reconstruction
    sv, sf, tv, tf, radar, grid = recon_setup()
    cfg = CfarParams()
    tcube, _, _ = oracle.simulate_cube(Workload("t", sv, sf, radar, grid, 2, {}))
    _, _, target = opc.power_map(tcube, radar, cfg)
    rec = Reconstruction(tv, tf, torch.from_numpy(target.astype(np.float32)), radar, grid, 2, cfg, lr=1e-3,
                         lap_weight=0.0, loss="image")
    rec.step()
    loss0 = float(rec.loss.item())
    rec.capture()
    rec.replay(30)
    torch.cuda.synchronize()
    loss1 = float(rec.loss.item())
    assert np.isfinite(loss1) and loss1 < loss0, (loss0, loss1)


def test_trace_adjoint_jittered_grid(sbr):
    """The trace adjoint on a jittered grid (its launch directions come from the offsets)."""
    import dataclasses
    from sbr_inputs import jittered
    wl = sphere_scene(G=32)
    check_trace_adjoint(sbr, dataclasses.replace(wl, grid=jittered(wl.grid, 6)))


def _fan(n_rim: int):
    """A flat fan: centre vertex 0 joined to n_rim rim vertices (centre degree n_rim)."""
    ang = np.linspace(0.0, 2 * np.pi, n_rim, endpoint=False)
    rng = np.random.default_rng(7)
    v = np.concatenate([[[0.0, 0.0, 0.1]], np.stack([np.cos(ang), np.sin(ang), 0.05 * rng.standard_normal(n_rim)], 1)])
    f = np.array([[0, 1 + i, 1 + (i + 1) % n_rim] for i in range(n_rim)], np.int32)
    return v.astype(np.float32), f


@pytest.mark.parametrize("mesh", ["icosphere4", "fan24"])
def test_laplacian_value_and_gradient(sbr, mesh):
    """sbr_laplacian against the oracle's uniform Laplacian (weight x mean_i |v_i - mean of its
    neighbours|^2): the value it adds to the loss within 1e-5 relative, and the gradient it adds
    within 1e-4 of the largest component against FP64 central differences of the oracle (exact
    for this quadratic up to rounding).  The icosphere (2,562 vertices) spans 11 CTAs with a
    ragged last one; the fan's centre has 24 neighbours, past the neighbours loaded together."""
    if mesh == "icosphere4":
        v, f = icosphere(4, 0.2)
        rng = np.random.default_rng(3)
        v = (v * (1.0 + 0.05 * rng.standard_normal((v.shape[0], 1)))).astype(np.float32)
    else:
        v, f = _fan(24)
    w = 0.1
    vt = torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
    adj = sbr.Adjacency(f, v.shape[0])
    l0, g0 = 2.0 ** -20, 2.0 ** -30  # the call adds to what is there (small, so no precision is lost)
    loss = torch.full((1,), l0, device="cuda")
    g = torch.full_like(vt, g0)
    sbr.laplacian(vt, adj, w, loss, g)
    torch.cuda.synchronize()
    v64 = v.astype(np.float64)
    ref = w * opc.laplacian(v64, f)
    assert abs((float(loss.item()) - l0) - ref) <= 1e-5 * ref
    gg = g.cpu().numpy().astype(np.float64) - g0
    rng = np.random.default_rng(11)
    chosen = np.unique(np.concatenate([[0], rng.choice(v.shape[0], size=min(20, v.shape[0]), replace=False)]))
    H = 1e-5
    fd = np.zeros((chosen.size, 3))
    for i, vi in enumerate(chosen):
        for ax in range(3):
            vp, vm = v64.copy(), v64.copy()
            vp[vi, ax] += H
            vm[vi, ax] -= H
            fd[i, ax] = w * (opc.laplacian(vp, f) - opc.laplacian(vm, f)) / (2 * H)
    scale = np.abs(fd).max()
    assert np.abs(gg[chosen] - fd).max() <= 1e-4 * scale, np.abs(gg[chosen] - fd).max() / scale
