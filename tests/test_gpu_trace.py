"""GPU trace parity: nearest-hit triangle indices bit-exact against the FP64 brute-force oracle
for every ray the oracle does not flag as within 1e-6 (barycentric) of an edge or tied."""
import numpy as np
import pytest
import torch

import oracle
from sbr_inputs import (C_LIGHT, icosphere, merge_meshes, radar_single_tx, ray_grid_for_sphere, ray_subset,
                        sphere_scene, superquadric_scene, Workload)
from tests._util import compare_tri, gpu_trace

pytestmark = pytest.mark.gpu


def check_paths(wl, tr, paths):
    """Hit points (FP64 refine), path count and per-antenna delays/strengths against the oracle."""
    mism, n_ok, tri_gpu = compare_tri(tr, paths)
    assert mism == 0, f"{mism} of {n_ok} unflagged rays chose a different triangle"
    ok = tr["flag"] == 0
    hp = paths.hit_points().cpu().numpy()
    valid = (tr["tri"] >= 0) & ok[:, None]
    np.testing.assert_allclose(hp[valid], tr["hit"][valid], rtol=0, atol=1e-9)
    P = paths.count()
    assert P == int((tri_gpu >= 0).sum())
    pa = oracle.paths(tr, wl.radar)
    if P:
        tau = paths.path_len().cpu().numpy()[:, :P] / C_LIGHT
        amp = paths.prep().cpu().numpy()[:, :P, 3]
        ray_gpu = paths.path_ray().cpu().numpy()[:P]
        # compare paths of unflagged rays, matched by (ray, bounce) order (both ray-major)
        sel_o = ok[pa["ray"]]
        sel_g = ok[ray_gpu]
        np.testing.assert_array_equal(pa["ray"][sel_o], ray_gpu[sel_g])
        np.testing.assert_allclose(tau[:, sel_g], pa["tau"][:, sel_o], rtol=1e-13)
        np.testing.assert_allclose(amp[:, sel_g], pa["amp"][:, sel_o], rtol=2e-6,
                                   atol=1e-6 * np.abs(pa["amp"]).max())
    return pa


def test_sphere_320_tris_64x64(sbr):
    wl = sphere_scene()
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, wl.max_bounces)
    _, paths = gpu_trace(sbr, wl)
    check_paths(wl, tr, paths)


def test_corner_reflector_three_bounces(sbr):
    from tests.test_oracle_pins import axis_grid, corner_reflector
    C = np.array([0.25, 0.125, 2.0])
    v, f = corner_reflector(C, 0.75)
    wl = Workload("corner", v, f, radar_single_tx(), axis_grid(96, 0.12, axis=C), 3, {})
    tr = oracle.trace(v, f, wl.grid, 3)
    _, paths = gpu_trace(sbr, wl)
    pa = check_paths(wl, tr, paths)
    assert (pa["bounce"] == 2).sum() > 500


def test_superquadric_ground_reduced_grid(sbr):
    """20,002-triangle superquadric + ground, 3 bounces, 96x96 rays (all traced by the oracle)."""
    wl = superquadric_scene(seed=1, G=96)
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, 3)
    _, paths = gpu_trace(sbr, wl)
    check_paths(wl, tr, paths)


def test_superquadric_full_grid_sampled_rays(sbr):
    """The 1024x1024-ray configuration as traced in the bench; 3000 sampled rays vs the oracle."""
    wl = superquadric_scene(seed=0, G=1024)
    _, paths = gpu_trace(sbr, wl)
    ids = ray_subset(123, wl.grid.n_rays, 3000)
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, 3, ray_ids=ids)
    tri_gpu = paths.hits()[0].cpu().numpy()[ids]
    ok = tr["flag"] == 0
    assert ((tri_gpu[ok] != tr["tri"][ok]).any(axis=1)).sum() == 0
    # same rays traced alone (ray-id list) give the same records
    _, sub = gpu_trace(sbr, wl, ray_ids=ids)
    np.testing.assert_array_equal(sub.hits()[0].cpu().numpy(), tri_gpu)


def test_superquadric_full_grid_every_ray(sbr):
    """All 1,048,576 rays of the bench configuration against the oracle.  A few dozen of them
    graze the surface after a bounce and run past the traversal's hand-over threshold, so
    their search is finished by the cooperative (warp-per-ray) kernel: they must choose the
    same triangles as every other ray."""
    wl = superquadric_scene(seed=0, G=1024)
    _, paths = gpu_trace(sbr, wl)
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, 3)
    mism, n_ok, tri_gpu = compare_tri(tr, paths)
    assert mism == 0, f"{mism} of {n_ok} unflagged rays chose a different triangle"
    ok = tr["flag"] == 0
    hp = paths.hit_points().cpu().numpy()
    valid = (tr["tri"] >= 0) & ok[:, None]
    np.testing.assert_allclose(hp[valid], tr["hit"][valid], rtol=0, atol=1e-9)
    assert paths.count() == int((tri_gpu >= 0).sum())


def test_empty_and_ragged_inputs(sbr):
    # a mesh the rays miss, a single triangle, a ray list of length 1 and 0
    wl = sphere_scene(G=8)
    far = Workload("miss", wl.verts + np.float32([50, 0, 0]), wl.faces, wl.radar, wl.grid, 2, {})
    _, paths = gpu_trace(sbr, far)
    assert paths.count() == 0
    one = Workload("one", np.float32([[-1, -1, 1], [1, -1, 1], [0, 1, 1]]), np.int32([[0, 1, 2]]), wl.radar,
                   wl.grid, 2, {})
    tr = oracle.trace(one.verts, one.faces, one.grid, 2)
    _, paths = gpu_trace(sbr, one)
    check_paths(one, tr, paths)
    _, p1 = gpu_trace(sbr, wl, ray_ids=[27])
    tr1 = oracle.trace(wl.verts, wl.faces, wl.grid, 2, ray_ids=np.int32([27]))
    assert (p1.hits()[0].cpu().numpy() == tr1["tri"]).all()
    _, p0 = gpu_trace(sbr, wl, ray_ids=np.zeros(0, np.int32))
    assert p0.count() == 0


def test_bad_face_index_reported(sbr):
    wl = sphere_scene(G=8)
    bad = wl.faces.copy()
    bad[5, 1] = 10_000
    v = torch.from_numpy(wl.verts).cuda()
    f = torch.from_numpy(bad).cuda()
    scene = sbr.Scene(v, f)
    with pytest.raises(sbr.SbrError):
        scene.check()


@pytest.mark.parametrize("nt", [2, 1023, 1024, 1025, 2049, 5000])
def test_tree_tile_boundaries(sbr, nt):
    """Meshes whose triangle counts sit on and around the 1024-leaf tiles of the fused tree
    build: the first nt faces of a 20,480-face sphere (open, so rays also reach its inside)."""
    c = (0.05, -0.02, 1.3)
    v, f = icosphere(5, 0.25, c)
    wl = Workload("tiles", v, np.ascontiguousarray(f[:nt]), radar_single_tx(), ray_grid_for_sphere(c, 0.25, 40), 2,
                  {})
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, 2)
    _, paths = gpu_trace(sbr, wl)
    check_paths(wl, tr, paths)


def test_fused_build_with_key_window(sbr):
    """50,000 triangles: inside the fused build's limit but above the 38,912 sorted keys it holds
    in shared memory, so the tree searches read a window of keys and global memory beyond it."""
    c = (0.0, 0.03, 1.1)
    v, f = icosphere(6, 0.25, c)
    wl = Workload("window", v, np.ascontiguousarray(f[:50000]), radar_single_tx(), ray_grid_for_sphere(c, 0.25, 32),
                  2, {})
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, 2)
    _, paths = gpu_trace(sbr, wl)
    check_paths(wl, tr, paths)


def test_large_mesh_multi_cta_build(sbr):
    """81,920 triangles: above the fused build's limit, so the Morton sort runs over many CTAs
    and the tree is refitted by global arrival counters."""
    c = (0.0, 0.03, 1.1)
    v, f = icosphere(6, 0.25, c)
    assert len(f) > 65536
    wl = Workload("large", v, f, radar_single_tx(), ray_grid_for_sphere(c, 0.25, 32), 2, {})
    tr = oracle.trace(wl.verts, wl.faces, wl.grid, 2)
    _, paths = gpu_trace(sbr, wl)
    check_paths(wl, tr, paths)


def test_jittered_sampling_matches_oracle(sbr):
    """Stratified jittered rays (seeded offsets inside each cell, Eq. 3): triangle indices
    bit-exact, hit points, delays and strengths against the oracle, on the sphere and on a
    superquadric subset; offsets of 1/2 give the cell-centre trace bitwise."""
    import dataclasses
    from sbr_inputs import jittered
    wl = sphere_scene(G=64)
    wj = dataclasses.replace(wl, grid=jittered(wl.grid, 9))
    tr = oracle.trace(wj.verts, wj.faces, wj.grid, wj.max_bounces)
    _, paths = gpu_trace(sbr, wj)
    check_paths(wj, tr, paths)
    assert not np.array_equal(tr["omega"], oracle.trace(wl.verts, wl.faces, wl.grid, 2)["omega"])
    half = dataclasses.replace(wl, grid=dataclasses.replace(wl.grid, jitter=np.full((64 * 64, 2), 0.5, np.float32)))
    _, p_half = gpu_trace(sbr, half)
    _, p_ctr = gpu_trace(sbr, wl)
    assert torch.equal(p_half.hits()[0], p_ctr.hits()[0])
    assert torch.equal(p_half.prep()[:, :p_ctr.count()], p_ctr.prep()[:, :p_ctr.count()])
    sq = superquadric_scene(seed=2, G=512)
    sqj = dataclasses.replace(sq, grid=jittered(sq.grid, 4))
    ids = ray_subset(8, sqj.grid.n_rays, 3000)
    tr = oracle.trace(sqj.verts, sqj.faces, sqj.grid, 3, ray_ids=ids)
    _, paths = gpu_trace(sbr, sqj, ray_ids=ids)
    check_paths(sqj, tr, paths)


@pytest.mark.parametrize("nt", [20002, 65536])
def test_fused_build_is_taken(sbr, nt):
    """The one-launch cooperative build (k_build_scene, then the 4-wide collapse: two launches)
    runs for the bench mesh and at its size limit: its shared memory fits a CTA, so it does not
    fall back to the multi-kernel build."""
    from sbr_inputs import superquadric_scene
    if nt == 20002:
        wl = superquadric_scene(seed=0, G=32)
        v, f = wl.verts, wl.faces
    else:
        v, f = icosphere(6, 0.25, (0.0, 0.0, 1.0))
        f = np.ascontiguousarray(f[:nt])
    vt, ft = torch.from_numpy(v).cuda(), torch.from_numpy(f).cuda()
    scene = sbr.Scene(vt, ft)
    L = sbr.load()
    torch.cuda.synchronize()
    n0 = int(L.sbr_launch_count())
    scene.update(vt)
    torch.cuda.synchronize()
    assert int(L.sbr_launch_count()) - n0 == 2


@pytest.mark.parametrize("G", [64, 200])
def test_trace_counts_variant(sbr, G):
    """sbr_trace_counts (the counting variant of the trace, warp per ray at 64^2 rays, thread per
    ray at 200^2): the same hits as sbr_trace, and exactly one traversal per ray and bounce until
    the ray's first miss; node and triangle counts positive."""
    from sbr_inputs import superquadric_scene
    wl = superquadric_scene(seed=2, G=G)
    v, f = torch.from_numpy(wl.verts).cuda(), torch.from_numpy(wl.faces).cuda()
    scene = sbr.Scene(v, f)
    a = sbr.trace(scene, wl.radar, wl.grid, wl.max_bounces)
    b = sbr.PathBuffers(wl.grid.n_rays, wl.max_bounces, wl.radar.n_virt)
    counts = sbr.sim.trace_counts(scene, wl.radar, wl.grid, wl.max_bounces, out=b)
    torch.cuda.synchronize()
    assert torch.equal(a.hits()[0], b.hits()[0])
    nh = (a.hits()[0] >= 0).sum(dim=1).cpu().numpy()
    expect = int(np.minimum(nh + 1, wl.max_bounces).sum())
    nodes, tris, trav = counts
    assert trav == expect and nodes > 0 and tris > 0


@pytest.mark.parametrize("kind", ["cluster", "cooperative", "multi-kernel"])
def test_refit_same_hits_as_rebuild(sbr, kind):
    """sbr_scene_refit keeps the last build's tree and recomputes its boxes for moved vertices:
    the trace then finds exactly what a scene built from the moved vertices finds (hits,
    float-float hit points, paths), on the three build paths (a cluster of up to 16 tiles, the
    cooperative launch, the multi-kernel build above 65,536 triangles)."""
    from sbr_inputs import superquadric_scene
    if kind == "cluster":
        v, f = icosphere(4, 0.25, (0.0, 0.02, 1.2))
        grid = ray_grid_for_sphere((0.0, 0.02, 1.2), 0.3, 96)
    elif kind == "cooperative":
        wl0 = superquadric_scene(seed=4, G=96)
        v, f, grid = wl0.verts, wl0.faces, wl0.grid
    else:
        v, f = icosphere(6, 0.25, (0.0, 0.03, 1.1))
        grid = ray_grid_for_sphere((0.0, 0.03, 1.1), 0.3, 64)
    radar = radar_single_tx()
    rng = np.random.default_rng(8)
    v1 = (v + rng.normal(scale=2e-3, size=v.shape) + np.array([0.01, -0.02, 0.05])).astype(np.float32)
    vt, ft, v1t = torch.from_numpy(v).cuda(), torch.from_numpy(f).cuda(), torch.from_numpy(v1).cuda()
    refit = sbr.Scene(vt, ft)
    L = sbr.load()
    torch.cuda.synchronize()
    n0 = int(L.sbr_launch_count())
    refit.refit(v1t)
    torch.cuda.synchronize()
    if kind != "multi-kernel":
        assert int(L.sbr_launch_count()) - n0 == 2  # the refit kernel and the 4-wide collapse
    refit.check()
    fresh = sbr.Scene(v1t, ft)
    a = sbr.trace(refit, radar, grid, 2)
    b = sbr.trace(fresh, radar, grid, 2)
    torch.cuda.synchronize()
    assert a.count() == b.count() > 0
    assert torch.equal(a.hits()[0], b.hits()[0])
    assert torch.equal(a.hit_pos(), b.hit_pos())
    P = a.count()
    assert torch.equal(a.prep()[:, :P], b.prep()[:, :P])  # the records written (the rest is scratch)
