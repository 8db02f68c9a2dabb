"""The forward step captured as one CUDA graph (sbr.Forward) gives what its separate launches
give, on the first replay and after the vertices move."""
import numpy as np
import pytest
import torch

from sbr_inputs import CfarParams, superquadric_scene

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager(sbr):
    wl = superquadric_scene(seed=6, G=256)
    cfg = CfarParams()
    v = torch.from_numpy(wl.verts).cuda()
    f = torch.from_numpy(wl.faces).cuda()
    g = sbr.Forward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg)
    e = sbr.Forward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, graph=False)
    for shift in (0.0, 0.01):  # then the whole mesh moved 1 cm along the boresight
        moved = v + torch.tensor([0.0, 0.0, shift], device="cuda")
        g.set_vertices(moved)
        e.set_vertices(moved)
        g.run()
        e.run()
        torch.cuda.synchronize()
        assert g.n_points() == e.n_points() > 0
        assert torch.equal(g.cube, e.cube)
        assert torch.equal(g.points, e.points)
    # the moved scene's nearest points are ~1 cm farther
    r_moved = np.linalg.norm(g.points[:g.n_points(), :3].cpu().numpy(), axis=1)
    assert r_moved.min() > 0


def test_host_io_graph_matches_eager(sbr):
    """Forward(host_io=True).run_host: the graph copies the vertices in and the points and their
    count out; the host buffers hold exactly what the separate launches compute, for the first
    vertex set and after new host vertices (moved 1 cm) go in."""
    wl = superquadric_scene(seed=6, G=256)
    cfg = CfarParams()
    v = torch.from_numpy(wl.verts).cuda()
    f = torch.from_numpy(wl.faces).cuda()
    h = sbr.Forward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, host_io=True)
    e = sbr.Forward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, graph=False)
    for shift in (0.0, 0.01):
        moved = wl.verts + np.array([0.0, 0.0, shift], np.float32)
        h.run_host(moved)
        e.set_vertices(torch.from_numpy(moved).cuda())
        e.run()
        h.done.synchronize()
        torch.cuda.synchronize()
        n = int(h.h_n.item())
        assert n == e.n_points() > 0
        assert torch.equal(h.h_points, e.points.cpu())
    with pytest.raises(RuntimeError):
        e.run_host(wl.verts)


@pytest.mark.parametrize("depth", [3, 4])
def test_pipelined_lags(sbr, depth):
    """sbr.PipelinedForward: step j traces batch j's tree beside the build of batch j+1 and the
    synthesis (depth 4) and point cloud of earlier batches.  With the vertices moving every step,
    step j's points equal (bitwise) those the serial step gives for the vertices set before step
    j - (depth - 1) (earlier steps: the constructor's), replayed from the two graphs, run eagerly,
    and with host buffers; the cube synthesized at step j is the serial cube of the vertices set
    before step j - depth + 2."""
    wl = superquadric_scene(seed=6, G=256)
    cfg = CfarParams()
    v = torch.from_numpy(wl.verts).cuda()
    f = torch.from_numpy(wl.faces).cuda()
    e = sbr.Forward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, graph=False)
    kw = dict(depth=depth)
    pg = sbr.PipelinedForward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, **kw)
    pe = sbr.PipelinedForward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, graph=False, **kw)
    ph = sbr.PipelinedForward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, host_io=True, **kw)
    shifts = [0.0, 0.01, 0.03, -0.02, 0.02]
    want = []
    for sh in shifts:  # the serial step's outputs per vertex set
        e.set_vertices(v + torch.tensor([0.0, 0.0, sh], device="cuda"))
        e.run()
        torch.cuda.synchronize()
        want.append((e.cube.clone(), e.points.clone(), e.n_points()))
    seq = shifts + [0.0] * depth  # the vertex set given before each step
    out = dict(zip(shifts, want))

    def given(k):  # the vertex set before step k (the constructor's before step 0)
        return seq[k] if k >= 0 else 0.0

    for j, sh in enumerate(seq):
        moved = v + torch.tensor([0.0, 0.0, sh], device="cuda")
        for fw in (pg, pe):
            fw.set_vertices(moved)
            fw.run()
        ph.run_host(moved.cpu().numpy())
        ph.done.synchronize()
        torch.cuda.synchronize()
        _, pts, n = out[given(j - depth + 1)]
        synthesized = out[given(j - depth + 2)][0]
        assert n > 0
        for fw in (pg, pe):
            assert fw.n_points() == n
            assert torch.equal(fw.points, pts)
            assert torch.equal(fw.synthesized(), synthesized)
        assert int(ph.h_n.item()) == n
        assert torch.equal(ph.h_points, pts.cpu())
    with pytest.raises(RuntimeError):
        pe.run_host(wl.verts)
    with pytest.raises(ValueError):
        sbr.PipelinedForward(v, f, wl.radar, wl.grid, wl.max_bounces, cfg, graph=False, depth=5)


def test_bench_step_full_cube_and_points_against_oracle(sbr):
    """The bench workload at full size (20,002 triangles, all 1,048,576 rays, 3 bounces,
    12 x 128 x 256 cube), run as the bench runs it (the graph-replayed sbr.Forward step):
    every ray traced and every path summed by the FP64 oracle.  IF cube relative L2 <= 1e-4
    and point cloud Chamfer <= 1 mm."""
    import oracle
    from oracle import pointcloud as opc
    from tests._util import cube_complex, rel_l2
    wl = superquadric_scene(seed=0, G=1024)
    cfg = CfarParams()
    fw = sbr.Forward(torch.from_numpy(wl.verts).cuda(), torch.from_numpy(wl.faces).cuda(), wl.radar, wl.grid,
                     wl.max_bounces, cfg)
    fw.run()
    torch.cuda.synchronize()
    ref, _, pa = oracle.simulate_cube(wl)
    assert fw.paths.count() == pa["P"]
    err = rel_l2(cube_complex(fw.cube), ref)
    ref_pts = opc.pointcloud(ref, wl.radar, cfg)["points"]
    n = fw.n_points()
    got = fw.points[:n].cpu().numpy().astype(np.float64)
    ch = opc.chamfer_parity(got, ref_pts)
    print(f"\nbench workload: {pa['P']} paths, cube rel L2 {err:.2e}, {n} points, Chamfer {ch:.2e} m")
    assert err <= 1e-4
    assert n > 0 and ch <= 1e-3
