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
