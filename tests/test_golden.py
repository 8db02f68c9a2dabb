"""Stored expected values (tests/golden/, written from the FP64 oracle by
tests/golden/make_golden.py): the oracle must still reproduce them, and the CUDA
path must match them within the parity bars (triangle ids bit-exact on rays the
oracle does not flag, IF cube relative L2 <= 1e-4, point cloud Chamfer <= 1 mm)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)


def stored():
    tr = load("sphere_g16_trace.txt").astype(np.int64)
    pa = load("sphere_g16_paths.txt")
    cu = load("sphere_g16_cube.txt")
    V, Ns = int(cu[:, 0].max()) + 1, int(cu[:, 1].max()) + 1
    cube = (cu[:, 2] + 1j * cu[:, 3]).reshape(V, Ns)
    P = pa.shape[0] // V
    return dict(tri=tr[:, 1:3], flag=tr[:, 3], tau=pa[:, 3].reshape(V, P), amp=pa[:, 4].reshape(V, P),
                ray=pa[:P, 1].astype(np.int64), bounce=pa[:P, 2].astype(np.int64), cube=cube,
                points=load("sphere_g64_points.txt"))


def test_oracle_reproduces_golden():
    from tests.golden.make_golden import compute
    g, d = stored(), compute()
    np.testing.assert_array_equal(d["tri"], g["tri"])
    np.testing.assert_array_equal(d["flag"], g["flag"])
    np.testing.assert_array_equal(d["ray"], g["ray"])
    np.testing.assert_array_equal(d["bounce"], g["bounce"])
    np.testing.assert_allclose(d["tau"], g["tau"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(d["amp"], g["amp"], rtol=1e-12, atol=0)
    assert np.linalg.norm(d["cube"] - g["cube"]) <= 1e-12 * np.linalg.norm(g["cube"])
    assert d["points"].shape == g["points"].shape
    np.testing.assert_allclose(d["points"], g["points"], rtol=0, atol=1e-9)


def test_golden_files_are_consistent():
    """Shapes and the structure the fixtures must have: 256 rays x 2 bounces, one path per
    hit and antenna, hits ordered ray-major, 4 x 256 samples, weights in (0.01, 1]."""
    g = stored()
    assert g["tri"].shape == (256, 2) and g["cube"].shape == (4, 256)
    hits = np.argwhere(g["tri"] >= 0)
    np.testing.assert_array_equal(hits[:, 0], g["ray"])
    np.testing.assert_array_equal(hits[:, 1], g["bounce"])
    assert (g["tau"] > 0).all() and g["points"].shape[1] == 4
    assert ((g["points"][:, 3] >= 0.01) & (g["points"][:, 3] <= 1.0)).all()
    # a hit's second bounce exists only after a first one
    assert not ((g["tri"][:, 0] < 0) & (g["tri"][:, 1] >= 0)).any()


@pytest.mark.gpu
def test_cuda_path_matches_golden(sbr):
    from oracle import pointcloud as opc
    from sbr_inputs import CfarParams, sphere_scene
    from tests._util import cube_complex, gpu_trace, rel_l2
    g = stored()
    wl = sphere_scene(G=16)
    _, paths = gpu_trace(sbr, wl)
    tri = paths.hits()[0].cpu().numpy()
    ok = g["flag"] == 0
    assert ok.sum() > 200
    np.testing.assert_array_equal(tri[ok], g["tri"][ok])
    cube = cube_complex(sbr.synthesize(paths, wl.radar))[:, 0, :]
    assert rel_l2(cube, g["cube"]) <= 1e-4
    wl64 = sphere_scene(G=64)
    _, p64 = gpu_trace(sbr, wl64)
    pts, st = sbr.pointcloud(sbr.synthesize(p64, wl64.radar), wl64.radar, CfarParams())
    n = st.n_points()
    got = pts.cpu().numpy()[:n].astype(np.float64)
    assert n > 0 and opc.chamfer_parity(got, g["points"]) <= 1e-3


def test_oracle_reproduces_precision_sweep():
    """The stored long-range sweep (sphere at 5/10/20 m, 1024-4096 samples, 4096 seeded rays
    of the 2048 x 2048 grid) is what the oracle computes now."""
    from tests.golden.make_golden import SWEEP_FILE, compute_sweep
    g = np.load(os.path.join(GOLDEN, SWEEP_FILE))
    d = compute_sweep()
    assert sorted(g.files) == sorted(d)
    for k in d:
        if k.startswith("cube_"):
            assert np.linalg.norm(d[k] - g[k]) <= 1e-12 * np.linalg.norm(g[k]), k
        elif k.startswith("points_"):
            assert d[k].shape == g[k].shape, k
            np.testing.assert_allclose(d[k], g[k], rtol=0, atol=1e-9, err_msg=k)
        else:
            assert int(d[k]) == int(g[k]), k
