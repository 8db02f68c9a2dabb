"""Helpers shared by the GPU parity tests (inputs and comparisons, no method arithmetic)."""
import numpy as np
import torch


def to_dev(wl, device="cuda"):
    v = torch.from_numpy(np.ascontiguousarray(wl.verts, dtype=np.float32)).to(device)
    f = torch.from_numpy(np.ascontiguousarray(wl.faces, dtype=np.int32)).to(device)
    return v, f


def gpu_trace(sbr, wl, ray_ids=None, K=None):
    v, f = to_dev(wl)
    scene = sbr.Scene(v, f)
    ids = None if ray_ids is None else torch.from_numpy(np.asarray(ray_ids, np.int32)).cuda()
    paths = sbr.trace(scene, wl.radar, wl.grid, K or wl.max_bounces, ids)
    torch.cuda.synchronize()
    scene.check()
    return scene, paths


def cube_complex(cube_t):
    c = cube_t.double().cpu().numpy()
    return c[..., 0] + 1j * c[..., 1]


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def compare_tri(tr, paths):
    """Exact triangle-index comparison on rays the oracle did not flag as edge/tie-near."""
    tri_gpu = paths.hits()[0].cpu().numpy()
    ok = tr["flag"] == 0
    mism = (tri_gpu[ok] != tr["tri"][ok]).any(axis=1)
    return int(mism.sum()), int(ok.sum()), tri_gpu
