"""Serving on the GPU: results are the same alone and in the mix, admission respects a
tight HBM budget, resident BVHs / IF cubes are reused, cancellation and host-side faults."""
import numpy as np
import pytest
import torch

from sbr_inputs import (CfarParams, bounding_sphere, icosphere, perturbed_icosphere, radar_single_tx,
                        ray_grid_for_sphere, superquadric)

pytestmark = pytest.mark.gpu

RADAR = radar_single_tx()
CFG = CfarParams()


def mesh(i):
    if i % 2:
        v, f, _ = superquadric(100 + i, n_lon=30, n_rings=30, center=(0.0, 0.0, 1.5 + 0.1 * i))
    else:
        v, f = perturbed_icosphere(200 + i, 3, 0.25, (0.0, 0.0, 1.2 + 0.1 * i))
    return v, f


def items(n=8, iters=4):
    from paper_2311_13182_gb300 import serving as S
    out = []
    for i in range(n):
        v, f = mesh(i)
        c, r = bounding_sphere(v)
        grid = ray_grid_for_sphere(c, r, 96 + 32 * (i % 3))
        if i % 3 == 2:
            target = S.plain_forward(v, f, RADAR, CFG, grid, 2)
            tmpl = (c + 0.9 * (v.astype(np.float64) - c)).astype(np.float32)
            out.append(dict(kind=S.RECON, verts=tmpl, faces=f, grid=grid, max_bounces=2, iterations=iters,
                            target=target, lr=1e-3, lap_weight=0.1, want_verts=True))
        else:
            out.append(dict(kind=S.FORWARD, verts=v, faces=f, grid=grid, max_bounces=2, mesh_id=i + 1))
    return out


def run(items_, arena=1 << 30, slots=4):
    from paper_2311_13182_gb300 import serving as S
    srv = S.Server(RADAR, CFG, arena, n_slots=slots)
    tickets = [srv.submit(**it) for it in items_]
    res = {r["ticket"]: r for r in srv.drain(300)}
    stats = srv.stats()
    srv.close()
    return [res[t] for t in tickets], stats


def test_alone_equals_mix(sbr):
    its = items()
    mix, stats = run(its, slots=4)
    assert all(r["status"] == 0 for r in mix)
    for it, m in zip(its, mix):
        alone, _ = run([it], slots=1)
        a = alone[0]
        assert a["status"] == 0 and a["n_points"] == m["n_points"]
        # every kernel, adjoints included, is deterministic: bitwise equal alone and in the mix
        np.testing.assert_array_equal(a["points"], m["points"])
        if it["kind"] == 1:
            assert a["loss"] == m["loss"]
            np.testing.assert_array_equal(a["verts"], m["verts"])


def test_served_forward_equals_plain_forward(sbr):
    from paper_2311_13182_gb300 import serving as S
    it = items(2)[1]
    res, _ = run([it])
    plain = S.plain_forward(it["verts"], it["faces"], RADAR, CFG, it["grid"], 2)
    np.testing.assert_array_equal(res[0]["points"], plain[: res[0]["n_points"]])


def test_tight_budget_admission(sbr):
    from paper_2311_13182_gb300 import serving as S
    its = [it for it in items(8) if it["kind"] == 0]
    probe = S.Server(RADAR, CFG, 1 << 30, n_slots=1)
    need = max(probe.request_bytes(**{k: v for k, v in it.items()}) for it in its)
    probe.close()
    budget = int(need * 2.2)          # room for two requests at a time, not more
    res, stats = run(its, arena=budget, slots=8)
    assert all(r["status"] == 0 for r in res)
    assert stats["peak_bytes"] <= budget
    # at most two ran at once: admission intervals overlap pairwise at most
    iv = sorted((r["t_admit_us"], r["t_done_us"]) for r in res)
    for i in range(len(iv)):
        overlapping = sum(1 for j in range(len(iv)) if iv[j][0] < iv[i][1] and iv[i][0] < iv[j][1])
        assert overlapping <= 3   # itself + at most two others across its lifetime boundaries


def test_resident_scene_and_cube_reuse(sbr):
    from paper_2311_13182_gb300 import serving as S
    v, f = mesh(1)
    c, r = bounding_sphere(v)
    g1, g2 = ray_grid_for_sphere(c, r, 64), ray_grid_for_sphere(c, r, 80)
    srv = S.Server(RADAR, CFG, 1 << 30, n_slots=2)
    res = []
    for g in (g1, g1, g2):
        t = srv.submit(kind=S.FORWARD, verts=v, faces=f, grid=g, max_bounces=2, mesh_id=77)
        res += srv.drain(60)
    st = srv.stats()
    srv.close()
    assert [x["scene_cached"] for x in res] == [False, True, True]
    assert [x["cube_cached"] for x in res] == [False, True, False]
    np.testing.assert_array_equal(res[0]["points"], res[1]["points"])
    plain = S.plain_forward(v, f, RADAR, CFG, g2, 2)
    np.testing.assert_array_equal(res[2]["points"], plain[: res[2]["n_points"]])
    assert st["cached_scenes"] == 1 and st["cached_cubes"] == 2 and st["cache_hits"] == 2


def test_cancel_and_host_side_faults(sbr):
    from paper_2311_13182_gb300 import serving as S
    from paper_2311_13182_gb300 import SbrError
    its = items(3)
    srv = S.Server(RADAR, CFG, 1 << 30, n_slots=1)
    t = [srv.submit(**it) for it in its]
    srv.cancel(t[2])                       # not yet admitted: no poll has run
    res = {r["ticket"]: r for r in srv.drain(120)}
    assert res[t[2]]["status"] == 6 and res[t[0]]["status"] == 0 and res[t[1]]["status"] == 0
    with pytest.raises(SbrError):
        srv.cancel(t[0])                   # already finished
    v, f = mesh(0)
    bad = f.copy()
    bad[3, 1] = v.shape[0] + 5             # out-of-range vertex index
    with pytest.raises(SbrError) as e:
        srv.submit(kind=S.FORWARD, verts=v, faces=bad, grid=its[0]["grid"], max_bounces=2)
    assert e.value.status == 1
    vn = v.copy()
    vn[7, 2] = np.nan                      # non-finite vertex
    with pytest.raises(SbrError):
        srv.submit(kind=S.FORWARD, verts=vn, faces=f, grid=its[0]["grid"], max_bounces=2)
    srv.close()
    tiny = S.Server(RADAR, CFG, 1 << 20, n_slots=1)   # 1 MiB arena: any request is larger
    with pytest.raises(SbrError) as e:
        tiny.submit(**its[0])
    assert e.value.status == 2
    # the server keeps working after rejected submissions
    ok = tiny.stats()
    assert ok["submitted"] == 0
    tiny.close()
