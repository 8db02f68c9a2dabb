"""Host logic of the serving layer without a GPU: the offset arena that places every
request's device buffers, and the admission footprint query."""
import numpy as np
import pytest

from sbr_inputs import CfarParams, radar_single_tx, ray_grid_for_sphere, serving_workload, sphere_scene


@pytest.fixture(scope="module")
def serving():
    from paper_2311_13182_gb300 import build
    build.build()
    from paper_2311_13182_gb300 import serving as s
    return s


def test_arena_first_fit_and_coalescing(serving):
    a = serving.Arena(1 << 20)
    offs = [a.alloc(1000) for _ in range(8)]
    assert offs == [i * 1024 for i in range(8)]          # 256-byte granules, first fit
    assert a.used() == 8 * 1024
    a.free(offs[1], 1000)
    a.free(offs[3], 1000)
    assert a.alloc(2000) == 8 * 1024                      # neither 1 KiB hole fits 2 KiB
    a.free(offs[2], 1000)                                 # 1, 2, 3 merge into one 3 KiB hole
    assert a.alloc(3000) == 1024
    assert a.peak() >= a.used()
    for o in (0, 4 * 1024, 5 * 1024, 6 * 1024, 7 * 1024):
        a.free(o, 1000)
    a.free(1024, 3000)
    a.free(8 * 1024, 2000)
    assert a.used() == 0 and a.largest_free() == 1 << 20  # everything merged back


def test_arena_exhaustion_and_random_churn(serving):
    a = serving.Arena(64 * 1024)
    assert a.alloc(65 * 1024) == -1
    rng = np.random.default_rng(0)
    live = {}
    for step in range(2000):
        if live and rng.random() < 0.5:
            off = rng.choice(list(live))
            a.free(off, live.pop(off))
        else:
            n = int(rng.integers(1, 4096))
            off = a.alloc(n)
            if off >= 0:
                # no overlap with any live block
                for o, m in live.items():
                    assert off + n <= o or o + m <= off
                live[off] = n
    assert a.used() == sum(((n + 255) // 256) * 256 for n in live.values())
    for o, n in list(live.items()):
        a.free(o, n)
    assert a.used() == 0 and a.largest_free() == 64 * 1024


def test_request_footprint_query_grows_with_budget(serving):
    import ctypes
    from paper_2311_13182_gb300 import sim
    lib = serving._declare()
    radar, cfg = radar_single_tx(), CfarParams()
    wl = sphere_scene(G=64)
    small = serving.Request()
    small.kind, small.max_bounces, small.nv, small.nt = serving.FORWARD, 2, 162, 320
    small.grid = sim.grid_struct(wl.grid)
    big = serving.Request()
    big.kind, big.max_bounces, big.nv, big.nt = serving.RECON, 2, 2562, 5120
    big.grid = sim.grid_struct(ray_grid_for_sphere((0, 0, 1), 0.2, 256))
    big.n_target = 100
    r, c = sim.radar_struct(radar), sim.cfar_struct(cfg)
    b_small = lib.sbr_server_request_bytes(ctypes.byref(r), ctypes.byref(c), ctypes.byref(small))
    b_big = lib.sbr_server_request_bytes(ctypes.byref(r), ctypes.byref(c), ctypes.byref(big))
    assert 0 < b_small < b_big
    # the path records of a 4096-ray, 2-bounce request dominate its footprint
    assert b_small >= lib.sbr_paths_bytes(4096, 2, 4)


def test_serving_workload_is_seeded_and_shaped():
    m1, r1 = serving_workload(3, n=200, pool=16)
    m2, r2 = serving_workload(3, n=200, pool=16)
    assert m1 == m2 and r1 == r2
    assert all(1_000 <= m["n_tris"] <= 200_000 for m in m1)
    assert all(256 <= q["G"] <= 2048 for q in r1)
    kinds = [q["kind"] for q in r1]
    assert 0.35 < kinds.count("forward") / len(kinds) < 0.65


def test_device_overlap_of_intervals():
    from paper_2311_13182_gb300.serving import device_overlap
    d = lambda a, b: dict(status=0, gpu_t0_ms=a, gpu_t1_ms=b)
    # [0, 4] and [2, 6]: busy 6 ms, two at once on [2, 4]
    o = device_overlap([d(0, 4), d(2, 6)])
    assert o["busy_ms"] == 6 and abs(o["two_or_more_frac"] - 2 / 6) < 1e-12
    # disjoint intervals never overlap; failed requests are ignored
    o = device_overlap([d(0, 1), d(2, 3), dict(status=4, gpu_t0_ms=0, gpu_t1_ms=3)])
    assert o["busy_ms"] == 2 and o["two_or_more_frac"] == 0
    # three nested
    o = device_overlap([d(0, 10), d(1, 9), d(2, 3)])
    assert o["busy_ms"] == 10 and abs(o["two_or_more_frac"] - 0.8) < 1e-12
