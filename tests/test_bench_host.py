"""bench.py's host-side bookkeeping on CPU: the roofline objects of the JSON line,
the ncu CSV -> per-stage DRAM traffic reduction, and the guard that drops stored
traffic once a stage's sources change."""
import json
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def workload(V=12, Ns=256, R=1 << 20, K=3):
    return types.SimpleNamespace(radar=types.SimpleNamespace(n_virt=V, n_samples=Ns),
                                 grid=types.SimpleNamespace(n_rays=R), max_bounces=K)


PEAKS = {"hbm_gbs": 6794.1, "bf16_tflops": 1899.0, "sm_max_mhz": 2070.0}


def test_rooflines_units_and_dominant_stage():
    wl = workload()
    P, counts = 471630, (6467118, 2506060, 1511588)
    dom, (trace, synth) = bench.rooflines({"trace": 0.33, "synthesize": 0.12}, wl, P, counts, PEAKS, "measured")
    assert dom is trace and trace["bound"] == "hbm" and trace["unit"] == "GB/s"
    tb = counts[0] * 112 + counts[1] * 48 + wl.grid.n_rays * 3 * 48 + wl.grid.n_rays * 8 + P * 12 * 24 + P * 4
    assert trace["bytes_per_launch"] == tb
    assert abs(trace["achieved"] - tb / 0.33e-3 / 1e9) < 1e-6 * trace["achieved"]
    assert abs(trace["frac"] - trace["achieved"] / PEAKS["hbm_gbs"]) < 1e-12
    # synthesis: Eq. 8 terms per second against 152 x 128 FP32 lanes x f_max / 4
    terms = P * 12 * 256
    assert synth["terms_per_launch"] == terms and synth["unit"] == "terms/s"
    assert abs(synth["peak"] - 152 * 128 * 2070e6 / 4) < 1.0
    assert abs(synth["frac"] - terms / 0.12e-3 / synth["peak"]) < 1e-12
    assert synth["grid_updates_per_launch"] == P * 12 * 8
    # a synthesis stage slower than the trace becomes the dominant one
    dom2, _ = bench.rooflines({"trace": 0.1, "synthesize": 0.2}, wl, P, counts, PEAKS, "measured")
    assert dom2["kernel"].startswith("k_nufft_spread")


def test_write_traffic_and_source_guard(tmp_path, monkeypatch):
    # a small ncu CSV: two launches of each trace kernel, one of each synthesis kernel
    rows = [["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]]
    lid = 0
    for name, n in (("k_trace", 2), ("k_prep", 2), ("k_nufft_spread", 1), ("k_nufft_finish", 1), ("k_reduce", 1)):
        for _ in range(n):
            rows.append([str(lid), f"void sbr::<unnamed>::{name}<0>(float*)", "dram__bytes_read.sum", "Mbyte", "1.5"])
            rows.append([str(lid), f"void sbr::<unnamed>::{name}<0>(float*)", "dram__bytes_write.sum", "Kbyte", "500"])
            lid += 1
    csv_path = tmp_path / "traffic.csv"
    csv_path.write_text("==PROF== noise line\n" + "\n".join(",".join(f'"{c}"' for c in r) for r in rows) + "\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    hashes = {st: bench.sources_sha1(st) for st in bench.TRAFFIC_SOURCES}  # of the real sources
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_sha1", lambda st: hashes[st])
    bench.write_traffic(str(csv_path))
    out = json.loads((prof / "traffic.json").read_text())["stages"]
    # per launch: trace = (2 k_trace + 2 k_prep) x 2 MB / 2 launches; synthesis = 3 x 2 MB / 1 launch
    assert abs(out["trace"]["bytes_per_launch"] - 4e6) < 1.0 and out["trace"]["launches"] == 2
    assert abs(out["synthesize"]["bytes_per_launch"] - 6e6) < 1.0 and out["synthesize"]["launches"] == 1
    assert set(bench.measured_traffic()) == {"trace", "synthesize"}
    # a stored hash that no longer matches the sources drops that stage
    d = json.loads((prof / "traffic.json").read_text())
    d["stages"]["trace"]["sources_sha1"] = "0" * 40
    (prof / "traffic.json").write_text(json.dumps(d))
    assert set(bench.measured_traffic()) == {"synthesize"}
