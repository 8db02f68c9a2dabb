"""bench.py's host-side bookkeeping on CPU: the roofline objects of the JSON line,
the ncu CSV -> per-stage counter reduction (DRAM bytes, warp instructions), and the
guard that drops stored counters once a stage's sources change."""
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


def test_rooflines_units_and_dominant_stage(monkeypatch):
    wl = workload()
    P, counts = 471630, (6467118, 2506060, 1511588)
    tb = counts[0] * 112 + counts[1] * 48 + wl.grid.n_rays * 3 * 48 + wl.grid.n_rays * 8 + P * 12 * 24 + P * 4
    ctr = {"trace": {"inst_per_launch": 1.5e8, "dram_bytes_per_launch": 2.4e8},
           "synthesize": {"inst_per_launch": 8.0e7, "dram_bytes_per_launch": 9.4e7}}
    monkeypatch.setattr(bench, "measured_counters", lambda: ctr)
    dom, (trace, synth) = bench.rooflines({"trace": 0.33, "synthesize": 0.12}, wl, P, counts, PEAKS, "measured")
    peak = 152 * 4 * 2070e6
    assert dom is trace and trace["bound"] == "alu" and trace["unit"] == "warp-inst/s"
    assert abs(trace["peak"] - peak) < 1.0
    assert abs(trace["achieved"] - 1.5e8 / 0.33e-3) < 1e-6 * trace["achieved"]
    assert abs(trace["frac"] - 1.5e8 / 0.33e-3 / peak) < 1e-12
    assert trace["traffic"] == 2.4e8
    assert abs(trace["dram"]["frac_of_hbm"] - 2.4e8 / 0.33e-3 / 1e9 / PEAKS["hbm_gbs"]) < 1e-12
    assert trace["served"]["bytes_per_launch"] == tb
    assert abs(trace["served"]["achieved_gbs"] - tb / 0.33e-3 / 1e9) < 1e-6 * trace["served"]["achieved_gbs"]
    # synthesis: issue slots as the bound; Eq. 8 terms against the direct-sum bound as a speed-up only
    terms = P * 12 * 256
    assert synth["terms_per_launch"] == terms and synth["unit"] == "warp-inst/s"
    assert abs(synth["frac"] - 8.0e7 / 0.12e-3 / peak) < 1e-12
    sp = synth["speedup_vs_direct_sum"]
    assert abs(sp["direct_sum_bound_terms_per_s"] - 152 * 128 * 2070e6 / 4) < 1.0
    assert abs(sp["ratio"] - terms / 0.12e-3 / sp["direct_sum_bound_terms_per_s"]) < 1e-12
    assert synth["grid_updates_per_launch"] == P * 12 * 8
    # a synthesis stage slower than the trace becomes the dominant one
    dom2, _ = bench.rooflines({"trace": 0.1, "synthesize": 0.2}, wl, P, counts, PEAKS, "measured")
    assert dom2["kernel"].startswith("k_nufft_spread")
    # without counters for the current sources: the bytes-served figure stands in, labelled
    monkeypatch.setattr(bench, "measured_counters", lambda: {})
    dom3, (t3, s3) = bench.rooflines({"trace": 0.33, "synthesize": 0.12}, wl, P, counts, PEAKS, "measured")
    assert t3["bound"] == "hbm" and t3["unit"] == "GB/s" and "absent" in t3["limiter"]
    assert abs(t3["frac"] - tb / 0.33e-3 / 1e9 / PEAKS["hbm_gbs"]) < 1e-12
    assert s3["bound"] == "hbm" and s3["achieved"] == s3["records"]["achieved_gbs"]


def test_write_counters_and_source_guard(tmp_path, monkeypatch):
    # one ncu CSV per captured kernel, two launches each
    prof = tmp_path / "profiles"
    prof.mkdir()
    paths = []
    for name in ("k_trace", "k_prep", "k_nufft_spread", "k_nufft_finish", "k_reduce"):
        rows = [["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]]
        for lid in range(2):
            kn = f"void sbr::<unnamed>::{name}<0>(float*)"
            rows.append([str(lid), kn, "dram__bytes_read.sum", "Mbyte", "1.5"])
            rows.append([str(lid), kn, "dram__bytes_write.sum", "Kbyte", "500"])
            rows.append([str(lid), kn, "smsp__inst_executed.sum", "inst", "1,000"])
            rows.append([str(lid), kn, "gpu__time_duration.sum", "usecond", "12"])
        p = tmp_path / f"{name}.csv"
        p.write_text("==PROF== noise line\n" + "\n".join(",".join(f'"{c}"' for c in r) for r in rows) + "\n")
        paths.append(str(p))
    hashes = {st: bench.sources_sha1(st) for st in bench.COUNTER_SOURCES}  # of the real sources
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_sha1", lambda st: hashes[st])
    bench.write_counters(paths)
    d = json.loads((prof / "counters.json").read_text())
    out = d["stages"]
    # per stage call: the sum over its kernels of each kernel's mean per launch
    assert abs(out["trace"]["dram_bytes_per_launch"] - 2 * 2e6) < 1.0
    assert abs(out["trace"]["inst_per_launch"] - 2 * 1000) < 1e-9
    assert abs(out["synthesize"]["dram_bytes_per_launch"] - 3 * 2e6) < 1.0
    assert d["kernels"]["k_trace"]["launches"] == 2
    assert set(bench.measured_counters()) == {"trace", "synthesize"}
    # a stored hash that no longer matches the sources drops that stage
    d["stages"]["trace"]["sources_sha1"] = "0" * 40
    (prof / "counters.json").write_text(json.dumps(d))
    assert set(bench.measured_counters()) == {"synthesize"}
