"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Run from the repository root:

    python tests/golden/make_golden.py

The script calls only ``oracle/`` (and the seeded input generators of
``sbr_inputs``); no value in these files comes from the CUDA library.  The
paper prints no worked numerical example of the simulator, so every stored
value is the oracle's FP64 result on a small seeded workload, kept as text so
that a change to the oracle's arithmetic shows up as a diff of these files.

Fixtures (workload: the icosphere scene of 320 triangles, radius 0.2 m,
centred 1.0 m on boresight; 77 GHz, 4 GHz over 40 us, 256 samples, 1 chirp;
1 Tx at the origin, 4 Rx at lambda/2 spacing; up to 2 specular bounces):

  sphere_g16_trace.txt   nearest-hit triangle per ray and bounce (Section 3.2.1,
                         Eq. 2-3), 16 x 16 ray grid, plus the oracle's edge/tie flag
  sphere_g16_paths.txt   per (antenna, path) delay tau and strength A (the I^t, I^s
                         of Section 3.2.1 under the amplitude reading of Eq. 1)
  sphere_g16_cube.txt    IF samples S[v, n] of Eq. 8 (one chirp: the scene is static)
  sphere_g64_points.txt  point cloud of the map T (Section 3.4, Eq. 16 reading) from the
                         64 x 64-ray cube: x, y, z, w
  precision_sweep_subset4096.npz
                         the long-range precision sweep: the same sphere centred 5, 10 and
                         20 m out, 1024, 2048 and 4096 samples per chirp, 2048 x 2048 ray
                         grid of which a seeded subset of 4096 rays (sbr_inputs.ray_subset,
                         seed 11) is traced; per (distance, samples) the oracle's FP64 IF
                         cube (Eq. 8, complex128 [4, N_s]) and its point cloud.  Binary
                         (numpy .npz) because the cubes hold 86,016 complex samples in all.
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import pointcloud as opc  # noqa: E402
from sbr_inputs import CfarParams, sphere_scene  # noqa: E402

WORKLOAD = ("icosphere 320 triangles, radius 0.2 m, centre (0, 0, 1.0) m; 77 GHz, 4 GHz / 40 us, "
            "256 samples, 1 chirp; 1 Tx at the origin, 4 Rx at lambda/2 along x; up to 2 bounces")
GENERATOR = "written by tests/golden/make_golden.py from oracle/ (FP64)"


def compute() -> dict:
    """The fixtures' contents, computed by the oracle (also used by the regression test)."""
    wl16 = sphere_scene(G=16)
    cube16, tr, pa = oracle.simulate_cube(wl16)
    wl64 = sphere_scene(G=64)
    cube64, _, _ = oracle.simulate_cube(wl64)
    pc = opc.pointcloud(cube64, wl64.radar, CfarParams())
    return dict(tri=tr["tri"], flag=tr["flag"], tau=pa["tau"], amp=pa["amp"], ray=pa["ray"],
                bounce=pa["bounce"], cube=cube16[:, 0, :], points=pc["points"])


SWEEP_DISTANCES = (5.0, 10.0, 20.0)
SWEEP_SAMPLES = (1024, 2048, 4096)
SWEEP_FILE = "precision_sweep_subset4096.npz"
SWEEP_RAYS = 4096
SWEEP_SEED = 11


def sweep_key(dist: float, ns: int) -> str:
    return f"d{int(dist)}_ns{ns}"


def compute_sweep() -> dict:
    """Oracle cubes and point clouds of the precision-sweep configurations (subset rays)."""
    from sbr_inputs import ray_subset
    out = {}
    for dist in SWEEP_DISTANCES:
        for ns in SWEEP_SAMPLES:
            wl = sphere_scene(G=2048, distance=dist, n_samples=ns)
            ids = ray_subset(SWEEP_SEED, wl.grid.n_rays, SWEEP_RAYS)
            cube, _, pa = oracle.simulate_cube(wl, ids)
            pc = opc.pointcloud(cube, wl.radar, CfarParams())
            k = sweep_key(dist, ns)
            out["cube_" + k] = cube[:, 0, :]
            out["points_" + k] = pc["points"]
            out["paths_" + k] = np.int64(pa["P"])
    return out


def _write(name: str, header: list, rows: list):
    with open(os.path.join(HERE, name), "w") as fh:
        for h in header:
            fh.write(f"# {h}\n")
        for r in rows:
            fh.write(r + "\n")


def main():
    d = compute()
    tri, flag = d["tri"], d["flag"]
    _write("sphere_g16_trace.txt",
           ["Nearest-hit triangle index per ray and bounce (-1: no hit); Section 3.2.1, Eq. 2-3:",
            "brute-force FP64 Moller-Trumbore, two-sided, |det| < 1e-12 misses, t > 1e-9 m, previous",
            "triangle skipped, exact ties to the lower index.  flag: first bounce (1-based) whose hit",
            "lies within 1e-6 of an edge or ties another surface (0: none); such rays are excluded",
            "from index parity.",
            f"workload: {WORKLOAD}; 16 x 16 ray grid over the sphere's bounding cone",
            GENERATOR,
            "columns: ray tri_bounce1 tri_bounce2 flag"],
           [f"{i} {tri[i, 0]} {tri[i, 1]} {flag[i]}" for i in range(tri.shape[0])])
    tau, amp, ray, bounce = d["tau"], d["amp"], d["ray"], d["bounce"]
    _write("sphere_g16_paths.txt",
           ["Per (virtual antenna, path) delay tau [s] and strength A: the I^t and I^s of Section",
            "3.2.1.  tau = (L_in + L_out) / c with L_in = |h_1 - Tx| + interior legs, L_out = |Rx - h_k|;",
            "A = omega (-1)^(k-1) |d_k . n_k| / (4 pi L_in L_out) (cos term and 1/(4 pi .) spreading",
            "of Eq. 1, perfect-conductor reflection).  Paths ray-major, bounce-minor.",
            f"workload: {WORKLOAD}; 16 x 16 ray grid",
            GENERATOR,
            "columns: antenna ray bounce(0-based) tau amp"],
           [f"{v} {ray[p]} {bounce[p]} {tau[v, p]:.17e} {amp[v, p]:.17e}"
            for v in range(tau.shape[0]) for p in range(tau.shape[1])])
    cube = d["cube"]
    _write("sphere_g16_cube.txt",
           ["IF samples of Eq. 8 (Section 3.2.2): S[v, n] = sum_p A exp(j 2 pi (f_c tau + mu tau t_n)),",
            "mu = B / T, t_n = n T / N_s, summed over every (hit, antenna) path, direct FP64 sum.",
            f"workload: {WORKLOAD}; 16 x 16 ray grid",
            GENERATOR,
            "columns: antenna sample re im"],
           [f"{v} {n} {cube[v, n].real:.17e} {cube[v, n].imag:.17e}"
            for v in range(cube.shape[0]) for n in range(cube.shape[1])])
    pts = d["points"]
    _write("sphere_g64_points.txt",
           ["Radar point cloud of the map T (Section 3.4, Eq. 16; the paper names only a signal",
            "processing algorithm): direct range DFT, angle DFT over 64 bins of u = sin(theta),",
            "power map, CA-CFAR (guard 2, train 8), soft weight w, 3x3 peaks, parabolic refine;",
            "order by (w desc, cell asc), w >= 0.01.",
            f"workload: {WORKLOAD}; 64 x 64 ray grid",
            GENERATOR,
            "columns: x y z w"],
           [" ".join(f"{x:.17e}" for x in p) for p in pts])
    np.savez_compressed(os.path.join(HERE, SWEEP_FILE), **compute_sweep())
    print("wrote", ", ".join(sorted(f for f in os.listdir(HERE) if f.endswith((".txt", ".npz")))))


if __name__ == "__main__":
    main()
