"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module builds scene meshes, radar parameter sets, ray-grid descriptors and
request streams.  It holds none of the simulator's arithmetic (no intersection,
no path length, no phase, no transform): every number it returns is an *input*
to the method.  Both the FP64 oracle and the GPU library consume these arrays
as they are; neither side's results feed back into this module.

Workload shapes follow the radar platforms of the paper's Section 4 (a 77 GHz
3 Tx x 4 Rx MIMO radar of the AWR1843 class) and car/human-scale objects at
1-3 m; the paper's real captures and ShapeNet/SMPL meshes are replaced by
seeded icospheres, superquadrics and a ground plane.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0  # m/s (exact SI value)

# ----------------------------------------------------------------------------
# Radar parameter sets
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class RadarConfig:
    """FMCW radar parameters (Section 3.2.2, Eq. 8: f_c, B, T; Section 4 platforms).

    Frame: origin at Tx0's phase centre, boresight +z, array along +x.
    Positions are metres in that frame; rays are launched from ``ray_origin``.
    """

    f0: float                 # carrier f_c [Hz]
    bandwidth: float          # sweep B [Hz]
    chirp_time: float         # chirp duration T [s]
    n_samples: int            # ADC samples per chirp N_s
    n_chirps: int             # chirps per frame C
    chirp_rep: float          # chirp repetition interval [s]
    tx: np.ndarray            # [n_tx, 3] float64
    rx: np.ndarray            # [n_rx, 3] float64

    @property
    def n_tx(self) -> int:
        return int(self.tx.shape[0])

    @property
    def n_rx(self) -> int:
        return int(self.rx.shape[0])

    @property
    def n_virt(self) -> int:
        return self.n_tx * self.n_rx

    @property
    def wavelength(self) -> float:
        return C_LIGHT / self.f0


def _radar(f0, bw, tc, ns, nc, n_tx, tx_spacing_wl, n_rx=4, trep=40e-6):
    lam = C_LIGHT / f0
    tx = np.array([[t * tx_spacing_wl * lam, 0.0, 0.0] for t in range(n_tx)], dtype=np.float64)
    rx = np.array([[r * 0.5 * lam, 0.0, 0.0] for r in range(n_rx)], dtype=np.float64)
    return RadarConfig(f0, bw, tc, ns, nc, trep, tx, rx)


def radar_single_tx(n_samples: int = 256, n_chirps: int = 1) -> RadarConfig:
    """77 GHz, 4 GHz over 40 us, 1 Tx at the origin, 4 Rx at lambda/2 along x."""
    return _radar(77e9, 4e9, 40e-6, n_samples, n_chirps, 1, 0.0)


def radar_awr1843(n_samples: int = 256, n_chirps: int = 128) -> RadarConfig:
    """77 GHz 3 Tx x 4 Rx with the middle transmitter raised by lambda/2 (the AWR1843
    layout): Tx at (0, 0), (lambda, lambda/2), (2 lambda, 0); Rx at r lambda/2 along x.
    Eight virtual elements span azimuth at y = 0 and four sit lambda/2 higher."""
    lam = C_LIGHT / 77e9
    tx = np.array([[0.0, 0.0, 0.0], [lam, 0.5 * lam, 0.0], [2 * lam, 0.0, 0.0]])
    rx = np.array([[r * 0.5 * lam, 0.0, 0.0] for r in range(4)])
    return RadarConfig(77e9, 4e9, 40e-6, n_samples, n_chirps, 40e-6, tx, rx)


def radar_mimo_3x4(n_samples: int = 256, n_chirps: int = 128) -> RadarConfig:
    """77 GHz 3 Tx x 4 Rx: Tx at t*2*lambda, Rx at r*lambda/2 -> 12 uniform virtual elements."""
    return _radar(77e9, 4e9, 40e-6, n_samples, n_chirps, 3, 2.0)


# ----------------------------------------------------------------------------
# Ray grids
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class RayGrid:
    """G x G stratified grid of launch directions over a cone (the sample set of Eq. 3).

    Directions are cell centres of the square [-tan_half, tan_half]^2 on the plane
    one unit along ``axis``, spanned by the orthonormal ``u_axis``/``v_axis``.
    Ray index = row * G + col, row along ``v_axis``.
    """

    G: int
    origin: np.ndarray   # [3]
    axis: np.ndarray     # [3] unit
    u_axis: np.ndarray   # [3] unit, orthogonal to axis
    v_axis: np.ndarray   # [3] unit, axis x u_axis
    tan_half: float
    jitter: np.ndarray | None = None   # [G*G, 2] float32 offsets in [0, 1) per ray, or None (cell centres)

    @property
    def n_rays(self) -> int:
        return self.G * self.G


def jittered(grid: RayGrid, seed: int) -> RayGrid:
    """The same grid sampled at seeded uniform offsets inside each cell (stratified jittered
    Monte-Carlo samples of Eq. 3); offsets are float32 in [0, 1)."""
    rng = np.random.default_rng(seed)
    off = rng.random((grid.G * grid.G, 2), dtype=np.float32)
    return dataclasses.replace(grid, jitter=off)


def ray_grid_for_sphere(center, radius: float, G: int, origin=(0.0, 0.0, 0.0)) -> RayGrid:
    """Grid whose square circumscribes the cone from ``origin`` onto a bounding sphere."""
    o = np.asarray(origin, dtype=np.float64)
    c = np.asarray(center, dtype=np.float64)
    dvec = c - o
    dist = float(np.linalg.norm(dvec))
    if dist <= radius:
        raise ValueError("ray origin inside the bounding sphere")
    axis = dvec / dist
    up = np.array([0.0, 1.0, 0.0]) if abs(axis[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    u = np.cross(up, axis)
    u /= np.linalg.norm(u)
    v = np.cross(axis, u)
    v /= np.linalg.norm(v)
    alpha = math.asin(radius / dist)
    return RayGrid(G, o, axis, u, v, math.tan(alpha))


def bounding_sphere(verts: np.ndarray):
    """AABB-centre bounding sphere of a vertex set (centre, radius)."""
    v = np.asarray(verts, dtype=np.float64)
    lo, hi = v.min(0), v.max(0)
    c = 0.5 * (lo + hi)
    r = float(np.sqrt(((v - c) ** 2).sum(1)).max())
    return c, r


def ray_subset(seed: int, n_rays_total: int, n: int) -> np.ndarray:
    """Seeded sorted subset of ray indices (int32)."""
    rng = np.random.default_rng(seed)
    n = min(n, n_rays_total)
    return np.sort(rng.choice(n_rays_total, size=n, replace=False)).astype(np.int32)


# ----------------------------------------------------------------------------
# Meshes
# ----------------------------------------------------------------------------


def icosphere(subdiv: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Subdivided icosahedron projected onto a sphere: 10*4^s+2 verts, 20*4^s tris."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    v = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    return v.astype(np.float32), np.array(faces, dtype=np.int32)


def _spow(x, e):
    return np.sign(x) * np.abs(x) ** e


def random_rotation(rng) -> np.ndarray:
    """Uniform random rotation from a normalised 4D Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def superquadric(seed: int, n_lon: int = 100, n_rings: int = 100, center=None):
    """Seeded superquadric: exponents U[0.3,2], half-axes U[0.1,0.5] m, random rotation,
    centre on boresight at range U[1,3] m.  Latitude-longitude mesh with pole fans:
    n_lon*n_rings+2 vertices, 2*n_lon*n_rings triangles (20,000 at the defaults)."""
    rng = np.random.default_rng(seed)
    e1, e2 = rng.uniform(0.3, 2.0, size=2)
    a = rng.uniform(0.1, 0.5, size=3)
    rot = random_rotation(rng)
    rng_c = rng.uniform(1.0, 3.0)
    if center is None:
        center = np.array([0.0, 0.0, rng_c])
    eta = -0.5 * np.pi + np.pi * (np.arange(1, n_rings + 1) / (n_rings + 1))   # interior rings
    om = -np.pi + 2 * np.pi * np.arange(n_lon) / n_lon
    E, O = np.meshgrid(eta, om, indexing="ij")
    ce, se = _spow(np.cos(E), e1), _spow(np.sin(E), e1)
    x = a[0] * ce * _spow(np.cos(O), e2)
    y = a[1] * ce * _spow(np.sin(O), e2)
    z = a[2] * se
    ring = np.stack([x, y, z], -1).reshape(-1, 3)
    south = np.array([[0.0, 0.0, -a[2]]])
    north = np.array([[0.0, 0.0, a[2]]])
    v = np.concatenate([ring, south, north], 0)
    v = v @ rot.T + np.asarray(center, dtype=np.float64)
    S, N = n_rings * n_lon, n_rings * n_lon + 1
    faces = []
    idx = lambda r, l: r * n_lon + (l % n_lon)
    for r in range(n_rings - 1):
        for l in range(n_lon):
            p00, p01, p10, p11 = idx(r, l), idx(r, l + 1), idx(r + 1, l), idx(r + 1, l + 1)
            faces.append((p00, p01, p11))
            faces.append((p00, p11, p10))
    for l in range(n_lon):
        faces.append((S, idx(0, l + 1), idx(0, l)))
        faces.append((N, idx(n_rings - 1, l), idx(n_rings - 1, l + 1)))
    params = dict(eps=(float(e1), float(e2)), axes=a.tolist(), center=list(map(float, center)))
    return v.astype(np.float32), np.array(faces, dtype=np.int32), params


def ground_plane(y: float, cx: float, cz: float, size: float = 4.0):
    """Horizontal square (2 triangles) in the plane y=const, centred at (cx, cz)."""
    h = 0.5 * size
    v = np.array([[cx - h, y, cz - h], [cx + h, y, cz - h], [cx + h, y, cz + h], [cx - h, y, cz + h]],
                 dtype=np.float32)
    f = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return v, f


def merge_meshes(*meshes):
    vs, fs, off = [], [], 0
    for v, f in meshes:
        vs.append(v)
        fs.append(f + off)
        off += v.shape[0]
    return np.concatenate(vs).astype(np.float32), np.concatenate(fs).astype(np.int32)


def perturbed_icosphere(seed: int, subdiv: int, radius: float, center, noise: float = 0.05):
    rng = np.random.default_rng(seed)
    v, f = icosphere(subdiv, 1.0)
    s = 1.0 + noise * rng.uniform(-1.0, 1.0, size=(v.shape[0], 1))
    v = v.astype(np.float64) * s * radius + np.asarray(center, dtype=np.float64)
    return v.astype(np.float32), f


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Workload:
    name: str
    verts: np.ndarray
    faces: np.ndarray
    radar: RadarConfig
    grid: RayGrid
    max_bounces: int
    meta: dict


def sphere_scene(G: int = 64, distance: float = 1.0, n_samples: int = 256, radius: float = 0.2,
                 subdiv: int = 2, max_bounces: int = 2) -> Workload:
    """Icosphere (320 tris at subdiv 2) of radius 0.2 m on boresight, 1 Tx / 4 Rx radar."""
    c = (0.0, 0.0, distance)
    v, f = icosphere(subdiv, radius, c)
    grid = ray_grid_for_sphere(c, radius, G)
    return Workload(f"sphere{len(f)}_d{distance:g}_G{G}_Ns{n_samples}", v, f,
                    radar_single_tx(n_samples, 1), grid, max_bounces,
                    dict(center=c, radius=radius))


def superquadric_scene(seed: int = 0, G: int = 1024, n_chirps: int = 128, n_samples: int = 256,
                       max_bounces: int = 3, n_lon: int = 100, n_rings: int = 100) -> Workload:
    """Seeded superquadric (20,000 tris) over a 4x4 m ground plane (2 tris), 3x4 MIMO radar."""
    ov, of, params = superquadric(seed, n_lon, n_rings)
    ymin = float(ov[:, 1].min())
    c, r = bounding_sphere(ov)
    gv, gf = ground_plane(ymin, float(c[0]), float(c[2]))
    v, f = merge_meshes((ov, of), (gv, gf))
    grid = ray_grid_for_sphere(c, r, G)
    return Workload(f"superquadric{len(f)}_s{seed}_G{G}", v, f, radar_mimo_3x4(n_samples, n_chirps),
                    grid, max_bounces, dict(params=params, center=c.tolist(), radius=r))


def serving_requests(seed: int, n: int = 512, nt_range=(1_000, 200_000), rays_range=(65_536, 4_194_304)):
    """Seeded request stream: Poisson inter-arrival gaps (unit mean; scale by the rate),
    log-uniform triangle and ray budgets, half forward-only, half reconstruction."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(n):
        t += rng.exponential(1.0)
        nt = int(math.exp(rng.uniform(math.log(nt_range[0]), math.log(nt_range[1]))))
        nr = math.exp(rng.uniform(math.log(rays_range[0]), math.log(rays_range[1])))
        G = max(8, int(round(math.sqrt(nr))))
        kind = "forward" if rng.random() < 0.5 else "recon"
        mesh = "superquadric" if rng.random() < 0.5 else "icosphere"
        reqs.append(dict(id=i, arrival=t, n_tris=nt, G=G, kind=kind, mesh=mesh,
                         seed=int(rng.integers(0, 2**31 - 1))))
    return reqs


def request_mesh(req: dict):
    """Mesh for a serving request with about ``req['n_tris']`` triangles at 1-3 m."""
    rng = np.random.default_rng(req["seed"])
    dist = float(rng.uniform(1.0, 3.0))
    if req["mesh"] == "superquadric":
        m = max(4, int(round(math.sqrt(req["n_tris"] / 2.0))))
        v, f, _ = superquadric(req["seed"], n_lon=m, n_rings=m, center=(0.0, 0.0, dist))
    else:
        s = max(1, int(round(math.log(max(req["n_tris"], 20) / 20.0, 4))))
        v, f = perturbed_icosphere(req["seed"], min(s, 6), 0.25, (0.0, 0.0, dist))
    return v, f


@dataclasses.dataclass
class CfarParams:
    """Point-extraction parameters (soft CA-CFAR over range, 3x3 peaks, top-k).

    Defaults: 64 angle bins, guard 2 / train 8 range cells, 12 dB CFAR scale,
    floor 40 dB below the map maximum, sigmoid temperature 0.5 (natural-log
    power units), minimum weight 0.01, at most 2000 points."""

    n_theta: int = 64
    guard: int = 2
    train: int = 8
    alpha_db: float = 12.0
    floor_rel: float = 1e-4
    beta: float = 0.5
    w_min: float = 0.01
    k_max: int = 2000
    n_elev: int = 1          # elevation bins (a 2D virtual array); 1: azimuth only

    @property
    def alpha(self) -> float:
        return 10.0 ** (self.alpha_db / 10.0)


def serving_workload(seed: int, n: int = 512, pool: int = 64, nt_range=(1_000, 200_000),
                     rays_range=(65_536, 4_194_304), recon_iterations: int = 50):
    """Seeded request stream over a pool of meshes (so BVHs can be reused).

    Pool mesh j: superquadric or perturbed icosphere (50/50) with a log-uniform
    triangle budget in ``nt_range`` at 1-3 m.  Request i: a pool mesh, a
    log-uniform ray budget in ``rays_range`` (rounded to G x G), and a kind:
    half forward-only, half ``recon_iterations``-iteration reconstructions."""
    rng = np.random.default_rng(seed)
    meshes = []
    for j in range(pool):
        nt = int(math.exp(rng.uniform(math.log(nt_range[0]), math.log(nt_range[1]))))
        kind = "superquadric" if rng.random() < 0.5 else "icosphere"
        meshes.append(dict(id=j + 1, n_tris=nt, mesh=kind, seed=int(rng.integers(0, 2**31 - 1))))
    reqs = []
    for i in range(n):
        nr = math.exp(rng.uniform(math.log(rays_range[0]), math.log(rays_range[1])))
        reqs.append(dict(id=i, mesh=int(rng.integers(0, pool)), G=max(8, int(round(math.sqrt(nr)))),
                         kind="forward" if rng.random() < 0.5 else "recon", iterations=recon_iterations))
    return meshes, reqs
