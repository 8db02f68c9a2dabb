"""FP64 CPU oracle of the SBR radar simulator (test infrastructure).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is
compared against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
bench's ``cpu_baseline`` / ``--impl reference`` legs may import it.  It shares
no code with the CUDA path; its only common dependency is the seeded input
module ``sbr_inputs``.

Layout:
  sbr_oracle.c   brute-force FP64 trace (every ray x every triangle), direct FP64
                 Eq. 8 synthesis and its Eq. 11-12 adjoint (OpenMP over rays/outputs)
  __init__.py    loader, ray paths -> per-antenna (tau, A), synthesis wrappers
  pointcloud.py  direct O(N^2) DFTs, angle DFT, CA-CFAR, soft detection, points,
                 Chamfer and Laplacian terms, frozen-structure evaluators for FD

Readings of passages the paper leaves open (amplitude constants, ray grid,
bounce count, the signal-processing chain T of Eq. 16) are written next to the
function that takes them.  "Parity unpinned": the amplitude constants and the
point-cloud chain beyond the closed-form special cases pinned by
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

from sbr_inputs import C_LIGHT

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbr_oracle.c")
_LIB = None

TMIN = 1e-9        # m, minimum accepted hit distance
EDGE_EPS = 1e-6    # barycentric edge band excluded from index parity
TIE_REL = 1e-9     # relative t band treated as a tie between surfaces


def lib_path() -> str:
    return os.path.join(_HERE, "_build", f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, no FP contraction)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_trace.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  P, P, P, P, P, P, P]
        lib.orc_synth.argtypes = [P, P, ctypes.c_long, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int, P, P]
        lib.orc_synth_grad.argtypes = [P, P, ctypes.c_long, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P, P, P]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def set_threads(n: int) -> int:
    """Threads the C oracle's loops use from now on (n >= 1); returns the previous count."""
    return int(_lib().orc_set_threads(int(n)))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def grid_array(grid) -> np.ndarray:
    return np.concatenate([grid.origin, grid.axis, grid.u_axis, grid.v_axis,
                           [grid.tan_half]]).astype(np.float64)


# ----------------------------------------------------------------------------
# Trace (Section 3.2.1, Eq. 2-3)
# ----------------------------------------------------------------------------


def trace(verts, faces, grid, max_bounces: int, ray_ids=None, tmin=TMIN, edge_eps=EDGE_EPS,
          tie_rel=TIE_REL) -> dict:
    """Brute-force FP64 trace of the G x G grid (or of ``ray_ids``); a grid with ``jitter``
    (offsets in [0, 1)^2 per ray) samples each cell there instead of at its centre.

    Returns arrays indexed [ray, bounce]: tri (-1 = no hit), t/u/v, hit point,
    incident direction, unit normal; per ray omega (solid-angle weight) and flag
    (first ambiguous bounce, 1-based, 0 if none)."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    g = grid_array(grid)
    ids = None if ray_ids is None else np.ascontiguousarray(ray_ids, dtype=np.int32)
    n = grid.n_rays if ids is None else int(ids.shape[0])
    K = int(max_bounces)
    tri = np.empty((n, K), np.int32)
    tuv = np.empty((n, K, 3), np.float64)
    hit = np.empty((n, K, 3), np.float64)
    din = np.empty((n, K, 3), np.float64)
    nrm = np.empty((n, K, 3), np.float64)
    omega = np.empty(n, np.float64)
    flag = np.empty(n, np.int32)
    jit = getattr(grid, "jitter", None)
    jit = None if jit is None else np.ascontiguousarray(jit, dtype=np.float32).reshape(-1, 2)
    if jit is not None and jit.shape[0] != grid.G * grid.G:
        raise ValueError("jitter must hold G*G offset pairs")
    rc = _lib().orc_trace(_ptr(v), v.shape[0], _ptr(f), f.shape[0], _ptr(g), grid.G, _ptr(jit), _ptr(ids), n, K,
                          tmin, edge_eps, tie_rel, _ptr(tri), _ptr(tuv), _ptr(hit), _ptr(din),
                          _ptr(nrm), _ptr(omega), _ptr(flag))
    if rc != 0:
        raise ValueError(f"orc_trace rejected its input (code {rc})")
    return dict(tri=tri, tuv=tuv, hit=hit, din=din, nrm=nrm, omega=omega, flag=flag,
                ray_ids=(np.arange(n, dtype=np.int32) if ids is None else ids), K=K)


def paths(tr: dict, radar) -> dict:
    """Per-path, per-virtual-antenna delay tau and strength A (the I^t, I^s of Section 3.2.1).

    Reading (the paper gives no constants): every hit k of a ray emits one path
    per virtual antenna (t, r), v = t * n_rx + r, with
      L_in  = |h_1 - Tx_t| + sum_{j=2..k} |h_j - h_{j-1}|
      L_out = |Rx_r - h_k|
      tau   = (L_in + L_out) / c
      A     = omega * (-1)^(k-1) * |d_k . n_k| / (4 pi L_in L_out)
    (per-interaction reflection -1 of a perfect conductor, the cos term and the
    1/(4 pi .) spreading of Eq. 1).  Paths are ordered ray-major, bounce-minor.
    """
    tri, hit, din, nrm, omega = tr["tri"], tr["hit"], tr["din"], tr["nrm"], tr["omega"]
    n, K = tri.shape
    valid = tri >= 0
    ray_of, k_of = np.nonzero(valid)              # row-major => ray-major, bounce-minor
    seg = np.zeros((n, K), np.float64)
    if K > 1:
        seg[:, 1:] = np.sqrt(((hit[:, 1:] - hit[:, :-1]) ** 2).sum(-1)) * valid[:, 1:]
    interior = np.cumsum(seg, axis=1)             # interior[i,k] = sum_{j<=k} |h_j - h_{j-1}|
    h1 = hit[ray_of, 0]
    hk = hit[ray_of, k_of]
    cos = np.abs((din[ray_of, k_of] * nrm[ray_of, k_of]).sum(-1))
    sign = np.where(k_of % 2 == 0, 1.0, -1.0)
    I = interior[ray_of, k_of]
    V = radar.n_virt
    P = ray_of.shape[0]
    tau = np.empty((V, P))
    amp = np.empty((V, P))
    lin = np.empty((V, P))
    lout = np.empty((V, P))
    for t in range(radar.n_tx):
        li = np.sqrt(((h1 - radar.tx[t]) ** 2).sum(-1)) + I
        for r in range(radar.n_rx):
            lo = np.sqrt(((radar.rx[r] - hk) ** 2).sum(-1))
            v = t * radar.n_rx + r
            lin[v], lout[v] = li, lo
            tau[v] = (li + lo) / C_LIGHT
            amp[v] = omega[ray_of] * sign * cos / (4.0 * np.pi * li * lo)
    return dict(tau=tau, amp=amp, ray=ray_of.astype(np.int32), bounce=k_of.astype(np.int32),
                lin=lin, lout=lout, cos=cos, P=P)


# ----------------------------------------------------------------------------
# Materials: Fresnel reflection (Section 3.2.2, Eq. 9-10)
# ----------------------------------------------------------------------------


def fresnel(cos_i, eps):
    """Fresnel reflection coefficients (r_s, r_p) of Eq. 9 for incidence cosines ``cos_i``
    (|d . n|, two-sided surfaces) from air onto a material of complex relative permittivity
    ``eps`` (eps' - j eps'' with eps'' = sigma / (omega eps_0) >= 0).

    Eq. 10 in the order the paper gives it, with two readings of its garbled parts:
      cos d_i = |i . n|,  sin d_i = sqrt(1 - cos^2 d_i),
      sin d_t = sin d_i / sqrt(eps)      (Snell's law from air into the material; the printed
                                          sqrt(eps) sin d_i inverts it),
      cos d_t = sqrt(1 - sin^2 d_t)      (principal complex root: Re >= 0, a decaying wave),
      eta     = sqrt(eps)                (used as the ratio of the two media's refractive
                                          indices, which makes Eq. 9 the textbook equations)
      r_p = (eta cos d_i - cos d_t) / (eta cos d_i + cos d_t),
      r_s = (cos d_i - eta cos d_t) / (cos d_i + eta cos d_t)."""
    c = np.asarray(cos_i, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.complex128)
    sin_i = np.sqrt(np.maximum(1.0 - c * c, 0.0))
    eta = np.sqrt(eps)
    sin_t = sin_i / eta
    cos_t = np.sqrt(1.0 - sin_t * sin_t)
    cos_t = np.where(cos_t.real < 0, -cos_t, cos_t)
    r_p = (eta * c - cos_t) / (eta * c + cos_t)
    r_s = (c - eta * cos_t) / (c + eta * cos_t)
    return r_s, r_p


def path_fresnel(tr: dict, pa: dict, tri_material, eps) -> np.ndarray:
    """Complex factor F of every path (ray-major, bounce-minor, as ``paths``): each surface
    interaction multiplies the path by its Fresnel coefficient (Section 3.2.2: "every time a
    ray interacts with a surface, these coefficients are applied and accumulated").

    Readings: the radar's polarisation is taken perpendicular to each plane of incidence, so
    the coefficient applied is r_s; a material with eps' <= 0 is a perfect conductor
    (r_s = -1).  Path k (1-based) reflects at hits 1..k-1 and scatters back at hit k:
      F = prod_{j<k} r_s(j) * (-r_s(k)),
    so with perfect conductors everywhere F = (-1)^(k-1), the factor of ``paths``."""
    tri = tr["tri"]
    cos = np.abs((tr["din"] * tr["nrm"]).sum(-1))          # [n, K] |d_j . n_j|
    mat = np.asarray(tri_material)[np.maximum(tri, 0)]
    e = np.asarray(eps, dtype=np.complex128)[mat]
    r, _ = fresnel(cos, e)
    r = np.where(e.real <= 0, -1.0 + 0j, r)
    F = np.empty(pa["P"], np.complex128)
    for i, (ray, k) in enumerate(zip(pa["ray"], pa["bounce"])):
        F[i] = -np.prod(r[ray, :k + 1])
    return F


# ----------------------------------------------------------------------------
# Synthesis (Section 3.2.2, Eq. 8) and its adjoint (Eq. 11-12)
# ----------------------------------------------------------------------------


def chirp_constants(radar):
    mu = radar.bandwidth / radar.chirp_time
    fs = radar.n_samples / radar.chirp_time
    return mu, fs


def synthesize(tau, amp, radar) -> np.ndarray:
    """IF cube [V, C, N_s] complex128 by the direct FP64 sum of Eq. 8.

    Reading: t_n = n / f_s with f_s = N_s / T (no ADC offset); the sum runs over
    every (hit, antenna) path; the scene is static, so every chirp is equal.
    A complex strength (material paths) enters through the linearity of Eq. 8 in
    I^s: the sum of Re(A) and j times the sum of Im(A)."""
    if np.iscomplexobj(amp):
        return synthesize(tau, np.real(amp), radar) + 1j * synthesize(tau, np.imag(amp), radar)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    V, P = tau.shape
    mu, fs = chirp_constants(radar)
    Ns = radar.n_samples
    re = np.empty((V, Ns))
    im = np.empty((V, Ns))
    rc = _lib().orc_synth(_ptr(tau), _ptr(amp), P, V, radar.f0, mu, fs, Ns, _ptr(re), _ptr(im))
    if rc:
        raise ValueError("orc_synth rejected its input")
    s = re + 1j * im
    return np.repeat(s[:, None, :], radar.n_chirps, axis=1)


def synthesize_grad(tau, amp, radar, g_cube):
    """(dL/dtau, dL/dA) [V, P] for upstream gradient g_cube [V, C, N_s] (Eq. 11-12).

    The static cube repeats one chirp C times, so the per-chirp gradients add."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    V, P = tau.shape
    mu, fs = chirp_constants(radar)
    g = np.asarray(g_cube).sum(axis=1)
    gr = np.ascontiguousarray(g.real, dtype=np.float64)
    gi = np.ascontiguousarray(g.imag, dtype=np.float64)
    gtau = np.empty((V, P))
    gamp = np.empty((V, P))
    rc = _lib().orc_synth_grad(_ptr(tau), _ptr(amp), P, V, radar.f0, mu, fs, radar.n_samples,
                               _ptr(gr), _ptr(gi), _ptr(gtau), _ptr(gamp))
    if rc:
        raise ValueError("orc_synth_grad rejected its input")
    return gtau, gamp


# ----------------------------------------------------------------------------
# Moving objects: path-length rates and the per-chirp IF signal (Section 3.1's
# scene dynamics; Eq. 8 evaluated chirp by chirp)
# ----------------------------------------------------------------------------


def path_rates(tr: dict, pa: dict, radar, tri_object, velocity) -> np.ndarray:
    """Rate of change dL/dt [V, P] of every path's length when each object translates with
    its velocity (m/s) and every hit point moves with its object.

    From L = |h_1 - Tx| + sum_{j=2..k} |h_j - h_{j-1}| + |Rx - h_k|:
      dL/dt = sum_j v_j . (u_in,j - u_out,j),
    u_in,j the unit vector of the leg arriving at h_j (from Tx for j = 1), u_out,j that of the
    leg leaving it (towards Rx for j = k)."""
    hit, tri = tr["hit"], tr["tri"]
    vel = np.asarray(velocity, dtype=np.float64).reshape(-1, 3)
    obj = np.asarray(tri_object)
    unit = lambda x: x / np.linalg.norm(x, axis=-1, keepdims=True)
    V = radar.n_virt
    out = np.zeros((V, pa["P"]))
    for i, (ray, k) in enumerate(zip(pa["ray"], pa["bounce"])):
        h = hit[ray, :k + 1]
        vj = vel[obj[tri[ray, :k + 1]]]
        interior = 0.0
        for j in range(k + 1):
            if j >= 1:
                interior += vj[j] @ unit(h[j] - h[j - 1])
            if j < k:
                interior -= vj[j] @ unit(h[j + 1] - h[j])
        for t in range(radar.n_tx):
            for r in range(radar.n_rx):
                out[t * radar.n_rx + r, i] = (interior + vj[0] @ unit(h[0] - radar.tx[t])
                                              - vj[k] @ unit(radar.rx[r] - h[k]))
    return out


def synthesize_moving(tau, amp, radar, rate) -> np.ndarray:
    """IF cube [V, C, N_s] of Eq. 8 chirp by chirp: chirp c starts at c T_rep, when every
    path's delay has become tau + c T_rep dL/dt / c (amplitudes held over the frame)."""
    C = radar.n_chirps
    out = []
    for c in range(C):
        tc = np.asarray(tau) + c * radar.chirp_rep * np.asarray(rate) / C_LIGHT
        one = synthesize(tc, amp, radar)[:, :1]
        out.append(one)
    return np.concatenate(out, axis=1)


def simulate_cube(wl, ray_ids=None, materials=None, motion=None) -> tuple:
    """Trace + paths + synthesis of a workload; returns (cube, trace, paths).  With
    ``materials = (tri_material, eps)`` every path carries its Fresnel factor (pa["amp_c"]);
    with ``motion = (tri_object, velocities)`` the chirps follow the moving objects."""
    tr = trace(wl.verts, wl.faces, wl.grid, wl.max_bounces, ray_ids)
    pa = paths(tr, wl.radar)
    if materials is not None:
        F = path_fresnel(tr, pa, *materials)
        # the perfect-conductor sign (-1)^(k-1) of pa["amp"] is replaced by F
        sign = np.where(pa["bounce"] % 2 == 0, 1.0, -1.0)
        pa["fresnel"] = F
        pa["amp_c"] = pa["amp"] * sign[None, :] * F[None, :]
    amp = pa.get("amp_c", pa["amp"])
    if motion is not None:
        pa["rate"] = path_rates(tr, pa, wl.radar, *motion)
        return synthesize_moving(pa["tau"], amp, wl.radar, pa["rate"]), tr, pa
    return synthesize(pa["tau"], amp, wl.radar), tr, pa


# ----------------------------------------------------------------------------
# Frozen-structure evaluation (finite-difference references of the adjoints)
# ----------------------------------------------------------------------------


def trace_frozen(verts, faces, tr_ref: dict, grid) -> dict:
    """Re-evaluate the geometry of ``tr_ref``'s rays in FP64 for new vertex positions
    with every ray's triangle sequence held fixed (the visibility structure of the
    reference trace).  Hit k is the intersection of the ray with the plane of its
    recorded triangle (Moller-Trumbore's t), then specular reflection as in ``trace``.
    The interior derivative of Eq. 4-5 is the derivative of this function."""
    return _frozen(verts, faces, tr_ref, grid, tr_ref["din"][:, 0].copy(), tr_ref["omega"].copy())


def trace_reparam(verts, faces, tr_ref: dict, grid, verts_ref) -> dict:
    """The ray samples of ``tr_ref`` under the change of variables of Eq. 6, for new vertex
    positions: T attaches each ray's first hit to its triangle at the reference barycentrics
    (u, v), so the launch direction follows the surface,
        d_1 = (x - o) / |x - o|,  x = (1 - u - v) a + u b + v c   (the moved triangle),
    and the ray's solid-angle weight takes the factor |det J_T|, the change of the solid angle
    the attached surface element subtends: with N = (b - a) x (c - a) (twice the area times the
    unit normal; an affine map of the triangle scales every area element with |N|),
        omega' = omega * J(verts) / J(verts_ref),  J = |N . (x - o)| / |x - o|^3.
    Later bounces follow as in ``trace_frozen`` (triangle sequence held).  At verts = verts_ref
    this is the reference trace; the derivative of a path sum under it is Eq. 7's integrand
    (df/dtheta with the sample moving along, plus f dlog|det J_T|/dtheta).  Rays without a first
    hit keep their direction and weight."""
    v = np.asarray(verts, dtype=np.float64)
    v0 = np.asarray(verts_ref, dtype=np.float64)
    f = np.asarray(faces)
    tri0 = tr_ref["tri"][:, 0]
    n = tri0.shape[0]
    o = np.asarray(grid.origin, np.float64)
    d = tr_ref["din"][:, 0].copy()
    omega = tr_ref["omega"].astype(np.float64).copy()
    idx = np.where(tri0 >= 0)[0]
    if idx.size:
        fa = f[tri0[idx]]
        u, w = tr_ref["tuv"][idx, 0, 1], tr_ref["tuv"][idx, 0, 2]

        def point_and_density(vv):
            a, b, c = vv[fa[:, 0]], vv[fa[:, 1]], vv[fa[:, 2]]
            x = (1.0 - u - w)[:, None] * a + u[:, None] * b + w[:, None] * c
            N = np.cross(b - a, c - a)
            r = np.linalg.norm(x - o, axis=1)
            return x, np.abs((N * (x - o)).sum(-1)) / r ** 3, r

        x, J, r = point_and_density(v)
        _, J0, _ = point_and_density(v0)
        d[idx] = (x - o) / r[:, None]
        omega[idx] *= J / J0
    return _frozen(verts, faces, tr_ref, grid, d, omega)


def _frozen(verts, faces, tr_ref: dict, grid, d, omega) -> dict:
    """Hits and reflections of ``tr_ref``'s triangle sequences from launch directions d."""
    v = np.asarray(verts, dtype=np.float64)
    f = np.asarray(faces)
    tri = tr_ref["tri"]
    n, K = tri.shape
    o = np.repeat(np.asarray(grid.origin, np.float64)[None], n, axis=0)
    hit = np.zeros((n, K, 3))
    din = np.zeros((n, K, 3))
    nrm = np.zeros((n, K, 3))
    tuv = np.zeros((n, K, 3))
    alive = np.ones(n, bool)
    for k in range(K):
        din[:, k] = d
        ok = alive & (tri[:, k] >= 0)
        alive = ok
        if not ok.any():
            continue
        idx = np.where(ok)[0]
        fa = f[tri[idx, k]]
        a, b, c = v[fa[:, 0]], v[fa[:, 1]], v[fa[:, 2]]
        N = np.cross(b - a, c - a)
        t = (N * (a - o[idx])).sum(-1) / (N * d[idx]).sum(-1)
        h = o[idx] + t[:, None] * d[idx]
        nh = N / np.linalg.norm(N, axis=1, keepdims=True)
        hit[idx, k] = h
        nrm[idx, k] = nh
        tuv[idx, k, 0] = t
        dd = d[idx]
        d[idx] = dd - 2.0 * (dd * nh).sum(-1, keepdims=True) * nh
        o[idx] = h
    return dict(tri=tri.copy(), tuv=tuv, hit=hit, din=din, nrm=nrm, omega=omega,
                flag=np.zeros(n, np.int32), ray_ids=tr_ref["ray_ids"], K=K)
