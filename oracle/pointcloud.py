"""FP64 oracle of the signal-processing chain T (Eq. 16) and of the reconstruction loss.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper names T only as "a signal processing algorithm" mapping MIMO IF
signals to a spatial image (Section 3.4, Eq. 16) and reports radar point
clouds (Section 4).  The reading implemented here, step by step in FP64:

  1. range DFT over samples    X[v,c,k] = sum_n S[v,c,n] e^{-j2pi kn/N_s}   (direct O(N^2))
  2. Doppler DFT over chirps   X[v,d,k] = sum_c X[v,c,k] e^{-j2pi dc/C}     (direct O(C^2))
  3. angle DFT                 Y[a,d,k] = sum_v W[a,v] X[v,d,k],
                               W[a,v] = e^{+j2pi (x_v u_a + y_v w_e) / lambda}, u_a = -1 + 2a/N_theta,
                               w_e = (2e + 1 - N_elev)/N_elev (w = 0 with one elevation bin),
                               x_v, y_v = position of Tx_t + Rx_r  (a target at direction
                               cosines (u, w) gives phase -2pi (x_v u + y_v w) / lambda across
                               the array, so W peaks there); rows e * N_theta + a;
                               lambda = c / (f_c + B/2), the sweep's centre wavelength: the
                               range DFT at the peak bin carries each element's delay at the
                               mean instantaneous frequency of the chirp, not at f_c
  4. power map                 Pw[a,k] = sum_d |Y[a,d,k]|^2
  5. CA-CFAR along range       N[a,k] = mean of Pw over `train` cells each side beyond
                               `guard` cells (cells outside [0, N_s) are skipped)
  6. soft detection            w = sigmoid((ln Pw - ln(alpha N + P_floor)) / beta),
                               P_floor = floor_rel * max Pw
  7. peaks                     local maxima of Pw over the 3x3x3 (elevation, azimuth, range) neighbourhood
                               that exceed P_floor (an all-zero map has no peak);
                               equal values: the lower linear index a*N_s+k wins
  8. sub-bin refine            3-point parabola on l = ln(max(Pw, 1e-30)) per axis (range, azimuth, elevation),
                               clamped to +-0.5 bin, 0 on the border
  9. points                    r = (k + dk) c / (2B), u = -1 + 2(a + da)/N_theta,
                               w = (2(e + de) + 1 - N_elev)/N_elev,
                               p = (r u, r w, r sqrt(1 - u^2 - w^2)), weight w;
                               keep w >= w_min, order by (w desc, linear index asc),
                               at most k_max points
"""
from __future__ import annotations

import numpy as np

from sbr_inputs import C_LIGHT, CfarParams


CfarConfig = CfarParams  # the parameter set is an input shared with the CUDA path


L_FLOOR = 1e-30


def dft_matrix(N: int) -> np.ndarray:
    k = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(k, k) / N)


def dft(x: np.ndarray, axis: int) -> np.ndarray:
    """Direct O(N^2) forward DFT along ``axis`` (e^{-j 2 pi k n / N})."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    y = x @ dft_matrix(x.shape[-1]).T
    return np.moveaxis(y, -1, axis)


def n_elev_of(cfg) -> int:
    return max(1, int(getattr(cfg, "n_elev", 1)))


def steering(radar, n_theta: int, n_elev: int = 1) -> np.ndarray:
    """W [n_elev * n_theta, V] = exp(+j 2 pi (x_v u_a + y_v w_e) / lambda_c),
    lambda_c = c / (f_c + B/2), row e * n_theta + a; u_a = -1 + 2a / n_theta (azimuth
    direction cosine), w_e = (2e + 1 - n_elev) / n_elev (elevation direction cosine, bin
    centres: w = 0 for a single bin); x_v, y_v the virtual element's position (Tx + Rx)."""
    lam = C_LIGHT / (radar.f0 + 0.5 * radar.bandwidth)
    pairs = [(t, r) for t in range(radar.n_tx) for r in range(radar.n_rx)]
    xv = np.array([radar.tx[t, 0] + radar.rx[r, 0] for t, r in pairs])
    yv = np.array([radar.tx[t, 1] + radar.rx[r, 1] for t, r in pairs])
    u = -1.0 + 2.0 * np.arange(n_theta) / n_theta
    w = (2.0 * np.arange(n_elev) + 1.0 - n_elev) / n_elev
    ph = (w[:, None, None] * yv[None, None, :] + u[None, :, None] * xv[None, None, :]) / lam
    return np.exp(2j * np.pi * ph.reshape(n_elev * n_theta, -1))


def cfar_noise(Pw: np.ndarray, guard: int, train: int) -> np.ndarray:
    A, N = Pw.shape
    noise = np.zeros_like(Pw)
    for k in range(N):
        idx = [j for j in range(k - guard - train, k - guard) if 0 <= j < N]
        idx += [j for j in range(k + guard + 1, k + guard + train + 1) if 0 <= j < N]
        if idx:
            noise[:, k] = Pw[:, idx].mean(axis=1)
    return noise


def local_max(Pw: np.ndarray, n_elev: int = 1) -> np.ndarray:
    """Local maxima over the 3 x 3 x 3 (elevation, azimuth, range) neighbourhood of the map
    [n_elev * n_theta, N]; equal values: the lower linear index wins."""
    R, N = Pw.shape
    E, A = n_elev, R // n_elev
    P3 = Pw.reshape(E, A, N)
    pad = np.full((E + 2, A + 2, N + 2), -np.inf)
    pad[1:-1, 1:-1, 1:-1] = P3
    peak = np.ones((E, A, N), bool)
    for de in (-1, 0, 1):
        for da in (-1, 0, 1):
            for dk in (-1, 0, 1):
                if de == 0 and da == 0 and dk == 0:
                    continue
                q = pad[1 + de:1 + de + E, 1 + da:1 + da + A, 1 + dk:1 + dk + N]
                earlier = (de, da, dk) < (0, 0, 0)
                peak &= (P3 > q) if earlier else (P3 >= q)
    return peak.reshape(R, N)


def _refine(l: np.ndarray, rows: np.ndarray, k: np.ndarray, n_elev: int = 1):
    """3-point parabola on l = ln Pw per axis (range, azimuth, elevation), clamped to +-1/2
    bin, 0 on the border of that axis."""
    R, N = l.shape
    A = R // n_elev

    def par(lm, l0, lp):
        den = lm - 2.0 * l0 + lp
        return np.clip(0.5 * (lm - lp) / den, -0.5, 0.5) if den < 0 else 0.0

    dk, da, de = np.zeros(rows.shape), np.zeros(rows.shape), np.zeros(rows.shape)
    for i in range(rows.shape[0]):
        ri, ki = rows[i], k[i]
        e, a = divmod(int(ri), A)
        if 0 < ki < N - 1:
            dk[i] = par(l[ri, ki - 1], l[ri, ki], l[ri, ki + 1])
        if 0 < a < A - 1:
            da[i] = par(l[ri - 1, ki], l[ri, ki], l[ri + 1, ki])
        if 0 < e < n_elev - 1:
            de[i] = par(l[ri - A, ki], l[ri, ki], l[ri + A, ki])
    return dk, da, de


def power_map(cube: np.ndarray, radar, cfg: CfarConfig):
    X = dft(cube, axis=2)                  # range
    X = dft(X, axis=1)                     # Doppler
    W = steering(radar, cfg.n_theta, n_elev_of(cfg))
    Y = np.einsum("av,vdk->adk", W, X)     # angle (azimuth x elevation rows)
    Pw = (np.abs(Y) ** 2).sum(axis=1)
    return X, Y, Pw


def points_at(Pw: np.ndarray, radar, cfg: CfarConfig, a: np.ndarray, k: np.ndarray):
    """Soft weights and refined 3D points at given (angle row, range) cells; row
    a = e * n_theta + azimuth bin."""
    E = n_elev_of(cfg)
    noise = cfar_noise(Pw, cfg.guard, cfg.train)
    floor = cfg.floor_rel * Pw.max()
    l = np.log(np.maximum(Pw, L_FLOOR))
    z = (l[a, k] - np.log(cfg.alpha * noise[a, k] + floor)) / cfg.beta
    w = 1.0 / (1.0 + np.exp(-z))
    dk, da, de = _refine(l, a, k, E)
    az, el = a % cfg.n_theta, a // cfg.n_theta
    r = (k + dk) * C_LIGHT / (2.0 * radar.bandwidth)
    u = np.clip(-1.0 + 2.0 * (az + da) / cfg.n_theta, -1.0, 1.0)
    v = (2.0 * (el + de) + 1.0 - E) / E
    pts = np.stack([r * u, r * v, r * np.sqrt(np.maximum(1.0 - u * u - v * v, 0.0)), w], axis=1)
    return pts


def pointcloud(cube: np.ndarray, radar, cfg: CfarConfig = None) -> dict:
    """Point cloud [n, 4] (x, y, z, w) from an IF cube [V, C, N_s]."""
    cfg = cfg or CfarConfig()
    X, Y, Pw = power_map(cube, radar, cfg)
    peak = local_max(Pw, n_elev_of(cfg)) & (Pw > cfg.floor_rel * Pw.max())
    a, k = np.nonzero(peak)
    pts = points_at(Pw, radar, cfg, a, k) if a.size else np.zeros((0, 4))
    keep = pts[:, 3] >= cfg.w_min if a.size else np.zeros(0, bool)
    a, k, pts = a[keep], k[keep], pts[keep]
    lin = a * Pw.shape[1] + k
    order = np.lexsort((lin, -pts[:, 3]))[: cfg.k_max]
    return dict(points=pts[order], a=a[order], k=k[order], Pw=Pw, X=X, Y=Y)


def image_loss(cube: np.ndarray, target: np.ndarray, radar, cfg: CfarConfig = None) -> float:
    """Spatial multi-antenna loss of Eq. 16 (Section 3.4): the mean over the N image cells of
    the squared difference between the image T(y) of the cube and a target image.

    Reading: T maps the MIMO IF cube to the range-angle power map Pw of steps 1-4 above
    (range DFT, Doppler DFT, angle DFT over n_theta bins, |Y|^2 summed over Doppler), a
    spatial image of n_theta x N_s cells (the 1D virtual array resolves azimuth only)."""
    cfg = cfg or CfarConfig()
    _, _, Pw = power_map(cube, radar, cfg)
    return float(((Pw - np.asarray(target, dtype=np.float64)) ** 2).mean())


# ----------------------------------------------------------------------------
# Chamfer terms and Laplacian smoothness
# ----------------------------------------------------------------------------


def _nn(P: np.ndarray, Q: np.ndarray):
    d2 = ((P[:, None, :3] - Q[None, :, :3]) ** 2).sum(-1)
    j = d2.argmin(axis=1)
    return j, d2[np.arange(P.shape[0]), j]


def chamfer_parity(P: np.ndarray, Q: np.ndarray) -> float:
    """Weighted mean nearest-neighbour Euclidean distance, both directions, averaged [m]."""
    if P.shape[0] == 0 and Q.shape[0] == 0:
        return 0.0
    if P.shape[0] == 0 or Q.shape[0] == 0:
        return float("inf")
    _, dpq = _nn(P, Q)
    _, dqp = _nn(Q, P)
    a = (P[:, 3] * np.sqrt(dpq)).sum() / P[:, 3].sum()
    b = (Q[:, 3] * np.sqrt(dqp)).sum() / Q[:, 3].sum()
    return float(0.5 * (a + b))


def chamfer_loss(P: np.ndarray, Q: np.ndarray, nn_pq=None, nn_qp=None) -> float:
    """Weighted squared Chamfer: sum_i w_i d_i^2 / sum w + sum_j w'_j e_j^2 / sum w'.

    P are the predicted points (x, y, z, w), Q the target.  With ``nn_pq`` /
    ``nn_qp`` given the nearest-neighbour assignment is frozen (FD checks)."""
    if nn_pq is None:
        nn_pq, _ = _nn(P, Q)
    if nn_qp is None:
        nn_qp, _ = _nn(Q, P)
    dpq = ((P[:, :3] - Q[nn_pq, :3]) ** 2).sum(-1)
    dqp = ((Q[:, :3] - P[nn_qp, :3]) ** 2).sum(-1)
    return float((P[:, 3] * dpq).sum() / P[:, 3].sum() + (Q[:, 3] * dqp).sum() / Q[:, 3].sum())


def mesh_neighbours(faces: np.ndarray, nv: int):
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    nb = [[] for _ in range(nv)]
    for i, j in e:
        nb[i].append(j)
        nb[j].append(i)
    return nb


def laplacian(verts: np.ndarray, faces: np.ndarray) -> float:
    """Uniform Laplacian smoothness: mean_i |v_i - mean_{j in N(i)} v_j|^2."""
    v = np.asarray(verts, dtype=np.float64)
    nb = mesh_neighbours(faces, v.shape[0])
    d = np.array([v[i] - v[n].mean(0) if n else np.zeros(3) for i, n in enumerate(nb)])
    return float((d ** 2).sum(-1).mean())
