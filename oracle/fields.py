"""Cell fields, NSF constitutive relations, higher-order terms and Kn_GLL.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy, FP64,
one formula per line as the paper writes it.

Field layout (18 per cell):
    0 rho, 1-3 u, 4 T_t, 5 T_r, 6-11 sigma (xx yy zz xy xz yz),
    12-14 q_t, 15-17 q_r
HoT layout (12 per cell): sigma (xx yy zz xy xz yz), q_t (3), q_r (3).
"""
from __future__ import annotations

import math
import numpy as np

F_RHO, F_U, F_TT, F_TR, F_SIG, F_QT, F_QR = 0, 1, 4, 5, 6, 12, 15
SIG_IJ = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def fields_from_sums(acc: np.ndarray, nsamples: int, fnum: float, vcell, d_r: float) -> np.ndarray:
    """Eq. (DSMC_macroscopic), time averaged over ``nsamples`` steps.

    The raw sums over all sampled steps are combined into central moments about
    the time-averaged mean velocity (cumulative sampling).  I_r is the
    rotational energy of a molecule, so T_r = 2 sum I_r / (d_r N) and
    q_r = n sum c I_r.  Cells that were never occupied return zeros.
    """
    acc = np.asarray(acc, dtype=np.float64)
    nc = acc.shape[0]
    out = np.zeros((nc, 18), np.float64)
    S = float(nsamples)
    for c in range(nc):
        a = acc[c]
        N = a[0]
        if N <= 0:
            continue
        sv = a[1:4]
        svv = np.array([[a[4], a[7], a[8]], [a[7], a[5], a[9]], [a[8], a[9], a[6]]])
        sv3 = a[10:13]
        si = a[13]
        siv = a[14:17]
        u = sv / N
        # sum c_i c_j with c = v - u
        scc = svv - np.outer(sv, u) - np.outer(u, sv) + N * np.outer(u, u)
        sc2 = np.trace(scc)
        # sum c_i |c|^2, expanded term by term from (v_i - u_i)(|v|^2 - 2 u.v + |u|^2)
        u2 = float(u @ u)
        sv2 = float(np.trace(svv))
        sc3 = (sv3 - 2.0 * (svv @ u) + u2 * sv
               - u * sv2 + 2.0 * u * float(u @ sv) - N * u * u2)
        vc = float(vcell[c]) if np.ndim(vcell) else vcell  # per-cell volumes (annulus)
        n_over_v = fnum / (vc * S)
        out[c, F_RHO] = fnum * N / (S * vc)
        out[c, F_U:F_U + 3] = u
        out[c, F_TT] = sc2 / (3.0 * N)
        out[c, F_TR] = 2.0 * si / (d_r * N)
        for k, (i, j) in enumerate(SIG_IJ):
            out[c, F_SIG + k] = n_over_v * (scc[i, j] - (sc2 / 3.0 if i == j else 0.0))
        out[c, F_QT:F_QT + 3] = 0.5 * n_over_v * sc3
        out[c, F_QR:F_QR + 3] = n_over_v * (siv - u * si)
    return out


def fields_from_particles(vx, vy, vz, ir, fnum, vcell, d_r) -> np.ndarray:
    """Eq. (DSMC_macroscopic) for one cell and one instant, straight from the
    particle list (used to pin ``fields_from_sums``)."""
    v = np.stack([vx, vy, vz], axis=1).astype(np.float64)
    ir = np.asarray(ir, np.float64)
    N = v.shape[0]
    out = np.zeros(18)
    u = v.mean(axis=0)
    c = v - u
    c2 = (c * c).sum(axis=1)
    n_over_v = fnum / vcell
    out[F_RHO] = n_over_v * N
    out[F_U:F_U + 3] = u
    out[F_TT] = c2.sum() / (3.0 * N)
    out[F_TR] = 2.0 * ir.sum() / (d_r * N)
    for k, (i, j) in enumerate(SIG_IJ):
        out[F_SIG + k] = n_over_v * (c[:, i] * c[:, j] - (c2 / 3.0 if i == j else 0.0)).sum()
    out[F_QT:F_QT + 3] = 0.5 * n_over_v * (c * c2[:, None]).sum(axis=0)
    out[F_QR:F_QR + 3] = n_over_v * (c * ir[:, None]).sum(axis=0)
    return out


def kappa_coefficients(a_matrix, d_r: float):
    """Eq. (kappa_A): (kappa_t, kappa_r) = (mu/2) A^-1 (5, d_r); returns the
    coefficients kappa/mu."""
    A = np.array([[a_matrix[0], a_matrix[1]], [a_matrix[2], a_matrix[3]]], np.float64)
    k = 0.5 * np.linalg.solve(A, np.array([5.0, d_r]))
    return float(k[0]), float(k[1])


def mu_ref_of(kn: float) -> float:
    """Non-dimensional viscosity at T0 from the Kn definition of Sec. 2."""
    return kn * math.sqrt(2.0 / math.pi)


def grad_cells(f: np.ndarray, nx: int, ny: int, dx: float, dy: float, dim: int):
    """Cell-centred gradients: central differences inside, one-sided first
    differences in the first and last cell of each line, zero along an axis
    with a single cell."""
    g = f.reshape(ny, nx)
    gx = np.zeros_like(g)
    gy = np.zeros_like(g)
    if nx >= 2:
        gx[:, 1:-1] = (g[:, 2:] - g[:, :-2]) / (2.0 * dx)
        gx[:, 0] = (g[:, 1] - g[:, 0]) / dx
        gx[:, -1] = (g[:, -1] - g[:, -2]) / dx
    if dim == 2 and ny >= 2:
        gy[1:-1, :] = (g[2:, :] - g[:-2, :]) / (2.0 * dy)
        gy[0, :] = (g[1, :] - g[0, :]) / dy
        gy[-1, :] = (g[-1, :] - g[-2, :]) / dy
    return gx.reshape(-1), gy.reshape(-1)


def ring_edges(cfg: dict) -> np.ndarray:
    """Ring radii R_0 = r_in < ... < R_ny = r_out of the annulus around a
    cylinder: widths growing by the factor `stretch` from ring to ring
    (uniform for stretch 1)."""
    nr, q = int(cfg["ny"]), float(cfg.get("stretch", 1.0))
    r_in, r_out = float(cfg["r_in"]), float(cfg["r_out"])
    j = np.arange(nr + 1, dtype=np.float64)
    f = j / nr if q == 1.0 else (q ** j - 1.0) / (q ** nr - 1.0)
    r = r_in + (r_out - r_in) * f
    r[0], r[-1] = r_in, r_out
    return r


def box_edges(n: int, length: float, q: float) -> np.ndarray:
    """Cell edges of the wall-refined box along one axis: n widths growing
    geometrically by q from both walls to the middle (w_i proportional to
    q^min(i, n-1-i)), summing to the length."""
    i = np.arange(n)
    w = q ** np.minimum(i, n - 1 - i).astype(np.float64)
    e = np.concatenate([[0.0], np.cumsum(length * w / w.sum())])
    e[-1] = length
    return e


def _d_nonuniform(g: np.ndarray, xc: np.ndarray, axis: int):
    """d/dx along `axis` of cell values g at centres xc: the three-point
    formula on the unequal spacing (exact for quadratics), one-sided first
    differences at the two ends."""
    g = np.moveaxis(g, axis, 0)
    d = np.zeros_like(g)
    hm = (xc[1:-1] - xc[:-2])[:, None]
    hp = (xc[2:] - xc[1:-1])[:, None]
    d[1:-1] = (hm * hm * g[2:] - hp * hp * g[:-2] + (hp * hp - hm * hm) * g[1:-1]) / (hp * hm * (hp + hm))
    d[0] = (g[1] - g[0]) / (xc[1] - xc[0])
    d[-1] = (g[-1] - g[-2]) / (xc[-1] - xc[-2])
    return np.moveaxis(d, 0, axis)


def grad_refined(f: np.ndarray, nx: int, ny: int, xe: np.ndarray, ye: np.ndarray):
    """Cell-centred gradient on the wall-refined box (cell centres at the
    middle of their edges)."""
    g = f.reshape(ny, nx)
    xc, yc = 0.5 * (xe[:-1] + xe[1:]), 0.5 * (ye[:-1] + ye[1:])
    return _d_nonuniform(g, xc, 1).reshape(-1), _d_nonuniform(g, yc, 0).reshape(-1)


def grad_annulus(f: np.ndarray, nt: int, nr: int, redges: np.ndarray):
    """Cartesian gradient (d/dx, d/dy) of a cell field on the annulus (cell j
    nt + k: ring j, sector k), from its polar derivatives at the cell centre
    (mid radius r_j, angle theta_k = 2 pi (k + 1/2) / nt):
      d/dr: the three-point formula on the stretched rings (exact for
            quadratics in r), a one-sided first difference in the first
            and the last ring;
      (1/r) d/dtheta: (f_{k+1} - f_{k-1}) / (2 r sin(dtheta)), periodic in
            k (second order, and exact for fields linear in x and y);
      d/dx = cos(theta) d/dr - sin(theta) (1/r) d/dtheta,
      d/dy = sin(theta) d/dr + cos(theta) (1/r) d/dtheta."""
    g = f.reshape(nr, nt)
    rc = 0.5 * (redges[:-1] + redges[1:])
    dr = np.zeros_like(g)
    if nr >= 2:
        hm = rc[1:-1] - rc[:-2]
        hp = rc[2:] - rc[1:-1]
        dr[1:-1, :] = ((hm * hm)[:, None] * g[2:, :] - (hp * hp)[:, None] * g[:-2, :]
                       + (hp * hp - hm * hm)[:, None] * g[1:-1, :]) / (hp * hm * (hp + hm))[:, None]
        dr[0, :] = (g[1, :] - g[0, :]) / (rc[1] - rc[0])
        dr[-1, :] = (g[-1, :] - g[-2, :]) / (rc[-1] - rc[-2])
    dth = 2.0 * math.pi / nt
    dt = (np.roll(g, -1, axis=1) - np.roll(g, 1, axis=1)) / (2.0 * rc[:, None] * math.sin(dth))
    th = 2.0 * math.pi * (np.arange(nt) + 0.5) / nt
    c, s = np.cos(th)[None, :], np.sin(th)[None, :]
    return (c * dr - s * dt).reshape(-1), (s * dr + c * dt).reshape(-1)


def gradient_of(cfg: dict):
    """The cell-centred gradient f -> (d/dx, d/dy) of the configuration's
    mesh: uniform box, annulus or wall-refined box."""
    dim, nx = int(cfg["dim"]), int(cfg["nx"])
    ny = int(cfg.get("ny", 1)) if dim == 2 else 1
    mesh = cfg.get("mesh", "box")
    if mesh == "annulus":
        re = ring_edges(cfg)
        return lambda f: grad_annulus(f, nx, ny, re)
    if mesh == "refined":
        q = float(cfg["stretch"])
        xe, ye = box_edges(nx, float(cfg["lx"]), q), box_edges(ny, float(cfg["ly"]), q)
        return lambda f: grad_refined(f, nx, ny, xe, ye)
    dx = float(cfg["lx"]) / nx
    dy = float(cfg.get("ly", 1.0)) / ny if dim == 2 else 1.0
    return lambda f: grad_cells(f, nx, ny, dx, dy, dim)


def hot_kngll(fields: np.ndarray, cfg: dict):
    """Eq. (ns_constitutive), Eq. (hot_constitutive) and Eq. (Kn_GLL).

    Returns (hot [ncells x 12] with zeros where Kn_GLL < Kn_ref, kn_gll,
    mask) where mask is True where the higher-order terms are kept.
    mu = mu_ref T^omega at the total temperature T = (3 T_t + d_r T_r)/(3+d_r);
    lambda = mu/(rho T) sqrt(pi T / 2); the velocity term of Kn_GLL is
    |grad |u|| / max(|u|, sqrt(gamma T)) so that it stays finite at rest.
    """
    dim, nx = int(cfg["dim"]), int(cfg["nx"])
    ny = int(cfg.get("ny", 1)) if dim == 2 else 1
    dx = float(cfg["lx"]) / nx
    dy = float(cfg.get("ly", 1.0)) / ny if dim == 2 else 1.0
    grad = gradient_of(cfg)
    d_r, omega = float(cfg["d_r"]), float(cfg["omega"])
    mu_ref = mu_ref_of(float(cfg["kn"]))
    kt_c, kr_c = kappa_coefficients(cfg["a_matrix"], d_r)
    rho = fields[:, F_RHO]
    u = fields[:, F_U:F_U + 3]
    tt = fields[:, F_TT]
    tr = fields[:, F_TR]
    T = (3.0 * tt + d_r * tr) / (3.0 + d_r)
    mu = mu_ref * T ** omega
    grads = {}
    for name, f in (("ux", u[:, 0]), ("uy", u[:, 1]), ("uz", u[:, 2]), ("tt", tt), ("tr", tr), ("rho", rho)):
        grads[name] = grad(f)
    (dux_dx, dux_dy), (duy_dx, duy_dy), (duz_dx, duz_dy) = grads["ux"], grads["uy"], grads["uz"]
    div_u = dux_dx + duy_dy
    # sigma_NSF = -mu (grad u + grad u^T - 2/3 div u I), d/dz = 0
    sig = np.zeros((len(rho), 6))
    sig[:, 0] = -mu * (2.0 * dux_dx - 2.0 / 3.0 * div_u)
    sig[:, 1] = -mu * (2.0 * duy_dy - 2.0 / 3.0 * div_u)
    sig[:, 2] = -mu * (0.0 - 2.0 / 3.0 * div_u)
    sig[:, 3] = -mu * (dux_dy + duy_dx)
    sig[:, 4] = -mu * (duz_dx)
    sig[:, 5] = -mu * (duz_dy)
    qt = np.zeros((len(rho), 3))
    qr = np.zeros((len(rho), 3))
    qt[:, 0] = -kt_c * mu * grads["tt"][0]
    qt[:, 1] = -kt_c * mu * grads["tt"][1]
    qr[:, 0] = -kr_c * mu * grads["tr"][0]
    qr[:, 1] = -kr_c * mu * grads["tr"][1]
    hot = np.zeros((len(rho), 12))
    hot[:, 0:6] = fields[:, F_SIG:F_SIG + 6] - sig
    hot[:, 6:9] = fields[:, F_QT:F_QT + 3] - qt
    hot[:, 9:12] = fields[:, F_QR:F_QR + 3] - qr
    # Kn_GLL
    gamma = (5.0 + d_r) / (3.0 + d_r)
    speed = np.sqrt((u * u).sum(axis=1))
    gs = grad(speed)
    lam = mu / (rho * T) * np.sqrt(math.pi * T / 2.0)
    g_rho = np.hypot(*grads["rho"]) / rho
    g_u = np.hypot(*gs) / np.maximum(speed, np.sqrt(gamma * T))
    g_tt = np.hypot(*grads["tt"]) / tt
    g_tr = np.hypot(*grads["tr"]) / tr
    kn_gll = lam * np.maximum(np.maximum(g_rho, g_u), np.maximum(g_tt, g_tr))
    mask = kn_gll >= float(cfg["kn_ref"])
    hot[~mask, :] = 0.0
    return hot, kn_gll, mask
