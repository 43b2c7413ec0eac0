"""Steady 2D synthetic equations of the DIG method, solved by Newton's method.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The steady form of Eq. (macroscopic_equation) on a rectangle of nx x ny
cells closed by walls (uniform, or the wall-refined grid of the cavity case
of Sec. 4.1, whose widths grow geometrically from each wall), with the constitutive relations of
Eq. (full_constitutive) (sigma = sigma_NSF + HoT, q = q_NSF + HoT; NSF terms
of Eq. ns_constitutive, kappa from Eq. kappa_A):

    div(rho u)                                               = 0
    div(rho u u + rho T_t I + sigma)                         = 0
    div(rho e u + rho T_t u + sigma . u + q_t + q_r)         = 0
    div(rho e_r u + q_r) = (d_r rho / 2) (T - T_r) / (Z tau)
    e = (3 T_t + d_r T_r) / 2 + |u|^2 / 2,  e_r = d_r T_r / 2,
    tau = mu / p,  p = rho T,  mu = mu_ref T^omega,  T = (3 T_t + d_r T_r) / (3 + d_r)

(u = (u_x, u_y); the flow is planar and u_z takes no part.)  Cell (i, j) is
cell j * nx + i.  Discretisation, the same as the 1D solver's where the two
overlap:

* finite volumes; the flux through a face is the mean of the two cells'
  convective fluxes plus the viscous and heat fluxes from compact normal
  differences and tangential differences averaged from the two cells (central
  within the domain, one-sided in the first and last row); differences are
  taken over the distances between the cell centres (the middle of each
  cell's edges) and a cell's balance divides by its own width; face viscosity
  mu(T_f) with T_f from the face means of T_t and T_r; face HoT the mean of
  the two cells' HoT;
* a fourth-difference dissipation eps4 * lambda_f * (W[i+2] - 3 W[i+1] +
  3 W[i] - W[i-1]) on the conserved variables W = (rho, rho u_x, rho u_y,
  rho e, rho e_r), lambda_f = |u_n| + sqrt(gamma T_f), added to every face
  flux whose four-cell stencil lies in the domain (it damps the odd-even modes
  of the collocated grid; its effect on a smooth solution is O(dx^3));
* the cells next to a wall keep the DSMC-sampled u_x, u_y, T_t, T_r
  (Dirichlet, carrying DSMC's slip and jump) and balance only their mass
  (no flux through a wall); every other cell balances all five;
* a corner cell touches no interior cell, so its mass balance would fix its
  density through its (near-zero) velocity alone: the four corner cells keep
  their whole sampled state and exchange no flux with their neighbours;
* the mass balances of the remaining cells then sum (weighted by the cell
  volumes) to zero identically, and the one of cell 1 is replaced by the
  total mass sum rho V (equal to the DSMC sample's), which the closed walls
  leave undetermined otherwise; the row is written as
  sum_c s_c (rho_c - rho_c,sampled) / n with s_c = n V_c / (L_x L_y) (1 on
  the uniform grid).

Unknowns per cell: rho, u_x, u_y, T_t, T_r.  Newton's method with a Jacobian
from central finite differences (25-colouring of the 5 x 5 stencil) and a
sparse direct solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fields import F_RHO, F_U, F_TT, F_TR, box_edges, kappa_coefficients, mu_ref_of

NV = 5  # rho, u_x, u_y, T_t, T_r
EPS4 = 1.0 / 32.0


def _geom(cfg):
    nx, ny = int(cfg["nx"]), int(cfg["ny"])
    return nx, ny, float(cfg["lx"]) / nx, float(cfg["ly"]) / ny


def _axis_metrics(n, length, mesh, q):
    """Along one axis: the cell widths, the distances between neighbouring
    cell centres (one per interior face) and the denominators of the per-cell
    tangential derivative (centre distance over the two neighbours inside,
    to the one neighbour in the first and last cell)."""
    if mesh == "refined":
        e = box_edges(n, length, q)
        w = np.diff(e)
        c = 0.5 * (e[:-1] + e[1:])
        dn = c[1:] - c[:-1]
        den = np.empty(n)
        den[1:-1] = c[2:] - c[:-2]
        den[0] = c[1] - c[0]
        den[-1] = c[-1] - c[-2]
        return w, dn, den
    h = length / n
    den = np.full(n, 2.0 * h)
    den[0] = den[-1] = h
    return np.full(n, h), np.full(n - 1, h), den


def _metrics(cfg):
    nx, ny = int(cfg["nx"]), int(cfg["ny"])
    mesh = cfg.get("mesh", "box")
    q = float(cfg.get("stretch", 1.0))
    return (_axis_metrics(nx, float(cfg["lx"]), mesh, q), _axis_metrics(ny, float(cfg["ly"]), mesh, q))


def _mass_scale(cfg):
    """s_c = n V_c / (L_x L_y) per cell (rows y, columns x); None on the
    uniform grid (s_c = 1)."""
    if cfg.get("mesh", "box") != "refined":
        return None
    (wx, _, _), (wy, _, _) = _metrics(cfg)
    n = len(wx) * len(wy)
    return n * np.outer(wy, wx) / (float(cfg["lx"]) * float(cfg["ly"]))


def _dy_cells(f, den):
    """d f / d y per cell (rows along axis 0): central inside, one-sided in
    the first and last row, over the centre distances in den."""
    g = np.empty_like(f)
    g[1:-1] = (f[2:] - f[:-2]) / den[1:-1, None]
    g[0] = (f[1] - f[0]) / den[0]
    g[-1] = (f[-1] - f[-2]) / den[-1]
    return g


def _face_fluxes(q, h, W, axis, d, dt, cfg, consts):
    """Fluxes (5 components) through the faces normal to ``axis`` (1: x
    faces between columns i and i+1; 0: y faces between rows j and j+1),
    written for the x direction on arrays transposed so that the face normal
    runs along the last axis.  d: centre distances across the faces (along
    the last axis); dt: the tangential-derivative denominators (rows)."""
    d_r, omega, mu_ref, kt_c, kr_c, gamma = consts
    rho, un, ut, tt, tr = q  # normal and tangential velocity
    # face means
    rf = 0.5 * (rho[:, :-1] + rho[:, 1:])
    unf = 0.5 * (un[:, :-1] + un[:, 1:])
    utf = 0.5 * (ut[:, :-1] + ut[:, 1:])
    ttf = 0.5 * (tt[:, :-1] + tt[:, 1:])
    trf = 0.5 * (tr[:, :-1] + tr[:, 1:])
    Tf = (3.0 * ttf + d_r * trf) / (3.0 + d_r)
    muf = mu_ref * Tf ** omega
    # normal (compact) and tangential (averaged) derivatives at the faces
    dun_n = (un[:, 1:] - un[:, :-1]) / d
    dut_n = (ut[:, 1:] - ut[:, :-1]) / d
    dtt_n = (tt[:, 1:] - tt[:, :-1]) / d
    dtr_n = (tr[:, 1:] - tr[:, :-1]) / d
    gun = _dy_cells(un, dt)
    gut = _dy_cells(ut, dt)
    dun_t = 0.5 * (gun[:, :-1] + gun[:, 1:])
    dut_t = 0.5 * (gut[:, :-1] + gut[:, 1:])
    hf = 0.5 * (h[:, :-1] + h[:, 1:])  # [.., 6]: s_nn, s_nt, q_t n, q_r n (+ unused)
    s_nn = -muf * ((4.0 / 3.0) * dun_n - (2.0 / 3.0) * dut_t) + hf[..., 0]
    s_nt = -muf * (dut_n + dun_t) + hf[..., 1]
    qt = -kt_c * muf * dtt_n + hf[..., 2]
    qr = -kr_c * muf * dtr_n + hf[..., 3]
    # convective fluxes: mean of the two cells' values
    e = 0.5 * (3.0 * tt + d_r * tr) + 0.5 * (un * un + ut * ut)
    er = 0.5 * d_r * tr
    cf = [rho * un, rho * un * un + rho * tt, rho * un * ut, rho * un * (e + tt), rho * un * er]
    F = [0.5 * (c[:, :-1] + c[:, 1:]) for c in cf]
    F[1] = F[1] + s_nn
    F[2] = F[2] + s_nt
    F[3] = F[3] + s_nn * unf + s_nt * utf + qt + qr
    F[4] = F[4] + qr
    # fourth-difference dissipation where the stencil i-1 .. i+2 exists
    lam = np.abs(unf) + np.sqrt(gamma * Tf)
    nf = F[0].shape[1]
    for k in range(NV):
        w = W[k]
        dk = np.zeros_like(F[k])
        if nf >= 3:
            dk[:, 1:-1] = w[:, 3:] - 3.0 * w[:, 2:-1] + 3.0 * w[:, 1:-2] - w[:, :-3]
        F[k] = F[k] + EPS4 * lam * dk
    return F


def residual(x: np.ndarray, dsmc: np.ndarray, hot: np.ndarray, cfg: dict) -> np.ndarray:
    nx, ny, _, _ = _geom(cfg)
    (wx, dnx, dtx), (wy, dny, dty) = _metrics(cfg)
    n = nx * ny
    d_r, omega, Z = float(cfg["d_r"]), float(cfg["omega"]), float(cfg["z_rot"])
    mu_ref = mu_ref_of(float(cfg["kn"]))
    kt_c, kr_c = kappa_coefficients(cfg["a_matrix"], d_r)
    gamma = (5.0 + d_r) / (3.0 + d_r)
    consts = (d_r, omega, mu_ref, kt_c, kr_c, gamma)
    X = x.reshape(NV, ny, nx)
    rho, ux, uy, tt, tr = X
    H = hot.reshape(ny, nx, 12)
    e = 0.5 * (3.0 * tt + d_r * tr) + 0.5 * (ux * ux + uy * uy)
    W = [rho, rho * ux, rho * uy, rho * e, rho * 0.5 * d_r * tr]
    # x faces: normal x, tangential y; HoT (s_xx, s_xy, q_t,x, q_r,x)
    hx = np.stack([H[..., 0], H[..., 3], H[..., 6], H[..., 9]], axis=-1)
    Fx = _face_fluxes((rho, ux, uy, tt, tr), hx, W, 1, dnx, dty, cfg, consts)
    # y faces: transpose so that y runs along the last axis; normal y,
    # tangential x; HoT (s_yy, s_xy, q_t,y, q_r,y)
    hy = np.stack([H[..., 1], H[..., 3], H[..., 7], H[..., 10]], axis=-1).transpose(1, 0, 2)
    Wy = [W[0].T, W[2].T, W[1].T, W[3].T, W[4].T]  # (rho, rho u_n, rho u_t, ...) with n = y
    Fy = _face_fluxes((rho.T, uy.T, ux.T, tt.T, tr.T), hy, Wy, 0, dny, dtx, cfg, consts)
    # momentum components of the y faces: (normal, tangential) = (y, x)
    Fy = [Fy[0].T, Fy[2].T, Fy[1].T, Fy[3].T, Fy[4].T]
    # no flux through the faces of the four corner cells
    for F in Fx:
        F[0, 0] = F[-1, 0] = F[0, -1] = F[-1, -1] = 0.0
    for F in Fy:
        F[0, 0] = F[-1, 0] = F[0, -1] = F[-1, -1] = 0.0
    div = []
    for k in range(NV):
        dk = np.zeros((ny, nx))
        dk[:, :-1] += Fx[k] / wx[None, :-1]
        dk[:, 1:] -= Fx[k] / wx[None, 1:]
        dk[:-1, :] += Fy[k] / wy[:-1, None]
        dk[1:, :] -= Fy[k] / wy[1:, None]
        div.append(dk)
    T = (3.0 * tt + d_r * tr) / (3.0 + d_r)
    mu = mu_ref * T ** omega
    src = 0.5 * d_r * rho * (rho * T) * (T - tr) / (Z * mu)
    R = np.stack([div[0], div[1], div[2], div[3], div[4] - src])
    # wall-adjacent cells: Dirichlet u_x, u_y, T_t, T_r; mass balance only
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    D = dsmc.reshape(ny, nx, -1)
    for k, col in ((1, F_U), (2, F_U + 1), (3, F_TT), (4, F_TR)):
        R[k][ring] = (X[k] - D[..., col])[ring]
    # corner cells keep their sampled state (density too)
    for cj, ci in ((0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)):
        R[0, cj, ci] = rho[cj, ci] - D[cj, ci, F_RHO]
    # the mass balances of the other cells sum to zero identically: the one of
    # cell 1 is replaced by the total mass
    s = _mass_scale(cfg)
    if s is None:
        R[0, 0, 1] = (rho.sum() - D[..., F_RHO].sum()) / n
    else:
        R[0, 0, 1] = ((s * rho).sum() - (s * D[..., F_RHO]).sum()) / n
    return R.reshape(-1)


def _jacobian(x, dsmc, hot, cfg):
    nx, ny, _, _ = _geom(cfg)
    n = nx * ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    ii, jj = ii.ravel(), jj.ravel()
    rows, cols, vals = [], [], []
    # residual of cell c depends on the cells within |di| <= 2, |dj| <= 2
    for v in range(NV):
        for cx in range(5):
            for cy in range(5):
                sel = np.nonzero((ii % 5 == cx) & (jj % 5 == cy))[0]
                if sel.size == 0:
                    continue
                hh = 1e-6 * np.maximum(np.abs(x[v * n + sel]), 1.0)
                xp = x.copy()
                xm = x.copy()
                xp[v * n + sel] += hh
                xm[v * n + sel] -= hh
                dR = (residual(xp, dsmc, hot, cfg) - residual(xm, dsmc, hot, cfg)).reshape(NV, n)
                hcell = np.zeros(n)
                hcell[sel] = hh
                for c in range(n):
                    # the perturbed cell in c's stencil, if any
                    ki = ii[c] + ((cx - ii[c]) % 5 if (cx - ii[c]) % 5 <= 2 else (cx - ii[c]) % 5 - 5)
                    kj = jj[c] + ((cy - jj[c]) % 5 if (cy - jj[c]) % 5 <= 2 else (cy - jj[c]) % 5 - 5)
                    if not (0 <= ki < nx and 0 <= kj < ny):
                        continue
                    k = kj * nx + ki
                    for r in range(NV):
                        val = dR[r, c]
                        if val != 0.0:
                            rows.append(r * n + c)
                            cols.append(v * n + k)
                            vals.append(val / (2.0 * hcell[k]))
    # the total-mass row (cell 1) depends on every cell
    keep = [t for t in range(len(rows)) if rows[t] != 1]
    rows = [rows[t] for t in keep] + [1] * n
    cols = [cols[t] for t in keep] + list(range(n))
    s = _mass_scale(cfg)
    vals = [vals[t] for t in keep] + (list(s.ravel() / n) if s is not None else [1.0 / n] * n)
    return sp.csr_matrix((vals, (rows, cols)), shape=(NV * n, NV * n))


def initial_state(dsmc: np.ndarray) -> np.ndarray:
    return np.concatenate([dsmc[:, F_RHO], dsmc[:, F_U], dsmc[:, F_U + 1], dsmc[:, F_TT], dsmc[:, F_TR]])


def synth_solve_2d(dsmc: np.ndarray, hot: np.ndarray, cfg: dict, tol: float = 1e-12, max_iter: int = 50):
    """Newton iterations from the DSMC fields until the largest relative
    update of a full step is below ``tol``.  Returns (out [ncells x 6] = rho,
    u_x, u_y, u_z (the sampled one), T_t, T_r; iterations; final max
    |residual|); when positivity cuts a step below 1/1024 (a stall: no
    solution near the state) out is the sampled fields."""
    nx, ny, _, _ = _geom(cfg)
    if nx < 3 or ny < 3:
        raise ValueError("synth_solve_2d needs at least 3 x 3 cells")
    n = nx * ny
    x = initial_state(dsmc)
    it = 0
    stalled = False
    for it in range(1, max_iter + 1):
        R = residual(x, dsmc, hot, cfg)
        J = _jacobian(x, dsmc, hot, cfg)
        dxv = spla.spsolve(J.tocsc(), -R)
        # halve the step (at most 60 times) until rho, T_t, T_r stay
        # positive and finite; a step cut below 1/1024 is a stall (no
        # solution near this state): the sampled fields are the answer
        lam = 1.0
        xn = x + dxv
        for _ in range(60):
            if np.all(np.isfinite(xn)) and not (np.any(xn[0:n] <= 0) or np.any(xn[3 * n:] <= 0)):
                break
            lam *= 0.5
            xn = x + lam * dxv
        if lam < 1.0 / 1024.0 or not np.all(np.isfinite(xn)):
            stalled = True
            break
        scale = np.maximum(np.abs(x), 1e-3)
        x = xn
        if lam == 1.0 and np.max(np.abs(dxv) / scale) < tol:
            break
    R = residual(x, dsmc, hot, cfg)
    X = x.reshape(NV, n)
    out = np.stack([X[0], X[1], X[2], dsmc[:, F_U + 2], X[3], X[4]], axis=1)
    if stalled:
        out = np.stack([dsmc[:, F_RHO], dsmc[:, F_U], dsmc[:, F_U + 1], dsmc[:, F_U + 2], dsmc[:, F_TT],
                        dsmc[:, F_TR]], axis=1)
    return out, it, float(np.max(np.abs(R)))
