"""Steady 1D synthetic equations of the DIG method, solved by Newton's method.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The steady form of Eq. (macroscopic_equation) on a 1D slab between two
impermeable walls (x is the wall-normal direction, so u_x = 0 at steady state)
with the constitutive relations of Eq. (full_constitutive):

    d/dx (rho T_t + sigma_xx)                  = 0     x-momentum
    d/dx (sigma_xy),  d/dx (sigma_xz)          = 0     y-, z-momentum
    d/dx (sigma_xy u_y + sigma_xz u_z + q_t + q_r) = 0 total energy
    d/dx (q_r) = (d_r rho / 2) (T - T_r) / (Z tau)     rotational energy
    tau = mu / p, p = rho T, mu = mu_ref T^omega, T = (3 T_t + d_r T_r)/(3 + d_r)

with sigma = sigma_NSF + HoT, q = q_NSF + HoT (Eq. ns_constitutive, kappa from
Eq. kappa_A).  The walls are not modelled by a slip law: the first and last
cell keep the DSMC-sampled u_y, u_z, T_t, T_r (Dirichlet), and the total mass
equals that of the DSMC sample.  Finite volumes with face fluxes from
compact differences; face viscosity at the mean of the two cell temperatures;
face HoT the mean of the two cell values.

Unknowns per cell: rho, u_y, u_z, T_t, T_r.  Newton's method with a Jacobian
from central finite differences (graph colouring over the 3-cell stencil) and
a sparse direct solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fields import F_RHO, F_U, F_TT, F_TR, kappa_coefficients, mu_ref_of

NV = 5  # rho, u_y, u_z, T_t, T_r


def _unpack(x, n):
    X = x.reshape(NV, n)
    return X[0], X[1], X[2], X[3], X[4]


def residual(x: np.ndarray, dsmc: np.ndarray, hot: np.ndarray, cfg: dict) -> np.ndarray:
    n = int(cfg["nx"])
    dx = float(cfg["lx"]) / n
    d_r, omega, Z = float(cfg["d_r"]), float(cfg["omega"]), float(cfg["z_rot"])
    mu_ref = mu_ref_of(float(cfg["kn"]))
    kt_c, kr_c = kappa_coefficients(cfg["a_matrix"], d_r)
    rho, uy, uz, tt, tr = _unpack(x, n)
    # faces i+1/2, i = 0..n-2
    ttf = 0.5 * (tt[:-1] + tt[1:])
    trf = 0.5 * (tr[:-1] + tr[1:])
    Tf = (3.0 * ttf + d_r * trf) / (3.0 + d_r)
    muf = mu_ref * Tf ** omega
    uyf = 0.5 * (uy[:-1] + uy[1:])
    uzf = 0.5 * (uz[:-1] + uz[1:])
    hf = 0.5 * (hot[:-1] + hot[1:])
    sxy = -muf * (uy[1:] - uy[:-1]) / dx + hf[:, 3]
    sxz = -muf * (uz[1:] - uz[:-1]) / dx + hf[:, 4]
    qt = -kt_c * muf * (tt[1:] - tt[:-1]) / dx + hf[:, 6]
    qr = -kr_c * muf * (tr[1:] - tr[:-1]) / dx + hf[:, 9]
    ef = sxy * uyf + sxz * uzf + qt + qr
    P = rho * tt + hot[:, 0]
    T = (3.0 * tt + d_r * tr) / (3.0 + d_r)
    mu = mu_ref * T ** omega
    src = 0.5 * d_r * rho * (rho * T) * (T - tr) / (Z * mu)
    R = np.zeros((NV, n))
    R[0, :-1] = P[1:] - P[:-1]
    R[0, -1] = rho.sum() * dx - dsmc[:, F_RHO].sum() * dx
    for v, (arr, flux, col) in enumerate(((uy, sxy, F_U + 1), (uz, sxz, F_U + 2)), start=1):
        R[v, 1:-1] = flux[1:] - flux[:-1]
        R[v, 0] = arr[0] - dsmc[0, col]
        R[v, -1] = arr[-1] - dsmc[-1, col]
    R[3, 1:-1] = ef[1:] - ef[:-1]
    R[3, 0] = tt[0] - dsmc[0, F_TT]
    R[3, -1] = tt[-1] - dsmc[-1, F_TT]
    R[4, 1:-1] = -(qr[1:] - qr[:-1]) / dx + src[1:-1]
    R[4, 0] = tr[0] - dsmc[0, F_TR]
    R[4, -1] = tr[-1] - dsmc[-1, F_TR]
    return R.reshape(-1)


def _jacobian(x, dsmc, hot, cfg):
    n = int(cfg["nx"])
    dx = float(cfg["lx"]) / n
    rows, cols, vals = [], [], []
    cell_of_row = np.tile(np.arange(n), NV)
    for v in range(NV):
        for r in range(3):
            cells = np.arange(r, n, 3)
            h = 1e-6 * np.maximum(np.abs(x[v * n + cells]), 1.0)
            xp = x.copy()
            xm = x.copy()
            xp[v * n + cells] += h
            xm[v * n + cells] -= h
            dR = residual(xp, dsmc, hot, cfg) - residual(xm, dsmc, hot, cfg)
            # the perturbed cell that row (cell j) sees is the one of j-1, j, j+1 with index = r mod 3
            for row in range(NV * n):
                j = cell_of_row[row]
                if row == n - 1:  # global mass row, filled below
                    continue
                for k in (j - 1, j, j + 1):
                    if 0 <= k < n and k % 3 == r:
                        val = dR[row] / (2.0 * h[(k - r) // 3])
                        if val != 0.0:
                            rows.append(row)
                            cols.append(v * n + k)
                            vals.append(val)
    for k in range(n):
        rows.append(n - 1)
        cols.append(k)
        vals.append(dx)
    return sp.csr_matrix((vals, (rows, cols)), shape=(NV * n, NV * n))


def synth_solve_1d(dsmc: np.ndarray, hot: np.ndarray, cfg: dict, tol: float = 1e-12, max_iter: int = 50):
    """Newton iterations from the DSMC fields until the largest relative
    update is below ``tol``.  Returns (out [ncells x 6] = rho, u_x = 0, u_y,
    u_z, T_t, T_r; iterations; final max |residual|)."""
    n = int(cfg["nx"])
    if n < 3:
        raise ValueError("synth_solve_1d needs at least 3 cells")
    x = np.concatenate([dsmc[:, F_RHO], dsmc[:, F_U + 1], dsmc[:, F_U + 2], dsmc[:, F_TT], dsmc[:, F_TR]])
    it = 0
    for it in range(1, max_iter + 1):
        R = residual(x, dsmc, hot, cfg)
        J = _jacobian(x, dsmc, hot, cfg)
        dxv = spla.spsolve(J.tocsc(), -R)
        lam = 1.0
        xn = x + dxv
        # keep densities and temperatures positive
        while np.any(xn[0:n] <= 0) or np.any(xn[3 * n:] <= 0):
            lam *= 0.5
            xn = x + lam * dxv
        scale = np.maximum(np.abs(x), 1e-3)
        x = xn
        if np.max(np.abs(lam * dxv) / scale) < tol:
            break
    R = residual(x, dsmc, hot, cfg)
    rho, uy, uz, tt, tr = _unpack(x, n)
    out = np.stack([rho, np.zeros(n), uy, uz, tt, tr], axis=1)
    return out, it, float(np.max(np.abs(R)))
