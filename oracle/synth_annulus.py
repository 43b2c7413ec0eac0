"""Steady synthetic equations of the DIG method on the annular mesh around a
cylinder (the flow past a cylinder of Sec. 4.2; Sec. 3 step 3), solved by
Newton's method.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The equations and constitutive relations are those of ``oracle/synth2d.py``
(Eq. macroscopic_equation with Eq. full_constitutive: sigma = sigma_NSF +
HoT, q = q_NSF + HoT, NSF terms of Eq. ns_constitutive, kappa from
Eq. kappa_A, the rotational relaxation source), with the velocity in
Cartesian components, on nt sectors x nr rings: cell j nt + k lies in ring
j (radii R_j .. R_{j+1}, ``fields.ring_edges``) and sector k (angles
2 pi k / nt .. 2 pi (k + 1) / nt).  Finite volumes:

* the face vector S of a face is the integral of its outward normal: an arc
  between rings at radius R, in sector k, has S = 2 R sin(dtheta / 2)
  e_r(theta_k) (theta_k the sector's middle angle); a ray between sectors at
  angle phi, in ring j, has S = (R_{j+1} - R_j) e_theta(phi); the cell volume
  is the sector's area (the DSMC cell's).  A cell's four face vectors sum to
  zero, so a uniform state is an exact discrete solution;
* the flux through a face is written in the face's frame (n = S / |S|,
  t = n turned by +90 degrees) as on the box: the mean of the two cells'
  convective fluxes, plus sigma_nn, sigma_nt and the heat fluxes from the
  difference of the two cells' u_n, u_t, T_t, T_r over the distance between
  their centres (the middle radius and angle of each cell; the two centres
  lie on the face's normal line) and the tangential derivatives t.grad u_n,
  t.grad u_t averaged from the two cells' Cartesian gradients (the polar
  formula of ``fields.grad_annulus``); face viscosity mu(T_f) from the face
  means of T_t and T_r; face HoT the mean of the two cells' HoT turned into
  the frame; the fourth-difference dissipation of the box on the conserved
  variables in the face's frame, along the ring index (arcs, where rings
  f-1 .. f+2 exist) or the sector index (rays, periodic);
* both boundary rings keep their whole sampled state: the one next to the
  cylinder (the wall's Knudsen layer, as the box's wall cells keep u, T)
  and the outer one, on the freestream side; every other cell balances all
  five.  The rings' densities fix the mass, so there is no total-mass row.
  (A first ring that balanced its mass with its velocity held, as the box's
  wall cells do, has no solution behind a hypersonic cylinder: its density
  collapses in the wake.)

Newton's method from the sampled fields, the Jacobian by central
differences (cells of one colour perturbed together), a dense solve (the
meshes of the tests are small); the update rule of ``synth2d``.
"""
from __future__ import annotations

import math

import numpy as np

from .fields import F_RHO, F_TR, F_TT, F_U, grad_annulus, kappa_coefficients, mu_ref_of, ring_edges

NV = 5
EPS4 = 1.0 / 32.0


def geometry(cfg: dict):
    """(nt, nr, R, rc, dth, thc): ring edges R, middle radii rc, sector
    angle dth, middle angles thc."""
    nt, nr = int(cfg["nx"]), int(cfg["ny"])
    R = ring_edges(cfg)
    rc = 0.5 * (R[:-1] + R[1:])
    dth = 2.0 * math.pi / nt
    thc = dth * (np.arange(nt) + 0.5)
    return nt, nr, R, rc, dth, thc


def volumes(cfg: dict) -> np.ndarray:
    nt, nr, R, _, dth, _ = geometry(cfg)
    return np.repeat(0.5 * dth * (R[1:] ** 2 - R[:-1] ** 2), nt)


def _consts(cfg):
    d_r, omega, Z = float(cfg["d_r"]), float(cfg["omega"]), float(cfg["z_rot"])
    kt, kr = kappa_coefficients(cfg["a_matrix"], d_r)
    return d_r, omega, mu_ref_of(float(cfg["kn"])), Z, kt, kr, (5.0 + d_r) / (3.0 + d_r)


def _conserved(rho, un, ut, tt, tr, d_r):
    e = 0.5 * (3.0 * tt + d_r * tr) + 0.5 * (un * un + ut * ut)
    return [rho, rho * un, rho * ut, rho * e, rho * 0.5 * d_r * tr]


def _frame(q, n):
    """(rho, u_n, u_t, T_t, T_r) of states q = (rho, u_x, u_y, T_t, T_r) in
    the frames n (m x 2), t = (-n_y, n_x)."""
    rho, ux, uy, tt, tr = q
    nx_, ny_ = n[:, 0], n[:, 1]
    return rho, ux * nx_ + uy * ny_, -ux * ny_ + uy * nx_, tt, tr


def _face_flux(qL, qR, gL, gR, hL, hR, n, d, c, diss=None):
    """Flux per unit face area through faces of unit normals n (m x 2)
    between cells of states qL, qR (tuples of m-arrays), Cartesian velocity
    gradients gL, gR (du_x/dx, du_x/dy, du_y/dx, du_y/dy), HoT hL, hR
    (m x 12) and centre distance d; diss = (qm, qp, mask): the dissipation's
    outer cells and where it applies.  Returns (mass, x-momentum,
    y-momentum, energy, rotational energy)."""
    d_r, omega, mu_ref, Z, kt_c, kr_c, gamma = c
    nx_, ny_ = n[:, 0], n[:, 1]
    tx_, ty_ = -ny_, nx_
    rl, unl, utl, ttl, trl = _frame(qL, n)
    rr, unr, utr, ttr, trr = _frame(qR, n)
    unf, utf = 0.5 * (unl + unr), 0.5 * (utl + utr)
    ttf, trf = 0.5 * (ttl + ttr), 0.5 * (trl + trr)
    Tf = (3.0 * ttf + d_r * trf) / (3.0 + d_r)
    muf = mu_ref * Tf ** omega
    dun_n, dut_n = (unr - unl) / d, (utr - utl) / d
    dtt_n, dtr_n = (ttr - ttl) / d, (trr - trl) / d

    def tangential(g):
        dxx, dxy, dyx, dyy = g
        tgx = tx_ * dxx + ty_ * dxy  # t . grad u_x
        tgy = tx_ * dyx + ty_ * dyy  # t . grad u_y
        return nx_ * tgx + ny_ * tgy, tx_ * tgx + ty_ * tgy

    gnl, gtl = tangential(gL)
    gnr, gtr = tangential(gR)
    dun_t, dut_t = 0.5 * (gnl + gnr), 0.5 * (gtl + gtr)

    def hot_frame(h):
        sxx, syy, sxy = h[:, 0], h[:, 1], h[:, 3]
        snn = sxx * nx_ * nx_ + 2.0 * sxy * nx_ * ny_ + syy * ny_ * ny_
        snt = sxx * nx_ * tx_ + sxy * (nx_ * ty_ + ny_ * tx_) + syy * ny_ * ty_
        return snn, snt, h[:, 6] * nx_ + h[:, 7] * ny_, h[:, 9] * nx_ + h[:, 10] * ny_

    hl, hr = hot_frame(hL), hot_frame(hR)
    h_nn, h_nt, h_qt, h_qr = (0.5 * (a + b) for a, b in zip(hl, hr))
    s_nn = -muf * ((4.0 / 3.0) * dun_n - (2.0 / 3.0) * dut_t) + h_nn
    s_nt = -muf * (dut_n + dun_t) + h_nt
    qt = -kt_c * muf * dtt_n + h_qt
    qr = -kr_c * muf * dtr_n + h_qr

    def convective(rho, un, ut, tt, tr):
        e = 0.5 * (3.0 * tt + d_r * tr) + 0.5 * (un * un + ut * ut)
        return [rho * un, rho * un * un + rho * tt, rho * un * ut, rho * un * (e + tt), rho * un * (0.5 * d_r * tr)]

    cl, cr = convective(rl, unl, utl, ttl, trl), convective(rr, unr, utr, ttr, trr)
    F = [0.5 * (a + b) for a, b in zip(cl, cr)]
    F[1] = F[1] + s_nn
    F[2] = F[2] + s_nt
    F[3] = F[3] + s_nn * unf + s_nt * utf + qt + qr
    F[4] = F[4] + qr
    if diss is not None:
        qm, qp, mask = diss
        wm = _conserved(*_frame(qm, n), d_r)
        w0 = _conserved(rl, unl, utl, ttl, trl, d_r)
        w1 = _conserved(rr, unr, utr, ttr, trr, d_r)
        wp = _conserved(*_frame(qp, n), d_r)
        lam = np.abs(unf) + np.sqrt(gamma * Tf)
        for k in range(NV):
            F[k] = F[k] + np.where(mask, EPS4 * lam * (wp[k] - 3.0 * w1[k] + 3.0 * w0[k] - wm[k]), 0.0)
    return [F[0], F[1] * nx_ + F[2] * tx_, F[1] * ny_ + F[2] * ty_, F[3], F[4]]


def residual(x: np.ndarray, dsmc: np.ndarray, hot: np.ndarray, cfg: dict) -> np.ndarray:
    """Residual rows (5 x ncells, flattened) of the state x (rho, u_x, u_y,
    T_t, T_r, each ncells long, cell j nt + k)."""
    nt, nr, R, rc, dth, thc = geometry(cfg)
    c = _consts(cfg)
    d_r, omega, mu_ref, Z = c[0], c[1], c[2], c[3]
    X = x.reshape(NV, nr, nt)
    H = hot.reshape(nr, nt, 12)
    G = [a.reshape(nr, nt) for a in (*grad_annulus(X[1].ravel(), nt, nr, R), *grad_annulus(X[2].ravel(), nt, nr, R))]
    s2 = math.sin(0.5 * dth)

    def cells(jj, kk):
        return tuple(X[v][jj, kk].ravel() for v in range(NV))

    def grads(jj, kk):
        return tuple(g[jj, kk].ravel() for g in G)

    # arcs between rings j and j + 1 (j = 0 .. nr - 2), every sector
    J, K = np.meshgrid(np.arange(nr - 1), np.arange(nt), indexing="ij")
    nA = np.stack([np.cos(thc)[K].ravel(), np.sin(thc)[K].ravel()], axis=1)
    dA = (rc[1:] - rc[:-1])[J].ravel()
    nf = nr - 1
    maskA = ((J >= 1) & (J <= nf - 2)).ravel() if nf >= 3 else np.zeros(J.size, bool)
    dissA = (cells(np.clip(J - 1, 0, nr - 1), K), cells(np.clip(J + 2, 0, nr - 1), K), maskA)
    FA = _face_flux(cells(J, K), cells(J + 1, K), grads(J, K), grads(J + 1, K), H[J, K].reshape(-1, 12),
                    H[J + 1, K].reshape(-1, 12), nA, dA, c, dissA)
    SA = (2.0 * R[1:nr] * s2)[:, None]
    # rays between sectors k and k + 1 (mod nt), every ring
    J, K = np.meshgrid(np.arange(nr), np.arange(nt), indexing="ij")
    phi = dth * (K + 1.0)
    nR = np.stack([-np.sin(phi).ravel(), np.cos(phi).ravel()], axis=1)
    dR = (2.0 * rc * s2)[J].ravel()
    dissR = (cells(J, (K - 1) % nt), cells(J, (K + 2) % nt), np.ones(J.size, bool))
    FR = _face_flux(cells(J, K), cells(J, (K + 1) % nt), grads(J, K), grads(J, (K + 1) % nt),
                    H[J, K].reshape(-1, 12), H[J, (K + 1) % nt].reshape(-1, 12), nR, dR, c, dissR)
    SR = (R[1:] - R[:-1])[:, None]
    V = (0.5 * dth * (R[1:] ** 2 - R[:-1] ** 2))[:, None]
    div = []
    for v in range(NV):
        fa = FA[v].reshape(nr - 1, nt) * SA
        fr = FR[v].reshape(nr, nt) * SR
        dv = np.zeros((nr, nt))
        dv[:-1] += fa
        dv[1:] -= fa
        dv += fr - np.roll(fr, 1, axis=1)
        div.append(dv / V)
    rho, tt, tr = X[0], X[3], X[4]
    T = (3.0 * tt + d_r * tr) / (3.0 + d_r)
    mu = mu_ref * T ** omega
    src = 0.5 * d_r * rho * (rho * T) * (T - tr) / (Z * mu)
    Rm = np.stack([div[0], div[1], div[2], div[3], div[4] - src])
    D = dsmc.reshape(nr, nt, -1)
    cols = (F_RHO, F_U, F_U + 1, F_TT, F_TR)
    for v in range(NV):  # the boundary rings: their whole sampled state
        Rm[v, 0] = X[v, 0] - D[0, :, cols[v]]
        Rm[v, -1] = X[v, -1] - D[-1, :, cols[v]]
    return Rm.reshape(-1)


def initial_state(dsmc: np.ndarray) -> np.ndarray:
    return np.concatenate([dsmc[:, F_RHO], dsmc[:, F_U], dsmc[:, F_U + 1], dsmc[:, F_TT], dsmc[:, F_TR]])


def jacobian(x: np.ndarray, dsmc: np.ndarray, hot: np.ndarray, cfg: dict) -> np.ndarray:
    """Dense Jacobian by central differences, h = 1e-6 max(|x|, 1).  A
    residual depends on the cells within two rings and two sectors of its
    own, so the cells of one colour (ring mod 5, sector mod 5 when nt is a
    multiple of 5, else the sector itself) are perturbed together."""
    nt, nr = int(cfg["nx"]), int(cfg["ny"])
    n = nt * nr
    pk = 5 if nt % 5 == 0 else nt
    jj_all, kk_all = np.divmod(np.arange(n), nt)
    J = np.zeros((NV * n, NV * n))

    def near(a, b, period):
        d = (b - a) % period
        return d - period if d > period // 2 else d

    for v in range(NV):
        for cj in range(5):
            for ck in range(pk):
                sel = np.nonzero((jj_all % 5 == cj) & (kk_all % pk == ck))[0]
                if sel.size == 0:
                    continue
                h = 1e-6 * np.maximum(np.abs(x[v * n + sel]), 1.0)
                xp, xm = x.copy(), x.copy()
                xp[v * n + sel] += h
                xm[v * n + sel] -= h
                dR = (residual(xp, dsmc, hot, cfg) - residual(xm, dsmc, hot, cfg)).reshape(NV, n)
                hc = np.zeros(n)
                hc[sel] = h
                for c in range(n):
                    j, k = jj_all[c], kk_all[c]
                    jp = j + near(j, cj, 5)
                    kp = (k + near(k, ck, 5)) % nt if pk == 5 else ck
                    if not 0 <= jp < nr:
                        continue
                    q = jp * nt + kp
                    if hc[q] == 0.0:
                        continue
                    J[np.arange(NV) * n + c, v * n + q] = dR[:, c] / (2.0 * hc[q])
    return J


def synth_solve_annulus(dsmc: np.ndarray, hot: np.ndarray, cfg: dict, tol: float = 1e-12, max_iter: int = 50):
    """Newton iterations from the sampled fields until the largest relative
    update of a full step is below tol.  Returns (out [ncells x 6] = rho,
    u_x, u_y, u_z (the sampled one), T_t, T_r; iterations; final max
    |residual|); when positivity cuts a step below 1/1024 (a stall: no
    solution near the state) out is the sampled fields."""
    nt, nr = int(cfg["nx"]), int(cfg["ny"])
    if nt < 4 or nr < 3:
        raise ValueError("synth_solve_annulus needs at least 4 sectors and 3 rings")
    n = nt * nr
    x = initial_state(dsmc)
    it = 0
    stalled = False
    for it in range(1, max_iter + 1):
        Rv = residual(x, dsmc, hot, cfg)
        dxv = np.linalg.solve(jacobian(x, dsmc, hot, cfg), -Rv)
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
    Rv = residual(x, dsmc, hot, cfg)
    X = x.reshape(NV, n)
    out = np.stack([X[0], X[1], X[2], dsmc[:, F_U + 2], X[3], X[4]], axis=1)
    if stalled:
        out = np.stack([dsmc[:, F_RHO], dsmc[:, F_U], dsmc[:, F_U + 1], dsmc[:, F_U + 2], dsmc[:, F_TT],
                        dsmc[:, F_TR]], axis=1)
    return out, it, float(np.max(np.abs(Rv)))
