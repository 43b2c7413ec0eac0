// dsmc_synth2d.cuh -- the steady 2D synthetic equations of the DIG method
// (Eq. macroscopic_equation with the constitutive relations of
// Eq. full_constitutive, Sec. 3 step 3) on a rectangle of nx x ny uniform
// cells closed by walls: per-cell residual, finite-difference Jacobian
// entries and the steps of a banded LU factorisation with partial pivoting.
//
// Everything here is __host__ __device__ and works on plain arrays, so the
// kernels of dsmc_synth2d.cu are thin loops over these functions.
//
// Discrete equations (unknowns per cell: rho, u_x, u_y, T_t, T_r; the flow is
// planar and u_z takes no part):
//   div(rho u) = 0,  div(rho u u + rho T_t I + sigma) = 0,
//   div(rho e u + rho T_t u + sigma.u + q_t + q_r) = 0,
//   div(rho e_r u + q_r) = (d_r rho / 2) (T - T_r) / (Z tau),
//   e = (3 T_t + d_r T_r) / 2 + |u|^2 / 2,  e_r = d_r T_r / 2,  tau = mu / p,
// with sigma = sigma_NSF + HoT and q = q_NSF + HoT (Eq. ns_constitutive,
// kappa from Eq. kappa_A).  Finite volumes: a face flux is the mean of the
// two cells' convective fluxes plus viscous and heat fluxes from compact
// normal differences and tangential differences averaged from the two cells
// (central inside, one-sided in the first and last row or column), face
// viscosity mu(T_f) with T_f from the face means of T_t and T_r, face HoT the
// mean of the two cells' HoT, and a fourth-difference dissipation
// (1/32) (|u_n| + sqrt(gamma T_f)) (W[i+2] - 3 W[i+1] + 3 W[i] - W[i-1]) on
// the conserved variables W wherever that stencil lies in the domain.
// Cells next to a wall keep the sampled u_x, u_y, T_t, T_r and balance only
// their mass; the four corner cells keep their whole sampled state and
// exchange no flux; cell (1, 0)'s mass balance is replaced by the total mass.
//
// Unknown ordering: cells are numbered along the shorter side first (band
// cell b = j nx + i when nx <= ny, else i ny + j) and the five unknowns of a
// cell are consecutive (u = 5 b + v), so that the Jacobian without the
// total-mass row is banded with kl = ku = 10 min(nx, ny) + 4.
#pragma once

#include <cmath>
#include <cstdint>

namespace dsmc {
namespace s2 {

constexpr int NV = 5;          // rho, u_x, u_y, T_t, T_r
constexpr double EPS4 = 1.0 / 32.0;
constexpr int NSTENCIL = 13;   // cells a residual depends on (the total-mass row aside)

// stencil offsets (di, dj): the cell, +-1 and +-2 along each axis, and the
// four diagonal neighbours
__host__ __device__ inline void stencil_offset(int s, int& di, int& dj) {
  const int8_t tab[NSTENCIL][2] = {{0, 0},  {-1, 0}, {1, 0},  {-2, 0}, {2, 0},   {0, -1}, {0, 1},
                                   {0, -2}, {0, 2},  {-1, -1}, {1, -1}, {-1, 1}, {1, 1}};
  di = tab[s][0];
  dj = tab[s][1];
}

// Geometry, constants and the inputs of one solve.
struct Grid {
  int nx, ny, n;           // cells
  int N, kl, ku, ld;       // unknowns, band widths, leading dimension of the band storage
  int xfast;               // 1: band cell b = j nx + i; 0: b = i ny + j
  double dx, dy;
  double d_r, omega, mu_ref, z_rot, kappa_t, kappa_r, gamma;
  const double* F;         // sampled fields, natural order (cell j nx + i) x 18
  const double* hot;       // HoT, natural order x 12
};

__host__ __device__ inline Grid make_grid(int nx, int ny, double dx, double dy, double d_r, double omega,
                                          double mu_ref, double z_rot, double kappa_t, double kappa_r,
                                          const double* F, const double* hot) {
  Grid g;
  g.nx = nx;
  g.ny = ny;
  g.n = nx * ny;
  g.N = NV * g.n;
  g.xfast = nx <= ny ? 1 : 0;
  const int nf = g.xfast ? nx : ny;
  g.kl = 10 * nf + 4;
  g.ku = g.kl;
  g.ld = 2 * g.kl + g.ku + 1;
  g.dx = dx;
  g.dy = dy;
  g.d_r = d_r;
  g.omega = omega;
  g.mu_ref = mu_ref;
  g.z_rot = z_rot;
  g.kappa_t = kappa_t;
  g.kappa_r = kappa_r;
  g.gamma = (5.0 + d_r) / (3.0 + d_r);
  g.F = F;
  g.hot = hot;
  return g;
}

__host__ __device__ inline int band_cell(const Grid& g, int i, int j) { return g.xfast ? j * g.nx + i : i * g.ny + j; }
__host__ __device__ inline void cell_of_band(const Grid& g, int b, int& i, int& j) {
  if (g.xfast) {
    j = b / g.nx;
    i = b - j * g.nx;
  } else {
    i = b / g.ny;
    j = b - i * g.ny;
  }
}
__host__ __device__ inline bool is_corner(const Grid& g, int i, int j) {
  return (i == 0 || i == g.nx - 1) && (j == 0 || j == g.ny - 1);
}

// The state x (band order) with one unknown (band cell pb, variable pv)
// shifted by delta, as the finite-difference Jacobian needs it.
struct View {
  const double* x;
  int pb, pv;
  double delta;
  __host__ __device__ double at(const Grid& g, int i, int j, int v) const {
    const int b = band_cell(g, i, j);
    const double val = x[NV * b + v];
    return (b == pb && v == pv) ? val + delta : val;
  }
};

// Face-frame state of cell (i, j) for faces normal to axis dir (0: x, 1: y):
// (rho, u_n, u_t, T_t, T_r).
__host__ __device__ inline void frame_state(const Grid& g, const View& X, int dir, int i, int j, double* q) {
  q[0] = X.at(g, i, j, 0);
  q[1] = X.at(g, i, j, dir == 0 ? 1 : 2);
  q[2] = X.at(g, i, j, dir == 0 ? 2 : 1);
  q[3] = X.at(g, i, j, 3);
  q[4] = X.at(g, i, j, 4);
}

// Tangential derivatives (d u_n / dt, d u_t / dt) at cell (i, j) in the frame
// of faces normal to dir: central inside, one-sided in the first and last
// row (dir 0) or column (dir 1).
__host__ __device__ inline void tangential(const Grid& g, const View& X, int dir, int i, int j, double& gn,
                                           double& gt) {
  const int vn = dir == 0 ? 1 : 2, vt = dir == 0 ? 2 : 1;
  const int t = dir == 0 ? j : i, nt = dir == 0 ? g.ny : g.nx;
  const double h = dir == 0 ? g.dy : g.dx;
  int lo = t - 1, hi = t + 1;
  double den = 2.0 * h;
  if (t == 0) {
    lo = 0;
    hi = 1;
    den = h;
  } else if (t == nt - 1) {
    lo = nt - 2;
    hi = nt - 1;
    den = h;
  }
  const int il = dir == 0 ? i : lo, jl = dir == 0 ? lo : j;
  const int ih = dir == 0 ? i : hi, jh = dir == 0 ? hi : j;
  gn = (X.at(g, ih, jh, vn) - X.at(g, il, jl, vn)) / den;
  gt = (X.at(g, ih, jh, vt) - X.at(g, il, jl, vt)) / den;
}

// conserved variables in the face frame: rho, rho u_n, rho u_t, rho e, rho e_r
__host__ __device__ inline void conserved(const Grid& g, const double* q, double* w) {
  const double e = 0.5 * (3.0 * q[3] + g.d_r * q[4]) + 0.5 * (q[1] * q[1] + q[2] * q[2]);
  w[0] = q[0];
  w[1] = q[0] * q[1];
  w[2] = q[0] * q[2];
  w[3] = q[0] * e;
  w[4] = q[0] * (0.5 * g.d_r * q[4]);
}

// Flux through the face between cell (i, j) and its neighbour along dir
// ((i+1, j) for dir 0, (i, j+1) for dir 1), in the face frame:
// (mass, normal momentum, tangential momentum, energy, rotational energy).
// A face of a corner cell carries nothing.
__host__ __device__ inline void face_flux(const Grid& g, const View& X, int dir, int i, int j, double* F) {
  const int i2 = dir == 0 ? i + 1 : i, j2 = dir == 0 ? j : j + 1;
  if (is_corner(g, i, j) || is_corner(g, i2, j2)) {
    for (int k = 0; k < NV; ++k) F[k] = 0.0;
    return;
  }
  const double d = dir == 0 ? g.dx : g.dy;
  const double d_r = g.d_r;
  double ql[NV], qr[NV];
  frame_state(g, X, dir, i, j, ql);
  frame_state(g, X, dir, i2, j2, qr);
  const double unf = 0.5 * (ql[1] + qr[1]);
  const double utf = 0.5 * (ql[2] + qr[2]);
  const double ttf = 0.5 * (ql[3] + qr[3]);
  const double trf = 0.5 * (ql[4] + qr[4]);
  const double Tf = (3.0 * ttf + d_r * trf) / (3.0 + d_r);
  const double muf = g.mu_ref * pow(Tf, g.omega);
  const double dun_n = (qr[1] - ql[1]) / d;
  const double dut_n = (qr[2] - ql[2]) / d;
  const double dtt_n = (qr[3] - ql[3]) / d;
  const double dtr_n = (qr[4] - ql[4]) / d;
  double gnl, gtl, gnr, gtr;
  tangential(g, X, dir, i, j, gnl, gtl);
  tangential(g, X, dir, i2, j2, gnr, gtr);
  const double dun_t = 0.5 * (gnl + gnr);
  const double dut_t = 0.5 * (gtl + gtr);
  // face HoT: (sigma_nn, sigma_nt, q_t,n, q_r,n)
  const double* hl = g.hot + (size_t)(j * g.nx + i) * 12;
  const double* hr = g.hot + (size_t)(j2 * g.nx + i2) * 12;
  const int hnn = dir == 0 ? 0 : 1, hqt = dir == 0 ? 6 : 7, hqr = dir == 0 ? 9 : 10;
  const double h_nn = 0.5 * (hl[hnn] + hr[hnn]);
  const double h_nt = 0.5 * (hl[3] + hr[3]);
  const double h_qt = 0.5 * (hl[hqt] + hr[hqt]);
  const double h_qr = 0.5 * (hl[hqr] + hr[hqr]);
  const double s_nn = -muf * ((4.0 / 3.0) * dun_n - (2.0 / 3.0) * dut_t) + h_nn;
  const double s_nt = -muf * (dut_n + dun_t) + h_nt;
  const double qt = -g.kappa_t * muf * dtt_n + h_qt;
  const double qrr = -g.kappa_r * muf * dtr_n + h_qr;
  // convective fluxes: mean of the two cells' values
  double cl[NV], cr[NV];
  {
    const double* q = ql;
    const double e = 0.5 * (3.0 * q[3] + d_r * q[4]) + 0.5 * (q[1] * q[1] + q[2] * q[2]);
    cl[0] = q[0] * q[1];
    cl[1] = q[0] * q[1] * q[1] + q[0] * q[3];
    cl[2] = q[0] * q[1] * q[2];
    cl[3] = q[0] * q[1] * (e + q[3]);
    cl[4] = q[0] * q[1] * (0.5 * d_r * q[4]);
  }
  {
    const double* q = qr;
    const double e = 0.5 * (3.0 * q[3] + d_r * q[4]) + 0.5 * (q[1] * q[1] + q[2] * q[2]);
    cr[0] = q[0] * q[1];
    cr[1] = q[0] * q[1] * q[1] + q[0] * q[3];
    cr[2] = q[0] * q[1] * q[2];
    cr[3] = q[0] * q[1] * (e + q[3]);
    cr[4] = q[0] * q[1] * (0.5 * d_r * q[4]);
  }
  for (int k = 0; k < NV; ++k) F[k] = 0.5 * (cl[k] + cr[k]);
  F[1] += s_nn;
  F[2] += s_nt;
  F[3] += s_nn * unf + s_nt * utf + qt + qrr;
  F[4] += qrr;
  // fourth-difference dissipation where cells f-1 .. f+2 along the normal exist
  const int f = dir == 0 ? i : j;
  const int nfaces = (dir == 0 ? g.nx : g.ny) - 1;
  if (nfaces >= 3 && f >= 1 && f <= nfaces - 2) {
    double qm[NV], qp[NV], wm[NV], w0[NV], w1[NV], wp[NV];
    frame_state(g, X, dir, dir == 0 ? i - 1 : i, dir == 0 ? j : j - 1, qm);
    frame_state(g, X, dir, dir == 0 ? i + 2 : i, dir == 0 ? j : j + 2, qp);
    conserved(g, qm, wm);
    conserved(g, ql, w0);
    conserved(g, qr, w1);
    conserved(g, qp, wp);
    const double lam = fabs(unf) + sqrt(g.gamma * Tf);
    for (int k = 0; k < NV; ++k) F[k] += EPS4 * lam * (wp[k] - 3.0 * w1[k] + 3.0 * w0[k] - wm[k]);
  }
}

// Residual rows (5) of cell (i, j).  mass_row is the total-mass residual
// (sum rho - sampled sum) / n, used by cell (1, 0).
__host__ __device__ inline void cell_residual(const Grid& g, const View& X, int i, int j, double mass_row, double* R) {
  const double* D = g.F + (size_t)(j * g.nx + i) * 18;
  if (is_corner(g, i, j)) {
    R[0] = X.at(g, i, j, 0) - D[0];
    R[1] = X.at(g, i, j, 1) - D[1];
    R[2] = X.at(g, i, j, 2) - D[2];
    R[3] = X.at(g, i, j, 3) - D[4];
    R[4] = X.at(g, i, j, 4) - D[5];
    return;
  }
  const bool ring = i == 0 || i == g.nx - 1 || j == 0 || j == g.ny - 1;
  double div[NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double Fa[NV];
  if (i < g.nx - 1) {
    face_flux(g, X, 0, i, j, Fa);
    for (int k = 0; k < NV; ++k) div[k] += Fa[k] / g.dx;
  }
  if (i > 0) {
    face_flux(g, X, 0, i - 1, j, Fa);
    for (int k = 0; k < NV; ++k) div[k] -= Fa[k] / g.dx;
  }
  // y faces: frame (normal y, tangential x) -> components 1 and 2 swap
  if (j < g.ny - 1) {
    face_flux(g, X, 1, i, j, Fa);
    div[0] += Fa[0] / g.dy;
    div[1] += Fa[2] / g.dy;
    div[2] += Fa[1] / g.dy;
    div[3] += Fa[3] / g.dy;
    div[4] += Fa[4] / g.dy;
  }
  if (j > 0) {
    face_flux(g, X, 1, i, j - 1, Fa);
    div[0] -= Fa[0] / g.dy;
    div[1] -= Fa[2] / g.dy;
    div[2] -= Fa[1] / g.dy;
    div[3] -= Fa[3] / g.dy;
    div[4] -= Fa[4] / g.dy;
  }
  R[0] = (i == 1 && j == 0) ? mass_row : div[0];
  if (ring) {
    R[1] = X.at(g, i, j, 1) - D[1];
    R[2] = X.at(g, i, j, 2) - D[2];
    R[3] = X.at(g, i, j, 3) - D[4];
    R[4] = X.at(g, i, j, 4) - D[5];
    return;
  }
  const double rho = X.at(g, i, j, 0), tt = X.at(g, i, j, 3), tr = X.at(g, i, j, 4);
  const double T = (3.0 * tt + g.d_r * tr) / (3.0 + g.d_r);
  const double mu = g.mu_ref * pow(T, g.omega);
  const double src = 0.5 * g.d_r * rho * (rho * T) * (T - tr) / (g.z_rot * mu);
  R[1] = div[1];
  R[2] = div[2];
  R[3] = div[3];
  R[4] = div[4] - src;
}

// row of the total-mass equation: unknown rho of cell (1, 0)
__host__ __device__ inline int mass_row(const Grid& g) { return NV * band_cell(g, 1, 0); }

// Band storage (column-major, leading dimension ld): entry (r, c) of the
// matrix at AB[c * ld + r - c + kl + ku], rows c - kl - ku .. c + kl of column
// c (the upper part grows to kl + ku under row interchanges).
__host__ __device__ inline size_t band_at(const Grid& g, int r, int c) {
  return (size_t)c * g.ld + (size_t)(r - c + g.kl + g.ku);
}

// Jacobian entries of one (cell, stencil neighbour, variable): column
// 5 k + v, rows 5 b .. 5 b + 4, by central differences with
// h = 1e-6 max(|x|, 1).  The total-mass row is left out (written by the
// caller as e_r / n; the rest of it is carried by a rank-one correction).
__host__ __device__ inline void jacobian_entries(const Grid& g, const double* x, int b, int s, int v, double* AB) {
  int i, j, di, dj;
  cell_of_band(g, b, i, j);
  stencil_offset(s, di, dj);
  const int ik = i + di, jk = j + dj;
  if (ik < 0 || ik >= g.nx || jk < 0 || jk >= g.ny) return;
  const int kb = band_cell(g, ik, jk);
  const double xv = x[NV * kb + v];
  const double h = 1e-6 * fmax(fabs(xv), 1.0);
  View Xp{x, kb, v, h}, Xm{x, kb, v, -h};
  double Rp[NV], Rm[NV];
  cell_residual(g, Xp, i, j, 0.0, Rp);
  cell_residual(g, Xm, i, j, 0.0, Rm);
  const int col = NV * kb + v;
  const int mr = mass_row(g);
  for (int r = 0; r < NV; ++r) {
    const int row = NV * b + r;
    if (row == mr) continue;
    AB[band_at(g, row, col)] = (Rp[r] - Rm[r]) / (2.0 * h);
  }
}

// Elimination step k (k = 0 .. N-2) on one column c in k+1 .. k+kl+ku:
// interchange rows k and p = piv[k], then subtract l_r times row k from rows
// r = k+1 .. min(k+kl, N-1), multipliers l_r in Lm[k kl + r - k - 1].  The
// two head entries (rows k and p) are read by every thread before any thread
// writes (col_head, then a barrier, then lu_column); thread 0 writes row k,
// the owner of row p writes row p from row k's old value, so no two threads
// touch one entry.
struct ColHead {
  double akc_old;  // A(k, c) before the interchange
  double ukc;      // U(k, c): A(p, c) before the interchange
};

__host__ __device__ inline ColHead col_head(const Grid& g, const double* AB, const int32_t* piv, int k, int c) {
  ColHead h;
  h.akc_old = AB[band_at(g, k, c)];
  h.ukc = AB[band_at(g, piv[k], c)];
  return h;
}

__host__ __device__ inline int last_row(const Grid& g, int k) { return k + g.kl < g.N - 1 ? k + g.kl : g.N - 1; }
__host__ __device__ inline int last_col(const Grid& g, int k) {
  return k + g.kl + g.ku < g.N - 1 ? k + g.kl + g.ku : g.N - 1;
}

__host__ __device__ inline void lu_column(const Grid& g, double* AB, const double* Lm, const int32_t* piv, int k,
                                          int c, const ColHead& h, int tid, int nthr) {
  const int p = piv[k];
  if (tid == 0 && p != k) AB[band_at(g, k, c)] = h.ukc;
  const double* l = Lm + (size_t)k * g.kl;
  const int rmax = last_row(g, k);
  for (int r = k + 1 + tid; r <= rmax; r += nthr) {
    const double a = (r == p) ? h.akc_old : AB[band_at(g, r, c)];
    AB[band_at(g, r, c)] = a - l[r - k - 1] * h.ukc;
  }
}

// Pivot of column k once steps 0 .. k-1 have updated it: the first row of
// largest |A(r, k)|, r = k .. min(k+kl, N-1) (sequential form; the kernel
// reduces the same order).
__host__ __device__ inline int pivot_seq(const Grid& g, const double* AB, int k) {
  int p = k;
  double best = fabs(AB[band_at(g, k, k)]);
  for (int r = k + 1; r <= last_row(g, k); ++r) {
    const double a = fabs(AB[band_at(g, r, k)]);
    if (a > best) {
      best = a;
      p = r;
    }
  }
  return p;
}

// With the pivot p of column k: U(k, k) into ud[k], p into piv[k] and the
// multipliers of rows k+1 .. into Lm (column k of the band is not written).
// Returns 1 when the pivot is zero (the matrix is singular; multipliers 0).
__host__ __device__ inline int pivot_write(const Grid& g, const double* AB, double* Lm, int32_t* piv, double* ud,
                                           int k, int p, int tid, int nthr) {
  const double up = AB[band_at(g, p, k)];
  const double akk = AB[band_at(g, k, k)];
  if (tid == 0) {
    ud[k] = up;
    piv[k] = p;
  }
  double* l = Lm + (size_t)k * g.kl;
  const int rmax = last_row(g, k);
  for (int r = k + 1 + tid; r <= rmax; r += nthr) {
    const double a = (r == p) ? akk : AB[band_at(g, r, k)];
    l[r - k - 1] = up != 0.0 ? a / up : 0.0;
  }
  return up == 0.0 ? 1 : 0;
}

// Forward substitution step k with P and L (two right-hand sides b0, b1;
// results y0[k], y1[k]).  Heads read first (fwd_head), barrier, then
// fwd_step, barrier.
struct FwdHead {
  double bk0, bk1;      // b(p) before the interchange: y(k)
  double old0, old1;    // b(k) before the interchange
};

__host__ __device__ inline FwdHead fwd_head(const int32_t* piv, int k, const double* b0, const double* b1) {
  const int p = piv[k];
  FwdHead h;
  h.bk0 = b0[p];
  h.bk1 = b1[p];
  h.old0 = b0[k];
  h.old1 = b1[k];
  return h;
}

__host__ __device__ inline void fwd_step(const Grid& g, const double* Lm, const int32_t* piv, int k, const FwdHead& h,
                                         double* b0, double* b1, double* y0, double* y1, int tid, int nthr) {
  const int p = piv[k];
  if (tid == 0) {
    y0[k] = h.bk0;
    y1[k] = h.bk1;
  }
  const double* l = Lm + (size_t)k * g.kl;
  const int rmax = last_row(g, k);
  for (int r = k + 1 + tid; r <= rmax; r += nthr) {
    const double a0 = (r == p) ? h.old0 : b0[r];
    const double a1 = (r == p) ? h.old1 : b1[r];
    b0[r] = a0 - l[r - k - 1] * h.bk0;
    b1[r] = a1 - l[r - k - 1] * h.bk1;
  }
}

// Back substitution step k (k = N-1 .. 0) with U: x(k) = y(k) / U(k, k), then
// y(r) -= U(r, k) x(k) for r = k-kl-ku .. k-1 (y overwritten; barrier after).
__host__ __device__ inline void back_step(const Grid& g, const double* AB, const double* ud, int k, double* y0,
                                          double* y1, double* x0, double* x1, int tid, int nthr) {
  const double xk0 = y0[k] / ud[k];
  const double xk1 = y1[k] / ud[k];
  if (tid == 0) {
    x0[k] = xk0;
    x1[k] = xk1;
  }
  const int rmin = k - g.kl - g.ku > 0 ? k - g.kl - g.ku : 0;
  for (int r = rmin + tid; r < k; r += nthr) {
    const double u = AB[band_at(g, r, k)];
    y0[r] -= u * xk0;
    y1[r] -= u * xk1;
  }
}

}  // namespace s2
}  // namespace dsmc
