// dsmc_synth2d.cuh -- the steady 2D synthetic equations of the DIG method
// (Eq. macroscopic_equation with the constitutive relations of
// Eq. full_constitutive, Sec. 3 step 3) on a rectangle of nx x ny cells
// closed by walls (uniform, or the wall-refined grid of the cavity case of
// Sec. 4.1: widths growing geometrically from each wall, see set_edges):
// per-cell residual, finite-difference Jacobian
// entries, and the steps of a blocked banded LU factorisation with partial
// pivoting in FP32 and of its substitutions.
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
// exchange no flux; cell (1, 0)'s mass balance is replaced by the total mass
// (sum rho V against the sampled one).
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
  double dx, dy;           // uniform grid: the cell size
  const double* xe;        // wall-refined grid: cell edges along x (nx + 1) and y (ny + 1); null: uniform
  const double* ye;
  double area;             // L_x L_y (wall-refined grid)
  int ann;                 // 1: the annulus around a cylinder (nx sectors, periodic; ny rings)
  const double* R;         // annulus: ring edges R_0 .. R_ny
  double dth, s2, sdth;    // annulus: sector angle, sin(dth / 2), sin(dth)
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
  g.xe = nullptr;
  g.ye = nullptr;
  g.area = 0.0;
  g.ann = 0;
  g.R = nullptr;
  g.dth = g.s2 = g.sdth = 0.0;
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

// The wall-refined grid of the cavity case (Sec. 4.1): cells between the
// given edges; differences are taken over the distances between cell centres
// (the middle of each cell's edges) and a balance divides by its cell's width.
__host__ __device__ inline void set_edges(Grid& g, const double* xe, const double* ye, double area) {
  g.xe = xe;
  g.ye = ye;
  g.area = area;
}

// width of cell k along axis dir (0: x, 1: y)
__host__ __device__ inline double width(const Grid& g, int dir, int k) {
  const double* e = dir == 0 ? g.xe : g.ye;
  return e ? e[k + 1] - e[k] : (dir == 0 ? g.dx : g.dy);
}

__host__ __device__ inline double centre(const double* e, int k) { return 0.5 * (e[k] + e[k + 1]); }

// The annulus around a cylinder (Sec. 4.2): cell (i, j) in sector i (angles
// dth i .. dth (i + 1)) and ring j (radii R_j .. R_{j+1}), cells numbered
// ring by ring (band cell j nx + i, periodic in i), so the band holds the
// wrap-around neighbours too: kl = ku = 10 nx + 4.  Needs nx >= 5 (the
// stencil's five sectors distinct) and ny >= 3.
__host__ __device__ inline void set_annulus(Grid& g, const double* R) {
  g.ann = 1;
  g.R = R;
  g.dth = 2.0 * 3.14159265358979323846 / g.nx;
  g.s2 = sin(0.5 * g.dth);
  g.sdth = sin(g.dth);
  g.xfast = 1;
  g.kl = 10 * g.nx + 4;
  g.ku = g.kl;
  g.ld = 2 * g.kl + g.ku + 1;
}

// Weight of cell (i, j)'s density in the total-mass row, times n: 1 on the
// uniform grid, n V_c / (L_x L_y) on the wall-refined one, so that the row
// holds the mass sum_c rho_c V_c against its sample; the annulus has no
// total-mass row (its outer ring keeps its sampled density).
__host__ __device__ inline double mass_scale(const Grid& g, int i, int j) {
  if (g.ann) return 0.0;
  if (!g.xe) return 1.0;
  return (double)g.n * (width(g, 0, i) * width(g, 1, j)) / g.area;
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
  return !g.ann && (i == 0 || i == g.nx - 1) && (j == 0 || j == g.ny - 1);
}

// the cell at stencil offset (di, dj) of cell (i, j); false outside the grid
// (the annulus wraps around in i)
__host__ __device__ inline bool stencil_cell(const Grid& g, int i, int j, int di, int dj, int& ik, int& jk) {
  ik = i + di;
  jk = j + dj;
  if (jk < 0 || jk >= g.ny) return false;
  if (g.ann) {
    ik = ik < 0 ? ik + g.nx : (ik >= g.nx ? ik - g.nx : ik);
    return true;
  }
  return ik >= 0 && ik < g.nx;
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
  const double* e = dir == 0 ? g.ye : g.xe;  // edges along the tangential axis
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
  if (e) den = centre(e, hi) - centre(e, lo);
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
  const double* en = dir == 0 ? g.xe : g.ye;  // edges along the normal
  const int fn = dir == 0 ? i : j;
  const double d = en ? centre(en, fn + 1) - centre(en, fn) : (dir == 0 ? g.dx : g.dy);
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

// ---------------------------------------------------------------------------
// The annulus (set_annulus): finite volumes with the exact face vectors (an
// arc at radius R in sector i: 2 R sin(dth / 2) e_r(theta_i), theta_i =
// dth (i + 1/2); a ray at angle phi in ring j: (R_{j+1} - R_j) e_theta(phi)),
// sector areas as volumes, the box's face flux in each face's frame (n, t =
// n turned by +90 degrees) with the tangential derivatives averaged from the
// two cells' Cartesian gradients; the ring next to the cylinder and the outer
// ring keep their whole sampled state.
// ---------------------------------------------------------------------------
__host__ __device__ inline double ann_rc(const Grid& g, int j) { return 0.5 * (g.R[j] + g.R[j + 1]); }

// Cartesian gradient (du_x/dx, du_x/dy, du_y/dx, du_y/dy) of cell (i, j):
// d/dr by the three-point formula on the ring centres (one-sided in the
// first and last ring), (1/r) d/dtheta = (f_{i+1} - f_{i-1}) / (2 r_c
// sin(dth)), turned to Cartesian at theta_i.
__host__ __device__ inline void ann_grad(const Grid& g, const View& X, int i, int j, double* gr) {
  const int nt = g.nx, nr = g.ny;
  const int ip = i + 1 < nt ? i + 1 : 0, im = i > 0 ? i - 1 : nt - 1;
  const double rc = ann_rc(g, j);
  const double th = g.dth * (i + 0.5);
  const double c = cos(th), s = sin(th);
  for (int q = 0; q < 2; ++q) {
    const int v = 1 + q;
    double dr;
    if (j == 0) {
      dr = (X.at(g, i, 1, v) - X.at(g, i, 0, v)) / (ann_rc(g, 1) - ann_rc(g, 0));
    } else if (j == nr - 1) {
      dr = (X.at(g, i, nr - 1, v) - X.at(g, i, nr - 2, v)) / (ann_rc(g, nr - 1) - ann_rc(g, nr - 2));
    } else {
      const double hm = rc - ann_rc(g, j - 1), hp = ann_rc(g, j + 1) - rc;
      dr = (hm * hm * X.at(g, i, j + 1, v) - hp * hp * X.at(g, i, j - 1, v) + (hp * hp - hm * hm) * X.at(g, i, j, v)) /
           (hp * hm * (hp + hm));
    }
    const double dt = (X.at(g, ip, j, v) - X.at(g, im, j, v)) / (2.0 * rc * g.sdth);
    gr[2 * q] = c * dr - s * dt;
    gr[2 * q + 1] = s * dr + c * dt;
  }
}

// Flux per unit area (mass, x-momentum, y-momentum, energy, rotational
// energy) through the ray between sectors i and i + 1 of ring j (dir 0) or
// the arc between rings j and j + 1 of sector i (dir 1).
__host__ __device__ inline void ann_face_flux(const Grid& g, const View& X, int dir, int i, int j, double* F) {
  const int nt = g.nx;
  const int i2 = dir == 0 ? (i + 1 < nt ? i + 1 : 0) : i, j2 = dir == 0 ? j : j + 1;
  const double ang = dir == 0 ? g.dth * (i + 1.0) : g.dth * (i + 0.5);
  const double nx = dir == 0 ? -sin(ang) : cos(ang), ny = dir == 0 ? cos(ang) : sin(ang);
  const double tx = -ny, ty = nx;
  const double d = dir == 0 ? 2.0 * ann_rc(g, j) * g.s2 : ann_rc(g, j + 1) - ann_rc(g, j);
  const double d_r = g.d_r;
  double q[2][NV];
  for (int side = 0; side < 2; ++side) {
    const int ci = side ? i2 : i, cj = side ? j2 : j;
    const double ux = X.at(g, ci, cj, 1), uy = X.at(g, ci, cj, 2);
    q[side][0] = X.at(g, ci, cj, 0);
    q[side][1] = ux * nx + uy * ny;
    q[side][2] = -ux * ny + uy * nx;
    q[side][3] = X.at(g, ci, cj, 3);
    q[side][4] = X.at(g, ci, cj, 4);
  }
  const double* ql = q[0];
  const double* qr = q[1];
  const double unf = 0.5 * (ql[1] + qr[1]), utf = 0.5 * (ql[2] + qr[2]);
  const double ttf = 0.5 * (ql[3] + qr[3]), trf = 0.5 * (ql[4] + qr[4]);
  const double Tf = (3.0 * ttf + d_r * trf) / (3.0 + d_r);
  const double muf = g.mu_ref * pow(Tf, g.omega);
  const double dun_n = (qr[1] - ql[1]) / d, dut_n = (qr[2] - ql[2]) / d;
  const double dtt_n = (qr[3] - ql[3]) / d, dtr_n = (qr[4] - ql[4]) / d;
  double gl[4], grr[4];
  ann_grad(g, X, i, j, gl);
  ann_grad(g, X, i2, j2, grr);
  double gn[2], gt[2];
  for (int side = 0; side < 2; ++side) {
    const double* gg = side ? grr : gl;
    const double tgx = tx * gg[0] + ty * gg[1], tgy = tx * gg[2] + ty * gg[3];
    gn[side] = nx * tgx + ny * tgy;
    gt[side] = tx * tgx + ty * tgy;
  }
  const double dun_t = 0.5 * (gn[0] + gn[1]), dut_t = 0.5 * (gt[0] + gt[1]);
  double hs[2][4];
  for (int side = 0; side < 2; ++side) {
    const double* h = g.hot + (size_t)((side ? j2 : j) * g.nx + (side ? i2 : i)) * 12;
    hs[side][0] = h[0] * nx * nx + 2.0 * h[3] * nx * ny + h[1] * ny * ny;
    hs[side][1] = h[0] * nx * tx + h[3] * (nx * ty + ny * tx) + h[1] * ny * ty;
    hs[side][2] = h[6] * nx + h[7] * ny;
    hs[side][3] = h[9] * nx + h[10] * ny;
  }
  const double s_nn = -muf * ((4.0 / 3.0) * dun_n - (2.0 / 3.0) * dut_t) + 0.5 * (hs[0][0] + hs[1][0]);
  const double s_nt = -muf * (dut_n + dun_t) + 0.5 * (hs[0][1] + hs[1][1]);
  const double qt = -g.kappa_t * muf * dtt_n + 0.5 * (hs[0][2] + hs[1][2]);
  const double qrr = -g.kappa_r * muf * dtr_n + 0.5 * (hs[0][3] + hs[1][3]);
  double Fn[NV];
  {
    double cl[NV], cr[NV];
    for (int side = 0; side < 2; ++side) {
      const double* qq = q[side];
      double* cc = side ? cr : cl;
      const double e = 0.5 * (3.0 * qq[3] + d_r * qq[4]) + 0.5 * (qq[1] * qq[1] + qq[2] * qq[2]);
      cc[0] = qq[0] * qq[1];
      cc[1] = qq[0] * qq[1] * qq[1] + qq[0] * qq[3];
      cc[2] = qq[0] * qq[1] * qq[2];
      cc[3] = qq[0] * qq[1] * (e + qq[3]);
      cc[4] = qq[0] * qq[1] * (0.5 * d_r * qq[4]);
    }
    for (int k = 0; k < NV; ++k) Fn[k] = 0.5 * (cl[k] + cr[k]);
  }
  Fn[1] += s_nn;
  Fn[2] += s_nt;
  Fn[3] += s_nn * unf + s_nt * utf + qt + qrr;
  Fn[4] += qrr;
  // fourth-difference dissipation: along the sectors (rays, periodic) or the
  // rings (arcs, where rings j-1 .. j+2 exist)
  const bool diss = dir == 0 || (g.ny - 1 >= 3 && j >= 1 && j <= g.ny - 3);
  if (diss) {
    const int im = dir == 0 ? (i > 0 ? i - 1 : nt - 1) : i, jm = dir == 0 ? j : j - 1;
    const int ip = dir == 0 ? (i + 2 < nt ? i + 2 : i + 2 - nt) : i, jp = dir == 0 ? j : j + 2;
    double qm[NV], qp[NV], wm[NV], w0[NV], w1[NV], wp[NV];
    const int cis[2] = {im, ip}, cjs[2] = {jm, jp};
    for (int side = 0; side < 2; ++side) {
      double* qq = side ? qp : qm;
      const double ux = X.at(g, cis[side], cjs[side], 1), uy = X.at(g, cis[side], cjs[side], 2);
      qq[0] = X.at(g, cis[side], cjs[side], 0);
      qq[1] = ux * nx + uy * ny;
      qq[2] = -ux * ny + uy * nx;
      qq[3] = X.at(g, cis[side], cjs[side], 3);
      qq[4] = X.at(g, cis[side], cjs[side], 4);
    }
    conserved(g, qm, wm);
    conserved(g, ql, w0);
    conserved(g, qr, w1);
    conserved(g, qp, wp);
    const double lam = fabs(unf) + sqrt(g.gamma * Tf);
    for (int k = 0; k < NV; ++k) Fn[k] += EPS4 * lam * (wp[k] - 3.0 * w1[k] + 3.0 * w0[k] - wm[k]);
  }
  F[0] = Fn[0];
  F[1] = Fn[1] * nx + Fn[2] * tx;
  F[2] = Fn[1] * ny + Fn[2] * ty;
  F[3] = Fn[3];
  F[4] = Fn[4];
}

__host__ __device__ inline void ann_cell_residual(const Grid& g, const View& X, int i, int j, double* R) {
  const double* D = g.F + (size_t)(j * g.nx + i) * 18;
  if (j == 0 || j == g.ny - 1) {  // the boundary rings: their sampled state
    R[0] = X.at(g, i, j, 0) - D[0];
    R[1] = X.at(g, i, j, 1) - D[1];
    R[2] = X.at(g, i, j, 2) - D[2];
    R[3] = X.at(g, i, j, 3) - D[4];
    R[4] = X.at(g, i, j, 4) - D[5];
    return;
  }
  double div[NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double Fa[NV];
  const double sa = 2.0 * g.R[j + 1] * g.s2, sr = g.R[j + 1] - g.R[j];
  ann_face_flux(g, X, 1, i, j, Fa);  // the outer arc
  for (int k = 0; k < NV; ++k) div[k] += Fa[k] * sa;
  ann_face_flux(g, X, 1, i, j - 1, Fa);  // the inner arc
  const double sb = 2.0 * g.R[j] * g.s2;
  for (int k = 0; k < NV; ++k) div[k] -= Fa[k] * sb;
  ann_face_flux(g, X, 0, i, j, Fa);  // the ray at the sector's upper angle
  for (int k = 0; k < NV; ++k) div[k] += Fa[k] * sr;
  ann_face_flux(g, X, 0, i > 0 ? i - 1 : g.nx - 1, j, Fa);  // and at its lower angle
  for (int k = 0; k < NV; ++k) div[k] -= Fa[k] * sr;
  const double V = 0.5 * g.dth * (g.R[j + 1] * g.R[j + 1] - g.R[j] * g.R[j]);
  for (int k = 0; k < NV; ++k) div[k] /= V;
  R[0] = div[0];
  const double rho = X.at(g, i, j, 0), tt = X.at(g, i, j, 3), tr = X.at(g, i, j, 4);
  const double T = (3.0 * tt + g.d_r * tr) / (3.0 + g.d_r);
  const double mu = g.mu_ref * pow(T, g.omega);
  const double src = 0.5 * g.d_r * rho * (rho * T) * (T - tr) / (g.z_rot * mu);
  R[1] = div[1];
  R[2] = div[2];
  R[3] = div[3];
  R[4] = div[4] - src;
}

// Residual rows (5) of cell (i, j).  mass_row is the total-mass residual
// sum_c mass_scale_c (rho_c - sampled rho_c) / n, used by cell (1, 0).
__host__ __device__ inline void cell_residual(const Grid& g, const View& X, int i, int j, double mass_row, double* R) {
  if (g.ann) {
    ann_cell_residual(g, X, i, j, R);
    return;
  }
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
  const double wx = width(g, 0, i), wy = width(g, 1, j);
  if (i < g.nx - 1) {
    face_flux(g, X, 0, i, j, Fa);
    for (int k = 0; k < NV; ++k) div[k] += Fa[k] / wx;
  }
  if (i > 0) {
    face_flux(g, X, 0, i - 1, j, Fa);
    for (int k = 0; k < NV; ++k) div[k] -= Fa[k] / wx;
  }
  // y faces: frame (normal y, tangential x) -> components 1 and 2 swap
  if (j < g.ny - 1) {
    face_flux(g, X, 1, i, j, Fa);
    div[0] += Fa[0] / wy;
    div[1] += Fa[2] / wy;
    div[2] += Fa[1] / wy;
    div[3] += Fa[3] / wy;
    div[4] += Fa[4] / wy;
  }
  if (j > 0) {
    face_flux(g, X, 1, i, j - 1, Fa);
    div[0] -= Fa[0] / wy;
    div[1] -= Fa[2] / wy;
    div[2] -= Fa[1] / wy;
    div[3] -= Fa[3] / wy;
    div[4] -= Fa[4] / wy;
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
__host__ __device__ inline int mass_row(const Grid& g) { return g.ann ? -1 : NV * band_cell(g, 1, 0); }

// Band storage (column-major, leading dimension ld): entry (r, c) of the
// matrix at AB[c * ld + r - c + kl + ku], rows c - kl - ku .. c + kl of column
// c (the upper part grows to kl + ku under row interchanges).
__host__ __device__ inline size_t band_at(const Grid& g, int r, int c) {
  return (size_t)c * g.ld + (size_t)(r - c + g.kl + g.ku);
}

// Jacobian entries of one (cell, stencil neighbour, variable): column
// 5 k + v, rows 5 b .. 5 b + 4, by central differences with
// h = 1e-6 max(|x|, 1).  Written twice: in FP32 into the band AB32 (for the
// factorisation; skipped when AB32 is null, as when an earlier factorisation
// is reused) and in FP64 into the compact blocks
// Jc[((b NSTENCIL + s) NV + r) NV + v] (for the refinement's products; zero
// where the neighbour is outside the domain).  The total-mass row is left out
// of both (its factorised row is e_r / n; the rest is carried by a rank-one
// correction).
__host__ __device__ inline size_t jc_at(int b, int s, int r, int v) {
  return (((size_t)b * NSTENCIL + s) * NV + r) * NV + v;
}

__host__ __device__ inline void jacobian_entries(const Grid& g, const double* x, int b, int s, int v, float* AB32,
                                                 double* Jc) {
  int i, j, di, dj;
  cell_of_band(g, b, i, j);
  stencil_offset(s, di, dj);
  int ik, jk;
  if (!stencil_cell(g, i, j, di, dj, ik, jk)) {
    for (int r = 0; r < NV; ++r) Jc[jc_at(b, s, r, v)] = 0.0;
    return;
  }
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
    const double val = row == mr ? 0.0 : (Rp[r] - Rm[r]) / (2.0 * h);
    Jc[jc_at(b, s, r, v)] = val;
    if (AB32 && row != mr) AB32[band_at(g, row, col)] = (float)val;
  }
}

// (B v) of unknown u in FP64 from the compact blocks; B's total-mass row is
// e_r u_1 / n (u_1 = mass_scale of cell (1, 0))
__host__ __device__ inline double bmv_row(const Grid& g, const double* Jc, const double* vec, int u) {
  if (u == mass_row(g)) return mass_scale(g, 1, 0) * vec[u] / g.n;
  const int b = u / NV, r = u - b * NV;
  int i, j;
  cell_of_band(g, b, i, j);
  double acc = 0.0;
  for (int s = 0; s < NSTENCIL; ++s) {
    int di, dj;
    stencil_offset(s, di, dj);
    int ik, jk;
    if (!stencil_cell(g, i, j, di, dj, ik, jk)) continue;
    const double* blk = Jc + jc_at(b, s, r, 0);
    const double* xv = vec + NV * band_cell(g, ik, jk);
    for (int v = 0; v < NV; ++v) acc += blk[v] * xv[v];
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Blocked factorisation in FP32 (right-looking, panels of w <= nb columns):
// the panel of columns k0 .. k0+w-1 and rows k0 .. k0+H-1 (H = min(w + kl,
// N - k0)) is factorised in shared memory with partial pivoting, row
// interchanges applied across the whole panel (its multipliers are stored in
// the panel's own final row order); then every column c of k0+w ..
// min(k0+w-1+kl+ku, N-1) takes the panel's interchanges, the unit-lower
// solve with the panel's top w x w block (rows k0 .. k0+w-1 of U) and the
// update of rows k0+w .. k0+H-1 by the panel's multipliers.  Substitution
// takes the panels in the same order (forward) and in reverse (backward).
//
// FP32 storage: AB32 the band as above (U above and on the diagonal; the
// diagonal also in ud32), piv[k] the row interchanged with row k, and the
// multipliers panel by panel: L(k0 + r, k0 + j) at
// Lp[(k0 / nb) nb (kl + nb) + j (kl + nb) + r], r = j+1 .. H-1 (a later
// interchange of the panel can move a multiplier of column j down to row
// w - 1 + kl, past the kl rows below the diagonal).  Panel arrays in shared
// memory are column-major with leading dimension H.
// ---------------------------------------------------------------------------
__host__ __device__ inline bool in_band(const Grid& g, int r, int c) {
  return r - c <= g.kl && c - r <= g.kl + g.ku;
}

__host__ __device__ inline int panel_width(const Grid& g, int nb, int k0) { return g.N - k0 < nb ? g.N - k0 : nb; }
__host__ __device__ inline int panel_height(const Grid& g, int w, int k0) {
  return g.N - k0 < w + g.kl ? g.N - k0 : w + g.kl;
}
// last row (local) column j of the panel reaches
__host__ __device__ inline int panel_rmax(const Grid& g, int H, int j) { return j + g.kl < H - 1 ? j + g.kl : H - 1; }

__host__ __device__ inline void panel_load(const Grid& g, const float* AB32, int k0, int w, int H, float* P, int tid,
                                           int nthr) {
  for (int c = 0; c < w; ++c) {
#pragma unroll 8
    for (int r = tid; r < H; r += nthr)
      P[(size_t)c * H + r] = in_band(g, k0 + r, k0 + c) ? AB32[band_at(g, k0 + r, k0 + c)] : 0.0f;
  }
}

// first row of largest |P(r, j)|, r = j .. panel_rmax (sequential form)
__host__ __device__ inline int panel_pivot_seq(const Grid& g, const float* P, int H, int j) {
  const float* col = P + (size_t)j * H;
  int p = j;
  float best = fabsf(col[j]);
  for (int r = j + 1; r <= panel_rmax(g, H, j); ++r) {
    const float a = fabsf(col[r]);
    if (a > best) {
      best = a;
      p = r;
    }
  }
  return p;
}

// interchange rows j and p of the panel (all w columns)
__host__ __device__ inline void panel_swap(float* P, int H, int w, int j, int p, int tid, int nthr) {
  if (p == j) return;
  for (int c = tid; c < w; c += nthr) {
    float* col = P + (size_t)c * H;
    const float t = col[j];
    col[j] = col[p];
    col[p] = t;
  }
}

// multipliers of column j (divided by the pivot; 0 if the pivot is 0)
__host__ __device__ inline void panel_scale(const Grid& g, float* P, int H, int j, int tid, int nthr) {
  float* lj = P + (size_t)j * H;
  const float piv = lj[j];
  const int rmax = panel_rmax(g, H, j);
  for (int r = j + 1 + tid; r <= rmax; r += nthr) lj[r] = piv != 0.0f ? lj[r] / piv : 0.0f;
}

// Rank-one update of columns j+1 .. w-1 by column j's multipliers; the
// threads split into ngrp column groups (thread tid: group tid % ngrp, rows
// strided by nthr / ngrp).
__host__ __device__ inline void panel_rank1(const Grid& g, float* P, int H, int w, int j, int tid, int nthr, int ngrp) {
  const float* lj = P + (size_t)j * H;
  const int rmax = panel_rmax(g, H, j);
  const int grp = tid % ngrp, rstride = nthr / ngrp;
  for (int r = j + 1 + tid / ngrp; r <= rmax; r += rstride) {
    const float l = lj[r];
    for (int c = j + 1 + grp; c < w; c += ngrp) {
      float* col = P + (size_t)c * H;
      col[r] -= l * col[j];
    }
  }
}

// start of panel k0's multipliers in Lp
__host__ __device__ inline size_t lp_base(const Grid& g, int nb, int k0) {
  return (size_t)(k0 / nb) * nb * (size_t)(g.kl + nb);
}

// U (rows above and on the diagonal), its diagonal and the multipliers back
// to global memory
__host__ __device__ inline void panel_store(const Grid& g, int nb, float* AB32, float* Lp, float* ud32, int k0, int w,
                                            int H, const float* P, int tid, int nthr) {
  const size_t base = lp_base(g, nb, k0);
  const int ldp = g.kl + nb;
  for (int c = 0; c < w; ++c) {
    const int k = k0 + c;
    for (int r = tid; r < H; r += nthr) {
      const float v = P[(size_t)c * H + r];
      if (r < c) {
        AB32[band_at(g, k0 + r, k)] = v;
      } else if (r == c) {
        ud32[k] = v;
        AB32[band_at(g, k, k)] = v;
      } else {
        Lp[base + (size_t)c * ldp + r] = v;
      }
    }
  }
}

// Trailing columns of the panel at k0: c0 .. c1 (c1 = min(k0+w-1+kl+ku, N-1)).
__host__ __device__ inline int trail_last(const Grid& g, int k0, int w) {
  return k0 + w - 1 + g.kl + g.ku < g.N - 1 ? k0 + w - 1 + g.kl + g.ku : g.N - 1;
}

// the panel's multipliers in shared memory: Ls[j H + r] = L(k0 + r, k0 + j)
__host__ __device__ inline void trail_load_l(const Grid& g, int nb, const float* Lp, int k0, int w, int H, float* Ls,
                                             int tid, int nthr) {
  const float* L = Lp + lp_base(g, nb, k0);
  const int ldp = g.kl + nb;
  for (int j = 0; j < w; ++j) {
#pragma unroll 8
    for (int r = tid; r < H; r += nthr) Ls[(size_t)j * H + r] = r > j ? L[(size_t)j * ldp + r] : 0.0f;
  }
}

// column segments (rows k0 .. k0+H-1) of columns cfirst .. cfirst+ncols-1
__host__ __device__ inline void trail_load_cols(const Grid& g, const float* AB32, int k0, int H, int cfirst, int ncols,
                                                float* Cs, int tid, int nthr) {
  for (int cc = 0; cc < ncols; ++cc) {
    const int c = cfirst + cc;
#pragma unroll 8
    for (int r = tid; r < H; r += nthr) Cs[(size_t)cc * H + r] = in_band(g, k0 + r, c) ? AB32[band_at(g, k0 + r, c)] : 0.0f;
  }
}

// the panel's interchanges, in order, on each column (one thread per column)
__host__ __device__ inline void trail_swaps(const int32_t* piv, int k0, int w, int H, int ncols, float* Cs, int tid,
                                            int nthr) {
  for (int cc = tid; cc < ncols; cc += nthr) {
    float* a = Cs + (size_t)cc * H;
    for (int j = 0; j < w; ++j) {
      const int p = piv[k0 + j] - k0;
      if (p != j) {
        const float t = a[j];
        a[j] = a[p];
        a[p] = t;
      }
    }
  }
}

// unit-lower solve, elimination j (rows j+1 .. w-1 of every column)
__host__ __device__ inline void trail_l11_step(const float* Ls, int w, int H, int ncols, int j, float* Cs, int tid,
                                               int nthr) {
  const int nr = w - j - 1;
  if (nr <= 0) return;
  const float* lj = Ls + (size_t)j * H;
  for (int t = tid; t < ncols * nr; t += nthr) {
    const int cc = t / nr;
    const int i = j + 1 + (t - cc * nr);
    float* a = Cs + (size_t)cc * H;
    a[i] -= lj[i] * a[j];
  }
}

// rows w .. H-1: a(r) -= sum_j L(r, j) a(j)
__host__ __device__ inline void trail_l21(const float* Ls, int w, int H, int ncols, float* Cs, int tid, int nthr) {
  for (int r = w + tid; r < H; r += nthr) {
    for (int cc = 0; cc < ncols; ++cc) {
      float* a = Cs + (size_t)cc * H;
      float acc = 0.0f;
      for (int j = 0; j < w; ++j) acc += Ls[(size_t)j * H + r] * a[j];
      a[r] -= acc;
    }
  }
}

__host__ __device__ inline void trail_store(const Grid& g, float* AB32, int k0, int H, int cfirst, int ncols,
                                            const float* Cs, int tid, int nthr) {
  for (int cc = 0; cc < ncols; ++cc) {
    const int c = cfirst + cc;
    for (int r = tid; r < H; r += nthr)
      if (in_band(g, k0 + r, c)) AB32[band_at(g, k0 + r, c)] = Cs[(size_t)cc * H + r];
  }
}

// ---------------------------------------------------------------------------
// Substitution with the FP32 factors on FP64 vectors (two right-hand sides).
// Forward, panel k0: window s[r] = b(k0 + r), r < H; the panel's
// interchanges; the unit-lower solve with L11 (the panel's y); rows w .. H-1
// less L21 y.  Backward, panel k0 (last to first): window rows
// k0 - kl - ku .. k0 + w - 1 (clipped at 0); the upper solve with U11 (x);
// the rows above less U12 x.
// ---------------------------------------------------------------------------
// L(k0 + r, k0 + j) of panel k0 for local rows j < r < H
__host__ __device__ inline float lmul(const Grid& g, int nb, const float* Lp, int k0, int r, int j) {
  return Lp[lp_base(g, nb, k0) + (size_t)j * (g.kl + nb) + r];
}

__host__ __device__ inline float umul(const Grid& g, const float* AB32, int r, int c) {
  return in_band(g, r, c) ? AB32[band_at(g, r, c)] : 0.0f;
}

}  // namespace s2
}  // namespace dsmc
