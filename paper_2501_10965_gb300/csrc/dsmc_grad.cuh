// dsmc_grad.cuh -- cell-centred gradients on the DSMC mesh, shared by the
// HoT / Kn_GLL kernel and the HoT surrogate's input features.
#pragma once

#include "dsmc_internal.h"

namespace dsmc {

// Annulus (nx sectors x ny rings, cell j nx + k): the Cartesian gradient at
// the cell centre (mid radius r_j, angle theta_k = 2 pi (k + 1/2) / nx) from
// the polar derivatives: d/dr by the three-point formula on the stretched
// rings (one-sided first difference in the first and last ring), (1/r)
// d/dtheta = (f_{k+1} - f_{k-1}) / (2 r_j sin(dtheta)) around the ring
// (exact for fields linear in x and y); then d/dx = cos d/dr - sin (1/r)
// d/dtheta, d/dy = sin d/dr + cos (1/r) d/dtheta.
template <typename F>
__device__ __forceinline__ void grad_ann(const CellParams& cp, int c, int lc, F f, double* gx, double* gy) {
  const int nt = cp.nx, nr = cp.ny;
  const int k = lc % nt, j = lc / nt;
  auto rmid = [&](int q) { return 0.5 * (sqrt(cp.r2t[q]) + sqrt(cp.r2t[q + 1])); };
  const double r = rmid(j);
  double dr = 0.0;
  if (nr >= 2) {
    if (j == 0) {
      dr = (f(c + nt) - f(c)) / (rmid(1) - r);
    } else if (j == nr - 1) {
      dr = (f(c) - f(c - nt)) / (r - rmid(j - 1));
    } else {
      const double hm = r - rmid(j - 1), hp = rmid(j + 1) - r;
      dr = (hm * hm * f(c + nt) - hp * hp * f(c - nt) + (hp * hp - hm * hm) * f(c)) / (hp * hm * (hp + hm));
    }
  }
  const int kp = (k == nt - 1) ? c - (nt - 1) : c + 1, km = (k == 0) ? c + (nt - 1) : c - 1;
  const double dth = 2.0 * PI_D / (double)nt;
  const double dt = (f(kp) - f(km)) / (2.0 * r * sin(dth));
  const double th = 2.0 * PI_D * ((double)k + 0.5) / (double)nt;
  const double ct = cos(th), st = sin(th);
  *gx = ct * dr - st * dt;
  *gy = st * dr + ct * dt;
}

// d/dx at cell i of a line with cell edges e (n cells; neighbours at
// cell-index distance `step`): the three-point formula on the unequal
// spacing of the cell centres, one-sided first differences at the ends
template <typename F>
__device__ __forceinline__ double d_nonuniform(const double* e, int n, int i, int c, int step, F f) {
  auto xc = [&](int q) { return 0.5 * (e[q] + e[q + 1]); };
  if (n < 2) return 0.0;
  if (i == 0) return (f(c + step) - f(c)) / (xc(1) - xc(0));
  if (i == n - 1) return (f(c) - f(c - step)) / (xc(n - 1) - xc(n - 2));
  const double hm = xc(i) - xc(i - 1), hp = xc(i + 1) - xc(i);
  return (hm * hm * f(c + step) - hp * hp * f(c - step) + (hp * hp - hm * hm) * f(c)) / (hp * hm * (hp + hm));
}

// Cell-centred gradient of field value f(cell): central inside, one-sided
// first difference in the first/last cell of a line, 0 with a single cell;
// on the annulus, grad_ann; on the wall-refined box, the three-point
// formula on the unequal cell widths along each axis.
template <typename F>
__device__ __forceinline__ void grad2(const CellParams& cp, int c, int lc, F f, double* gx, double* gy) {
  if (cp.mesh == 1) {
    grad_ann(cp, c, lc, f, gx, gy);
    return;
  }
  if (cp.mesh == 2) {
    const int ix = lc % cp.nx, iy = lc / cp.nx;
    *gx = d_nonuniform(cp.xe, cp.nx, ix, c, 1, f);
    *gy = d_nonuniform(cp.ye, cp.ny, iy, c, cp.nx, f);
    return;
  }
  const int ix = lc % cp.nx, iy = lc / cp.nx;
  *gx = 0.0;
  *gy = 0.0;
  if (cp.nx >= 2) {
    if (ix == 0) *gx = (f(c + 1) - f(c)) / cp.dx;
    else if (ix == cp.nx - 1) *gx = (f(c) - f(c - 1)) / cp.dx;
    else *gx = (f(c + 1) - f(c - 1)) / (2.0 * cp.dx);
  }
  if (cp.dim == 2 && cp.ny >= 2) {
    const int nx = cp.nx;
    if (iy == 0) *gy = (f(c + nx) - f(c)) / cp.dy;
    else if (iy == cp.ny - 1) *gy = (f(c) - f(c - nx)) / cp.dy;
    else *gy = (f(c + nx) - f(c - nx)) / (2.0 * cp.dy);
  }
}

}  // namespace dsmc
