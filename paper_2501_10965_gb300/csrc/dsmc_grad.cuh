// dsmc_grad.cuh -- cell-centred gradients on the DSMC mesh, shared by the
// HoT / Kn_GLL kernel and the HoT surrogate's input features.
#pragma once

#include "dsmc_internal.h"

namespace dsmc {

// Cell-centred gradient of field value f(cell): central inside, one-sided
// first difference in the first/last cell of a line, 0 with a single cell.
template <typename F>
__device__ __forceinline__ void grad2(const CellParams& cp, int c, int lc, F f, double* gx, double* gy) {
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
