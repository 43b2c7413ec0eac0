// dsmc_fields.cu -- FP64 per-cell kernels: sampled fields of
// Eq. (DSMC_macroscopic), the NSF relations of Eq. (ns_constitutive), the
// higher-order terms of Eq. (hot_constitutive) with the Kn_GLL mask of
// Sec. 3.1, and the steady 1D synthetic equations of Eq. (macroscopic_equation)
// solved by Newton's method (Sec. 3 step 3).
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "dsmc_internal.h"

namespace dsmc {

// ---------------------------------------------------------------------------
// fields from the accumulated raw sums (time average over nsamples steps;
// central moments about the averaged velocity)
// ---------------------------------------------------------------------------
__global__ void k_fields(CellParams cp, const double* __restrict__ acc, const double* __restrict__ comp,
                         double nsamples, double* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cp.ncells; c += gridDim.x * blockDim.x) {
    double a[NMOM];
    for (int q = 0; q < NMOM; ++q) a[q] = acc[(size_t)c * NMOM + q] + comp[(size_t)c * NMOM + q];
    double* f = out + (size_t)c * 18;
    const double N = a[0];
    if (!(N > 0.0) || !(nsamples > 0.0)) {
      for (int q = 0; q < 18; ++q) f[q] = 0.0;
      continue;
    }
    const double ux = a[1] / N, uy = a[2] / N, uz = a[3] / N;
    // sum c_i c_j = sum v_i v_j - N u_i u_j
    const double cxx = a[4] - N * ux * ux, cyy = a[5] - N * uy * uy, czz = a[6] - N * uz * uz;
    const double cxy = a[7] - N * ux * uy, cxz = a[8] - N * ux * uz, cyz = a[9] - N * uy * uz;
    const double c2 = cxx + cyy + czz;
    // sum c_i |c|^2 = sum v_i|v|^2 - 2 (S u)_i - u_i tr S + 2 N u_i |u|^2, S = sum v v^T
    const double trS = a[4] + a[5] + a[6];
    const double u2 = ux * ux + uy * uy + uz * uz;
    const double Sux = a[4] * ux + a[7] * uy + a[8] * uz;
    const double Suy = a[7] * ux + a[5] * uy + a[9] * uz;
    const double Suz = a[8] * ux + a[9] * uy + a[6] * uz;
    const double q3x = a[10] - 2.0 * Sux - ux * trS + 2.0 * N * ux * u2;
    const double q3y = a[11] - 2.0 * Suy - uy * trS + 2.0 * N * uy * u2;
    const double q3z = a[12] - 2.0 * Suz - uz * trS + 2.0 * N * uz * u2;
    const double nv = cp.fnum / (cp.vcell * nsamples);
    f[0] = cp.fnum * N / (nsamples * cp.vcell);
    f[1] = ux;
    f[2] = uy;
    f[3] = uz;
    f[4] = c2 / (3.0 * N);
    f[5] = 2.0 * a[13] / (cp.d_r * N);
    f[6] = nv * (cxx - c2 / 3.0);
    f[7] = nv * (cyy - c2 / 3.0);
    f[8] = nv * (czz - c2 / 3.0);
    f[9] = nv * cxy;
    f[10] = nv * cxz;
    f[11] = nv * cyz;
    f[12] = 0.5 * nv * q3x;
    f[13] = 0.5 * nv * q3y;
    f[14] = 0.5 * nv * q3z;
    f[15] = nv * (a[14] - ux * a[13]);
    f[16] = nv * (a[15] - uy * a[13]);
    f[17] = nv * (a[16] - uz * a[13]);
  }
}

void launch_fields(const CellParams& cp, const double* acc, const double* comp, int64_t nsamples, double* out,
                   cudaStream_t st) {
  const int g = (cp.ncells + 255) / 256;
  k_fields<<<g > 0 ? g : 1, 256, 0, st>>>(cp, acc, comp, (double)nsamples, out);
}

__global__ void k_acc_sum(int n, const double* __restrict__ acc, const double* __restrict__ comp,
                          double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = acc[i] + comp[i];
}

void launch_acc_sum(int ncells, const double* acc, const double* comp, double* out, cudaStream_t st) {
  const int n = ncells * NMOM;
  k_acc_sum<<<(n + 255) / 256, 256, 0, st>>>(n, acc, comp, out);
}

// ---------------------------------------------------------------------------
// HoT and Kn_GLL
// ---------------------------------------------------------------------------
// Cell-centred gradient of field value f(cell): central inside, one-sided
// first difference in the first/last cell of a line, 0 with a single cell.
template <typename F>
__device__ __forceinline__ void grad2(const CellParams& cp, int c, F f, double* gx, double* gy) {
  const int ix = c % cp.nx, iy = c / cp.nx;
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

__global__ void k_hot(CellParams cp, const double* __restrict__ F, double* __restrict__ hot,
                      double* __restrict__ kngll, uint8_t* __restrict__ mask) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cp.ncells; c += gridDim.x * blockDim.x) {
    const double* f = F + (size_t)c * 18;
    const double rho = f[0], ux = f[1], uy = f[2], tt = f[4], tr = f[5];
    const double T = (3.0 * tt + cp.d_r * tr) / (3.0 + cp.d_r);
    const double mu = cp.mu_ref * pow(T, cp.omega);
    double duxx, duxy, duyx, duyy, duzx, duzy, dttx, dtty, dtrx, dtry, drx, dry, dsx, dsy;
    grad2(cp, c, [&](int k) { return F[(size_t)k * 18 + 1]; }, &duxx, &duxy);
    grad2(cp, c, [&](int k) { return F[(size_t)k * 18 + 2]; }, &duyx, &duyy);
    grad2(cp, c, [&](int k) { return F[(size_t)k * 18 + 3]; }, &duzx, &duzy);
    grad2(cp, c, [&](int k) { return F[(size_t)k * 18 + 4]; }, &dttx, &dtty);
    grad2(cp, c, [&](int k) { return F[(size_t)k * 18 + 5]; }, &dtrx, &dtry);
    grad2(cp, c, [&](int k) { return F[(size_t)k * 18 + 0]; }, &drx, &dry);
    grad2(cp, c, [&](int k) {
            const double* g = F + (size_t)k * 18;
            return sqrt(g[1] * g[1] + g[2] * g[2] + g[3] * g[3]);
          },
          &dsx, &dsy);
    const double div = duxx + duyy;
    double sig[6];
    sig[0] = -mu * (2.0 * duxx - 2.0 / 3.0 * div);
    sig[1] = -mu * (2.0 * duyy - 2.0 / 3.0 * div);
    sig[2] = -mu * (0.0 - 2.0 / 3.0 * div);
    sig[3] = -mu * (duxy + duyx);
    sig[4] = -mu * duzx;
    sig[5] = -mu * duzy;
    const double qt[3] = {-cp.kappa_t * mu * dttx, -cp.kappa_t * mu * dtty, 0.0};
    const double qr[3] = {-cp.kappa_r * mu * dtrx, -cp.kappa_r * mu * dtry, 0.0};
    // Kn_GLL
    const double gamma = (5.0 + cp.d_r) / (3.0 + cp.d_r);
    const double speed = sqrt(ux * ux + uy * uy + f[3] * f[3]);
    const double lam = mu / (rho * T) * sqrt(PI_D * T / 2.0);
    const double g_rho = hypot(drx, dry) / rho;
    const double g_u = hypot(dsx, dsy) / fmax(speed, sqrt(gamma * T));
    const double g_tt = hypot(dttx, dtty) / tt;
    const double g_tr = hypot(dtrx, dtry) / tr;
    const double kn = lam * fmax(fmax(g_rho, g_u), fmax(g_tt, g_tr));
    const bool keep = kn >= cp.kn_ref;
    double* h = hot + (size_t)c * 12;
    for (int q = 0; q < 6; ++q) h[q] = keep ? f[6 + q] - sig[q] : 0.0;
    for (int q = 0; q < 3; ++q) h[6 + q] = keep ? f[12 + q] - qt[q] : 0.0;
    for (int q = 0; q < 3; ++q) h[9 + q] = keep ? f[15 + q] - qr[q] : 0.0;
    if (kngll) kngll[c] = kn;
    if (mask) mask[c] = keep ? 1 : 0;
  }
}

void launch_hot(const CellParams& cp, const double* fields, double* hot, double* kngll, uint8_t* mask,
                cudaStream_t st) {
  const int g = (cp.ncells + 255) / 256;
  k_hot<<<g > 0 ? g : 1, 256, 0, st>>>(cp, fields, hot, kngll, mask);
}

// ---------------------------------------------------------------------------
// steady 1D synthetic equations (slab between impermeable walls, u_x = 0)
//
// unknowns per cell y = (u_y, u_z, T_t, T_r) and the uniform normal stress
// P = rho T_t + sigma_xx (x-momentum), so rho_i = (P - HoT_xx,i) / T_t,i.
// Faces i+1/2: mean of the two cells for T_t, T_r, u and HoT; mu at the face
// temperature.  Rows: boundary cells keep the sampled (u_y, u_z, T_t, T_r);
// inside, d/dx sigma_xy = 0, d/dx sigma_xz = 0,
// d/dx (sigma_xy u_y + sigma_xz u_z + q_t + q_r) = 0,
// -d/dx q_r + (d_r/2) rho p (T - T_r) / (Z mu) = 0 with p = rho T;
// plus sum rho_i dx = sampled mass.  Newton with a Jacobian by central
// differences of each cell's local residual, and a bordered block-tridiagonal
// solve (block Thomas, one thread).
// ---------------------------------------------------------------------------
struct SynthArgs {
  CellParams cp;
  const double* F;    // sampled fields, ncells x 18
  const double* hot;  // ncells x 12
};

__device__ __forceinline__ void face_flux(const SynthArgs& a, int i, const double* yl, const double* yr,
                                          double* sxy, double* sxz, double* qr, double* e) {
  const CellParams& cp = a.cp;
  const double ttf = 0.5 * (yl[2] + yr[2]);
  const double trf = 0.5 * (yl[3] + yr[3]);
  const double Tf = (3.0 * ttf + cp.d_r * trf) / (3.0 + cp.d_r);
  const double muf = cp.mu_ref * pow(Tf, cp.omega);
  const double* hl = a.hot + (size_t)i * 12;
  const double* hr = a.hot + (size_t)(i + 1) * 12;
  const double h3 = 0.5 * (hl[3] + hr[3]), h4 = 0.5 * (hl[4] + hr[4]);
  const double h6 = 0.5 * (hl[6] + hr[6]), h9 = 0.5 * (hl[9] + hr[9]);
  *sxy = -muf * (yr[0] - yl[0]) / cp.dx + h3;
  *sxz = -muf * (yr[1] - yl[1]) / cp.dx + h4;
  const double qt = -cp.kappa_t * muf * (yr[2] - yl[2]) / cp.dx + h6;
  *qr = -cp.kappa_r * muf * (yr[3] - yl[3]) / cp.dx + h9;
  const double uyf = 0.5 * (yl[0] + yr[0]), uzf = 0.5 * (yl[1] + yr[1]);
  *e = *sxy * uyf + *sxz * uzf + qt + *qr;
}

// residual rows of cell i from y_{i-1}, y_i, y_{i+1} and P
__device__ void local_res(const SynthArgs& a, int i, int n, const double* ym, const double* y0,
                          const double* yp, double P, double* R) {
  const CellParams& cp = a.cp;
  if (i == 0 || i == n - 1) {
    const double* f = a.F + (size_t)i * 18;
    R[0] = y0[0] - f[2];
    R[1] = y0[1] - f[3];
    R[2] = y0[2] - f[4];
    R[3] = y0[3] - f[5];
    return;
  }
  double sxy_p, sxz_p, qr_p, e_p, sxy_m, sxz_m, qr_m, e_m;
  face_flux(a, i, y0, yp, &sxy_p, &sxz_p, &qr_p, &e_p);
  face_flux(a, i - 1, ym, y0, &sxy_m, &sxz_m, &qr_m, &e_m);
  const double rho = (P - a.hot[(size_t)i * 12 + 0]) / y0[2];
  const double T = (3.0 * y0[2] + cp.d_r * y0[3]) / (3.0 + cp.d_r);
  const double mu = cp.mu_ref * pow(T, cp.omega);
  const double src = 0.5 * cp.d_r * rho * (rho * T) * (T - y0[3]) / (cp.z_rot * mu);
  R[0] = sxy_p - sxy_m;
  R[1] = sxz_p - sxz_m;
  R[2] = e_p - e_m;
  R[3] = -(qr_p - qr_m) / cp.dx + src;
}

__device__ void inv4(const double* m, double* r) {
  // Gauss-Jordan with partial pivoting on a 4x4 matrix
  double a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      a[i][j] = m[i * 4 + j];
      a[i][4 + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int i = c + 1; i < 4; ++i)
      if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
    if (piv != c)
      for (int j = 0; j < 8; ++j) {
        const double t = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = t;
      }
    const double d = a[c][c];
    for (int j = 0; j < 8; ++j) a[c][j] /= d;
    for (int i = 0; i < 4; ++i)
      if (i != c) {
        const double fct = a[i][c];
        for (int j = 0; j < 8; ++j) a[i][j] -= fct * a[c][j];
      }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r[i * 4 + j] = a[i][4 + j];
}

__device__ __forceinline__ void mm4(const double* a, const double* b, double* c) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[i * 4 + k] * b[k * 4 + j];
      c[i * 4 + j] = s;
    }
}

__device__ __forceinline__ void mv4(const double* a, const double* x, double* y) {
  for (int i = 0; i < 4; ++i) {
    double s = 0.0;
    for (int k = 0; k < 4; ++k) s += a[i * 4 + k] * x[k];
    y[i] = s;
  }
}

size_t synth1d_work_doubles(int n) { return (size_t)n * (4 * 6 + 16 * 4 + 4) + 64; }

__global__ void __launch_bounds__(256) k_synth1d(SynthArgs a, double* __restrict__ out, double* __restrict__ work,
                                                 int n_m, double tol, double* __restrict__ info) {
  const CellParams& cp = a.cp;
  const int n = cp.nx;
  double* y = work;             // 4n
  double* R = y + 4 * n;        // 4n
  double* Gp = R + 4 * n;       // 4n  dR_i/dP
  double* z1 = Gp + 4 * n;      // 4n
  double* z2 = z1 + 4 * n;      // 4n
  double* yn = z2 + 4 * n;      // 4n
  double* A = yn + 4 * n;       // 16n dR_i/dy_{i-1}
  double* B = A + 16 * n;       // 16n dR_i/dy_i
  double* C = B + 16 * n;       // 16n dR_i/dy_{i+1}
  double* W = C + 16 * n;       // 16n Thomas: inverse of the reduced diagonal
  double* hvec = W + 16 * n;    // 4n  dR_P/dy_i
  __shared__ double s_P, s_M, s_red[256];
  __shared__ int s_done, s_it, s_bad;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) {
    const double* f = a.F + (size_t)i * 18;
    y[4 * i + 0] = f[2];
    y[4 * i + 1] = f[3];
    y[4 * i + 2] = f[4];
    y[4 * i + 3] = f[5];
  }
  // sampled mass and the initial P (mean of rho T_t + HoT_xx)
  double m = 0.0, pm = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    const double* f = a.F + (size_t)i * 18;
    m += f[0] * cp.dx;
    pm += f[0] * f[4] + a.hot[(size_t)i * 12];
  }
  s_red[tid] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o) s_red[tid] += s_red[tid + o];
    __syncthreads();
  }
  if (tid == 0) s_M = s_red[0];
  __syncthreads();
  s_red[tid] = pm;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o) s_red[tid] += s_red[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    s_P = s_red[0] / n;
    s_done = 0;
    s_it = 0;
    s_bad = 0;
  }
  __syncthreads();
  for (int it = 1; it <= n_m; ++it) {
    const double P = s_P;
    // residuals, local Jacobian blocks and the border
    for (int i = tid; i < n; i += blockDim.x) {
      double ym[4], y0[4], yp[4];
      for (int v = 0; v < 4; ++v) {
        y0[v] = y[4 * i + v];
        ym[v] = (i > 0) ? y[4 * (i - 1) + v] : y0[v];
        yp[v] = (i < n - 1) ? y[4 * (i + 1) + v] : y0[v];
      }
      local_res(a, i, n, ym, y0, yp, P, R + 4 * i);
      double rp[4], rm[4];
      for (int blk = 0; blk < 3; ++blk) {
        double* J = (blk == 0 ? A : (blk == 1 ? B : C)) + 16 * i;
        double* yy = (blk == 0 ? ym : (blk == 1 ? y0 : yp));
        const bool exists = (blk == 1) || (blk == 0 && i > 0) || (blk == 2 && i < n - 1);
        for (int v = 0; v < 4; ++v) {
          if (!exists) {
            for (int r = 0; r < 4; ++r) J[r * 4 + v] = 0.0;
            continue;
          }
          const double sv = yy[v];
          const double h = 1e-6 * fmax(fabs(sv), 1.0);
          yy[v] = sv + h;
          local_res(a, i, n, ym, y0, yp, P, rp);
          yy[v] = sv - h;
          local_res(a, i, n, ym, y0, yp, P, rm);
          yy[v] = sv;
          for (int r = 0; r < 4; ++r) J[r * 4 + v] = (rp[r] - rm[r]) / (2.0 * h);
        }
      }
      const double hP = 1e-6 * fmax(fabs(P), 1.0);
      local_res(a, i, n, ym, y0, yp, P + hP, rp);
      local_res(a, i, n, ym, y0, yp, P - hP, rm);
      for (int r = 0; r < 4; ++r) Gp[4 * i + r] = (rp[r] - rm[r]) / (2.0 * hP);
      // mass row: d(sum rho dx)/dT_t,i = -dx (P - H_i)/T_t,i^2
      const double Hi = a.hot[(size_t)i * 12];
      hvec[4 * i + 0] = 0.0;
      hvec[4 * i + 1] = 0.0;
      hvec[4 * i + 2] = -cp.dx * (P - Hi) / (y0[2] * y0[2]);
      hvec[4 * i + 3] = 0.0;
    }
    __syncthreads();
    if (tid == 0) {
      // mass residual and dR_P/dP
      double mass = 0.0, dP = 0.0;
      for (int i = 0; i < n; ++i) {
        const double Hi = a.hot[(size_t)i * 12];
        mass += (P - Hi) / y[4 * i + 2] * cp.dx;
        dP += cp.dx / y[4 * i + 2];
      }
      const double RP = mass - s_M;
      // block Thomas for T z1 = -R and T z2 = Gp
      for (int i = 0; i < n; ++i) {
        double Bi[16], r1[4], r2[4];
        for (int q = 0; q < 16; ++q) Bi[q] = B[16 * i + q];
        for (int v = 0; v < 4; ++v) {
          r1[v] = -R[4 * i + v];
          r2[v] = Gp[4 * i + v];
        }
        if (i > 0) {
          // Bi -= A_i W_{i-1} C_{i-1};  r -= A_i W_{i-1} r_{i-1}
          double AW[16], AWC[16], t1[4], t2[4];
          mm4(A + 16 * i, W + 16 * (i - 1), AW);
          mm4(AW, C + 16 * (i - 1), AWC);
          for (int q = 0; q < 16; ++q) Bi[q] -= AWC[q];
          mv4(AW, z1 + 4 * (i - 1), t1);
          mv4(AW, z2 + 4 * (i - 1), t2);
          for (int v = 0; v < 4; ++v) {
            r1[v] -= t1[v];
            r2[v] -= t2[v];
          }
        }
        inv4(Bi, W + 16 * i);
        for (int v = 0; v < 4; ++v) {
          z1[4 * i + v] = r1[v];
          z2[4 * i + v] = r2[v];
        }
      }
      // back substitution: x_i = W_i (r_i - C_i x_{i+1})
      for (int i = n - 1; i >= 0; --i) {
        double t1[4], t2[4];
        for (int v = 0; v < 4; ++v) {
          t1[v] = z1[4 * i + v];
          t2[v] = z2[4 * i + v];
        }
        if (i < n - 1) {
          double c1[4], c2[4];
          mv4(C + 16 * i, z1 + 4 * (i + 1), c1);
          mv4(C + 16 * i, z2 + 4 * (i + 1), c2);
          for (int v = 0; v < 4; ++v) {
            t1[v] -= c1[v];
            t2[v] -= c2[v];
          }
        }
        mv4(W + 16 * i, t1, z1 + 4 * i);
        mv4(W + 16 * i, t2, z2 + 4 * i);
      }
      // bordered correction: [T g; h^T d] [dy; dP] = [-R; -RP]
      double hz1 = 0.0, hz2 = 0.0;
      for (int i = 0; i < n; ++i)
        for (int v = 0; v < 4; ++v) {
          hz1 += hvec[4 * i + v] * z1[4 * i + v];
          hz2 += hvec[4 * i + v] * z2[4 * i + v];
        }
      const double dPstep = (-RP - hz1) / (dP - hz2);
      // damped update keeping rho > 0, T > 0
      double lam = 1.0;
      int ok = 0;
      for (int tries = 0; tries < 40 && !ok; ++tries) {
        ok = 1;
        const double Pn = P + lam * dPstep;
        for (int i = 0; i < n && ok; ++i) {
          for (int v = 0; v < 4; ++v) yn[4 * i + v] = y[4 * i + v] + lam * (z1[4 * i + v] - z2[4 * i + v] * dPstep);
          const double rho = (Pn - a.hot[(size_t)i * 12]) / yn[4 * i + 2];
          if (!(yn[4 * i + 2] > 0.0) || !(yn[4 * i + 3] > 0.0) || !(rho > 0.0)) ok = 0;
        }
        if (!ok) lam *= 0.5;
      }
      double dmax = 0.0;
      if (ok) {
        for (int i = 0; i < n; ++i)
          for (int v = 0; v < 4; ++v) {
            const double d = fabs(yn[4 * i + v] - y[4 * i + v]) / fmax(fabs(y[4 * i + v]), 1e-3);
            dmax = fmax(dmax, d);
            y[4 * i + v] = yn[4 * i + v];
          }
        const double Pn = P + lam * dPstep;
        dmax = fmax(dmax, fabs(Pn - P) / fmax(fabs(P), 1e-3));
        s_P = Pn;
      } else {
        s_bad = 1;
      }
      s_it = it;
      if (!ok || dmax < tol) s_done = 1;
    }
    __syncthreads();
    if (s_done) break;
  }
  // final residual and output
  const double P = s_P;
  double rmax = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    double ym[4], y0[4], yp[4], r[4];
    for (int v = 0; v < 4; ++v) {
      y0[v] = y[4 * i + v];
      ym[v] = (i > 0) ? y[4 * (i - 1) + v] : y0[v];
      yp[v] = (i < n - 1) ? y[4 * (i + 1) + v] : y0[v];
    }
    local_res(a, i, n, ym, y0, yp, P, r);
    for (int v = 0; v < 4; ++v) rmax = fmax(rmax, fabs(r[v]));
    double* o = out + (size_t)i * 6;
    o[0] = (P - a.hot[(size_t)i * 12]) / y0[2];
    o[1] = 0.0;
    o[2] = y0[0];
    o[3] = y0[1];
    o[4] = y0[2];
    o[5] = y0[3];
  }
  s_red[tid] = rmax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o) s_red[tid] = fmax(s_red[tid], s_red[tid + o]);
    __syncthreads();
  }
  if (tid == 0) {
    info[0] = (double)s_it;
    info[1] = s_red[0];
    info[2] = s_bad ? 2.0 : (s_done ? 0.0 : 1.0);  // 0 converged, 1 not converged, 2 numeric
  }
}

void launch_synth1d(const CellParams& cp, const double* fields, const double* hot, double* out, double* work,
                    int n_m, double tol, double* dev_info, cudaStream_t st) {
  SynthArgs a{cp, fields, hot};
  k_synth1d<<<1, 256, 0, st>>>(a, out, work, n_m, tol, dev_info);
}

}  // namespace dsmc
