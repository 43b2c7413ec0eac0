// dsmc_fields.cu -- FP64 per-cell kernels: sampled fields of
// Eq. (DSMC_macroscopic), the NSF relations of Eq. (ns_constitutive), the
// higher-order terms of Eq. (hot_constitutive) with the Kn_GLL mask of
// Sec. 3.1, and the steady 1D synthetic equations of Eq. (macroscopic_equation)
// solved by Newton's method (Sec. 3 step 3).
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "dsmc_internal.h"
#include "dsmc_grad.cuh"

namespace dsmc {

// ---------------------------------------------------------------------------
// fields from the accumulated raw sums (time average over nsamples steps;
// central moments about the averaged velocity)
// ---------------------------------------------------------------------------
__global__ void k_fields(const CellParams* __restrict__ cps, const int32_t* __restrict__ cell_case, int ncells,
                         const double* __restrict__ acc, const double* __restrict__ comp, double nsamples,
                         double* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    const CellParams& cp = cps[cell_case[c]];
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
    const double vc = cp.vol ? cp.vol[c] : cp.vcell;  // annulus: one case, global cell = local cell
    const double nv = cp.fnum / (vc * nsamples);
    f[0] = cp.fnum * N / (nsamples * vc);
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

void launch_fields(const CellParams* cp, const int32_t* cell_case, int ncells, const double* acc, const double* comp,
                   int64_t nsamples, double* out, cudaStream_t st) {
  const int g = (ncells + 255) / 256;
  k_fields<<<g > 0 ? g : 1, 256, 0, st>>>(cp, cell_case, ncells, acc, comp, (double)nsamples, out);
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
__global__ void k_hot(const CellParams* __restrict__ cps, const int32_t* __restrict__ cell_case,
                      const int32_t* __restrict__ cell0, int ncells, const double* __restrict__ F,
                      double* __restrict__ hot, double* __restrict__ kngll, uint8_t* __restrict__ mask) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    const int cs = cell_case[c];
    const CellParams& cp = cps[cs];
    const int lc = c - cell0[cs];
    const double* f = F + (size_t)c * 18;
    const double rho = f[0], ux = f[1], uy = f[2], tt = f[4], tr = f[5];
    const double T = (3.0 * tt + cp.d_r * tr) / (3.0 + cp.d_r);
    const double mu = cp.mu_ref * pow(T, cp.omega);
    double duxx, duxy, duyx, duyy, duzx, duzy, dttx, dtty, dtrx, dtry, drx, dry, dsx, dsy;
    grad2(cp, c, lc, [&](int k) { return F[(size_t)k * 18 + 1]; }, &duxx, &duxy);
    grad2(cp, c, lc, [&](int k) { return F[(size_t)k * 18 + 2]; }, &duyx, &duyy);
    grad2(cp, c, lc, [&](int k) { return F[(size_t)k * 18 + 3]; }, &duzx, &duzy);
    grad2(cp, c, lc, [&](int k) { return F[(size_t)k * 18 + 4]; }, &dttx, &dtty);
    grad2(cp, c, lc, [&](int k) { return F[(size_t)k * 18 + 5]; }, &dtrx, &dtry);
    grad2(cp, c, lc, [&](int k) { return F[(size_t)k * 18 + 0]; }, &drx, &dry);
    grad2(cp, c, lc, [&](int k) {
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

void launch_hot(const CellParams* cp, const int32_t* cell_case, const int32_t* cell0, int ncells,
                const double* fields, double* hot, double* kngll, uint8_t* mask, cudaStream_t st) {
  const int g = (ncells + 255) / 256;
  k_hot<<<g > 0 ? g : 1, 256, 0, st>>>(cp, cell_case, cell0, ncells, fields, hot, kngll, mask);
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
// plus sum rho_i dx = sampled mass.  Newton: the residual in FP64 (each face's
// fluxes once, then each cell's rows), the Jacobian by central differences in
// FP32, a bordered block-tridiagonal solve by cyclic reduction in FP32 with
// the mass row in FP64.
// ---------------------------------------------------------------------------
struct SynthArgs {
  CellParams cp;
  const double* F;    // sampled fields, ncells x 18
  const double* hot;  // ncells x 12
};

// The slabs of a solve: either one slab described by cp1 (tables null) or
// several, case c with parameters cps[c], cells [cell0[c], cell0[c+1]) and
// work at work + woff[c].
struct SynthCases {
  CellParams cp1;
  const CellParams* cps;
  const int32_t* cell_case;
  const int32_t* cell0;
  const int64_t* woff;
  const double* F;
  const double* hot;
  double* work;
  double* info;  // 3 per case + a count of finished cases
  int ncases;
  int ncells;
};

__device__ __forceinline__ SynthArgs case_args(const SynthCases& sc, int c) {
  const int off = sc.cell0 ? sc.cell0[c] : 0;
  SynthArgs a;
  a.cp = sc.cps ? sc.cps[c] : sc.cp1;
  a.F = sc.F + (size_t)off * 18;
  a.hot = sc.hot + (size_t)off * 12;
  return a;
}

__device__ __forceinline__ double* case_work(const SynthCases& sc, int c) {
  return sc.work + (sc.woff ? sc.woff[c] : 0);
}

// FP64 fluxes at face i+1/2 from the states of cells i (yl) and i+1 (yr):
// f = (sigma_xy, sigma_xz, q_r, sigma_xy u_y + sigma_xz u_z + q_t + q_r)
__device__ __forceinline__ void face_flux(const SynthArgs& a, int i, const double* yl, const double* yr, double* f) {
  const CellParams& cp = a.cp;
  const double d_r = cp.d_r, dx = cp.dx;
  const double ttf = 0.5 * (yl[2] + yr[2]);
  const double trf = 0.5 * (yl[3] + yr[3]);
  const double Tf = (3.0 * ttf + d_r * trf) / (3.0 + d_r);
  const double muf = cp.mu_ref * pow(Tf, cp.omega);
  const double* hl = a.hot + (size_t)i * 12;
  const double* hr = a.hot + (size_t)(i + 1) * 12;
  const double h3 = 0.5 * (hl[3] + hr[3]), h4 = 0.5 * (hl[4] + hr[4]);
  const double h6 = 0.5 * (hl[6] + hr[6]), h9 = 0.5 * (hl[9] + hr[9]);
  const double sxy = -muf * (yr[0] - yl[0]) / dx + h3;
  const double sxz = -muf * (yr[1] - yl[1]) / dx + h4;
  const double qt = -cp.kappa_t * muf * (yr[2] - yl[2]) / dx + h6;
  const double qr = -cp.kappa_r * muf * (yr[3] - yl[3]) / dx + h9;
  const double uyf = 0.5 * (yl[0] + yr[0]), uzf = 0.5 * (yl[1] + yr[1]);
  f[0] = sxy;
  f[1] = sxz;
  f[2] = qr;
  f[3] = sxy * uyf + sxz * uzf + qt + qr;
}

// FP64 residual rows of cell i from its state y0, the fluxes fm, fp of faces
// i-1/2 and i+1/2, and P
__device__ __forceinline__ void cell_rows(const SynthArgs& a, int i, int n, const double* y0, const double* fm,
                                          const double* fp, double P, double* R) {
  const CellParams& cp = a.cp;
  if (i == 0 || i == n - 1) {
    const double* f = a.F + (size_t)i * 18;
    R[0] = y0[0] - f[2];
    R[1] = y0[1] - f[3];
    R[2] = y0[2] - f[4];
    R[3] = y0[3] - f[5];
    return;
  }
  const double d_r = cp.d_r;
  const double rho = (P - a.hot[(size_t)i * 12 + 0]) / y0[2];
  const double Tc = (3.0 * y0[2] + d_r * y0[3]) / (3.0 + d_r);
  const double mu = cp.mu_ref * pow(Tc, cp.omega);
  const double src = 0.5 * d_r * rho * (rho * Tc) * (Tc - y0[3]) / (cp.z_rot * mu);
  R[0] = fp[0] - fm[0];
  R[1] = fp[1] - fm[1];
  R[2] = fp[3] - fm[3];
  R[3] = -(fp[2] - fm[2]) / cp.dx + src;
}

// Work layout, n cells.  Doubles: y (4n), yn (4n; also the face fluxes of
// the residual), R (4n), scalars (32).  Floats: A, B, C, Binv (16n each;
// the blocks d R_i / d y_{i-1}, d y_i, d y_{i+1}), r1, r2 (4n each; -R and
// dR/dP, overwritten by the reduction), yf (4n; y in FP32), hf (4n; HoT
// sigma_xy, sigma_xz, q_t,x, q_r,x at face i+1/2), h0 (n; HoT sigma_xx per
// cell), kf (16; constants and P in FP32).
size_t synth1d_work_doubles(int n) { return (size_t)n * 12 + 32 + ((size_t)n * 85 + 16 + 1) / 2 + 64; }

struct SynthWork {
  double *y, *yn, *R, *sc;
  float *A, *B, *C, *Bi, *r1, *r2, *yf, *hf, *h0, *kf;
};

__host__ __device__ inline SynthWork synth_work(double* w, int n) {
  SynthWork s;
  s.y = w;
  s.yn = s.y + 4 * n;
  s.R = s.yn + 4 * n;
  s.sc = s.R + 4 * n;
  float* f = reinterpret_cast<float*>(s.sc + 32);
  s.A = f;
  s.B = s.A + 16 * n;
  s.C = s.B + 16 * n;
  s.Bi = s.C + 16 * n;
  s.r1 = s.Bi + 16 * n;
  s.r2 = s.r1 + 4 * n;
  s.yf = s.r2 + 4 * n;
  s.hf = s.yf + 4 * n;
  s.h0 = s.hf + 4 * n;
  s.kf = s.h0 + n;
  return s;
}

// scalar slots: 0 P, 1 mass, 2 done, 3 iterations, 4 status (0 converged,
// 1 not (yet) converged, 2 numeric), 5 last max relative change
enum { SC_P = 0, SC_M = 1, SC_DONE = 2, SC_IT = 3, SC_STATUS = 4, SC_DMAX = 5 };
// FP32 constants of the Jacobian
enum { KF_DR = 0, KF_IDX, KF_I3DR, KF_MUREF, KF_OMEGA, KF_KT, KF_KR, KF_IZ, KF_P };

template <int NT>
__device__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
#pragma unroll
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

template <int NT>
__device__ double block_max(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
#pragma unroll
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// FP64 residual of every cell into w.R (the face fluxes go through w.yn)
template <int NT>
__device__ void residual_fp64(const SynthArgs& a, const SynthWork& w, int n, double P) {
  const int tid = threadIdx.x;
  for (int i = tid; i < n - 1; i += NT) face_flux(a, i, w.y + 4 * i, w.y + 4 * (i + 1), w.yn + 4 * i);
  __syncthreads();
  for (int i = tid; i < n; i += NT) {
    const double* fm = (i > 0) ? w.yn + 4 * (i - 1) : nullptr;
    const double* fp = (i < n - 1) ? w.yn + 4 * i : nullptr;
    cell_rows(a, i, n, w.y + 4 * i, fm, fp, P, w.R + 4 * i);
  }
  __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) k_synth_init(const __grid_constant__ SynthCases scs) {
  __shared__ double red[NT];
  const int cs = blockIdx.x;
  const SynthArgs a = case_args(scs, cs);
  double* work = case_work(scs, cs);
  const int n = a.cp.nx;
  SynthWork w = synth_work(work, n);
  double m = 0.0, pm = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    const double* f = a.F + (size_t)i * 18;
    const double* h = a.hot + (size_t)i * 12;
    for (int v = 0; v < 4; ++v) {
      w.y[4 * i + v] = f[2 + v];
      w.yf[4 * i + v] = (float)f[2 + v];
    }
    w.h0[i] = (float)h[0];
    if (i < n - 1) {
      const double* hr = h + 12;
      w.hf[4 * i + 0] = (float)(0.5 * (h[3] + hr[3]));
      w.hf[4 * i + 1] = (float)(0.5 * (h[4] + hr[4]));
      w.hf[4 * i + 2] = (float)(0.5 * (h[6] + hr[6]));
      w.hf[4 * i + 3] = (float)(0.5 * (h[9] + hr[9]));
    }
    m += f[0] * a.cp.dx;
    pm += f[0] * f[4] + h[0];
  }
  const double M = block_sum<NT>(m, red);
  const double PM = block_sum<NT>(pm, red);
  if (threadIdx.x == 0) {
    const CellParams& cp = a.cp;
    w.sc[SC_P] = PM / n;
    w.sc[SC_M] = M;
    w.sc[SC_DONE] = 0.0;
    w.sc[SC_IT] = 0.0;
    w.sc[SC_STATUS] = 1.0;
    w.sc[SC_DMAX] = 0.0;
    w.kf[KF_DR] = (float)cp.d_r;
    w.kf[KF_IDX] = (float)(1.0 / cp.dx);
    w.kf[KF_I3DR] = (float)(1.0 / (3.0 + cp.d_r));
    w.kf[KF_MUREF] = (float)cp.mu_ref;
    w.kf[KF_OMEGA] = (float)cp.omega;
    w.kf[KF_KT] = (float)cp.kappa_t;
    w.kf[KF_KR] = (float)cp.kappa_r;
    w.kf[KF_IZ] = (float)(1.0 / cp.z_rot);
    w.kf[KF_P] = (float)(PM / n);
  }
}

// FP32 counterparts for the Jacobian (they only steer Newton's steps: the
// FP64 residual decides the solution)
struct SynthKf {
  float d_r, idx, i3dr, mu_ref, omega, kt, kr, iz;
};

__device__ __forceinline__ float synth_powf(float x, float e) { return exp2f(e * __log2f(x)); }

__device__ __forceinline__ void face_flux_f(const SynthKf& k, const float* hf, const float* yl, const float* yr,
                                            float* f) {
  const float ttf = 0.5f * (yl[2] + yr[2]);
  const float trf = 0.5f * (yl[3] + yr[3]);
  const float Tf = (3.f * ttf + k.d_r * trf) * k.i3dr;
  const float muf = k.mu_ref * synth_powf(Tf, k.omega);
  const float sxy = -muf * (yr[0] - yl[0]) * k.idx + hf[0];
  const float sxz = -muf * (yr[1] - yl[1]) * k.idx + hf[1];
  const float qt = -k.kt * muf * (yr[2] - yl[2]) * k.idx + hf[2];
  const float qr = -k.kr * muf * (yr[3] - yl[3]) * k.idx + hf[3];
  f[0] = sxy;
  f[1] = sxz;
  f[2] = qr;
  f[3] = sxy * (0.5f * (yl[0] + yr[0])) + sxz * (0.5f * (yl[1] + yr[1])) + qt + qr;
}

__device__ __forceinline__ float source_f(const SynthKf& k, float h0, const float* y0, float P) {
  const float rho = __fdividef(P - h0, y0[2]);
  const float Tc = (3.f * y0[2] + k.d_r * y0[3]) * k.i3dr;
  const float mu = k.mu_ref * synth_powf(Tc, k.omega);
  return __fdividef(0.5f * k.d_r * rho * (rho * Tc) * (Tc - y0[3]) * k.iz, mu);
}

__device__ __forceinline__ void rows_f(const SynthKf& k, const float* hfm, const float* hfp, float h0,
                                       const float* ym, const float* y0, const float* yp, float P, float* R) {
  float fm[4], fp[4];
  face_flux_f(k, hfm, ym, y0, fm);
  face_flux_f(k, hfp, y0, yp, fp);
  R[0] = fp[0] - fm[0];
  R[1] = fp[1] - fm[1];
  R[2] = fp[3] - fm[3];
  R[3] = -(fp[2] - fm[2]) * k.idx + source_f(k, h0, y0, P);
}

// one thread per (cell, column): columns 0..11 are d R_i / d(y_{i-1}, y_i,
// y_{i+1}) by central differences, written into the blocks A, B, C; column
// 12 is dR_i/dP (only the rotational source depends on P), written into r2.
// A column of a neighbour's state changes only that face's fluxes.
__global__ void k_synth_jac(const __grid_constant__ SynthCases scs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= scs.ncells * 13) return;
  const int g = t / 13, col = t - 13 * (t / 13);
  const int cs = scs.cell_case ? scs.cell_case[g] : 0;
  const int i = g - (scs.cell0 ? scs.cell0[cs] : 0);
  const int n = scs.cps ? scs.cps[cs].nx : scs.cp1.nx;
  SynthWork w = synth_work(case_work(scs, cs), n);
  if (w.sc[SC_DONE] != 0.0) return;
  const int blk = col >> 2, v = col & 3;
  float* J = (blk == 0) ? w.A + 16 * i : ((blk == 1) ? w.B + 16 * i : w.C + 16 * i);
  if (i == 0 || i == n - 1) {
    // boundary rows R = y_i - sampled: the identity in B
    if (col < 12)
      for (int r = 0; r < 4; ++r) J[r * 4 + v] = (blk == 1 && r == v) ? 1.f : 0.f;
    else
      for (int r = 0; r < 4; ++r) w.r2[4 * i + r] = 0.f;
    return;
  }
  const SynthKf k{w.kf[KF_DR], w.kf[KF_IDX], w.kf[KF_I3DR], w.kf[KF_MUREF],
                  w.kf[KF_OMEGA], w.kf[KF_KT], w.kf[KF_KR], w.kf[KF_IZ]};
  const float P = w.kf[KF_P];
  float ym[4], y0[4], yp[4];
  for (int q = 0; q < 4; ++q) {
    ym[q] = w.yf[4 * (i - 1) + q];
    y0[q] = w.yf[4 * i + q];
    yp[q] = w.yf[4 * (i + 1) + q];
  }
  const float* hfm = w.hf + 4 * (i - 1);
  const float* hfp = w.hf + 4 * i;
  if (col == 12) {
    const float hP = 1e-3f * fmaxf(fabsf(P), 1.0f);
    const float h2 = (P + hP) - (P - hP);
    const float ds = source_f(k, w.h0[i], y0, P + hP) - source_f(k, w.h0[i], y0, P - hP);
    w.r2[4 * i + 0] = 0.f;
    w.r2[4 * i + 1] = 0.f;
    w.r2[4 * i + 2] = 0.f;
    w.r2[4 * i + 3] = ds / h2;
    return;
  }
  // step ~ sqrt of the FP32 rounding unit
  float* yy = (blk == 0) ? ym : ((blk == 1) ? y0 : yp);
  const float sv = yy[v];
  const float hh = 1e-3f * fmaxf(fabsf(sv), 1.0f);
  const float h2 = (sv + hh) - (sv - hh);  // the step actually taken
  float d[4];
  if (blk == 1) {
    float rp[4], rm[4];
    yy[v] = sv + hh;
    rows_f(k, hfm, hfp, w.h0[i], ym, y0, yp, P, rp);
    yy[v] = sv - hh;
    rows_f(k, hfm, hfp, w.h0[i], ym, y0, yp, P, rm);
    for (int r = 0; r < 4; ++r) d[r] = rp[r] - rm[r];
  } else {
    // the face shared with the perturbed neighbour: R = f(i+1/2) - f(i-1/2)
    // in rows 0..2 and -(q_r(i+1/2) - q_r(i-1/2)) / dx in row 3
    float fp[4], fm[4];
    const float* hfc = (blk == 0) ? hfm : hfp;
    const float* yl = (blk == 0) ? ym : y0;
    const float* yr = (blk == 0) ? y0 : yp;
    yy[v] = sv + hh;
    face_flux_f(k, hfc, yl, yr, fp);
    yy[v] = sv - hh;
    face_flux_f(k, hfc, yl, yr, fm);
    const float sg = (blk == 0) ? -1.f : 1.f;
    d[0] = sg * (fp[0] - fm[0]);
    d[1] = sg * (fp[1] - fm[1]);
    d[2] = sg * (fp[3] - fm[3]);
    d[3] = -sg * (fp[2] - fm[2]) * k.idx;
  }
  for (int r = 0; r < 4; ++r) J[r * 4 + v] = d[r] / h2;
}

__device__ void inv4f(const float* m, float* r) {
  // Gauss-Jordan with partial pivoting on a 4x4 matrix
  float a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      a[i][j] = m[i * 4 + j];
      a[i][4 + j] = (i == j) ? 1.f : 0.f;
    }
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int i = c + 1; i < 4; ++i)
      if (fabsf(a[i][c]) > fabsf(a[piv][c])) piv = i;
    if (piv != c)
      for (int j = 0; j < 8; ++j) {
        const float t = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = t;
      }
    const float dinv = 1.f / a[c][c];
    for (int j = 0; j < 8; ++j) a[c][j] *= dinv;
    for (int i = 0; i < 4; ++i)
      if (i != c) {
        const float fct = a[i][c];
        for (int j = 0; j < 8; ++j) a[i][j] = __fmaf_rn(-fct, a[c][j], a[i][j]);
      }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r[i * 4 + j] = a[i][4 + j];
}

__device__ __forceinline__ void mm4f(const float* a, const float* b, float* c) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      float s = 0.f;
      for (int k = 0; k < 4; ++k) s = __fmaf_rn(a[i * 4 + k], b[k * 4 + j], s);
      c[i * 4 + j] = s;
    }
}

__device__ __forceinline__ void mv4f(const float* a, const float* x, float* y) {
  for (int i = 0; i < 4; ++i) {
    float s = 0.f;
    for (int k = 0; k < 4; ++k) s = __fmaf_rn(a[i * 4 + k], x[k], s);
    y[i] = s;
  }
}

// Newton update: block cyclic reduction (FP32) of J z1 = -R, J z2 = G; the
// bordered mass row in FP64; a damped update that keeps rho, T positive.
// count_done: add 1 to the finished-slab count (info[3 ncases]) for every
// slab that is finished after this launch
template <int NT>
__global__ void __launch_bounds__(NT) k_synth_solve(const __grid_constant__ SynthCases scs, int n_m, double tol,
                                                    int count_done) {
  __shared__ double red[NT];
  const int cs = blockIdx.x;
  const SynthArgs a = case_args(scs, cs);
  const int n = a.cp.nx;
  SynthWork w = synth_work(case_work(scs, cs), n);
  if (w.sc[SC_DONE] != 0.0) {
    if (count_done && threadIdx.x == 0) atomicAdd(scs.info + 3 * scs.ncases, 1.0);
    return;
  }
  const int tid = threadIdx.x, nt = NT;
  const double P = w.sc[SC_P];
  residual_fp64<NT>(a, w, n, P);
  for (int i = tid; i < n; i += nt)
    for (int v = 0; v < 4; ++v) w.r1[4 * i + v] = (float)(-w.R[4 * i + v]);
  __syncthreads();
  // forward reduction: at stride s the rows i = 2s-1 (mod 2s) eliminate their
  // neighbours i -/+ s, which keep their equations for back substitution
  int s = 1;
  for (; 2 * s - 1 < n; s *= 2) {
    for (int j = s - 1 + tid * 2 * s; j < n; j += nt * 2 * s) inv4f(w.B + 16 * j, w.Bi + 16 * j);
    __syncthreads();
    for (int i = 2 * s - 1 + tid * 2 * s; i < n; i += nt * 2 * s) {
      const int lo = i - s, hi = i + s;
      float al[16], ga[16], t1[16], t2[16];
      mm4f(w.A + 16 * i, w.Bi + 16 * lo, al);
      for (int q = 0; q < 16; ++q) al[q] = -al[q];
      float Bn[16], An[16], Cn[16], x1[4], x2[4], v1[4], v2[4];
      mm4f(al, w.A + 16 * lo, An);
      mm4f(al, w.C + 16 * lo, t1);
      for (int q = 0; q < 16; ++q) Bn[q] = w.B[16 * i + q] + t1[q];
      mv4f(al, w.r1 + 4 * lo, v1);
      mv4f(al, w.r2 + 4 * lo, v2);
      for (int v = 0; v < 4; ++v) {
        x1[v] = w.r1[4 * i + v] + v1[v];
        x2[v] = w.r2[4 * i + v] + v2[v];
      }
      if (hi < n) {
        mm4f(w.C + 16 * i, w.Bi + 16 * hi, ga);
        for (int q = 0; q < 16; ++q) ga[q] = -ga[q];
        mm4f(ga, w.C + 16 * hi, Cn);
        mm4f(ga, w.A + 16 * hi, t2);
        for (int q = 0; q < 16; ++q) Bn[q] += t2[q];
        mv4f(ga, w.r1 + 4 * hi, v1);
        mv4f(ga, w.r2 + 4 * hi, v2);
        for (int v = 0; v < 4; ++v) {
          x1[v] += v1[v];
          x2[v] += v2[v];
        }
      } else {
        for (int q = 0; q < 16; ++q) Cn[q] = 0.f;
      }
      for (int q = 0; q < 16; ++q) {
        w.A[16 * i + q] = An[q];
        w.B[16 * i + q] = Bn[q];
        w.C[16 * i + q] = Cn[q];
      }
      for (int v = 0; v < 4; ++v) {
        w.r1[4 * i + v] = x1[v];
        w.r2[4 * i + v] = x2[v];
      }
    }
    __syncthreads();
  }
  // the last remaining row (index s-1) is solved directly; z lives in r1, r2
  if (tid == 0) {
    const int i = s - 1;
    float x1[4], x2[4];
    inv4f(w.B + 16 * i, w.Bi + 16 * i);
    mv4f(w.Bi + 16 * i, w.r1 + 4 * i, x1);
    mv4f(w.Bi + 16 * i, w.r2 + 4 * i, x2);
    for (int v = 0; v < 4; ++v) {
      w.r1[4 * i + v] = x1[v];
      w.r2[4 * i + v] = x2[v];
    }
  }
  __syncthreads();
  for (s /= 2; s >= 1; s /= 2) {
    for (int j = s - 1 + tid * 2 * s; j < n; j += nt * 2 * s) {
      float t1[4], t2[4], c1[4], c2[4];
      for (int v = 0; v < 4; ++v) {
        t1[v] = w.r1[4 * j + v];
        t2[v] = w.r2[4 * j + v];
      }
      if (j - s >= 0) {
        mv4f(w.A + 16 * j, w.r1 + 4 * (j - s), c1);
        mv4f(w.A + 16 * j, w.r2 + 4 * (j - s), c2);
        for (int v = 0; v < 4; ++v) {
          t1[v] -= c1[v];
          t2[v] -= c2[v];
        }
      }
      if (j + s < n) {
        mv4f(w.C + 16 * j, w.r1 + 4 * (j + s), c1);
        mv4f(w.C + 16 * j, w.r2 + 4 * (j + s), c2);
        for (int v = 0; v < 4; ++v) {
          t1[v] -= c1[v];
          t2[v] -= c2[v];
        }
      }
      mv4f(w.Bi + 16 * j, t1, c1);
      mv4f(w.Bi + 16 * j, t2, c2);
      for (int v = 0; v < 4; ++v) {
        w.r1[4 * j + v] = c1[v];
        w.r2[4 * j + v] = c2[v];
      }
    }
    __syncthreads();
  }
  // bordered correction in FP64: [J G; h^T d] [dy; dP] = [-R; -(mass - M)],
  // h the derivative of the mass sum dx (P - H_i) / T_t,i by T_t,i
  double mass = 0.0, dP = 0.0, hz1 = 0.0, hz2 = 0.0;
  for (int i = tid; i < n; i += nt) {
    const double Hi = a.hot[(size_t)i * 12];
    const double tt = w.y[4 * i + 2];
    const double itt = 1.0 / tt;
    mass += (P - Hi) / tt * a.cp.dx;
    dP += a.cp.dx * itt;
    const double hi = -a.cp.dx * (P - Hi) * itt * itt;
    hz1 += hi * (double)w.r1[4 * i + 2];
    hz2 += hi * (double)w.r2[4 * i + 2];
  }
  mass = block_sum<NT>(mass, red);
  dP = block_sum<NT>(dP, red);
  hz1 = block_sum<NT>(hz1, red);
  hz2 = block_sum<NT>(hz2, red);
  const double RP = mass - w.sc[SC_M];
  const double dPstep = (-RP - hz1) / (dP - hz2);
  double lam = 1.0;
  int ok = 0;
  for (int tries = 0; tries < 40; ++tries) {
    const double Pn = P + lam * dPstep;
    int bad = 0;
    for (int i = tid; i < n; i += nt) {
      for (int v = 0; v < 4; ++v)
        w.yn[4 * i + v] = w.y[4 * i + v] + lam * ((double)w.r1[4 * i + v] - (double)w.r2[4 * i + v] * dPstep);
      const double rho = (Pn - a.hot[(size_t)i * 12]) / w.yn[4 * i + 2];
      if (!(w.yn[4 * i + 2] > 0.0) || !(w.yn[4 * i + 3] > 0.0) || !(rho > 0.0)) bad = 1;
    }
    ok = !__syncthreads_or(bad);
    if (ok) break;
    lam *= 0.5;
  }
  double dmax = 0.0;
  if (ok) {
    for (int i = tid; i < n; i += nt)
      for (int v = 0; v < 4; ++v) {
        dmax = fmax(dmax, fabs(w.yn[4 * i + v] - w.y[4 * i + v]) / fmax(fabs(w.y[4 * i + v]), 1e-3));
        w.y[4 * i + v] = w.yn[4 * i + v];
        w.yf[4 * i + v] = (float)w.yn[4 * i + v];
      }
  }
  dmax = block_max<NT>(dmax, red);
  if (tid == 0) {
    const double it = w.sc[SC_IT] + 1.0;
    w.sc[SC_IT] = it;
    if (!ok) {
      w.sc[SC_STATUS] = 2.0;
      w.sc[SC_DONE] = 1.0;
    } else {
      const double Pn = P + lam * dPstep;
      dmax = fmax(dmax, fabs(Pn - P) / fmax(fabs(P), 1e-3));
      w.sc[SC_P] = Pn;
      w.kf[KF_P] = (float)Pn;
      w.sc[SC_DMAX] = dmax;
      if (dmax < tol) {
        w.sc[SC_STATUS] = 0.0;
        w.sc[SC_DONE] = 1.0;
      } else if (it >= n_m) {
        w.sc[SC_DONE] = 1.0;
      }
    }
    if (count_done && w.sc[SC_DONE] != 0.0) atomicAdd(scs.info + 3 * scs.ncases, 1.0);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_synth_final(const __grid_constant__ SynthCases scs, double* out_all) {
  __shared__ double red[NT];
  __shared__ double s_status;
  const int cs = blockIdx.x;
  const SynthArgs a = case_args(scs, cs);
  const int n = a.cp.nx;
  SynthWork w = synth_work(case_work(scs, cs), n);
  double* out = out_all + (size_t)(scs.cell0 ? scs.cell0[cs] : 0) * 6;
  double* info = scs.info + 3 * cs;
  const double P = w.sc[SC_P];
  // an iterate is used (converged, or at the iteration cap) only if it is
  // finite and positive and keeps the sampled mass (the mass condition is
  // not linear in the unknowns, so an unconverged iterate may break it);
  // otherwise the slab keeps its sampled fields
  residual_fp64<NT>(a, w, n, P);
  double rmax = 0.0, msol = 0.0, msmp = 0.0, bad = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    const double* y0 = w.y + 4 * i;
    for (int v = 0; v < 4; ++v) rmax = fmax(rmax, fabs(w.R[4 * i + v]));
    const double rho = (P - a.hot[(size_t)i * 12]) / y0[2];
    if (!(rho > 0.0) || !(y0[2] > 0.0) || !(y0[3] > 0.0) || !isfinite(rho) || !isfinite(y0[0]) || !isfinite(y0[1]))
      bad = 1.0;
    msol += rho;
    msmp += a.F[(size_t)i * 18];
  }
  rmax = block_max<NT>(rmax, red);
  bad = block_max<NT>(bad, red);
  msol = block_sum<NT>(msol, red);
  msmp = block_sum<NT>(msmp, red);
  if (threadIdx.x == 0) {
    double st = w.sc[SC_STATUS];  // 0 converged, 1 iteration cap, 2 numeric
    if (st != 2.0 && (bad > 0.0 || !(fabs(msol - msmp) <= 1e-6 * msmp))) st = 2.0;
    s_status = st;
  }
  __syncthreads();
  const bool keep = s_status == 2.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    double* o = out + (size_t)i * 6;
    if (keep) {
      const double* f = a.F + (size_t)i * 18;
      for (int v = 0; v < 6; ++v) o[v] = f[v];
    } else {
      const double* y0 = w.y + 4 * i;
      o[0] = (P - a.hot[(size_t)i * 12]) / y0[2];
      o[1] = 0.0;
      o[2] = y0[0];
      o[3] = y0[1];
      o[4] = y0[2];
      o[5] = y0[3];
    }
  }
  if (threadIdx.x == 0) {
    info[0] = w.sc[SC_IT];
    info[1] = rmax;
    info[2] = s_status;
  }
}

// Newton iterations are launched in batches of 4 (a finished slab makes the
// remaining launches return at once); the host reads the count of finished
// slabs between batches.  One CTA per slab, NT threads: the smallest power
// of two from 128 to 1024 that covers the largest slab.  The first CUDA
// error (a launch, the copy of the count or the wait) stops the loop before
// any further launch and is returned.
template <int NT>
static cudaError_t run_synth_nt(const SynthCases& sc, double* out, int n_m, double tol, cudaStream_t st) {
  k_synth_init<NT><<<sc.ncases, NT, 0, st>>>(sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int jt = 128, jb = (sc.ncells * 13 + jt - 1) / jt;
  int it = 0;
  while (it < n_m) {
    const int batch = (n_m - it) < 4 ? (n_m - it) : 4;
    e = cudaMemsetAsync(sc.info + 3 * sc.ncases, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    for (int b = 0; b < batch; ++b) {
      k_synth_jac<<<jb, jt, 0, st>>>(sc);
      k_synth_solve<NT><<<sc.ncases, NT, 0, st>>>(sc, n_m, tol, b == batch - 1 ? 1 : 0);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    it += batch;
    double done = 0.0;
    e = cudaMemcpyAsync(&done, sc.info + 3 * sc.ncases, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (done >= (double)sc.ncases) break;
  }
  k_synth_final<NT><<<sc.ncases, NT, 0, st>>>(sc, out);
  return cudaGetLastError();
}

static cudaError_t run_synth(const SynthCases& sc, const int32_t* host_nx, double* out, int n_m, double tol,
                             cudaStream_t st) {
  int nmax = 1;
  for (int c = 0; c < sc.ncases; ++c) nmax = host_nx[c] > nmax ? host_nx[c] : nmax;
  if (nmax <= 128) return run_synth_nt<128>(sc, out, n_m, tol, st);
  if (nmax <= 256) return run_synth_nt<256>(sc, out, n_m, tol, st);
  if (nmax <= 512) return run_synth_nt<512>(sc, out, n_m, tol, st);
  return run_synth_nt<1024>(sc, out, n_m, tol, st);
}

cudaError_t launch_synth1d(const CellParams* cp, const int32_t* cell_case, const int32_t* cell0, int ncases,
                           int ncells, const int32_t* host_nx, const double* fields, const double* hot, double* out,
                           double* work, const int64_t* woff, int n_m, double tol, double* info, cudaStream_t st) {
  SynthCases sc{};
  sc.cps = cp;
  sc.cell_case = cell_case;
  sc.cell0 = cell0;
  sc.woff = woff;
  sc.F = fields;
  sc.hot = hot;
  sc.work = work;
  sc.info = info;
  sc.ncases = ncases;
  sc.ncells = ncells;
  return run_synth(sc, host_nx, out, n_m, tol, st);
}

// one slab given by value (no device tables): used where nothing may be
// allocated
cudaError_t launch_synth1d_single(const CellParams& cp, const double* fields, const double* hot, double* out,
                                  double* work, int n_m, double tol, double* info, cudaStream_t st) {
  SynthCases sc{};
  sc.cp1 = cp;
  sc.F = fields;
  sc.hot = hot;
  sc.work = work;
  sc.info = info;
  sc.ncases = 1;
  sc.ncells = cp.nx;
  return run_synth(sc, &cp.nx, out, n_m, tol, st);
}

}  // namespace dsmc
