// dsmc_synth2d.cu -- the steady 2D synthetic equations of the DIG method
// (Sec. 3 step 3) on the GPU: Newton's method with the residual and a
// central-difference Jacobian in FP64 (dsmc_synth2d.cuh), and a direct
// banded LU factorisation with partial pivoting for each Newton step.
//
// The total-mass row (cell (1, 0)'s mass balance replaced by the total mass)
// couples every cell; the factorised matrix B has e_r / n there instead, and
// the Newton step of J = B + e_r w^T (w = 1/n on the density of every other
// cell) follows from two solves with B (Sherman-Morrison).
//
// The factorisation runs one launch per pivot column k: CTA b updates column
// k + 1 + b (interchange and elimination with the multipliers of column k),
// and CTA 0, which owns column k + 1, then finds that column's pivot and
// multipliers for the next launch.  The launches on one stream order the
// steps; within a launch no two CTAs touch one column.
#include <climits>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "dsmc_internal.h"
#include "dsmc_synth2d.cuh"

namespace dsmc {

namespace {

// scalar slots of the work area
enum {
  S2_SUMD = 0,   // sampled total density (sum over cells)
  S2_MASS = 1,   // total-mass residual (sum rho - sampled sum) / n
  S2_DONE = 2,
  S2_IT = 3,
  S2_STATUS = 4, // 0 converged, 1 not (yet) converged, 2 numeric
  S2_DMAX = 5,
  S2_SING = 6,   // a zero pivot was met
  S2_RMAX = 7,
  S2_LAM = 8,
  S2_NSC = 16
};

struct S2Work {
  double *x, *R, *d, *b0, *b1, *y0, *y1, *z, *yv, *ud, *sc, *AB, *Lm;
  int32_t* piv;
};

inline size_t round32(size_t n) { return (n + 31) & ~(size_t)31; }  // 256-byte multiples

inline size_t s2_doubles(const s2::Grid& g) {
  const size_t N = (size_t)g.N;
  const size_t vec = (N + 31) & ~(size_t)31;
  return 10 * vec + 32 + (((size_t)g.ld * N + 31) & ~(size_t)31) + (((size_t)g.kl * N + 31) & ~(size_t)31) +
         ((N / 2 + 1 + 31) & ~(size_t)31);
}

S2Work s2_carve(const s2::Grid& g, double* w) {
  const size_t vec = round32((size_t)g.N);
  S2Work s;
  double* p = w;
  s.x = p; p += vec;
  s.R = p; p += vec;
  s.d = p; p += vec;
  s.b0 = p; p += vec;
  s.b1 = p; p += vec;
  s.y0 = p; p += vec;
  s.y1 = p; p += vec;
  s.z = p; p += vec;
  s.yv = p; p += vec;
  s.ud = p; p += vec;
  s.sc = p; p += 32;
  s.AB = p; p += round32((size_t)g.ld * g.N);
  s.Lm = p; p += round32((size_t)g.kl * g.N);
  s.piv = reinterpret_cast<int32_t*>(p);
  return s;
}

template <int NT>
__device__ double s2_block_sum(double v, double* red) {
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
__device__ double s2_block_max(double v, double* red) {
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

// First row of largest |A(r, k)|, r = k .. min(k + kl, N - 1), as
// s2::pivot_seq; rows whose magnitude is not a number never win, and a
// column without any number pivots on its diagonal.
template <int NT>
__device__ int s2_block_argmax(const s2::Grid& g, const double* AB, int k, double* sv, int* si) {
  const int tid = threadIdx.x;
  double best = -1.0;
  int bi = INT_MAX;
  const int rmax = s2::last_row(g, k);
  for (int r = k + tid; r <= rmax; r += NT) {
    const double a = fabs(AB[s2::band_at(g, r, k)]);
    if (a > best) {
      best = a;
      bi = r;
    }
  }
  sv[tid] = best;
  si[tid] = bi;
  __syncthreads();
#pragma unroll
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (tid < o) {
      const double v2 = sv[tid + o];
      const int i2 = si[tid + o];
      if (v2 > sv[tid] || (v2 == sv[tid] && i2 < si[tid])) {
        sv[tid] = v2;
        si[tid] = i2;
      }
    }
    __syncthreads();
  }
  const int p = si[0];
  __syncthreads();
  return p == INT_MAX ? k : p;
}

constexpr int S2_NT = 256;    // single-CTA kernels
constexpr int S2_STEP_NT = 128;
constexpr int S2_SOLVE_NT = 512;

__global__ void __launch_bounds__(S2_NT) k_s2_init(const s2::Grid g, S2Work w) {
  __shared__ double red[S2_NT];
  double s = 0.0;
  for (int b = threadIdx.x; b < g.n; b += S2_NT) {
    int i, j;
    s2::cell_of_band(g, b, i, j);
    const double* D = g.F + (size_t)(j * g.nx + i) * 18;
    double* x = w.x + s2::NV * b;
    x[0] = D[0];
    x[1] = D[1];
    x[2] = D[2];
    x[3] = D[4];
    x[4] = D[5];
  }
  for (int c = threadIdx.x; c < g.n; c += S2_NT) s += g.F[(size_t)c * 18];
  s = s2_block_sum<S2_NT>(s, red);
  if (threadIdx.x == 0) {
    w.sc[S2_SUMD] = s;
    w.sc[S2_DONE] = 0.0;
    w.sc[S2_IT] = 0.0;
    w.sc[S2_STATUS] = 1.0;
    w.sc[S2_DMAX] = 0.0;
    w.sc[S2_SING] = 0.0;
    w.sc[S2_RMAX] = 0.0;
    w.sc[S2_LAM] = 0.0;
  }
}

// total-mass residual of the current state
__global__ void __launch_bounds__(S2_NT) k_s2_mass(const s2::Grid g, S2Work w) {
  __shared__ double red[S2_NT];
  double s = 0.0;
  for (int b = threadIdx.x; b < g.n; b += S2_NT) s += w.x[s2::NV * b];
  s = s2_block_sum<S2_NT>(s, red);
  if (threadIdx.x == 0) w.sc[S2_MASS] = (s - w.sc[S2_SUMD]) / g.n;
}

__global__ void k_s2_res(const s2::Grid g, S2Work w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.n) return;
  int i, j;
  s2::cell_of_band(g, b, i, j);
  const s2::View X{w.x, -1, 0, 0.0};
  s2::cell_residual(g, X, i, j, w.sc[S2_MASS], w.R + s2::NV * b);
}

__global__ void k_s2_jac(const s2::Grid g, S2Work w) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    const int mr = s2::mass_row(g);
    w.AB[s2::band_at(g, mr, mr)] = 1.0 / g.n;
  }
  if (t >= g.n * s2::NSTENCIL * s2::NV) return;
  const int b = t / (s2::NSTENCIL * s2::NV);
  const int rem = t - b * (s2::NSTENCIL * s2::NV);
  s2::jacobian_entries(g, w.x, b, rem / s2::NV, rem % s2::NV, w.AB);
}

// pivot and multipliers of column 0
__global__ void __launch_bounds__(S2_STEP_NT) k_s2_piv0(const s2::Grid g, S2Work w) {
  __shared__ double sv[S2_STEP_NT];
  __shared__ int si[S2_STEP_NT];
  const int p = s2_block_argmax<S2_STEP_NT>(g, w.AB, 0, sv, si);
  const int sing = s2::pivot_write(g, w.AB, w.Lm, w.piv, w.ud, 0, p, threadIdx.x, S2_STEP_NT);
  if (sing && threadIdx.x == 0) w.sc[S2_SING] = 1.0;
}

// elimination step k on columns k+1 .. last_col(k) (one CTA each); CTA 0 then
// pivots column k + 1
__global__ void __launch_bounds__(S2_STEP_NT) k_s2_step(const s2::Grid g, S2Work w, int k) {
  __shared__ double sv[S2_STEP_NT];
  __shared__ int si[S2_STEP_NT];
  const int c = k + 1 + blockIdx.x;
  if (c > s2::last_col(g, k)) return;
  const s2::ColHead h = s2::col_head(g, w.AB, w.piv, k, c);
  __syncthreads();
  s2::lu_column(g, w.AB, w.Lm, w.piv, k, c, h, threadIdx.x, S2_STEP_NT);
  if (blockIdx.x != 0) return;
  __syncthreads();
  const int p = s2_block_argmax<S2_STEP_NT>(g, w.AB, k + 1, sv, si);
  const int sing = s2::pivot_write(g, w.AB, w.Lm, w.piv, w.ud, k + 1, p, threadIdx.x, S2_STEP_NT);
  if (sing && threadIdx.x == 0) w.sc[S2_SING] = 1.0;
}

// Solves with the factors (right-hand sides -R and e_r), the rank-one
// correction for the total-mass row, the damped update that keeps rho, T_t,
// T_r positive and finite (step halved up to 60 times), and the convergence
// test on the largest relative update (|lam dx| / max(|x|, 1e-3) < tol).
__global__ void __launch_bounds__(S2_SOLVE_NT) k_s2_solve(const s2::Grid g, S2Work w, int n_m, double tol) {
  __shared__ double red[S2_SOLVE_NT];
  const int tid = threadIdx.x;
  const int N = g.N;
  const int mr = s2::mass_row(g);
  for (int u = tid; u < N; u += S2_SOLVE_NT) {
    w.b0[u] = -w.R[u];
    w.b1[u] = u == mr ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    const s2::FwdHead h = s2::fwd_head(w.piv, k, w.b0, w.b1);
    __syncthreads();
    s2::fwd_step(g, w.Lm, w.piv, k, h, w.b0, w.b1, w.y0, w.y1, tid, S2_SOLVE_NT);
    __syncthreads();
  }
  for (int k = N - 1; k >= 0; --k) {
    s2::back_step(g, w.AB, w.ud, k, w.y0, w.y1, w.z, w.yv, tid, S2_SOLVE_NT);
    __syncthreads();
  }
  double wz = 0.0, wy = 0.0;
  for (int b = tid; b < g.n; b += S2_SOLVE_NT) {
    if (s2::NV * b == mr) continue;
    wz += w.z[s2::NV * b];
    wy += w.yv[s2::NV * b];
  }
  wz = s2_block_sum<S2_SOLVE_NT>(wz, red) / g.n;
  wy = s2_block_sum<S2_SOLVE_NT>(wy, red) / g.n;
  const double f = wz / (1.0 + wy);
  for (int u = tid; u < N; u += S2_SOLVE_NT) w.d[u] = w.z[u] - w.yv[u] * f;
  __syncthreads();
  double lam = 1.0;
  bool ok = false;
  for (int hv = 0; hv < 60 && !ok; ++hv) {
    double bad = 0.0;
    for (int u = tid; u < N; u += S2_SOLVE_NT) {
      const double xn = w.x[u] + lam * w.d[u];
      const int v = u % s2::NV;
      if (!isfinite(xn) || ((v == 0 || v >= 3) && xn <= 0.0)) bad = 1.0;
    }
    ok = s2_block_max<S2_SOLVE_NT>(bad, red) == 0.0;
    if (!ok) lam *= 0.5;
  }
  if (!ok) {
    if (tid == 0) {
      w.sc[S2_STATUS] = 2.0;
      w.sc[S2_DONE] = 1.0;
    }
    return;
  }
  double dm = 0.0;
  for (int u = tid; u < N; u += S2_SOLVE_NT) {
    const double x = w.x[u];
    const double step = lam * w.d[u];
    dm = fmax(dm, fabs(step) / fmax(fabs(x), 1e-3));
    w.x[u] = x + step;
  }
  dm = s2_block_max<S2_SOLVE_NT>(dm, red);
  if (tid == 0) {
    const double it = w.sc[S2_IT] + 1.0;
    w.sc[S2_IT] = it;
    w.sc[S2_DMAX] = dm;
    w.sc[S2_LAM] = lam;
    if (dm < tol) {
      w.sc[S2_STATUS] = 0.0;
      w.sc[S2_DONE] = 1.0;
    } else if (it >= n_m) {
      w.sc[S2_DONE] = 1.0;
    }
  }
}

// outputs (natural cell order, rho, u_x, u_y, sampled u_z, T_t, T_r; the
// sampled fields for a numeric failure) and (iterations, max |R|, status)
__global__ void __launch_bounds__(S2_NT) k_s2_final(const s2::Grid g, S2Work w, double* out, double* info) {
  __shared__ double red[S2_NT];
  const int status = (int)w.sc[S2_STATUS];
  double rm = 0.0;
  for (int u = threadIdx.x; u < g.N; u += S2_NT) rm = fmax(rm, fabs(w.R[u]));
  rm = s2_block_max<S2_NT>(rm, red);
  for (int b = threadIdx.x; b < g.n; b += S2_NT) {
    int i, j;
    s2::cell_of_band(g, b, i, j);
    const size_t c = (size_t)j * g.nx + i;
    const double* D = g.F + c * 18;
    const double* x = w.x + s2::NV * b;
    double* o = out + c * 6;
    if (status == 2) {
      o[0] = D[0];
      o[1] = D[1];
      o[2] = D[2];
      o[4] = D[4];
      o[5] = D[5];
    } else {
      o[0] = x[0];
      o[1] = x[1];
      o[2] = x[2];
      o[4] = x[3];
      o[5] = x[4];
    }
    o[3] = D[3];
  }
  if (threadIdx.x == 0) {
    info[0] = w.sc[S2_IT];
    info[1] = rm;
    info[2] = status;
  }
}

}  // namespace

size_t synth2d_work_doubles(int nx, int ny) {
  const s2::Grid g = s2::make_grid(nx, ny, 1.0, 1.0, 2.0, 0.75, 1.0, 1.0, 1.0, 1.0, nullptr, nullptr);
  return s2_doubles(g);
}

int launch_synth2d(const CellParams& cp, const double* fields, const double* hot, double* out, double* work,
                   int n_m, double tol, double* info, int* singular, cudaStream_t st) {
  const s2::Grid g = s2::make_grid(cp.nx, cp.ny, cp.dx, cp.dy, cp.d_r, cp.omega, cp.mu_ref, cp.z_rot, cp.kappa_t,
                                   cp.kappa_r, fields, hot);
  const S2Work w = s2_carve(g, work);
  const int nb = 256;
  const int res_grid = (g.n + nb - 1) / nb;
  const long long jac_threads = (long long)g.n * s2::NSTENCIL * s2::NV;
  const int jac_grid = (int)((jac_threads + nb - 1) / nb);
  double sc[S2_NSC];
  k_s2_init<<<1, S2_NT, 0, st>>>(g, w);
  for (int it = 0; it < n_m; ++it) {
    k_s2_mass<<<1, S2_NT, 0, st>>>(g, w);
    k_s2_res<<<res_grid, nb, 0, st>>>(g, w);
    cudaMemsetAsync(w.AB, 0, sizeof(double) * (size_t)g.ld * g.N, st);
    k_s2_jac<<<jac_grid, nb, 0, st>>>(g, w);
    k_s2_piv0<<<1, S2_STEP_NT, 0, st>>>(g, w);
    for (int k = 0; k < g.N - 1; ++k) k_s2_step<<<s2::last_col(g, k) - k, S2_STEP_NT, 0, st>>>(g, w, k);
    k_s2_solve<<<1, S2_SOLVE_NT, 0, st>>>(g, w, n_m, tol);
    cudaMemcpyAsync(sc, w.sc, sizeof(double) * 9, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    if (sc[S2_DONE] != 0.0) break;
  }
  k_s2_mass<<<1, S2_NT, 0, st>>>(g, w);
  k_s2_res<<<res_grid, nb, 0, st>>>(g, w);
  k_s2_final<<<1, S2_NT, 0, st>>>(g, w, out, info);
  cudaMemcpyAsync(sc, w.sc, sizeof(double) * 9, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  if (singular) *singular = sc[S2_SING] != 0.0;
  return 0;
}

}  // namespace dsmc
