// dsmc_synth2d.cu -- the steady 2D synthetic equations of the DIG method
// (Sec. 3 step 3) on the GPU: Newton's method with the residual and a
// central-difference Jacobian in FP64 (dsmc_synth2d.cuh); each Newton step
// solves with a blocked banded LU factorisation (partial pivoting) of the
// Jacobian in FP32, substitutions in FP32 and iterative refinement with FP64
// residuals; later Newton steps reuse the factorisation while the updates
// keep shrinking.
//
// The total-mass row (cell (1, 0)'s mass balance replaced by the total mass)
// couples every cell; the factorised matrix B has e_r / n there instead, and
// the Newton step of J = B + e_r w^T (w = mass_scale / n on the density of
// every other cell) follows from two solves with B (Sherman-Morrison).
//
// Factorisation: per panel of nb columns, one CTA factorises the panel in
// shared memory, then one launch applies it to the up to kl + ku trailing
// columns, up to 16 columns per CTA.  Substitution: a cluster of 8 CTAs walks the
// panels, forward then backward, one cluster barrier per panel
// (k_s2_subst_cl; one CTA, k_s2_subst, where no cluster fits).  The launches
// on one stream order the factorisation's panels.
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
  S2_SUMD = 0,   // sampled total density (sum over cells, weighted by mass_scale)
  S2_MASS = 1,   // total-mass residual (weighted sum rho - sampled sum) / n
  S2_DONE = 2,
  S2_IT = 3,
  S2_STATUS = 4, // 0 converged, 1 not (yet) converged, 2 numeric
  S2_DMAX = 5,
  S2_SING = 6,   // a zero pivot was met
  S2_LAM = 7,    // length of the last Newton update (1 = full step)
  S2_NSC = 16
};

constexpr int S2_NT = 256;        // threads of the factorisation and substitution kernels
constexpr int S2_UPD_NT = 512;    // the Newton update
constexpr int S2_SUB_NT = 512;    // the substitutions
constexpr int S2_PNL_NT = 512;    // the panel factorisation
constexpr int S2_NREF = 1;        // refinement sweeps after a fresh factorisation
constexpr int S2_NREF_REUSE = 3;  // refinement sweeps when an earlier factorisation is reused
constexpr int S2_SMEM_CAP = 200 * 1024;

// Panel width nb and trailing columns per CTA cb (4: enough CTAs to fill the
// GPU for the kl + ku trailing columns): the largest nb of 32, 16, 8 whose
// panel and nb + cb trailing columns (H = kl + nb rows, FP32) fit the
// shared-memory budget.
struct S2Blocking {
  int nb, cb;
};

inline S2Blocking s2_blocking(const s2::Grid& g) {
  for (int nb = 32; nb >= 8; nb /= 2) {
    const long long col = 4LL * (g.kl + nb);
    const long long cb = S2_SMEM_CAP / col - nb;
    if (cb >= 4 || (nb == 8 && cb >= 1)) return {nb, cb >= 4 ? 4 : (int)cb};
  }
  return {0, 0};
}

struct S2Work {
  double *x, *R, *d, *rhs0, *rhs1, *b0, *b1, *y0, *y1, *v0, *v1, *s0, *s1, *sc, *Jc;
  float *AB, *Lp, *ud;
  int32_t* piv;
  float* q;  // 4 FP32 vectors of N: the clustered substitution's ping-pong right-hand sides
  int nb, cb;
};

inline size_t round32(size_t n) { return (n + 31) & ~(size_t)31; }  // 256-byte multiples

inline size_t s2_lp_floats(const s2::Grid& g, int nb) { return (size_t)((g.N + nb - 1) / nb) * nb * (g.kl + nb); }

inline size_t s2_doubles(const s2::Grid& g) {
  const S2Blocking bl = s2_blocking(g);
  const size_t N = (size_t)g.N;
  const size_t vec = round32(N);
  const size_t jc = round32((size_t)g.n * s2::NSTENCIL * s2::NV * s2::NV);
  const size_t f32 = (size_t)g.ld * N + s2_lp_floats(g, bl.nb) + N + N + 4 * N;  // AB, Lp, ud, piv, q
  return 13 * vec + 32 + jc + round32((f32 + 1) / 2) + 32;
}

S2Work s2_carve(const s2::Grid& g, double* w) {
  const S2Blocking bl = s2_blocking(g);
  const size_t vec = round32((size_t)g.N);
  S2Work s;
  double* p = w;
  double** vecs[13] = {&s.x, &s.R, &s.d, &s.rhs0, &s.rhs1, &s.b0, &s.b1, &s.y0, &s.y1, &s.v0, &s.v1, &s.s0, &s.s1};
  for (double** v : vecs) {
    *v = p;
    p += vec;
  }
  s.sc = p;
  p += 32;
  s.Jc = p;
  p += round32((size_t)g.n * s2::NSTENCIL * s2::NV * s2::NV);
  float* f = reinterpret_cast<float*>(p);
  s.AB = f;
  f += (size_t)g.ld * g.N;
  s.Lp = f;
  f += s2_lp_floats(g, bl.nb);
  s.ud = f;
  f += g.N;
  s.piv = reinterpret_cast<int32_t*>(f);
  f += g.N;
  s.q = f;
  s.nb = bl.nb;
  s.cb = bl.cb;
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

extern __shared__ __align__(16) unsigned char s2_smem[];

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
  for (int c = threadIdx.x; c < g.n; c += S2_NT) s += g.F[(size_t)c * 18] * s2::mass_scale(g, c % g.nx, c / g.nx);
  s = s2_block_sum<S2_NT>(s, red);
  if (threadIdx.x == 0) {
    w.sc[S2_SUMD] = s;
    w.sc[S2_DONE] = 0.0;
    w.sc[S2_IT] = 0.0;
    w.sc[S2_STATUS] = 1.0;
    w.sc[S2_DMAX] = 0.0;
    w.sc[S2_SING] = 0.0;
    w.sc[S2_LAM] = 0.0;
  }
}

// total-mass residual of the current state
__global__ void __launch_bounds__(S2_NT) k_s2_mass(const s2::Grid g, S2Work w) {
  __shared__ double red[S2_NT];
  double s = 0.0;
  for (int b = threadIdx.x; b < g.n; b += S2_NT) {
    int i, j;
    s2::cell_of_band(g, b, i, j);
    s += w.x[s2::NV * b] * s2::mass_scale(g, i, j);
  }
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

// the Jacobian: compact FP64 blocks always, the FP32 band only when it is
// to be factorised
__global__ void k_s2_jac(const s2::Grid g, S2Work w, int band) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (band && t == 0) {
    const int mr = s2::mass_row(g);  // none on the annulus
    if (mr >= 0) w.AB[s2::band_at(g, mr, mr)] = (float)(s2::mass_scale(g, 1, 0) / g.n);
  }
  if (t >= g.n * s2::NSTENCIL * s2::NV) return;
  const int b = t / (s2::NSTENCIL * s2::NV);
  const int rem = t - b * (s2::NSTENCIL * s2::NV);
  s2::jacobian_entries(g, w.x, b, rem / s2::NV, rem % s2::NV, band ? w.AB : nullptr, w.Jc);
}

__device__ __forceinline__ void s2_cp_async4(float* sdst, const float* gsrc, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gsrc), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void s2_cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Block-wide first row of largest magnitude from each thread's candidate
// (best, bi): warps reduce by shuffles and write one candidate each into
// buffer buf; after one barrier every warp reduces those candidates itself
// (the same order, so the same answer everywhere).  Magnitudes that are not
// numbers never win; no candidate gives row `fallback` with magnitude -1.
__device__ __forceinline__ int s2_block_argmax(float best, int bi, float (*cbest)[S2_PNL_NT / 32],
                                               int (*cidx)[S2_PNL_NT / 32], int buf, int fallback,
                                               float& best_out) {
  constexpr int NW = S2_PNL_NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    cbest[buf][warp] = best;
    cidx[buf][warp] = bi;
  }
  __syncthreads();
  best = lane < NW ? cbest[buf][lane] : -1.0f;
  bi = lane < NW ? cidx[buf][lane] : INT_MAX;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  best_out = best;
  return bi == INT_MAX ? fallback : bi;
}

// Factorisation of the panel at column k0 (one CTA; panel in shared memory,
// column-major).  Thread t owns the panel rows r = t (mod S2_PNL_NT): in
// step j it scales its rows' multipliers of column j, updates its rows of
// columns j+1 .. w-1 (the arithmetic of s2::panel_scale and panel_rank1)
// and scans its rows of column j+1 for the next pivot, so that a step needs
// two barriers: one in the pivot search, one after the interchange.
__global__ void __launch_bounds__(S2_PNL_NT) k_s2_panel(const s2::Grid g, S2Work w, int k0) {
  __shared__ float cbest[2][S2_PNL_NT / 32];
  __shared__ int cidx[2][S2_PNL_NT / 32];
  float* P = reinterpret_cast<float*>(s2_smem);
  const int tid = threadIdx.x;
  const int wd = s2::panel_width(g, w.nb, k0), H = s2::panel_height(g, wd, k0);
  // the panel arrives by asynchronous copies, all in flight at once (zero
  // outside the band: the values of s2::panel_load)
  for (int e = tid; e < wd * H; e += S2_PNL_NT) {
    const int c = e / H, r = e - c * H;
    const bool in = s2::in_band(g, k0 + r, k0 + c);
    s2_cp_async4(P + e, w.AB + (in ? s2::band_at(g, k0 + r, k0 + c) : 0), in ? 4 : 0);
  }
  s2_cp_async_wait_all();
  __syncthreads();
  float best = -1.0f, pbest = -1.0f;
  int bi = INT_MAX;
  for (int r = tid; r <= s2::panel_rmax(g, H, 0); r += S2_PNL_NT) {
    const float a = fabsf(P[r]);
    if (a > best) {
      best = a;
      bi = r;
    }
  }
  int p = s2_block_argmax(best, bi, cbest, cidx, 0, 0, pbest);
  for (int j = 0; j < wd; ++j) {
    if (tid == 0) {
      w.piv[k0 + j] = k0 + p;
      if (!(pbest > 0.0f)) w.sc[S2_SING] = 1.0;
    }
    if (p != j && tid < wd) {
      float* col = P + (size_t)tid * H;
      const float t = col[j];
      col[j] = col[p];
      col[p] = t;
    }
    __syncthreads();
    const float* lj0 = P + (size_t)j * H;
    const float piv = lj0[j];
    const int rm = s2::panel_rmax(g, H, j);
    const int rm1 = j + 1 < wd ? s2::panel_rmax(g, H, j + 1) : -1;
    const int rend = rm > rm1 ? rm : rm1;
    best = -1.0f;
    bi = INT_MAX;
    int r = tid;
    if (r <= j) r += ((j - tid) / S2_PNL_NT + 1) * S2_PNL_NT;
    for (; r <= rend; r += S2_PNL_NT) {
      if (r <= rm) {
        float* lj = P + (size_t)j * H;
        const float l = piv != 0.0f ? lj[r] / piv : 0.0f;
        lj[r] = l;
        for (int c = j + 1; c < wd; ++c) {
          float* col = P + (size_t)c * H;
          col[r] -= l * col[j];
        }
      }
      if (r <= rm1) {
        const float a = fabsf(P[(size_t)(j + 1) * H + r]);
        if (a > best) {
          best = a;
          bi = r;
        }
      }
    }
    if (j + 1 < wd) p = s2_block_argmax(best, bi, cbest, cidx, (j + 1) & 1, j + 1, pbest);
  }
  __syncthreads();
  s2::panel_store(g, w.nb, w.AB, w.Lp, w.ud, k0, wd, H, P, tid, S2_PNL_NT);
}

// The panel's interchanges and eliminations on up to cbt trailing columns per
// CTA (the arithmetic of s2::trail_swaps, trail_l11_step and trail_l21, in
// their order): the column segments arrive by asynchronous copies (zero
// outside the band), a thread per column applies the interchanges, a warp
// per column the unit-lower solve with L11 (lane i holding L11's row i), and
// a thread per row of L21 (its multipliers in registers) updates that row of
// every column of the CTA.  No copy of the multipliers in shared memory, so
// the CTAs stay small and many.
__global__ void __launch_bounds__(S2_NT) k_s2_trail(const s2::Grid g, S2Work w, int k0, int cbt) {
  __shared__ int spv[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = w.nb, ldp = g.kl + nb;
  const int wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
  const int cfirst = k0 + wd + blockIdx.x * cbt;
  const int clast = s2::trail_last(g, k0, wd);
  const int ncols = clast - cfirst + 1 < cbt ? clast - cfirst + 1 : cbt;
  if (ncols <= 0) return;
  float* Cs = reinterpret_cast<float*>(s2_smem);
  const float* Lk = w.Lp + s2::lp_base(g, nb, k0);
  for (int e = tid; e < ncols * H; e += S2_NT) {
    const int cc = e / H, r = e - cc * H, c = cfirst + cc;
    const bool in = s2::in_band(g, k0 + r, c);
    s2_cp_async4(Cs + e, w.AB + (in ? s2::band_at(g, k0 + r, c) : 0), in ? 4 : 0);
  }
  if (tid < wd) spv[tid] = w.piv[k0 + tid] - k0;
  s2_cp_async_wait_all();
  __syncthreads();
  for (int cc = tid; cc < ncols; cc += S2_NT) {
    float* a = Cs + (size_t)cc * H;
    for (int j = 0; j < wd; ++j) {
      const int p = spv[j];
      if (p != j) {
        const float t = a[j];
        a[j] = a[p];
        a[p] = t;
      }
    }
  }
  __syncthreads();
  {
    const int i = lane, ic = i < wd ? i : wd - 1;
    float lr[32];
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const float l = Lk[(size_t)(jj < wd ? jj : wd - 1) * ldp + ic];
      lr[jj] = (jj < i && i < wd) ? l : 0.0f;
    }
    for (int cc = warp; cc < ncols; cc += S2_NT / 32) {
      float* a = Cs + (size_t)cc * H;
      float ai = lane < wd ? a[lane] : 0.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < wd) {
          const float aj = __shfl_sync(0xffffffffu, ai, j);
          if (lane > j && lane < wd) ai -= lr[j] * aj;
        }
      }
      if (lane < wd) a[lane] = ai;
    }
  }
  __syncthreads();
  for (int r = wd + tid; r < H; r += S2_NT) {
    float l[32];
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) l[jj] = Lk[(size_t)(jj < wd ? jj : wd - 1) * ldp + r];
    for (int cc = 0; cc < ncols; ++cc) {
      const float* a = Cs + (size_t)cc * H;
      float acc = 0.0f;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj)
        if (jj < wd) acc += l[jj] * a[jj];
      Cs[(size_t)cc * H + r] -= acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < ncols * H; e += S2_NT) {
    const int cc = e / H, r = e - cc * H, c = cfirst + cc;
    if (s2::in_band(g, k0 + r, c)) w.AB[s2::band_at(g, k0 + r, c)] = Cs[e];
  }
}

// Forward and backward substitution with the FP32 factors for two
// right-hand sides in FP32 arithmetic (the refinement's FP64 residuals make
// up the precision): b0, b1 (consumed) -> o0, o1; y0, y1 scratch.  One CTA;
// the current panel's window of the right-hand sides and its pivots in
// shared memory.
__global__ void __launch_bounds__(S2_SUB_NT) k_s2_subst(const s2::Grid g, S2Work w, double* b0, double* b1, double* o0,
                                                        double* o1) {
  __shared__ int spiv[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = w.nb, N = g.N;
  const int span = g.kl + g.ku + nb;
  const int ldp = g.kl + nb;
  float* t0 = reinterpret_cast<float*>(s2_smem);
  float* t1 = t0 + span;
  double* y0 = w.y0;
  double* y1 = w.y1;
  for (int k0 = 0; k0 < N; k0 += nb) {
    const int wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
#pragma unroll 4
    for (int r = tid; r < H; r += S2_SUB_NT) {
      t0[r] = (float)b0[k0 + r];
      t1[r] = (float)b1[k0 + r];
    }
    if (tid < wd) spiv[tid] = w.piv[k0 + tid] - k0;
    __syncthreads();
    if (tid == 0) {
      for (int j = 0; j < wd; ++j) {
        const int p = spiv[j];
        if (p != j) {
          float t = t0[j];
          t0[j] = t0[p];
          t0[p] = t;
          t = t1[j];
          t1[j] = t1[p];
          t1[p] = t;
        }
      }
    }
    __syncthreads();
    const float* Lk = w.Lp + s2::lp_base(g, nb, k0);
    if (warp == 0) {
      const int i = lane;
      float a0 = i < wd ? t0[i] : 0.0f, a1 = i < wd ? t1[i] : 0.0f;
      // every lane loads all 32 entries at clamped (valid) indices, so the
      // loads issue together; the unused ones are dropped by the selects
      const int ic = i < wd ? i : wd - 1;
      float lr[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const float l = Lk[(size_t)(jj < wd ? jj : wd - 1) * ldp + ic];
        lr[jj] = (jj < i && i < wd) ? l : 0.0f;
      }
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        if (jj < wd) {
          const float y0j = __shfl_sync(0xffffffffu, a0, jj);
          const float y1j = __shfl_sync(0xffffffffu, a1, jj);
          if (i > jj && i < wd) {
            a0 -= lr[jj] * y0j;
            a1 -= lr[jj] * y1j;
          }
        }
      }
      if (i < wd) {
        t0[i] = a0;
        t1[i] = a1;
        y0[k0 + i] = a0;
        y1[k0 + i] = a1;
      }
    }
    __syncthreads();
    for (int r = wd + tid; r < H; r += S2_SUB_NT) {
      float lv[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) lv[jj] = Lk[(size_t)(jj < wd ? jj : wd - 1) * ldp + r];
      float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        acc0 += jj < wd ? lv[jj] * t0[jj] : 0.0f;
        acc1 += jj < wd ? lv[jj] * t1[jj] : 0.0f;
      }
      b0[k0 + r] = t0[r] - acc0;
      b1[k0 + r] = t1[r] - acc1;
    }
    __syncthreads();
  }
  for (int k0 = ((N - 1) / nb) * nb; k0 >= 0; k0 -= nb) {
    const int wd = s2::panel_width(g, nb, k0);
    const int lo = k0 - g.kl - g.ku > 0 ? k0 - g.kl - g.ku : 0;
    const int nwin = k0 + wd - lo;
#pragma unroll 4
    for (int r = tid; r < nwin; r += S2_SUB_NT) {
      t0[r] = (float)y0[lo + r];
      t1[r] = (float)y1[lo + r];
    }
    __syncthreads();
    if (warp == 0) {
      const int i = lane;
      float a0 = i < wd ? t0[k0 - lo + i] : 0.0f, a1 = i < wd ? t1[k0 - lo + i] : 0.0f;
      const float dg = i < wd ? w.ud[k0 + i] : 1.0f;
      const int ic = i < wd ? i : wd - 1;
      float ur[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const float u = s2::umul(g, w.AB, k0 + ic, k0 + (jj < wd ? jj : wd - 1));
        ur[jj] = (jj > i && jj < wd) ? u : 0.0f;
      }
      float x0i = 0.0f, x1i = 0.0f;
#pragma unroll
      for (int jj = 31; jj >= 0; --jj) {
        if (jj < wd) {
          const float x0j = __shfl_sync(0xffffffffu, a0 / dg, jj);
          const float x1j = __shfl_sync(0xffffffffu, a1 / dg, jj);
          if (i == jj) {
            x0i = x0j;
            x1i = x1j;
          }
          if (i < jj) {
            a0 -= ur[jj] * x0j;
            a1 -= ur[jj] * x1j;
          }
        }
      }
      if (i < wd) {
        t0[k0 - lo + i] = x0i;
        t1[k0 - lo + i] = x1i;
        o0[k0 + i] = x0i;
        o1[k0 + i] = x1i;
      }
    }
    __syncthreads();
    for (int r = lo + tid; r < k0; r += S2_SUB_NT) {
      float uv[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) uv[jj] = s2::umul(g, w.AB, r, k0 + (jj < wd ? jj : wd - 1));
      float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        acc0 += jj < wd ? uv[jj] * t0[k0 - lo + jj] : 0.0f;
        acc1 += jj < wd ? uv[jj] * t1[k0 - lo + jj] : 0.0f;
      }
      y0[r] = t0[r - lo] - acc0;
      y1[r] = t1[r - lo] - acc1;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The same substitutions across a cluster of SC_CL CTAs (SC_CL SMs) instead
// of one CTA.  Per panel, warp 0 of every CTA applies the panel's
// interchanges and multiplies the panel's head by the inverse of its 32 x 32
// triangle (a product of 32 independent terms instead of a chain of 32
// dependent eliminations); warp 1 computes those inverses two panels ahead;
// the other warps update their share of the rows below (above, going
// backward), one row per lane, with the factor entries of the panel loaded
// between a thread's arrival at the previous panel's cluster barrier and its
// wait there.  One cluster barrier per panel.  The right-hand sides live in
// FP32 ping-pong vectors in global memory (read and written at L2): panel k
// reads pair k % 2 and writes pair (k + 1) % 2, so no CTA overwrites a value
// another may still read.  Rows a panel does not write keep their value in
// both pairs (both start as the input), which is what the next panel needs.
// ---------------------------------------------------------------------------
constexpr int SC_CL = 8;                 // CTAs: one cluster (the portable maximum)
constexpr int SC_UW = 8;                 // update warps per CTA (warps 2 .. SC_UW + 1)
constexpr int SC_NT = 32 * (2 + SC_UW);  // warp 0 solves, warp 1 inverts ahead

__device__ __forceinline__ void sc_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void sc_cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void sc_cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// barrier 1 of the CTA for the solver and update warps only (warp 1 keeps
// to its own pace between cluster barriers)
__device__ __forceinline__ void sc_bar_solve_update() {
  asm volatile("bar.sync 1, %0;" ::"r"(32 * (1 + SC_UW)) : "memory");
}

__device__ __forceinline__ unsigned sc_cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// The panel's interchanges as a map of window positions: m[r] = the window
// row whose value ends at position r (identity elsewhere); the entries the
// previous use touched are put back first.
__device__ void sc_build_map(const s2::Grid& g, const int32_t* piv, int nb, int k0, int* m, int* touched, int& nt) {
  for (int q = 0; q < nt; ++q) m[touched[q]] = touched[q];
  nt = 0;
  const int wd = s2::panel_width(g, nb, k0);
  for (int j = 0; j < wd; ++j) {
    const int p = piv[k0 + j] - k0;
    if (p != j) {
      const int t = m[j];
      m[j] = m[p];
      m[p] = t;
      touched[nt++] = j;
      touched[nt++] = p;
    }
  }
}

// Row `lane` of the panel at k0's 32 x 32 triangle (identity rows past the
// panel's width): the unit lower L11 (forward, below the diagonal only) or
// the upper U11 with its diagonal (backward).
__device__ __forceinline__ void sc_tri_row(const s2::Grid& g, const S2Work& w, bool lower, int k0, int lane,
                                           float* row) {
  const int nb = w.nb, ldp = g.kl + nb;
  const int wd = s2::panel_width(g, nb, k0);
  const float* Lk = w.Lp + s2::lp_base(g, nb, k0);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float v = j == lane ? 1.0f : 0.0f;
    if (lane < wd && j < wd) {
      if (lower)
        v = j < lane ? __ldg(Lk + (size_t)j * ldp + lane) : (j == lane ? 1.0f : 0.0f);
      else
        v = j >= lane ? s2::umul(g, w.AB, k0 + lane, k0 + j) : 0.0f;
    }
    row[j] = v;
  }
}

// The inverse of a triangle given by rows (row[j] of lane i = T[i][j]) into
// inv[i][j]: lane c solves T x = e_c, forward (lower, unit diagonal) or
// backward (upper), with the triangle staged in sc.
__device__ __forceinline__ void sc_tri_inverse(bool lower, const float* row, float (*sc)[33], float (*inv)[33],
                                               int lane) {
#pragma unroll
  for (int j = 0; j < 32; ++j) sc[lane][j] = row[j];
  __syncwarp();
  float x[32];
  if (lower) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < i; ++j) acc += sc[i][j] * x[j];
      x[i] = i == lane ? 1.0f : (i > lane ? -acc : 0.0f);
    }
  } else {
#pragma unroll
    for (int i = 31; i >= 0; --i) {
      float acc = 0.0f;
#pragma unroll
      for (int j = i + 1; j < 32; ++j) acc += sc[i][j] * x[j];
      const float rd = 1.0f / sc[i][i];
      x[i] = i == lane ? rd : (i < lane ? -acc * rd : 0.0f);
    }
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) inv[i][lane] = x[i];
  __syncwarp();
}

__global__ void __launch_bounds__(SC_NT) k_s2_subst_cl(const s2::Grid g, S2Work w, const double* b0,
                                                       const double* b1, double* o0, double* o1) {
  __shared__ float ty0[32], ty1[32];
  __shared__ int touched[2][64];
  __shared__ int ntouch[2];
  __shared__ float invs[3][32][33];  // triangle inverses: panels k, k + 1, k + 2
  __shared__ float scr[32][33];      // warp 1's staging of a triangle
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned rank = sc_cluster_rank();
  const int nb = w.nb, N = g.N, ldp = g.kl + nb, hcap = g.kl + nb;
  const int nk = (N + nb - 1) / nb;
  const int nup = SC_CL * SC_UW;                  // update warps in the cluster
  const int uq = (int)rank * SC_UW + (warp - 2);  // this warp's place among them (warp >= 2)
  int* const map0 = reinterpret_cast<int*>(s2_smem);  // two maps of hcap entries
  auto map = [&](int k) { return map0 + (k & 1) * hcap; };
  // pair p of right-hand-side vectors: rhs 0 at qv(p, 0), rhs 1 at qv(p, 1)
  auto qv = [&](int p, int c) { return w.q + (size_t)(2 * (p & 1) + c) * N; };
  auto fill = [&](const double* v0s, const double* v1s) {
    for (int u = (int)rank * SC_NT + tid; u < N; u += SC_CL * SC_NT) {
      const float v0 = (float)__ldcg(v0s + u), v1 = (float)__ldcg(v1s + u);
      __stcg(qv(0, 0) + u, v0);
      __stcg(qv(0, 1) + u, v1);
      __stcg(qv(1, 0) + u, v0);
      __stcg(qv(1, 1) + u, v1);
    }
  };
  float fr[32];  // warp 1: a triangle's row `lane`, fetched ahead; update warps: the lane's row of L21 or U12
  // ---- forward: L y = P b ----
  auto load_l21 = [&](int k0) {
    const int wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
    const float* Lk = w.Lp + s2::lp_base(g, nb, k0);
    const int r = wd + 32 * uq + lane;
    const int rc = r < H ? r : H - 1;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) fr[jj] = __ldg(Lk + (size_t)(jj < wd ? jj : wd - 1) * ldp + rc);
  };
  fill(b0, b1);
  for (int r = tid; r < 2 * hcap; r += SC_NT) map0[r] = r < hcap ? r : r - hcap;
  if (tid < 2) ntouch[tid] = 0;
  __syncthreads();
  if (warp == 0 && lane == 0) sc_build_map(g, w.piv, nb, 0, map(0), touched[0], ntouch[0]);
  if (warp == 1) {
    for (int q = 0; q < 2 && q < nk; ++q) {
      sc_tri_row(g, w, true, q * nb, lane, fr);
      sc_tri_inverse(true, fr, scr, invs[q], lane);
    }
    if (nk > 2) sc_tri_row(g, w, true, 2 * nb, lane, fr);
  }
  if (warp >= 2) load_l21(0);
  sc_cluster_sync();
  for (int k = 0; k < nk; ++k) {
    const int k0 = k * nb;
    const int wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
    const float* qa0 = qv(k, 0);
    const float* qa1 = qv(k, 1);
    float* qb0 = qv(k + 1, 0);
    float* qb1 = qv(k + 1, 1);
    const int* m = map(k);
    const int r = wd + 32 * uq + lane;
    float v0 = 0.0f, v1 = 0.0f;
    if (warp == 0) {
      const int i = lane;
      const float a0 = i < wd ? __ldcg(qa0 + k0 + m[i]) : 0.0f, a1 = i < wd ? __ldcg(qa1 + k0 + m[i]) : 0.0f;
      float (*inv)[33] = invs[k % 3];
      float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const float b0j = __shfl_sync(0xffffffffu, a0, jj), b1j = __shfl_sync(0xffffffffu, a1, jj);
        const float t = inv[i][jj];
        y0 += t * b0j;
        y1 += t * b1j;
      }
      if (i < wd) {
        ty0[i] = y0;
        ty1[i] = y1;
        if (rank == 0) {
          w.y0[k0 + i] = y0;
          w.y1[k0 + i] = y1;
        }
      }
    } else if (warp >= 2 && r < H) {
      v0 = __ldcg(qa0 + k0 + m[r]);
      v1 = __ldcg(qa1 + k0 + m[r]);
    }
    if (warp != 1) sc_bar_solve_update();
    if (warp == 0) {
      if (k + 1 < nk && lane == 0)
        sc_build_map(g, w.piv, nb, k0 + nb, map(k + 1), touched[(k + 1) & 1], ntouch[(k + 1) & 1]);
      __syncwarp();
      sc_cluster_arrive();
    } else if (warp == 1) {
      if (k + 2 < nk) sc_tri_inverse(true, fr, scr, invs[(k + 2) % 3], lane);
      sc_cluster_arrive();
      if (k + 3 < nk) sc_tri_row(g, w, true, k0 + 3 * nb, lane, fr);
    } else {
      if (r < H) {
        float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          acc0 += jj < wd ? fr[jj] * ty0[jj] : 0.0f;
          acc1 += jj < wd ? fr[jj] * ty1[jj] : 0.0f;
        }
        __stcg(qb0 + k0 + r, v0 - acc0);
        __stcg(qb1 + k0 + r, v1 - acc1);
      }
      // rows past the cluster's lanes (bands wider than 32 x SC_CL x SC_UW rows)
      const float* Lk = w.Lp + s2::lp_base(g, nb, k0);
      for (int rr = r + 32 * nup; rr < H; rr += 32 * nup) {
        const float x0 = __ldcg(qa0 + k0 + m[rr]), x1 = __ldcg(qa1 + k0 + m[rr]);
        float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll 8
        for (int jj = 0; jj < 32; ++jj) {
          const float l = __ldg(Lk + (size_t)(jj < wd ? jj : wd - 1) * ldp + rr);
          acc0 += jj < wd ? l * ty0[jj] : 0.0f;
          acc1 += jj < wd ? l * ty1[jj] : 0.0f;
        }
        __stcg(qb0 + k0 + rr, x0 - acc0);
        __stcg(qb1 + k0 + rr, x1 - acc1);
      }
      sc_cluster_arrive();
      if (k + 1 < nk) load_l21(k0 + nb);
    }
    sc_cluster_wait();
  }
  // ---- backward: U x = y ----
  auto load_u12 = [&](int k0) {
    const int wd = s2::panel_width(g, nb, k0);
    const int lo = k0 - g.kl - g.ku > 0 ? k0 - g.kl - g.ku : 0;
    const int r = lo + 32 * uq + lane;
    const int rc = r < k0 ? r : (k0 > 0 ? k0 - 1 : 0);
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) fr[jj] = s2::umul(g, w.AB, rc, k0 + (jj < wd ? jj : wd - 1));
  };
  fill(w.y0, w.y1);
  const int klast = (nk - 1) * nb;
  if (warp == 1) {
    for (int q = 0; q < 2 && q < nk; ++q) {
      sc_tri_row(g, w, false, klast - q * nb, lane, fr);
      sc_tri_inverse(false, fr, scr, invs[q], lane);
    }
    if (nk > 2) sc_tri_row(g, w, false, klast - 2 * nb, lane, fr);
  }
  if (warp >= 2) load_u12(klast);
  sc_cluster_sync();
  for (int k = nk - 1, it = 0; k >= 0; --k, ++it) {
    const int k0 = k * nb;
    const int wd = s2::panel_width(g, nb, k0);
    const int lo = k0 - g.kl - g.ku > 0 ? k0 - g.kl - g.ku : 0;
    const float* qa0 = qv(it, 0);
    const float* qa1 = qv(it, 1);
    float* qb0 = qv(it + 1, 0);
    float* qb1 = qv(it + 1, 1);
    const int r = lo + 32 * uq + lane;
    float v0 = 0.0f, v1 = 0.0f;
    if (warp == 0) {
      const int i = lane;
      const float a0 = i < wd ? __ldcg(qa0 + k0 + i) : 0.0f, a1 = i < wd ? __ldcg(qa1 + k0 + i) : 0.0f;
      float (*inv)[33] = invs[it % 3];
      float x0 = 0.0f, x1 = 0.0f;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const float y0j = __shfl_sync(0xffffffffu, a0, jj), y1j = __shfl_sync(0xffffffffu, a1, jj);
        const float t = inv[i][jj];
        x0 += t * y0j;
        x1 += t * y1j;
      }
      if (i < wd) {
        ty0[i] = x0;
        ty1[i] = x1;
        if (rank == 0) {
          o0[k0 + i] = x0;
          o1[k0 + i] = x1;
        }
      }
    } else if (warp >= 2 && r < k0) {
      v0 = __ldcg(qa0 + r);
      v1 = __ldcg(qa1 + r);
    }
    if (warp != 1) sc_bar_solve_update();
    if (warp == 0) {
      sc_cluster_arrive();
    } else if (warp == 1) {
      if (it + 2 < nk) sc_tri_inverse(false, fr, scr, invs[(it + 2) % 3], lane);
      sc_cluster_arrive();
      if (it + 3 < nk) sc_tri_row(g, w, false, k0 - 3 * nb, lane, fr);
    } else {
      if (r < k0) {
        float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          acc0 += jj < wd ? fr[jj] * ty0[jj] : 0.0f;
          acc1 += jj < wd ? fr[jj] * ty1[jj] : 0.0f;
        }
        __stcg(qb0 + r, v0 - acc0);
        __stcg(qb1 + r, v1 - acc1);
      }
      for (int rr = r + 32 * nup; rr < k0; rr += 32 * nup) {
        const float x0 = __ldcg(qa0 + rr), x1 = __ldcg(qa1 + rr);
        float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll 8
        for (int jj = 0; jj < 32; ++jj) {
          const float u = s2::umul(g, w.AB, rr, k0 + (jj < wd ? jj : wd - 1));
          acc0 += jj < wd ? u * ty0[jj] : 0.0f;
          acc1 += jj < wd ? u * ty1[jj] : 0.0f;
        }
        __stcg(qb0 + rr, x0 - acc0);
        __stcg(qb1 + rr, x1 - acc1);
      }
      sc_cluster_arrive();
      if (k > 0) load_u12(k0 - nb);
    }
    sc_cluster_wait();
  }
}

// right-hand sides of a Newton step: -R and e_r (the total-mass row)
__global__ void k_s2_prep(const s2::Grid g, S2Work w) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= g.N) return;
  const double r0 = -w.R[u], r1 = u == s2::mass_row(g) ? 1.0 : 0.0;
  w.rhs0[u] = r0;
  w.rhs1[u] = r1;
  w.b0[u] = r0;
  w.b1[u] = r1;
}

// refinement residuals in FP64: b = rhs - B v
__global__ void k_s2_bmv(const s2::Grid g, S2Work w) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= g.N) return;
  w.b0[u] = w.rhs0[u] - s2::bmv_row(g, w.Jc, w.v0, u);
  w.b1[u] = w.rhs1[u] - s2::bmv_row(g, w.Jc, w.v1, u);
}

__global__ void k_s2_add(const s2::Grid g, S2Work w) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= g.N) return;
  w.v0[u] += w.s0[u];
  w.v1[u] += w.s1[u];
}

// The rank-one correction for the total-mass row (z = v0, y = v1), the damped
// update that keeps rho, T_t, T_r positive and finite (step halved up to 60
// times), and the convergence test on the largest relative update of a full
// step (|dx| / max(|x|, 1e-3) < tol); a step cut below 1/1024 is a stall.
__global__ void __launch_bounds__(S2_UPD_NT) k_s2_newton(const s2::Grid g, S2Work w, int n_m, double tol) {
  __shared__ double red[S2_UPD_NT];
  const int tid = threadIdx.x;
  const int N = g.N;
  const int mr = s2::mass_row(g);
  double wz = 0.0, wy = 0.0;
  for (int b = tid; b < g.n; b += S2_UPD_NT) {
    if (s2::NV * b == mr) continue;
    int i, j;
    s2::cell_of_band(g, b, i, j);
    const double ms = s2::mass_scale(g, i, j);
    wz += w.v0[s2::NV * b] * ms;
    wy += w.v1[s2::NV * b] * ms;
  }
  wz = s2_block_sum<S2_UPD_NT>(wz, red) / g.n;
  wy = s2_block_sum<S2_UPD_NT>(wy, red) / g.n;
  const double f = wz / (1.0 + wy);
  for (int u = tid; u < N; u += S2_UPD_NT) w.d[u] = w.v0[u] - w.v1[u] * f;
  __syncthreads();
  double lam = 1.0;
  bool ok = false;
  for (int hv = 0; hv < 60 && !ok; ++hv) {
    double bad = 0.0;
    for (int u = tid; u < N; u += S2_UPD_NT) {
      const double xn = w.x[u] + lam * w.d[u];
      const int v = u % s2::NV;
      if (!isfinite(xn) || ((v == 0 || v >= 3) && xn <= 0.0)) bad = 1.0;
    }
    ok = s2_block_max<S2_UPD_NT>(bad, red) == 0.0;
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
  for (int u = tid; u < N; u += S2_UPD_NT) {
    const double x = w.x[u];
    const double step = lam * w.d[u];
    dm = fmax(dm, fabs(step) / fmax(fabs(x), 1e-3));
    w.x[u] = x + step;
  }
  dm = s2_block_max<S2_UPD_NT>(dm, red);
  if (tid == 0) {
    const double it = w.sc[S2_IT] + 1.0;
    w.sc[S2_IT] = it;
    w.sc[S2_DMAX] = dm;
    w.sc[S2_LAM] = lam;
    if (dm < tol && lam == 1.0) {
      // converged: a full Newton step below the tolerance
      w.sc[S2_STATUS] = 0.0;
      w.sc[S2_DONE] = 1.0;
    } else if (lam < 1.0 / 1024.0) {
      // stalled: positivity holds the step to a sliver, so the equations
      // have no solution near this state (e.g. a shock the central
      // differences cannot carry); the sampled fields are the output
      w.sc[S2_STATUS] = 2.0;
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

// shared-memory limits of the dynamic-size kernels, raised (never lowered)
// to what a solve needs
void s2_smem_limits(size_t panel, size_t trail, size_t subst) {
  static size_t set[3] = {48 * 1024, 48 * 1024, 48 * 1024};
  const void* fn[3] = {(const void*)k_s2_panel, (const void*)k_s2_trail, (const void*)k_s2_subst};
  const size_t need[3] = {panel, trail, subst};
  for (int k = 0; k < 3; ++k) {
    if (need[k] > set[k]) {
      cudaFuncSetAttribute(fn[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need[k]);
      set[k] = need[k];
    }
  }
}

}  // namespace

// One substitution (two right-hand sides): on a cluster of SC_CL CTAs where
// the device can run one, else on one CTA (k_s2_subst).
cudaError_t s2_subst(const s2::Grid& g, const S2Work& w, double* b0, double* b1, double* o0, double* o1,
                     size_t sm_subst, cudaStream_t st) {
  static int cluster_ok = -1;  // per process: 1 when an SC_CL-CTA cluster of k_s2_subst_cl fits
  const size_t sm_cl = sizeof(int) * 2 * ((size_t)g.kl + w.nb);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = SC_CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(SC_CL);
  cfg.blockDim = dim3(SC_NT);
  cfg.dynamicSmemBytes = sm_cl;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cluster_ok < 0) {
    int n = 0;
    cluster_ok = (sm_cl <= 48 * 1024 && cudaOccupancyMaxActiveClusters(&n, k_s2_subst_cl, &cfg) == cudaSuccess &&
                  n >= 1)
                     ? 1
                     : 0;
    cudaGetLastError();  // a refused query leaves no error behind
  }
  if (cluster_ok && sm_cl <= 48 * 1024)
    return cudaLaunchKernelEx(&cfg, k_s2_subst_cl, g, w, (const double*)b0, (const double*)b1, o0, o1);
  k_s2_subst<<<1, S2_SUB_NT, sm_subst, st>>>(g, w, b0, b1, o0, o1);
  return cudaGetLastError();
}

size_t synth2d_work_doubles(int nx, int ny, int annulus) {
  s2::Grid g = s2::make_grid(nx, ny, 1.0, 1.0, 2.0, 0.75, 1.0, 1.0, 1.0, 1.0, nullptr, nullptr);
  if (annulus) s2::set_annulus(g, nullptr);  // the band of the annulus's ordering
  return s2_doubles(g);
}

int launch_synth2d(const CellParams& cp, const double* fields, const double* hot, double* out, double* work,
                   int n_m, double tol, double* info, int* singular, cudaStream_t st) {
  s2::Grid g = s2::make_grid(cp.nx, cp.ny, cp.dx, cp.dy, cp.d_r, cp.omega, cp.mu_ref, cp.z_rot, cp.kappa_t,
                             cp.kappa_r, fields, hot);
  if (cp.mesh == 2) s2::set_edges(g, cp.xe, cp.ye, cp.lx * cp.ly);  // the wall-refined grid (device edges)
  if (cp.mesh == 1) s2::set_annulus(g, cp.rt);  // the annulus (device ring radii)
  const S2Work w = s2_carve(g, work);
  if (w.nb == 0) return (int)cudaErrorInvalidValue;
  const int nb = w.nb;
  const size_t hmax = (size_t)g.kl + nb;
  const size_t sm_panel = sizeof(float) * nb * hmax;
  // trailing columns per CTA of the trailing update: up to 16, as shared
  // memory allows (column segments of hmax rows)
  int cbt = (int)(S2_SMEM_CAP / (sizeof(float) * hmax));
  if (cbt > 16) cbt = 16;
  if (cbt < 1) cbt = 1;
  const size_t sm_trail = sizeof(float) * (size_t)cbt * hmax;
  const size_t sm_subst = sizeof(float) * 2 * ((size_t)g.kl + g.ku + nb);
  s2_smem_limits(sm_panel, sm_trail, sm_subst);
  const int nt = 256;
  const int cell_grid = (g.n + nt - 1) / nt;
  const int vec_grid = (g.N + nt - 1) / nt;
  const long long jac_threads = (long long)g.n * s2::NSTENCIL * s2::NV;
  const int jac_grid = (int)((jac_threads + nt - 1) / nt);
  double sc[S2_NSC];
  k_s2_init<<<1, S2_NT, 0, st>>>(g, w);
  // The factorisation of the first Newton step is reused while the updates
  // keep shrinking (by half or more per step), with more refinement sweeps
  // against each step's fresh FP64 Jacobian; otherwise the next step
  // refactorises.
  bool refactor = true;
  double dm_prev = 0.0;
  for (int it = 0; it < n_m; ++it) {
    k_s2_mass<<<1, S2_NT, 0, st>>>(g, w);
    k_s2_res<<<cell_grid, nt, 0, st>>>(g, w);
    if (refactor) cudaMemsetAsync(w.AB, 0, sizeof(float) * (size_t)g.ld * g.N, st);
    k_s2_jac<<<jac_grid, nt, 0, st>>>(g, w, refactor ? 1 : 0);
    if (refactor) {
      for (int k0 = 0; k0 < g.N; k0 += nb) {
        const int wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
        k_s2_panel<<<1, S2_PNL_NT, sizeof(float) * (size_t)wd * H, st>>>(g, w, k0);
        const int ntrail = s2::trail_last(g, k0, wd) - (k0 + wd) + 1;
        if (ntrail > 0)
          k_s2_trail<<<(ntrail + cbt - 1) / cbt, S2_NT, sizeof(float) * (size_t)cbt * H, st>>>(g, w, k0, cbt);
      }
    }
    const int nsweep = refactor ? S2_NREF : S2_NREF_REUSE;
    k_s2_prep<<<vec_grid, nt, 0, st>>>(g, w);
    cudaError_t le = s2_subst(g, w, w.b0, w.b1, w.v0, w.v1, sm_subst, st);
    for (int r = 0; r < nsweep && le == cudaSuccess; ++r) {
      k_s2_bmv<<<vec_grid, nt, 0, st>>>(g, w);
      le = s2_subst(g, w, w.b0, w.b1, w.s0, w.s1, sm_subst, st);
      k_s2_add<<<vec_grid, nt, 0, st>>>(g, w);
    }
    if (le != cudaSuccess) return (int)le;
    k_s2_newton<<<1, S2_UPD_NT, 0, st>>>(g, w, n_m, tol);
    cudaMemcpyAsync(sc, w.sc, sizeof(double) * (S2_LAM + 1), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    if (sc[S2_DONE] != 0.0) break;
    refactor = it > 0 && !(sc[S2_DMAX] <= 0.5 * dm_prev);
    dm_prev = sc[S2_DMAX];
  }
  k_s2_mass<<<1, S2_NT, 0, st>>>(g, w);
  k_s2_res<<<cell_grid, nt, 0, st>>>(g, w);
  k_s2_final<<<1, S2_NT, 0, st>>>(g, w, out, info);
  cudaMemcpyAsync(sc, w.sc, sizeof(double) * (S2_LAM + 1), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  if (singular) *singular = sc[S2_SING] != 0.0;
  return 0;
}

}  // namespace dsmc
