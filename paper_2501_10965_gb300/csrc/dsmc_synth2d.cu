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
// Factorisation: per panel of nb columns, one CTA factorises the panel (its
// rows in registers, k_s2_panel_rot, or in shared memory for taller panels),
// then one launch applies it to the up to kl + ku trailing columns, up to 8
// columns per CTA.  Substitution: a cluster of 8 CTAs walks the panels,
// forward then backward, as a data flow (k_s2_subst_df; with one cluster
// barrier per panel, k_s2_subst_cl, where its rows do not fit the cluster's
// shared memory; one CTA, k_s2_subst, where no cluster fits).  The launches
// on one stream order the factorisation's panels.
#include <climits>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

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
  S2_TOUT = 8,   // a wait of the substitution gave up
  S2_EPS0 = 9,   // step of the directional differences along v0, v1
  S2_EPS1 = 10,
  S2_NSC = 16
};

constexpr int S2_NT = 256;        // threads of the factorisation and substitution kernels
constexpr int S2_UPD_NT = 512;    // the Newton update
constexpr int S2_SUB_NT = 512;    // the substitutions
constexpr int S2_PNL_NT = 512;    // the panel factorisation
constexpr int S2_NREF = 1;        // refinement sweeps after a fresh factorisation
constexpr int S2_NREF_REUSE = 3;  // refinement sweeps when an earlier factorisation is reused
constexpr int S2_SMEM_CAP = 200 * 1024;
constexpr int S2_SMAP = 256;  // ints of a panel's row maps (k_s2_sprep, k_s2_spush)
constexpr size_t S2_DF_SMEM_CAP = 200 * 1024;  // rows of the data-flow substitution per CTA (4 copies of 32 floats a block)

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
  float* inv;     // per panel: the inverses of its L11 and U11 triangles (2 x 32 x 32)
  float* mh;      // per panel k: inv(L11_k) times panel k - 1's multipliers of its head rows (32 x 32)
  int32_t* smap;  // per panel: its interchanges as maps of rows (S2_SMAP entries, k_s2_sprep, k_s2_spush)
  int nb, cb;
};

inline size_t round32(size_t n) { return (n + 31) & ~(size_t)31; }  // 256-byte multiples

inline size_t s2_lp_floats(const s2::Grid& g, int nb) { return (size_t)((g.N + nb - 1) / nb) * nb * (g.kl + nb); }

inline size_t s2_doubles(const s2::Grid& g) {
  const S2Blocking bl = s2_blocking(g);
  const size_t N = (size_t)g.N;
  const size_t vec = round32(N);
  const size_t jc = round32((size_t)g.n * s2::NSTENCIL * s2::NV * s2::NV);
  const size_t nk = (N + bl.nb - 1) / bl.nb;
  // AB, Lp, ud, piv, q, inv, smap
  const size_t f32 = (size_t)g.ld * N + s2_lp_floats(g, bl.nb) + N + N + 4 * N + 3072 * nk + S2_SMAP * nk;
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
  f += 4 * (size_t)g.N;
  s.inv = f;
  f += 2048 * (size_t)((g.N + bl.nb - 1) / bl.nb);
  s.mh = f;
  f += 1024 * (size_t)((g.N + bl.nb - 1) / bl.nb);
  s.smap = reinterpret_cast<int32_t*>(f);
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

// the sampled fields as Newton's first state (warm: keep the state the work
// area holds, the previous solve's solution), the sampled total mass, and the
// scalar slots
__global__ void __launch_bounds__(S2_NT) k_s2_init(const s2::Grid g, S2Work w, int warm) {
  __shared__ double red[S2_NT];
  double s = 0.0;
  for (int b = threadIdx.x; b < g.n && !warm; b += S2_NT) {
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
    w.sc[S2_TOUT] = 0.0;
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

// a pivot candidate's key: 1 + the bits of its magnitude (0: not a
// candidate; magnitudes that are not numbers never win)
__device__ __forceinline__ unsigned s2_cand_key(float v, bool cand) {
  const float a = fabsf(v);
  return (cand && a == a) ? __float_as_uint(a) + 1u : 0u;
}

// The panel factorisation with the rows in registers.  Thread t holds the
// rows loaded from positions t + s T (s < RPT, T threads), each as 32
// columns of a frame that starts at column 4 g in steps 4 g .. 4 g + 3 (the
// frame shifts by four columns every four steps, so one loop body of four
// unrolled steps serves the panel; columns past the panel's width are
// skipped eight at a time).  Interchanges move no row: each row carries its
// current position.  One barrier per step: in the pivot search each warp
// writes its best candidate row (from the pivot column on) to shared memory
// with its key, so the row the block chooses is already there for the
// rank-one update of the next step.  The pivot row's U entries go to global
// memory at once, each row's multipliers to shared memory (Ls, by load
// index) until the end, when they are stored at the rows' final positions.
// The pivots are chosen as in k_s2_panel (largest magnitude, lowest position
// among equals), and each entry takes the same operations in the same order.
template <int RPT>
__global__ void __launch_bounds__(512) k_s2_panel_rot(const s2::Grid g, S2Work w, int k0) {
  __shared__ unsigned ckey[2][32];
  __shared__ int cpos[2][32];
  __shared__ __align__(16) float crow[2][32][32];  // per warp: its candidate row (frame of the next step)
  const int T = blockDim.x, NS = T * RPT, nw = T >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wd = s2::panel_width(g, w.nb, k0), H = s2::panel_height(g, wd, k0);
  float* Ls = reinterpret_cast<float*>(s2_smem);  // [32][NS]
  float a[RPT][32];
  int pos[RPT];
  bool act[RPT];
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int r = tid + s * T;
    pos[s] = r;
    act[s] = r < H;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const bool in = r < H && c < wd && s2::in_band(g, k0 + r, k0 + c);
      a[s][c] = in ? w.AB[s2::band_at(g, k0 + r, k0 + c)] : 0.0f;
    }
  }
  float pbest = -1.0f;
  int p = 0, pwin = 0;
  // pivot search on frame column fc among positions lo .. hi; the winning
  // rows go to crow[buf] in the frame shifted by sh columns
  // (lim: the frame columns inside the panel before the shift; the columns
  // past it are written eight at a time only where a chunk reaches inside)
  auto search = [&](auto fct, auto sht, int lo, int hi, int buf, int fallback, int lim) {
    constexpr int fc = decltype(fct)::value, sh = decltype(sht)::value;
    unsigned key = 0u;
    int bp = INT_MAX, bs = 0;
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const unsigned kq = s2_cand_key(a[s][fc], act[s] && pos[s] >= lo && pos[s] <= hi);
      if (kq > key || (kq == key && kq != 0u && pos[s] < bp)) {
        key = kq;
        bp = pos[s];
        bs = s;
      }
    }
    const unsigned kw = __reduce_max_sync(0xffffffffu, key);
    const int pw = __reduce_min_sync(0xffffffffu, key == kw ? bp : INT_MAX);
    if (kw != 0u && key == kw && bp == pw) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (8 * q + 7 >= fc && 8 * q < lim) {  // chunk q of the frame before the shift
#pragma unroll
          for (int c = (8 * q > fc ? 8 * q : fc); c < 8 * q + 8; ++c) {
            float v = a[0][c];
#pragma unroll
            for (int s = 1; s < RPT; ++s)
              if (s == bs) v = a[s][c];
            crow[buf][warp][c - sh] = v;
          }
        }
      }
    }
    if (lane == 0) {
      ckey[buf][warp] = kw;
      cpos[buf][warp] = pw;
    }
    __syncthreads();
    const unsigned k2 = lane < nw ? ckey[buf][lane] : 0u;
    const int p2 = lane < nw ? cpos[buf][lane] : INT_MAX;
    const unsigned km = __reduce_max_sync(0xffffffffu, k2);
    const int pm = __reduce_min_sync(0xffffffffu, k2 == km ? p2 : INT_MAX);
    const unsigned won = __ballot_sync(0xffffffffu, lane < nw && k2 == km && p2 == pm);
    pbest = km == 0u ? -1.0f : __uint_as_float(km - 1u);
    p = km == 0u ? fallback : pm;
    pwin = km == 0u ? 0 : __ffs(won) - 1;
  };
  search(std::integral_constant<int, 0>{}, std::integral_constant<int, 0>{}, 0, s2::panel_rmax(g, H, 0), 0, 0, wd);
  const int ld = g.ld;
#pragma unroll 1
  for (int jb = 0; jb < wd; jb += 4) {
    const int live = wd - jb;  // frame columns inside the panel
    // step j = jb + jj, its pivot column at frame column jj
    auto step = [&](auto jjt) {
      constexpr int jj = decltype(jjt)::value;
      const int j = jb + jj;
      if (j >= wd) return;
      const float* prow = crow[j & 1][pwin];
      // the interchange: the pivot row takes position j, the row there takes p
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        if (act[s] && pos[s] == p) {
          act[s] = false;
          pos[s] = j;
        } else if (act[s] && pos[s] == j) {
          pos[s] = p;
        }
      }
      if (tid == 0) {
        w.piv[k0 + j] = k0 + p;
        if (!(pbest > 0.0f)) w.sc[S2_SING] = 1.0;
      }
      // U(j, j + c) of the pivot row
      if (tid < wd - j) {
        const float v = prow[jj + tid];
        w.AB[(size_t)(k0 + j + tid) * ld + (size_t)(g.kl + g.ku - tid)] = v;
        if (tid == 0) w.ud[k0 + j] = v;
      }
      const float piv = prow[jj];
      const int rm = s2::panel_rmax(g, H, j);
      float l[RPT];
      bool upd[RPT];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        upd[s] = act[s] && pos[s] <= rm;
        l[s] = piv != 0.0f ? a[s][jj] / piv : 0.0f;
        if (act[s]) Ls[(size_t)j * NS + tid + s * T] = upd[s] ? l[s] : a[s][jj];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (8 * q + 7 > jj && 8 * q < live) {
#pragma unroll
          for (int c = (8 * q > jj ? 8 * q : jj + 1); c < 8 * q + 8; ++c) {
            const float pc = prow[c];
#pragma unroll
            for (int s = 0; s < RPT; ++s)
              if (upd[s]) a[s][c] -= l[s] * pc;
          }
        }
      }
      if (j + 1 < wd) {
        const int rm1 = s2::panel_rmax(g, H, j + 1);
        if constexpr (jj < 3)
          search(std::integral_constant<int, jj + 1>{}, std::integral_constant<int, 0>{}, j + 1, rm1, (j + 1) & 1,
                 j + 1, live);
        else
          search(std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{}, j + 1, rm1, (j + 1) & 1, j + 1,
                 live);
      }
    };
    step(std::integral_constant<int, 0>{});
    step(std::integral_constant<int, 1>{});
    step(std::integral_constant<int, 2>{});
    step(std::integral_constant<int, 3>{});
    // the next frame: columns jb + 4 .. (those inside the panel)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (8 * q + 4 < live) {
#pragma unroll
        for (int c = 8 * q; c < 8 * q + 8 && c + 4 < 32; ++c) {
#pragma unroll
          for (int s = 0; s < RPT; ++s) a[s][c] = a[s][c + 4];
        }
      }
    }
  }
  __syncthreads();
  // multipliers at the rows' final positions (zero rows past the band included)
  const size_t base = s2::lp_base(g, w.nb, k0);
  const int ldp = g.kl + w.nb;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int id = tid + s * T;
    if (id < H) {
      const int ps = pos[s], cend = ps < wd ? ps : wd;
      for (int c = 0; c < cend; ++c) w.Lp[base + (size_t)c * ldp + ps] = Ls[(size_t)c * NS + id];
    }
  }
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

// ---------------------------------------------------------------------------
// Substitution tables of one factorisation, a warp per panel k (used by
// k_s2_subst_df): the inverses of the panel's unit-lower L11 and upper U11
// triangles (sc_tri_row / sc_tri_inverse, row-major 32 x 32 at inv + 2048 k
// and inv + 2048 k + 1024), and the panel's interchanges as a map of rows:
// smap[S k + i], i < 32 (S = S2_SMAP), the row whose value ends at head
// position k0 + i (k0 + i itself past the panel's width); smap[S k + 32 + q]
// and smap[S k + 64 + q], q < smap[S k + 96], the rows past the head whose
// value changes (ascending) and the head position each takes it from.
// ---------------------------------------------------------------------------
constexpr int SP_WPB = 4;  // warps (panels) per CTA of k_s2_sprep

__global__ void __launch_bounds__(SP_WPB * 32) k_s2_sprep(const s2::Grid g, S2Work w) {
  __shared__ float scr[SP_WPB][32][33];
  __shared__ float inv[SP_WPB][32][33];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nb = w.nb, N = g.N, nk = (N + nb - 1) / nb;
  const int k = blockIdx.x * SP_WPB + wp;
  if (k >= nk) return;
  const int k0 = k * nb, wd = s2::panel_width(g, nb, k0);
  float fr[32];
  for (int t = 0; t < 2; ++t) {
    sc_tri_row(g, w, t == 0, k0, lane, fr);
    sc_tri_inverse(t == 0, fr, scr[wp], inv[wp], lane);
    float* dst = w.inv + (size_t)k * 2048 + t * 1024;
#pragma unroll 4
    for (int i = 0; i < 32; ++i) dst[i * 32 + lane] = inv[wp][i][lane];
    __syncwarp();
  }
  if (lane == 0) {
    // the interchanges applied in order to a sparse map (touched rows only)
    int pos[64], val[64], nt = 0;
    auto find = [&](int r) {
      for (int q = 0; q < nt; ++q)
        if (pos[q] == r) return q;
      pos[nt] = r;
      val[nt] = r;
      return nt++;
    };
    for (int j = 0; j < wd; ++j) {
      const int p = w.piv[k0 + j];
      if (p != k0 + j) {
        const int a = find(k0 + j), b = find(p);
        const int t = val[a];
        val[a] = val[b];
        val[b] = t;
      }
    }
    int32_t* sm = w.smap + (size_t)k * S2_SMAP;
    for (int i = 0; i < 32; ++i) sm[i] = k0 + i;
    int ntail = 0;
    for (int q = 0; q < nt; ++q) {
      if (pos[q] < k0 + wd) {
        sm[pos[q] - k0] = val[q];
      } else if (val[q] != pos[q]) {
        // insertion in ascending order of the row
        int z = ntail++;
        while (z > 0 && sm[32 + z - 1] > pos[q]) {
          sm[32 + z] = sm[32 + z - 1];
          sm[64 + z] = sm[64 + z - 1];
          --z;
        }
        sm[32 + z] = pos[q];
        sm[64 + z] = val[q];
      }
    }
    sm[96] = ntail;
  }
}

// The rows each head of the data-flow substitution needs, a warp per panel
// k (after k_s2_sprep): the head position i < wd takes the value, after
// step k - 1, of row h_i = smap[S k + i], and the tail entry q that of head
// position t_q = smap[S k + 64 + q]; both follow from the value after step
// k - 2 of the row that panel k - 1's interchanges move there,
// smap[S k + 128 + d] (d = i, or 32 + q; -1 where there is none).  Those of
// them that step k - 2 updates (rows of its window) are sent to the head by
// their owners (bit d of smap[S k + 192 + d / 32]; smap[S k + 194] of them);
// the others still hold their input.
__global__ void __launch_bounds__(SP_WPB * 32) k_s2_spush(const s2::Grid g, S2Work w) {
  __shared__ float lb[SP_WPB][32][33];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nb = w.nb, N = g.N, nk = (N + nb - 1) / nb, ldp = g.kl + nb;
  const int k = blockIdx.x * SP_WPB + wp;
  if (k >= nk) return;
  const int k0 = k * nb, wd = s2::panel_width(g, nb, k0);
  int32_t* sm = w.smap + (size_t)k * S2_SMAP;
  const int ntail = sm[96];
  int rh = lane < wd ? sm[lane] : -1, rt = lane < ntail ? sm[64 + lane] : -1;
  // mh = inv(L11_k) times panel k - 1's multipliers of the head's rows (row
  // l: those of row h_l, zero where h_l is past that panel's window): the
  // head's result is then inv(L11_k) a - mh y_{k-1}
  {
    const int p0 = k0 - nb;
    const bool hin = k > 0 && rh >= 0 && rh - p0 < s2::panel_height(g, nb, p0 > 0 ? p0 : 0);
    const float* Lk = w.Lp + s2::lp_base(g, nb, p0 > 0 ? p0 : 0);
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) lb[wp][lane][jj] = hin ? Lk[(size_t)jj * ldp + (rh - p0)] : 0.0f;
    __syncwarp();
    float ir[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) ir[l] = w.inv[(size_t)k * 2048 + lane * 32 + l];
    for (int j = 0; j < 32; ++j) {
      float m = 0.0f;
#pragma unroll
      for (int l = 0; l < 32; ++l) m += ir[l] * lb[wp][l][j];
      w.mh[(size_t)k * 1024 + lane * 32 + j] = m;
    }
  }
  if (k > 0) {
    const int32_t* smp = sm - S2_SMAP;
    const int ntp = smp[96];
    const int td = lane < ntp ? smp[32 + lane] : -1, ts = lane < ntp ? smp[64 + lane] : 0;
    int sh = rh, st = rt;
    for (int q = 0; q < ntp; ++q) {
      const int d = __shfl_sync(0xffffffffu, td, q), sv = __shfl_sync(0xffffffffu, ts, q);
      if (rh >= 0 && d == rh) sh = sv;
      if (rt >= 0 && d == rt) st = sv;
    }
    rh = sh;
    rt = st;
  }
  bool ph = false, pt = false;
  if (k >= 2) {
    const int p0 = k0 - 2 * nb, lo = p0 + nb, hi = p0 + s2::panel_height(g, nb, p0);
    ph = rh >= lo && rh < hi;
    pt = rt >= lo && rt < hi;
  }
  sm[128 + lane] = rh;
  sm[160 + lane] = rt;
  const unsigned mh = __ballot_sync(0xffffffffu, ph), mt = __ballot_sync(0xffffffffu, pt);
  if (lane == 0) {
    sm[192] = (int)mh;
    sm[193] = (int)mt;
    sm[194] = __popc(mh) + __popc(mt);
  }
}

// ---------------------------------------------------------------------------
// The substitutions as a data flow across a cluster of DF_C CTAs, with no
// cluster-wide barrier per panel.  Rows are owned by 32-row block: block b
// (rows 32 b .. 32 b + 31) by CTA b % DF_C, its values in that CTA's shared
// memory in two copies (parities): step s reads copy s % 2 and writes copy
// (s + 1) % 2, so that values read remotely are never overwritten while
// still needed (rows outside a step's window keep their value in both).
//
// Warp 0 of the owner of panel k's head block computes the head's values
// itself: each source row's value after step k - 2 (sent into a buffer of
// the head's CTA by the row's owner, by an asynchronous store that completes
// the buffer's mbarrier phase, as soon as step k - 2 has updated it; rows
// that step did not reach still hold their input) less the previous panel's
// multipliers times the previous step's result.  It applies the inverse of
// the panel's triangle and sends the 32 results (two right-hand sides) into
// a ring of DF_S slots in every CTA by asynchronous stores, which complete
// the slot's mbarrier phase there; with them go the head values that the
// panel's interchanges move to rows below the head, computed the same way.
// Warps 1 .. DF_UW of every CTA, in two groups that take alternate steps
// (a group waits, on a CTA-local mbarrier, for the other group's previous
// step), take each step's result from the ring, update their CTA's rows of
// the step's window and send the new values a later head needs; warp
// DF_UW + 1 arms each slot's next phase and, once the step's group has
// finished, publishes the number of steps done (release).  Warp
// 0 writes a ring slot only once every CTA has finished the slot's previous
// step, and (backward) reads its own rows once this CTA's count covers them.
// Each wait gives up after DF_WAIT_NS (the kernel then records the timeout in
// the work area, drains the buffers still armed and every CTA leaves at the
// next cluster barrier).
//
// Each row takes the operations of k_s2_subst_cl (the dot products in four
// partial sums); forward, then (after one cluster barrier) backward.
// ---------------------------------------------------------------------------
constexpr int DF_C = 8;                  // CTAs of the cluster
constexpr int DF_UWG = 5;                // update warps per group
constexpr int DF_UW = 2 * DF_UWG;        // update warps per CTA: group 0 takes the even steps, group 1 the odd
constexpr int DF_NT = 32 * (2 + DF_UW);  // warp 0 solves the heads, warp DF_UW + 1 publishes
constexpr int DF_S = 32;                 // ring slots (steps in flight)
constexpr unsigned long long DF_WAIT_NS = 500000000ull;  // 0.5 s
constexpr unsigned long long DF_DRAIN_NS = 1000000ull;   // 1 ms
// step barriers of the update-warp groups: more than the DF_S steps the
// groups can run ahead of the publishing warp (the ring's back-pressure), so
// a phase is never overtaken by the next use of its slot
constexpr int DF_GD = 64;
constexpr unsigned DF_SUSPEND_NS = 2000;                  // longest suspension of one wait test

__device__ __forceinline__ unsigned long long df_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned df_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// shared::cluster address of the same shared variable in CTA `cta`
__device__ __forceinline__ unsigned df_mapa(const void* p, unsigned cta) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(df_smem_addr(p)), "r"(cta));
  return r;
}

__device__ __forceinline__ unsigned df_ld_acquire(unsigned addr) {
  unsigned v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void df_st_release(unsigned addr, unsigned v) {
  asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// asynchronous store of 16 bytes into another CTA's shared memory, counted
// on that CTA's mbarrier at `mbar` (complete_tx) once it has landed
__device__ __forceinline__ void df_st_async4(unsigned addr, float4 v, unsigned mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void df_st_async2(unsigned addr, float a, float b, unsigned mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(a), "f"(b), "r"(mbar)
               : "memory");
}

// a count in this CTA's shared memory, published and read at CTA scope
__device__ __forceinline__ void df_st_release_cta(const unsigned* p, unsigned v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(df_smem_addr(p)), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned df_ld_acquire_cta(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(df_smem_addr(p)) : "memory");
  return v;
}

// this CTA's arrival on its mbarrier, expecting `bytes` of asynchronous stores in the phase
__device__ __forceinline__ void df_arm(const uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(df_smem_addr(bar)), "r"(bytes)
               : "memory");
}

// test for the completion of the phase of parity `parity`; the thread may be
// suspended until then, for at most DF_SUSPEND_NS, instead of spinning (a
// spinning warp takes issue slots from the warps that compute)
__device__ __forceinline__ bool df_try_wait(const uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(df_smem_addr(bar)), "r"(parity), "r"(DF_SUSPEND_NS)
      : "memory");
  return ok != 0;
}

// until the ring slot's phase `parity` completes; false after DF_WAIT_NS
__device__ __forceinline__ bool df_wait_slot(const uint64_t* bar, unsigned parity) {
  if (df_try_wait(bar, parity)) return true;
  const unsigned long long t0 = df_clock_ns();
  for (;;) {
    for (int q = 0; q < 8; ++q)
      if (df_try_wait(bar, parity)) return true;
    if (df_clock_ns() - t0 > DF_WAIT_NS) return false;
  }
}

// until the step count at `addr` (any CTA of the cluster) reaches `need`;
// false after DF_WAIT_NS
__device__ __forceinline__ bool df_wait_count(unsigned addr, unsigned need, unsigned* seen = nullptr) {
  unsigned v = df_ld_acquire(addr);
  if (v < need) {
    const unsigned long long t0 = df_clock_ns();
    for (;;) {
      for (int q = 0; q < 64 && v < need; ++q) v = df_ld_acquire(addr);
      if (v >= need) break;
      if (df_clock_ns() - t0 > DF_WAIT_NS) return false;
    }
  }
  if (seen) *seen = v;
  return true;
}

// *p where pred holds, else 0, as one predicated load: nothing waits for the
// value until it is used (a select after the load would stall the warp for
// the memory round trip at once)
__device__ __forceinline__ float df_ldg_or0(const float* p, bool pred) {
  float v;
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ne.u32 q, %2, 0;\n\t"
      "mov.f32 %0, 0f00000000;\n\t"
      "@q ld.global.nc.f32 %0, [%1];\n\t}"
      : "=f"(v)
      : "l"(p), "r"((unsigned)pred));
  return v;
}

// acc0 = l . y.x, acc1 = l . y.y over a ring slot of 32 float4 (four
// partial sums each)
__device__ __forceinline__ void df_dot2i(const float (&l)[32], const float4* y4, float& acc0, float& acc1) {
  float p0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, p1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float4 v = y4[j];
    p0[j & 3] += l[j] * v.x;
    p1[j & 3] += l[j] * v.y;
  }
  acc0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
  acc1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
}

// the two dot products of df_dot2i for the rows l and m at once (each ring
// entry read once)
__device__ __forceinline__ void df_dot4i(const float (&l)[32], const float (&m)[32], const float4* y4, float& a0,
                                         float& a1, float& b0, float& b1) {
  float p0[2] = {0.0f, 0.0f}, p1[2] = {0.0f, 0.0f}, q0[2] = {0.0f, 0.0f}, q1[2] = {0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float4 v = y4[j];
    p0[j & 1] += l[j] * v.x;
    p1[j & 1] += l[j] * v.y;
    q0[j & 1] += m[j] * v.x;
    q1[j & 1] += m[j] * v.y;
  }
  a0 = p0[0] + p0[1];
  a1 = p1[0] + p1[1];
  b0 = q0[0] + q0[1];
  b1 = q1[0] + q1[1];
}

// *p issued here (an asm load the compiler does not move down to its use)
__device__ __forceinline__ int df_ldg_s32(const int32_t* p) {
  int v;
  asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// acc0 = l . y[0:32], acc1 = l . y[32:64] (y 16-byte aligned; four partial
// sums each, for a short dependency chain)
__device__ __forceinline__ void df_dot2(const float (&l)[32], const float* y, float& acc0, float& acc1) {
  const float4* y4 = reinterpret_cast<const float4*>(y);
  float p0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, p1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 a = y4[q], b = y4[8 + q];
    p0[0] += l[4 * q] * a.x;
    p1[0] += l[4 * q] * b.x;
    p0[1] += l[4 * q + 1] * a.y;
    p1[1] += l[4 * q + 1] * b.y;
    p0[2] += l[4 * q + 2] * a.z;
    p1[2] += l[4 * q + 2] * b.z;
    p0[3] += l[4 * q + 3] * a.w;
    p1[3] += l[4 * q + 3] * b.w;
  }
  acc0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
  acc1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
}

__global__ void __launch_bounds__(DF_NT, 1) k_s2_subst_df(const s2::Grid g, S2Work w, const double* b0,
                                                         const double* b1, double* o0, double* o1) {
  // step results, entry j = (rhs 0, rhs 1) of head position j and, forward,
  // the values the step's interchanges move below the head (list entry j:
  // rhs 0, rhs 1)
  __shared__ __align__(16) float4 ring[DF_S][32];
  __shared__ __align__(16) float hsol[64];    // warp 0: the head's values before the triangle solve
  __shared__ __align__(8) uint64_t full[DF_S];
  // this CTA's forward heads k = rank + DF_C u: the values of the rows they
  // need after step k - 2, sent by the rows' owners (entry d: rhs 0, rhs 1 at
  // 2 d, 2 d + 1), in buffer u % 2, completed on hbar[u % 2]
  __shared__ __align__(16) float hbuf[2][128];
  __shared__ __align__(8) uint64_t hbar[2];
  // gdone[t % DF_GD]: the update warps of step t's group have finished it (a
  // phase per use, DF_UWG arrivals)
  __shared__ __align__(8) uint64_t gdone[DF_GD];
  // per update warp: lane -> list entry maps for the scatter of its lookups (-1: none)
  __shared__ int lsc[DF_UW][3][32];
  __shared__ unsigned done;       // steps this CTA's update warps have finished
  __shared__ unsigned done_l;     // the same, published at CTA scope
  __shared__ unsigned abort_all;  // set in every CTA once a wait gave up
  float* const As = reinterpret_cast<float*>(s2_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned rank = sc_cluster_rank();
  constexpr int nb = 32;
  const int N = g.N, nk = (N + nb - 1) / nb, nbl = (nk + DF_C - 1) / DF_C, ldp = g.kl + nb;
  // copy `par` of right-hand side `rhs` at row R, in the shared memory of R's owner
  auto aloc = [&](int par, int rhs, int R) -> float* {
    return As + ((size_t)(2 * par + rhs) * nbl + (size_t)((R >> 5) / DF_C)) * 32 + (R & 31);
  };
  auto fail = [&]() {
    for (unsigned c = 0; c < DF_C; ++c)
      asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(df_mapa(&abort_all, c)), "r"(1u) : "memory");
    w.sc[S2_TOUT] = 1.0;
  };
  // both copies of this CTA's rows from v0s, v1s (FP64 or FP32)
  auto fill = [&](auto v0s, auto v1s) {
    for (int e = tid; e < nbl * 32; e += DF_NT) {
      const int R = ((e >> 5) * DF_C + (int)rank) * 32 + (e & 31);
      const float v0 = R < N ? (float)__ldcg(v0s + R) : 0.0f, v1 = R < N ? (float)__ldcg(v1s + R) : 0.0f;
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        As[(size_t)(2 * par) * nbl * 32 + e] = v0;
        As[(size_t)(2 * par + 1) * nbl * 32 + e] = v1;
      }
    }
  };
  if (tid == 0) {
    done = 0;
    done_l = 0;
    abort_all = 0;
  }
  // bytes a step's result brings into each CTA's ring slot
  auto step_bytes = [&](int t) -> unsigned { return t < 2 * nk ? 512u : 0u; };
  if (tid < DF_S) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(df_smem_addr(&full[tid])) : "memory");
    if (tid < 2 * nk) df_arm(&full[tid], step_bytes(tid));
  }
  if (tid < DF_GD)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(df_smem_addr(&gdone[tid])), "r"(DF_UWG) : "memory");
  for (int i = tid; i < DF_UW * 3 * 32; i += DF_NT) (&lsc[0][0][0])[i] = -1;
  if (tid < 2) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(df_smem_addr(&hbar[tid])) : "memory");
    const int k = (int)rank + DF_C * tid;
    if (k < nk) df_arm(&hbar[tid], 8u * (unsigned)w.smap[(size_t)k * S2_SMAP + 194]);
  }
  fill(b0, b1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  sc_cluster_sync();
  unsigned known = 0;  // warp 0, lane c < DF_C: steps CTA c is known to have finished
  // warp 0: send this lane's entry v of the step's result into every CTA's
  // ring slot t % DF_S by asynchronous stores, which complete the slot's
  // phase there (its publishing warp armed it for 32 entries), once every CTA
  // has finished step t - DF_S (the slot's previous use)
  // this lane's ring entry of slot 0 and slot 0's mbarrier, in each CTA
  unsigned rbase[DF_C], fbase[DF_C];
#pragma unroll
  for (unsigned c = 0; c < DF_C; ++c) {
    rbase[c] = df_mapa(&ring[0][lane], c);
    fbase[c] = df_mapa(&full[0], c);
  }
  auto send = [&](int t, float4 v) -> bool {
    const unsigned need = t >= DF_S ? (unsigned)(t - DF_S + 1) : 0u;
    bool ok = true;
    if (lane < DF_C && known < need) ok = df_wait_count(df_mapa(&done, lane), need, &known);
    if (!__all_sync(0xffffffffu, ok)) return false;
    const unsigned slot = (unsigned)(t % DF_S);
#pragma unroll
    for (unsigned c = 0; c < DF_C; ++c)
      df_st_async4(rbase[c] + slot * (unsigned)sizeof(ring[0]), v, fbase[c] + slot * (unsigned)sizeof(full[0]));
    return true;
  };
  // the publishing warp's lane 0: the first step whose slot it has not consumed
  int tnext = 0;
  // warp 0: how many of this CTA's head buffers it has consumed
  int hcons = 0;
  // after a cluster barrier that ends the sends: wait (briefly) for the slots
  // armed but not consumed, so that no asynchronous store is still on its way
  // into this CTA when it exits (only after a wait gave up)
  auto drain = [&]() {
    if (warp == 0 && lane == 0) {
      for (int u = hcons; u < hcons + 2 && (int)rank + DF_C * u < nk; ++u) {
        const unsigned long long t0 = df_clock_ns();
        while (!df_try_wait(&hbar[u & 1], (unsigned)(u >> 1) & 1u))
          if (df_clock_ns() - t0 > DF_DRAIN_NS) break;
      }
    }
    if (warp == DF_UW + 1 && lane == 0) {
      const int tend = tnext + DF_S < 2 * nk ? tnext + DF_S : 2 * nk;
      for (int t = tnext; t < tend; ++t) {
        const unsigned long long t0 = df_clock_ns();
        while (!df_try_wait(&full[t % DF_S], (unsigned)(t / DF_S) & 1u))
          if (df_clock_ns() - t0 > DF_DRAIN_NS) break;
      }
    }
  };
  // ---- forward: L y = P b ----
  if (warp == 0) {
    for (int k = (int)rank, u = 0; k < nk; k += DF_C, ++u) {
      const int k0 = k * nb, wd = s2::panel_width(g, nb, k0);
      const int32_t* sm = w.smap + (size_t)k * S2_SMAP;
      // lane i follows two rows to their values after step k - 1: the row
      // whose value ends at head position k0 + i, and (i < ntail) tp, the
      // head position whose value the interchanges move to the i-th row of
      // the list past the head; each from the value after step k - 2 of the
      // row panel k - 1's interchanges move there (rh, rt: sent by its owner
      // if step k - 2 updated it, else its input)
      const int ntail = sm[96], tpl = sm[64 + lane];
      const int tp = lane < ntail ? tpl : -1;
      const int rh = sm[128 + lane], rt = sm[160 + lane];
      // the byte count of this buffer's next use (loaded now: the arm after the
      // wait must not wait for memory)
      const unsigned nnext = k + 2 * DF_C < nk ? 8u * (unsigned)w.smap[(size_t)(k + 2 * DF_C) * S2_SMAP + 194] : 0u;
      const bool sh = (((unsigned)sm[192] >> lane) & 1u) != 0, st = (((unsigned)sm[193] >> lane) & 1u) != 0;
      float a0 = 0.0f, a1 = 0.0f, c0 = 0.0f, c1 = 0.0f;
      if (lane < wd && !sh) {
        a0 = (float)__ldcg(b0 + rh);
        a1 = (float)__ldcg(b1 + rh);
      }
      if (tp >= 0 && !st) {
        c0 = (float)__ldcg(b0 + rt);
        c1 = (float)__ldcg(b1 + rt);
      }
      float invr[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) invr[jj] = __ldg(w.inv + (size_t)k * 2048 + lane * 32 + jj);
      // row `lane` of mh (the previous panel's multipliers of the head's rows,
      // through the triangle's inverse), and that panel's multipliers of tp
      // (a head position of panel k: inside panel k - 1's window)
      bool tin = false;
      float mrow[32], lt[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        mrow[jj] = __ldg(w.mh + (size_t)k * 1024 + lane * 32 + jj);
        lt[jj] = 0.0f;
      }
      if (k > 0) {
        const int p0 = k0 - nb;
        const float* Lk = w.Lp + s2::lp_base(g, nb, p0);
        tin = tp >= 0;
        if (tin) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) lt[jj] = __ldg(Lk + (size_t)jj * ldp + (tp - p0));
        }
      }
      // the values sent by their owners (slot u % 2 of this CTA's head buffers)
      bool ok = df_wait_slot(&hbar[u & 1], (unsigned)(u >> 1) & 1u);
      if (ok) {
        if (lane < wd && sh) {
          a0 = hbuf[u & 1][2 * lane];
          a1 = hbuf[u & 1][2 * lane + 1];
        }
        if (tp >= 0 && st) {
          c0 = hbuf[u & 1][64 + 2 * lane];
          c1 = hbuf[u & 1][64 + 2 * lane + 1];
        }
      }
      __syncwarp();
      if (lane == 0 && ok) {
        hcons = u + 1;
        if (k + 2 * DF_C < nk) df_arm(&hbar[u & 1], nnext);
      }
      // inv(L11) times the head's values after step k - 2, before the
      // previous step's result is there
      hsol[lane] = a0;
      hsol[32 + lane] = a1;
      __syncwarp();
      float y0, y1;
      df_dot2(invr, hsol, y0, y1);
      if (k > 0 && ok) {
        const int t = k - 1;
        ok = df_wait_slot(&full[t % DF_S], (unsigned)(t / DF_S) & 1u);
        if (ok) {
          const float4* yp = ring[t % DF_S];
          float acc0, acc1, bcc0, bcc1;
          df_dot4i(mrow, lt, yp, acc0, acc1, bcc0, bcc1);  // lt is zero where tin is false
          y0 -= acc0;
          y1 -= acc1;
          c0 -= bcc0;
          c1 -= bcc1;
        }
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        break;
      }
      if (lane >= wd) y0 = y1 = 0.0f;
      if (!send(k, make_float4(y0, y1, c0, c1))) {
        if (lane == 0) fail();
        break;
      }
      // the forward result, right-hand side of the backward pass (stored
      // after the send, whose release would otherwise wait for these stores)
      if (lane < wd) {
        w.q[k0 + lane] = y0;
        w.q[(size_t)N + k0 + lane] = y1;
      }
    }
  } else if (warp == DF_UW + 1) {
    // publisher: waits for each step's slot and arms its next use, then, once
    // the step's group has finished it, publishes the count of steps done
    // (its release waits for no loads of its own, unlike the update warps')
    for (int s = 0; s < nk; ++s) {
      bool bad = false;
      if (lane == 0) {
        bad = !df_wait_slot(&full[s % DF_S], (unsigned)(s / DF_S) & 1u);
        if (!bad) {
          tnext = s + 1;
          if (s + DF_S < 2 * nk) df_arm(&full[s % DF_S], step_bytes(s + DF_S));
          bad = !df_wait_slot(&gdone[s % DF_GD], (unsigned)(s / DF_GD) & 1u);
        }
        if (!bad) {
          df_st_release_cta(&done_l, (unsigned)(s + 1));
          df_st_release(df_mapa(&done, rank), (unsigned)(s + 1));
        }
      }
      if (__shfl_sync(0xffffffffu, (int)bad, 0)) break;
    }
  } else {
    // update warps: group grp takes the steps of its parity; its warp u the
    // u-th, (u + DF_UWG)-th, ... of this CTA's blocks in a step's window,
    // lane = row in the block; a step's multipliers and interchanges are
    // loaded when the group's previous step is done (two steps ahead)
    const int grp = (warp - 1) / DF_UWG, u = (warp - 1) % DF_UWG;
    // this warp's first block of forward step s (rows 32 (s + 1) .. k0 + H - 1), or -1
    auto first_block = [&](int s) -> int {
      const int k0 = s * nb, H = s2::panel_height(g, s2::panel_width(g, nb, k0), k0);
      const int bf = s + 1, bl = (k0 + H - 1) >> 5;
      const int b = bf + (((int)rank - bf) % DF_C + DF_C) % DF_C + u * DF_C;
      return b <= bl ? b : -1;
    };
    // this group's arrival once its warps have finished step t (after this
    // lane's stores)
    auto finished = [&](int t) {
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(df_smem_addr(&gdone[t % DF_GD])) : "memory");
    };
    // multipliers of step s for this lane's row of block b (zero outside the
    // window and past the panel's width)
    auto load_l = [&](float (&lr)[32], int s, int b) {
      const int k0 = s * nb, wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
      const int r = 32 * b + lane - k0;
      const float* Lk = w.Lp + s2::lp_base(g, nb, k0);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) lr[jj] = df_ldg_or0(Lk + (size_t)jj * ldp + r, b >= 0 && r < H && jj < wd);
    };
    // the step's interchanges past the head: entry `lane` of its list
    // step s's rows past the head that take a head value (entry `lane`), and
    // the rows whose values after step s the head of step s + 2 needs
    // (entries lane and 32 + lane, with their bits of the send masks)
    struct Tail {
      int n, d, r0, r1;
      unsigned m0, m1;
    };
    auto load_tail = [&](int s) -> Tail {
      const int32_t* sm = w.smap + (size_t)s * S2_SMAP;
      Tail t;
      // loaded as they are (entries past the count are masked where used: a
      // select here would stall the warp for the memory round trip)
      t.n = df_ldg_s32(sm + 96);
      t.d = df_ldg_s32(sm + 32 + lane);
      t.r0 = t.r1 = -1;
      t.m0 = t.m1 = 0u;
      if (s + 2 < nk) {
        const int32_t* sp = sm + 2 * S2_SMAP;
        t.r0 = df_ldg_s32(sp + 128 + lane);
        t.r1 = df_ldg_s32(sp + 160 + lane);
        t.m0 = (unsigned)df_ldg_s32(sp + 192);
        t.m1 = (unsigned)df_ldg_s32(sp + 193);
      }
      return t;
    };
    // step s with this warp's first block b and its multipliers lr; false once a wait gave up
    auto step = [&](int s, int bfirst, float (&lr)[32], const Tail& tl) -> bool {
      const int k0 = s * nb, wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
      const int bl = (k0 + H - 1) >> 5;
      const float4* y = ring[s % DF_S];
      // where the new values go: the head of step s + 2 (its owner's buffer u % 2)
      const unsigned ho = (unsigned)((s + 2) % DF_C);
      const int hslot = ((s + 2) / DF_C) & 1;
      // row R's entry in the step's list of rows past the head that take a
      // head value (-1: none; the value came with the step's result), and the
      // entries of the head's list that row R's new value serves (masks over
      // d and 32 + d); found before the wait, for the first block
      int* const sc = lsc[warp - 1][0];
      auto lists = [&](int b, int& qi, unsigned& pm0, unsigned& pm1) {
        // each entry lane writes its index at its row's lane (rows in a list are distinct)
        const bool et = lane < tl.n && (tl.d >> 5) == b;
        if (et) sc[tl.d & 31] = lane;
        __syncwarp();
        qi = sc[lane];
        __syncwarp();
        if (et) sc[tl.d & 31] = -1;
        pm0 = __ballot_sync(0xffffffffu, ((tl.m0 >> lane) & 1u) && (tl.r0 >> 5) == b);
        pm1 = __ballot_sync(0xffffffffu, ((tl.m1 >> lane) & 1u) && (tl.r1 >> 5) == b);
      };
      int qi = -1;
      unsigned pm0 = 0u, pm1 = 0u;
      if (bfirst >= 0 && bfirst <= bl) lists(bfirst, qi, pm0, pm1);
      bool ok = df_wait_slot(&full[s % DF_S], (unsigned)(s / DF_S) & 1u);
      // the rows' values after step s - 1: the other group's step
      if (ok && s >= 1) ok = df_wait_slot(&gdone[(s - 1) % DF_GD], (unsigned)((s - 1) / DF_GD) & 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        return false;
      }
      for (int b = bfirst; b >= 0 && b <= bl; b += DF_UWG * DF_C) {
        if (b != bfirst) {  // a window wider than DF_UWG x DF_C blocks
          load_l(lr, s, b);
          lists(b, qi, pm0, pm1);
        }
        const int R = 32 * b + lane;
        const bool in = R - k0 < H;
        float v0 = 0.0f, v1 = 0.0f;
        if (in) {
          const int par = s & 1;
          if (qi < 0) {
            v0 = *aloc(par, 0, R);
            v1 = *aloc(par, 1, R);
          } else {
            v0 = y[qi].z;
            v1 = y[qi].w;
          }
          float acc0 = 0.0f, acc1 = 0.0f;
          df_dot2i(lr, y, acc0, acc1);
          v0 -= acc0;
          v1 -= acc1;
          *aloc(par ^ 1, 0, R) = v0;
          *aloc(par ^ 1, 1, R) = v1;
        }
        // send the new values that the head of step s + 2 takes from this
        // block: the entry lanes (bits of pm) name their rows, scattered to the
        // rows' lanes, so each lane sends its own (one entry at a time where
        // two entries share a row)
        auto send_part = [&](unsigned pm, int rs, int base, int* scp) {
          if (pm == 0u) return;
          const bool e = ((pm >> lane) & 1u) != 0u;
          const unsigned same = __match_any_sync(0xffffffffu, e ? rs : -1 - lane);
          if (__any_sync(0xffffffffu, e && __popc(same) > 1)) {
            for (unsigned m = pm; m; m &= m - 1) {
              const int q = __ffs(m) - 1;
              if (__shfl_sync(0xffffffffu, rs, q) == R && in)
                df_st_async2(df_mapa(&hbuf[hslot][2 * (base + q)], ho), v0, v1, df_mapa(&hbar[hslot], ho));
            }
            return;
          }
          if (e) scp[rs & 31] = lane;
          __syncwarp();
          const int q = scp[lane];
          if (q >= 0 && in) df_st_async2(df_mapa(&hbuf[hslot][2 * (base + q)], ho), v0, v1, df_mapa(&hbar[hslot], ho));
          __syncwarp();
          if (e) scp[rs & 31] = -1;
        };
        send_part(pm0, tl.r0, 0, sc + 32);
        send_part(pm1, tl.r1, 32, sc + 64);
      }
      finished(s);
      return true;
    };
    float lr[32];
    int bc = -1;
    Tail tc{0, -1, -1, -1, 0u, 0u};
    if (grp < nk) {
      bc = first_block(grp);
      tc = load_tail(grp);
      load_l(lr, grp, bc);
    }
    for (int s = grp; s < nk; s += 2) {
      if (!step(s, bc, lr, tc)) break;
      if (s + 2 < nk) {
        bc = first_block(s + 2);
        tc = load_tail(s + 2);
        load_l(lr, s + 2, bc);
      }
    }
  }
  // ---- backward: U x = y, steps t = nk + it for panel k = nk - 1 - it ----
  sc_cluster_sync();
  if (abort_all) {
    drain();
    sc_cluster_sync();
    return;
  }
  fill(w.q, w.q + N);
  __syncthreads();
  if (warp == 0) {
    const int klast = nk - 1;
    for (int k = klast - ((klast - (int)rank) % DF_C + DF_C) % DF_C; k >= 0; k -= DF_C) {
      const int it = klast - k, t = nk + it;
      const int k0 = k * nb, wd = s2::panel_width(g, nb, k0);
      const int R = k0 + lane;
      float invr[32], ur[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) invr[jj] = __ldg(w.inv + (size_t)k * 2048 + 1024 + lane * 32 + jj);
      // row R after step it - 1: less U(R, columns of panel k + 1) times x_{k+1}
      const int kn0 = k0 + nb, wdn = k + 1 < nk ? s2::panel_width(g, nb, kn0) : 0;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) ur[jj] = (lane < wd && jj < wdn) ? s2::umul(g, w.AB, R, kn0 + jj) : 0.0f;
      bool ok = true;
      if (it >= 2 && df_ld_acquire_cta(&done_l) < (unsigned)(t - 1)) {
        // this CTA's update warps finish step t - 2 (a count at CTA scope)
        const unsigned long long t0 = df_clock_ns();
        while (df_ld_acquire_cta(&done_l) < (unsigned)(t - 1))
          if (df_clock_ns() - t0 > DF_WAIT_NS) {
            ok = false;
            break;
          }
      }
      float a0 = 0.0f, a1 = 0.0f;
      if (lane < wd) {
        a0 = *aloc((it + 1) & 1, 0, R);
        a1 = *aloc((it + 1) & 1, 1, R);
      }
      if (it > 0 && ok) {
        ok = df_wait_slot(&full[(t - 1) % DF_S], (unsigned)((t - 1) / DF_S) & 1u);
        if (ok && lane < wd) {
          float acc0 = 0.0f, acc1 = 0.0f;
          df_dot2i(ur, ring[(t - 1) % DF_S], acc0, acc1);
          a0 -= acc0;
          a1 -= acc1;
        }
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        break;
      }
      // x = (inverse of U11) times the head's values
      hsol[lane] = a0;
      hsol[32 + lane] = a1;
      __syncwarp();
      float x0, x1;
      df_dot2(invr, hsol, x0, x1);
      if (lane >= wd) x0 = x1 = 0.0f;
      if (!send(t, make_float4(x0, x1, 0.0f, 0.0f))) {
        if (lane == 0) fail();
        break;
      }
      if (lane < wd) {
        o0[R] = x0;
        o1[R] = x1;
      }
    }
  } else if (warp == DF_UW + 1) {
    for (int it = 0; it < nk; ++it) {
      const int t = nk + it;
      bool bad = false;
      if (lane == 0) {
        bad = !df_wait_slot(&full[t % DF_S], (unsigned)(t / DF_S) & 1u);
        if (!bad) {
          tnext = t + 1;
          if (t + DF_S < 2 * nk) df_arm(&full[t % DF_S], step_bytes(t + DF_S));
          bad = !df_wait_slot(&gdone[t % DF_GD], (unsigned)(t / DF_GD) & 1u);
        }
        if (!bad) {
          df_st_release_cta(&done_l, (unsigned)(t + 1));
          df_st_release(df_mapa(&done, rank), (unsigned)(t + 1));
        }
      }
      if (__shfl_sync(0xffffffffu, (int)bad, 0)) break;
    }
  } else {
    // the groups take the backward steps t = nk + it of their parity
    const int grp = (warp - 1) / DF_UWG, u = (warp - 1) % DF_UWG;
    // rows lo .. k0 - 1 of backward step it (panel k = nk - 1 - it): this warp's first block, or -1
    auto first_block = [&](int it) -> int {
      const int k = nk - 1 - it, k0 = k * nb;
      const int lo = k0 - g.kl - g.ku > 0 ? k0 - g.kl - g.ku : 0;
      const int bf = lo >> 5, bl = k - 1;
      const int b = bf + (((int)rank - bf) % DF_C + DF_C) % DF_C + u * DF_C;
      return b <= bl ? b : -1;
    };
    auto finished = [&](int t) {
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(df_smem_addr(&gdone[t % DF_GD])) : "memory");
    };
    auto load_u = [&](float (&ur)[32], int it, int b) {
      const int k = nk - 1 - it, k0 = k * nb, wd = s2::panel_width(g, nb, k0);
      const int lo = k0 - g.kl - g.ku > 0 ? k0 - g.kl - g.ku : 0;
      const int R = 32 * b + lane;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj)
        ur[jj] = df_ldg_or0(w.AB + s2::band_at(g, R, k0 + jj),
                            b >= 0 && R >= lo && jj < wd && s2::in_band(g, R, k0 + jj));  // U(R, k0 + jj)
    };
    auto step = [&](int it, int bfirst, float (&ur)[32]) -> bool {
      const int t = nk + it, k = nk - 1 - it, k0 = k * nb;
      const int lo = k0 - g.kl - g.ku > 0 ? k0 - g.kl - g.ku : 0;
      const float4* x = ring[t % DF_S];
      bool ok = df_wait_slot(&full[t % DF_S], (unsigned)(t / DF_S) & 1u);
      if (ok) ok = df_wait_slot(&gdone[(t - 1) % DF_GD], (unsigned)((t - 1) / DF_GD) & 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        return false;
      }
      for (int b = bfirst; b >= 0 && b <= k - 1; b += DF_UWG * DF_C) {
        if (b != bfirst) load_u(ur, it, b);
        const int R = 32 * b + lane;
        if (R >= lo) {
          const int par = it & 1;
          float acc0 = 0.0f, acc1 = 0.0f;
          df_dot2i(ur, x, acc0, acc1);
          const float v0 = *aloc(par, 0, R), v1 = *aloc(par, 1, R);
          *aloc(par ^ 1, 0, R) = v0 - acc0;
          *aloc(par ^ 1, 1, R) = v1 - acc1;
        }
      }
      finished(t);
      return true;
    };
    float ur[32];
    const int it0 = (nk + grp) & 1;  // first backward step of this group's parity (t = nk + it)
    int bc = -1;
    if (it0 < nk) {
      bc = first_block(it0);
      load_u(ur, it0, bc);
    }
    for (int it = it0; it < nk; it += 2) {
      if (!step(it, bc, ur)) break;
      if (it + 2 < nk) {
        bc = first_block(it + 2);
        load_u(ur, it + 2, bc);
      }
    }
  }
  sc_cluster_sync();
  drain();
  sc_cluster_sync();
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

// The same refinement residuals without the stored Jacobian (on Newton steps
// that keep an earlier factorisation): B v from central differences of the
// FP64 residual along v, (R(x + e v) - R(x - e v)) / (2 e), e = S2_JV_H
// max(1, |x|) / |v| (maxima over the unknowns), and the total-mass row as in
// bmv_row.  The differences use y0, y1 (the states) and s0, s1 (their
// residuals), which the sweep overwrites later.
constexpr double S2_JV_H = 1e-6;
// from this many cells on (measured: slower below ~3 000 cells, where the
// Jacobian is cheaper than the extra launches; 100 x 100 gains 5 %, a solve
// from an earlier factorisation 12 %)
constexpr int S2_JV_MIN_CELLS = 4096;

__global__ void __launch_bounds__(S2_UPD_NT) k_s2_jveps(const s2::Grid g, S2Work w) {
  __shared__ double red[S2_UPD_NT];
  double mx = 0.0, m0 = 0.0, m1 = 0.0;
  for (int u = threadIdx.x; u < g.N; u += S2_UPD_NT) {
    mx = fmax(mx, fabs(w.x[u]));
    m0 = fmax(m0, fabs(w.v0[u]));
    m1 = fmax(m1, fabs(w.v1[u]));
  }
  mx = s2_block_max<S2_UPD_NT>(mx, red);
  m0 = s2_block_max<S2_UPD_NT>(m0, red);
  m1 = s2_block_max<S2_UPD_NT>(m1, red);
  if (threadIdx.x == 0) {
    const double h = S2_JV_H * fmax(1.0, mx);
    w.sc[S2_EPS0] = m0 > 0.0 ? h / m0 : 1.0;
    w.sc[S2_EPS1] = m1 > 0.0 ? h / m1 : 1.0;
  }
}

// y0 = x + e v_c, y1 = x - e v_c
__global__ void k_s2_jvx(const s2::Grid g, S2Work w, int c) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= g.N) return;
  const double e = w.sc[c ? S2_EPS1 : S2_EPS0], v = (c ? w.v1 : w.v0)[u];
  w.y0[u] = w.x[u] + e * v;
  w.y1[u] = w.x[u] - e * v;
}

// s0 = R(y0), s1 = R(y1) (the total-mass row is replaced below)
__global__ void k_s2_jvres(const s2::Grid g, S2Work w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.n) return;
  int i, j;
  s2::cell_of_band(g, b, i, j);
  s2::cell_residual(g, s2::View{w.y0, -1, 0, 0.0}, i, j, 0.0, w.s0 + s2::NV * b);
  s2::cell_residual(g, s2::View{w.y1, -1, 0, 0.0}, i, j, 0.0, w.s1 + s2::NV * b);
}

// b_c = rhs_c - B v_c
__global__ void k_s2_jvb(const s2::Grid g, S2Work w, int c) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= g.N) return;
  const double e = w.sc[c ? S2_EPS1 : S2_EPS0];
  const double* v = c ? w.v1 : w.v0;
  const double bv = u == s2::mass_row(g) ? s2::mass_scale(g, 1, 0) * v[u] / g.n : (w.s0[u] - w.s1[u]) / (2.0 * e);
  (c ? w.b1 : w.b0)[u] = (c ? w.rhs1 : w.rhs0)[u] - bv;
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
  // the register-row panels: multipliers of up to 3 x 512 rows
  static bool rot_set = false;
  if (!rot_set) {
    const int cap = (int)(sizeof(float) * 32 * 3 * S2_PNL_NT);
    cudaFuncSetAttribute(k_s2_panel_rot<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    cudaFuncSetAttribute(k_s2_panel_rot<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    cudaFuncSetAttribute(k_s2_panel_rot<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    rot_set = true;
  }
}

}  // namespace

// One substitution (two right-hand sides): on a cluster of SC_CL CTAs where
// the device can run one, else on one CTA (k_s2_subst).
cudaError_t s2_subst(const s2::Grid& g, const S2Work& w, double* b0, double* b1, double* o0, double* o1,
                     size_t sm_subst, cudaStream_t st) {
  // the data-flow form where its rows fit the cluster's shared memory
  static int df_ok = -1;  // per process: 1 when a DF_C-CTA cluster of k_s2_subst_df fits
  static size_t df_set = 0;
  const size_t nk = (size_t)(g.N + 31) / 32;
  const size_t sm_df = sizeof(float) * 4 * 32 * ((nk + DF_C - 1) / DF_C);
  if (w.nb == 32 && sm_df <= S2_DF_SMEM_CAP) {
    if (df_set < sm_df) {
      if (cudaFuncSetAttribute(k_s2_subst_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S2_DF_SMEM_CAP) ==
          cudaSuccess)
        df_set = S2_DF_SMEM_CAP;
      cudaGetLastError();
    }
    cudaLaunchConfig_t dc = {};
    cudaLaunchAttribute da[1];
    da[0].id = cudaLaunchAttributeClusterDimension;
    da[0].val.clusterDim.x = DF_C;
    da[0].val.clusterDim.y = 1;
    da[0].val.clusterDim.z = 1;
    dc.gridDim = dim3(DF_C);
    dc.blockDim = dim3(DF_NT);
    dc.dynamicSmemBytes = S2_DF_SMEM_CAP;
    dc.stream = st;
    dc.attrs = da;
    dc.numAttrs = 1;
    if (df_ok < 0) {
      int n = 0;
      df_ok = (df_set >= S2_DF_SMEM_CAP && cudaOccupancyMaxActiveClusters(&n, k_s2_subst_df, &dc) == cudaSuccess &&
               n >= 1)
                  ? 1
                  : 0;
      cudaGetLastError();
    }
    if (df_ok) {
      dc.dynamicSmemBytes = sm_df;
      return cudaLaunchKernelEx(&dc, k_s2_subst_df, g, w, (const double*)b0, (const double*)b1, o0, o1);
    }
  }
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
                   int n_m, double tol, double* info, int* singular, int reuse, int warm, cudaStream_t st) {
  s2::Grid g = s2::make_grid(cp.nx, cp.ny, cp.dx, cp.dy, cp.d_r, cp.omega, cp.mu_ref, cp.z_rot, cp.kappa_t,
                             cp.kappa_r, fields, hot);
  if (cp.mesh == 2) s2::set_edges(g, cp.xe, cp.ye, cp.lx * cp.ly);  // the wall-refined grid (device edges)
  if (cp.mesh == 1) s2::set_annulus(g, cp.rt);  // the annulus (device ring radii)
  const S2Work w = s2_carve(g, work);
  if (w.nb == 0) return (int)cudaErrorInvalidValue;
  const int nb = w.nb;
  const size_t hmax = (size_t)g.kl + nb;
  const size_t sm_panel = sizeof(float) * nb * hmax;
  // trailing columns per CTA of the trailing update: up to 8, as shared
  // memory allows (column segments of hmax rows; 8 beat 16 by 5 % at 100 x
  // 100: twice the CTAs, each with half the serial work)
  int cbt = (int)(S2_SMEM_CAP / (sizeof(float) * hmax));
  if (cbt > 8) cbt = 8;
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
  k_s2_init<<<1, S2_NT, 0, st>>>(g, w, warm);
  // The factorisation of the first Newton step (with `reuse`, the one the
  // work area holds from the previous solve) is reused while the updates
  // keep shrinking (by half or more per step), with more refinement sweeps
  // against each step's fresh FP64 Jacobian; otherwise the next step
  // refactorises.
  bool refactor = !reuse;
  double dm_prev = 0.0;
  for (int it = 0; it < n_m; ++it) {
    k_s2_mass<<<1, S2_NT, 0, st>>>(g, w);
    k_s2_res<<<cell_grid, nt, 0, st>>>(g, w);
    // on large grids the Jacobian only where it is factorised: a step that
    // keeps an earlier factorisation refines with directional differences
    const bool jv = !refactor && g.n >= S2_JV_MIN_CELLS;
    if (refactor) cudaMemsetAsync(w.AB, 0, sizeof(float) * (size_t)g.ld * g.N, st);
    if (!jv) k_s2_jac<<<jac_grid, nt, 0, st>>>(g, w, refactor ? 1 : 0);
    if (refactor) {
      for (int k0 = 0; k0 < g.N; k0 += nb) {
        const int wd = s2::panel_width(g, nb, k0), H = s2::panel_height(g, wd, k0);
        // rows in registers (up to 3 a thread, 512 threads) where they fit
        const int rpt = (H + S2_PNL_NT - 1) / S2_PNL_NT;
        const int tpb = rpt <= 3 ? (H + 32 * rpt - 1) / (32 * rpt) * 32 : 0;
        const size_t smr = tpb ? sizeof(float) * 32 * (size_t)tpb * rpt : 0;
        if (nb == 32 && rpt == 1)
          k_s2_panel_rot<1><<<1, tpb, smr, st>>>(g, w, k0);
        else if (nb == 32 && rpt == 2)
          k_s2_panel_rot<2><<<1, tpb, smr, st>>>(g, w, k0);
        else if (nb == 32 && rpt == 3)
          k_s2_panel_rot<3><<<1, tpb, smr, st>>>(g, w, k0);
        else
          k_s2_panel<<<1, S2_PNL_NT, sizeof(float) * (size_t)wd * H, st>>>(g, w, k0);
        const int ntrail = s2::trail_last(g, k0, wd) - (k0 + wd) + 1;
        if (ntrail > 0)
          k_s2_trail<<<(ntrail + cbt - 1) / cbt, S2_NT, sizeof(float) * (size_t)cbt * H, st>>>(g, w, k0, cbt);
      }
      const int nk = (g.N + nb - 1) / nb;
      k_s2_sprep<<<(nk + SP_WPB - 1) / SP_WPB, SP_WPB * 32, 0, st>>>(g, w);
      k_s2_spush<<<(nk + SP_WPB - 1) / SP_WPB, SP_WPB * 32, 0, st>>>(g, w);
    }
    const int nsweep = refactor ? S2_NREF : S2_NREF_REUSE;
    k_s2_prep<<<vec_grid, nt, 0, st>>>(g, w);
    cudaError_t le = s2_subst(g, w, w.b0, w.b1, w.v0, w.v1, sm_subst, st);
    for (int r = 0; r < nsweep && le == cudaSuccess; ++r) {
      if (!jv) {
        k_s2_bmv<<<vec_grid, nt, 0, st>>>(g, w);
      } else {
        k_s2_jveps<<<1, S2_UPD_NT, 0, st>>>(g, w);
        for (int c = 0; c < 2; ++c) {
          k_s2_jvx<<<vec_grid, nt, 0, st>>>(g, w, c);
          k_s2_jvres<<<cell_grid, nt, 0, st>>>(g, w);
          k_s2_jvb<<<vec_grid, nt, 0, st>>>(g, w, c);
        }
      }
      le = s2_subst(g, w, w.b0, w.b1, w.s0, w.s1, sm_subst, st);
      k_s2_add<<<vec_grid, nt, 0, st>>>(g, w);
    }
    if (le != cudaSuccess) return (int)le;
    k_s2_newton<<<1, S2_UPD_NT, 0, st>>>(g, w, n_m, tol);
    cudaMemcpyAsync(sc, w.sc, sizeof(double) * (S2_TOUT + 1), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    if (sc[S2_TOUT] != 0.0) return S2_TIMEOUT_RC;
    if (sc[S2_DONE] != 0.0) break;
    refactor = it > 0 && !(sc[S2_DMAX] <= 0.5 * dm_prev);
    dm_prev = sc[S2_DMAX];
  }
  k_s2_mass<<<1, S2_NT, 0, st>>>(g, w);
  k_s2_res<<<cell_grid, nt, 0, st>>>(g, w);
  k_s2_final<<<1, S2_NT, 0, st>>>(g, w, out, info);
  cudaMemcpyAsync(sc, w.sc, sizeof(double) * (S2_TOUT + 1), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  // a solve that started from an earlier factorisation and did not
  // converge is repeated from a fresh one
  if ((reuse || warm) && sc[S2_STATUS] != 0.0)
    return launch_synth2d(cp, fields, hot, out, work, n_m, tol, info, singular, 0, 0, st);
  if (singular) *singular = sc[S2_SING] != 0.0;
  return 0;
}

}  // namespace dsmc
