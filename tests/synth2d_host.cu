// Host build of the 2D synthetic solve's __host__ __device__ functions
// (paper_2501_10965_gb300/csrc/dsmc_synth2d.cuh), run in the order of the
// GPU kernels with one thread per loop: the blocked FP32 banded LU with
// partial pivoting, the FP32 substitutions, FP64 refinement and Newton's
// method.  Test infrastructure: compiled by tests/test_synth2d_host.py with
// nvcc as host code and compared with the oracle and with numpy.
#include <vector>
#include <cstdio>
#include <algorithm>
#include "dsmc_synth2d.cuh"
using namespace dsmc::s2;

// the wall-refined grid's edges for the calls that follow (null: uniform)
static const double* g_xe = nullptr;
static const double* g_ye = nullptr;
static double g_area = 0.0;
extern "C" void h_set_edges(const double* xe, const double* ye, double area) {
  g_xe = xe;
  g_ye = ye;
  g_area = area;
}
// the annulus's ring edges for the calls that follow (null: a box)
static const double* g_R = nullptr;
extern "C" void h_set_annulus(const double* R) { g_R = R; }
static Grid G(int nx, int ny, double dx, double dy, const double* c, const double* F, const double* hot) {
  Grid g = make_grid(nx, ny, dx, dy, c[0], c[1], c[2], c[3], c[4], c[5], F, hot);
  if (g_xe) set_edges(g, g_xe, g_ye, g_area);
  if (g_R) set_annulus(g, g_R);
  return g;
}
static void residual_all(const Grid& g, const double* xb, double* Rb) {
  double sx = 0, sd = 0;
  for (int b = 0; b < g.n; ++b) { int i, j; cell_of_band(g, b, i, j); sx += xb[NV * b] * mass_scale(g, i, j); }
  for (int c = 0; c < g.n; ++c) sd += g.F[(size_t)c * 18] * mass_scale(g, c % g.nx, c / g.nx);
  const double mrow = (sx - sd) / g.n;
  View X{xb, -1, 0, 0.0};
  for (int b = 0; b < g.n; ++b) { int i, j; cell_of_band(g, b, i, j); cell_residual(g, X, i, j, mrow, Rb + NV * b); }
}
struct F32 {
  std::vector<float> AB, Lm, ud;
  std::vector<int32_t> piv;
};
static size_t lp_size(const Grid& g, int nb) { return (size_t)((g.N + nb - 1) / nb) * nb * (g.kl + nb); }

static int factor(const Grid& g, int nb, F32& f) {
  int sing = 0;
  std::vector<float> P, Ls, Cs;
  for (int k0 = 0; k0 < g.N; k0 += nb) {
    const int w = panel_width(g, nb, k0), H = panel_height(g, w, k0);
    P.assign((size_t)w * H, 0.f);
    panel_load(g, f.AB.data(), k0, w, H, P.data(), 0, 1);
    for (int j = 0; j < w; ++j) {
      const int p = panel_pivot_seq(g, P.data(), H, j);
      f.piv[k0 + j] = k0 + p;
      if (P[(size_t)j * H + p] == 0.0f) sing = 1;
      panel_swap(P.data(), H, w, j, p, 0, 1);
      panel_scale(g, P.data(), H, j, 0, 1);
      panel_rank1(g, P.data(), H, w, j, 0, 1, 1);
    }
    panel_store(g, nb, f.AB.data(), f.Lm.data(), f.ud.data(), k0, w, H, P.data(), 0, 1);
    const int c0 = k0 + w, c1 = trail_last(g, k0, w);
    const int CB = 8;
    for (int cf = c0; cf <= c1; cf += CB) {
      const int nc = std::min(CB, c1 - cf + 1);
      Ls.assign((size_t)w * H, 0.f); Cs.assign((size_t)nc * H, 0.f);
      trail_load_l(g, nb, f.Lm.data(), k0, w, H, Ls.data(), 0, 1);
      trail_load_cols(g, f.AB.data(), k0, H, cf, nc, Cs.data(), 0, 1);
      trail_swaps(f.piv.data(), k0, w, H, nc, Cs.data(), 0, 1);
      for (int j = 0; j < w; ++j) trail_l11_step(Ls.data(), w, H, nc, j, Cs.data(), 0, 1);
      trail_l21(Ls.data(), w, H, nc, Cs.data(), 0, 1);
      trail_store(g, f.AB.data(), k0, H, cf, nc, Cs.data(), 0, 1);
    }
  }
  return sing;
}

// two right-hand sides b0, b1 (consumed); outputs o0, o1 -- arithmetic in FP32
static void subst(const Grid& g, int nb, const F32& f, double* b0, double* b1, double* y0, double* y1, double* o0, double* o1) {
  for (int k0 = 0; k0 < g.N; k0 += nb) {
    const int w = panel_width(g, nb, k0), H = panel_height(g, w, k0);
    std::vector<float> s0(H), s1(H);
    for (int r = 0; r < H; ++r) { s0[r] = (float)b0[k0 + r]; s1[r] = (float)b1[k0 + r]; }
    for (int j = 0; j < w; ++j) { const int p = f.piv[k0 + j] - k0; std::swap(s0[j], s0[p]); std::swap(s1[j], s1[p]); }
    for (int j = 0; j < w; ++j) for (int i = j + 1; i < w; ++i) {
      const float l = lmul(g, nb, f.Lm.data(), k0, i, j); s0[i] -= l * s0[j]; s1[i] -= l * s1[j]; }
    for (int i = 0; i < w; ++i) { y0[k0 + i] = s0[i]; y1[k0 + i] = s1[i]; }
    for (int r = w; r < H; ++r) {
      float a0 = 0, a1 = 0;
      for (int j = 0; j < w; ++j) { const float l = lmul(g, nb, f.Lm.data(), k0, r, j); a0 += l * s0[j]; a1 += l * s1[j]; }
      b0[k0 + r] = s0[r] - a0; b1[k0 + r] = s1[r] - a1;
    }
  }
  const int last = ((g.N - 1) / nb) * nb;
  for (int k0 = last; k0 >= 0; k0 -= nb) {
    const int w = panel_width(g, nb, k0);
    const int lo = std::max(0, k0 - g.kl - g.ku);
    std::vector<float> x0(w), x1(w), a0(w), a1(w);
    for (int i = 0; i < w; ++i) { a0[i] = (float)y0[k0 + i]; a1[i] = (float)y1[k0 + i]; }
    for (int j = w - 1; j >= 0; --j) {
      x0[j] = a0[j] / f.ud[k0 + j]; x1[j] = a1[j] / f.ud[k0 + j];
      for (int i = 0; i < j; ++i) { const float u = umul(g, f.AB.data(), k0 + i, k0 + j); a0[i] -= u * x0[j]; a1[i] -= u * x1[j]; }
    }
    for (int j = 0; j < w; ++j) { o0[k0 + j] = x0[j]; o1[k0 + j] = x1[j]; }
    for (int r = lo; r < k0; ++r) {
      float s0 = 0, s1 = 0;
      for (int j = 0; j < w; ++j) { const float u = umul(g, f.AB.data(), r, k0 + j); s0 += u * x0[j]; s1 += u * x1[j]; }
      y0[r] = (float)y0[r] - s0; y1[r] = (float)y1[r] - s1;
    }
  }
}

// Newton as the GPU runs it: a fresh factorisation with nref refinement
// sweeps; with reuse, later steps keep the factorisation (nref_reuse sweeps
// against their fresh FP64 Jacobian) while each update is at most half the
// previous one.
extern "C" int h_solve_blk(int nx, int ny, double dx, double dy, const double* c, const double* F, const double* hot,
                           int n_m, double tol, int nb, int nref, int reuse, int nref_reuse, double* out, int* iters,
                           double* resid, int* status, int* nfactor) {
  Grid g = G(nx, ny, dx, dy, c, F, hot);
  const int N = g.N;
  F32 f; f.AB.assign((size_t)N * g.ld, 0.f); f.Lm.assign(lp_size(g, nb), 0.f); f.ud.assign(N, 0.f); f.piv.assign(N, 0);
  std::vector<double> x(N), R(N), Jc((size_t)g.n * NSTENCIL * NV * NV), rhs0(N), rhs1(N), b0(N), b1(N), y0(N), y1(N),
      v0(N), v1(N), s0(N), s1(N), d(N);
  for (int b = 0; b < g.n; ++b) {
    int i, j; cell_of_band(g, b, i, j);
    const double* D = F + (size_t)(j * nx + i) * 18;
    x[NV * b + 0] = D[0]; x[NV * b + 1] = D[1]; x[NV * b + 2] = D[2]; x[NV * b + 3] = D[4]; x[NV * b + 4] = D[5];
  }
  const int mr = mass_row(g);
  int st = 1, it = 0, sing = 0, nf = 0;
  bool refac = true;
  double dm_prev = 0.0;
  for (it = 1; it <= n_m; ++it) {
    residual_all(g, x.data(), R.data());
    if (refac) std::fill(f.AB.begin(), f.AB.end(), 0.f);
    for (int b = 0; b < g.n; ++b) for (int s = 0; s < NSTENCIL; ++s) for (int v = 0; v < NV; ++v)
      jacobian_entries(g, x.data(), b, s, v, refac ? f.AB.data() : nullptr, Jc.data());
    if (refac) {
      if (mr >= 0) f.AB[band_at(g, mr, mr)] = (float)(mass_scale(g, 1, 0) / g.n);
      sing |= factor(g, nb, f);
      ++nf;
    }
    const int nsw = refac ? nref : nref_reuse;
    for (int u = 0; u < N; ++u) { rhs0[u] = -R[u]; rhs1[u] = u == mr ? 1.0 : 0.0; b0[u] = rhs0[u]; b1[u] = rhs1[u]; }
    subst(g, nb, f, b0.data(), b1.data(), y0.data(), y1.data(), v0.data(), v1.data());
    for (int rr = 0; rr < nsw; ++rr) {
      for (int u = 0; u < N; ++u) { b0[u] = rhs0[u] - bmv_row(g, Jc.data(), v0.data(), u); b1[u] = rhs1[u] - bmv_row(g, Jc.data(), v1.data(), u); }
      subst(g, nb, f, b0.data(), b1.data(), y0.data(), y1.data(), s0.data(), s1.data());
      for (int u = 0; u < N; ++u) { v0[u] += s0[u]; v1[u] += s1[u]; }
    }
    double wz = 0, wy = 0;
    for (int b = 0; b < g.n; ++b) if (NV * b != mr) {
      int i, j; cell_of_band(g, b, i, j); const double ms = mass_scale(g, i, j);
      wz += v0[NV * b] * ms; wy += v1[NV * b] * ms; }
    wz /= g.n; wy /= g.n;
    const double fct = wz / (1.0 + wy);
    for (int u = 0; u < N; ++u) d[u] = v0[u] - v1[u] * fct;
    double lam = 1.0; bool ok = false;
    for (int h = 0; h < 60 && !ok; ++h) {
      ok = true;
      for (int u = 0; u < N; ++u) {
        const double xn = x[u] + lam * d[u]; const int v = u % NV;
        if (!std::isfinite(xn) || ((v == 0 || v >= 3) && xn <= 0.0)) { ok = false; break; }
      }
      if (!ok) lam *= 0.5;
    }
    if (!ok) { st = 2; break; }
    double dm = 0;
    for (int u = 0; u < N; ++u) { dm = std::max(dm, std::fabs(lam * d[u]) / std::max(std::fabs(x[u]), 1e-3)); x[u] += lam * d[u]; }
    if (dm < tol) { st = 0; break; }
    refac = !reuse || (it > 1 && !(dm <= 0.5 * dm_prev));
    dm_prev = dm;
  }
  if (it > n_m) it = n_m;
  residual_all(g, x.data(), R.data());
  double rm = 0; for (int u = 0; u < N; ++u) rm = std::max(rm, std::fabs(R[u]));
  for (int b = 0; b < g.n; ++b) {
    int i, j; cell_of_band(g, b, i, j); const int cn = j * nx + i;
    const double* D = F + (size_t)cn * 18;
    double* o = out + (size_t)cn * 6;
    o[0] = x[NV * b]; o[1] = x[NV * b + 1]; o[2] = x[NV * b + 2]; o[3] = D[3]; o[4] = x[NV * b + 3]; o[5] = x[NV * b + 4];
  }
  *iters = it; *resid = rm; *status = st | (sing ? 4 : 0);
  if (nfactor) *nfactor = nf;
  return 0;
}

// factor + solve a band matrix given densely (A row-major N x N, within kl of the diagonal)
extern "C" int h_band_test(int N, int kl, int nb, const double* A, const double* b, double* x) {
  Grid g{};
  g.N = N; g.kl = kl; g.ku = kl; g.ld = 2 * kl + kl + 1;
  F32 f; f.AB.assign((size_t)N * g.ld, 0.f); f.Lm.assign(lp_size(g, nb), 0.f); f.ud.assign(N, 0.f); f.piv.assign(N, 0);
  for (int r = 0; r < N; ++r) for (int c = 0; c < N; ++c) if (std::abs(r - c) <= kl) f.AB[band_at(g, r, c)] = (float)A[(size_t)r * N + c];
  factor(g, nb, f);
  std::vector<double> b0(b, b + N), b1(N, 0.0), y0(N), y1(N), o1(N);
  subst(g, nb, f, b0.data(), b1.data(), y0.data(), y1.data(), x, o1.data());
  return 0;
}

extern "C" int h_residual(int nx, int ny, double dx, double dy, const double* c, const double* F, const double* hot,
                          const double* x_nat, double* R_nat) {
  Grid g = G(nx, ny, dx, dy, c, F, hot);
  std::vector<double> xb(g.N), Rb(g.N);
  for (int j = 0; j < g.ny; ++j)
    for (int i = 0; i < g.nx; ++i)
      for (int v = 0; v < NV; ++v) xb[NV * band_cell(g, i, j) + v] = x_nat[(size_t)v * g.n + j * g.nx + i];
  residual_all(g, xb.data(), Rb.data());
  for (int j = 0; j < g.ny; ++j)
    for (int i = 0; i < g.nx; ++i)
      for (int v = 0; v < NV; ++v) R_nat[(size_t)v * g.n + j * g.nx + i] = Rb[NV * band_cell(g, i, j) + v];
  return 0;
}

// the FP32 factors of a band matrix given densely, for checks of the
// substitution's data flow: AB (N x ld), Lp, ud, piv
extern "C" int h_band_factor(int N, int kl, int nb, const double* A, float* AB, float* Lp, float* ud, int32_t* piv) {
  Grid g{};
  g.N = N; g.kl = kl; g.ku = kl; g.ld = 2 * kl + kl + 1;
  F32 f; f.AB.assign((size_t)N * g.ld, 0.f); f.Lm.assign(lp_size(g, nb), 0.f); f.ud.assign(N, 0.f); f.piv.assign(N, 0);
  for (int r = 0; r < N; ++r) for (int c = 0; c < N; ++c) if (std::abs(r - c) <= kl) f.AB[band_at(g, r, c)] = (float)A[(size_t)r * N + c];
  factor(g, nb, f);
  std::copy(f.AB.begin(), f.AB.end(), AB);
  std::copy(f.Lm.begin(), f.Lm.end(), Lp);
  std::copy(f.ud.begin(), f.ud.end(), ud);
  std::copy(f.piv.begin(), f.piv.end(), piv);
  return 0;
}
