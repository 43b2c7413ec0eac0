/*
 * dsmc_oracle.c -- plain, single-threaded FP64 reference implementation of the
 * DSMC particle step of the DIG method (arXiv 2501.10965) for a polyatomic gas
 * with continuous rotational energy.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: it is used by the tests, by the CPU-baseline leg of the
 * benchmark and by the smoke check, to decide whether the CUDA library is
 * right.  It shares no source with the CUDA library.
 *
 * Every function follows the paper's text in the paper's order, one particle
 * and one candidate pair at a time, with no blocking, fusion or reordering:
 *
 *   move + diffuse walls   Sec. 2.2 (free flight, then collisions) and Sec. 4
 *                          ("fully diffuse" gas-surface interaction); for the
 *                          flow past a cylinder (Sec. 4.2, annular mesh) the
 *                          cylinder is a diffuse wall, particles leave through
 *                          the outer circle and the freestream enters through
 *                          it with the one-sided flux of a drifting Maxwellian
 *   cell index + sort      implied by the per-cell collisions of Sec. 2.2
 *   NTC / VHS / BL         Sec. 2.2, Eq. (P_inelastic); Sec. 4 gas constants
 *   sampling               Eq. (DSMC_macroscopic), time averaged (Sec. 3 step 2)
 *   particle modification  Sec. 3.2 steps i-iv
 *
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11,
 * "Parallel random numbers: as easy as 1, 2, 3"), keyed by the 64-bit seed,
 * with the counter (index, cell, step, tag<<24 | block).  A uniform deviate
 * takes two 32-bit words: u = (m + 1/2) 2^-52 with m the top 52 bits of
 * (w0, w1), so u lies strictly inside (0, 1).
 *
 * Units: lengths in L0, density in rho0, temperature in T0, speed in
 * sqrt(R T0), so a particle has unit mass and k/m = 1.  I_r is the rotational
 * energy per unit mass in units of R T0, so <I_r> = (d_r/2) T_r.
 *
 * Compile with -ffp-contract=off: no fused multiply-add may change rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_CAPACITY (-2)
#define OR_ERR_NUMERIC (-3)

#define OR_TAG_INIT 1u
#define OR_TAG_WALL 2u
#define OR_TAG_NTC 3u
#define OR_TAG_COLL 4u
#define OR_TAG_DIG_N 5u
#define OR_TAG_DIG_SEL 6u
#define OR_TAG_DIG_POS 7u
#define OR_TAG_INJ 8u

#define OR_MAX_HITS 8
#define OR_NMOM 17

typedef struct or_config {
  int32_t dim, nx, ny, ppc;
  double lx, ly;
  double kn, omega, alpha, z_rot, d_r;
  double dt;
  int32_t wall_kind[4]; /* 0 diffuse, 1 specular */
  double wall_t[4];
  double wall_u[4][3];
  double init_rho, init_tt, init_tr;
  double init_u[3];
  int32_t collisions;
  int32_t pad0;
  uint64_t seed;
  int64_t capacity;
  /* mesh 1: annulus r_in <= r <= r_out around a cylinder, nx angular x ny
   * radial cells, cell = j nx + k; the radial width grows by the factor
   * stretch from ring to ring; wall 0 is the cylinder; the freestream
   * (fs_rho, fs_t, fs_u) enters through the outer circle */
  int32_t mesh;
  int32_t pad1;
  double r_in, r_out, stretch;
  double fs_rho, fs_t, fs_u[3];
} or_config;

typedef struct or_state {
  or_config c;
  int ncells;
  int64_t n, cap;
  double *x, *y, *vx, *vy, *vz, *ir;
  double *tx, *ty, *tvx, *tvy, *tvz, *tir;
  int32_t *key;   /* cell of each slot, after the last move */
  int32_t *cell;  /* cell of each slot in the current (sorted) layout */
  int64_t *start; /* ncells + 1 */
  int64_t *cnt;
  double *sgmax;
  double *acc; /* ncells x 17 raw sums */
  int64_t nsamples;
  uint32_t step, dig_iter;
  double dx, dy, vcell, fnum, mu_ref, k_visc, c_sigma, p_inel;
  int64_t n_cand, n_coll, n_clip, n_inel, n_hits, n_maxhit;
  double wall_tally[4][5];
  double *vol;      /* ncells cell volumes (areas per unit depth in 2D) */
  double *rt, *r2t; /* annulus: ny + 1 ring radii and their squares */
  double *xe, *ye;  /* wall-refined box: nx + 1 and ny + 1 cell edges */
  double *rc, *rs;  /* annulus: nx + 1 rays (cos, sin of 2 pi k / nx) */
  double *fc, *fs;  /* annulus: nx outer-face centre directions */
  int64_t n_inj, n_out;
} or_state;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64        */
/* multiplies, key bumped by the Weyl constants after every round.          */
/* ------------------------------------------------------------------------ */
void or_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
               uint32_t k1, uint32_t out[4]) {
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* A named stream of uniforms: uniform j lives in block j/2, words 2(j%2),
 * 2(j%2)+1 of philox(c0, c1, c2, tag<<24 | block). */
typedef struct {
  uint64_t seed;
  uint32_t c0, c1, c2, tag;
  int64_t blk;
  uint32_t w[4];
} or_stream;

static void or_stream_init(or_stream *s, uint64_t seed, uint32_t tag, uint32_t c0,
                           uint32_t c1, uint32_t c2) {
  s->seed = seed;
  s->tag = tag;
  s->c0 = c0;
  s->c1 = c1;
  s->c2 = c2;
  s->blk = -1;
}

static double or_uni(or_stream *s, uint32_t j) {
  uint32_t b = j / 2u, k = j % 2u;
  if ((int64_t)b != s->blk) {
    or_philox(s->c0, s->c1, s->c2, (s->tag << 24) | b, (uint32_t)(s->seed & 0xffffffffu),
              (uint32_t)(s->seed >> 32), s->w);
    s->blk = (int64_t)b;
  }
  uint32_t hi = s->w[2 * k], lo = s->w[2 * k + 1];
  uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
  return ((double)m + 0.5) * 0x1p-52;
}

double or_uniform(uint64_t seed, uint32_t tag, uint32_t c0, uint32_t c1, uint32_t c2,
                  uint32_t j) {
  or_stream s;
  or_stream_init(&s, seed, tag, c0, c1, c2);
  return or_uni(&s, j);
}

/* Iround (Sec. 3.2 step i): floor(x) + 1 with probability x - floor(x). */
static int64_t or_iround(double x, double u) {
  double f = floor(x);
  return (int64_t)f + ((u < x - f) ? 1 : 0);
}

int64_t or_iround_pub(double x, double u) { return or_iround(x, u); }

/* ------------------------------------------------------------------------ */
/* Constants                                                                */
/* ------------------------------------------------------------------------ */

/* Kn = mu(T0)/(p0 L0) sqrt(pi R T0 / 2) (Sec. 2) gives the non-dimensional
 * reference viscosity mu_ref = Kn sqrt(2/pi).  The VHS/VSS first-order
 * viscosity makes the equilibrium collision frequency nu = K p / mu with
 * K = 5(a+1)(a+2) / (a (5-2w)(7-2w)); <g^k> over the relative-speed
 * distribution at temperature T is (4T)^{k/2} (2/sqrt(pi)) Gamma((k+3)/2),
 * so sigma g = C_sigma g^{2-2w} with the C_sigma below reproduces nu at
 * rho = T = 1. */
/* Annulus geometry: ring radii R_j = r_in + (r_out - r_in) (q^j - 1) / (q^ny
 * - 1) (q = stretch; uniform for q = 1), rays at 2 pi k / nx, cell volume
 * (pi / nx) (R_{j+1}^2 - R_j^2). */
static void or_annulus_tables(or_state *S) {
  const or_config *c = &S->c;
  int nr = c->ny, nt = c->nx;
  double q = c->stretch;
  for (int j = 0; j <= nr; ++j) {
    double f = (q == 1.0) ? (double)j / (double)nr : (pow(q, (double)j) - 1.0) / (pow(q, (double)nr) - 1.0);
    S->rt[j] = c->r_in + (c->r_out - c->r_in) * f;
  }
  S->rt[0] = c->r_in;
  S->rt[nr] = c->r_out;
  for (int j = 0; j <= nr; ++j) S->r2t[j] = S->rt[j] * S->rt[j];
  for (int k = 0; k < nt; ++k) {
    double th = 2.0 * M_PI * (double)k / (double)nt;
    S->rc[k] = cos(th);
    S->rs[k] = sin(th);
    double tm = 2.0 * M_PI * ((double)k + 0.5) / (double)nt;
    S->fc[k] = cos(tm);
    S->fs[k] = sin(tm);
  }
  S->rc[nt] = S->rc[0];
  S->rs[nt] = S->rs[0];
  double half = M_PI / (double)nt;
  for (int j = 0; j < nr; ++j)
    for (int k = 0; k < nt; ++k) S->vol[j * nt + k] = half * (S->r2t[j + 1] - S->r2t[j]);
}

/* Wall-refined box (mesh 2, the non-uniform cavity grid of Sec. 4.1): n
 * cells along an axis of length L whose widths grow geometrically by the
 * factor q from both walls towards the middle, w_i proportional to
 * q^min(i, n-1-i), scaled to sum to L; e[0] = 0, e[n] = L. */
static void or_box_edges(int n, double L, double q, double *e) {
  double sum = 0.0;
  for (int i = 0; i < n; ++i) sum += pow(q, (double)(i < n - 1 - i ? i : n - 1 - i));
  e[0] = 0.0;
  for (int i = 0; i < n; ++i) e[i + 1] = e[i] + L * pow(q, (double)(i < n - 1 - i ? i : n - 1 - i)) / sum;
  e[n] = L;
}

static void or_constants_compute(or_state *S) {
  const or_config *c = &S->c;
  double w = c->omega, a = c->alpha;
  if (c->mesh == 2) {
    or_box_edges(c->nx, c->lx, c->stretch, S->xe);
    or_box_edges(c->ny, c->ly, c->stretch, S->ye);
    S->dx = c->lx / (double)c->nx;
    S->dy = c->ly / (double)c->ny;
    S->vcell = S->dx * S->dy;
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) S->vol[j * c->nx + i] = (S->xe[i + 1] - S->xe[i]) * (S->ye[j + 1] - S->ye[j]);
  } else if (c->mesh == 1) {
    or_annulus_tables(S);
    S->dx = 2.0 * M_PI / (double)c->nx;
    S->dy = (c->r_out - c->r_in) / (double)c->ny;
    double area = 0.0;
    for (int i = 0; i < S->ncells; ++i) area += S->vol[i];
    S->vcell = area / (double)S->ncells;
  } else {
    S->dx = c->lx / (double)c->nx;
    S->dy = (c->dim == 2) ? c->ly / (double)c->ny : 1.0;
    S->vcell = S->dx * S->dy;
    for (int i = 0; i < S->ncells; ++i) S->vol[i] = S->vcell;
  }
  /* particle weight F = rho V / N_p (Eq. DSMC_macroscopic) with the mean cell
   * volume; a state created empty is weighted as if it had one particle per
   * cell */
  S->fnum = c->init_rho * S->vcell / (double)(c->ppc > 0 ? c->ppc : 1);
  S->mu_ref = c->kn * sqrt(2.0 / M_PI);
  S->k_visc = 5.0 * (a + 1.0) * (a + 2.0) / (a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w));
  S->c_sigma = S->k_visc /
               (S->mu_ref * pow(4.0, 1.0 - w) * (2.0 / sqrt(M_PI)) * tgamma(2.5 - w));
  /* Eq. (P_inelastic) */
  S->p_inel = a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (a + 1.0) * (a + 2.0) * c->z_rot);
}

void or_constants(const or_state *S, double out[8]) {
  out[0] = S->dx;
  out[1] = S->dy;
  out[2] = S->vcell;
  out[3] = S->fnum;
  out[4] = S->mu_ref;
  out[5] = S->k_visc;
  out[6] = S->c_sigma;
  out[7] = S->p_inel;
}

/* Annulus: ring j is the largest with R_j^2 <= r^2 (the first ring below
 * r_in, which rounding can give); sector k holds the points with
 * cross(ray_k, p) >= 0 > cross(ray_{k+1}, p), found from the atan2 guess by
 * those two signs; -1 outside r_out (the particle has left). */
static int or_cell_of_annulus(const or_state *S, double x, double y) {
  const or_config *c = &S->c;
  int nr = c->ny, nt = c->nx;
  double r2 = x * x + y * y;
  if (!(r2 < S->r2t[nr])) return -1;
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (S->r2t[mid] <= r2) lo = mid;
    else hi = mid - 1;
  }
  double th = atan2(y, x);
  if (th < 0.0) th += 2.0 * M_PI;
  int k = (int)(th * ((double)nt / (2.0 * M_PI)));
  if (k < 0) k = 0;
  if (k > nt - 1) k = nt - 1;
  for (int it = 0; it < 4; ++it) {
    if (S->rc[k] * y - S->rs[k] * x < 0.0) k = (k == 0) ? nt - 1 : k - 1;
    else if (S->rc[k + 1] * y - S->rs[k + 1] * x >= 0.0) k = (k == nt - 1) ? 0 : k + 1;
    else break;
  }
  return lo * nt + k;
}

/* the largest i with e[i] <= v, clamped to [0, n - 1] */
static int or_edge_index(const double *e, int n, double v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (e[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

static int or_cell_of(const or_state *S, double x, double y) {
  const or_config *c = &S->c;
  if (c->mesh == 1) return or_cell_of_annulus(S, x, y);
  if (c->mesh == 2) return or_edge_index(S->ye, c->ny, y) * c->nx + or_edge_index(S->xe, c->nx, x);
  int ix = (int)(x * ((double)c->nx / c->lx));
  if (ix < 0) ix = 0;
  if (ix > c->nx - 1) ix = c->nx - 1;
  if (c->dim == 1) return ix;
  int iy = (int)(y * ((double)c->ny / c->ly));
  if (iy < 0) iy = 0;
  if (iy > c->ny - 1) iy = c->ny - 1;
  return iy * c->nx + ix;
}

/* ------------------------------------------------------------------------ */
/* Creation                                                                 */
/* ------------------------------------------------------------------------ */
static int or_alloc(or_state *S, int64_t cap) {
  S->cap = cap;
  double **arrs[12] = {&S->x, &S->y, &S->vx, &S->vy, &S->vz, &S->ir,
                       &S->tx, &S->ty, &S->tvx, &S->tvy, &S->tvz, &S->tir};
  for (int i = 0; i < 12; ++i) {
    *arrs[i] = (double *)calloc((size_t)(cap > 0 ? cap : 1), sizeof(double));
    if (!*arrs[i]) return OR_ERR_CAPACITY;
  }
  S->key = (int32_t *)calloc((size_t)(cap > 0 ? cap : 1), sizeof(int32_t));
  S->cell = (int32_t *)calloc((size_t)(cap > 0 ? cap : 1), sizeof(int32_t));
  S->start = (int64_t *)calloc((size_t)S->ncells + 1, sizeof(int64_t));
  S->cnt = (int64_t *)calloc((size_t)S->ncells + 1, sizeof(int64_t));
  S->sgmax = (double *)calloc((size_t)S->ncells, sizeof(double));
  S->acc = (double *)calloc((size_t)S->ncells * OR_NMOM, sizeof(double));
  if (!S->key || !S->cell || !S->start || !S->cnt || !S->sgmax || !S->acc) return OR_ERR_CAPACITY;
  S->vol = (double *)calloc((size_t)S->ncells, sizeof(double));
  S->rt = (double *)calloc((size_t)S->c.ny + 1, sizeof(double));
  S->r2t = (double *)calloc((size_t)S->c.ny + 1, sizeof(double));
  S->rc = (double *)calloc((size_t)S->c.nx + 1, sizeof(double));
  S->rs = (double *)calloc((size_t)S->c.nx + 1, sizeof(double));
  S->fc = (double *)calloc((size_t)S->c.nx, sizeof(double));
  S->fs = (double *)calloc((size_t)S->c.nx, sizeof(double));
  S->xe = (double *)calloc((size_t)S->c.nx + 1, sizeof(double));
  S->ye = (double *)calloc((size_t)S->c.ny + 1, sizeof(double));
  if (!S->vol || !S->rt || !S->r2t || !S->rc || !S->rs || !S->fc || !S->fs || !S->xe || !S->ye)
    return OR_ERR_CAPACITY;
  return OR_OK;
}

void or_destroy(or_state *S) {
  if (!S) return;
  double *arrs[12] = {S->x, S->y, S->vx, S->vy, S->vz, S->ir,
                      S->tx, S->ty, S->tvx, S->tvy, S->tvz, S->tir};
  for (int i = 0; i < 12; ++i) free(arrs[i]);
  free(S->key);
  free(S->cell);
  free(S->start);
  free(S->cnt);
  free(S->sgmax);
  free(S->acc);
  free(S->vol);
  free(S->rt);
  free(S->r2t);
  free(S->rc);
  free(S->rs);
  free(S->fc);
  free(S->fs);
  free(S->xe);
  free(S->ye);
  free(S);
}

/* Box-Muller: two standard normals from two uniforms. */
static void or_box_muller(double ua, double ub, double *n1, double *n2) {
  double r = sqrt(-2.0 * log(ua));
  double th = 2.0 * M_PI * ub;
  *n1 = r * cos(th);
  *n2 = r * sin(th);
}

/* Rotational energy of one molecule in equilibrium at temperature T: d_r
 * quadratic degrees of freedom share (d_r/2) T on average, so I_r / T is
 * Gamma(d_r/2) distributed (Sec. 2.1, e_r = d_r T_r / 2).  d_r = 2 (linear
 * molecules): -T ln u with u the draw's main uniform.  d_r = 3 (non-linear
 * molecules): Gamma(3/2) = Gamma(1) + Gamma(1/2), the Gamma(1/2) part as
 * Z^2/2 of a Box-Muller normal Z = sqrt(-2 ln u_a) cos(2 pi u_b), with u_a,
 * u_b the uniforms jx, jx + 1 of the same stream. */
static double or_ir_draw(const or_state *S, double T, double u, or_stream *st, uint32_t jx) {
  double e = -log(u);
  if (S->c.d_r == 3.0) {
    double cb = cos(2.0 * M_PI * or_uni(st, jx + 1u));
    e += -log(or_uni(st, jx)) * cb * cb;
  }
  return T * e;
}

/* Uniform indices of the extra draws (d_r = 3 only): I_r of a particle's own
 * stream takes 1024-1025; the wall hit whose four uniforms start at jh takes
 * 1026 + jh/2 and 1027 + jh/2; the Borgnakke-Larsen acceptance-rejection of
 * candidate pair k takes 2048 + 4t .. 2051 + 4t (try t). */
#define OR_JX_OWN 1024u
#define OR_JX_HIT(jh) (1026u + (jh) / 2u)
#define OR_JX_BL 2048u
#define OR_BL_TRIES 32

/* Fraction x = I_r,k' / E_c kept as rotational energy in one
 * Borgnakke-Larsen exchange (Sec. 2.2): the equilibrium partition of E_c
 * between the d_r rotational degrees of freedom of one molecule and the
 * relative translation of a VHS/VSS pair, whose collision-weighted energy
 * has 5/2 - w degrees of freedom in units of 2, i.e. x ~ Beta(a, b) with a =
 * d_r/2, b = 5/2 - w.  d_r = 2 (a = 1): x = 1 - u^{1/b} (inverse CDF, u the
 * main uniform).  d_r = 3: acceptance-rejection under the uniform envelope
 * of the density x^{a-1} (1-x)^{b-1}, whose maximum is at x* = (a-1)/(a+b-2):
 * try t proposes x (the main uniform at t = 0, else uniform jx + 4t) and
 * accepts it when ln(uniform jx + 4t + 1) < (a-1) ln(x/x*) + (b-1) ln((1-x)/
 * (1-x*)); after OR_BL_TRIES rejections (odds below 1e-18) it takes x*. */
static double or_bl_fraction(const or_state *S, double u, or_stream *st, uint32_t jx) {
  double b = 2.5 - S->c.omega;
  if (S->c.d_r == 2.0) return 1.0 - pow(u, 1.0 / b);
  double a = 0.5 * S->c.d_r;
  double xs = (a - 1.0) / (a + b - 2.0);
  for (int t = 0; t < OR_BL_TRIES; ++t) {
    double x = (t == 0) ? u : or_uni(st, jx + 4u * (uint32_t)t);
    double acc = or_uni(st, jx + 4u * (uint32_t)t + 1u);
    if (log(acc) < (a - 1.0) * log(x / xs) + (b - 1.0) * log((1.0 - x) / (1.0 - xs))) return x;
  }
  return xs;
}

/* Post-collision relative velocity h = g'/2 of magnitude gn/2.  VHS (alpha
 * = 1): isotropic, cos(theta) = 2 u - 1 and azimuth 2 pi v in the lab frame.
 * VSS (alpha != 1, Sec. 2.2): the deflection chi from the pre-collision
 * direction e = g/|g| has cos(chi) = 2 u^{1/alpha} - 1 and the azimuth 2 pi
 * v about e, measured from e1 = the unit vector along the coordinate axis
 * least aligned with e, made orthogonal to e (e2 = e x e1). */
static void or_scatter(const or_state *S, double gx, double gy, double gz, double gn, double u, double v,
                       double h[3]) {
  double ph = 2.0 * M_PI * v;
  if (S->c.alpha == 1.0) {
    double cth = 2.0 * u - 1.0;
    double sth = sqrt(1.0 - cth * cth);
    h[0] = 0.5 * gn * cth;
    h[1] = 0.5 * gn * sth * cos(ph);
    h[2] = 0.5 * gn * sth * sin(ph);
    return;
  }
  double g = sqrt(gx * gx + gy * gy + gz * gz);
  double e[3] = {gx / g, gy / g, gz / g};
  double ax[3] = {0.0, 0.0, 0.0};
  double m0 = fabs(e[0]), m1 = fabs(e[1]), m2 = fabs(e[2]);
  ax[(m0 <= m1 && m0 <= m2) ? 0 : (m1 <= m2 ? 1 : 2)] = 1.0;
  double d = ax[0] * e[0] + ax[1] * e[1] + ax[2] * e[2];
  double e1[3] = {ax[0] - d * e[0], ax[1] - d * e[1], ax[2] - d * e[2]};
  double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  e1[0] /= l1;
  e1[1] /= l1;
  e1[2] /= l1;
  double e2[3] = {e[1] * e1[2] - e[2] * e1[1], e[2] * e1[0] - e[0] * e1[2], e[0] * e1[1] - e[1] * e1[0]};
  double cch = 2.0 * pow(u, 1.0 / S->c.alpha) - 1.0;
  double sch = sqrt(1.0 - cch * cch);
  double cp = cos(ph), sp = sin(ph);
  for (int k = 0; k < 3; ++k) h[k] = 0.5 * gn * (cch * e[k] + sch * (cp * e1[k] + sp * e2[k]));
}

/* exported for the tests of the Borgnakke-Larsen partition, the rotational
 * energy draw and the scattering law */
double or_bl_fraction_pub(double omega, double d_r, uint64_t seed, uint32_t k, uint32_t cell, uint32_t step,
                          double u, uint32_t jx) {
  or_state S;
  memset(&S, 0, sizeof S);
  S.c.omega = omega;
  S.c.d_r = d_r;
  or_stream st;
  or_stream_init(&st, seed, OR_TAG_COLL, k, cell, step);
  return or_bl_fraction(&S, u, &st, jx);
}
void or_scatter_pub(double alpha, double gx, double gy, double gz, double gn, double u, double v, double h[3]) {
  or_state S;
  memset(&S, 0, sizeof S);
  S.c.alpha = alpha;
  or_scatter(&S, gx, gy, gz, gn, u, v, h);
}

/* Equilibrium (Maxwellian) initial state, ppc particles per cell, cell by cell
 * (Sec. 3 step 1; Sec. 4: particles sampled from an equilibrium distribution),
 * I_r drawn at T_r (or_ir_draw). */
int or_create(const or_config *cfg, or_state **out) {
  *out = NULL;
  if (cfg->dim != 1 && cfg->dim != 2) return OR_ERR_ARG;
  if (cfg->nx <= 0 || (cfg->dim == 2 && cfg->ny <= 0) || cfg->ppc < 0) return OR_ERR_ARG;
  /* d_r = 2 (linear) or 3 (non-linear molecules); VSS exponent 0 < alpha <= 2 */
  if ((cfg->d_r != 2.0 && cfg->d_r != 3.0) || !(cfg->alpha > 0.0 && cfg->alpha <= 2.0)) return OR_ERR_ARG;
  if (cfg->mesh != 0 && cfg->mesh != 1 && cfg->mesh != 2) return OR_ERR_ARG;
  if (cfg->mesh == 2 && (cfg->dim != 2 || !(cfg->stretch > 0.0))) return OR_ERR_ARG;
  if (cfg->mesh == 1 && (cfg->dim != 2 || cfg->nx < 3 || !(cfg->r_in > 0.0) || !(cfg->r_out > cfg->r_in) ||
                         !(cfg->stretch > 0.0) || !(cfg->fs_t > 0.0) || !(cfg->fs_rho >= 0.0)))
    return OR_ERR_ARG;
  or_state *S = (or_state *)calloc(1, sizeof(or_state));
  if (!S) return OR_ERR_CAPACITY;
  S->c = *cfg;
  if (S->c.dim == 1) {
    S->c.ny = 1;
    S->c.ly = 1.0;
  }
  S->ncells = S->c.nx * S->c.ny;
  int64_t n0 = (int64_t)S->ncells * (int64_t)S->c.ppc;
  int64_t cap = S->c.capacity > 0 ? S->c.capacity : n0 * 2 + 64;
  if (S->c.mesh == 0 && n0 > cap) {
    free(S);
    return OR_ERR_CAPACITY;
  }
  int rc = or_alloc(S, cap);
  if (rc) {
    or_destroy(S);
    return rc;
  }
  or_constants_compute(S);
  const or_config *c = &S->c;
  double stt = sqrt(c->init_tt);
  int64_t s = 0;
  for (int cell = 0; cell < S->ncells; ++cell) {
    int ix = cell % c->nx, iy = cell / c->nx;
    S->start[cell] = s;
    int64_t np = c->ppc;
    if (c->mesh != 0) {
      /* annulus, wall-refined box: the equilibrium density in cells of
       * unequal volume */
      or_stream sc;
      or_stream_init(&sc, c->seed, OR_TAG_INIT, 0xFFFFFFFFu, (uint32_t)cell, 0u);
      np = or_iround(c->init_rho * S->vol[cell] / S->fnum, or_uni(&sc, 0));
      if (s + np > cap) {
        or_destroy(S);
        return OR_ERR_CAPACITY;
      }
    }
    for (int k = 0; k < np; ++k, ++s) {
      or_stream st;
      or_stream_init(&st, c->seed, OR_TAG_INIT, (uint32_t)k, (uint32_t)cell, 0u);
      double u0 = or_uni(&st, 0), u1 = or_uni(&st, 1);
      double n1, n2, n3, n4;
      or_box_muller(or_uni(&st, 2), or_uni(&st, 3), &n1, &n2);
      or_box_muller(or_uni(&st, 4), or_uni(&st, 5), &n3, &n4);
      (void)n4;
      if (c->mesh == 1) {
        /* uniform in the annular sector: r^2 uniform, angle uniform */
        double r = sqrt(S->r2t[iy] + u0 * (S->r2t[iy + 1] - S->r2t[iy]));
        double th = 2.0 * M_PI * ((double)ix + u1) / (double)c->nx;
        S->x[s] = r * cos(th);
        S->y[s] = r * sin(th);
      } else if (c->mesh == 2) {
        S->x[s] = S->xe[ix] + u0 * (S->xe[ix + 1] - S->xe[ix]);
        S->y[s] = S->ye[iy] + u1 * (S->ye[iy + 1] - S->ye[iy]);
      } else {
        S->x[s] = ((double)ix + u0) * S->dx;
        S->y[s] = (c->dim == 2) ? ((double)iy + u1) * S->dy : 0.0;
      }
      S->vx[s] = c->init_u[0] + stt * n1;
      S->vy[s] = c->init_u[1] + stt * n2;
      S->vz[s] = c->init_u[2] + stt * n3;
      S->ir[s] = or_ir_draw(S, c->init_tr, or_uni(&st, 6), &st, OR_JX_OWN);
      S->cell[s] = cell;
    }
  }
  S->start[S->ncells] = s;
  S->n = s;
  /* (sigma g)_max starts at C_sigma g_ref^{2-2w}, g_ref = 4 sqrt(T_ref) + U_ref */
  double tref = c->init_tt, uref = sqrt(c->init_u[0] * c->init_u[0] + c->init_u[1] * c->init_u[1] +
                                        c->init_u[2] * c->init_u[2]);
  double umax = 0.0;
  int nwalls = (c->mesh == 1) ? 1 : 2 * c->dim;
  for (int w = 0; w < nwalls; ++w) {
    if (c->wall_kind[w] == 0 && c->wall_t[w] > tref) tref = c->wall_t[w];
    double uw = sqrt(c->wall_u[w][0] * c->wall_u[w][0] + c->wall_u[w][1] * c->wall_u[w][1] +
                     c->wall_u[w][2] * c->wall_u[w][2]);
    if (uw > umax) umax = uw;
  }
  uref += umax;
  double sg0 = S->c_sigma * pow(4.0 * sqrt(tref) + uref, 2.0 - 2.0 * c->omega);
  for (int i = 0; i < S->ncells; ++i) S->sgmax[i] = sg0;
  *out = S;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Stage (a): free flight with wall interaction                             */
/* ------------------------------------------------------------------------ */

/* Re-emission at wall w (0: x=0, 1: x=lx, 2: y=0, 3: y=ly).  Fully diffuse
 * (Sec. 4): the normal speed follows the flux-weighted half-range Maxwellian
 * at the wall temperature, sqrt(-2 T_w ln u); the tangential components are
 * Maxwellian about the wall velocity; the rotational energy is re-drawn at
 * T_w (full accommodation).  Specular walls mirror the normal component. */
static void or_wall_emit(or_state *S, int w, or_stream *st, int hit, double v[3], double *ir) {
  const or_config *c = &S->c;
  int axis = (w < 2) ? 0 : 1;
  double sgn = (w % 2 == 0) ? 1.0 : -1.0;
  double vin[3] = {v[0], v[1], v[2]}, irin = *ir;
  if (c->wall_kind[w] == 1) {
    v[axis] = -v[axis];
  } else {
    double T = c->wall_t[w];
    double ua = or_uni(st, (uint32_t)(4 * hit + 0));
    double ub = or_uni(st, (uint32_t)(4 * hit + 1));
    double uc = or_uni(st, (uint32_t)(4 * hit + 2));
    double ud = or_uni(st, (uint32_t)(4 * hit + 3));
    double vn = sqrt(-2.0 * T * log(ua));
    double n1, n2;
    or_box_muller(ub, uc, &n1, &n2);
    double sT = sqrt(T);
    if (axis == 0) {
      v[0] = sgn * vn;
      v[1] = c->wall_u[w][1] + sT * n1;
      v[2] = c->wall_u[w][2] + sT * n2;
    } else {
      v[0] = c->wall_u[w][0] + sT * n1;
      v[1] = sgn * vn;
      v[2] = c->wall_u[w][2] + sT * n2;
    }
    *ir = or_ir_draw(S, T, ud, st, OR_JX_HIT((uint32_t)(4 * hit)));
  }
  double *t = S->wall_tally[w];
  t[0] += 1.0;
  t[1] += vin[0] - v[0];
  t[2] += vin[1] - v[1];
  t[3] += vin[2] - v[2];
  t[4] += (0.5 * (vin[0] * vin[0] + vin[1] * vin[1] + vin[2] * vin[2]) + irin) -
          (0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + *ir);
  S->n_hits += 1;
}

/* Re-emission from the cylinder (wall 0 of the annulus) at the surface point
 * with outward unit normal (nx, ny): diffuse at T_w about a resting wall
 * (normal speed sqrt(-2 T_w ln u), Maxwellian tangential and z components,
 * I_r drawn at T_w) or specular (normal component reversed). */
static void or_cyl_emit(or_state *S, or_stream *st, uint32_t j0, double nx, double ny, double v[3], double *ir) {
  const or_config *c = &S->c;
  double vin[3] = {v[0], v[1], v[2]}, irin = *ir;
  if (c->wall_kind[0] == 1) {
    double vn = v[0] * nx + v[1] * ny;
    v[0] = v[0] - 2.0 * vn * nx;
    v[1] = v[1] - 2.0 * vn * ny;
  } else {
    double T = c->wall_t[0];
    double ua = or_uni(st, j0 + 0u), ub = or_uni(st, j0 + 1u), uc = or_uni(st, j0 + 2u), ud = or_uni(st, j0 + 3u);
    double vn = sqrt(-2.0 * T * log(ua));
    double n1, n2;
    or_box_muller(ub, uc, &n1, &n2);
    double sT = sqrt(T);
    double vt = sT * n1;
    v[0] = vn * nx - vt * ny;
    v[1] = vn * ny + vt * nx;
    v[2] = sT * n2;
    *ir = or_ir_draw(S, T, ud, st, OR_JX_HIT(j0));
  }
  double *t = S->wall_tally[0];
  t[0] += 1.0;
  t[1] += vin[0] - v[0];
  t[2] += vin[1] - v[1];
  t[3] += vin[2] - v[2];
  t[4] += (0.5 * (vin[0] * vin[0] + vin[1] * vin[1] + vin[2] * vin[2]) + irin) -
          (0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + *ir);
  S->n_hits += 1;
}

/* Free flight for time t in the annulus.  The first crossing of the cylinder
 * r = r_in along the straight path p + v s is the smaller root of
 * |p + v s|^2 = r_in^2 (taken when the particle moves inward); the particle
 * is put on the circle, re-emitted and flies the rest of the step (a path
 * leaving a convex body does not meet it again).  Hit h draws uniforms
 * j0 + 4h .. j0 + 4h + 3 of the stream.  Returns 0 if the particle ends at or
 * beyond r_out (it has left the domain). */
static int or_fly_annulus(or_state *S, or_stream *st, uint32_t j0, double *px, double *py, double v[3], double *ir,
                          double t) {
  double x = *px, y = *py;
  int hits = 0;
  for (;;) {
    double a = v[0] * v[0] + v[1] * v[1];
    double b = x * v[0] + y * v[1];
    double s1 = INFINITY;
    if (b < 0.0 && a > 0.0) {
      double cc = x * x + y * y - S->r2t[0];
      double disc = b * b - a * cc;
      if (disc > 0.0) {
        s1 = (-b - sqrt(disc)) / a;
        if (s1 < 0.0) s1 = 0.0;
      }
    }
    if (!(s1 < t)) {
      x = x + v[0] * t;
      y = y + v[1] * t;
      break;
    }
    double xh = x + v[0] * s1, yh = y + v[1] * s1;
    double rh = sqrt(xh * xh + yh * yh);
    double nx = xh / rh, ny = yh / rh;
    x = S->rt[0] * nx;
    y = S->rt[0] * ny;
    if (hits == OR_MAX_HITS) {
      S->n_maxhit += 1;
      break;
    }
    t = t - s1;
    if (t < 0.0) t = 0.0;
    or_cyl_emit(S, st, j0 + 4u * (uint32_t)hits, nx, ny, v, ir);
    hits += 1;
  }
  *px = x;
  *py = y;
  return (x * x + y * y < S->r2t[S->c.ny]) ? 1 : 0;
}

/* One-sided number flux (per unit length and time) of a Maxwellian of
 * density rho, temperature T and velocity component un along the inward
 * normal: rho sqrt(T/(2 pi)) [exp(-s^2) + sqrt(pi) s erfc(-s)], s = un /
 * sqrt(2T), written as rho G(inf) / (beta sqrt(pi)) with beta = 1/sqrt(2T). */
static double or_inflow_ginf(double s) { return 0.5 * exp(-s * s) + s * (0.5 * sqrt(M_PI)) * erfc(-s); }

/* Inward normal speed of an entering particle, in units of 1/beta: the
 * density of z = beta v_n > 0 is proportional to z exp(-(z - s)^2), with
 * CDF G(z) = [exp(-s^2) - exp(-(z-s)^2)] / 2 + s (sqrt(pi)/2) [erfc(-s) -
 * erfc(z - s)]; G(z) = u G(inf) is solved by Newton steps kept inside a
 * bisection bracket (at most 100 steps). */
static double or_inflow_speed(double s, double u) {
  double target = u * or_inflow_ginf(s);
  double lo = 0.0, hi = (s > 0.0 ? s : 0.0) + 8.0;
  double z = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    double w = z - s;
    double g = 0.5 * (exp(-s * s) - exp(-w * w)) + s * (0.5 * sqrt(M_PI)) * (erfc(-s) - erfc(w));
    double f = g - target;
    if (f > 0.0) hi = z;
    else lo = z;
    double d = z * exp(-w * w);
    double zn = (d > 0.0) ? z - f / d : 0.5 * (lo + hi);
    if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
    if (fabs(zn - z) <= 1e-15 * (1.0 + z) || hi - lo <= 1e-15 * (1.0 + z)) {
      z = zn;
      break;
    }
    z = zn;
  }
  return z;
}

/* Freestream entry through the outer circle during one step.  Outer face k
 * (between rays k and k+1 at r_out) admits Iround(flux L dt / F) particles,
 * the flux taken with the face-centre inward normal n and L = r_out 2 pi /
 * nx.  Particle q of face k (stream (q, k, step)): normal speed from the
 * inflow distribution, tangential and z components Maxwellian about the
 * freestream, I_r at the freestream temperature, the entry angle uniform on
 * the face, and a flight over a uniform fraction of the step.  New
 * particles follow the existing ones, face by face. */
static void or_inject(or_state *S) {
  const or_config *c = &S->c;
  int nt = c->nx;
  double T = c->fs_t, sT = sqrt(T), beta = 1.0 / sqrt(2.0 * T);
  double len = c->r_out * 2.0 * M_PI / (double)nt;
  for (int k = 0; k < nt; ++k) {
    double nx = -S->fc[k], ny = -S->fs[k]; /* inward normal */
    double tx = -ny, ty = nx;
    double un = c->fs_u[0] * nx + c->fs_u[1] * ny, ut = c->fs_u[0] * tx + c->fs_u[1] * ty;
    double sn = un * beta;
    double mu = c->fs_rho * or_inflow_ginf(sn) / (beta * sqrt(M_PI)) * len * c->dt / S->fnum;
    or_stream sc;
    or_stream_init(&sc, c->seed, OR_TAG_INJ, 0xFFFFFFFFu, (uint32_t)k, S->step);
    int64_t m = or_iround(mu, or_uni(&sc, 0));
    for (int64_t q = 0; q < m; ++q) {
      or_stream st;
      or_stream_init(&st, c->seed, OR_TAG_INJ, (uint32_t)q, (uint32_t)k, S->step);
      double vn = or_inflow_speed(sn, or_uni(&st, 0)) / beta;
      double n1, n2;
      or_box_muller(or_uni(&st, 1), or_uni(&st, 2), &n1, &n2);
      double vt = ut + sT * n1;
      double v[3] = {vn * nx + vt * tx, vn * ny + vt * ty, c->fs_u[2] + sT * n2};
      double th = 2.0 * M_PI * ((double)k + or_uni(&st, 3)) / (double)nt;
      double ir = or_ir_draw(S, T, or_uni(&st, 4), &st, OR_JX_OWN);
      double x = c->r_out * cos(th), y = c->r_out * sin(th);
      int in = or_fly_annulus(S, &st, 8u, &x, &y, v, &ir, or_uni(&st, 5) * c->dt);
      if (!in || S->n >= S->cap) continue; /* it does not enter */
      int64_t s = S->n++;
      S->x[s] = x;
      S->y[s] = y;
      S->vx[s] = v[0];
      S->vy[s] = v[1];
      S->vz[s] = v[2];
      S->ir[s] = ir;
      S->key[s] = or_cell_of(S, x, y);
      S->n_inj += 1;
    }
  }
}

/* exported for the tests of the inflow sampler */
double or_inflow_ginf_pub(double s) { return or_inflow_ginf(s); }
double or_inflow_speed_pub(double s, double u) { return or_inflow_speed(s, u); }

void or_move(or_state *S) {
  const or_config *c = &S->c;
  if (c->mesh == 1) {
    /* annulus: particles in slot order, each with its cell's wall stream;
     * leavers get key -1 and the sort drops them; then the freestream entry */
    for (int cell = 0; cell < S->ncells; ++cell) {
      for (int64_t s = S->start[cell]; s < S->start[cell + 1]; ++s) {
        or_stream st;
        or_stream_init(&st, c->seed, OR_TAG_WALL, (uint32_t)(s - S->start[cell]), (uint32_t)cell, S->step);
        double x = S->x[s], y = S->y[s];
        double v[3] = {S->vx[s], S->vy[s], S->vz[s]};
        double ir = S->ir[s];
        int in = or_fly_annulus(S, &st, 0u, &x, &y, v, &ir, c->dt);
        S->x[s] = x;
        S->y[s] = y;
        S->vx[s] = v[0];
        S->vy[s] = v[1];
        S->vz[s] = v[2];
        S->ir[s] = ir;
        S->key[s] = in ? or_cell_of(S, x, y) : -1;
        if (!in) S->n_out += 1;
      }
    }
    or_inject(S);
    return;
  }
  for (int cell = 0; cell < S->ncells; ++cell) {
    for (int64_t s = S->start[cell]; s < S->start[cell + 1]; ++s) {
      or_stream st;
      or_stream_init(&st, c->seed, OR_TAG_WALL, (uint32_t)(s - S->start[cell]), (uint32_t)cell,
                     S->step);
      double x = S->x[s], y = S->y[s];
      double v[3] = {S->vx[s], S->vy[s], S->vz[s]};
      double ir = S->ir[s];
      double t = c->dt;
      int hits = 0;
      for (;;) {
        double xn = x + v[0] * t;
        double yn = (c->dim == 2) ? y + v[1] * t : y;
        double tx = INFINITY, ty = INFINITY;
        int wx = -1, wy = -1;
        if (xn < 0.0) {
          tx = -x / v[0];
          wx = 0;
        } else if (xn > c->lx) {
          tx = (c->lx - x) / v[0];
          wx = 1;
        }
        if (c->dim == 2) {
          if (yn < 0.0) {
            ty = -y / v[1];
            wy = 2;
          } else if (yn > c->ly) {
            ty = (c->ly - y) / v[1];
            wy = 3;
          }
        }
        if (wx < 0 && wy < 0) {
          x = xn;
          y = yn;
          break;
        }
        int w;
        double tw;
        if (wy < 0 || (wx >= 0 && tx <= ty)) {
          w = wx;
          tw = tx;
        } else {
          w = wy;
          tw = ty;
        }
        if (w < 2) {
          x = (w == 0) ? 0.0 : c->lx;
          if (c->dim == 2) {
            y = y + v[1] * tw;
            if (y < 0.0) y = 0.0;
            if (y > c->ly) y = c->ly;
          }
        } else {
          y = (w == 2) ? 0.0 : c->ly;
          x = x + v[0] * tw;
          if (x < 0.0) x = 0.0;
          if (x > c->lx) x = c->lx;
        }
        if (hits == OR_MAX_HITS) {
          S->n_maxhit += 1;
          break;
        }
        t = t - tw;
        if (t < 0.0) t = 0.0;
        or_wall_emit(S, w, &st, hits, v, &ir);
        hits += 1;
      }
      S->x[s] = x;
      S->y[s] = y;
      S->vx[s] = v[0];
      S->vy[s] = v[1];
      S->vz[s] = v[2];
      S->ir[s] = ir;
      S->key[s] = or_cell_of(S, x, y);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Stage (b): stable counting sort by cell                                  */
/* ------------------------------------------------------------------------ */
void or_sort(or_state *S) {
  int nc = S->ncells;
  for (int i = 0; i <= nc; ++i) S->cnt[i] = 0;
  for (int64_t s = 0; s < S->n; ++s)
    if (S->key[s] >= 0) S->cnt[S->key[s]] += 1;
  int64_t acc = 0;
  for (int i = 0; i < nc; ++i) {
    S->start[i] = acc;
    acc += S->cnt[i];
    S->cnt[i] = S->start[i];
  }
  S->start[nc] = acc;
  for (int64_t s = 0; s < S->n; ++s) {
    int k = S->key[s];
    if (k < 0) continue; /* left the domain */
    int64_t d = S->cnt[k]++;
    S->tx[d] = S->x[s];
    S->ty[d] = S->y[s];
    S->tvx[d] = S->vx[s];
    S->tvy[d] = S->vy[s];
    S->tvz[d] = S->vz[s];
    S->tir[d] = S->ir[s];
    S->cell[d] = k;
  }
  double *t;
  t = S->x; S->x = S->tx; S->tx = t;
  t = S->y; S->y = S->ty; S->ty = t;
  t = S->vx; S->vx = S->tvx; S->tvx = t;
  t = S->vy; S->vy = S->tvy; S->tvy = t;
  t = S->vz; S->vz = S->tvz; S->tvz = t;
  t = S->ir; S->ir = S->tir; S->tir = t;
  S->n = acc;
  for (int64_t s = 0; s < S->n; ++s) S->key[s] = S->cell[s];
}

/* ------------------------------------------------------------------------ */
/* Stage (c): No-Time-Counter selection, VHS acceptance, Borgnakke-Larsen    */
/* ------------------------------------------------------------------------ */

/* One cell.  The number of candidate pairs is Iround(N(N-1)/2 F (sigma g)_max
 * dt / V).  For each candidate in turn: pick i uniformly, j uniformly among
 * the others; accept with probability sigma g / (sigma g)_max; if accepted,
 * each of i then j independently undergoes a Borgnakke-Larsen exchange with
 * probability P_inelastic (Bird's particle selection permitting double
 * relaxation, Sec. 2.2): with E_c = E_t + I_r,k the particle keeps
 * I_r,k' = x E_c, x from or_bl_fraction (Beta(d_r/2, 5/2 - w)), and
 * E_t = E_c - I_r,k'.  The pair then scatters about the centre-of-mass
 * velocity with |g'| = sqrt(4 E_t) (or_scatter: isotropic for VHS, alpha =
 * 1; the VSS deflection law otherwise).  (sigma g)_max stays fixed over the
 * candidates of the step and takes the largest sigma g seen afterwards. */
static void or_collide_cell(or_state *S, int cell) {
  const or_config *c = &S->c;
  int64_t s0 = S->start[cell];
  int64_t n = S->start[cell + 1] - s0;
  if (!c->collisions || n < 2) return;
  double sgmax = S->sgmax[cell];
  double xm = 0.5 * (double)n * (double)(n - 1) * S->fnum * sgmax * c->dt / S->vol[cell];
  or_stream sn;
  or_stream_init(&sn, c->seed, OR_TAG_NTC, 0u, (uint32_t)cell, S->step);
  int64_t m = or_iround(xm, or_uni(&sn, 0));
  double e = 2.0 - 2.0 * c->omega;
  double obs = 0.0;
  for (int64_t k = 0; k < m; ++k) {
    or_stream st;
    or_stream_init(&st, c->seed, OR_TAG_COLL, (uint32_t)k, (uint32_t)cell, S->step);
    int64_t i = (int64_t)(or_uni(&st, 0) * (double)n);
    if (i > n - 1) i = n - 1;
    int64_t j = (int64_t)(or_uni(&st, 1) * (double)(n - 1));
    if (j > n - 2) j = n - 2;
    if (j >= i) j += 1;
    int64_t pi = s0 + i, pj = s0 + j;
    double gx = S->vx[pi] - S->vx[pj];
    double gy = S->vy[pi] - S->vy[pj];
    double gz = S->vz[pi] - S->vz[pj];
    double g2 = gx * gx + gy * gy + gz * gz;
    double g = sqrt(g2);
    double sg = S->c_sigma * pow(g, e);
    if (sg > obs) obs = sg;
    S->n_cand += 1;
    if (!(or_uni(&st, 2) * sgmax < sg)) continue;
    S->n_coll += 1;
    if (sg > sgmax) S->n_clip += 1;
    double et = 0.25 * g2;
    if (or_uni(&st, 3) < S->p_inel) {
      double ec = et + S->ir[pi];
      S->ir[pi] = ec * or_bl_fraction(S, or_uni(&st, 4), &st, OR_JX_BL);
      et = ec - S->ir[pi];
      S->n_inel += 1;
    }
    if (or_uni(&st, 5) < S->p_inel) {
      double ec = et + S->ir[pj];
      S->ir[pj] = ec * or_bl_fraction(S, or_uni(&st, 6), &st, OR_JX_BL + 2u);
      et = ec - S->ir[pj];
      S->n_inel += 1;
    }
    double gn = 2.0 * sqrt(et);
    double h[3];
    or_scatter(S, gx, gy, gz, gn, or_uni(&st, 7), or_uni(&st, 8), h);
    double hx = h[0], hy = h[1], hz = h[2];
    double cx = 0.5 * (S->vx[pi] + S->vx[pj]);
    double cy = 0.5 * (S->vy[pi] + S->vy[pj]);
    double cz = 0.5 * (S->vz[pi] + S->vz[pj]);
    S->vx[pi] = cx + hx;
    S->vy[pi] = cy + hy;
    S->vz[pi] = cz + hz;
    S->vx[pj] = cx - hx;
    S->vy[pj] = cy - hy;
    S->vz[pj] = cz - hz;
  }
  if (obs > sgmax) S->sgmax[cell] = obs;
}

void or_collide(or_state *S) {
  for (int cell = 0; cell < S->ncells; ++cell) or_collide_cell(S, cell);
}

/* ------------------------------------------------------------------------ */
/* Stage (d): sampling of raw sums for Eq. (DSMC_macroscopic)               */
/* ------------------------------------------------------------------------ */
/* Per cell, per sampled step: N; sum v_i; sum v_i v_j (xx yy zz xy xz yz);
 * sum v_i |v|^2; sum I_r; sum I_r v_i. */
void or_sample(or_state *S) {
  for (int cell = 0; cell < S->ncells; ++cell) {
    double *a = S->acc + (size_t)cell * OR_NMOM;
    for (int64_t s = S->start[cell]; s < S->start[cell + 1]; ++s) {
      double vx = S->vx[s], vy = S->vy[s], vz = S->vz[s], ir = S->ir[s];
      double v2 = vx * vx + vy * vy + vz * vz;
      a[0] += 1.0;
      a[1] += vx;
      a[2] += vy;
      a[3] += vz;
      a[4] += vx * vx;
      a[5] += vy * vy;
      a[6] += vz * vz;
      a[7] += vx * vy;
      a[8] += vx * vz;
      a[9] += vy * vz;
      a[10] += vx * v2;
      a[11] += vy * v2;
      a[12] += vz * v2;
      a[13] += ir;
      a[14] += ir * vx;
      a[15] += ir * vy;
      a[16] += ir * vz;
    }
  }
  S->nsamples += 1;
}

/* One DSMC time step in the paper's order: move, index, collide, sample. */
void or_step(or_state *S, int nsteps, int sample) {
  for (int k = 0; k < nsteps; ++k) {
    or_move(S);
    or_sort(S);
    or_collide(S);
    if (sample) or_sample(S);
    S->step += 1;
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: particle modification to the target fields M^{n+1}              */
/* ------------------------------------------------------------------------ */
/* target: ncells x 6 = (rho, u_x, u_y, u_z, T_t, T_r). */
int or_dig_correct(or_state *S, const double *target) {
  const or_config *c = &S->c;
  int nc = S->ncells;
  for (int cell = 0; cell < nc; ++cell) {
    const double *t = target + (size_t)cell * 6;
    for (int q = 0; q < 6; ++q)
      if (!isfinite(t[q])) return OR_ERR_NUMERIC;
    /* an empty target cell (rho 0) has no particles whose T would matter */
    if (!(t[0] >= 0.0) || (t[0] > 0.0 && (!(t[4] > 0.0) || !(t[5] > 0.0)))) return OR_ERR_NUMERIC;
  }
  /* step i: target counts */
  int64_t *nt = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
  int64_t total = 0;
  for (int cell = 0; cell < nc; ++cell) {
    or_stream st;
    or_stream_init(&st, c->seed, OR_TAG_DIG_N, 0u, (uint32_t)cell, S->dig_iter);
    /* the cell's own volume: the annulus's cells differ */
    nt[cell] = or_iround(target[(size_t)cell * 6] * S->vol[cell] / S->fnum, or_uni(&st, 0));
    total += nt[cell];
  }
  if (total > S->cap) {
    free(nt);
    return OR_ERR_CAPACITY;
  }
  int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->n > 0 ? S->n : 1));
  int64_t d = 0;
  for (int cell = 0; cell < nc; ++cell) {
    const double *t = target + (size_t)cell * 6;
    int64_t s0 = S->start[cell], n = S->start[cell + 1] - s0;
    int64_t ntg = nt[cell];
    int64_t d0 = d;
    int ix = cell % c->nx, iy = cell / c->nx;
    /* step ii */
    if (ntg <= n) {
      int64_t k = n - ntg;
      for (int64_t q = 0; q < n; ++q) idx[q] = q;
      /* partial Fisher-Yates: the first k entries are removed */
      for (int64_t q = 0; q < k; ++q) {
        or_stream st;
        or_stream_init(&st, c->seed, OR_TAG_DIG_SEL, (uint32_t)q, (uint32_t)cell, S->dig_iter);
        int64_t r = q + (int64_t)(or_uni(&st, 0) * (double)(n - q));
        if (r > n - 1) r = n - 1;
        int64_t tmp = idx[q];
        idx[q] = idx[r];
        idx[r] = tmp;
      }
      /* keep the rest in their original order */
      char *rm = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
      for (int64_t q = 0; q < k; ++q) rm[idx[q]] = 1;
      for (int64_t q = 0; q < n; ++q) {
        if (rm[q]) continue;
        S->tx[d] = S->x[s0 + q];
        S->ty[d] = S->y[s0 + q];
        S->tvx[d] = S->vx[s0 + q];
        S->tvy[d] = S->vy[s0 + q];
        S->tvz[d] = S->vz[s0 + q];
        S->tir[d] = S->ir[s0 + q];
        ++d;
      }
      free(rm);
    } else {
      for (int64_t q = 0; q < n; ++q) {
        S->tx[d] = S->x[s0 + q];
        S->ty[d] = S->y[s0 + q];
        S->tvx[d] = S->vx[s0 + q];
        S->tvy[d] = S->vy[s0 + q];
        S->tvz[d] = S->vz[s0 + q];
        S->tir[d] = S->ir[s0 + q];
        ++d;
      }
      for (int64_t q = 0; q < ntg - n; ++q) {
        or_stream sp;
        or_stream_init(&sp, c->seed, OR_TAG_DIG_POS, (uint32_t)q, (uint32_t)cell, S->dig_iter);
        if (c->mesh == 1) {
          /* uniform in the annular sector: r^2 and the angle uniform */
          double r = sqrt(S->r2t[iy] + or_uni(&sp, 0) * (S->r2t[iy + 1] - S->r2t[iy]));
          double th = 2.0 * M_PI * ((double)ix + or_uni(&sp, 1)) / (double)c->nx;
          S->tx[d] = r * cos(th);
          S->ty[d] = r * sin(th);
        } else if (c->mesh == 2) {
          S->tx[d] = S->xe[ix] + or_uni(&sp, 0) * (S->xe[ix + 1] - S->xe[ix]);
          S->ty[d] = S->ye[iy] + or_uni(&sp, 1) * (S->ye[iy + 1] - S->ye[iy]);
        } else {
          S->tx[d] = ((double)ix + or_uni(&sp, 0)) * S->dx;
          S->ty[d] = (c->dim == 2) ? ((double)iy + or_uni(&sp, 1)) * S->dy : 0.0;
        }
        if (n > 0) {
          /* replicate a randomly chosen pre-existing particle */
          or_stream st;
          or_stream_init(&st, c->seed, OR_TAG_DIG_SEL, (uint32_t)q, (uint32_t)cell, S->dig_iter);
          int64_t src = (int64_t)(or_uni(&st, 0) * (double)n);
          if (src > n - 1) src = n - 1;
          S->tvx[d] = S->vx[s0 + src];
          S->tvy[d] = S->vy[s0 + src];
          S->tvz[d] = S->vz[s0 + src];
          S->tir[d] = S->ir[s0 + src];
        } else {
          /* empty cell: draw from the Maxwellian of the target state */
          double n1, n2, n3, n4, st_ = sqrt(t[4]);
          or_box_muller(or_uni(&sp, 2), or_uni(&sp, 3), &n1, &n2);
          or_box_muller(or_uni(&sp, 4), or_uni(&sp, 5), &n3, &n4);
          (void)n4;
          S->tvx[d] = t[1] + st_ * n1;
          S->tvy[d] = t[2] + st_ * n2;
          S->tvz[d] = t[3] + st_ * n3;
          S->tir[d] = or_ir_draw(S, t[5], or_uni(&sp, 6), &sp, OR_JX_OWN);
        }
        ++d;
      }
    }
    /* step iii: u*, T_t*, T_r* of the current particles, Eq. (DSMC_macroscopic).
       The mean is taken about the first particle's velocity, so that copies
       of one particle (a cell that held one particle and was refilled) have
       u* equal to that velocity and T_t* = 0 exactly (then a = 1). */
    int64_t np = d - d0;
    if (np > 0) {
      const double rx = S->tvx[d0], ry = S->tvy[d0], rz = S->tvz[d0];
      double sx = 0, sy = 0, sz = 0, si = 0;
      for (int64_t q = d0; q < d; ++q) {
        sx += S->tvx[q] - rx;
        sy += S->tvy[q] - ry;
        sz += S->tvz[q] - rz;
        si += S->tir[q];
      }
      double ux = rx + sx / (double)np, uy = ry + sy / (double)np, uz = rz + sz / (double)np;
      double c2 = 0;
      for (int64_t q = d0; q < d; ++q) {
        double cx = S->tvx[q] - ux, cy = S->tvy[q] - uy, cz = S->tvz[q] - uz;
        c2 += cx * cx + cy * cy + cz * cz;
      }
      double tts = c2 / (3.0 * (double)np);
      double trs = 2.0 * si / (c->d_r * (double)np);
      /* step iv: v <- a v + b, I_r <- c I_r */
      double a = (np >= 2 && tts > 0.0) ? sqrt(t[4] / tts) : 1.0;
      double bx = t[1] - ux * a, by = t[2] - uy * a, bz = t[3] - uz * a;
      double cc = (trs > 0.0) ? t[5] / trs : 1.0;
      for (int64_t q = d0; q < d; ++q) {
        S->tvx[q] = a * S->tvx[q] + bx;
        S->tvy[q] = a * S->tvy[q] + by;
        S->tvz[q] = a * S->tvz[q] + bz;
        S->tir[q] = cc * S->tir[q];
      }
    }
    S->cnt[cell] = d0;
  }
  for (int cell = 0; cell < nc; ++cell) S->start[cell] = S->cnt[cell];
  S->start[nc] = d;
  S->n = d;
  double *tp;
  tp = S->x; S->x = S->tx; S->tx = tp;
  tp = S->y; S->y = S->ty; S->ty = tp;
  tp = S->vx; S->vx = S->tvx; S->tvx = tp;
  tp = S->vy; S->vy = S->tvy; S->tvy = tp;
  tp = S->vz; S->vz = S->tvz; S->tvz = tp;
  tp = S->ir; S->ir = S->tir; S->tir = tp;
  for (int cell = 0; cell < nc; ++cell)
    for (int64_t s = S->start[cell]; s < S->start[cell + 1]; ++s) {
      S->cell[s] = cell;
      S->key[s] = cell;
    }
  S->dig_iter += 1;
  free(idx);
  free(nt);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Accessors                                                                */
/* ------------------------------------------------------------------------ */
int64_t or_num_particles(const or_state *S) { return S->n; }
int or_num_cells(const or_state *S) { return S->ncells; }
uint32_t or_get_step(const or_state *S) { return S->step; }
int64_t or_get_nsamples(const or_state *S) { return S->nsamples; }

void or_get_particles(const or_state *S, double *x, double *y, double *vx, double *vy, double *vz,
                      double *ir, int32_t *cell) {
  size_t nb = sizeof(double) * (size_t)S->n;
  memcpy(x, S->x, nb);
  memcpy(y, S->y, nb);
  memcpy(vx, S->vx, nb);
  memcpy(vy, S->vy, nb);
  memcpy(vz, S->vz, nb);
  memcpy(ir, S->ir, nb);
  memcpy(cell, S->cell, sizeof(int32_t) * (size_t)S->n);
}

void or_get_start(const or_state *S, int64_t *start) {
  memcpy(start, S->start, sizeof(int64_t) * ((size_t)S->ncells + 1));
}

/* Replace the particle state; particles are binned by position (stable). */
int or_set_particles(or_state *S, int64_t n, const double *x, const double *y, const double *vx,
                     const double *vy, const double *vz, const double *ir) {
  if (n < 0 || n > S->cap) return OR_ERR_CAPACITY;
  S->n = n;
  for (int64_t s = 0; s < n; ++s) {
    S->x[s] = x[s];
    S->y[s] = (S->c.dim == 2) ? y[s] : 0.0;
    S->vx[s] = vx[s];
    S->vy[s] = vy[s];
    S->vz[s] = vz[s];
    S->ir[s] = ir[s];
    S->key[s] = or_cell_of(S, S->x[s], S->y[s]);
  }
  or_sort(S);
  return OR_OK;
}

void or_get_acc(const or_state *S, double *out) {
  memcpy(out, S->acc, sizeof(double) * (size_t)S->ncells * OR_NMOM);
}

void or_reset_acc(or_state *S) {
  memset(S->acc, 0, sizeof(double) * (size_t)S->ncells * OR_NMOM);
  S->nsamples = 0;
}

void or_get_sgmax(const or_state *S, double *out) {
  memcpy(out, S->sgmax, sizeof(double) * (size_t)S->ncells);
}

void or_set_sgmax(or_state *S, const double *in) {
  memcpy(S->sgmax, in, sizeof(double) * (size_t)S->ncells);
}

void or_set_step(or_state *S, uint32_t step, uint32_t dig_iter) {
  S->step = step;
  S->dig_iter = dig_iter;
}

/* n_cand, n_coll, n_clip, n_inel, n_hits, n_maxhit */
void or_get_stats(const or_state *S, int64_t out[6]) {
  out[0] = S->n_cand;
  out[1] = S->n_coll;
  out[2] = S->n_clip;
  out[3] = S->n_inel;
  out[4] = S->n_hits;
  out[5] = S->n_maxhit;
}

/* cell volumes */
void or_get_vol(const or_state *S, double *out) { memcpy(out, S->vol, sizeof(double) * (size_t)S->ncells); }

/* particles that entered (annulus freestream) and that left; an entering
 * particle whose partial flight ends outside never entered and is in neither */
void or_get_flow(const or_state *S, int64_t out[2]) {
  out[0] = S->n_inj;
  out[1] = S->n_out;
}

/* per wall: hits, momentum delivered (3), energy delivered */
void or_get_wall(const or_state *S, double out[20]) { memcpy(out, S->wall_tally, sizeof(double) * 20); }
