// dsmc_capi.cu -- the extern "C" entry points declared in include/dig_dsmc.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dig_dsmc.h"
#include "dsmc_internal.h"

using namespace dsmc;

struct dsmc_handle {
  dsmc_config cfg;              // case 0 (the simulation, for a single case)
  std::vector<dsmc_config> cfgs;  // every case
  std::vector<int32_t> cell0;     // host copy of the case offsets (ncases + 1)
  std::vector<int32_t> nx;        // cells per case
  int ncases = 1;
  Params<double>* d_pd = nullptr;  // device tables (see dsmc::Cases)
  Params<float>* d_pf = nullptr;
  CellParams* d_cp = nullptr;
  int32_t* d_cell0 = nullptr;
  int32_t* d_cell_case = nullptr;
  int64_t* d_woff = nullptr;
  int ncells = 0;
  int det = 1;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  Params<double> pd{};
  Params<float> pf{};
  CellParams cp{};
  State<double> sd{};
  State<float> sf{};
  int cur = 0, lay = 0;
  uint32_t step = 0, dig_iter = 0;
  int64_t nsamples = 0;
  int64_t rebuilds = 0;
  double* synth_work = nullptr;
  double* synth_info = nullptr;
  int synth_reuse = 0;       // 2D: start synth_solve from the previous call's factorisation
  int synth_fact_valid = 0;  // 2D: the workspace holds a factorisation of this grid's Jacobian
  int synth_warm = 0;        // 2D: start Newton from the previous call's solution
  int synth_last_ok = 0;     // 2D: the previous call converged (its solution is in the workspace)
  Mlp mlp{};       // HoT surrogate network
  int mlp_t = 0;   // Adam steps taken since the parameters were set
  // annulus tables (device): squared ring radii, rays, outer-face
  // directions, cell volumes, in FP64 and FP32
  double *ann_r2t_d = nullptr, *ann_ray_d = nullptr, *ann_fn_d = nullptr, *ann_vol_d = nullptr;
  double* ann_rt_d = nullptr;  // ring radii (the annulus's synthetic solve)
  double *ref_xe_d = nullptr, *ref_ye_d = nullptr;  // wall-refined box: cell edges (volumes in ann_vol_*)
  float *ref_xe_f = nullptr, *ref_ye_f = nullptr;
  double* ann_mu_d = nullptr;  // expected freestream entries of every outer face per step
  float *ann_r2t_f = nullptr, *ann_ray_f = nullptr, *ann_fn_f = nullptr, *ann_vol_f = nullptr;
  std::string err;
  ~dsmc_handle() {
    // the side stream of the annulus's freestream entry (FP32 layout)
    if (sf.side) {
      cudaStreamSynchronize(sf.side);
      cudaStreamDestroy(sf.side);
    }
    if (sf.ev_fork) cudaEventDestroy(sf.ev_fork);
    if (sf.ev_join) cudaEventDestroy(sf.ev_join);
  }
};

namespace {

int set_err(dsmc_handle* h, int code, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return code;
}

int check_cuda(dsmc_handle* h, const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
  return DSMC_OK;
}

int sync_check(dsmc_handle* h, const char* where) {
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
  return check_cuda(h, where);
}

int32_t host_bin_cap(int32_t count, double slack) {
  const int32_t c = (int32_t)std::ceil(slack * (double)count) + 32;
  return (c + 7) & ~7;
}

int validate(const dsmc_config* c, char* why, size_t n) {
  if (!c) return snprintf(why, n, "null config"), DSMC_ERR_ARG;
  if (c->version != DSMC_ABI_VERSION) return snprintf(why, n, "config version %d != %d", c->version, DSMC_ABI_VERSION), DSMC_ERR_ARG;
  if (c->dim != 1 && c->dim != 2) return snprintf(why, n, "dim must be 1 or 2"), DSMC_ERR_ARG;
  if (c->nx <= 0 || (c->dim == 2 && c->ny <= 0)) return snprintf(why, n, "cell counts must be positive"), DSMC_ERR_ARG;
  if (c->ppc < 0) return snprintf(why, n, "ppc must be >= 0"), DSMC_ERR_ARG;
  if (c->mesh != DSMC_MESH_BOX && c->mesh != DSMC_MESH_ANNULUS && c->mesh != DSMC_MESH_REFINED)
    return snprintf(why, n, "bad mesh"), DSMC_ERR_ARG;
  if (c->mesh == DSMC_MESH_REFINED && (c->dim != 2 || !(c->stretch > 0)))
    return snprintf(why, n, "the wall-refined box is 2D with stretch > 0"), DSMC_ERR_ARG;
  const bool ann = c->mesh == DSMC_MESH_ANNULUS;
  if (ann) {
    if (c->dim != 2 || c->nx < 3) return snprintf(why, n, "the annulus is 2D with nx >= 3"), DSMC_ERR_ARG;
    if (!(c->r_in > 0) || !(c->r_out > c->r_in) || !(c->stretch > 0))
      return snprintf(why, n, "annulus needs 0 < r_in < r_out and stretch > 0"), DSMC_ERR_ARG;
    if (!(c->fs_t > 0) || !(c->fs_rho >= 0) || !std::isfinite(c->fs_u[0]) || !std::isfinite(c->fs_u[1]) ||
        !std::isfinite(c->fs_u[2]))
      return snprintf(why, n, "bad freestream"), DSMC_ERR_ARG;
    if (c->wall_kind[0] != DSMC_WALL_DIFFUSE && c->wall_kind[0] != DSMC_WALL_SPECULAR)
      return snprintf(why, n, "bad wall kind"), DSMC_ERR_ARG;
    if (c->wall_kind[0] == DSMC_WALL_DIFFUSE && !(c->wall_t[0] > 0))
      return snprintf(why, n, "wall temperature must be positive"), DSMC_ERR_ARG;
    if (c->wall_u[0][0] != 0.0 || c->wall_u[0][1] != 0.0 || c->wall_u[0][2] != 0.0)
      return snprintf(why, n, "the cylinder is at rest"), DSMC_ERR_ARG;
  } else if (!(c->lx > 0) || (c->dim == 2 && !(c->ly > 0))) {
    return snprintf(why, n, "domain lengths must be positive"), DSMC_ERR_ARG;
  }
  if (!(c->kn > 0) || !(c->dt > 0) || !(c->z_rot > 0)) return snprintf(why, n, "kn, dt, z_rot must be positive"), DSMC_ERR_ARG;
  if (!(c->omega > 0.5 && c->omega <= 1.0)) return snprintf(why, n, "omega must lie in (0.5, 1]"), DSMC_ERR_ARG;
  if (!(c->alpha > 0.0 && c->alpha <= 2.0)) return snprintf(why, n, "alpha (VSS) must lie in (0, 2]"), DSMC_ERR_ARG;
  if (c->d_r != 2.0 && c->d_r != 3.0) return snprintf(why, n, "d_r must be 2 or 3"), DSMC_ERR_ARG;
  if (c->precision != DSMC_PREC_FP64_DET && c->precision != DSMC_PREC_FP32) return snprintf(why, n, "bad precision"), DSMC_ERR_ARG;
  if (!(c->init_rho > 0) || !(c->init_tt > 0) || !(c->init_tr > 0)) return snprintf(why, n, "initial rho, T must be positive"), DSMC_ERR_ARG;
  const int nw = ann ? 0 : 2 * c->dim;
  for (int w = 0; w < nw; ++w) {
    if (c->wall_kind[w] != DSMC_WALL_DIFFUSE && c->wall_kind[w] != DSMC_WALL_SPECULAR) return snprintf(why, n, "bad wall kind"), DSMC_ERR_ARG;
    if (c->wall_kind[w] == DSMC_WALL_DIFFUSE && !(c->wall_t[w] > 0)) return snprintf(why, n, "wall temperature must be positive"), DSMC_ERR_ARG;
    const int axis = w < 2 ? 0 : 1;
    if (c->wall_u[w][axis] != 0.0) return snprintf(why, n, "wall %d moves along its normal", w), DSMC_ERR_ARG;
  }
  const long long ncells = (long long)c->nx * (c->dim == 2 ? c->ny : 1);
  if (ncells > (1LL << 26)) return snprintf(why, n, "too many cells"), DSMC_ERR_ARG;
  if (c->synth2d != 0 && c->synth2d != 1) return snprintf(why, n, "synth2d must be 0 or 1"), DSMC_ERR_ARG;
  if (c->synth2d) {
    if (c->dim != 2 || (ann ? (c->nx < 5 || c->ny < 3) : (c->nx < 3 || c->ny < 3)))
      return snprintf(why, n, "synth2d needs a 2D box of at least 3 x 3 cells or an annulus of at least 5 x 3"),
             DSMC_ERR_ARG;
    if ((ann ? c->nx : std::min(c->nx, c->ny)) > 500)
      return snprintf(why, n, "synth2d: at most 500 cells on the band's side (the sectors of an annulus)"),
             DSMC_ERR_ARG;
    // the band storage must stay addressable with 64-bit offsets and the
    // unknowns with int
    if (ncells * 5 > (1LL << 28)) return snprintf(why, n, "synth2d: too many cells"), DSMC_ERR_ARG;
  }
  if (ncells * (long long)c->ppc > (1LL << 30)) return snprintf(why, n, "too many particles"), DSMC_ERR_ARG;
  if (c->precision == DSMC_PREC_FP32 && !(c->bin_slack >= 1.0)) return snprintf(why, n, "bin_slack must be >= 1"), DSMC_ERR_ARG;
  return DSMC_OK;
}

struct Plan {
  int ncells, det, tile, ovf_cap;
  int64_t capacity;
  size_t bytes;
};

struct Carver {
  char* base;
  size_t off = 0;
  template <typename P>
  P* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    P* p = base ? reinterpret_cast<P*>(base + off) : nullptr;
    off += sizeof(P) * (count ? count : 1);
    return p;
  }
};

template <typename T>
void carve_state(Carver& cv, const Plan& pl, State<T>& s) {
  const size_t cap = (size_t)pl.capacity, nc = (size_t)pl.ncells;
  for (int b = 0; b < 2; ++b) {
    s.buf[b].x = cv.take<T>(cap);
    s.buf[b].y = cv.take<T>(cap);
    s.buf[b].vx = cv.take<T>(cap);
    s.buf[b].vy = cv.take<T>(cap);
    s.buf[b].vz = cv.take<T>(cap);
    s.buf[b].ir = cv.take<T>(cap);
    s.start[b] = cv.take<int32_t>(nc + 1);
    s.count[b] = cv.take<int32_t>(nc);
  }
  s.cellof = cv.take<int32_t>(cap);
  s.key = cv.take<int32_t>(cap);
  s.dest = cv.take<int32_t>(cap);
  s.scratch_i = cv.take<int32_t>(cap);
  s.owner = cv.take<uint32_t>(cap);
  s.nt = cv.take<int32_t>(nc + 1);
  s.tmp_start = cv.take<int32_t>(nc + 1);
  s.tmp2 = cv.take<int32_t>(nc + 1);
  s.sgmax = cv.take<T>(nc);
  s.acc = cv.take<double>(nc * NMOM);
  s.comp = cv.take<double>(nc * NMOM);
  s.stg = pl.det ? nullptr : cv.take<float>(nc * NMOM);
  s.stc = pl.det ? nullptr : cv.take<float>(nc * NMOM);
  s.tally = cv.take<double>(20);
  s.stats = cv.take<unsigned long long>(ST_NSLOTS);
  s.flags = cv.take<int32_t>(16);
  for (int b = 0; b < 2; ++b) {
    const size_t oc = pl.det ? 1 : (size_t)pl.ovf_cap;
    s.ovf[b].x = reinterpret_cast<float*>(cv.take<float>(oc));
    s.ovf[b].y = cv.take<float>(oc);
    s.ovf[b].vx = cv.take<float>(oc);
    s.ovf[b].vy = cv.take<float>(oc);
    s.ovf[b].vz = cv.take<float>(oc);
    s.ovf[b].ir = cv.take<float>(oc);
    s.ovf[b].dest = cv.take<int32_t>(oc);
    s.ovf[b].count = cv.take<int32_t>(1);
  }
  s.capacity = pl.capacity;
  s.ovf_cap = pl.ovf_cap;
  s.tile = pl.tile;
}

Plan make_plan(const dsmc_config* cs, int ncases, char* base, dsmc_handle* h) {
  Plan pl{};
  pl.det = cs[0].precision == DSMC_PREC_FP64_DET;
  pl.ncells = 0;
  int64_t capacity = 0;
  int tile = 64;
  size_t synth = 0;
  for (int k = 0; k < ncases; ++k) {
    const dsmc_config* c = &cs[k];
    const int nc = c->nx * (c->dim == 2 ? c->ny : 1);
    pl.ncells += nc;
    const int64_t n0 = (int64_t)nc * c->ppc;
    if (pl.det) {
      capacity += c->capacity > 0 ? c->capacity : 2 * n0 + 64;
    } else {
      const int64_t bins = (int64_t)nc * host_bin_cap(c->ppc, c->bin_slack);
      capacity += c->capacity > 0 ? c->capacity : bins + bins / 4 + 1024;
    }
    // particles staged per warp: room for density fluctuations above ppc;
    // larger cells are processed in global memory
    int t = pl.det ? 2 * c->ppc : (5 * c->ppc) / 4 + 32;
    if (t > tile) tile = t;
    if (c->dim == 1) synth += synth1d_work_doubles(nc);
    if (c->dim == 2 && c->synth2d) synth += synth2d_work_doubles(c->nx, c->ny, c->mesh == DSMC_MESH_ANNULUS);
  }
  pl.capacity = capacity;
  tile = pl.det ? (tile + 31) & ~31 : (tile + 15) & ~15;  // FP32: 16-float multiple for bulk copies
  const int tmax = pl.det ? TILE_MAX_OF<double> : TILE_MAX_OF<float>;
  if (tile > tmax) tile = tmax;
  pl.tile = tile;
  pl.ovf_cap = pl.det ? 1 : (int)(pl.capacity / 16 + 1024);
  Carver cv{base};
  if (pl.det) {
    State<double> st{};
    carve_state(cv, pl, st);
    if (h) h->sd = st;
  } else {
    State<float> st{};
    carve_state(cv, pl, st);
    if (h) h->sf = st;
  }
  double* sw = cv.take<double>(synth > 0 ? synth : 1);
  double* si = cv.take<double>(3 * (size_t)ncases + 8);
  Params<double>* pd = cv.take<Params<double>>(ncases);
  Params<float>* pf = cv.take<Params<float>>(ncases);
  CellParams* cp = cv.take<CellParams>(ncases);
  int32_t* c0 = cv.take<int32_t>(ncases + 1);
  int32_t* cc = cv.take<int32_t>(pl.ncells);
  int64_t* wo = cv.take<int64_t>(ncases);
  Mlp ml{};
  ml.theta = cv.take<float>(MLP_NPARAM);
  ml.wbf = cv.take<uint16_t>(MLP_NPARAM);
  ml.m = cv.take<float>(MLP_NPARAM);
  ml.v = cv.take<float>(MLP_NPARAM);
  ml.grad = cv.take<float>(MLP_NPARAM);
  ml.partial = cv.take<float>((size_t)MLP_GRID * MLP_NPARAM);
  ml.part_loss = cv.take<double>(MLP_GRID);
  ml.X = cv.take<float>((size_t)pl.ncells * 12);
  ml.Y = cv.take<float>((size_t)pl.ncells * 5);
  ml.S = cv.take<float>((size_t)pl.ncells * 4);
  ml.w = cv.take<float>(pl.ncells);
  ml.out = cv.take<float>((size_t)pl.ncells * 5);
  ml.scal = cv.take<double>(8);
  ml.count = cv.take<int32_t>(4);
  ml.jacc = cv.take<double>((size_t)pl.ncells * 16);
  const bool ann = cs[0].mesh == DSMC_MESH_ANNULUS, ref = cs[0].mesh == DSMC_MESH_REFINED;
  const size_t nr1 = ann ? (size_t)cs[0].ny + 1 : 1, nray = ann ? 2 * ((size_t)cs[0].nx + 1) : 1;
  const size_t nfn = ann ? 2 * (size_t)cs[0].nx : 1, nvol = (ann || ref) ? (size_t)pl.ncells : 1;
  const size_t nxe = ref ? (size_t)cs[0].nx + 1 : 1, nye = ref ? (size_t)cs[0].ny + 1 : 1;
  double* r_xed = cv.take<double>(nxe);
  double* r_yed = cv.take<double>(nye);
  float* r_xef = cv.take<float>(nxe);
  float* r_yef = cv.take<float>(nye);
  double* a_r2d = cv.take<double>(nr1);
  double* a_rtd = cv.take<double>(nr1);
  double* a_rayd = cv.take<double>(nray);
  double* a_fnd = cv.take<double>(nfn);
  double* a_vold = cv.take<double>(nvol);
  float* a_r2f = cv.take<float>(nr1);
  float* a_rayf = cv.take<float>(nray);
  float* a_fnf = cv.take<float>(nfn);
  float* a_volf = cv.take<float>(nvol);
  double* a_mu = cv.take<double>(ann ? (size_t)cs[0].nx : 1);
  if (h) {
    h->ref_xe_d = r_xed;
    h->ref_ye_d = r_yed;
    h->ref_xe_f = r_xef;
    h->ref_ye_f = r_yef;
    h->ann_mu_d = a_mu;
    h->ann_r2t_d = a_r2d;
    h->ann_rt_d = a_rtd;
    h->ann_ray_d = a_rayd;
    h->ann_fn_d = a_fnd;
    h->ann_vol_d = a_vold;
    h->ann_r2t_f = a_r2f;
    h->ann_ray_f = a_rayf;
    h->ann_fn_f = a_fnf;
    h->ann_vol_f = a_volf;
    h->mlp = ml;
    h->synth_work = sw;
    h->synth_info = si;
    h->d_pd = pd;
    h->d_pf = pf;
    h->d_cp = cp;
    h->d_cell0 = c0;
    h->d_cell_case = cc;
    h->d_woff = wo;
  }
  pl.bytes = cv.off + 256;
  return pl;
}

// Annulus geometry: ring radii R_j = r_in + (r_out - r_in) (q^j - 1) / (q^ny -
// 1) (q = stretch, uniform for q = 1) and their squares, rays (cos, sin) at
// 2 pi k / nx (ray nx = ray 0), outer-face centre directions at 2 pi (k +
// 1/2) / nx, cell volumes (pi / nx) (R_{j+1}^2 - R_j^2).
struct AnnTables {
  std::vector<double> rt, r2t, ray, fn, vol;
  double area = 0.0;
};

AnnTables ann_tables(const dsmc_config* c) {
  AnnTables t;
  const int nr = c->ny, nt = c->nx;
  const double q = c->stretch;
  std::vector<double> rt(nr + 1);
  for (int j = 0; j <= nr; ++j) {
    const double f = (q == 1.0) ? (double)j / (double)nr : (std::pow(q, (double)j) - 1.0) / (std::pow(q, (double)nr) - 1.0);
    rt[j] = c->r_in + (c->r_out - c->r_in) * f;
  }
  rt[0] = c->r_in;
  rt[nr] = c->r_out;
  t.rt = rt;
  t.r2t.resize(nr + 1);
  for (int j = 0; j <= nr; ++j) t.r2t[j] = rt[j] * rt[j];
  t.ray.resize(2 * (nt + 1));
  t.fn.resize(2 * nt);
  for (int k = 0; k < nt; ++k) {
    const double th = 2.0 * M_PI * (double)k / (double)nt;
    t.ray[2 * k] = std::cos(th);
    t.ray[2 * k + 1] = std::sin(th);
    const double tm = 2.0 * M_PI * ((double)k + 0.5) / (double)nt;
    t.fn[2 * k] = std::cos(tm);
    t.fn[2 * k + 1] = std::sin(tm);
  }
  t.ray[2 * nt] = t.ray[0];
  t.ray[2 * nt + 1] = t.ray[1];
  const double half = M_PI / (double)nt;
  t.vol.resize((size_t)nr * nt);
  for (int j = 0; j < nr; ++j)
    for (int k = 0; k < nt; ++k) t.vol[(size_t)j * nt + k] = half * (t.r2t[j + 1] - t.r2t[j]);
  for (double v : t.vol) t.area += v;
  return t;
}

// Wall-refined box: cell edges along an axis of n cells and length L, widths
// proportional to q^min(i, n-1-i) (growing by q from both walls to the
// middle), scaled to sum to L; e[0] = 0, e[n] = L
std::vector<double> refined_edges(int n, double L, double q) {
  std::vector<double> e(n + 1);
  double sum = 0.0;
  for (int i = 0; i < n; ++i) sum += std::pow(q, (double)(i < n - 1 - i ? i : n - 1 - i));
  e[0] = 0.0;
  for (int i = 0; i < n; ++i) e[i + 1] = e[i] + L * std::pow(q, (double)(i < n - 1 - i ? i : n - 1 - i)) / sum;
  e[n] = L;
  return e;
}

template <typename T>
void fill_params(const dsmc_config* c, Params<T>& p, CellParams& cp) {
  const double w = c->omega, a = c->alpha;
  const bool ann = c->mesh == DSMC_MESH_ANNULUS;
  const int ny = (c->dim == 2) ? c->ny : 1;
  const double lx = ann ? 2.0 * M_PI : c->lx, ly = ann ? c->r_out - c->r_in : ((c->dim == 2) ? c->ly : 1.0);
  const double dx = lx / (double)c->nx;
  const double dy = (c->dim == 2) ? ly / (double)ny : 1.0;
  // annulus: the mean cell volume (cells differ; per-cell volumes in tables)
  const double vcell = ann ? ann_tables(c).area / (double)(c->nx * ny) : dx * dy;
  const double fnum = c->init_rho * vcell / (double)(c->ppc > 0 ? c->ppc : 1);
  const double mu_ref = c->kn * std::sqrt(2.0 / M_PI);
  const double kv = 5.0 * (a + 1.0) * (a + 2.0) / (a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w));
  const double c_sigma = kv / (mu_ref * std::pow(4.0, 1.0 - w) * (2.0 / std::sqrt(M_PI)) * std::tgamma(2.5 - w));
  const double p_inel = a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (a + 1.0) * (a + 2.0) * c->z_rot);
  p.dim = c->dim;
  p.nx = c->nx;
  p.ny = ny;
  p.ncells = c->nx * ny;
  p.lx = (T)lx;
  p.ly = (T)ly;
  p.dx = (T)dx;
  p.dy = (T)dy;
  p.sx = (T)((double)c->nx / lx);
  p.sy = (T)((double)ny / ly);
  p.vcell = (T)vcell;
  p.fnum = (T)fnum;
  p.dt = (T)c->dt;
  p.c_sigma = (T)c_sigma;
  p.p_inel = (T)p_inel;
  p.vhs_e = (T)(2.0 - 2.0 * w);
  p.bl_exp = (T)(1.0 / (2.5 - w));
  {
    // Borgnakke-Larsen partition Beta(a, b) and its mode (used for d_r = 3)
    const double ba = 0.5 * c->d_r, bb = 2.5 - w;
    p.d_r3 = (c->d_r == 3.0) ? 1 : 0;
    p.bl_am1 = (T)(ba - 1.0);
    p.bl_bm1 = (T)(bb - 1.0);
    p.bl_xs = (T)((ba - 1.0) / (ba + bb - 2.0));
  }
  p.vss = (a != 1.0) ? 1 : 0;
  p.vss_ia = (T)(1.0 / a);
  p.collisions = c->collisions ? 1 : 0;
  for (int k = 0; k < 4; ++k) {
    p.wall_kind[k] = c->wall_kind[k];
    p.wall_t[k] = (T)c->wall_t[k];
    for (int q = 0; q < 3; ++q) p.wall_u[k][q] = (T)c->wall_u[k][q];
  }
  p.k0 = (uint32_t)(c->seed & 0xffffffffu);
  p.k1 = (uint32_t)(c->seed >> 32);
  p.ppc = c->ppc;
  p.init_tt = (T)c->init_tt;
  p.init_tr = (T)c->init_tr;
  for (int q = 0; q < 3; ++q) p.init_u[q] = (T)c->init_u[q];
  p.init_rho = (T)c->init_rho;
  p.mesh = ann ? 1 : (c->mesh == DSMC_MESH_REFINED ? 2 : 0);
  p.r2t = p.ray = p.fnrm = p.vol = nullptr;  // annulus / refined-box tables: set_ann_tables, set_ref_tables
  p.xe = p.ye = nullptr;
  p.r_in = (T)c->r_in;
  p.r_out = (T)c->r_out;
  p.fs_rho = (T)c->fs_rho;
  p.fs_t = (T)c->fs_t;
  for (int q = 0; q < 3; ++q) p.fs_u[q] = (T)c->fs_u[q];
  // FP64 cell parameters
  cp.dim = c->dim;
  cp.nx = c->nx;
  cp.ny = ny;
  cp.ncells = c->nx * ny;
  cp.lx = lx;
  cp.ly = ly;
  cp.dx = dx;
  cp.dy = dy;
  cp.vcell = vcell;
  cp.fnum = fnum;
  cp.d_r = c->d_r;
  cp.omega = w;
  cp.mu_ref = mu_ref;
  cp.z_rot = c->z_rot;
  // Eq. (kappa_A): (kappa_t, kappa_r) = (mu/2) A^-1 (5, d_r)
  const double* A = c->a_matrix;
  const double det = A[0] * A[3] - A[1] * A[2];
  cp.kappa_t = 0.5 * (A[3] * 5.0 - A[1] * c->d_r) / det;
  cp.kappa_r = 0.5 * (-A[2] * 5.0 + A[0] * c->d_r) / det;
  cp.kn_ref = c->kn_ref;
  cp.k0 = p.k0;
  cp.k1 = p.k1;
  cp.mesh = p.mesh;
  cp.vol = nullptr;
  cp.r2t = nullptr;
  cp.rt = nullptr;
  cp.xe = cp.ye = nullptr;
}

// annulus: upload the tables (FP64 and FP32) and point the parameters at them
int set_ann_tables(dsmc_handle* h) {
  const AnnTables t = ann_tables(&h->cfg);
  auto f32 = [](const std::vector<double>& v) {
    std::vector<float> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
    return o;
  };
  const std::vector<float> r2f = f32(t.r2t), rayf = f32(t.ray), fnf = f32(t.fn), volf = f32(t.vol);
  cudaStream_t st = h->stream;
  cudaMemcpyAsync(h->ann_r2t_d, t.r2t.data(), sizeof(double) * t.r2t.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_rt_d, t.rt.data(), sizeof(double) * t.rt.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_ray_d, t.ray.data(), sizeof(double) * t.ray.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_fn_d, t.fn.data(), sizeof(double) * t.fn.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_vol_d, t.vol.data(), sizeof(double) * t.vol.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_r2t_f, r2f.data(), sizeof(float) * r2f.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_ray_f, rayf.data(), sizeof(float) * rayf.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_fn_f, fnf.data(), sizeof(float) * fnf.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_vol_f, volf.data(), sizeof(float) * volf.size(), cudaMemcpyHostToDevice, st);
  const cudaError_t e = cudaStreamSynchronize(st);  // the host vectors die here
  if (e != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "annulus tables: %s", cudaGetErrorString(e));
  h->pd.r2t = h->ann_r2t_d;
  h->pd.ray = h->ann_ray_d;
  h->pd.fnrm = h->ann_fn_d;
  h->pd.vol = h->ann_vol_d;
  h->pf.r2t = h->ann_r2t_f;
  h->pf.ray = h->ann_ray_f;
  h->pf.fnrm = h->ann_fn_f;
  h->pf.vol = h->ann_vol_f;
  h->cp.vol = h->ann_vol_d;
  h->cp.r2t = h->ann_r2t_d;
  h->cp.rt = h->ann_rt_d;
  return DSMC_OK;
}

// wall-refined box: upload the edge and volume tables (FP64 and FP32) and
// point the parameters at them
int set_ref_tables(dsmc_handle* h) {
  const dsmc_config* c = &h->cfg;
  const std::vector<double> xe = refined_edges(c->nx, c->lx, c->stretch);
  const std::vector<double> ye = refined_edges(c->ny, c->ly, c->stretch);
  std::vector<double> vol((size_t)c->nx * c->ny);
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) vol[(size_t)j * c->nx + i] = (xe[i + 1] - xe[i]) * (ye[j + 1] - ye[j]);
  auto f32 = [](const std::vector<double>& v) {
    std::vector<float> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
    return o;
  };
  const std::vector<float> xef = f32(xe), yef = f32(ye), volf = f32(vol);
  cudaStream_t st = h->stream;
  cudaMemcpyAsync(h->ref_xe_d, xe.data(), sizeof(double) * xe.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ref_ye_d, ye.data(), sizeof(double) * ye.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_vol_d, vol.data(), sizeof(double) * vol.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ref_xe_f, xef.data(), sizeof(float) * xef.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ref_ye_f, yef.data(), sizeof(float) * yef.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ann_vol_f, volf.data(), sizeof(float) * volf.size(), cudaMemcpyHostToDevice, st);
  const cudaError_t e = cudaStreamSynchronize(st);  // the host vectors die here
  if (e != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "refined-box tables: %s", cudaGetErrorString(e));
  h->pd.xe = h->ref_xe_d;
  h->pd.ye = h->ref_ye_d;
  h->pd.vol = h->ann_vol_d;
  h->pf.xe = h->ref_xe_f;
  h->pf.ye = h->ref_ye_f;
  h->pf.vol = h->ann_vol_f;
  h->cp.vol = h->ann_vol_d;
  h->cp.xe = h->ref_xe_d;
  h->cp.ye = h->ref_ye_d;
  return DSMC_OK;
}

// cell volumes of the wall-refined box (host)
std::vector<double> refined_volumes(const dsmc_config* c) {
  const std::vector<double> xe = refined_edges(c->nx, c->lx, c->stretch);
  const std::vector<double> ye = refined_edges(c->ny, c->ly, c->stretch);
  std::vector<double> vol((size_t)c->nx * c->ny);
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) vol[(size_t)j * c->nx + i] = (xe[i + 1] - xe[i]) * (ye[j + 1] - ye[j]);
  return vol;
}

double sgmax0(const dsmc_config* c, double c_sigma) {
  double tref = c->init_tt;
  double uref = std::sqrt(c->init_u[0] * c->init_u[0] + c->init_u[1] * c->init_u[1] + c->init_u[2] * c->init_u[2]);
  double umax = 0.0;
  const int nw = (c->mesh == DSMC_MESH_ANNULUS) ? 1 : 2 * c->dim;  // annulus: the cylinder
  for (int w = 0; w < nw; ++w) {
    if (c->wall_kind[w] == 0 && c->wall_t[w] > tref) tref = c->wall_t[w];
    const double uw = std::sqrt(c->wall_u[w][0] * c->wall_u[w][0] + c->wall_u[w][1] * c->wall_u[w][1] +
                                c->wall_u[w][2] * c->wall_u[w][2]);
    if (uw > umax) umax = uw;
  }
  uref += umax;
  return c_sigma * std::pow(4.0 * std::sqrt(tref) + uref, 2.0 - 2.0 * c->omega);
}

template <typename T>
__global__ void k_fill(T* a, int n, T v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = v;
}

template <typename T>
int init_state(dsmc_handle* h, State<T>& s, Params<T>& p0, Params<T>* d_p) {
  cudaStream_t st = h->stream;
  const int nc = h->ncells;
  const int ncases = h->ncases;
  cudaMemsetAsync(s.stats, 0, sizeof(unsigned long long) * ST_NSLOTS, st);
  cudaMemsetAsync(s.tally, 0, sizeof(double) * 20, st);
  cudaMemsetAsync(s.flags, 0, sizeof(int32_t) * 16, st);
  cudaMemsetAsync(s.acc, 0, sizeof(double) * nc * NMOM, st);
  cudaMemsetAsync(s.comp, 0, sizeof(double) * nc * NMOM, st);
  if (s.stg) {
    cudaMemsetAsync(s.stg, 0, sizeof(float) * nc * NMOM, st);
    cudaMemsetAsync(s.stc, 0, sizeof(float) * nc * NMOM, st);
  }
  for (int b = 0; b < 2; ++b) {
    cudaMemsetAsync(s.count[b], 0, sizeof(int32_t) * nc, st);
    cudaMemsetAsync(s.ovf[b].count, 0, sizeof(int32_t), st);
  }
  cudaMemsetAsync(s.buf[0].y, 0, sizeof(T) * (size_t)s.capacity, st);
  cudaMemsetAsync(s.buf[1].y, 0, sizeof(T) * (size_t)s.capacity, st);
  // per-case tables, per-cell layout and (sigma g)_max
  std::vector<Params<T>> pt(ncases);
  std::vector<Params<double>> pdv(ncases);
  std::vector<CellParams> cpt(ncases);
  std::vector<int32_t> cell_case(nc), start(nc + 1);
  std::vector<T> sg(nc);
  std::vector<int64_t> woff(ncases);
  int64_t total = 0, wacc = 0;
  int32_t slot = 0;
  // annulus, wall-refined box (one case): the initial count of every cell,
  // drawn on the device from its volume
  const bool ann = h->cfg.mesh != DSMC_MESH_BOX;
  std::vector<int32_t> counts;
  std::vector<double> vol;
  if (ann) {
    counts.resize(nc);
    vol = h->cfg.mesh == DSMC_MESH_ANNULUS ? ann_tables(&h->cfg).vol : refined_volumes(&h->cfg);
    Ops<T>::ann_counts(h->pd, nc, s.nt, st);
    cudaMemcpyAsync(counts.data(), s.nt, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "dsmc_init: %s", cudaGetErrorString(e));
  }
  for (int k = 0; k < ncases; ++k) {
    const dsmc_config* c = &h->cfgs[k];
    fill_params<T>(c, pt[k], cpt[k]);
    fill_params<double>(c, pdv[k], cpt[k]);
    if (ann) {
      pt[k] = p0;  // with the table pointers
      pdv[k] = h->pd;
      cpt[k] = h->cp;
    }
    const int32_t cap0 = h->det ? c->ppc : host_bin_cap(c->ppc, c->bin_slack);
    const T sg0 = (T)sgmax0(c, (double)pdv[k].c_sigma);
    for (int i = h->cell0[k]; i < h->cell0[k + 1]; ++i) {
      cell_case[i] = k;
      start[i] = slot;
      if (ann) {
        const int32_t nominal = (int32_t)(vol[i] / h->cp.fnum + 0.5);
        slot += h->det ? counts[i] : host_bin_cap(std::max(counts[i], nominal), c->bin_slack);
        total += counts[i];
      } else {
        slot += cap0;
      }
      sg[i] = sg0;
    }
    if (!ann) total += (int64_t)(h->cell0[k + 1] - h->cell0[k]) * c->ppc;
    woff[k] = wacc;
    if (c->dim == 1) wacc += (int64_t)synth1d_work_doubles(h->nx[k]);
  }
  s.pinj = h->pd;
  s.inj_mu = nullptr;
  s.inj_max = 0;
  if (h->cfg.mesh == DSMC_MESH_ANNULUS) {
    // expected entries per face and step, and a bound on one step's entries
    std::vector<double> mu(h->cfg.nx);
    Ops<T>::inflow_means(h->pd, h->ann_mu_d, st);
    cudaMemcpyAsync(mu.data(), h->ann_mu_d, sizeof(double) * mu.size(), cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "dsmc_init: %s", cudaGetErrorString(e));
    long long bound = 0;
    for (double m : mu) bound += (long long)std::floor(m) + 1;
    if (bound > (1LL << 30)) return set_err(h, DSMC_ERR_ARG, "freestream entry too large per step");
    s.inj_mu = h->ann_mu_d;
    s.inj_max = (int)bound;
    if (!h->det) {
      if (cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming) != cudaSuccess)
        return set_err(h, DSMC_ERR_CUDA, "dsmc_init: side stream");
    }
  }
  start[nc] = slot;
  if ((int64_t)slot > s.capacity)
    return set_err(h, DSMC_ERR_CAPACITY, "initial bins need %lld slots, capacity %lld", (long long)slot,
                   (long long)s.capacity);
  cudaMemcpyAsync(d_p, pt.data(), sizeof(Params<T>) * ncases, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->d_cp, cpt.data(), sizeof(CellParams) * ncases, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->d_cell0, h->cell0.data(), sizeof(int32_t) * (ncases + 1), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->d_cell_case, cell_case.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->d_woff, woff.data(), sizeof(int64_t) * ncases, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s.start[0], start.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s.sgmax, sg.data(), sizeof(T) * nc, cudaMemcpyHostToDevice, st);
  s.cases = Cases<T>{d_p, h->d_cp, h->d_cell0, h->d_cell_case, ncases};
  s.batch = ncases > 1;
  s.gen = false;
  for (int k = 0; k < ncases; ++k)
    if (h->cfgs[k].d_r != 2.0 || h->cfgs[k].alpha != 1.0) s.gen = true;
  s.ncells = nc;
  h->cur = 0;
  h->lay = 0;
  Ops<T>::init_batch(p0, s, nc, 0, 0, st, ann ? s.nt : nullptr);
  s.nparticles = (int)total;
  s.slack = h->cfgs[0].bin_slack;
  // the host vectors above must outlive the copies
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "dsmc_init: %s", cudaGetErrorString(e));
  return check_cuda(h, "dsmc_init");
}

// HoT network: Glorot-uniform weights (bounds sqrt(6 / (n_in + n_out))) and
// zero biases from a splitmix64 stream, uploaded with the bfloat16 copies;
// the Adam state is cleared
int mlp_upload(dsmc_handle* h, const float* host) {
  cudaMemcpyAsync(h->mlp.theta, host, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, h->stream);
  cudaMemsetAsync(h->mlp.m, 0, sizeof(float) * MLP_NPARAM, h->stream);
  cudaMemsetAsync(h->mlp.v, 0, sizeof(float) * MLP_NPARAM, h->stream);
  // a new network starts the judge's statistics afresh
  cudaMemsetAsync(h->mlp.jacc, 0, sizeof(double) * 16 * (size_t)h->ncells, h->stream);
  mlp_to_bf16(h->mlp, h->stream);
  h->mlp_t = 0;
  return sync_check(h, "hot_mlp parameters");
}

int mlp_init_params(dsmc_handle* h, uint64_t seed) {
  static const int nin[4] = {12, 64, 64, 64}, nout[4] = {64, 64, 64, 5};
  std::vector<float> th(MLP_NPARAM, 0.f);
  uint64_t z = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto next = [&]() {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return ((double)(x >> 11) + 0.5) * 0x1p-53;
  };
  int o = 0;
  for (int k = 0; k < 4; ++k) {
    const double lim = std::sqrt(6.0 / (double)(nin[k] + nout[k]));
    for (int q = 0; q < nin[k] * nout[k]; ++q) th[o + q] = (float)((2.0 * next() - 1.0) * lim);
    o += nin[k] * nout[k] + nout[k];
  }
  return mlp_upload(h, th.data());
}

// inputs of the cells (and targets where hot is given)
void mlp_data(dsmc_handle* h, const double* fields, const double* hot, const double* kngll, const uint8_t* mask) {
  mlp_prepare(h->mlp, h->d_cp, h->d_cell_case, h->d_cell0, h->ncells, fields, hot, kngll, mask, h->stream);
}

int mlp_count(dsmc_handle* h, int* n) {
  cudaMemcpyAsync(n, h->mlp.count, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  return sync_check(h, "hot_mlp");
}

int init_cases(const dsmc_config* cfgs, int ncases, void* dev_workspace, size_t bytes, void* stream,
               dsmc_handle** out) {
  if (!out || !cfgs || ncases < 1) return DSMC_ERR_ARG;
  *out = nullptr;
  char why[256];
  for (int k = 0; k < ncases; ++k) {
    const int rc = validate(&cfgs[k], why, sizeof why);
    if (rc) return rc;
    if (cfgs[k].dim != cfgs[0].dim || cfgs[k].precision != cfgs[0].precision) return DSMC_ERR_ARG;
    if (cfgs[k].mesh != DSMC_MESH_BOX && ncases != 1) return DSMC_ERR_ARG;  // the annulus, the refined box run alone
    if (cfgs[k].synth2d && ncases != 1) return DSMC_ERR_ARG;                    // so does the 2D solve
    // the FP32 fused step has its d_r = 3 / VSS instantiation for single cases only
    if (ncases != 1 && cfgs[k].precision == DSMC_PREC_FP32 && (cfgs[k].d_r != 2.0 || cfgs[k].alpha != 1.0))
      return DSMC_ERR_ARG;
  }
  const Plan pl = make_plan(cfgs, ncases, nullptr, nullptr);
  if (!dev_workspace || bytes < pl.bytes) return DSMC_ERR_ARG;
  dsmc_handle* h = new (std::nothrow) dsmc_handle();
  if (!h) return DSMC_ERR_ARG;
  h->cfgs.assign(cfgs, cfgs + ncases);
  h->ncases = ncases;
  h->cell0.assign(ncases + 1, 0);
  h->nx.assign(ncases, 0);
  for (int k = 0; k < ncases; ++k) {
    dsmc_config& c = h->cfgs[k];
    if (c.dim == 1) {
      c.ny = 1;
      c.ly = 1.0;
    }
    h->nx[k] = c.nx;
    h->cell0[k + 1] = h->cell0[k] + c.nx * c.ny;
  }
  h->cfg = h->cfgs[0];
  h->ncells = pl.ncells;
  h->det = pl.det;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->ws = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(dev_workspace) + 255) & ~(uintptr_t)255);
  h->ws_bytes = bytes;
  make_plan(h->cfgs.data(), ncases, h->ws, h);
  fill_params<double>(&h->cfg, h->pd, h->cp);
  fill_params<float>(&h->cfg, h->pf, h->cp);
  int r;
  if (h->cfg.mesh == DSMC_MESH_ANNULUS || h->cfg.mesh == DSMC_MESH_REFINED) {
    r = h->cfg.mesh == DSMC_MESH_ANNULUS ? set_ann_tables(h) : set_ref_tables(h);
    if (r) {
      delete h;
      return r;
    }
  }
  if (h->det) {
    Ops<double>::configure(pl.tile);
    r = init_state<double>(h, h->sd, h->pd, h->d_pd);
  } else {
    Ops<float>::configure(pl.tile);
    r = init_state<float>(h, h->sf, h->pf, h->d_pf);
  }
  if (!r) r = mlp_init_params(h, h->cfg.seed);
  if (r) {
    delete h;
    return r;
  }
  *out = h;
  return DSMC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int dsmc_workspace_size(const dsmc_config* cfg, size_t* bytes) {
  return dsmc_batch_workspace_size(cfg, 1, bytes);
}

int dsmc_init(const dsmc_config* cfg, void* dev_workspace, size_t bytes, void* stream, dsmc_handle** out) {
  return init_cases(cfg, 1, dev_workspace, bytes, stream, out);
}

int dsmc_batch_workspace_size(const dsmc_config* cfgs, int ncases, size_t* bytes) {
  char why[256];
  if (!bytes || !cfgs || ncases < 1) return DSMC_ERR_ARG;
  for (int k = 0; k < ncases; ++k) {
    const int rc = validate(&cfgs[k], why, sizeof why);
    if (rc) return rc;
    if (cfgs[k].dim != cfgs[0].dim || cfgs[k].precision != cfgs[0].precision) return DSMC_ERR_ARG;
    if (cfgs[k].mesh != DSMC_MESH_BOX && ncases != 1) return DSMC_ERR_ARG;
    if (cfgs[k].synth2d && ncases != 1) return DSMC_ERR_ARG;
    if (ncases != 1 && cfgs[k].precision == DSMC_PREC_FP32 && (cfgs[k].d_r != 2.0 || cfgs[k].alpha != 1.0))
      return DSMC_ERR_ARG;
  }
  *bytes = make_plan(cfgs, ncases, nullptr, nullptr).bytes;
  return DSMC_OK;
}

int dsmc_batch_init(const dsmc_config* cfgs, int ncases, void* dev_workspace, size_t bytes, void* stream,
                    dsmc_handle** out) {
  return init_cases(cfgs, ncases, dev_workspace, bytes, stream, out);
}

int dsmc_destroy(dsmc_handle* h) {
  delete h;
  return DSMC_OK;
}

const char* dsmc_last_error(const dsmc_handle* h) { return h ? h->err.c_str() : "null handle"; }

int dsmc_step(dsmc_handle* h, int nsteps, int sample) {
  if (!h || nsteps < 0) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  if (nsteps == 0) return DSMC_OK;
  if (h->det) {
    for (int k = 0; k < nsteps; ++k) {
      Ops<double>::step_det(h->pd, h->sd, h->cur, h->lay, h->step, sample, h->stream);
      h->step += 1;
      if (sample) h->nsamples += 1;
      if (h->sd.lost) return set_err(h, DSMC_ERR_CAPACITY, "dsmc_step: freestream entries exceed the capacity");
    }
    return check_cuda(h, "dsmc_step");
  }
  Ops<float>::step_bins(h->pf, h->sf, h->cur, h->lay, h->step, nsteps, sample, h->stream);
  h->step += (uint32_t)nsteps;
  if (sample) h->nsamples += nsteps;
  int r = check_cuda(h, "dsmc_step");
  if (r) return r;
  // rebuild the bins if a particle overflowed or a bin came near its capacity
  int32_t ovf = 0, timeout = 0;
  unsigned long long nearfull = 0;
  cudaMemcpyAsync(&ovf, h->sf.ovf[h->cur].count, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(&nearfull, h->sf.stats + ST_NEARFULL, sizeof(nearfull), cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(&timeout, h->sf.flags + 8, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  r = sync_check(h, "dsmc_step (bin check)");
  if (r) return r;
  if (timeout & 1) return set_err(h, DSMC_ERR_TIMEOUT, "dsmc_step: a cell's bulk copy did not complete in time");
  if ((timeout & 2) || ovf > h->sf.ovf_cap)
    return set_err(h, DSMC_ERR_CAPACITY, "dsmc_step: the overflow list was full, particles were lost");
  if (ovf > 0 || nearfull > 0) {
    Ops<float>::rebin(h->pf, h->sf, h->cur, h->lay, 1, h->sf.slack, h->stream);
    cudaMemsetAsync(h->sf.stats + ST_NEARFULL, 0, sizeof(unsigned long long), h->stream);
    int32_t fl[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(fl, h->sf.flags, sizeof fl, cudaMemcpyDeviceToHost, h->stream);
    r = sync_check(h, "dsmc_step (rebin)");
    if (r) return r;
    h->rebuilds += 1;
    if (fl[2]) return set_err(h, DSMC_ERR_CAPACITY, "cell bins do not fit the capacity");
  }
  return DSMC_OK;
}

int dsmc_sample(dsmc_handle* h, double* dev_fields, int reset) {
  if (!h || !dev_fields) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  const double* acc = h->det ? h->sd.acc : h->sf.acc;
  double* comp = h->det ? h->sd.comp : h->sf.comp;
  launch_fields(h->d_cp, h->d_cell_case, h->ncells, acc, comp, h->nsamples, dev_fields, h->stream);
  if (reset) {
    cudaMemsetAsync(const_cast<double*>(acc), 0, sizeof(double) * h->ncells * NMOM, h->stream);
    cudaMemsetAsync(comp, 0, sizeof(double) * h->ncells * NMOM, h->stream);
    h->nsamples = 0;
  }
  return check_cuda(h, "dsmc_sample");
}

int dsmc_hot(dsmc_handle* h, const double* dev_fields, double* dev_hot, double* dev_kngll, uint8_t* dev_mask) {
  if (!h || !dev_fields || !dev_hot) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  launch_hot(h->d_cp, h->d_cell_case, h->d_cell0, h->ncells, dev_fields, dev_hot, dev_kngll, dev_mask, h->stream);
  return check_cuda(h, "dsmc_hot");
}

// the 2D box (single case, workspace reserved by synth2d)
static int synth_solve_2d(dsmc_handle* h, const double* dev_fields, const double* dev_hot, double* dev_out,
                          int* host_iters, double* host_resid) {
  const dsmc_config& c = h->cfg;
  if (h->ncases != 1 || !c.synth2d)
    return set_err(h, DSMC_ERR_ARG, "synth_solve: a 2D case needs synth2d = 1 (workspace for the banded solve)");
  const int n_m = std::min(c.n_m > 0 ? c.n_m : 2000, 100);
  const double tol = c.synth_tol > 0 ? c.synth_tol : 1e-5;
  int singular = 0;
  const int e = launch_synth2d(h->cp, dev_fields, dev_hot, dev_out, h->synth_work, n_m, tol, h->synth_info,
                               &singular, h->synth_reuse && h->synth_fact_valid,
                               h->synth_warm && h->synth_last_ok, h->stream);
  h->synth_fact_valid = e == 0;
  h->synth_last_ok = 0;
  if (e == S2_TIMEOUT_RC) return set_err(h, DSMC_ERR_TIMEOUT, "synth_solve: a wait of the substitution gave up");
  if (e) return set_err(h, DSMC_ERR_CUDA, "synth_solve: %s", cudaGetErrorString((cudaError_t)e));
  double info[3];
  cudaMemcpyAsync(info, h->synth_info, sizeof info, cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "synth_solve");
  if (r) return r;
  if (host_iters) *host_iters = (int)info[0];
  if (host_resid) *host_resid = info[1];
  const int status = (int)info[2];
  if (status == 2)
    return set_err(h, DSMC_ERR_NUMERIC, "synth_solve: no update keeps rho, T positive%s",
                   singular ? " (singular Jacobian)" : "");
  if (status == 1) return set_err(h, DSMC_ERR_NOT_CONVERGED, "synth_solve: %d iterations without convergence", n_m);
  h->synth_last_ok = 1;
  return DSMC_OK;
}

int dsmc_synth_reuse(dsmc_handle* h, int on) {
  if (!h || h->cfg.dim != 2 || !h->cfg.synth2d || h->ncases != 1)
    return set_err(h, DSMC_ERR_ARG, "dsmc_synth_reuse: needs a single 2D case with synth2d = 1");
  h->synth_reuse = (on & 1) != 0;
  h->synth_warm = (on & 2) != 0;
  return DSMC_OK;
}

int synth_solve(dsmc_handle* h, const double* dev_fields, const double* dev_hot, double* dev_out, int* host_iters,
                double* host_resid) {
  if (!h || !dev_fields || !dev_hot || !dev_out) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  if (h->cfg.dim == 2) return synth_solve_2d(h, dev_fields, dev_hot, dev_out, host_iters, host_resid);
  int n_m = 0;
  double tol = 1.0;
  for (int k = 0; k < h->ncases; ++k) {
    const dsmc_config& c = h->cfgs[k];
    if (c.dim != 1) return set_err(h, DSMC_ERR_ARG, "synth_solve: only the 1D slab is implemented");
    if (c.nx < 3) return set_err(h, DSMC_ERR_ARG, "synth_solve needs at least 3 cells per slab");
    const int nm = c.n_m > 0 ? c.n_m : 2000;
    const double tl = c.synth_tol > 0 ? c.synth_tol : 1e-5;
    if (nm > n_m) n_m = nm;
    if (tl < tol) tol = tl;
  }
  const cudaError_t le = launch_synth1d(h->d_cp, h->d_cell_case, h->d_cell0, h->ncases, h->ncells, h->nx.data(),
                                        dev_fields, dev_hot, dev_out, h->synth_work, h->d_woff, n_m, tol,
                                        h->synth_info, h->stream);
  if (le != cudaSuccess) return set_err(h, DSMC_ERR_CUDA, "synth_solve: %s", cudaGetErrorString(le));
  std::vector<double> info(3 * (size_t)h->ncases);
  cudaMemcpyAsync(info.data(), h->synth_info, sizeof(double) * info.size(), cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "synth_solve");
  if (r) return r;
  int its = 0, worst = 0;
  double res = 0.0;
  for (int k = 0; k < h->ncases; ++k) {
    its = std::max(its, (int)info[3 * k]);
    res = std::max(res, info[3 * k + 1]);
    worst = std::max(worst, (int)info[3 * k + 2]);
  }
  if (host_iters) *host_iters = its;
  if (host_resid) *host_resid = res;
  if (worst == 2) return set_err(h, DSMC_ERR_NUMERIC, "synth_solve: no update keeps rho, T positive");
  if (worst == 1) return set_err(h, DSMC_ERR_NOT_CONVERGED, "synth_solve: %d iterations without convergence", n_m);
  return DSMC_OK;
}

int dig_correct(dsmc_handle* h, const double* dev_target) {
  if (!h || !dev_target) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  int32_t fl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (h->det) Ops<double>::dig_counts(h->sd, h->ncells, h->lay, dev_target, h->dig_iter, 1, h->stream);
  else Ops<float>::dig_counts(h->sf, h->ncells, h->lay, dev_target, h->dig_iter, 0, h->stream);
  int32_t* flags = h->det ? h->sd.flags : h->sf.flags;
  cudaMemcpyAsync(fl, flags, sizeof fl, cudaMemcpyDeviceToHost, h->stream);
  int r = sync_check(h, "dig_correct (counts)");
  if (r) return r;
  unsigned long long tot64 = 0, caps64 = 0;
  std::memcpy(&tot64, fl + 4, sizeof tot64);
  std::memcpy(&caps64, fl + 6, sizeof caps64);
  const unsigned long long cap = (unsigned long long)(h->det ? h->sd.capacity : h->sf.capacity);
  if (fl[0] & 1) return set_err(h, DSMC_ERR_NUMERIC, "dig_correct: non-finite or non-positive target");
  if ((fl[0] & 6) || tot64 > cap || caps64 > cap)
    return set_err(h, DSMC_ERR_CAPACITY, "dig_correct: new particle count does not fit");
  if (h->det) {
    Ops<double>::dig_apply(h->cp, h->sd, h->ncells, h->cur, h->lay, dev_target, h->dig_iter, 1, h->stream);
    h->sd.nparticles = fl[1];
  } else {
    Ops<float>::dig_apply(h->cp, h->sf, h->ncells, h->cur, h->lay, dev_target, h->dig_iter, 0, h->stream);
    h->sf.nparticles = fl[3];
  }
  h->dig_iter += 1;
  return check_cuda(h, "dig_correct");
}

int dsmc_num_particles(dsmc_handle* h, int64_t* host_n) {
  if (!h || !host_n) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  int32_t* cnt = h->det ? h->sd.count[h->lay] : h->sf.count[h->cur];
  int32_t* tmp = h->det ? h->sd.tmp_start : h->sf.tmp_start;
  if (h->det) Ops<double>::total_count(h->sd, cnt, h->ncells, h->stream);
  else Ops<float>::total_count(h->sf, cnt, h->ncells, h->stream);
  int32_t tot = 0, ov = 0;
  cudaMemcpyAsync(&tot, tmp + h->ncells, sizeof tot, cudaMemcpyDeviceToHost, h->stream);
  if (!h->det) cudaMemcpyAsync(&ov, h->sf.ovf[h->cur].count, sizeof ov, cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "dsmc_num_particles");
  if (r) return r;
  *host_n = (int64_t)tot + (ov < h->sf.ovf_cap || h->det ? ov : h->sf.ovf_cap);
  return DSMC_OK;
}

int dsmc_get_particles(dsmc_handle* h, double* x, double* y, double* vx, double* vy, double* vz, double* ir,
                       int32_t* cell, int64_t capacity_out, int64_t* host_n) {
  if (!h || !x || !y || !vx || !vy || !vz || !ir || !cell) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  int64_t n = 0;
  int r = dsmc_num_particles(h, &n);
  if (r) return r;
  if (host_n) *host_n = n;
  if (n > capacity_out) return set_err(h, DSMC_ERR_CAPACITY, "output holds %lld, need %lld", (long long)capacity_out, (long long)n);
  if (h->det) Ops<double>::export_particles(h->pd, h->sd, h->cur, h->lay, x, y, vx, vy, vz, ir, cell, h->stream);
  else Ops<float>::export_particles(h->pf, h->sf, h->cur, h->lay, x, y, vx, vy, vz, ir, cell, h->stream);
  return check_cuda(h, "dsmc_get_particles");
}

int dsmc_set_particles(dsmc_handle* h, int64_t n, const double* x, const double* y, const double* vx,
                       const double* vy, const double* vz, const double* ir) {
  if (!h || n < 0 || (n > 0 && (!x || !vx || !vy || !vz || !ir || (h->cfg.dim == 2 && !y))))
    return set_err(h, DSMC_ERR_ARG, "bad arguments");
  if (h->ncases > 1) return set_err(h, DSMC_ERR_ARG, "dsmc_set_particles: not available for a batch of cases");
  const int64_t cap = h->det ? h->sd.capacity : h->sf.capacity;
  if (n > cap) return set_err(h, DSMC_ERR_CAPACITY, "%lld particles exceed capacity %lld", (long long)n, (long long)cap);
  int32_t* flags = h->det ? h->sd.flags : h->sf.flags;
  cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, h->stream);
  if (h->det) Ops<double>::import_particles(h->pd, h->sd, h->cur, h->lay, n, x, y, vx, vy, vz, ir, 1, h->stream);
  else Ops<float>::import_particles(h->pf, h->sf, h->cur, h->lay, n, x, y, vx, vy, vz, ir, 0, h->stream);
  int32_t fl[4] = {0, 0, 0, 0};
  cudaMemcpyAsync(fl, flags, sizeof fl, cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "dsmc_set_particles");
  if (r) return r;
  if (fl[2]) return set_err(h, DSMC_ERR_CAPACITY, "cell bins do not fit the capacity");
  return DSMC_OK;
}

int dsmc_get_accumulators(dsmc_handle* h, double* dev_out, int64_t* host_nsamples) {
  if (!h || !dev_out) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  if (h->det) launch_acc_sum(h->ncells, h->sd.acc, h->sd.comp, dev_out, h->stream);
  else launch_acc_sum(h->ncells, h->sf.acc, h->sf.comp, dev_out, h->stream);
  if (host_nsamples) *host_nsamples = h->nsamples;
  return check_cuda(h, "dsmc_get_accumulators");
}

int dsmc_get_sgmax(dsmc_handle* h, double* dev_out) {
  if (!h || !dev_out) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  if (h->det) Ops<double>::sgmax_io(h->sd, h->ncells, dev_out, nullptr, h->stream);
  else Ops<float>::sgmax_io(h->sf, h->ncells, dev_out, nullptr, h->stream);
  return check_cuda(h, "dsmc_get_sgmax");
}

int dsmc_set_sgmax(dsmc_handle* h, const double* dev_in) {
  if (!h || !dev_in) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  if (h->det) Ops<double>::sgmax_io(h->sd, h->ncells, nullptr, dev_in, h->stream);
  else Ops<float>::sgmax_io(h->sf, h->ncells, nullptr, dev_in, h->stream);
  return check_cuda(h, "dsmc_set_sgmax");
}

int dsmc_get_counters(dsmc_handle* h, uint32_t* host_step, uint32_t* host_dig_iter) {
  if (!h) return DSMC_ERR_ARG;
  if (host_step) *host_step = h->step;
  if (host_dig_iter) *host_dig_iter = h->dig_iter;
  return DSMC_OK;
}

int dsmc_set_counters(dsmc_handle* h, uint32_t step, uint32_t dig_iter) {
  if (!h) return DSMC_ERR_ARG;
  h->step = step;
  h->dig_iter = dig_iter;
  return DSMC_OK;
}

int dsmc_get_stats(dsmc_handle* h, int64_t* out8) {
  if (!h || !out8) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  unsigned long long s[ST_NSLOTS];
  cudaMemcpyAsync(s, h->det ? h->sd.stats : h->sf.stats, sizeof s, cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "dsmc_get_stats");
  if (r) return r;
  out8[0] = (int64_t)s[ST_CAND];
  out8[1] = (int64_t)s[ST_COLL];
  out8[2] = (int64_t)s[ST_CLIP];
  out8[3] = (int64_t)s[ST_INEL];
  out8[4] = (int64_t)s[ST_HITS];
  out8[5] = (int64_t)s[ST_MAXHIT];
  out8[6] = (int64_t)s[ST_OVF];
  out8[7] = h->rebuilds;
  return DSMC_OK;
}

int dsmc_get_flow(dsmc_handle* h, int64_t* out2) {
  if (!h || !out2) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  unsigned long long s[ST_NSLOTS];
  cudaMemcpyAsync(s, h->det ? h->sd.stats : h->sf.stats, sizeof s, cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "dsmc_get_flow");
  if (r) return r;
  out2[0] = (int64_t)s[ST_INJ];
  out2[1] = (int64_t)s[ST_OUT];
  return DSMC_OK;
}

int dsmc_get_volumes(dsmc_handle* h, double* host_out) {
  if (!h || !host_out) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  if (h->cfg.mesh != DSMC_MESH_BOX) {
    cudaMemcpyAsync(host_out, h->ann_vol_d, sizeof(double) * h->ncells, cudaMemcpyDeviceToHost, h->stream);
    return sync_check(h, "dsmc_get_volumes");
  }
  for (int k = 0; k < h->ncases; ++k) {
    Params<double> p;
    CellParams cp;
    fill_params<double>(&h->cfgs[k], p, cp);
    for (int i = h->cell0[k]; i < h->cell0[k + 1]; ++i) host_out[i] = cp.vcell;
  }
  return DSMC_OK;
}

int dsmc_get_wall_tally(dsmc_handle* h, double* out20) {
  if (!h || !out20) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  cudaMemcpyAsync(out20, h->det ? h->sd.tally : h->sf.tally, sizeof(double) * 20, cudaMemcpyDeviceToHost, h->stream);
  return sync_check(h, "dsmc_get_wall_tally");
}

int dsmc_get_constants(dsmc_handle* h, double* out8) {
  if (!h || !out8) return DSMC_ERR_ARG;
  Params<double> p;
  CellParams cp;
  fill_params<double>(&h->cfg, p, cp);
  const double w = h->cfg.omega, a = h->cfg.alpha;
  out8[0] = cp.dx;
  out8[1] = cp.dy;
  out8[2] = cp.vcell;
  out8[3] = cp.fnum;
  out8[4] = cp.mu_ref;
  out8[5] = 5.0 * (a + 1.0) * (a + 2.0) / (a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w));
  out8[6] = p.c_sigma;
  out8[7] = p.p_inel;
  return DSMC_OK;
}

int dsmc_get_launch_shape(dsmc_handle* h, int* host_warps_per_cta, int* host_tile) {
  if (!h || !host_warps_per_cta || !host_tile) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  *host_warps_per_cta = h->det ? 0 : h->sf.fwpb;
  *host_tile = (h->det || h->sf.fwpb == 0) ? 0 : (h->sf.ftile > 0 ? h->sf.ftile : h->sf.tile);
  return DSMC_OK;
}

int dsmc_get_launch_config(dsmc_handle* h, int* host_warps_per_cta) {
  if (!h || !host_warps_per_cta) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  *host_warps_per_cta = h->det ? 0 : h->sf.fwpb;
  return DSMC_OK;
}

int hot_mlp_init(dsmc_handle* h, uint64_t seed) {
  if (!h) return DSMC_ERR_ARG;
  return mlp_init_params(h, seed);
}

int hot_mlp_set_params(dsmc_handle* h, const float* host_params) {
  if (!h || !host_params) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  for (int q = 0; q < MLP_NPARAM; ++q)
    if (!std::isfinite(host_params[q])) return set_err(h, DSMC_ERR_NUMERIC, "hot_mlp_set_params: parameter %d", q);
  return mlp_upload(h, host_params);
}

int hot_mlp_get_params(dsmc_handle* h, float* host_params) {
  if (!h || !host_params) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  cudaMemcpyAsync(host_params, h->mlp.theta, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, h->stream);
  return sync_check(h, "hot_mlp_get_params");
}

int hot_mlp_grad(dsmc_handle* h, const double* dev_fields, const double* dev_hot, const double* dev_kngll,
                 const uint8_t* dev_mask, float* host_grad, double* host_loss) {
  if (!h || !dev_fields || !dev_hot || !dev_kngll || !dev_mask) return set_err(h, DSMC_ERR_ARG, "bad arguments");
  mlp_data(h, dev_fields, dev_hot, dev_kngll, dev_mask);
  int n = 0;
  int r = mlp_count(h, &n);
  if (r) return r;
  if (n == 0) return set_err(h, DSMC_ERR_ARG, "hot_mlp_grad: no cell with mask = 1");
  mlp_grad(h->mlp, h->ncells, h->stream);
  double loss = 0.0;
  cudaMemcpyAsync(&loss, h->mlp.scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (host_grad)
    cudaMemcpyAsync(host_grad, h->mlp.grad, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, h->stream);
  r = sync_check(h, "hot_mlp_grad");
  if (r) return r;
  if (host_loss) *host_loss = loss;
  return DSMC_OK;
}

int hot_mlp_train(dsmc_handle* h, const double* dev_fields, const double* dev_hot, const double* dev_kngll,
                  const uint8_t* dev_mask, int nsteps, double lr, double* host_loss) {
  if (!h || !dev_fields || !dev_hot || !dev_kngll || !dev_mask || nsteps < 0 || !(lr > 0.0))
    return set_err(h, DSMC_ERR_ARG, "bad arguments");
  mlp_data(h, dev_fields, dev_hot, dev_kngll, dev_mask);
  int n = 0;
  int r = mlp_count(h, &n);
  if (r) return r;
  if (n == 0) return set_err(h, DSMC_ERR_ARG, "hot_mlp_train: no cell with mask = 1");
  for (int k = 0; k < nsteps; ++k) {
    mlp_grad(h->mlp, h->ncells, h->stream);
    h->mlp_t += 1;
    mlp_adam(h->mlp, h->mlp_t, lr, h->stream);
  }
  double loss = 0.0;
  cudaMemcpyAsync(&loss, h->mlp.scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  r = sync_check(h, "hot_mlp_train");
  if (r) return r;
  if (host_loss) *host_loss = loss;
  return DSMC_OK;
}

int hot_mlp_apply(dsmc_handle* h, const double* dev_fields, const double* dev_hot, const double* dev_kngll,
                  const uint8_t* dev_mask, double* dev_hot_out, double* host_judge) {
  if (!h || !dev_fields || !dev_hot || !dev_kngll || !dev_mask || !dev_hot_out)
    return set_err(h, DSMC_ERR_ARG, "bad arguments");
  mlp_data(h, dev_fields, dev_hot, dev_kngll, dev_mask);
  mlp_apply(h->mlp, h->ncells, dev_hot, dev_hot_out, h->stream);
  double j[2] = {0.0, 0.0};
  cudaMemcpyAsync(j, h->mlp.scal + 2, sizeof j, cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "hot_mlp_apply");
  if (r) return r;
  if (host_judge) *host_judge = j[1] > 0.0 ? j[0] / j[1] : 0.0;
  return DSMC_OK;
}

int hot_mlp_judge_reset(dsmc_handle* h) {
  if (!h) return DSMC_ERR_ARG;
  cudaMemsetAsync(h->mlp.jacc, 0, sizeof(double) * 16 * (size_t)h->ncells, h->stream);
  return check_cuda(h, "hot_mlp_judge_reset");
}

int hot_mlp_apply_judged(dsmc_handle* h, const double* dev_fields, const double* dev_hot, const double* dev_kngll,
                         const uint8_t* dev_mask, const int32_t* dev_group, double z, int min_samples, double rel,
                         double* dev_hot_out, double* host_judge, int64_t* host_nnet) {
  if (!h || !dev_fields || !dev_hot || !dev_kngll || !dev_mask || !dev_hot_out || !(z > 0.0) || min_samples < 2 ||
      !(rel > 0.0))
    return set_err(h, DSMC_ERR_ARG, "bad arguments");
  mlp_data(h, dev_fields, dev_hot, dev_kngll, dev_mask);
  mlp_apply(h->mlp, h->ncells, dev_hot, dev_hot_out, h->stream, dev_group, z, min_samples, rel);
  double j[3] = {0.0, 0.0, 0.0};
  cudaMemcpyAsync(j, h->mlp.scal + 2, sizeof j, cudaMemcpyDeviceToHost, h->stream);
  const int r = sync_check(h, "hot_mlp_apply_judged");
  if (r) return r;
  if (host_judge) *host_judge = j[1] > 0.0 ? j[0] / j[1] : 0.0;
  if (host_nnet) *host_nnet = (int64_t)j[2];
  return DSMC_OK;
}

}  // extern "C"
