// dsmc_internal.h -- host-side views shared by the C ABI and the kernel
// launch wrappers.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dsmc_device.cuh"

namespace dsmc {

template <typename T>
struct PBuf {
  T *x, *y, *vx, *vy, *vz, *ir;
};

// largest particles-per-warp tile of a layout (a handle caps its tile here)
template <typename T>
constexpr int TILE_MAX_OF = sizeof(T) == 8 ? 256 : 512;

// Particles that did not fit their destination bin (FP32 layout only).
struct Ovf {
  float *x, *y, *vx, *vy, *vz, *ir;
  int32_t* dest;
  int32_t* count;  // one word
};

// Parameters of the per-cell DIG and field kernels (always FP64).
struct CellParams {
  int dim, nx, ny, ncells;
  double lx, ly, dx, dy, vcell, fnum, d_r, omega, mu_ref, z_rot;
  double kappa_t, kappa_r;  // kappa / mu from Eq. (kappa_A)
  double kn_ref;
  uint32_t k0, k1;
  int mesh;            // 0 Cartesian box, 1 annulus, 2 wall-refined box (1, 2: single case)
  const double* vol;   // annulus: cell volumes (null on the box: vcell)
  const double* r2t;   // annulus: ny + 1 squared ring radii (nx sectors x ny rings)
  const double* rt;    // annulus: the ny + 1 ring radii themselves
  const double* xe;    // wall-refined box: nx + 1 and ny + 1 cell edges
  const double* ye;
};

// Per-case tables of a handle (device memory).  A single simulation is one
// case; a batch holds several independent cases whose cells are numbered
// consecutively: case c owns global cells [cell0[c], cell0[c+1]).
template <typename T>
struct Cases {
  const Params<T>* p;        // per case
  const CellParams* cp;      // per case
  const int32_t* cell0;      // ncases + 1
  const int32_t* cell_case;  // per global cell
  int n;
};

// Everything a launch needs, carved out of the caller's workspace.
template <typename T>
struct State {
  int64_t capacity;
  int nparticles;  // host copy of the particle count (compact layout)
  int ncells;      // total cells (all cases)
  int ovf_cap;
  int tile;        // particles staged per warp in shared memory
  double slack;    // FP32 bin capacity = slack * count + 32
  PBuf<T> buf[2];  // particle buffers; buf[cur] holds the state
  int32_t* start[2];  // layout: bin starts (ncells + 1) ...
  int32_t* count[2];  // ... and occupancies (ncells)
  int32_t* cellof;    // FP64 compact layout: cell of each slot
  int32_t* key;       // scratch: new cell per slot
  int32_t* dest;      // scratch: destination slot
  int32_t* scratch_i; // scratch (capacity) for DIG index lists / export offsets
  uint32_t* owner;    // scratch (capacity) for the collision scheduler of big cells
  int32_t* nt;        // scratch (ncells): DIG target counts
  int32_t* tmp_start; // scratch (ncells + 1)
  int32_t* tmp2;      // scratch (ncells + 1)
  T* sgmax;           // ncells
  double* acc;        // ncells x 17
  double* comp;       // ncells x 17
  float* stg;         // FP32 layout: staged per-step sums (ncells x 17) ...
  float* stc;         // ... and their Kahan compensations
  double* tally;      // 20
  unsigned long long* stats;  // ST_NSLOTS
  int32_t* flags;     // 16 device words: [0] error bits, [1] total, [2] over-capacity
  Ovf ovf[2];
  Cases<T> cases;
  bool batch;  // several cases: kernels read their parameters per cell
  bool gen;    // a gas with d_r = 3 or VSS scattering: the fused step's general instantiation
  int fwpb;    // FP32 fused step: warps per CTA (0: not tuned yet)
  int ftile;   // FP32 fused step: particles staged per warp (0: tile)
  Params<double> pinj;  // annulus: FP64 parameters of the freestream entry
  double* inj_mu;       // annulus: expected entries of every outer face per step
  int inj_max;          // annulus: bound on the entries of one step (sum of floor(mu) + 1)
  // annulus, FP32 layout: the freestream entry of a step runs on a side
  // stream beside the fused step (both append to the next step's bins with
  // atomics); fork after the previous launch, join before the next
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  bool lost;  // FP64 annulus: freestream entries did not fit the workspace
};

template <typename T>
struct Ops {
  static void configure(int tile);
  static void init(const Params<T>& p, State<T>& s, int cur, int lay, int ppc, int cap0, double tt,
                   double tr, const double* u3, cudaStream_t st);
  // batch: the layout s.start[lay] is set; every case fills its cells
  // (counts[c] particles in cell c when counts is given, else ppc)
  static void init_batch(const Params<T>& p0, State<T>& s, int ncells, int cur, int lay, cudaStream_t st,
                         const int32_t* counts = nullptr);
  // annulus: initial particles per cell (FP64 draws, both layouts)
  static void ann_counts(const Params<double>& pd, int ncells, int32_t* counts, cudaStream_t st);
  // annulus: expected entries of every outer face per step
  static void inflow_means(const Params<double>& pd, double* mu, cudaStream_t st);
  static void step_det(const Params<T>& p, State<T>& s, int& cur, int& lay, uint32_t step,
                       int do_sample, cudaStream_t st);
  static void step_bins(const Params<T>& p, State<T>& s, int& cur, int lay, uint32_t step0,
                        int nsteps, int do_sample, cudaStream_t st);
  static void rebin(const Params<T>& p, State<T>& s, int& cur, int& lay, int with_ovf, double slack,
                    cudaStream_t st);
  static void export_particles(const Params<T>& p, State<T>& s, int cur, int lay, double* x,
                               double* y, double* vx, double* vy, double* vz, double* ir,
                               int32_t* cell, cudaStream_t st);
  static void import_particles(const Params<T>& p, State<T>& s, int& cur, int& lay, int64_t n,
                               const double* x, const double* y, const double* vx,
                               const double* vy, const double* vz, const double* ir, int det,
                               cudaStream_t st);
  static void dig_counts(State<T>& s, int ncells, int lay, const double* target, uint32_t iter, int det,
                         cudaStream_t st);
  static void dig_apply(const CellParams& cp0, State<T>& s, int ncells, int& cur, int& lay,
                        const double* target, uint32_t iter, int det, cudaStream_t st);
  // writes the total of cnt[0..ncells) to s.tmp_start[ncells]
  static void total_count(State<T>& s, const int32_t* cnt, int ncells, cudaStream_t st);
  static void sgmax_io(State<T>& s, int ncells, double* out, const double* in, cudaStream_t st);
};

// FP64 cell-field kernels (dsmc_fields.cu); cp / cell_case / cell0 are
// device tables (see Cases), ncells the total number of cells
void launch_fields(const CellParams* cp, const int32_t* cell_case, int ncells, const double* acc,
                   const double* comp, int64_t nsamples, double* out, cudaStream_t st);
void launch_hot(const CellParams* cp, const int32_t* cell_case, const int32_t* cell0, int ncells,
                const double* fields, double* hot, double* kngll, uint8_t* mask, cudaStream_t st);
void launch_acc_sum(int ncells, const double* acc, const double* comp, double* out,
                    cudaStream_t st);
// 1D synthetic equations of ncases slabs; case c uses work + woff[c] (device
// table of offsets in doubles) and writes (iterations, max residual, status)
// to info[3c .. 3c+2]; host_nx[c] are the slab sizes (host memory)
cudaError_t launch_synth1d(const CellParams* cp, const int32_t* cell_case, const int32_t* cell0, int ncases,
                           int ncells, const int32_t* host_nx, const double* fields, const double* hot,
                           double* out, double* work, const int64_t* woff, int n_m, double tol, double* info,
                           cudaStream_t st);
// one slab given by value, no device tables (info: 4 doubles)
cudaError_t launch_synth1d_single(const CellParams& cp, const double* fields, const double* hot, double* out,
                                  double* work, int n_m, double tol, double* info, cudaStream_t st);
size_t synth1d_work_doubles(int ncells);
// 2D synthetic equations of one box case (dsmc_synth2d.cu): doubles of work,
// and the solve (info = iterations, max residual, status; *singular set when
// a zero pivot was met); returns a cudaError_t value, or S2_TIMEOUT_RC when a
// bounded wait of the substitution gave up
constexpr int S2_TIMEOUT_RC = -2;
size_t synth2d_work_doubles(int nx, int ny, int annulus);
int launch_synth2d(const CellParams& cp, const double* fields, const double* hot, double* out, double* work,
                   int n_m, double tol, double* info, int* singular, int reuse, int warm, cudaStream_t st);

// HoT surrogate network (dsmc_mlp.cu): 12 -> 64 -> 64 -> 64 -> 5, tanh
// hidden layers; parameters per layer: W (n_out x n_in, row major), then b.
constexpr int MLP_NPARAM = 9477;
constexpr int MLP_GRID = 304;  // largest grid of the forward/backward kernel
struct Mlp {
  float* theta;      // MLP_NPARAM FP32 master parameters
  uint16_t* wbf;     // MLP_NPARAM bfloat16 copies used by the kernels
  float* m;          // Adam first moments
  float* v;          // Adam second moments
  float* grad;       // MLP_NPARAM
  float* partial;    // MLP_GRID x MLP_NPARAM per-CTA gradient sums
  double* part_loss; // MLP_GRID per-CTA loss sums
  float* X;          // ncells x 12 inputs
  float* Y;          // ncells x 5 normalised DSMC HoT
  float* S;          // ncells x 4: p, p sqrt(T), e_x, e_y
  float* w;          // ncells: 1 for a training / replaced cell, else 0
  float* out;        // ncells x 5 network outputs
  double* scal;      // [0] loss, [2] judge sum, [3] judge count, [4] cells given the network's HoT
  int32_t* count;    // [0] number of cells with w = 1
  double* jacc;      // ncells x 16 judge statistics per group: sum r (5), sum r^2 (5), count, sum Y (5)
};
// inputs, scales, targets (hot may be null) and weights of every cell
void mlp_prepare(const Mlp& m, const CellParams* cp, const int32_t* cell_case, const int32_t* cell0, int ncells,
                 const double* fields, const double* hot, const double* kngll, const uint8_t* mask,
                 cudaStream_t st);
// loss (scal[0]) and gradient (grad) of the weighted cells
void mlp_grad(const Mlp& m, int ncells, cudaStream_t st);
// one Adam step (step number t >= 1) and the bfloat16 copies
void mlp_adam(const Mlp& m, int t, double lr, cudaStream_t st);
// bfloat16 copies of the master parameters
void mlp_to_bf16(const Mlp& m, cudaStream_t st);
// network outputs, the HoT for the synthetic equations and the judge sums;
// with z > 0 a cell takes the network's HoT only where its group's running
// residual statistics pass the judge (see hot_mlp_apply_judged)
void mlp_apply(const Mlp& m, int ncells, const double* hot, double* hot_out, cudaStream_t st,
               const int32_t* group = nullptr, double z = 0.0, int min_samples = 0, double rel = 0.0);

}  // namespace dsmc
