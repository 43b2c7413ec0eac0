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
};

// Everything a launch needs, carved out of the caller's workspace.
template <typename T>
struct State {
  int64_t capacity;
  int nparticles;  // host copy of the particle count (compact layout)
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
};

template <typename T>
struct Ops {
  static void configure(int tile);
  static void init(const Params<T>& p, State<T>& s, int cur, int lay, int ppc, int cap0, double tt,
                   double tr, const double* u3, cudaStream_t st);
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
  static void dig_counts(const CellParams& cp, State<T>& s, int lay, const double* target,
                         uint32_t iter, int det, cudaStream_t st);
  static void dig_apply(const CellParams& cp, State<T>& s, int& cur, int& lay, const double* target,
                        uint32_t iter, int det, cudaStream_t st);
  // writes the total of cnt[0..ncells) to s.tmp_start[ncells]
  static void total_count(State<T>& s, const int32_t* cnt, int ncells, cudaStream_t st);
  static void sgmax_io(State<T>& s, int ncells, double* out, const double* in, cudaStream_t st);
};

// FP64 cell-field kernels (dsmc_fields.cu)
void launch_fields(const CellParams& cp, const double* acc, const double* comp, int64_t nsamples,
                   double* out, cudaStream_t st);
void launch_hot(const CellParams& cp, const double* fields, double* hot, double* kngll,
                uint8_t* mask, cudaStream_t st);
void launch_acc_sum(int ncells, const double* acc, const double* comp, double* out,
                    cudaStream_t st);
// 1D synthetic equations; writes iterations / residual / status to dev_info (3 doubles)
void launch_synth1d(const CellParams& cp, const double* fields, const double* hot, double* out,
                    double* work, int n_m, double tol, double* dev_info, cudaStream_t st);
size_t synth1d_work_doubles(int ncells);

}  // namespace dsmc
