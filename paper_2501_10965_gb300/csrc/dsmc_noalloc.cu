// dsmc_noalloc.cu -- synth_solve_noalloc: the 1D synthetic-equation solve for
// callers that cannot allocate device memory.
//
// The ordinary entry point (synth_solve) needs a handle, and a handle needs a
// workspace that the caller allocates.  Some callers cannot do that: a host
// code whose device memory belongs to another allocator (a pool it may not
// grow or bypass), or one that runs under a device-memory budget fixed at
// start-up, where a new allocation is not permitted.  This variant takes the
// configuration and the field arrays directly and keeps the solver's scratch
// (the Newton iterate, residuals, Jacobian blocks and the cyclic-reduction
// factors) in a fixed, file-scope device array instead.  That array belongs to the library: every
// GPU that loads the library holds it until the process exits.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/dig_dsmc.h"
#include "dsmc_internal.h"

namespace {

// scratch doubles for DSMC_SYNTH_NOALLOC_MAX_CELLS cells (the solver needs
// 104 per cell + 96) plus 8 for the iteration count / residual / status
constexpr size_t kScratchDoubles = (size_t)DSMC_SYNTH_NOALLOC_MAX_CELLS * 112 + 256;
constexpr size_t kInfoOffset = kScratchDoubles - 8;

static __device__ __align__(256) double g_synth_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_synth_scratch on the current device, looked up once per
// device (the host-side name is only a stand-in, not a device address).
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DSMC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_synth_scratch);
    if (e != cudaSuccess || !p) return DSMC_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DSMC_OK;
}

}  // namespace

extern "C" int synth_solve_noalloc(const dsmc_config* cfg, const double* dev_fields, const double* dev_hot,
                                   double* dev_out, void* stream, int* host_iters, double* host_resid) {
  if (!cfg || !dev_fields || !dev_hot || !dev_out) return DSMC_ERR_ARG;
  if (cfg->version != DSMC_ABI_VERSION || cfg->dim != 1 || cfg->nx < 3) return DSMC_ERR_ARG;
  if (!(cfg->lx > 0) || !(cfg->kn > 0) || !(cfg->z_rot > 0) || cfg->d_r != 2.0) return DSMC_ERR_ARG;
  if (cfg->nx > DSMC_SYNTH_NOALLOC_MAX_CELLS) return DSMC_ERR_CAPACITY;
  if (dsmc::synth1d_work_doubles(cfg->nx) + 8 > kScratchDoubles) return DSMC_ERR_CAPACITY;
  const double* A = cfg->a_matrix;
  const double det = A[0] * A[3] - A[1] * A[2];
  if (!(det != 0.0) || !std::isfinite(det)) return DSMC_ERR_ARG;
  // the call waits on the stream, which a capturing stream cannot do:
  // refuse before launching anything (an implicit capture of the legacy
  // stream reports itself as an error of the query)
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t qe = cudaStreamIsCapturing(st, &cap);
  if (qe == cudaErrorStreamCaptureImplicit) return DSMC_ERR_ARG;
  if (qe != cudaSuccess) return DSMC_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return DSMC_ERR_ARG;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  // the parameters the 1D solver reads (same definitions as the handle's)
  dsmc::CellParams cp{};
  cp.dim = 1;
  cp.nx = cfg->nx;
  cp.ny = 1;
  cp.ncells = cfg->nx;
  cp.lx = cfg->lx;
  cp.ly = 1.0;
  cp.dx = cfg->lx / (double)cfg->nx;
  cp.dy = 1.0;
  cp.vcell = cp.dx;
  cp.d_r = cfg->d_r;
  cp.omega = cfg->omega;
  cp.mu_ref = cfg->kn * std::sqrt(2.0 / M_PI);
  cp.z_rot = cfg->z_rot;
  cp.kappa_t = 0.5 * (A[3] * 5.0 - A[1] * cfg->d_r) / det;
  cp.kappa_r = 0.5 * (-A[2] * 5.0 + A[0] * cfg->d_r) / det;
  cp.kn_ref = cfg->kn_ref;
  const int n_m = cfg->n_m > 0 ? cfg->n_m : 2000;
  const double tol = cfg->synth_tol > 0 ? cfg->synth_tol : 1e-5;
  double* info_dev = scratch + kInfoOffset;
  // every scratch word the kernel reads it has written first in the same
  // call, so nothing needs clearing between calls
  if (dsmc::launch_synth1d_single(cp, dev_fields, dev_hot, dev_out, scratch, n_m, tol, info_dev, st) != cudaSuccess)
    return DSMC_ERR_CUDA;
  double info[3] = {0, 0, 0};
  if (cudaMemcpyAsync(info, info_dev, sizeof info, cudaMemcpyDeviceToHost, st) != cudaSuccess) return DSMC_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DSMC_ERR_CUDA;
  if (host_iters) *host_iters = (int)info[0];
  if (host_resid) *host_resid = info[1];
  if (info[2] == 2.0) return DSMC_ERR_NUMERIC;
  if (info[2] == 1.0) return DSMC_ERR_NOT_CONVERGED;
  return DSMC_OK;
}
