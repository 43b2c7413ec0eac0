// dsmc_ops.cuh -- kernels of the DSMC step and of the particle modification,
// templated on the particle precision T and the dimension DIM, and their
// launch wrappers.  Included by one translation unit per precision.
//
// Two particle layouts:
//  * FP64-deterministic: compact, cell-sorted arrays; each step runs
//    move (one thread per particle) -> stable counting sort (one CTA) ->
//    collide + sample (one warp per cell).  The event order equals the
//    sequential definition, so results match a sequential implementation.
//  * FP32: each cell owns a padded bin; one fused kernel per step runs, per
//    cell (one warp): stage the cell in shared memory, collide, sample, move,
//    and append each particle to its new cell's bin in the other buffer
//    (warp-aggregated atomics).  Particles read once and written once per step.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "dsmc_device.cuh"
#include "dsmc_internal.h"

namespace dsmc {

constexpr int WPB = 8;  // warps per CTA for the per-cell kernels
constexpr int CTA_SCAN = 1024;

// ---------------------------------------------------------------------------
// single-CTA exclusive scan: out[i] = sum_{k<i} value(k), out[n] = total
// ---------------------------------------------------------------------------
template <typename F>
__device__ void cta_exclusive_scan(int n, F value, int32_t* out) {
  // each thread takes SCAN_ITEMS consecutive entries per pass, so that a pass
  // covers SCAN_ITEMS x blockDim.x entries and its loads are issued together
  constexpr int SCAN_ITEMS = 8;
  __shared__ int32_t wsum[32];
  __shared__ int32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x * SCAN_ITEMS) {
    const int i0 = base + threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t tsum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
      v[j] = (i0 + j < n) ? value(i0 + j) : 0;
      tsum += v[j];
    }
    int32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t w = (lane < nw) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int32_t run = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - tsum;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
      if (i0 + j < n) out[i0 + j] = run;
      run += v[j];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = run;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
  __syncthreads();
}

__device__ __forceinline__ int32_t bin_cap_of(int32_t count, double slack) {
  const int32_t c = (int32_t)ceil(slack * (double)count) + 32;
  return (c + 7) & ~7;
}

// ---------------------------------------------------------------------------
// initial equilibrium state (Sec. 3 step 1)
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void k_init(Params<T> p, PBuf<T> b, const int32_t* __restrict__ start,
                       int32_t* __restrict__ count, int32_t* __restrict__ cellof, int ppc, T tt,
                       T tr, T u0x, T u0y, T u0z) {
  const long long total = (long long)p.ncells * ppc;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < total;
       s += (long long)gridDim.x * blockDim.x) {
    const int cell = (int)(s / ppc), k = (int)(s % ppc);
    const int ix = cell % p.nx, iy = cell / p.nx;
    Stream<T> st(TAG_INIT, (uint32_t)k, (uint32_t)cell, 0u, p.k0, p.k1);
    const T a0 = st.u(0), a1 = st.u(1);
    T n1, n2, n3, n4;
    box_muller(st.u(2), st.u(3), &n1, &n2);
    box_muller(st.u(4), st.u(5), &n3, &n4);
    const T stt = m_sqrt(tt);
    const int slot = start[cell] + k;
    b.x[slot] = ((T)ix + a0) * p.dx;
    b.y[slot] = (DIM == 2) ? ((T)iy + a1) * p.dy : T(0);
    b.vx[slot] = u0x + stt * n1;
    b.vy[slot] = u0y + stt * n2;
    b.vz[slot] = u0z + stt * n3;
    b.ir[slot] = rot_energy(p.d_r3 != 0, tr, st.u(6), st, JX_OWN);
    if (cellof) cellof[slot] = cell;
    if (k == 0) count[cell] = ppc;
  }
}

// Batch initial state: one warp per cell, the cell's case supplies ppc, the
// initial state and the random key (same draws as k_init).
template <typename T, int DIM>
__global__ void k_init_cells(Cases<T> cases, int ncells, PBuf<T> b, const int32_t* __restrict__ start,
                             int32_t* __restrict__ count, int32_t* __restrict__ cellof,
                             const int32_t* __restrict__ counts) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int cell = warp;
  if (cell >= ncells) return;
  const int cs = cases.cell_case[cell];
  const Params<T>& p = cases.p[cs];
  const int lcell = cell - cases.cell0[cs];
  const int ix = lcell % p.nx, iy = lcell / p.nx;
  const int ppc = counts ? counts[cell] : p.ppc;
  const T stt = m_sqrt(p.init_tt);
  for (int k = lane; k < ppc; k += 32) {
    Stream<T> st(TAG_INIT, (uint32_t)k, (uint32_t)lcell, 0u, p.k0, p.k1);
    const T a0 = st.u(0), a1 = st.u(1);
    T n1, n2, n3, n4;
    box_muller(st.u(2), st.u(3), &n1, &n2);
    box_muller(st.u(4), st.u(5), &n3, &n4);
    const int slot = start[cell] + k;
    if (p.mesh == 1) {
      // annulus: uniform in the sector (r^2 and the angle uniform)
      const T r = m_sqrt(p.r2t[iy] + a0 * (p.r2t[iy + 1] - p.r2t[iy]));
      const T th = T(2.0 * PI_D) * ((T)ix + a1) / (T)p.nx;
      b.x[slot] = r * m_cos(th);
      b.y[slot] = r * m_sin(th);
    } else if (DIM == 2 && p.mesh == 2) {
      // wall-refined box: uniform between the cell's edges
      b.x[slot] = p.xe[ix] + a0 * (p.xe[ix + 1] - p.xe[ix]);
      b.y[slot] = p.ye[iy] + a1 * (p.ye[iy + 1] - p.ye[iy]);
    } else {
      b.x[slot] = ((T)ix + a0) * p.dx;
      b.y[slot] = (DIM == 2) ? ((T)iy + a1) * p.dy : T(0);
    }
    b.vx[slot] = p.init_u[0] + stt * n1;
    b.vy[slot] = p.init_u[1] + stt * n2;
    b.vz[slot] = p.init_u[2] + stt * n3;
    b.ir[slot] = rot_energy(p.d_r3 != 0, p.init_tr, st.u(6), st, JX_OWN);
    if (cellof) cellof[slot] = cell;
  }
  if (lane == 0) count[cell] = ppc;
}

// Annulus: initial particles of every cell, Iround(rho V_cell / F) with the
// draw (~0, cell, 0) of the initial stream (FP64 in both layouts)
static __global__ void k_ann_counts(const __grid_constant__ Params<double> pd, int ncells, int32_t* __restrict__ counts) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    Stream<double> st(TAG_INIT, 0xFFFFFFFFu, (uint32_t)c, 0u, pd.k0, pd.k1);
    counts[c] = (int32_t)iround(pd.init_rho * pd.vol[c] / pd.fnum, st.u(0));
  }
}

static __global__ void k_layout_uniform(int ncells, int32_t cap, int32_t* start) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncells; c += gridDim.x * blockDim.x)
    start[c] = c * cap;
}

// ---------------------------------------------------------------------------
// FP64-deterministic layout: move, stable sort, collide + sample
// ---------------------------------------------------------------------------
template <typename T, int DIM, bool BATCH, bool ANN>
__global__ void __launch_bounds__(256) k_move_det(const __grid_constant__ Params<T> pk, Cases<T> cases, PBuf<T> b,
                                                  const int32_t* __restrict__ cellof,
                                                  const int32_t* __restrict__ start, int n,
                                                  uint32_t step, int32_t* __restrict__ key,
                                                  double* __restrict__ tally_g,
                                                  unsigned long long* __restrict__ stats) {
  __shared__ T s_tally[20];
  if (threadIdx.x < 20) s_tally[threadIdx.x] = T(0);
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int c = cellof[s];
    const int cs = BATCH ? cases.cell_case[c] : 0;
    const Params<T>& p = BATCH ? cases.p[cs] : pk;
    const int c0 = BATCH ? cases.cell0[cs] : 0;
    T x = b.x[s], y = b.y[s], vx = b.vx[s], vy = b.vy[s], vz = b.vz[s], ir = b.ir[s];
    bool in = true;
    if constexpr (ANN)
      in = fly_ann<T, true>(p, x, y, vx, vy, vz, ir, TAG_WALL, (uint32_t)(s - start[c]), (uint32_t)c, step, 0u, p.dt,
                            s_tally, stats + ST_HITS, stats + ST_MAXHIT);
    else
      fly<T, DIM, true>(p, x, y, vx, vy, vz, ir, (uint32_t)(s - start[c]), (uint32_t)(c - c0), step, s_tally,
                        stats + ST_HITS, stats + ST_MAXHIT);
    b.x[s] = x;
    b.y[s] = y;
    b.vx[s] = vx;
    b.vy[s] = vy;
    b.vz[s] = vz;
    b.ir[s] = ir;
    if constexpr (ANN) {
      // a particle that left keeps key -1: the sort drops it
      key[s] = in ? cell_of_ann<T>(p, x, y) : -1;
      if (!in) atomicAdd(stats + ST_OUT, 1ull);
    } else {
      key[s] = c0 + cell_of<T, DIM>(p, x, y);
    }
  }
  __syncthreads();
  if (threadIdx.x < 20 && s_tally[threadIdx.x] != T(0))
    atomicAdd(tally_g + threadIdx.x, (double)s_tally[threadIdx.x]);
}

// Stable counting sort by key (one CTA of 1024 threads): histogram, scan,
// then one warp assigns destinations 32 slots at a time in slot order (ties
// keep their order), then every thread scatters.  Tin -> Tout conversion.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(1024) k_sort_stable(const Tin* __restrict__ ix, const Tin* __restrict__ iy,
                                                      const Tin* __restrict__ ivx, const Tin* __restrict__ ivy,
                                                      const Tin* __restrict__ ivz, const Tin* __restrict__ iir,
                                                      PBuf<Tout> o, const int32_t* __restrict__ key, int n,
                                                      int ncells, int32_t* __restrict__ start_out,
                                                      int32_t* __restrict__ count_out,
                                                      int32_t* __restrict__ fill,
                                                      int32_t* __restrict__ dest,
                                                      int32_t* __restrict__ cellof_out) {
  for (int c = threadIdx.x; c < ncells; c += blockDim.x) count_out[c] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x)
    if (key[s] >= 0) atomicAdd(&count_out[key[s]], 1);  // key -1: the particle left
  __syncthreads();
  cta_exclusive_scan(ncells, [&](int i) { return count_out[i]; }, start_out);
  for (int c = threadIdx.x; c < ncells; c += blockDim.x) fill[c] = start_out[c];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int base = 0; base < n; base += 32) {
      const int s = base + lane;
      const int k = (s < n) ? key[s] : -1;
      const unsigned peers = __match_any_sync(FULL, k);
      const int leader = __ffs(peers) - 1;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      int b = 0;
      if (s < n && k >= 0 && lane == leader) {
        b = fill[k];
        fill[k] = b + __popc(peers);
      }
      b = __shfl_sync(FULL, b, leader);
      if (s < n) dest[s] = (k >= 0) ? b + rank : -1;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const int d = dest[s];
    if (d < 0) continue;
    o.x[d] = (Tout)ix[s];
    o.y[d] = (Tout)iy[s];
    o.vx[d] = (Tout)ivx[s];
    o.vy[d] = (Tout)ivy[s];
    o.vz[d] = (Tout)ivz[s];
    o.ir[d] = (Tout)iir[s];
    if (cellof_out) cellof_out[d] = key[s];
  }
}

// ---------------------------------------------------------------------------
// Freestream entry through the outer circle of the annulus (FP64 arithmetic
// in both layouts).  Outer face k (between rays k and k+1 at r_out) admits
// Iround(flux L dt / F) particles, the flux that of the drifting freestream
// Maxwellian through the face with its centre normal, L = r_out 2 pi / nx.
// Particle q of face k (stream (q, k, step)): inward normal speed from the
// inflow distribution, tangential and z components Maxwellian about the
// freestream, I_r at its temperature, entry angle uniform on the face, then
// a flight over a uniform fraction of the step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long inflow_count(const Params<double>& p, int k, uint32_t step) {
  const double beta = 1.0 / sqrt(2.0 * p.fs_t);
  const double len = p.r_out * 2.0 * PI_D / (double)p.nx;
  const double nx = -p.fnrm[2 * k], ny = -p.fnrm[2 * k + 1];  // inward normal
  const double sn = (p.fs_u[0] * nx + p.fs_u[1] * ny) * beta;
  const double mu = p.fs_rho * inflow_ginf(sn) / (beta * sqrt(PI_D)) * len * p.dt / p.fnum;
  Stream<double> sc(TAG_INJ, 0xFFFFFFFFu, (uint32_t)k, step, p.k0, p.k1);
  return iround(mu, sc.u(0));
}

// false if the entering particle ends outside (it does not enter)
template <bool TALLY>
__device__ __forceinline__ bool inflow_particle(const Params<double>& p, int k, int q, uint32_t step, double* tally,
                                                unsigned long long* hits, unsigned long long* maxhit, double& x,
                                                double& y, double& vx, double& vy, double& vz, double& ir) {
  const double sT = sqrt(p.fs_t), beta = 1.0 / sqrt(2.0 * p.fs_t);
  const double nx = -p.fnrm[2 * k], ny = -p.fnrm[2 * k + 1];
  const double tx = -ny, ty = nx;
  const double un = p.fs_u[0] * nx + p.fs_u[1] * ny, ut = p.fs_u[0] * tx + p.fs_u[1] * ty;
  Stream<double> st(TAG_INJ, (uint32_t)q, (uint32_t)k, step, p.k0, p.k1);
  const double vn = inflow_speed(un * beta, st.u(0)) / beta;
  double n1, n2;
  box_muller(st.u(1), st.u(2), &n1, &n2);
  const double vt = ut + sT * n1;
  vx = vn * nx + vt * tx;
  vy = vn * ny + vt * ty;
  vz = p.fs_u[2] + sT * n2;
  const double th = 2.0 * PI_D * ((double)k + st.u(3)) / (double)p.nx;
  ir = rot_energy(p.d_r3 != 0, p.fs_t, st.u(4), st, JX_OWN);
  x = p.r_out * cos(th);
  y = p.r_out * sin(th);
  return fly_ann<double, TALLY>(p, x, y, vx, vy, vz, ir, TAG_INJ, (uint32_t)q, (uint32_t)k, step, 8u, st.u(5) * p.dt,
                                tally, hits, maxhit);
}

// FP64 layout, one CTA: a scan gives each face its run of slots after the n
// moved particles, so that new particles follow face by face and, within a
// face, in draw order (the sequential algorithm's order).  One that ends
// outside keeps key -1 (the sort drops it).  cnt, off: nx and nx + 1 ints;
// off[nx] is the number of slots used.
template <typename T>
__global__ void __launch_bounds__(1024) k_inject_det(const __grid_constant__ Params<double> p, PBuf<T> b,
                                                     int32_t* __restrict__ key, int n, long long capacity,
                                                     uint32_t step, int32_t* __restrict__ cnt,
                                                     int32_t* __restrict__ off, int32_t* __restrict__ flags,
                                                     double* __restrict__ tally_g,
                                                     unsigned long long* __restrict__ stats) {
  __shared__ double s_tally[5];
  if (threadIdx.x < 5) s_tally[threadIdx.x] = 0.0;
  const int nt = p.nx;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const long long m = inflow_count(p, k, step);
    cnt[k] = (int32_t)(m < 0 ? 0 : (m > (1 << 24) ? (1 << 24) : m));
  }
  __syncthreads();
  cta_exclusive_scan(nt, [&](int i) { return cnt[i]; }, off);
  if (threadIdx.x == 0 && (long long)n + off[nt] > capacity) atomicOr(flags, 4);
  unsigned long long nin = 0;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    for (int q = 0; q < cnt[k]; ++q) {
      const long long slot = (long long)n + off[k] + q;
      if (slot >= capacity) break;
      double x, y, vx, vy, vz, ir;
      const bool in = inflow_particle<true>(p, k, q, step, s_tally, stats + ST_HITS, stats + ST_MAXHIT, x, y, vx, vy,
                                            vz, ir);
      b.x[slot] = (T)x;
      b.y[slot] = (T)y;
      b.vx[slot] = (T)vx;
      b.vy[slot] = (T)vy;
      b.vz[slot] = (T)vz;
      b.ir[slot] = (T)ir;
      key[slot] = in ? cell_of_ann<double>(p, x, y) : -1;
      if (in) ++nin;  // one that ends outside never entered
    }
  }
  if (nin) atomicAdd(stats + ST_INJ, nin);
  __syncthreads();
  if (threadIdx.x < 5 && s_tally[threadIdx.x] != 0.0) atomicAdd(tally_g + threadIdx.x, s_tally[threadIdx.x]);
}

template <int DIM>
__device__ __forceinline__ void append_particle(const Params<float>& p, const PBuf<float>& o,
                                                const int32_t* __restrict__ start,
                                                int32_t* __restrict__ cnt_out, const Ovf& ovo,
                                                int ovf_cap, bool active, int d, float x, float y,
                                                float vx, float vy, float vz, float ir,
                                                unsigned* s_misc, int32_t* errflag);

// FP32 layout: the same inflow speed distribution, density z exp(-(z -
// s)^2) on z > 0, sampled exactly by acceptance-rejection in FP32 from
// uniforms 64 + 4t .. 67 + 4t of the particle's stream (try t):
//   s >= 0: with w = z - s the density is (s + w) exp(-w^2) <= (s + |w|)
//     exp(-w^2), a mixture of s exp(-w^2) (weight s sqrt(pi); w normal with
//     variance 1/2) and |w| exp(-w^2) (weight 1; |w| = sqrt(-ln u), random
//     sign); accept z > 0 with probability z / (s + |w|);
//   -1 <= s < 0: with a = -s and w = z + a > a the density is (w - a)
//     exp(-w^2) <= w exp(-w^2), whose tail beyond a is w = sqrt(a^2 - ln u);
//     accept with probability (w - a) / w;
//   s < -1: the density is proportional to z exp(-2 a z) exp(-z^2): z from
//     Gamma(2, rate 2a), accepted with probability exp(-z^2).
// The acceptance rate is at least ~24 %; after 64 rejected tries (odds
// below 1e-7) returns -1 and the caller takes the FP64 inverse.
__device__ __forceinline__ float inflow_speed_f32(float s, Stream<float>& st) {
  const float SQRTPI = 1.7724538509055159f;
  for (uint32_t t = 0; t < 64u; ++t) {
    const uint32_t j = 64u + 4u * t;
    const float ua = st.u(j), ub = st.u(j + 1), uc = st.u(j + 2), ud = st.u(j + 3);
    if (s >= 0.f) {
      float w;
      if (ua * (s * SQRTPI + 1.f) < s * SQRTPI) {
        float sn, cn;
        m_sincos_2pi(uc, &sn, &cn);
        w = sqrtf(-__logf(ub)) * cn;
      } else {
        w = sqrtf(-__logf(ub));
        if (uc < 0.5f) w = -w;
      }
      const float z = s + w;
      if (z > 0.f && ud * (s + fabsf(w)) < z) return z;
    } else if (s >= -1.f) {
      const float a = -s;
      const float w = sqrtf(a * a - __logf(ub));
      if (ud * w < w - a) return w - a;
    } else {
      const float a = -s;
      const float z = -(__logf(ub) + __logf(uc)) / (2.f * a);
      if (ud < __expf(-z * z)) return z;
    }
  }
  return -1.f;
}

// FP32 layout: particle q of face k in FP32 (the draws of inflow_particle,
// the speed from inflow_speed_f32); false if it ends outside
__device__ __forceinline__ bool inflow_particle_f32(const Params<float>& p, int k, int q, uint32_t step, float* tally,
                                                    unsigned long long* hits, unsigned long long* maxhit, float& x,
                                                    float& y, float& vx, float& vy, float& vz, float& ir) {
  const float sT = sqrtf(p.fs_t), beta = rsqrtf(2.f * p.fs_t);
  const float nx = -p.fnrm[2 * k], ny = -p.fnrm[2 * k + 1];
  const float tx = -ny, ty = nx;
  const float un = p.fs_u[0] * nx + p.fs_u[1] * ny, ut = p.fs_u[0] * tx + p.fs_u[1] * ty;
  Stream<float> st(TAG_INJ, (uint32_t)q, (uint32_t)k, step, p.k0, p.k1);
  float z = inflow_speed_f32(un * beta, st);
  if (z < 0.f) z = (float)inflow_speed((double)(un * beta), (double)st.u(0));
  const float vn = z / beta;
  float n1, n2;
  box_muller(st.u(1), st.u(2), &n1, &n2);
  const float vt = ut + sT * n1;
  vx = vn * nx + vt * tx;
  vy = vn * ny + vt * ty;
  vz = p.fs_u[2] + sT * n2;
  const float th = 6.283185307179586f * ((float)k + st.u(3)) / (float)p.nx;
  ir = rot_energy(p.d_r3 != 0, p.fs_t, st.u(4), st, JX_OWN);
  x = p.r_out * cosf(th);
  y = p.r_out * sinf(th);
  return fly_ann<float, true>(p, x, y, vx, vy, vz, ir, TAG_INJ, (uint32_t)q, (uint32_t)k, step, 8u, st.u(5) * p.dt,
                              tally, hits, maxhit);
}

// Expected entries of every outer face per step, mu_k (the mean of
// inflow_count's Iround), written once per handle
static __global__ void k_inflow_means(const __grid_constant__ Params<double> p, double* __restrict__ mu) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < p.nx; k += gridDim.x * blockDim.x) {
    const double beta = 1.0 / sqrt(2.0 * p.fs_t);
    const double len = p.r_out * 2.0 * PI_D / (double)p.nx;
    const double nx = -p.fnrm[2 * k], ny = -p.fnrm[2 * k + 1];
    const double sn = (p.fs_u[0] * nx + p.fs_u[1] * ny) * beta;
    mu[k] = p.fs_rho * inflow_ginf(sn) / (beta * sqrt(PI_D)) * len * p.dt / p.fnum;
  }
}

// FP32 layout: one thread per entering particle.  Every CTA (one warp) draws
// the faces' counts from the precomputed means (the same Iround draws as
// inflow_count) and scans them in shared memory; lane t of the grid takes
// the t-th new particle, finds its face by bisection, samples it and appends
// it to the next step's bins (warp-aggregated, overflow list when a bin is
// full).  off: dynamic shared memory, nx + 1 ints.
static __global__ void __launch_bounds__(32) k_inject_bins(const __grid_constant__ Params<double> pd,
                                                           const __grid_constant__ Params<float> pf,
                                                           const double* __restrict__ mu, PBuf<float> out,
                                                           const int32_t* __restrict__ start,
                                                           int32_t* __restrict__ cnt_out, Ovf ovo, int ovf_cap,
                                                           uint32_t step, double* __restrict__ tally_g,
                                                           unsigned long long* __restrict__ stats,
                                                           int32_t* __restrict__ errflag) {
  extern __shared__ int32_t off[];
  __shared__ float s_tally[5];
  __shared__ unsigned s_misc[2];
  __shared__ unsigned long long s_hits[2];
  const int lane = threadIdx.x;
  if (lane < 5) s_tally[lane] = 0.f;
  if (lane < 2) {
    s_misc[lane] = 0;
    s_hits[lane] = 0;
  }
  const int nt = pd.nx;
  // counts and their exclusive scan, 32 faces at a time
  int run = 0;
  for (int k0 = 0; k0 < nt; k0 += 32) {
    const int k = k0 + lane;
    int c = 0;
    if (k < nt) {
      Stream<double> sc(TAG_INJ, 0xFFFFFFFFu, (uint32_t)k, step, pd.k0, pd.k1);
      const long long m = iround(mu[k], sc.u(0));
      c = (int)(m < 0 ? 0 : (m > (1 << 20) ? (1 << 20) : m));
    }
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (k < nt) off[k] = run + x - c;
    run += __shfl_sync(FULL, x, 31);
  }
  if (lane == 0) off[nt] = run;
  __syncwarp();
  const int total = run;
  unsigned nin = 0;
  for (int t0 = blockIdx.x * 32; t0 < total; t0 += gridDim.x * 32) {
    const int t = t0 + lane;
    float x = 0.f, y = 0.f, vx = 0.f, vy = 0.f, vz = 0.f, ir = 0.f;
    int d = -1;
    if (t < total) {
      int lo = 0, hi = nt - 1;  // the face k with off[k] <= t < off[k + 1]
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      if (inflow_particle_f32(pf, lo, t - off[lo], step, s_tally, &s_hits[0], &s_hits[1], x, y, vx, vy, vz, ir))
        d = cell_of_ann<float>(pf, x, y);
      if (d >= 0) ++nin;  // one that ends outside never entered
    }
    append_particle<2>(pf, out, start, cnt_out, ovo, ovf_cap, d >= 0, d, x, y, vx, vy, vz, ir, s_misc, errflag);
  }
  __syncwarp();
  for (int o = 16; o > 0; o >>= 1) nin += __shfl_xor_sync(FULL, nin, o);
  if (lane == 0 && nin) atomicAdd(stats + ST_INJ, (unsigned long long)nin);
  if (lane < 5 && s_tally[lane] != 0.f) atomicAdd(tally_g + lane, (double)s_tally[lane]);
  if (lane == 5 && s_misc[0]) atomicAdd(stats + ST_OVF, (unsigned long long)s_misc[0]);
  if (lane == 6 && s_misc[1]) atomicAdd(stats + ST_NEARFULL, (unsigned long long)s_misc[1]);
  if (lane == 7 && s_hits[0]) atomicAdd(stats + ST_HITS, s_hits[0]);
  if (lane == 8 && s_hits[1]) atomicAdd(stats + ST_MAXHIT, s_hits[1]);
}

template <typename T>
__device__ __forceinline__ void flush_counts(const CollCount& cc, unsigned* s_cnt) {
  unsigned a = cc.cand, b = cc.coll, c = cc.clip, d = cc.inel;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(FULL, a, o);
    b += __shfl_xor_sync(FULL, b, o);
    c += __shfl_xor_sync(FULL, c, o);
    d += __shfl_xor_sync(FULL, d, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(s_cnt + 0, a);
    atomicAdd(s_cnt + 1, b);
    atomicAdd(s_cnt + 2, c);
    atomicAdd(s_cnt + 3, d);
  }
}

// One warp per cell: stage the cell's velocities and rotational energies in
// shared memory (cells above `tile` particles work in global memory), run
// NTC collisions and/or sampling, write back.  flags: 1 collide, 2 sample.
template <typename T, bool BATCH>
__global__ void __launch_bounds__(WPB * 32) k_collide_sample(const __grid_constant__ Params<T> pk, Cases<T> cases,
                                                             int ncells, PBuf<T> b,
                                                             const int32_t* __restrict__ start,
                                                             const int32_t* __restrict__ count,
                                                             T* __restrict__ sgmax, double* __restrict__ acc,
                                                             double* __restrict__ comp,
                                                             uint32_t* __restrict__ owner_g,
                                                             uint32_t step, int flags, int tile,
                                                             unsigned long long* __restrict__ stats,
                                                             float* __restrict__ stg = nullptr,
                                                             float* __restrict__ stc = nullptr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_cnt[4];
  if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * WPB + warp;
  if (cell < ncells) {
    const int cs = BATCH ? cases.cell_case[cell] : 0;
    const Params<T>& p = BATCH ? cases.p[cs] : pk;
    const int lcell = cell - (BATCH ? cases.cell0[cs] : 0);
    const int base = start[cell], n = count[cell];
    T* tv = reinterpret_cast<T*>(smem) + (size_t)warp * tile * 4;
    uint32_t* tow = reinterpret_cast<uint32_t*>(smem + (size_t)WPB * tile * 4 * sizeof(T)) + (size_t)warp * tile;
    const bool staged = n <= tile;
    T *vx, *vy, *vz, *ir;
    uint32_t* own;
    if (staged) {
      vx = tv;
      vy = tv + tile;
      vz = tv + 2 * tile;
      ir = tv + 3 * tile;
      own = tow;
      for (int q = lane; q < n; q += 32) {
        vx[q] = b.vx[base + q];
        vy[q] = b.vy[base + q];
        vz[q] = b.vz[base + q];
        ir[q] = b.ir[base + q];
      }
    } else {
      vx = b.vx + base;
      vy = b.vy + base;
      vz = b.vz + base;
      ir = b.ir + base;
      own = owner_g + base;
    }
    __syncwarp();
    if (flags & 1) {
      CollCount cc{0, 0, 0, 0};
      collide_cell<T>(p, vx, vy, vz, ir, n, (uint32_t)lcell, step, sgmax + cell, own, cc);
      flush_counts<T>(cc, s_cnt);
      __syncwarp();
    }
    if (flags & 2) {
      if (stg) {
        // FP32 staging accumulators: always folded here (last step of a call)
        float pre32[2] = {0.f, 0.f};
        if (lane < NMOM) {
          pre32[0] = stg[(size_t)cell * NMOM + lane];
          pre32[1] = stc[(size_t)cell * NMOM + lane];
        }
        sample_cell<T>(vx, vy, vz, ir, n, acc + (size_t)cell * NMOM, comp + (size_t)cell * NMOM, nullptr,
                       stg + (size_t)cell * NMOM, stc + (size_t)cell * NMOM, pre32, true);
      } else {
        sample_cell<T>(vx, vy, vz, ir, n, acc + (size_t)cell * NMOM, comp + (size_t)cell * NMOM);
      }
    }
    if (staged && (flags & 1)) {
      for (int q = lane; q < n; q += 32) {
        b.vx[base + q] = vx[q];
        b.vy[base + q] = vy[q];
        b.vz[base + q] = vz[q];
        b.ir[base + q] = ir[q];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(stats + threadIdx.x, (unsigned long long)s_cnt[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// FP32 padded-bin layout: the fused step
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void append_particle(const Params<float>& p, const PBuf<float>& o,
                                                const int32_t* __restrict__ start,
                                                int32_t* __restrict__ cnt_out, const Ovf& ovo,
                                                int ovf_cap, bool active, int d, float x, float y,
                                                float vx, float vy, float vz, float ir,
                                                unsigned* s_misc, int32_t* errflag) {
  const int lane = threadIdx.x & 31;
  const int key = active ? d : -1;
  const unsigned peers = __match_any_sync(FULL, key);
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  int b = 0;
  if (active && lane == leader) b = atomicAdd(&cnt_out[d], __popc(peers));
  b = __shfl_sync(FULL, b, leader);
  if (!active) return;
  const int slot = b + rank;
  const int s0 = start[d], cap = start[d + 1] - s0;
  if (slot < cap) {
    const int w = s0 + slot;
    o.x[w] = x;
    if (DIM == 2) o.y[w] = y;
    o.vx[w] = vx;
    o.vy[w] = vy;
    o.vz[w] = vz;
    o.ir[w] = ir;
    if (slot >= cap - 8) atomicAdd(s_misc + 1, 1u);
  } else {
    // the slot was reserved but is not used: give it back, so that the bin's
    // count ends at its capacity
    atomicSub(&cnt_out[d], 1);
    const int q = atomicAdd(ovo.count, 1);
    atomicAdd(s_misc + 0, 1u);
    if (q < ovf_cap) {
      ovo.x[q] = x;
      ovo.y[q] = y;
      ovo.vx[q] = vx;
      ovo.vy[q] = vy;
      ovo.vz[q] = vz;
      ovo.ir[q] = ir;
      ovo.dest[q] = d;
    } else {
      atomicOr(errflag, 2);  // the overflow list is full: the particle is lost
    }
  }
}

// Destination of a particle that left cell `cell` for cell `d`, as an index
// into the 3 x 3 neighbourhood of `cell` (4 = stays), or 9 for a farther cell.
template <int DIM>
__device__ __forceinline__ int neighbour_code(const Params<float>& p, int ix, int iy, float x, float y) {
  int jx, jy = 0;
  if (DIM == 2 && p.mesh == 2) {
    // wall-refined box: the cell from its edge tables
    jx = edge_index(p.xe, p.nx, x);
    jy = edge_index(p.ye, p.ny, y);
  } else {
    jx = (int)(x * p.sx);
    jx = jx < 0 ? 0 : (jx > p.nx - 1 ? p.nx - 1 : jx);
    if (DIM == 2) {
      jy = (int)(y * p.sy);
      jy = jy < 0 ? 0 : (jy > p.ny - 1 ? p.ny - 1 : jy);
    }
  }
  const int dx = jx - ix, dy = jy - iy;
  if (dx < -1 || dx > 1 || dy < -1 || dy > 1) return 9;
  return (dy + 1) * 3 + (dx + 1);
}

__device__ __forceinline__ int neighbour_cell(int nx, int cell, int code) {
  return cell + (code / 3 - 1) * nx + (code % 3 - 1);
}

// Annulus: the geometry one cell's moves need, read from the tables once
// per cell: the squared radii of rings j-1 .. j+2 (sentinels where a ring is
// missing) and the rays of sectors k-1 .. k+2 (wrapping around).
struct AnnCell {
  float rin2, r2m, r2lo, r2hi, r2p;
  float cm, sm, clo, slo, cup, sup, cp, sp;
};

__device__ __forceinline__ AnnCell ann_cell(const Params<float>& p, int k, int j) {
  AnnCell g;
  const int nt = p.nx;
  g.rin2 = p.r2t[0];
  g.r2lo = p.r2t[j];
  g.r2hi = p.r2t[j + 1];
  g.r2m = (j > 0) ? p.r2t[j - 1] : -1.f;            // below ring 0: stays in ring 0
  g.r2p = (j + 1 < p.ny) ? p.r2t[j + 2] : -1.f;  // none beyond the outer ring
  const int km = (k == 0) ? nt - 1 : k - 1, kp = (k + 2 > nt) ? k + 2 - nt : k + 2;
  g.cm = p.ray[2 * km];
  g.sm = p.ray[2 * km + 1];
  g.clo = p.ray[2 * k];
  g.slo = p.ray[2 * k + 1];
  g.cup = p.ray[2 * k + 2];
  g.sup = p.ray[2 * k + 3];
  g.cp = p.ray[2 * kp];
  g.sp = p.ray[2 * kp + 1];
  return g;
}

// Annulus: the straight flight over dt, true if it does not meet the
// cylinder (the test of fly_ann)
__device__ __forceinline__ bool ann_straight(const Params<float>& p, float rin2, float x, float y, float vx, float vy,
                                             float* xn, float* yn) {
  *xn = x + vx * p.dt;
  *yn = y + vy * p.dt;
  const float a = vx * vx + vy * vy, b = x * vx + y * vy;
  if (b < 0.f && a > 0.f) {
    const float cc = x * x + y * y - rin2;
    const float disc = b * b - a * cc;
    if (disc > 0.f) {
      float s1 = (-b - sqrtf(disc)) / a;
      if (s1 < 0.f) s1 = 0.f;
      if (s1 < p.dt) return false;
    }
  }
  return true;
}

// Annulus: code (dj + 1) * 3 + (dk + 1) of the cell (ring j + dj, sector
// k + dk mod nx) holding (x, y), from the squared radii of ring j's
// neighbours and the signs against sector k's neighbouring rays; 9 when the
// particle is farther or outside r_out.
__device__ __forceinline__ int neighbour_code_ann(const AnnCell& g, int j, float x, float y) {
  const float r2 = x * x + y * y;
  int dj = 0;
  if (r2 < g.r2lo) {
    if (j > 0) {
      if (!(r2 >= g.r2m)) return 9;
      dj = -1;
    }
  } else if (!(r2 < g.r2hi)) {
    if (!(r2 < g.r2p)) return 9;  // r2p = -1 past the outer ring
    dj = 1;
  }
  const bool lo = g.clo * y - g.slo * x >= 0.f;
  const bool up = g.cup * y - g.sup * x >= 0.f;
  int dk = 0;
  if (!lo) {
    if (!(g.cm * y - g.sm * x >= 0.f)) return 9;
    dk = -1;
  } else if (up) {
    if (!(g.cp * y - g.sp * x < 0.f)) return 9;
    dk = 1;
  }
  return (dj + 1) * 3 + (dk + 1);
}

__device__ __forceinline__ int neighbour_cell_ann(int nx, int cell, int code) {
  const int j = cell / nx + code / 3 - 1;
  int k = cell % nx + code % 3 - 1;
  k = (k < 0) ? k + nx : (k >= nx ? k - nx : k);
  return j * nx + k;
}

// warps per CTA of the fused step: 2 or 4, chosen per handle with the tile
// by timing real steps of the handle's first long dsmc_step call (step_bins)
constexpr int FWPB_MAX = 4;
constexpr uint32_t MBAR_POLL_LIMIT = 1u << 22;  // bounded wait for a cell's bulk copies

// shared memory of the fused step: per warp, tile x (vx, vy, vz, I_r, x, y)
// floats and tile x u32 (collision owners, then destination tags)
inline size_t fused_smem_bytes(int tile, int fwpb) { return (size_t)fwpb * tile * 28; }

// flags: 1 collide (step_c), 2 sample, 4 move (step_m) into `out`, 8 fold the
// FP32 staging sums into the FP64 accumulators after sampling.
// Blocks [0, ncell_blocks) take FWPB cells each, one warp per cell; the
// remaining blocks move the particles of the input overflow list.
//
// Staging: one lane issues bulk asynchronous copies (TMA, cp.async.bulk) of
// the cell's six arrays into shared memory, completed on the warp's mbarrier,
// so a cell costs one memory round trip however many particles it holds.
// Move and append: (M1) fly every particle to find its destination and its
// rank among the cell's particles bound for the same neighbour (shared-memory
// counters over the 3 x 3 neighbourhood); (M2) one global atomicAdd per
// destination bin reserves the slots; (M3) fly again (the same counter-based
// random stream, so the same result) and store.  Counters are flushed by the
// last warp of the block to finish, so warps never wait for one another.
template <int DIM, bool BATCH, int FWPB, bool ANN, bool GEN>
__global__ void __launch_bounds__(FWPB * 32, 32 / FWPB) k_fused(const __grid_constant__ Params<float> pk,
                                                        Cases<float> cases, int ncells, PBuf<float> in,
                                                        PBuf<float> out,
                                                        const int32_t* __restrict__ start,
                                                        int32_t* __restrict__ cnt_in,
                                                        int32_t* __restrict__ cnt_out,
                                                        float* __restrict__ sgmax, double* __restrict__ acc,
                                                        double* __restrict__ comp,
                                                        uint32_t* __restrict__ owner_g, Ovf ovi, Ovf ovo,
                                                        int ovf_cap, uint32_t step_c, uint32_t step_m,
                                                        int flags, int tile, int ncell_blocks,
                                                        double* __restrict__ tally_g,
                                                        unsigned long long* __restrict__ stats,
                                                        int32_t* __restrict__ errflag, float* __restrict__ stg,
                                                        float* __restrict__ stc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_cnt[4];
  __shared__ unsigned s_misc[2];
  __shared__ float s_tally[20];
  __shared__ unsigned long long s_hits[2];
  __shared__ unsigned s_done;
  __shared__ unsigned s_out;  // annulus: particles that left
  __shared__ int s_nb[FWPB][4][12];  // per warp: count, base, bin start, bin capacity
  __shared__ __align__(8) uint64_t s_bar[FWPB];
  if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x < 2) s_misc[threadIdx.x] = 0;
  if (threadIdx.x < 20) s_tally[threadIdx.x] = 0.f;
  if (threadIdx.x < 2) s_hits[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_done = 0;
  if (threadIdx.x == 0) s_out = 0;
  if (threadIdx.x < FWPB) mbar_init(&s_bar[threadIdx.x], 1);
  mbar_fence_init();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((int)blockIdx.x < ncell_blocks) {
    const int cell = blockIdx.x * FWPB + warp;
    if (cell < ncells) {
      const int cs = BATCH ? cases.cell_case[cell] : 0;
      const Params<float>& p = BATCH ? cases.p[cs] : pk;
      const int c0 = BATCH ? cases.cell0[cs] : 0;
      const int lcell = cell - c0;
      const int base = start[cell], n = cnt_in[cell];
      const bool flush = (flags & 8) != 0;
      double pre[2] = {0.0, 0.0};
      float pre32[2] = {0.f, 0.f};
      const int mom = halving_moment(lane);
      if ((flags & 2) && mom >= 0) {
        pre32[0] = stg[(size_t)cell * NMOM + mom];
        pre32[1] = stc[(size_t)cell * NMOM + mom];
        if (flush) {
          pre[0] = acc[(size_t)cell * NMOM + mom];
          pre[1] = comp[(size_t)cell * NMOM + mom];
        }
      }
      float* tvx = reinterpret_cast<float*>(smem + (size_t)warp * tile * 28);
      uint32_t* tow = reinterpret_cast<uint32_t*>(tvx + 6 * tile);
      const bool staged = n <= tile;
      const int narr = (DIM == 2) ? 6 : 5;
      // bulk copies of particles [q0, q0 + m) of the cell into the tile on the
      // warp's mbarrier at phase ph (bounded wait; false on a timeout)
      auto stage = [&](int q0, int m, uint32_t ph) -> bool {
        if (lane == 0) {
          const uint32_t bytes = (uint32_t)((m + 3) & ~3) * 4u;
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&s_bar[warp], bytes * narr);
          bulk_g2s(tvx, in.vx + base + q0, bytes, &s_bar[warp]);
          bulk_g2s(tvx + tile, in.vy + base + q0, bytes, &s_bar[warp]);
          bulk_g2s(tvx + 2 * tile, in.vz + base + q0, bytes, &s_bar[warp]);
          bulk_g2s(tvx + 3 * tile, in.ir + base + q0, bytes, &s_bar[warp]);
          bulk_g2s(tvx + 4 * tile, in.x + base + q0, bytes, &s_bar[warp]);
          if (DIM == 2) bulk_g2s(tvx + 5 * tile, in.y + base + q0, bytes, &s_bar[warp]);
        }
        const bool r = mbar_wait_bounded(&s_bar[warp], ph, MBAR_POLL_LIMIT);
        if (!r && lane == 0) atomicOr(errflag, 1);
        return __all_sync(FULL, r);
      };
      bool ok = true;
      if (staged && n > 0) ok = stage(0, n, 0u);
      float* vx = tvx;
      float* vy = tvx + tile;
      float* vz = tvx + 2 * tile;
      float* ir = tvx + 3 * tile;
      const float* px = tvx + 4 * tile;
      const float* py = tvx + 5 * tile;
      uint32_t* own = tow;
      float mtot = 0.f;  // cell above the tile: this lane's moment summed over the chunks
      // The cell body on the shared-memory tile, for particles [q0, q0 + m)
      // of the cell: the whole cell when it fits the tile (WHOLE), or one
      // chunk of a larger cell, whose collisions ran in global memory and
      // whose sums, reduced per chunk, add up over the chunks.
      auto body = [&](auto whole_tag, int q0, int m) {
        constexpr bool whole = decltype(whole_tag)::value;
        if (whole && (flags & 1)) {
          CollCount cc{0, 0, 0, 0};
          collide_cell<float, GEN>(p, vx, vy, vz, ir, m, (uint32_t)lcell, step_c, sgmax + cell, own, cc);
          flush_counts<float>(cc, s_cnt);
          __syncwarp();
        }
        if (flags & 2) {
          if constexpr (whole)
            sample_cell_staged(vx, vy, vz, ir, m, mom, acc + (size_t)cell * NMOM, comp + (size_t)cell * NMOM, pre,
                               stg + (size_t)cell * NMOM, stc + (size_t)cell * NMOM, pre32, flush);
          else
            mtot += sample_chunk(vx, vy, vz, ir, m);
        }
        if (flags & 4) {
          int* nb_cnt = s_nb[warp][0];
          int* nb_base = s_nb[warp][1];
          int* nb_s0 = s_nb[warp][2];
          int* nb_cap = s_nb[warp][3];
          if (lane < 12) nb_cnt[lane] = 0;
          __syncwarp();
          // M1: destinations and ranks; a particle that reaches a wall is
          // placed individually in M3 (code 9)
          const int cix = lcell % p.nx, ciy = lcell / p.nx;
          AnnCell ag;
          if constexpr (ANN) ag = ann_cell(p, cix, ciy);
          for (int q = lane; q < m; q += 32) {
            float xn, yn;
            int code = 9;
            if constexpr (ANN) {
              if (ann_straight(p, ag.rin2, px[q], py[q], vx[q], vy[q], &xn, &yn))
                code = neighbour_code_ann(ag, ciy, xn, yn);
            } else {
              if (flight_stays_inside<float, DIM>(p, px[q], (DIM == 2) ? py[q] : 0.f, vx[q], vy[q], &xn, &yn))
                code = neighbour_code<DIM>(p, cix, ciy, xn, yn);
            }
            const int r = atomicAdd(&nb_cnt[code], 1);
            own[q] = ((uint32_t)code << 24) | (uint32_t)r;
          }
          __syncwarp();
          // M2: reserve the slots, one atomic per destination bin
          if (lane < 9 && nb_cnt[lane] > 0) {
            const int d = ANN ? neighbour_cell_ann(p.nx, cell, lane) : neighbour_cell(p.nx, cell, lane);
            nb_base[lane] = atomicAdd(&cnt_out[d], nb_cnt[lane]);
            const int s0 = start[d];
            nb_s0[lane] = s0;
            nb_cap[lane] = start[d + 1] - s0;
          }
          __syncwarp();
          // M3: fly again (identical result) with wall tallies, and store
          for (int q = lane; q < m; q += 32) {
            float x = px[q], y = (DIM == 2) ? py[q] : 0.f;
            float a = vx[q], b = vy[q], c = vz[q], e = ir[q];
            const uint32_t tag = own[q];
            const int code = (int)(tag >> 24), r = (int)(tag & 0xFFFFFFu);
            if constexpr (ANN) {
              if (code < 9) {
                x = x + a * p.dt;
                y = y + b * p.dt;
              } else if (!fly_ann<float, true, GEN>(p, x, y, a, b, c, e, TAG_WALL, (uint32_t)(q0 + q), (uint32_t)lcell, step_m, 0u,
                                               p.dt, s_tally, &s_hits[0], &s_hits[1])) {
                atomicAdd(&s_out, 1u);  // left through the outer circle
                continue;
              }
            } else {
              fly<float, DIM, true, GEN>(p, x, y, a, b, c, e, (uint32_t)(q0 + q), (uint32_t)lcell, step_m, s_tally, &s_hits[0],
                                    &s_hits[1]);
            }
            int d = -1, slot, s0, cap;
            if (code < 9) {
              slot = nb_base[code] + r;
              s0 = nb_s0[code];
              cap = nb_cap[code];
            } else {
              d = ANN ? cell_of_ann<float>(p, x, y) : c0 + cell_of<float, DIM>(p, x, y);
              if (ANN && d < 0) {
                atomicAdd(&s_out, 1u);
                continue;
              }
              slot = atomicAdd(&cnt_out[d], 1);
              s0 = start[d];
              cap = start[d + 1] - s0;
            }
            if (slot < cap) {
              const int w = s0 + slot;
              out.x[w] = x;
              if (DIM == 2) out.y[w] = y;
              out.vx[w] = a;
              out.vy[w] = b;
              out.vz[w] = c;
              out.ir[w] = e;
              if (slot >= cap - 8) atomicAdd(s_misc + 1, 1u);
            } else {
              // reserved but unused slot: give it back (the bin's count ends
              // at its capacity)
              if (d < 0) d = ANN ? neighbour_cell_ann(p.nx, cell, code) : neighbour_cell(p.nx, cell, code);
              atomicSub(&cnt_out[d], 1);
              const int qo = atomicAdd(ovo.count, 1);
              atomicAdd(s_misc + 0, 1u);
              if (qo < ovf_cap) {
                ovo.x[qo] = x;
                ovo.y[qo] = y;
                ovo.vx[qo] = a;
                ovo.vy[qo] = b;
                ovo.vz[qo] = c;
                ovo.ir[qo] = e;
                ovo.dest[qo] = d;
              } else {
                atomicOr(errflag, 2);  // the overflow list is full: the particle is lost
              }
            }
          }
        } else if (whole && (flags & 1)) {
          for (int q = lane; q < m; q += 32) {
            in.vx[base + q] = vx[q];
            in.vy[base + q] = vy[q];
            in.vz[base + q] = vz[q];
            in.ir[base + q] = ir[q];
          }
        }
      };
      if (ok) {
        if (staged) {
          body(std::true_type{}, 0, n);
        } else {
          // a cell above the tile: collisions in place in global memory (the
          // candidates pick particles anywhere in the cell), then sampling
          // and the move chunk by chunk through the tile
          if (flags & 1) {
            CollCount cc{0, 0, 0, 0};
            collide_cell<float, GEN>(p, in.vx + base, in.vy + base, in.vz + base, in.ir + base, n, (uint32_t)lcell, step_c,
                                sgmax + cell, owner_g + base, cc);
            flush_counts<float>(cc, s_cnt);
            fence_proxy_async_global();  // the bulk copies below read these velocities
            __syncwarp();
          }
          if (flags & 6) {
            uint32_t ph = 0u;
            for (int q0 = 0; q0 < n && ok; q0 += tile, ph ^= 1u) {
              const int m = min(tile, n - q0);
              __syncwarp();  // every lane is done with the previous chunk
              ok = stage(q0, m, ph);
              if (ok) body(std::false_type{}, q0, m);
            }
          }
          if (ok && (flags & 2))
            sample_fold(mtot, mom, acc + (size_t)cell * NMOM, comp + (size_t)cell * NMOM, pre,
                        stg + (size_t)cell * NMOM, stc + (size_t)cell * NMOM, pre32, flush);
        }
        if (ok && (flags & 4)) {
          __syncwarp();
          if (lane == 0) cnt_in[cell] = 0;
        }
      }
    }
  } else if (flags & 4) {
    // overflow list of the previous step: move and append (no collision)
    const int nov = min(*ovi.count, ovf_cap);
    const int gw = (blockIdx.x - ncell_blocks) * FWPB + warp;
    const int nwarps = (gridDim.x - ncell_blocks) * FWPB;
    for (int base = gw * 32; base < nov; base += nwarps * 32) {
      const int q = base + lane;
      const bool active = q < nov;
      float x = 0.f, y = 0.f, a = 0.f, bb = 0.f, c = 0.f, e = 0.f;
      int d = 0;
      if (active) {
        const int cs = BATCH ? cases.cell_case[ovi.dest[q]] : 0;
        const Params<float>& p = BATCH ? cases.p[cs] : pk;
        const int c0 = BATCH ? cases.cell0[cs] : 0;
        x = ovi.x[q];
        y = ovi.y[q];
        a = ovi.vx[q];
        bb = ovi.vy[q];
        c = ovi.vz[q];
        e = ovi.ir[q];
        if constexpr (ANN) {
          d = fly_ann<float, true, GEN>(p, x, y, a, bb, c, e, TAG_WALL, (uint32_t)q, (uint32_t)(p.ncells + 1), step_m, 0u,
                                   p.dt, s_tally, &s_hits[0], &s_hits[1])
                  ? cell_of_ann<float>(p, x, y)
                  : -1;
          if (d < 0) atomicAdd(&s_out, 1u);
        } else {
          fly<float, DIM, true, GEN>(p, x, y, a, bb, c, e, (uint32_t)q, (uint32_t)(p.ncells + 1), step_m, s_tally,
                                &s_hits[0], &s_hits[1]);
          d = c0 + cell_of<float, DIM>(p, x, y);
        }
      }
      append_particle<DIM>(pk, out, start, cnt_out, ovo, ovf_cap, active && d >= 0, d, x, y, a, bb, c, e, s_misc,
                           errflag);
    }
  }
  // the last warp of the block to finish flushes the block's counters
  __syncwarp();
  __threadfence_block();
  unsigned done = 0;
  if (lane == 0) done = atomicAdd(&s_done, 1u);
  done = __shfl_sync(FULL, done, 0);
  if (done == FWPB - 1) {
    __threadfence_block();
    if (lane < 4 && s_cnt[lane]) atomicAdd(stats + lane, (unsigned long long)s_cnt[lane]);
    if (lane == 4 && s_misc[0]) atomicAdd(stats + ST_OVF, (unsigned long long)s_misc[0]);
    if (lane == 5 && s_misc[1]) atomicAdd(stats + ST_NEARFULL, (unsigned long long)s_misc[1]);
    if (lane == 6 && s_hits[0]) atomicAdd(stats + ST_HITS, s_hits[0]);
    if (lane == 7 && s_hits[1]) atomicAdd(stats + ST_MAXHIT, s_hits[1]);
    if (lane == 8 && s_out) atomicAdd(stats + ST_OUT, (unsigned long long)s_out);
    if (lane < 20 && s_tally[lane] != 0.f) atomicAdd(tally_g + lane, (double)s_tally[lane]);
  }
}

static __global__ void k_zero_i32(int32_t* a, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = 0;
}

// ---------------------------------------------------------------------------
// FP32 layout rebuild: new bin capacities from the occupancies (+ overflow)
// ---------------------------------------------------------------------------
static __global__ void k_rebin_add_ovf(const Ovf ov, int ovf_cap, int32_t* __restrict__ tot) {
  const int nov = min(*ov.count, ovf_cap);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nov; q += gridDim.x * blockDim.x)
    atomicAdd(&tot[ov.dest[q]], 1);
}

// caps = bin_cap_of(tot, slack); halve the slack until the bins fit.
// nominal particles per cell of a cell's case: rho = 1 with weight F
__device__ __forceinline__ int32_t nominal_count(const CellParams* cps, const int32_t* cell_case, int c) {
  if (!cps) return 0;
  const CellParams& cp = cps[cell_case[c]];
  return (int32_t)((cp.vol ? cp.vol[c] : cp.vcell) / cp.fnum + 0.5);
}

static __global__ void __launch_bounds__(1024) k_caps_scan(const int32_t* __restrict__ tot, int ncells,
                                                    double slack, long long capacity,
                                                    int32_t* __restrict__ start_out,
                                                    int32_t* __restrict__ flags,
                                                    const CellParams* __restrict__ cps = nullptr,
                                                    const int32_t* __restrict__ cell_case = nullptr) {
  __shared__ double s_slack;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    s_slack = slack;
    s_ok = 0;
  }
  __syncthreads();
  for (int attempt = 0; attempt < 8; ++attempt) {
    const double sl = s_slack;
    cta_exclusive_scan(ncells, [&](int i) { return bin_cap_of(max(tot[i], nominal_count(cps, cell_case, i)), sl); },
                       start_out);
    if (threadIdx.x == 0) {
      if ((long long)start_out[ncells] <= capacity) s_ok = 1;
      else s_slack = 1.0 + 0.5 * (s_slack - 1.0);
    }
    __syncthreads();
    if (s_ok) break;
  }
  if (threadIdx.x == 0 && !s_ok) flags[2] = 1;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(WPB * 32) k_rebin_copy(PBuf<T> in, PBuf<T> out,
                                                         const int32_t* __restrict__ start_in,
                                                         const int32_t* __restrict__ cnt_in,
                                                         const int32_t* __restrict__ start_out,
                                                         int32_t* __restrict__ cnt_out, int ncells) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * WPB + warp;
  if (cell >= ncells) return;
  const int si = start_in[cell], so = start_out[cell], n = cnt_in[cell];
  for (int q = lane; q < n; q += 32) {
    out.x[so + q] = in.x[si + q];
    if (DIM == 2) out.y[so + q] = in.y[si + q];
    out.vx[so + q] = in.vx[si + q];
    out.vy[so + q] = in.vy[si + q];
    out.vz[so + q] = in.vz[si + q];
    out.ir[so + q] = in.ir[si + q];
  }
  if (lane == 0) cnt_out[cell] = n;
}

template <int DIM>
__global__ void k_rebin_ovf(const Ovf ov, int ovf_cap, PBuf<float> out, const int32_t* __restrict__ start_out,
                            int32_t* __restrict__ cnt_out) {
  const int nov = min(*ov.count, ovf_cap);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nov; q += gridDim.x * blockDim.x) {
    const int d = ov.dest[q];
    const int w = start_out[d] + atomicAdd(&cnt_out[d], 1);
    out.x[w] = ov.x[q];
    if (DIM == 2) out.y[w] = ov.y[q];
    out.vx[w] = ov.vx[q];
    out.vy[w] = ov.vy[q];
    out.vz[w] = ov.vz[q];
    out.ir[w] = ov.ir[q];
  }
}

// ---------------------------------------------------------------------------
// export / import
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(1024) k_scan_counts(const int32_t* __restrict__ cnt, int ncells,
                                                      int32_t* __restrict__ out) {
  cta_exclusive_scan(ncells, [&](int i) { return cnt[i]; }, out);
}

template <typename T>
__global__ void __launch_bounds__(WPB * 32) k_export(PBuf<T> b, const int32_t* __restrict__ start,
                                                     const int32_t* __restrict__ cnt,
                                                     const int32_t* __restrict__ ostart, int ncells,
                                                     double* x, double* y, double* vx, double* vy,
                                                     double* vz, double* ir, int32_t* cell_out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * WPB + warp;
  if (cell >= ncells) return;
  const int si = start[cell], so = ostart[cell], n = cnt[cell];
  for (int q = lane; q < n; q += 32) {
    x[so + q] = (double)b.x[si + q];
    y[so + q] = (double)b.y[si + q];
    vx[so + q] = (double)b.vx[si + q];
    vy[so + q] = (double)b.vy[si + q];
    vz[so + q] = (double)b.vz[si + q];
    ir[so + q] = (double)b.ir[si + q];
    cell_out[so + q] = cell;
  }
}

// DIM 3: the annulus (key -1 outside it)
template <typename T, int DIM>
__global__ void k_keys_from_pos(Params<T> p, const double* __restrict__ x, const double* __restrict__ y,
                                int n, int32_t* __restrict__ key) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    if constexpr (DIM == 3) key[s] = cell_of_ann<T>(p, (T)x[s], (T)y[s]);
    else key[s] = cell_of<T, DIM>(p, (T)x[s], (DIM == 2) ? (T)y[s] : T(0));
  }
}

// FP32 import: occupancy of every cell (one atomic per group of lanes with
// the same cell: imported particles often come ordered by cell)
static __global__ void k_count_keys(const int32_t* __restrict__ key, int n, int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (int s0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); s0 < n; s0 += gridDim.x * blockDim.x) {
    const int s = s0 + lane;
    const int k = (s < n) ? key[s] : -1;
    const unsigned peers = __match_any_sync(FULL, k);
    if (k >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[k], __popc(peers));
  }
}

// FP32 import: every particle into a slot of its cell's padded bin (the
// order inside a bin is that of the atomics; the FP32 layout keeps none)
template <int DIM>
static __global__ void k_scatter_bins(const double* __restrict__ x, const double* __restrict__ y,
                                      const double* __restrict__ vx, const double* __restrict__ vy,
                                      const double* __restrict__ vz, const double* __restrict__ ir,
                                      const int32_t* __restrict__ key, int n, const int32_t* __restrict__ start,
                                      int32_t* __restrict__ cnt, PBuf<float> o) {
  const int lane = threadIdx.x & 31;
  for (int s0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); s0 < n; s0 += gridDim.x * blockDim.x) {
    const int s = s0 + lane;
    const int k = (s < n) ? key[s] : -1;
    const unsigned peers = __match_any_sync(FULL, k);
    const int leader = __ffs(peers) - 1;
    int b = 0;
    if (k >= 0 && lane == leader) b = atomicAdd(&cnt[k], __popc(peers));
    b = __shfl_sync(FULL, b, leader);
    if (k < 0) continue;
    const int w = start[k] + b + __popc(peers & ((1u << lane) - 1u));
    o.x[w] = (float)x[s];
    o.y[w] = (DIM == 2) ? (float)y[s] : 0.f;
    o.vx[w] = (float)vx[s];
    o.vy[w] = (float)vy[s];
    o.vz[w] = (float)vz[s];
    o.ir[w] = (float)ir[s];
  }
}

static __global__ void k_fill_zero_d(double* a, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = 0.0;
}

// ---------------------------------------------------------------------------
// Sec. 3.2: particle modification
// ---------------------------------------------------------------------------
static __global__ void k_dig_counts(const CellParams* __restrict__ cps, const int32_t* __restrict__ cell_case,
                                    const int32_t* __restrict__ cell0, int ncells,
                                    const double* __restrict__ target, uint32_t iter,
                                    int det, double slack, int32_t* __restrict__ nt,
                                    int32_t* __restrict__ caps, int32_t* __restrict__ flags) {
  // the loop runs the same number of times in every lane of a warp, so that
  // the new total is summed per warp and added with one atomic
  const int stride = gridDim.x * blockDim.x;
  for (int c0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < ncells; c0 += stride) {
    const int c = c0 + (threadIdx.x & 31);
    int32_t nv = 0;
    if (c < ncells) {
      const int cs = cell_case[c];
      const CellParams& cp = cps[cs];
      const int lcell = c - cell0[cs];
      const double* t = target + (size_t)c * 6;
      bool bad = false;
      for (int q = 0; q < 6; ++q)
        if (!isfinite(t[q])) bad = true;
      // an empty target cell (rho 0, as an unsampled cell's fields read)
      // has no particles whose temperatures would matter
      if (!(t[0] >= 0.0) || (t[0] > 0.0 && (!(t[4] > 0.0) || !(t[5] > 0.0)))) bad = true;
      if (bad) {
        atomicOr(flags, 1);
        nt[c] = 0;
        caps[c] = 0;
      } else {
        Stream<double> st(TAG_DIG_N, 0u, (uint32_t)lcell, iter, cp.k0, cp.k1);
        const double vc = cp.vol ? cp.vol[lcell] : cp.vcell;  // the annulus's cells differ
        const double xm = t[0] * vc / cp.fnum;
        long long v = iround(xm, st.u(0));
        if (v > 0x3fffffffLL) {
          atomicOr(flags, 2);
          v = 0;
        }
        nv = (int32_t)v;
        nt[c] = nv;
        // FP32 bins: room for slack x the larger of the new and the nominal count
        const int32_t nominal = (int32_t)(vc / cp.fnum + 0.5);
        caps[c] = det ? nv : bin_cap_of(max(nv, nominal), slack);
      }
    }
    const int32_t wtot = __reduce_add_sync(FULL, nv);
    if ((threadIdx.x & 31) == 0 && wtot) atomicAdd(&flags[3], wtot);
    // the totals of the new counts and of the bin capacities in 64 bits
    // (flags 4-5 and 6-7), so that the host sees a target too large for
    // the workspace before an int32 sum or the layout scan could wrap
    unsigned long long c64 = (unsigned long long)nv, k64 = (c < ncells) ? (unsigned long long)caps[c] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c64 += __shfl_xor_sync(FULL, c64, o);
      k64 += __shfl_xor_sync(FULL, k64, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (c64) atomicAdd(reinterpret_cast<unsigned long long*>(flags + 4), c64);
      if (k64) atomicAdd(reinterpret_cast<unsigned long long*>(flags + 6), k64);
    }
  }
}

static __global__ void __launch_bounds__(1024) k_scan_caps(const int32_t* __restrict__ caps, int ncells,
                                                    long long capacity, int32_t* __restrict__ start_out,
                                                    int32_t* __restrict__ flags) {
  cta_exclusive_scan(ncells, [&](int i) { return caps[i]; }, start_out);
  if (threadIdx.x == 0) {
    flags[1] = start_out[ncells];
    if ((long long)start_out[ncells] > capacity) atomicOr(flags, 4);
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(WPB * 32) k_dig_apply(const CellParams* __restrict__ cps,
                                                        const int32_t* __restrict__ cell_case,
                                                        const int32_t* __restrict__ cell0, int ncells,
                                                        PBuf<T> in, PBuf<T> out,
                                                        const int32_t* __restrict__ start_in,
                                                        const int32_t* __restrict__ cnt_in,
                                                        const int32_t* __restrict__ start_out,
                                                        int32_t* __restrict__ cnt_out,
                                                        const int32_t* __restrict__ nt,
                                                        const double* __restrict__ target, uint32_t iter,
                                                        int32_t* __restrict__ idx_g,
                                                        int32_t* __restrict__ cellof_out, int tile) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * WPB + warp;
  if (cell >= ncells) return;
  const int cs = cell_case[cell];
  const CellParams& cp = cps[cs];
  const int lcell = cell - cell0[cs];
  const int s0 = start_in[cell], n = cnt_in[cell], d0 = start_out[cell], ntg = nt[cell];
  const double* t = target + (size_t)cell * 6;
  const int ix = lcell % cp.nx, iy = lcell / cp.nx;
  int32_t* idx = (n <= tile) ? reinterpret_cast<int32_t*>(smem) + (size_t)warp * tile * 2 : idx_g + s0;
  int32_t* rm = (n <= tile) ? reinterpret_cast<int32_t*>(smem) + (size_t)warp * tile * 2 + tile : nullptr;
  // step ii
  if (ntg <= n) {
    const int k = n - ntg;
    if (k > 0) {
      for (int q = lane; q < n; q += 32) idx[q] = q;
      __syncwarp();
      // partial Fisher-Yates: swap q draws r_q = q + floor(u_q (n - q)), which
      // does not depend on the earlier swaps, so 32 lanes draw at once and
      // lane 0 applies the swaps in order
      for (int qb = 0; qb < k; qb += 32) {
        const int q = qb + lane;
        int r = 0;
        if (q < k) {
          Stream<double> st(TAG_DIG_SEL, (uint32_t)q, (uint32_t)lcell, iter, cp.k0, cp.k1);
          r = q + (int)(st.u(0) * (double)(n - q));
          if (r > n - 1) r = n - 1;
        }
        const int m = min(32, k - qb);
        for (int j = 0; j < m; ++j) {
          const int rj = __shfl_sync(FULL, r, j);
          if (lane == 0) {
            const int tmp = idx[qb + j];
            idx[qb + j] = idx[rj];
            idx[rj] = tmp;
          }
        }
      }
      __syncwarp();
    }
    // mark the removed slots: in shared memory when the cell fits, else by
    // negating entries of idx (idx holds a permutation of 0..n-1)
    if (rm) {
      for (int q = lane; q < n; q += 32) rm[q] = 0;
      __syncwarp();
      for (int q = lane; q < k; q += 32) rm[idx[q]] = 1;
    } else if (k > 0) {
      // cell larger than the tile: idx lives in global scratch; mark removed
      // slot r by setting bit 30 of idx[r] (entries are < 2^30)
      for (int q = lane; q < k; q += 32) {
        const int slot = idx[q] & 0x3fffffff;
        atomicOr(&idx[slot], 0x40000000);
      }
    }
    __syncwarp();
    int kept_before = 0;
    for (int base = 0; base < n; base += 32) {
      const int q = base + lane;
      bool keep = false;
      if (q < n) {
        if (rm) keep = rm[q] == 0;
        else keep = (k == 0) || ((idx[q] & 0x40000000) == 0);
      }
      const unsigned m = __ballot_sync(FULL, keep);
      if (keep) {
        const int w = d0 + kept_before + __popc(m & ((1u << lane) - 1u));
        const T vx = in.vx[s0 + q], vy = in.vy[s0 + q], vz = in.vz[s0 + q], ir = in.ir[s0 + q];
        out.x[w] = in.x[s0 + q];
        out.y[w] = in.y[s0 + q];
        out.vx[w] = vx;
        out.vy[w] = vy;
        out.vz[w] = vz;
        out.ir[w] = ir;
      }
      kept_before += __popc(m);
    }
  } else {
    for (int q = lane; q < n; q += 32) {
      const T vx = in.vx[s0 + q], vy = in.vy[s0 + q], vz = in.vz[s0 + q], ir = in.ir[s0 + q];
      out.x[d0 + q] = in.x[s0 + q];
      out.y[d0 + q] = in.y[s0 + q];
      out.vx[d0 + q] = vx;
      out.vy[d0 + q] = vy;
      out.vz[d0 + q] = vz;
      out.ir[d0 + q] = ir;
    }
    for (int q = lane; q < ntg - n; q += 32) {
      Stream<double> sp(TAG_DIG_POS, (uint32_t)q, (uint32_t)lcell, iter, cp.k0, cp.k1);
      const int w = d0 + n + q;
      if (cp.mesh == 1) {
        // annulus: uniform in the sector (r^2 and the angle uniform)
        const double r = sqrt(cp.r2t[iy] + sp.u(0) * (cp.r2t[iy + 1] - cp.r2t[iy]));
        const double th = 2.0 * PI_D * ((double)ix + sp.u(1)) / (double)cp.nx;
        out.x[w] = (T)(r * cos(th));
        out.y[w] = (T)(r * sin(th));
      } else if (cp.mesh == 2) {
        // wall-refined box: uniform between the cell's edges
        out.x[w] = (T)(cp.xe[ix] + sp.u(0) * (cp.xe[ix + 1] - cp.xe[ix]));
        out.y[w] = (T)(cp.ye[iy] + sp.u(1) * (cp.ye[iy + 1] - cp.ye[iy]));
      } else {
        out.x[w] = (T)(((double)ix + sp.u(0)) * cp.dx);
        out.y[w] = (T)((cp.dim == 2) ? ((double)iy + sp.u(1)) * cp.dy : 0.0);
      }
      if (n > 0) {
        Stream<double> ss(TAG_DIG_SEL, (uint32_t)q, (uint32_t)lcell, iter, cp.k0, cp.k1);
        int src = (int)(ss.u(0) * (double)n);
        if (src > n - 1) src = n - 1;
        const T vx = in.vx[s0 + src], vy = in.vy[s0 + src], vz = in.vz[s0 + src], ir = in.ir[s0 + src];
        out.vx[w] = vx;
        out.vy[w] = vy;
        out.vz[w] = vz;
        out.ir[w] = ir;
      } else {
        double n1, n2, n3, n4;
        box_muller(sp.u(2), sp.u(3), &n1, &n2);
        box_muller(sp.u(4), sp.u(5), &n3, &n4);
        const double stt = sqrt(t[4]);
        const T vx = (T)(t[1] + stt * n1), vy = (T)(t[2] + stt * n2), vz = (T)(t[3] + stt * n3);
        const T ir = (T)rot_energy(cp.d_r == 3.0, t[5], sp.u(6), sp, JX_OWN);
        out.vx[w] = vx;
        out.vy[w] = vy;
        out.vz[w] = vz;
        out.ir[w] = ir;
      }
    }
  }
  __syncwarp();
  // step iii: u*, T_t*, T_r* of the new population, in FP64 in both layouts
  // (the factors of step iv too; FP32 particles are rounded once).  The mean
  // is taken about the first particle's velocity: copies of one particle (a
  // cell that held one particle and was refilled) then give u* equal to that
  // velocity and T_t* = 0 exactly (a = 1), and the second pass about u*
  // keeps the digits of the thermal spread.
  const int np = ntg;
  if (np > 0) {
    const double rx = (double)out.vx[d0], ry = (double)out.vy[d0], rz = (double)out.vz[d0];
    double sx = 0, sy = 0, sz = 0, si = 0;
    for (int q = lane; q < np; q += 32) {
      sx += (double)out.vx[d0 + q] - rx;
      sy += (double)out.vy[d0 + q] - ry;
      sz += (double)out.vz[d0 + q] - rz;
      si += (double)out.ir[d0 + q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(FULL, sx, o);
      sy += __shfl_xor_sync(FULL, sy, o);
      sz += __shfl_xor_sync(FULL, sz, o);
      si += __shfl_xor_sync(FULL, si, o);
    }
    const double ux = rx + sx / (double)np, uy = ry + sy / (double)np, uz = rz + sz / (double)np;
    double c2 = 0;
    for (int q = lane; q < np; q += 32) {
      const double cx = (double)out.vx[d0 + q] - ux, cy = (double)out.vy[d0 + q] - uy,
                   cz = (double)out.vz[d0 + q] - uz;
      c2 += cx * cx + cy * cy + cz * cz;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(FULL, c2, o);
    const double tts = c2 / (3.0 * (double)np);
    const double trs = 2.0 * si / (cp.d_r * (double)np);
    // step iv
    const double a = (np >= 2 && tts > 0.0) ? sqrt(t[4] / tts) : 1.0;
    const double bx = t[1] - ux * a, by = t[2] - uy * a, bz = t[3] - uz * a;
    const double cc = (trs > 0.0) ? t[5] / trs : 1.0;
    for (int q = lane; q < np; q += 32) {
      const int w = d0 + q;
      out.vx[w] = (T)(a * (double)out.vx[w] + bx);
      out.vy[w] = (T)(a * (double)out.vy[w] + by);
      out.vz[w] = (T)(a * (double)out.vz[w] + bz);
      out.ir[w] = (T)(cc * (double)out.ir[w]);
      if (cellof_out) cellof_out[w] = cell;
    }
  }
  if (lane == 0) cnt_out[cell] = ntg;
}

template <typename T>
__global__ void k_sgmax_io(T* sg, int n, double* out, const double* in) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    if (out) out[c] = (double)sg[c];
    if (in) sg[c] = (T)in[c];
  }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
inline int grid_for(long long n, int threads, int maxblocks = 152 * 16) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > maxblocks) b = maxblocks;
  return (int)b;
}

template <typename T>
void Ops<T>::init(const Params<T>& p, State<T>& s, int cur, int lay, int ppc, int cap0, double tt, double tr,
                  const double* u3, cudaStream_t st) {
  k_layout_uniform<<<grid_for(p.ncells + 1, 256), 256, 0, st>>>(p.ncells, (int32_t)cap0, s.start[lay]);
  const long long total = (long long)p.ncells * ppc;
  const int g = grid_for(total, 256);
  if (p.dim == 1)
    k_init<T, 1><<<g, 256, 0, st>>>(p, s.buf[cur], s.start[lay], s.count[lay], s.cellof, ppc, (T)tt, (T)tr,
                                    (T)u3[0], (T)u3[1], (T)u3[2]);
  else
    k_init<T, 2><<<g, 256, 0, st>>>(p, s.buf[cur], s.start[lay], s.count[lay], s.cellof, ppc, (T)tt, (T)tr,
                                    (T)u3[0], (T)u3[1], (T)u3[2]);
  if (ppc == 0) k_zero_i32<<<grid_for(p.ncells, 256), 256, 0, st>>>(s.count[lay], p.ncells);
}

template <typename T>
void Ops<T>::init_batch(const Params<T>& p0, State<T>& s, int ncells, int cur, int lay, cudaStream_t st,
                        const int32_t* counts) {
  const int blocks = (ncells * 32 + 255) / 256;
  if (p0.dim == 1)
    k_init_cells<T, 1><<<blocks, 256, 0, st>>>(s.cases, ncells, s.buf[cur], s.start[lay], s.count[lay], s.cellof,
                                               counts);
  else
    k_init_cells<T, 2><<<blocks, 256, 0, st>>>(s.cases, ncells, s.buf[cur], s.start[lay], s.count[lay], s.cellof,
                                               counts);
}

template <typename T>
void Ops<T>::ann_counts(const Params<double>& pd, int ncells, int32_t* counts, cudaStream_t st) {
  k_ann_counts<<<grid_for(ncells, 256), 256, 0, st>>>(pd, ncells, counts);
}

template <typename T>
void Ops<T>::inflow_means(const Params<double>& pd, double* mu, cudaStream_t st) {
  k_inflow_means<<<grid_for(pd.nx, 256), 256, 0, st>>>(pd, mu);
}

template <typename T>
static size_t tile_smem(int tile) {
  return (size_t)WPB * tile * (4 * sizeof(T) + sizeof(uint32_t));
}

template <typename T, bool BATCH>
static void launch_collide_sample(const Params<T>& p, State<T>& s, int ncells, const PBuf<T>& b, const int32_t* start,
                                  const int32_t* count, uint32_t step, int flags, float* stg, float* stc,
                                  cudaStream_t st) {
  const int blocks = (ncells + WPB - 1) / WPB;
  k_collide_sample<T, BATCH><<<blocks, WPB * 32, tile_smem<T>(s.tile), st>>>(
      p, s.cases, ncells, b, start, count, s.sgmax, s.acc, s.comp, s.owner, step, flags, s.tile, s.stats, stg, stc);
}

template <typename T>
void Ops<T>::step_det(const Params<T>& p, State<T>& s, int& cur, int& lay, uint32_t step, int do_sample,
                      cudaStream_t st) {
  const int n = s.nparticles;
  const int ncells = s.ncells;
  const int other = cur ^ 1, olay = lay ^ 1;
  if (n > 0) {
    const int g = grid_for(n, 256);
    if (p.mesh == 1) {
      k_move_det<T, 2, false, true><<<g, 256, 0, st>>>(p, s.cases, s.buf[cur], s.cellof, s.start[lay], n, step,
                                                       s.key, s.tally, s.stats);
    } else if (p.dim == 1) {
      if (s.batch)
        k_move_det<T, 1, true, false><<<g, 256, 0, st>>>(p, s.cases, s.buf[cur], s.cellof, s.start[lay], n, step,
                                                         s.key, s.tally, s.stats);
      else
        k_move_det<T, 1, false, false><<<g, 256, 0, st>>>(p, s.cases, s.buf[cur], s.cellof, s.start[lay], n, step,
                                                          s.key, s.tally, s.stats);
    } else {
      if (s.batch)
        k_move_det<T, 2, true, false><<<g, 256, 0, st>>>(p, s.cases, s.buf[cur], s.cellof, s.start[lay], n, step,
                                                         s.key, s.tally, s.stats);
      else
        k_move_det<T, 2, false, false><<<g, 256, 0, st>>>(p, s.cases, s.buf[cur], s.cellof, s.start[lay], n, step,
                                                          s.key, s.tally, s.stats);
    }
  }
  int ntot = n;
  if (p.mesh == 1) {
    // annulus: freestream entry after the moved particles; the host learns
    // how many slots it used, the sort drops the particles that left
    k_inject_det<T><<<1, 1024, 0, st>>>(s.pinj, s.buf[cur], s.key, n, (long long)s.capacity, step, s.nt, s.tmp2,
                                        s.flags, s.tally, s.stats);
    int32_t add = 0;
    cudaMemcpyAsync(&add, s.tmp2 + p.nx, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    const long long tot = (long long)n + add;
    ntot = (int)(tot < s.capacity ? tot : s.capacity);
    if (tot > s.capacity) s.lost = true;  // entries beyond the workspace were not written
  }
  const PBuf<T>& a = s.buf[cur];
  k_sort_stable<T, T><<<1, 1024, 0, st>>>(a.x, a.y, a.vx, a.vy, a.vz, a.ir, s.buf[other], s.key, ntot, ncells,
                                          s.start[olay], s.count[olay], s.tmp2, s.dest, s.cellof);
  cur = other;
  lay = olay;
  if (p.mesh == 1) {
    int32_t kept = 0;
    cudaMemcpyAsync(&kept, s.start[lay] + ncells, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    s.nparticles = kept;
  }
  const int flags = 1 | (do_sample ? 2 : 0);
  if (s.batch)
    launch_collide_sample<T, true>(p, s, ncells, s.buf[cur], s.start[lay], s.count[lay], step, flags, nullptr,
                                   nullptr, st);
  else
    launch_collide_sample<T, false>(p, s, ncells, s.buf[cur], s.start[lay], s.count[lay], step, flags, nullptr,
                                    nullptr, st);
}

template <typename T>
void Ops<T>::step_bins(const Params<T>& p, State<T>& s, int& cur, int lay, uint32_t step0, int nsteps,
                       int do_sample, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (nsteps <= 0) return;
    const int ncells = s.ncells;
    const int oblocks = 8;
    auto launch = [&](int flags, uint32_t sc, uint32_t sm_step, int F, int ftile) {
      const int other = cur ^ 1;
      const int cblocks = (ncells + F - 1) / F;
      const size_t smf = fused_smem_bytes(ftile, F);
#define DSMC_FUSED_ARGS                                                                                         \
  p, s.cases, ncells, s.buf[cur], s.buf[other], s.start[lay], s.count[cur], s.count[other], s.sgmax, s.acc,      \
      s.comp, s.owner, s.ovf[cur], s.ovf[other], s.ovf_cap, sc, sm_step, flags, ftile, cblocks, s.tally, s.stats, \
      s.flags + 8, s.stg, s.stc
#define DSMC_FUSED_LAUNCH(D, B, W, A) k_fused<D, B, W, A, false><<<cblocks + oblocks, W * 32, smf, st>>>(DSMC_FUSED_ARGS)
#define DSMC_FUSED_LAUNCH_GEN(D, A) k_fused<D, false, 4, A, true><<<cblocks + oblocks, 128, smf, st>>>(DSMC_FUSED_ARGS)
      const bool inject = p.mesh == 1 && (flags & 4);
      if (inject) {
        // annulus: the freestream entry of this step, on the side stream,
        // into the bins the fused step fills (their counts were cleared by
        // the previous launch)
        cudaEventRecord(s.ev_fork, st);
        cudaStreamWaitEvent(s.side, s.ev_fork, 0);
        const int nb = (s.inj_max + 31) / 32;
        k_inject_bins<<<nb > 0 ? nb : 1, 32, sizeof(int32_t) * (p.nx + 1), s.side>>>(
            s.pinj, p, s.inj_mu, s.buf[other], s.start[lay], s.count[other], s.ovf[other], s.ovf_cap, sm_step,
            s.tally, s.stats, s.flags + 8);
        cudaEventRecord(s.ev_join, s.side);
      }
      if (s.gen) {
        // d_r = 3 or VSS: one instantiation per mesh, 4 warps per CTA
        if (p.mesh == 1) DSMC_FUSED_LAUNCH_GEN(2, true);
        else if (p.dim == 1) DSMC_FUSED_LAUNCH_GEN(1, false);
        else DSMC_FUSED_LAUNCH_GEN(2, false);
      } else if (p.mesh == 1) {
        if (F == 2) DSMC_FUSED_LAUNCH(2, false, 2, true);
        else DSMC_FUSED_LAUNCH(2, false, 4, true);
      } else if (F == 2) {
        if (p.dim == 1) {
          if (s.batch) DSMC_FUSED_LAUNCH(1, true, 2, false);
          else DSMC_FUSED_LAUNCH(1, false, 2, false);
        } else {
          if (s.batch) DSMC_FUSED_LAUNCH(2, true, 2, false);
          else DSMC_FUSED_LAUNCH(2, false, 2, false);
        }
      } else {
        if (p.dim == 1) {
          if (s.batch) DSMC_FUSED_LAUNCH(1, true, 4, false);
          else DSMC_FUSED_LAUNCH(1, false, 4, false);
        } else {
          if (s.batch) DSMC_FUSED_LAUNCH(2, true, 4, false);
          else DSMC_FUSED_LAUNCH(2, false, 4, false);
        }
      }
#undef DSMC_FUSED_LAUNCH
#undef DSMC_FUSED_LAUNCH_GEN
#undef DSMC_FUSED_ARGS
      if (inject) cudaStreamWaitEvent(st, s.ev_join, 0);
      // the input overflow list has been consumed
      cudaMemsetAsync(s.ovf[cur].count, 0, sizeof(int32_t), st);
      cur = other;
    };
    // move of step0, then per step: collide (+sample) of step k and move of step k+1
    const int tile0 = s.ftile > 0 ? s.ftile : s.tile;
    launch(4, step0, step0, s.fwpb > 0 ? s.fwpb : FWPB_MAX, tile0);
    // sampled sums are staged in FP32 and folded into FP64 every
    // STAGE_STEPS steps and on the last step of the call
    constexpr int STAGE_STEPS = 16;
    auto fused_flags = [&](int i) {
      const int fold = ((i + 1) % STAGE_STEPS == 0) ? 8 : 0;
      return 1 | (do_sample ? 2 | fold : 0) | 4;
    };
    int i0 = 0;
    if (s.gen) s.fwpb = 4;  // the general gas has the 4-warp shape only
    if (s.fwpb == 0 && nsteps >= 20) {
      // launch shape of the fused step, tuned on real steps of the call:
      // warps (cells) per CTA and the shared-memory tile (particles staged
      // per warp; larger cells go through the chunked path).  Each shape
      // runs one warm-up step and three timed steps; the first shape (4
      // warps, the tile sized from the particles per cell) is kept unless
      // another is faster by more than 1 % (the timing's resolution).
      const int t0 = s.tile;
      const int tlo = t0 - 32 >= 64 ? t0 - 32 : t0, thi = t0 + 32 <= TILE_MAX_OF<T> ? t0 + 32 : t0;
      const int shapes[4][2] = {{4, t0}, {2, t0}, {4, tlo}, {4, thi}};
      cudaEvent_t ev[8];
      for (auto& e : ev) cudaEventCreate(&e);
      int i = 0;
      for (int k = 0; k < 4; ++k) {
        for (int r = 0; r < 4; ++r, ++i) {
          if (r == 1) cudaEventRecord(ev[2 * k], st);
          const uint32_t sc = step0 + (uint32_t)i;
          launch(fused_flags(i), sc, sc + 1, shapes[k][0], shapes[k][1]);
        }
        cudaEventRecord(ev[2 * k + 1], st);
      }
      cudaEventSynchronize(ev[7]);
      float tk[4];
      for (int k = 0; k < 4; ++k) cudaEventElapsedTime(&tk[k], ev[2 * k], ev[2 * k + 1]);
      for (auto& e : ev) cudaEventDestroy(e);
      int best = 0;
      for (int k = 1; k < 4; ++k)
        if (tk[k] > 0.f && tk[k] < 0.99f * tk[best]) best = k;
      s.fwpb = shapes[best][0];
      s.ftile = shapes[best][1];
      i0 = i;
    }
    const int F = s.fwpb > 0 ? s.fwpb : FWPB_MAX;
    const int FT = s.ftile > 0 ? s.ftile : s.tile;
    for (int i = i0; i < nsteps; ++i) {
      const bool last = (i == nsteps - 1);
      const uint32_t sc = step0 + (uint32_t)i;
      if (!last) {
        launch(fused_flags(i), sc, sc + 1, F, FT);
      } else {
        const int flags = 1 | (do_sample ? 2 : 0);
        if (s.batch)
          launch_collide_sample<T, true>(p, s, ncells, s.buf[cur], s.start[lay], s.count[cur], sc, flags, s.stg,
                                         s.stc, st);
        else
          launch_collide_sample<T, false>(p, s, ncells, s.buf[cur], s.start[lay], s.count[cur], sc, flags, s.stg,
                                          s.stc, st);
      }
    }
  } else {
    (void)p; (void)s; (void)cur; (void)lay; (void)step0; (void)nsteps; (void)do_sample; (void)st;
  }
}

template <typename T>
void Ops<T>::rebin(const Params<T>& p, State<T>& s, int& cur, int& lay, int with_ovf, double slack, cudaStream_t st) {
  // tot (tmp in s.nt) = occupancy (+ overflow destinations)
  const int ncells = s.ncells;
  const int other = cur ^ 1, olay = lay ^ 1;
  cudaMemcpyAsync(s.nt, s.count[cur], sizeof(int32_t) * ncells, cudaMemcpyDeviceToDevice, st);
  if constexpr (sizeof(T) == 4) {
    if (with_ovf) k_rebin_add_ovf<<<64, 256, 0, st>>>(s.ovf[cur], s.ovf_cap, s.nt);
  }
  k_caps_scan<<<1, 1024, 0, st>>>(s.nt, ncells, slack, (long long)s.capacity, s.start[olay], s.flags,
                                  s.cases.cp, s.cases.cell_case);
  const int blocks = (ncells + WPB - 1) / WPB;
  if (p.dim == 1)
    k_rebin_copy<T, 1><<<blocks, WPB * 32, 0, st>>>(s.buf[cur], s.buf[other], s.start[lay], s.count[cur],
                                                    s.start[olay], s.count[other], ncells);
  else
    k_rebin_copy<T, 2><<<blocks, WPB * 32, 0, st>>>(s.buf[cur], s.buf[other], s.start[lay], s.count[cur],
                                                    s.start[olay], s.count[other], ncells);
  if constexpr (sizeof(T) == 4) {
    if (with_ovf) {
      if (p.dim == 1)
        k_rebin_ovf<1><<<64, 256, 0, st>>>(s.ovf[cur], s.ovf_cap, s.buf[other], s.start[olay], s.count[other]);
      else
        k_rebin_ovf<2><<<64, 256, 0, st>>>(s.ovf[cur], s.ovf_cap, s.buf[other], s.start[olay], s.count[other]);
      cudaMemsetAsync(s.ovf[cur].count, 0, sizeof(int32_t), st);
    }
  }
  // the old buffer's occupancies are cleared so that it can take appends
  k_zero_i32<<<grid_for(ncells, 256), 256, 0, st>>>(s.count[cur], ncells);
  cur = other;
  lay = olay;
}

template <typename T>
void Ops<T>::export_particles(const Params<T>& p, State<T>& s, int cur, int lay, double* x, double* y, double* vx,
                              double* vy, double* vz, double* ir, int32_t* cell, cudaStream_t st) {
  (void)p;
  const int cntlay = (sizeof(T) == 4) ? cur : lay;
  k_scan_counts<<<1, 1024, 0, st>>>(s.count[cntlay], s.ncells, s.tmp_start);
  const int blocks = (s.ncells + WPB - 1) / WPB;
  k_export<T><<<blocks, WPB * 32, 0, st>>>(s.buf[cur], s.start[lay], s.count[cntlay], s.tmp_start, s.ncells, x, y,
                                          vx, vy, vz, ir, cell);
}

template <typename T>
void Ops<T>::import_particles(const Params<T>& p, State<T>& s, int& cur, int& lay, int64_t n, const double* x,
                              const double* y, const double* vx, const double* vy, const double* vz,
                              const double* ir, int det, cudaStream_t st) {
  const int other = cur ^ 1, olay = lay ^ 1;
  if (n > 0) {
    if (p.mesh == 1)
      k_keys_from_pos<T, 3><<<grid_for(n, 256), 256, 0, st>>>(p, x, y, (int)n, s.key);
    else if (p.dim == 1)
      k_keys_from_pos<T, 1><<<grid_for(n, 256), 256, 0, st>>>(p, x, y, (int)n, s.key);
    else
      k_keys_from_pos<T, 2><<<grid_for(n, 256), 256, 0, st>>>(p, x, y, (int)n, s.key);
  }
  const double* yy = (p.dim == 2) ? y : x;  // y is not read in 1D; pass any valid pointer
  s.nparticles = (int)n;
  if (det) {
    // stable sort of the input into the other buffer: the compact layout
    k_sort_stable<double, T><<<1, 1024, 0, st>>>(x, yy, vx, vy, vz, ir, s.buf[other], s.key, (int)n, p.ncells,
                                                 s.start[olay], s.count[olay], s.tmp2, s.dest, s.cellof);
    cur = other;
    lay = olay;
    if (p.mesh == 1) {
      // particles outside the annulus were dropped
      int32_t kept = 0;
      cudaMemcpyAsync(&kept, s.start[lay] + p.ncells, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      s.nparticles = kept;
    }
    if (p.dim == 1) cudaMemsetAsync(s.buf[cur].y, 0, sizeof(T) * (size_t)n, st);
    return;
  }
  if constexpr (sizeof(T) == 4) {
    // occupancies, bin layout lay, then every particle straight into its bin
    // of buffer cur (all in parallel; no order is kept inside a bin)
    const int g = grid_for(p.ncells, 256);
    k_zero_i32<<<g, 256, 0, st>>>(s.nt, p.ncells);
    if (n > 0) k_count_keys<<<grid_for(n, 256), 256, 0, st>>>(s.key, (int)n, s.nt);
    k_caps_scan<<<1, 1024, 0, st>>>(s.nt, p.ncells, s.slack, (long long)s.capacity, s.start[lay], s.flags);
    k_zero_i32<<<g, 256, 0, st>>>(s.count[cur], p.ncells);
    if (n > 0) {
      if (p.dim == 1)
        k_scatter_bins<1><<<grid_for(n, 256), 256, 0, st>>>(x, yy, vx, vy, vz, ir, s.key, (int)n, s.start[lay],
                                                            s.count[cur], s.buf[cur]);
      else
        k_scatter_bins<2><<<grid_for(n, 256), 256, 0, st>>>(x, yy, vx, vy, vz, ir, s.key, (int)n, s.start[lay],
                                                            s.count[cur], s.buf[cur]);
    }
    k_zero_i32<<<g, 256, 0, st>>>(s.count[other], p.ncells);
    cudaMemsetAsync(s.ovf[0].count, 0, sizeof(int32_t), st);
    cudaMemsetAsync(s.ovf[1].count, 0, sizeof(int32_t), st);
  }
}

template <typename T>
void Ops<T>::dig_counts(State<T>& s, int ncells, int lay, const double* target, uint32_t iter, int det,
                        cudaStream_t st) {
  cudaMemsetAsync(s.flags, 0, sizeof(int32_t) * 8, st);
  // caps go to tmp_start (ncells), then scanned into the other layout's start
  k_dig_counts<<<grid_for(ncells, 256), 256, 0, st>>>(s.cases.cp, s.cases.cell_case, s.cases.cell0, ncells, target,
                                                      iter, det, s.slack, s.nt, s.tmp_start, s.flags);
  k_scan_caps<<<1, 1024, 0, st>>>(s.tmp_start, ncells, (long long)s.capacity, s.start[lay ^ 1], s.flags);
}

template <typename T>
void Ops<T>::dig_apply(const CellParams& cp0, State<T>& s, int ncells, int& cur, int& lay, const double* target,
                       uint32_t iter, int det, cudaStream_t st) {
  const int other = cur ^ 1, olay = lay ^ 1;
  const int cin = det ? lay : cur;    // occupancy array of the current state
  const int cout = det ? olay : other;
  const int blocks = (ncells + WPB - 1) / WPB;
  const size_t sm = (size_t)WPB * s.tile * 2 * sizeof(int32_t);
  if (cp0.dim == 1)
    k_dig_apply<T, 1><<<blocks, WPB * 32, sm, st>>>(s.cases.cp, s.cases.cell_case, s.cases.cell0, ncells, s.buf[cur],
                                                    s.buf[other], s.start[lay], s.count[cin], s.start[olay],
                                                    s.count[cout], s.nt, target, iter, s.scratch_i,
                                                    det ? s.cellof : nullptr, s.tile);
  else
    k_dig_apply<T, 2><<<blocks, WPB * 32, sm, st>>>(s.cases.cp, s.cases.cell_case, s.cases.cell0, ncells, s.buf[cur],
                                                    s.buf[other], s.start[lay], s.count[cin], s.start[olay],
                                                    s.count[cout], s.nt, target, iter, s.scratch_i,
                                                    det ? s.cellof : nullptr, s.tile);
  if (!det) k_zero_i32<<<grid_for(ncells, 256), 256, 0, st>>>(s.count[cur], ncells);
  cur = other;
  lay = olay;
}

template <typename T>
void Ops<T>::total_count(State<T>& s, const int32_t* cnt, int ncells, cudaStream_t st) {
  k_scan_counts<<<1, 1024, 0, st>>>(cnt, ncells, s.tmp_start);
}

template <typename T>
void Ops<T>::configure(int tile) {
  // The limit is an attribute of the kernel, shared by every handle in the
  // process: it is set for the largest tile a handle of this layout can
  // have (only a limit; each launch still asks for its own tile's bytes),
  // so that a later handle with a smaller tile cannot lower it under an
  // earlier one's launches.
  tile = TILE_MAX_OF<T>;
  const int sm = (int)tile_smem<T>(tile);
  const int smd = WPB * tile * 2 * (int)sizeof(int32_t);
  cudaFuncSetAttribute(k_collide_sample<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_collide_sample<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_dig_apply<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smd);
  cudaFuncSetAttribute(k_dig_apply<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smd);
  if constexpr (sizeof(T) == 4) {
    const int sm4 = (int)fused_smem_bytes(tile, 4), sm2 = (int)fused_smem_bytes(tile, 2);
    cudaFuncSetAttribute(k_fused<2, false, 4, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<1, false, 4, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<2, false, 4, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<2, false, 4, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<2, false, 2, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    cudaFuncSetAttribute(k_fused<1, false, 4, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<2, false, 4, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<1, true, 4, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<2, true, 4, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm4);
    cudaFuncSetAttribute(k_fused<1, false, 2, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    cudaFuncSetAttribute(k_fused<2, false, 2, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    cudaFuncSetAttribute(k_fused<1, true, 2, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    cudaFuncSetAttribute(k_fused<2, true, 2, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
  }
}

template <typename T>
void Ops<T>::sgmax_io(State<T>& s, int ncells, double* out, const double* in, cudaStream_t st) {
  k_sgmax_io<T><<<grid_for(ncells, 256), 256, 0, st>>>(s.sgmax, ncells, out, in);
}

}  // namespace dsmc
