// dsmc_mlp.cu -- the HoT surrogate network: input features, forward and
// backward passes with bfloat16 weights and FP32 accumulation, Adam, and the
// HoT it hands to the synthetic equations.  An extension: the paper takes
// the higher-order terms of Eq. (hot_constitutive) from DSMC moments alone.
//
// Forward / backward: a CTA takes tiles of MLP_TILE cells.  The weights
// (bfloat16 in global memory) are widened to FP32 in shared memory once per
// CTA, rows padded by one word so that the threads of a warp, which work on
// consecutive output neurons, read different banks.  A tile's activations of
// all layers stay in shared memory for the backward pass.  Each thread owns
// a fixed set of parameter gradients and sums its products over the tile's
// cells, so the per-CTA sums need no atomics; the CTAs' sums are added in a
// fixed order by a second kernel (the result does not depend on scheduling).
#include <cmath>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dsmc_grad.cuh"
#include "dsmc_internal.h"

namespace dsmc {

namespace {

constexpr int MLP_TILE = 32;
constexpr int MLP_THREADS = 256;
__host__ __device__ constexpr int nin(int k) { return k == 0 ? 12 : 64; }
__host__ __device__ constexpr int nout(int k) { return k == 3 ? 5 : 64; }

// offsets of W_k and b_k in the parameter vector, and of the padded W_k /
// b_k in shared memory
__host__ __device__ constexpr int poff_w(int k) {
  return k == 0 ? 0 : poff_w(k - 1) + nin(k - 1) * nout(k - 1) + nout(k - 1);
}
__host__ __device__ constexpr int poff_b(int k) { return poff_w(k) + nin(k) * nout(k); }
__host__ __device__ constexpr int soff_w(int k) {
  return k == 0 ? 0 : soff_w(k - 1) + (nin(k - 1) + 1) * nout(k - 1) + nout(k - 1);
}
__host__ __device__ constexpr int soff_b(int k) { return soff_w(k) + (nin(k) + 1) * nout(k); }
constexpr int SW_FLOATS = soff_b(3) + nout(3);
static_assert(poff_b(3) + nout(3) == MLP_NPARAM, "parameter count");

// shared memory: padded weights, gradient sums (training), activations
// A0 (TILE x 12), A1..A3 (TILE x 64), output (TILE x 5), two delta buffers
// (TILE x 64), cell weights (TILE)
constexpr int ACT_FLOATS = MLP_TILE * (12 + 3 * 64 + 5 + 2 * 64 + 1);
inline size_t fb_smem_bytes(bool train) {
  return sizeof(float) * ((size_t)SW_FLOATS + (train ? (size_t)MLP_NPARAM : 0) + ACT_FLOATS);
}

__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// per cell: inputs (12), scales (4), normalised HoT targets (5, if hot) and
// weight (1 where mask = 1 and the cell state admits the inputs)
__global__ void k_mlp_data(const CellParams* __restrict__ cps, const int32_t* __restrict__ cell_case,
                           const int32_t* __restrict__ cell0, int ncells, const double* __restrict__ F,
                           const double* __restrict__ hot, const double* __restrict__ kngll,
                           const uint8_t* __restrict__ mask, float* __restrict__ X, float* __restrict__ Y,
                           float* __restrict__ S, float* __restrict__ w, int32_t* __restrict__ count) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    const int cs = cell_case[c];
    const CellParams& cp = cps[cs];
    const int lc = c - cell0[cs];
    const double* f = F + (size_t)c * 18;
    const double rho = f[0], tt = f[4], tr = f[5];
    const double T = (3.0 * tt + cp.d_r * tr) / (3.0 + cp.d_r);
    double x[12], sc[4], y[5];
    bool ok = rho > 0.0 && tt > 0.0 && tr > 0.0 && isfinite(T);
    if (ok) {
      const double mu = cp.mu_ref * pow(T, cp.omega);
      const double lam = mu / (rho * T) * sqrt(M_PI * T / 2.0);
      const double sq = sqrt(T);
      const int cols[5] = {0, 1, 2, 4, 5};
      const double norm[5] = {rho, sq, sq, T, T};
      for (int k = 0; k < 5; ++k) {
        double gx, gy;
        const int col = cols[k];
        grad2(cp, c, lc, [&](int q) { return F[(size_t)q * 18 + col]; }, &gx, &gy);
        x[2 * k] = lam * gx / norm[k];
        x[2 * k + 1] = lam * gy / norm[k];
      }
      x[10] = kngll[c];
      x[11] = tr / tt;
      double gTx, gTy;
      grad2(cp, c, lc,
            [&](int q) {
              const double* g = F + (size_t)q * 18;
              return (3.0 * g[4] + cp.d_r * g[5]) / (3.0 + cp.d_r);
            },
            &gTx, &gTy);
      const double gn = sqrt(gTx * gTx + gTy * gTy);
      const double ex = gn > 0.0 ? gTx / gn : 1.0, ey = gn > 0.0 ? gTy / gn : 0.0;
      const double p = rho * T;
      sc[0] = p;
      sc[1] = p * sq;
      sc[2] = ex;
      sc[3] = ey;
      if (hot) {
        const double* h = hot + (size_t)c * 12;
        y[0] = h[0] / p;
        y[1] = h[3] / p;
        y[2] = h[1] / p;
        y[3] = (h[6] * ex + h[7] * ey) / sc[1];
        y[4] = (h[9] * ex + h[10] * ey) / sc[1];
      } else {
        for (int k = 0; k < 5; ++k) y[k] = 0.0;
      }
      for (int k = 0; k < 12; ++k) ok = ok && isfinite(x[k]);
      for (int k = 0; k < 5; ++k) ok = ok && isfinite(y[k]);
    }
    if (!ok) {
      for (int k = 0; k < 12; ++k) x[k] = 0.0;
      for (int k = 0; k < 5; ++k) y[k] = 0.0;
      sc[0] = sc[1] = 1.0;
      sc[2] = 1.0;
      sc[3] = 0.0;
    }
    for (int k = 0; k < 12; ++k) X[(size_t)c * 12 + k] = (float)x[k];
    for (int k = 0; k < 5; ++k) Y[(size_t)c * 5 + k] = (float)y[k];
    for (int k = 0; k < 4; ++k) S[(size_t)c * 4 + k] = (float)sc[k];
    const bool use = ok && mask[c] != 0;
    w[c] = use ? 1.f : 0.f;
    if (use) atomicAdd(count, 1);
  }
}

template <int L, bool TANH>
__device__ __forceinline__ void layer_fwd(const float* sw, const float* ain, float* aout) {
  constexpr int ni = nin(L), no = nout(L);
  const float* W = sw + soff_w(L);
  const float* b = sw + soff_b(L);
  for (int idx = threadIdx.x; idx < MLP_TILE * no; idx += blockDim.x) {
    const int c = idx / no, j = idx % no;
    const float* wr = W + j * (ni + 1);
    const float* a = ain + c * ni;
    float z = b[j];
#pragma unroll 16
    for (int i = 0; i < ni; ++i) z = fmaf(wr[i], a[i], z);
    aout[idx] = TANH ? tanhf(z) : z;
  }
}

// gradient sums of layer L from its output deltas d (TILE x no) and input
// activations ain (TILE x ni); then, for L > 0, the deltas of the layer below
// (through tanh' = 1 - a^2 of ain) into dnext
template <int L>
__device__ __forceinline__ void layer_bwd(const float* sw, float* g, const float* d, const float* ain,
                                          float* dnext) {
  constexpr int ni = nin(L), no = nout(L);
  float* gW = g + poff_w(L);
  float* gb = g + poff_b(L);
  for (int idx = threadIdx.x; idx < no * ni; idx += blockDim.x) {
    const int j = idx / ni, i = idx % ni;
    float s = 0.f;
#pragma unroll 8
    for (int c = 0; c < MLP_TILE; ++c) s = fmaf(d[c * no + j], ain[c * ni + i], s);
    gW[idx] += s;
  }
  for (int j = threadIdx.x; j < no; j += blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < MLP_TILE; ++c) s += d[c * no + j];
    gb[j] += s;
  }
  if (L > 0) {
    const float* W = sw + soff_w(L);
    for (int idx = threadIdx.x; idx < MLP_TILE * ni; idx += blockDim.x) {
      const int c = idx / ni, i = idx % ni;
      float s = 0.f;
#pragma unroll 8
      for (int j = 0; j < no; ++j) s = fmaf(d[c * no + j], W[j * (ni + 1) + i], s);
      const float a = ain[idx];
      dnext[idx] = s * (1.f - a * a);
    }
  }
}

template <bool TRAIN>
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_fb(const uint16_t* __restrict__ wbf, const float* __restrict__ X,
                                                        const float* __restrict__ Y, const float* __restrict__ wc,
                                                        const int32_t* __restrict__ count, int ncells,
                                                        float* __restrict__ partial, double* __restrict__ part_loss,
                                                        float* __restrict__ out) {
  extern __shared__ __align__(16) float sm[];
  float* sw = sm;
  float* g = sw + SW_FLOATS;
  float* a0 = g + (TRAIN ? MLP_NPARAM : 0);
  float* a1 = a0 + MLP_TILE * 12;
  float* a2 = a1 + MLP_TILE * 64;
  float* a3 = a2 + MLP_TILE * 64;
  float* ao = a3 + MLP_TILE * 64;
  float* d0 = ao + MLP_TILE * 5;
  float* d1 = d0 + MLP_TILE * 64;
  float* wt = d1 + MLP_TILE * 64;
  __shared__ double red[MLP_THREADS];
  // widen the weights into padded rows
  for (int k = 0; k < 4; ++k) {
    const int ni = nin(k), no = nout(k);
    for (int idx = threadIdx.x; idx < no * ni; idx += blockDim.x) {
      const int j = idx / ni, i = idx % ni;
      sw[soff_w(k) + j * (ni + 1) + i] = bf16_to_f(wbf[poff_w(k) + idx]);
    }
    for (int j = threadIdx.x; j < no; j += blockDim.x) sw[soff_b(k) + j] = bf16_to_f(wbf[poff_b(k) + j]);
  }
  if (TRAIN)
    for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x) g[q] = 0.f;
  const float inv_n = TRAIN ? 1.f / (5.f * (float)max(*count, 1)) : 0.f;
  double lsum = 0.0;
  __syncthreads();
  const int ntiles = (ncells + MLP_TILE - 1) / MLP_TILE;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int c0 = t * MLP_TILE;
    for (int idx = threadIdx.x; idx < MLP_TILE * 12; idx += blockDim.x) {
      const int c = c0 + idx / 12;
      a0[idx] = (c < ncells) ? X[(size_t)c0 * 12 + idx] : 0.f;
    }
    for (int c = threadIdx.x; c < MLP_TILE; c += blockDim.x) wt[c] = (c0 + c < ncells) ? wc[c0 + c] : 0.f;
    __syncthreads();
    layer_fwd<0, true>(sw, a0, a1);
    __syncthreads();
    layer_fwd<1, true>(sw, a1, a2);
    __syncthreads();
    layer_fwd<2, true>(sw, a2, a3);
    __syncthreads();
    layer_fwd<3, false>(sw, a3, ao);
    __syncthreads();
    if (!TRAIN) {
      for (int idx = threadIdx.x; idx < MLP_TILE * 5; idx += blockDim.x)
        if (c0 + idx / 5 < ncells) out[(size_t)c0 * 5 + idx] = ao[idx];
    } else {
      // output deltas of the mean squared error over the weighted cells
      for (int idx = threadIdx.x; idx < MLP_TILE * 5; idx += blockDim.x) {
        const int c = idx / 5;
        const float y = (c0 + c < ncells) ? Y[(size_t)c0 * 5 + idx] : 0.f;
        const float r = (ao[idx] - y) * wt[c];
        lsum += (double)r * (double)r;
        d0[idx] = 2.f * r * inv_n;
      }
      __syncthreads();
      layer_bwd<3>(sw, g, d0, a3, d1);
      __syncthreads();
      layer_bwd<2>(sw, g, d1, a2, d0);
      __syncthreads();
      layer_bwd<1>(sw, g, d0, a1, d1);
      __syncthreads();
      layer_bwd<0>(sw, g, d1, a0, nullptr);
    }
    __syncthreads();
  }
  if (TRAIN) {
    for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x) partial[(size_t)blockIdx.x * MLP_NPARAM + q] = g[q];
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part_loss[blockIdx.x] = red[0];
  }
}

// the CTAs' gradient sums in block order; the loss
__global__ void k_mlp_reduce(const float* __restrict__ partial, const double* __restrict__ part_loss, int nblk,
                             const int32_t* __restrict__ count, float* __restrict__ grad, double* __restrict__ scal) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < MLP_NPARAM) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * MLP_NPARAM + q];
    grad[q] = s;
  }
  if (q == 0) {
    double l = 0.0;
    for (int b = 0; b < nblk; ++b) l += part_loss[b];
    scal[0] = l / (5.0 * (double)max(*count, 1));
  }
}

__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, uint16_t* __restrict__ wbf, float c1, float c2, float lr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= MLP_NPARAM) return;
  const float gq = grad[q];
  const float mq = 0.9f * m[q] + 0.1f * gq;
  const float vq = 0.999f * v[q] + 0.001f * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float th = theta[q] - lr * (mq / c1) / (sqrtf(vq / c2) + 1e-8f);
  theta[q] = th;
  wbf[q] = __bfloat16_as_ushort(__float2bfloat16_rn(th));
}

__global__ void k_mlp_bf16(const float* __restrict__ theta, uint16_t* __restrict__ wbf) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < MLP_NPARAM) wbf[q] = __bfloat16_as_ushort(__float2bfloat16_rn(theta[q]));
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores: every layer is one product of the tile's
// activations (16 cells x K, bfloat16) with the layer's weights (K x N,
// bfloat16) accumulated in FP32 by mma.sync m16n8k16; bias and tanh in FP32,
// and the result, rounded to bfloat16, is already laid out as the next
// layer's A operand (the accumulator fragment of two adjacent 8-column tiles
// is the operand fragment of one 16-column k-slice).  A warp takes 16 cells
// at a time; the CTA's warps share the weights, staged in shared memory in
// rows padded so that the fragment loads of a warp hit 32 distinct banks.
// ---------------------------------------------------------------------------
constexpr int TC_WARPS = 4;
constexpr int TC_K0 = 16;        // the 12 inputs padded to one k-slice
constexpr int TC_LD0 = 12;       // words per row of the padded layer-0 weights (8 used)
constexpr int TC_LD = 36;        // words per row of the 64-input weights (32 used)
constexpr int TC_W0 = 64 * TC_LD0, TC_W1 = 64 * TC_LD, TC_W3 = 8 * TC_LD;
constexpr int TC_WORDS = TC_W0 + 2 * TC_W1 + TC_W3;        // bfloat16 pairs
constexpr int TC_BIAS = 64 * 3 + 8;                         // FP32 biases
inline size_t tc_smem_bytes() { return sizeof(uint32_t) * (size_t)TC_WORDS + sizeof(float) * TC_BIAS; }

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One layer for the warp's 16 cells: a[KT][4] operand fragments (KT
// k-slices of 16 inputs) times the NT 8-column tiles of the weights W
// (rows of ld words, row n = output n), plus bias; d[NT][4] accumulators.
template <int KT, int NT>
__device__ __forceinline__ void tc_layer(const uint32_t (*a)[4], const uint32_t* W, int ld, const float* bias,
                                         float (*d)[4], int g, int t) {
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
    d[j][0] = b0;
    d[j][1] = b1;
    d[j][2] = b0;
    d[j][3] = b1;
    const uint32_t* wr = W + (8 * j + g) * ld;
#pragma unroll
    for (int k = 0; k < KT; ++k) mma16816(d[j], a[k], wr[8 * k + t], wr[8 * k + 4 + t]);
  }
}

// tanh of the accumulators of 2 KT tiles, packed as KT operand fragments
template <int KT>
__device__ __forceinline__ void tc_to_operand(float (*d)[4], uint32_t (*a)[4]) {
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    a[k][0] = bf16x2(tanhf(d[2 * k][0]), tanhf(d[2 * k][1]));
    a[k][1] = bf16x2(tanhf(d[2 * k][2]), tanhf(d[2 * k][3]));
    a[k][2] = bf16x2(tanhf(d[2 * k + 1][0]), tanhf(d[2 * k + 1][1]));
    a[k][3] = bf16x2(tanhf(d[2 * k + 1][2]), tanhf(d[2 * k + 1][3]));
  }
}

__global__ void __launch_bounds__(TC_WARPS * 32) k_mlp_fwd_tc(const uint16_t* __restrict__ wbf,
                                                              const float* __restrict__ theta,
                                                              const float* __restrict__ X, int ncells,
                                                              float* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t smw[];
  uint32_t* W0 = smw;
  uint32_t* W1 = W0 + TC_W0;
  uint32_t* W2 = W1 + TC_W1;
  uint32_t* W3 = W2 + TC_W1;
  float* bs = reinterpret_cast<float*>(W3 + TC_W3);
  // stage the bfloat16 weights as pairs along the input index (zero padded)
  auto pair = [&](int k, int n, int i) -> uint32_t {  // inputs i, i + 1 of output n of layer k
    const int ni = nin(k);
    if (n >= nout(k) || i >= ni) return 0u;
    const uint32_t lo = wbf[poff_w(k) + n * ni + i];
    const uint32_t hi = (i + 1 < ni) ? wbf[poff_w(k) + n * ni + i + 1] : 0u;
    return lo | (hi << 16);
  };
  for (int q = threadIdx.x; q < 64 * TC_LD0; q += blockDim.x) {
    const int n = q / TC_LD0, w = q % TC_LD0;
    W0[q] = (w < TC_K0 / 2) ? pair(0, n, 2 * w) : 0u;
  }
  for (int q = threadIdx.x; q < 64 * TC_LD; q += blockDim.x) {
    const int n = q / TC_LD, w = q % TC_LD;
    W1[q] = (w < 32) ? pair(1, n, 2 * w) : 0u;
    W2[q] = (w < 32) ? pair(2, n, 2 * w) : 0u;
  }
  for (int q = threadIdx.x; q < 8 * TC_LD; q += blockDim.x) {
    const int n = q / TC_LD, w = q % TC_LD;
    W3[q] = (w < 32) ? pair(3, n, 2 * w) : 0u;
  }
  for (int q = threadIdx.x; q < TC_BIAS; q += blockDim.x) {
    const int k = q / 64, j = q % 64;
    bs[q] = (k < 3) ? theta[poff_b(k) + j] : (j < 5 ? theta[poff_b(3) + j] : 0.f);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int ntiles = (ncells + 15) / 16;
  for (int tile = blockIdx.x * TC_WARPS + warp; tile < ntiles; tile += gridDim.x * TC_WARPS) {
    const int c0 = tile * 16;
    const int ca = c0 + g, cb = c0 + g + 8;
    auto xin = [&](int c, int i) { return (c < ncells && i < 12) ? X[(size_t)c * 12 + i] : 0.f; };
    uint32_t a0[1][4];
    a0[0][0] = bf16x2(xin(ca, 2 * t), xin(ca, 2 * t + 1));
    a0[0][1] = bf16x2(xin(cb, 2 * t), xin(cb, 2 * t + 1));
    a0[0][2] = bf16x2(xin(ca, 2 * t + 8), xin(ca, 2 * t + 9));
    a0[0][3] = bf16x2(xin(cb, 2 * t + 8), xin(cb, 2 * t + 9));
    float d[8][4];
    uint32_t a[4][4];
    tc_layer<1, 8>(a0, W0, TC_LD0, bs, d, g, t);
    tc_to_operand<4>(d, a);
    tc_layer<4, 8>(a, W1, TC_LD, bs + 64, d, g, t);
    tc_to_operand<4>(d, a);
    tc_layer<4, 8>(a, W2, TC_LD, bs + 128, d, g, t);
    tc_to_operand<4>(d, a);
    float o[1][4];
    tc_layer<4, 1>(a, W3, TC_LD, bs + 192, o, g, t);
    // row g: outputs 2t, 2t + 1 in o[0][0..1]; row g + 8 in o[0][2..3]
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = h ? cb : ca;
      if (c >= ncells) continue;
      if (2 * t < 5) out[(size_t)c * 5 + 2 * t] = o[0][2 * h];
      if (2 * t + 1 < 5) out[(size_t)c * 5 + 2 * t + 1] = o[0][2 * h + 1];
    }
  }
}

// The judge's statistics: every cell of the network (w = 1, finite
// outputs) adds its residual r = network - DSMC (5 normalised outputs), r^2
// and the DSMC terms Y to its group's sums, and 1 to its count (FP64):
// JACC doubles per group.
constexpr int JACC = 16;
__global__ void k_mlp_judge_acc(int ncells, const float* __restrict__ out, const float* __restrict__ Y,
                                const float* __restrict__ w, const int32_t* __restrict__ group,
                                double* __restrict__ jacc) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    const float* o = out + (size_t)c * 5;
    bool fin = true;
    for (int k = 0; k < 5; ++k) fin = fin && isfinite(o[k]);
    if (w[c] == 0.f || !fin) continue;
    double* a = jacc + (size_t)(group ? group[c] : c) * JACC;
    for (int k = 0; k < 5; ++k) {
      const double y = (double)Y[(size_t)c * 5 + k];
      const double r = (double)o[k] - y;
      atomicAdd(a + k, r);
      atomicAdd(a + 5 + k, r * r);
      atomicAdd(a + 11 + k, y);
    }
    atomicAdd(a + 10, 1.0);
  }
}

// true if the group's residuals show the network's bias to be small: at
// least min_samples of them and, for every output, |mean r| + z SE(r) <=
// rel |mean Y| (an equivalence test: the bias is bounded, with z standard
// errors of confidence, by the fraction rel of the DSMC terms themselves)
__device__ __forceinline__ bool judge_pass(const double* a, double z, int min_samples, double rel) {
  const double n = a[10];
  if (n < (double)min_samples) return false;
  for (int k = 0; k < 5; ++k) {
    const double m = a[k] / n;
    const double var = fmax(a[5 + k] / n - m * m, 0.0) * n / (n - 1.0);
    if (fabs(m) + z * sqrt(var / n) > rel * fabs(a[11 + k] / n)) return false;
  }
  return true;
}

// HoT for the synthetic equations and the judge sums (network against DSMC);
// hot and hot_out may be the same array (each thread reads its cell first).
// With z > 0 a network cell keeps the DSMC HoT unless its group passes the
// judge (judge_pass).
__global__ void k_mlp_hot(int ncells, const float* __restrict__ out, const float* __restrict__ Y,
                          const float* __restrict__ S, const float* __restrict__ w, const double* hot,
                          double* hot_out, double* __restrict__ scal, const int32_t* __restrict__ group,
                          const double* __restrict__ jacc, double z, int min_samples, double rel) {
  double jsum = 0.0, jcnt = 0.0, nnet = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    double h[12];
    for (int k = 0; k < 12; ++k) h[k] = hot[(size_t)c * 12 + k];
    const float* o = out + (size_t)c * 5;
    bool fin = true;
    for (int k = 0; k < 5; ++k) fin = fin && isfinite(o[k]);
    const bool judged = z > 0.0 && w[c] != 0.f && fin;
    const bool pass = !judged || judge_pass(jacc + (size_t)(group ? group[c] : c) * JACC, z, min_samples, rel);
    if (w[c] != 0.f && fin) {
      for (int k = 0; k < 5; ++k) {
        const double r = (double)o[k] - (double)Y[(size_t)c * 5 + k];
        jsum += r * r;
      }
      jcnt += 5.0;
    }
    if (w[c] != 0.f && fin && pass) {
      nnet += 1.0;
      const double p = S[(size_t)c * 4], ps = S[(size_t)c * 4 + 1];
      const double ex = S[(size_t)c * 4 + 2], ey = S[(size_t)c * 4 + 3];
      h[0] = (double)o[0] * p;
      h[3] = (double)o[1] * p;
      h[1] = (double)o[2] * p;
      const int base[2] = {6, 9};
      for (int r = 0; r < 2; ++r) {
        const double along = h[base[r]] * ex + h[base[r] + 1] * ey;
        const double nw = (double)o[3 + r] * ps;
        h[base[r]] += (nw - along) * ex;
        h[base[r] + 1] += (nw - along) * ey;
      }
    }
    for (int k = 0; k < 12; ++k) hot_out[(size_t)c * 12 + k] = h[k];
  }
  if (jcnt > 0.0) {
    atomicAdd(scal + 2, jsum);
    atomicAdd(scal + 3, jcnt);
  }
  if (nnet > 0.0) atomicAdd(scal + 4, nnet);
}

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

void configure_fb() {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_mlp_fb<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_bytes(true));
    cudaFuncSetAttribute(k_mlp_fb<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_bytes(false));
    configured = true;
  }
}

}  // namespace

void mlp_prepare(const Mlp& m, const CellParams* cp, const int32_t* cell_case, const int32_t* cell0, int ncells,
                 const double* fields, const double* hot, const double* kngll, const uint8_t* mask,
                 cudaStream_t st) {
  cudaMemsetAsync(m.count, 0, sizeof(int32_t), st);
  k_mlp_data<<<blocks_for(ncells, 256), 256, 0, st>>>(cp, cell_case, cell0, ncells, fields, hot, kngll, mask, m.X,
                                                       m.Y, m.S, m.w, m.count);
}

void mlp_grad(const Mlp& m, int ncells, cudaStream_t st) {
  configure_fb();
  const int ntiles = blocks_for(ncells, MLP_TILE);
  const int grid = ntiles < MLP_GRID ? ntiles : MLP_GRID;
  k_mlp_fb<true><<<grid, MLP_THREADS, fb_smem_bytes(true), st>>>(m.wbf, m.X, m.Y, m.w, m.count, ncells, m.partial,
                                                                  m.part_loss, m.out);
  k_mlp_reduce<<<blocks_for(MLP_NPARAM, 256), 256, 0, st>>>(m.partial, m.part_loss, grid, m.count, m.grad, m.scal);
}

void mlp_adam(const Mlp& m, int t, double lr, cudaStream_t st) {
  const float c1 = (float)(1.0 - pow(0.9, t)), c2 = (float)(1.0 - pow(0.999, t));
  k_mlp_adam<<<blocks_for(MLP_NPARAM, 256), 256, 0, st>>>(m.theta, m.m, m.v, m.grad, m.wbf, c1, c2, (float)lr);
}

void mlp_to_bf16(const Mlp& m, cudaStream_t st) {
  k_mlp_bf16<<<blocks_for(MLP_NPARAM, 256), 256, 0, st>>>(m.theta, m.wbf);
}

void mlp_apply(const Mlp& m, int ncells, const double* hot, double* hot_out, cudaStream_t st,
               const int32_t* group, double z, int min_samples, double rel) {
  // inference on the tensor cores (bfloat16 weights and activations, FP32 sums)
  const int tiles = blocks_for(ncells, 16);
  const int grid = blocks_for(tiles, TC_WARPS) < MLP_GRID ? blocks_for(tiles, TC_WARPS) : MLP_GRID;
  k_mlp_fwd_tc<<<grid, TC_WARPS * 32, tc_smem_bytes(), st>>>(m.wbf, m.theta, m.X, ncells, m.out);
  cudaMemsetAsync(m.scal + 2, 0, 3 * sizeof(double), st);
  const int hb = blocks_for(ncells, 256) < 1024 ? blocks_for(ncells, 256) : 1024;
  if (z > 0.0) k_mlp_judge_acc<<<hb, 256, 0, st>>>(ncells, m.out, m.Y, m.w, group, m.jacc);
  k_mlp_hot<<<hb, 256, 0, st>>>(ncells, m.out, m.Y, m.S, m.w, hot, hot_out, m.scal, group, m.jacc, z, min_samples,
                                rel);
}

}  // namespace dsmc
