// dsmc_device.cuh -- device building blocks of the DSMC step (sm_103a).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
// the 64-bit seed, counter = (c0, c1, c2, tag << 24 | block).  A stream is a
// (tag, c0, c1, c2) tuple; its uniform number j lives in block j / P, where
// P = 2 in FP64 (two words per uniform: the top 52 bits of (w_hi, w_lo),
// u = (m + 1/2) 2^-52) and P = 4 in FP32 (u = (w >> 9 + 1/2) 2^-23).  Both
// lie strictly inside (0, 1).  Streams used by the step:
//   TAG_INIT  (k, cell, 0)      initial particle k of a cell
//   TAG_WALL  (k, cell, step)   wall hits of the k-th particle of a cell
//   TAG_NTC   (0, cell, step)   Iround of the candidate-pair count
//   TAG_COLL  (m, cell, step)   candidate pair m of a cell
//   TAG_DIG_* (q, cell, iter)   particle modification, always FP64 layout
//   TAG_INJ   (q, face, step)   freestream entry through outer face `face` of
//                               the annulus, always FP64; (~0, face, step)
//                               draws the face's count
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dsmc {

constexpr uint32_t TAG_INIT = 1u, TAG_WALL = 2u, TAG_NTC = 3u, TAG_COLL = 4u;
constexpr uint32_t TAG_DIG_N = 5u, TAG_DIG_SEL = 6u, TAG_DIG_POS = 7u, TAG_INJ = 8u;
constexpr int MAX_HITS = 8;
constexpr int NMOM = 17;
constexpr uint32_t OWNER_FREE = 0xFFFFFFFFu;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr double PI_D = 3.141592653589793;

// Simulation constants in the particle precision T.
template <typename T>
struct Params {
  int dim, nx, ny, ncells;
  T lx, ly, dx, dy, sx, sy;  // sx = nx / lx, sy = ny / ly
  T vcell, fnum, dt;
  T c_sigma, p_inel, vhs_e, bl_exp;  // vhs_e = 2 - 2 omega, bl_exp = 1/(5/2 - omega)
  // rotational degrees of freedom: d_r3 = 0 for d_r = 2, 1 for d_r = 3; the
  // Borgnakke-Larsen partition Beta(a, b), a = d_r/2, b = 5/2 - omega, for
  // d_r = 3 by acceptance-rejection: bl_am1 = a - 1, bl_bm1 = b - 1 and its
  // mode bl_xs = (a - 1)/(a + b - 2)
  int d_r3;
  T bl_am1, bl_bm1, bl_xs;
  // VSS scattering (vss = 1 for alpha != 1): cos chi = 2 u^{vss_ia} - 1, vss_ia = 1/alpha
  int vss;
  T vss_ia;
  int collisions;
  int wall_kind[4];
  T wall_t[4];
  T wall_u[4][3];
  uint32_t k0, k1;
  int ppc;                           // initial particles per cell
  T init_tt, init_tr, init_u[3];     // initial equilibrium state
  T init_rho;
  // mesh 1: annulus r_in <= r <= r_out around a cylinder (Sec. 4.2), nx
  // angular x ny radial cells, cell = j nx + k; wall 0 is the cylinder
  int mesh;
  const T* r2t;   // ny + 1 squared ring radii
  const T* ray;   // nx + 1 rays (cos, sin) at 2 pi k / nx; ray nx = ray 0
  const T* fnrm;  // nx outer-face centre directions (cos, sin)
  const T* vol;   // cell volumes (null on the box: vcell)
  // mesh 2: the wall-refined box, nx + 1 and ny + 1 cell edges
  const T* xe;
  const T* ye;
  T r_in, r_out;
  T fs_rho, fs_t, fs_u[3];  // freestream entering through the outer circle
};

// Per-step device counters (unsigned long long so they can be added atomically).
enum StatSlot {
  ST_CAND = 0, ST_COLL = 1, ST_CLIP = 2, ST_INEL = 3, ST_HITS = 4, ST_MAXHIT = 5, ST_OVF = 6,
  ST_REBIN = 7, ST_NEARFULL = 8, ST_OUT = 9, ST_INJ = 10, ST_NSLOTS = 16
};

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ double u01_from_words(uint32_t hi, uint32_t lo) {
  const unsigned long long m = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
  return ((double)m + 0.5) * 0x1p-52;
}

__device__ __forceinline__ float u01_from_word(uint32_t w) {
  return ((float)(w >> 9) + 0.5f) * 0x1p-23f;
}

template <typename T>
struct Stream;

template <>
struct Stream<double> {
  uint32_t c0, c1, c2, tag, k0, k1;
  int blk;
  uint4 w;
  __device__ Stream(uint32_t tag_, uint32_t c0_, uint32_t c1_, uint32_t c2_, uint32_t k0_, uint32_t k1_)
      : c0(c0_), c1(c1_), c2(c2_), tag(tag_ << 24), k0(k0_), k1(k1_), blk(-1) {}
  __device__ __forceinline__ double u(uint32_t j) {
    const uint32_t b = j >> 1;
    if ((int)b != blk) {
      w = philox4x32_10(c0, c1, c2, tag | b, k0, k1);
      blk = (int)b;
    }
    return (j & 1u) ? u01_from_words(w.z, w.w) : u01_from_words(w.x, w.y);
  }
};

template <>
struct Stream<float> {
  uint32_t c0, c1, c2, tag, k0, k1;
  int blk;
  uint4 w;
  __device__ Stream(uint32_t tag_, uint32_t c0_, uint32_t c1_, uint32_t c2_, uint32_t k0_, uint32_t k1_)
      : c0(c0_), c1(c1_), c2(c2_), tag(tag_ << 24), k0(k0_), k1(k1_), blk(-1) {}
  __device__ __forceinline__ float u(uint32_t j) {
    const uint32_t b = j >> 2;
    if ((int)b != blk) {
      w = philox4x32_10(c0, c1, c2, tag | b, k0, k1);
      blk = (int)b;
    }
    const uint32_t s = j & 3u;
    const uint32_t word = s == 0 ? w.x : (s == 1 ? w.y : (s == 2 ? w.z : w.w));
    return u01_from_word(word);
  }
};

// Uniforms j0 .. j0+3 of a stream (j0 a multiple of 4): one Philox block in
// FP32, two in FP64.
__device__ __forceinline__ void draw4(uint32_t tag, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t j0,
                                      uint32_t k0, uint32_t k1, float* u) {
  const uint4 w = philox4x32_10(c0, c1, c2, (tag << 24) | (j0 >> 2), k0, k1);
  u[0] = u01_from_word(w.x);
  u[1] = u01_from_word(w.y);
  u[2] = u01_from_word(w.z);
  u[3] = u01_from_word(w.w);
}

__device__ __forceinline__ void draw4(uint32_t tag, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t j0,
                                      uint32_t k0, uint32_t k1, double* u) {
  const uint4 a = philox4x32_10(c0, c1, c2, (tag << 24) | (j0 >> 1), k0, k1);
  const uint4 b = philox4x32_10(c0, c1, c2, (tag << 24) | ((j0 >> 1) + 1), k0, k1);
  u[0] = u01_from_words(a.x, a.y);
  u[1] = u01_from_words(a.z, a.w);
  u[2] = u01_from_words(b.x, b.y);
  u[3] = u01_from_words(b.z, b.w);
}

// Post-collision uniforms u4 .. u8 of candidate stream (m, cell, step).  FP64:
// uniforms 4..8 of the stream (blocks 2, 3, 4).  FP32: one block gives
// u4..u7 from the top 23 bits of its four words and u8 from 23 of the 36
// unused low bits (9 of word 0, 9 of word 1, 5 of word 2).
__device__ __forceinline__ uint4 post_block(uint32_t m, uint32_t cell, uint32_t step, uint32_t k0, uint32_t k1) {
  return philox4x32_10(m, cell, step, (4u << 24) | 1u, k0, k1);
}

__device__ __forceinline__ void post_from_block(const uint4& w, float* u) {
  u[0] = u01_from_word(w.x);
  u[1] = u01_from_word(w.y);
  u[2] = u01_from_word(w.z);
  u[3] = u01_from_word(w.w);
  const uint32_t m8 = ((w.x & 0x1FFu) << 14) | ((w.y & 0x1FFu) << 5) | (w.z & 0x1Fu);
  u[4] = ((float)m8 + 0.5f) * 0x1p-23f;
}

__device__ __forceinline__ void draw_post(uint32_t m, uint32_t cell, uint32_t step, uint32_t k0, uint32_t k1,
                                          float* u) {
  post_from_block(post_block(m, cell, step, k0, k1), u);
}

__device__ __forceinline__ void draw_post(uint32_t m, uint32_t cell, uint32_t step, uint32_t k0, uint32_t k1,
                                          double* u) {
  Stream<double> st(4u, m, cell, step, k0, k1);
  for (int j = 0; j < 5; ++j) u[j] = st.u(4 + j);
}

// ---------------------------------------------------------------------------
// Precision-dispatched math.  FP64 calls the CUDA double functions (the
// oracle calls the C library ones; both are within a few ulp).  FP32 uses the
// hardware approximations where the error is far below the statistical noise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return __logf(x); }
__device__ __forceinline__ double m_pow(double x, double e) { return pow(x, e); }
__device__ __forceinline__ float m_pow(float x, float e) {
  // x >= 0; exp2(e log2 x) with log2(0) = -inf giving 0 for e > 0
  return exp2f(e * __log2f(x));
}
__device__ __forceinline__ void m_sincos_2pi(double u, double* s, double* c) {
  const double th = 2.0 * PI_D * u;
  *c = cos(th);
  *s = sin(th);
}
__device__ __forceinline__ void m_sincos_2pi(float u, float* s, float* c) {
  sincospif(2.0f * u, s, c);
}
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ double m_sin(double x) { return sin(x); }
__device__ __forceinline__ float m_sin(float x) { return sinf(x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }

// Indices of the extra uniforms that only d_r = 3 draws (rot_energy) and the
// Borgnakke-Larsen acceptance-rejection (bl_fraction) take from a stream:
// 1024-1025 for the I_r of a particle's own stream, 1026 + jh/2 and 1027 +
// jh/2 for a wall hit whose four uniforms start at jh, 2048 + 4t .. 2051 + 4t
// for try t of a candidate pair (2048 + 4t, +1: particle i; +2, +3: j).
constexpr uint32_t JX_OWN = 1024u, JX_BL = 2048u;
constexpr int BL_TRIES = 32;
__host__ __device__ __forceinline__ uint32_t jx_hit(uint32_t jh) { return 1026u + jh / 2u; }

template <typename T>
__device__ __forceinline__ void box_muller(T ua, T ub, T* n1, T* n2) {
  const T r = m_sqrt(T(-2) * m_log(ua));
  T s, c;
  m_sincos_2pi(ub, &s, &c);
  *n1 = r * c;
  *n2 = r * s;
}

// Rotational energy of one molecule in equilibrium at temperature tq (Sec.
// 2.1, e_r = d_r T_r / 2): I_r / tq is Gamma(d_r / 2).  d_r = 2: -tq ln u
// with u the draw's main uniform; d_r = 3: Gamma(1) + Gamma(1/2), the second
// as Z^2 / 2 of a Box-Muller normal, -ln(u_a) cos^2(2 pi u_b), with u_a, u_b
// the uniforms jx, jx + 1 of stream st.
// (The d_r = 3 and VSS parts are compiled only where the GEN template switch
// of the caller asks for them, so that the fused step of an N2-like gas keeps
// its registers.)
template <typename T, typename S>
__device__ __forceinline__ T gamma_half_part(S& st, uint32_t jx) {
  T sb, cb;
  m_sincos_2pi(st.u(jx + 1u), &sb, &cb);
  return -m_log(st.u(jx)) * cb * cb;
}

template <typename T, typename S>
__device__ __forceinline__ T rot_energy(bool d_r3, T tq, T u, S& st, uint32_t jx) {
  T e = -m_log(u);
  if (d_r3) e += gamma_half_part<T>(st, jx);
  return tq * e;
}

// Fraction x = I_r,k' / E_c kept as rotational energy in one
// Borgnakke-Larsen exchange (Sec. 2.2): x ~ Beta(d_r/2, 5/2 - omega).  d_r
// = 2: the inverse CDF 1 - u^{1/(5/2 - omega)} at the main uniform u.  d_r =
// 3: acceptance-rejection under the uniform envelope of x^{a-1} (1-x)^{b-1}
// (maximum at its mode x*): try t proposes x (u at t = 0, else uniform jx +
// 4t) and accepts it when ln(uniform jx + 4t + 1) < (a-1) ln(x/x*) + (b-1)
// ln((1-x)/(1-x*)); after BL_TRIES rejections (odds below 1e-18) x = x*.
template <typename T>
__device__ __forceinline__ T bl_fraction_ar(const Params<T>& p, T u, uint32_t k, uint32_t cell, uint32_t step,
                                         uint32_t jx) {
  Stream<T> st(4u, k, cell, step, p.k0, p.k1);  // the candidate's stream (TAG_COLL)
  const T xs = p.bl_xs;
  for (int t = 0; t < BL_TRIES; ++t) {
    const T x = (t == 0) ? u : st.u(jx + 4u * (uint32_t)t);
    const T acc = st.u(jx + 4u * (uint32_t)t + 1u);
    if (m_log(acc) < p.bl_am1 * m_log(x / xs) + p.bl_bm1 * m_log((T(1) - x) / (T(1) - xs))) return x;
  }
  return xs;
}

template <typename T, bool GEN>
__device__ __forceinline__ T bl_fraction(const Params<T>& p, T u, uint32_t k, uint32_t cell, uint32_t step,
                                         uint32_t jx) {
  if (!GEN || !p.d_r3) return T(1) - m_pow(u, p.bl_exp);
  return bl_fraction_ar(p, u, k, cell, step, jx);
}

// Half the post-collision relative velocity, h = g'/2, |g'| = gn.  VHS
// (alpha = 1): isotropic, cos(theta) = 2 u - 1 and azimuth 2 pi v in the lab
// frame.  VSS (Sec. 2.2): deflection chi from the pre-collision direction e
// = g/|g| with cos(chi) = 2 u^{1/alpha} - 1, azimuth 2 pi v about e measured
// from e1, the coordinate axis least aligned with e made orthogonal to e (e2
// = e x e1).
template <typename T>
__device__ __forceinline__ void scatter_vss(const Params<T>& p, T gx, T gy, T gz, T gn, T u, T v, T* h) {
  T sph, cph;
  m_sincos_2pi(v, &sph, &cph);
  const T g = m_sqrt(gx * gx + gy * gy + gz * gz);
  const T e[3] = {gx / g, gy / g, gz / g};
  const T m0 = e[0] < T(0) ? -e[0] : e[0], m1 = e[1] < T(0) ? -e[1] : e[1], m2 = e[2] < T(0) ? -e[2] : e[2];
  const int ax = (m0 <= m1 && m0 <= m2) ? 0 : (m1 <= m2 ? 1 : 2);
  const T d = e[ax];
  T e1[3];
  for (int k = 0; k < 3; ++k) e1[k] = ((k == ax) ? T(1) : T(0)) - d * e[k];
  const T l1 = m_sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int k = 0; k < 3; ++k) e1[k] = e1[k] / l1;
  const T e2[3] = {e[1] * e1[2] - e[2] * e1[1], e[2] * e1[0] - e[0] * e1[2], e[0] * e1[1] - e[1] * e1[0]};
  const T cch = T(2) * m_pow(u, p.vss_ia) - T(1);
  const T sch = m_sqrt(T(1) - cch * cch);
  for (int k = 0; k < 3; ++k) h[k] = T(0.5) * gn * (cch * e[k] + sch * (cph * e1[k] + sph * e2[k]));
}

template <typename T, bool GEN>
__device__ __forceinline__ void scatter(const Params<T>& p, T gx, T gy, T gz, T gn, T u, T v, T* h) {
  if (GEN && p.vss) {
    scatter_vss(p, gx, gy, gz, gn, u, v, h);
    return;
  }
  T sph, cph;
  m_sincos_2pi(v, &sph, &cph);
  const T cth = T(2) * u - T(1);
  const T sth = m_sqrt(T(1) - cth * cth);
  h[0] = T(0.5) * gn * cth;
  h[1] = T(0.5) * gn * sth * cph;
  h[2] = T(0.5) * gn * sth * sph;
}

// Iround of Sec. 3.2 step i: floor(x) + 1 with probability x - floor(x).
template <typename T>
__device__ __forceinline__ long long iround(T x, T u) {
  const T f = m_floor(x);
  return (long long)f + ((u < x - f) ? 1 : 0);
}

// the largest i with e[i] <= v, clamped to [0, n - 1]
template <typename T>
__device__ __forceinline__ int edge_index(const T* e, int n, T v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (e[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, int DIM>
__device__ __forceinline__ int cell_of(const Params<T>& p, T x, T y) {
  if (DIM == 2 && p.mesh == 2) return edge_index(p.ye, p.ny, y) * p.nx + edge_index(p.xe, p.nx, x);
  int ix = (int)(x * p.sx);
  ix = ix < 0 ? 0 : (ix > p.nx - 1 ? p.nx - 1 : ix);
  if (DIM == 1) return ix;
  int iy = (int)(y * p.sy);
  iy = iy < 0 ? 0 : (iy > p.ny - 1 ? p.ny - 1 : iy);
  return iy * p.nx + ix;
}

// Annulus cell of (x, y), -1 at or beyond r_out (the particle has left).
// Ring j is the largest with R_j^2 <= r^2 (ring 0 below r_in, where rounding
// can put a particle); sector k holds the points with cross(ray_k, p) >= 0 >
// cross(ray_{k+1}, p), reached from the atan2 guess by those two signs.
template <typename T>
__device__ __forceinline__ int cell_of_ann(const Params<T>& p, T x, T y) {
  const int nr = p.ny, nt = p.nx;
  const T r2 = x * x + y * y;
  if (!(r2 < p.r2t[nr])) return -1;
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.r2t[mid] <= r2) lo = mid;
    else hi = mid - 1;
  }
  T th = m_atan2(y, x);
  if (th < T(0)) th += T(2.0 * PI_D);
  int k = (int)(th * ((T)nt / T(2.0 * PI_D)));
  k = k < 0 ? 0 : (k > nt - 1 ? nt - 1 : k);
  for (int it = 0; it < 4; ++it) {
    if (p.ray[2 * k] * y - p.ray[2 * k + 1] * x < T(0)) k = (k == 0) ? nt - 1 : k - 1;
    else if (p.ray[2 * k + 2] * y - p.ray[2 * k + 3] * x >= T(0)) k = (k == nt - 1) ? 0 : k + 1;
    else break;
  }
  return lo * nt + k;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory, completed
// on an mbarrier.  Addresses and sizes must be multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// generic-proxy accesses to shared memory are ordered before later
// async-proxy (bulk copy) accesses
// generic-proxy writes to global memory before later bulk copies read it
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for the phase with the given parity; gives up after `limit` polls
// (each poll may suspend the thread for a while) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// d_r = 3: rotational energy re-emitted by a wall hit whose four uniforms of
// stream (tag, idx, cell, step) start at jh (ud the fourth), out of line
template <typename T>
__device__ __forceinline__ T wall_rot_energy3(const Params<T>& p, T tw, T ud, uint32_t tag, uint32_t idx, uint32_t cell,
                                           uint32_t step, uint32_t jh) {
  Stream<T> sx(tag, idx, cell, step, p.k0, p.k1);
  return rot_energy(true, tw, ud, sx, jx_hit(jh));
}

// ---------------------------------------------------------------------------
// Stage (a): free flight with wall interaction (Sec. 2.2; fully diffuse
// walls of Sec. 4).  A diffuse wall re-emits with normal speed
// sqrt(-2 T_w ln u) (flux-weighted half-range Maxwellian), Maxwellian
// tangential components about the wall velocity and a rotational energy drawn
// at T_w; the particle then flies the rest of the step; at most MAX_HITS hits.
// tally[w*5 + q]: hits, momentum (3) and energy delivered to wall w.
// ---------------------------------------------------------------------------
template <typename T, int DIM, bool TALLY, bool GEN = true>
__device__ void fly_walls(const Params<T>& p, T& x, T& y, T& vx, T& vy, T& vz, T& ir, uint32_t idx,
                          uint32_t cell, uint32_t step, T* tally, unsigned long long* hits_out,
                          unsigned long long* maxhit_out) {
  T t = p.dt;
  int hits = 0;
  for (;;) {
    const T xn = x + vx * t;
    const T yn = (DIM == 2) ? y + vy * t : y;
    T tx = T(0), ty = T(0);
    int wx = -1, wy = -1;
    if (xn < T(0)) {
      tx = -x / vx;
      wx = 0;
    } else if (xn > p.lx) {
      tx = (p.lx - x) / vx;
      wx = 1;
    }
    if (DIM == 2) {
      if (yn < T(0)) {
        ty = -y / vy;
        wy = 2;
      } else if (yn > p.ly) {
        ty = (p.ly - y) / vy;
        wy = 3;
      }
    }
    if (wx < 0 && wy < 0) {
      x = xn;
      y = yn;
      break;
    }
    int w;
    T tw;
    if (wy < 0 || (wx >= 0 && tx <= ty)) {
      w = wx;
      tw = tx;
    } else {
      w = wy;
      tw = ty;
    }
    if (w < 2) {
      x = (w == 0) ? T(0) : p.lx;
      if (DIM == 2) {
        y = y + vy * tw;
        if (y < T(0)) y = T(0);
        if (y > p.ly) y = p.ly;
      }
    } else {
      y = (w == 2) ? T(0) : p.ly;
      x = x + vx * tw;
      if (x < T(0)) x = T(0);
      if (x > p.lx) x = p.lx;
    }
    if (hits == MAX_HITS) {
      if (TALLY) atomicAdd(maxhit_out, 1ull);
      break;
    }
    t = t - tw;
    if (t < T(0)) t = T(0);
    // re-emission
    const T vix = vx, viy = vy, viz = vz, iri = ir;
    const int axis = (w < 2) ? 0 : 1;
    const T sgn = (w % 2 == 0) ? T(1) : T(-1);
    if (p.wall_kind[w] == 1) {
      if (axis == 0) vx = -vx;
      else vy = -vy;
    } else {
      const T Tw = p.wall_t[w];
      T u4[4];
      draw4(TAG_WALL, idx, cell, step, 4u * (uint32_t)hits, p.k0, p.k1, u4);
      const T ua = u4[0], ub = u4[1], uc = u4[2], ud = u4[3];
      const T vn = m_sqrt(T(-2) * Tw * m_log(ua));
      T n1, n2;
      box_muller(ub, uc, &n1, &n2);
      const T sT = m_sqrt(Tw);
      if (axis == 0) {
        vx = sgn * vn;
        vy = p.wall_u[w][1] + sT * n1;
        vz = p.wall_u[w][2] + sT * n2;
      } else {
        vx = p.wall_u[w][0] + sT * n1;
        vy = sgn * vn;
        vz = p.wall_u[w][2] + sT * n2;
      }
      ir = -Tw * m_log(ud);
      if (GEN && p.d_r3) ir = wall_rot_energy3(p, Tw, ud, TAG_WALL, idx, cell, step, 4u * (uint32_t)hits);
    }
    if (TALLY) {
      T* tl = tally + 5 * w;
      atomicAdd(tl + 0, T(1));
      atomicAdd(tl + 1, vix - vx);
      atomicAdd(tl + 2, viy - vy);
      atomicAdd(tl + 3, viz - vz);
      atomicAdd(tl + 4, (T(0.5) * (vix * vix + viy * viy + viz * viz) + iri) -
                            (T(0.5) * (vx * vx + vy * vy + vz * vz) + ir));
    }
    hits += 1;
  }
  if (TALLY && hits) atomicAdd(hits_out, (unsigned long long)hits);
}

// Free flight over t in the annulus (flow past a cylinder).  The first
// crossing of the cylinder along p + v s is the smaller root of |p + v s|^2 =
// r_in^2, taken when the particle moves inward; the particle is put on the
// circle, re-emitted (diffuse at T_w about the resting wall, or specular)
// and flies the rest of the step; a path leaving a convex body does not
// meet it again.  Hit h draws uniforms j0 + 4h .. j0 + 4h + 3 of stream
// (tag, idx, cell, step).  Returns false if the particle ends at or beyond
// r_out (it leaves the domain).  tally[0..4]: hits, momentum (3) and energy
// delivered to the cylinder.
template <typename T, bool TALLY, bool GEN = true>
__device__ bool fly_ann(const Params<T>& p, T& x, T& y, T& vx, T& vy, T& vz, T& ir, uint32_t tag, uint32_t idx,
                        uint32_t cell, uint32_t step, uint32_t j0, T t, T* tally, unsigned long long* hits_out,
                        unsigned long long* maxhit_out) {
  int hits = 0;
  const T rin2 = p.r2t[0];
  for (;;) {
    const T a = vx * vx + vy * vy;
    const T b = x * vx + y * vy;
    T s1 = T(0);
    bool hit = false;
    if (b < T(0) && a > T(0)) {
      const T cc = x * x + y * y - rin2;
      const T disc = b * b - a * cc;
      if (disc > T(0)) {
        s1 = (-b - m_sqrt(disc)) / a;
        if (s1 < T(0)) s1 = T(0);
        hit = s1 < t;
      }
    }
    if (!hit) {
      x = x + vx * t;
      y = y + vy * t;
      break;
    }
    const T xh = x + vx * s1, yh = y + vy * s1;
    const T rh = m_sqrt(xh * xh + yh * yh);
    const T nx = xh / rh, ny = yh / rh;
    x = p.r_in * nx;
    y = p.r_in * ny;
    if (hits == MAX_HITS) {
      if (TALLY) atomicAdd(maxhit_out, 1ull);
      break;
    }
    t = t - s1;
    if (t < T(0)) t = T(0);
    const T vix = vx, viy = vy, viz = vz, iri = ir;
    if (p.wall_kind[0] == 1) {
      const T vn = vx * nx + vy * ny;
      vx = vx - T(2) * vn * nx;
      vy = vy - T(2) * vn * ny;
    } else {
      const T Tw = p.wall_t[0];
      T u4[4];
      draw4(tag, idx, cell, step, j0 + 4u * (uint32_t)hits, p.k0, p.k1, u4);
      const T vn = m_sqrt(T(-2) * Tw * m_log(u4[0]));
      T n1, n2;
      box_muller(u4[1], u4[2], &n1, &n2);
      const T sT = m_sqrt(Tw);
      const T vt = sT * n1;
      vx = vn * nx - vt * ny;
      vy = vn * ny + vt * nx;
      vz = sT * n2;
      ir = -Tw * m_log(u4[3]);
      if (GEN && p.d_r3) ir = wall_rot_energy3(p, Tw, u4[3], tag, idx, cell, step, j0 + 4u * (uint32_t)hits);
    }
    if (TALLY) {
      atomicAdd(tally + 0, T(1));
      atomicAdd(tally + 1, vix - vx);
      atomicAdd(tally + 2, viy - vy);
      atomicAdd(tally + 3, viz - vz);
      atomicAdd(tally + 4, (T(0.5) * (vix * vix + viy * viy + viz * viz) + iri) -
                               (T(0.5) * (vx * vx + vy * vy + vz * vz) + ir));
    }
    hits += 1;
  }
  if (TALLY && hits) atomicAdd(hits_out, (unsigned long long)hits);
  return x * x + y * y < p.r2t[p.ny];
}

// Freestream entry (annulus), FP64.  One-sided number flux per unit length
// and time of a Maxwellian (rho, T, normal drift u_n inward) through a
// boundary: rho G(inf) / (beta sqrt(pi)), beta = 1/sqrt(2T), s = u_n beta,
// G(inf) = exp(-s^2)/2 + s (sqrt(pi)/2) erfc(-s).
__device__ __forceinline__ double inflow_ginf(double s) {
  return 0.5 * exp(-s * s) + s * (0.5 * sqrt(PI_D)) * erfc(-s);
}

// Inward normal speed of an entering particle in units of 1/beta: z > 0 has
// density z exp(-(z - s)^2) with CDF G(z) = [exp(-s^2) - exp(-(z-s)^2)] / 2 +
// s (sqrt(pi)/2) [erfc(-s) - erfc(z - s)]; G(z) = u G(inf) is solved by
// Newton steps kept inside a bisection bracket, at most 100 of them.
__device__ inline double inflow_speed(double s, double u) {
  const double target = u * inflow_ginf(s);
  const double es = exp(-s * s), cs = erfc(-s);  // loop invariants
  double lo = 0.0, hi = (s > 0.0 ? s : 0.0) + 8.0;
  double z = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double w = z - s;
    const double g = 0.5 * (es - exp(-w * w)) + s * (0.5 * sqrt(PI_D)) * (cs - erfc(w));
    const double f = g - target;
    if (f > 0.0) hi = z;
    else lo = z;
    const double d = z * exp(-w * w);
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

// true if a free flight over dt stays inside the domain (no wall is reached)
template <typename T, int DIM>
__device__ __forceinline__ bool flight_stays_inside(const Params<T>& p, T x, T y, T vx, T vy, T* xn, T* yn) {
  *xn = x + vx * p.dt;
  *yn = (DIM == 2) ? y + vy * p.dt : y;
  bool in = !(*xn < T(0)) && !(*xn > p.lx);
  if (DIM == 2) in = in && !(*yn < T(0)) && !(*yn > p.ly);
  return in;
}

// Full flight: the common straight flight inline, the wall loop only when a
// wall is reached (the loop repeats the first straight step identically).
template <typename T, int DIM, bool TALLY, bool GEN = true>
__device__ __forceinline__ void fly(const Params<T>& p, T& x, T& y, T& vx, T& vy, T& vz, T& ir, uint32_t idx,
                                    uint32_t cell, uint32_t step, T* tally, unsigned long long* hits_out,
                                    unsigned long long* maxhit_out) {
  T xn, yn;
  if (flight_stays_inside<T, DIM>(p, x, y, vx, vy, &xn, &yn)) {
    x = xn;
    y = yn;
    return;
  }
  fly_walls<T, DIM, TALLY, GEN>(p, x, y, vx, vy, vz, ir, idx, cell, step, tally, hits_out, maxhit_out);
}

// ---------------------------------------------------------------------------
// Stage (c): NTC / VHS / Borgnakke-Larsen for one cell, one warp.
//
// The candidate pairs m = 0 .. M-1 are those of the sequential algorithm
// (Sec. 2.2): pick i, then j != i, accept with sigma g / (sigma g)_max, then
// Borgnakke-Larsen for i and for j (each with probability P_inelastic, Bird's
// particle selection permitting double relaxation) and isotropic scattering.
// (sigma g)_max is frozen during the step, so the only coupling between
// candidates is through shared particles.  The warp keeps a window of the
// (up to) 32 earliest unprocessed candidates; a candidate runs once no
// earlier unprocessed candidate uses either of its particles (it owns both:
// owner[] holds the smallest claiming index).  Candidates that run together
// touch disjoint particles, and every candidate sees exactly the particle
// state the sequential loop would give it, so the result is the sequential
// one, pair for pair.
// ---------------------------------------------------------------------------
struct CollCount {
  unsigned cand, coll, clip, inel;
};

template <typename T, bool GEN = true>
__device__ __forceinline__ void collide_cell(const Params<T>& p, T* __restrict__ vx, T* __restrict__ vy,
                             T* __restrict__ vz, T* __restrict__ ir, int n, uint32_t cell,
                             uint32_t step, T* sgmax_ptr, uint32_t* owner, CollCount& cc) {
  const int lane = threadIdx.x & 31;
  if (!p.collisions || n < 2) return;
  const T sgmax = *sgmax_ptr;
  const T vc = p.vol ? p.vol[cell] : p.vcell;  // the annulus's cells differ in volume
  const T xm = T(0.5) * T(n) * T(n - 1) * p.fnum * sgmax * p.dt / vc;
  Stream<T> sn(TAG_NTC, 0u, cell, step, p.k0, p.k1);
  const long long Mll = iround(xm, sn.u(0));
  const uint32_t M = (uint32_t)(Mll < 0 ? 0 : Mll);
  if (M == 0) return;
  for (int q = lane; q < n; q += 32) owner[q] = OWNER_FREE;
  __syncwarp();
  T obs = T(0);
  uint32_t next = 0;
  bool has = false;
  uint32_t k = 0;
  int pi = 0, pj = 0;
  T uacc = T(0), uinel = T(0);
  // FP32: the candidate's post-collision block is drawn with it, while every
  // lane still has a candidate to draw (later rounds run with few lanes)
  uint4 wpost = make_uint4(0u, 0u, 0u, 0u);
  const T fn = T(n), fn1 = T(n - 1);
  const unsigned below = (1u << lane) - 1u;
  // A lane keeps its candidate until it runs; free lanes take the next
  // candidates in order, so the window is always every unprocessed candidate
  // below `next` (which lane holds which does not matter).
  for (;;) {
    const unsigned freem = __ballot_sync(FULL, !has);
    if (!has) {
      const uint32_t kk = next + (uint32_t)__popc(freem & below);
      if (kk < M) {
        T u4[4];
        draw4(TAG_COLL, kk, cell, step, 0u, p.k0, p.k1, u4);
        if constexpr (sizeof(T) == 4) wpost = post_block(kk, cell, step, p.k0, p.k1);
        const T u0 = u4[0], u1 = u4[1];
        uacc = u4[2];
        uinel = u4[3];
        int i = (int)(u0 * fn);
        if (i > n - 1) i = n - 1;
        int j = (int)(u1 * fn1);
        if (j > n - 2) j = n - 2;
        if (j >= i) j += 1;
        pi = i;
        pj = j;
        k = kk;
        has = true;
      }
    }
    {
      const uint32_t room = (uint32_t)__popc(freem);
      next = (M - next > room) ? next + room : M;
    }
    if (__ballot_sync(FULL, has) == 0u) break;
    if (has) {
      atomicMin(&owner[pi], k);
      atomicMin(&owner[pj], k);
    }
    __syncwarp();
    const bool ready = has && owner[pi] == k && owner[pj] == k;
    __syncwarp();
    if (has) {
      owner[pi] = OWNER_FREE;
      owner[pj] = OWNER_FREE;
    }
    __syncwarp();
    if (ready) {
      const T gx = vx[pi] - vx[pj];
      const T gy = vy[pi] - vy[pj];
      const T gz = vz[pi] - vz[pj];
      const T g2 = gx * gx + gy * gy + gz * gz;
      T sg;
      if constexpr (sizeof(T) == 4) {
        // g^(2 - 2 omega) = (g^2)^(1 - omega): no square root
        const T he = T(0.5) * p.vhs_e;
        sg = p.c_sigma * ((g2 > T(0)) ? m_pow(g2, he) : (he == T(0) ? T(1) : T(0)));
      } else {
        sg = p.c_sigma * m_pow(m_sqrt(g2), p.vhs_e);
      }
      if (sg > obs) obs = sg;
      cc.cand += 1;
      if (uacc * sgmax < sg) {
        cc.coll += 1;
        if (sg > sgmax) cc.clip += 1;
        T up[5];
        if constexpr (sizeof(T) == 4) post_from_block(wpost, up);
        else draw_post(k, cell, step, p.k0, p.k1, up);
        T et = T(0.25) * g2;
        if (uinel < p.p_inel) {
          const T ec = et + ir[pi];
          ir[pi] = ec * bl_fraction<T, GEN>(p, up[0], k, cell, step, JX_BL);
          et = ec - ir[pi];
          cc.inel += 1;
        }
        if (up[1] < p.p_inel) {
          const T ec = et + ir[pj];
          ir[pj] = ec * bl_fraction<T, GEN>(p, up[2], k, cell, step, JX_BL + 2u);
          et = ec - ir[pj];
          cc.inel += 1;
        }
        const T gn = T(2) * m_sqrt(et);
        T hv[3];
        scatter<T, GEN>(p, gx, gy, gz, gn, up[3], up[4], hv);
        const T hx = hv[0], hy = hv[1], hz = hv[2];
        const T cx = T(0.5) * (vx[pi] + vx[pj]);
        const T cy = T(0.5) * (vy[pi] + vy[pj]);
        const T cz = T(0.5) * (vz[pi] + vz[pj]);
        vx[pi] = cx + hx;
        vy[pi] = cy + hy;
        vz[pi] = cz + hz;
        vx[pj] = cx - hx;
        vy[pj] = cy - hy;
        vz[pj] = cz - hz;
      }
    }
    __syncwarp();
    has = has && !ready;
  }
  // (sigma g)_max takes the largest sigma g seen in the step
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T other = __shfl_xor_sync(FULL, obs, o);
    obs = other > obs ? other : obs;
  }
  __syncwarp();
  if (lane == 0 && obs > sgmax) *sgmax_ptr = obs;
}

// ---------------------------------------------------------------------------
// Stage (d): raw sums of one cell for Eq. (DSMC_macroscopic), added to
// Neumaier-compensated FP64 accumulators (acc, comp: 17 per cell).
// ---------------------------------------------------------------------------
//
// FP32 particles: each step's sums go to Kahan-compensated FP32 staging
// accumulators (stg, stc: 17 per cell; pre32 holds this lane's values loaded
// earlier); when `flush` is set they are folded into the FP64 accumulators
// and cleared.  FP64 particles add to the FP64 accumulators every step (pre
// holds this lane's (acc, comp) loaded earlier, or is null).
template <typename T>
__device__ void sample_cell(const T* __restrict__ vx, const T* __restrict__ vy,
                            const T* __restrict__ vz, const T* __restrict__ ir, int n,
                            double* __restrict__ acc, double* __restrict__ comp,
                            const double* pre = nullptr, float* __restrict__ stg = nullptr,
                            float* __restrict__ stc = nullptr, const float* pre32 = nullptr,
                            bool flush = true) {
  const int lane = threadIdx.x & 31;
  T s[NMOM];
#pragma unroll
  for (int q = 0; q < NMOM; ++q) s[q] = T(0);
  for (int q = lane; q < n; q += 32) {
    const T a = vx[q], b = vy[q], c = vz[q], e = ir[q];
    const T v2 = a * a + b * b + c * c;
    s[0] += T(1);
    s[1] += a;
    s[2] += b;
    s[3] += c;
    s[4] += a * a;
    s[5] += b * b;
    s[6] += c * c;
    s[7] += a * b;
    s[8] += a * c;
    s[9] += b * c;
    s[10] += a * v2;
    s[11] += b * v2;
    s[12] += c * v2;
    s[13] += e;
    s[14] += e * a;
    s[15] += e * b;
    s[16] += e * c;
  }
#pragma unroll
  for (int q = 0; q < NMOM; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(FULL, s[q], o);
  }
  T mine = T(0);
#pragma unroll
  for (int q = 0; q < NMOM; ++q)
    if (lane == q) mine = s[q];
  if (lane < NMOM) {
    double v;
    if (stg) {
      // Kahan step into the FP32 staging pair
      const float s0 = pre32[0], c0 = pre32[1];
      const float yk = (float)mine - c0;
      const float tk = s0 + yk;
      const float ck = (tk - s0) - yk;
      if (!flush) {
        stg[lane] = tk;
        stc[lane] = ck;
        return;
      }
      stg[lane] = 0.f;
      stc[lane] = 0.f;
      v = (double)tk - (double)ck;
    } else {
      v = (double)mine;
    }
    const double a = pre ? pre[0] : acc[lane];
    const double cprev = pre ? pre[1] : comp[lane];
    const double t = a + v;
    const double cmp = (fabs(a) >= fabs(v)) ? ((a - t) + v) : ((v - t) + a);
    acc[lane] = t;
    comp[lane] = cprev + cmp;
  }
}

// ---------------------------------------------------------------------------
// Warp sum of 17 per-lane values by recursive halving (reduce-scatter): at
// each level a lane keeps half of its values and adds its partner's copy of
// that half (offsets 16, 8, 4, 2, 1; sizes 17 -> 9 -> 5 -> 3 -> 2 -> 1), 20
// shuffles instead of 17 x 5.  Lane L ends with the warp total of value
// halving_moment(L), or nothing (-1); every value lands on exactly one lane.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int halving_moment(int lane) {
  int j = (lane & 1) ? 1 : 0;
  bool ok = true;
  j = (lane & 2) ? 2 + j : j;
  ok = ok && j < 3;
  j = (lane & 4) ? 3 + j : j;
  ok = ok && j < 5;
  j = (lane & 8) ? 5 + j : j;
  ok = ok && j < 9;
  j = (lane & 16) ? 9 + j : j;
  ok = ok && j < 17;
  return ok ? j : -1;
}

template <int S, int OFF>
__device__ __forceinline__ void halving_level(const float* in, float* out, int lane) {
  constexpr int H = (S + 1) / 2;
  const bool up = (lane & OFF) != 0;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float lo = in[i];
    const float hi = (i + H < S) ? in[i + H] : 0.f;
    out[i] = (up ? hi : lo) + __shfl_xor_sync(FULL, up ? lo : hi, OFF);
  }
}

__device__ __forceinline__ float halving_sum17(const float* v, int lane) {
  float a[9], b[5], c[3], d[2], e[1];
  halving_level<17, 16>(v, a, lane);
  halving_level<9, 8>(a, b, lane);
  halving_level<5, 4>(b, c, lane);
  halving_level<3, 2>(c, d, lane);
  halving_level<2, 1>(d, e, lane);
  return e[0];
}

// FP32 particles: this step's sums of one cell, added to the Kahan-compensated
// FP32 staging pair of moment `mom` (the lane's moment, halving_moment(lane);
// pre32 holds the lane's (stg, stc) loaded earlier).  With `flush` the staged
// sum is folded into the compensated FP64 accumulators (pre: the lane's acc,
// comp) and the staging pair is cleared.
__device__ __forceinline__ void sample_accumulate(const float* __restrict__ vx, const float* __restrict__ vy,
                                                  const float* __restrict__ vz, const float* __restrict__ ir, int n,
                                                  float* s) {
  const int lane = threadIdx.x & 31;
  for (int q = lane; q < n; q += 32) {
    const float a = vx[q], b = vy[q], c = vz[q], e = ir[q];
    const float v2 = a * a + b * b + c * c;
    s[0] += 1.f;
    s[1] += a;
    s[2] += b;
    s[3] += c;
    s[4] += a * a;
    s[5] += b * b;
    s[6] += c * c;
    s[7] += a * b;
    s[8] += a * c;
    s[9] += b * c;
    s[10] += a * v2;
    s[11] += b * v2;
    s[12] += c * v2;
    s[13] += e;
    s[14] += e * a;
    s[15] += e * b;
    s[16] += e * c;
  }
}

// the cell's sum of moment `mom` (tot, this lane's) staged / folded as
// described above
__device__ __forceinline__ void sample_fold(float tot, int mom, double* __restrict__ acc, double* __restrict__ comp,
                                            const double* pre, float* __restrict__ stg, float* __restrict__ stc,
                                            const float* pre32, bool flush) {
  if (mom < 0) return;
  const float s0 = pre32[0], c0 = pre32[1];
  const float yk = tot - c0;
  const float tk = s0 + yk;
  const float ck = (tk - s0) - yk;
  if (!flush) {
    stg[mom] = tk;
    stc[mom] = ck;
    return;
  }
  stg[mom] = 0.f;
  stc[mom] = 0.f;
  const double v = (double)tk - (double)ck;
  const double a = pre[0], cprev = pre[1];
  const double t = a + v;
  const double cmp = (fabs(a) >= fabs(v)) ? ((a - t) + v) : ((v - t) + a);
  acc[mom] = t;
  comp[mom] = cprev + cmp;
}

__device__ __forceinline__ void sample_cell_staged(const float* __restrict__ vx, const float* __restrict__ vy,
                                   const float* __restrict__ vz, const float* __restrict__ ir, int n, int mom,
                                   double* __restrict__ acc, double* __restrict__ comp, const double* pre,
                                   float* __restrict__ stg, float* __restrict__ stc, const float* pre32,
                                   bool flush) {
  float s[NMOM];
#pragma unroll
  for (int q = 0; q < NMOM; ++q) s[q] = 0.f;
  sample_accumulate(vx, vy, vz, ir, n, s);
  sample_fold(halving_sum17(s, threadIdx.x & 31), mom, acc, comp, pre, stg, stc, pre32, flush);
}

// one chunk of a cell's particles: its sums reduced across the warp (the
// lane's moment returned, to be added over the chunks)
__device__ __forceinline__ float sample_chunk(const float* __restrict__ vx, const float* __restrict__ vy,
                                              const float* __restrict__ vz, const float* __restrict__ ir, int n) {
  float s[NMOM];
#pragma unroll
  for (int q = 0; q < NMOM; ++q) s[q] = 0.f;
  sample_accumulate(vx, vy, vz, ir, n, s);
  return halving_sum17(s, threadIdx.x & 31);
}

}  // namespace dsmc
